// The per-mode work of the FP64 descent step (paper §4, steps 1-5) as three streaming kernels
// over groups of instances.
//
// k_mode performs the Chebyshev analysis, the Stokes solve and the Chebyshev synthesis of a
// few Fourier modes of one instance in one CTA.  Every instance of a batch on the same grid
// applies the same matrices to its own columns, so the descent step instead runs each phase
// as a small batched matrix product whose right-hand sides are the columns of a group of up
// to G instances (real and imaginary parts: 2 G columns), one CTA per sub-problem:
//   k_yanalysis  CTA (group, mode, component c): parity-folded Chebyshev analysis of the
//                product y-values and the right-hand side F = (state/step + product)/nu,
//                written class-split to frg
//   k_ysolve     CTA (group, mode, parity group g): the dense Stokes operators of group g
//                (v of class g; xi = -dv/dy and eta of class 1-g), the assembly of v (class g)
//                and u, w (class 1-g), and the finite-difference quotient: r1 = (u+ - u)/dt
//                (PHI) or f = -(q+ - q)/dtau_hat followed by u += dtau f (PSI_UPDATE)
//   k_ysynth     CTA (group, mode, output field q): Chebyshev synthesis of values
//                (u, v, w) or y-derivative values (u_y, w_y) of u or r1 into yv
// Matrices are staged in shared memory (the Chebyshev tables, and the five operator blocks of
// the CTA's mode and parity group).  On GB300 a warp's FP64 instruction holds the FP64 pipe
// for the same time whatever its active lanes, so every warp is kept full and branch-uniform:
// a lane owns one column and two matrix rows (two independent accumulations sharing each
// right-hand-side load), the columns of a group are padded to SP = 2, 4, 8 or 16 and a warp
// covers 32/SP row pairs, and row lists with different loop structure (even / odd
// Chebyshev rows; v and xi / eta) start on warp boundaries.  Shared-memory column arrays
// have the odd row stride SP + 1 (no bank conflicts when a warp walks down a column).  Each
// output is the same sequence of operations as in k_mode, so both paths give bit-identical
// results.
#include <algorithm>
#include <type_traits>

#include "pcf_ff.cuh"
#include "pcf_kernels.cuh"

namespace pcf {

// Threads per CTA of the split synthesis and analysis kernels.
#ifndef PCF_SPLIT_THREADS
#define PCF_SPLIT_THREADS 128
#endif
#ifndef PCF_ANALYSIS_THREADS
#define PCF_ANALYSIS_THREADS 256
#endif
constexpr int kSplitThreads = PCF_SPLIT_THREADS;
constexpr int kAnalysisThreads = PCF_ANALYSIS_THREADS;
// Launch bounds of the split synthesis and analysis kernels: the host sizes each launch to
// one pass over a CTA's row tasks (split_ysynth_threads, split_yanalysis_threads), within
// these bounds; the register budgets (five and four resident CTAs) are those of the 128- and
// 256-thread kernels with ten and five resident CTAs.
constexpr int kSynthMaxThreads = 256;
constexpr int kAnalysisMaxThreads = 320;
#ifndef PCF_SOLVE_THREADS
#define PCF_SOLVE_THREADS 128
#endif
constexpr int kSolveThreads = PCF_SOLVE_THREADS;  // threads per CTA of the persistent solve
constexpr int kMaxGroup = 8;  // instances per group (16 columns)

// frg of one instance: [mode][3][2][L2] doubles, L2 = 2 (N/2 + 1); class-split (even n at
// n/2, odd n at N/2 + 1 + n/2).

__device__ __forceinline__ int find_group(const GroupLaunch& gl, int cta, int* local) {
  int lo = 0, hi = gl.ngroups - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (gl.prefix[mid] <= cta) lo = mid; else hi = mid - 1;
  }
  *local = cta - gl.prefix[lo];
  return lo;
}

// Columns of a group of nI instances, padded to a power of two (SP divides 32).
__device__ __forceinline__ int col_pad(int nI) {
  int sp = 2;
  while (sp < 2 * nI) sp <<= 1;
  return sp;
}
__device__ __forceinline__ int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Element t of the Chebyshev table in the arithmetic A (float-float: the precomputed pairs)
template <class A> __device__ __forceinline__ A cheb_at(const Inst& I, int t);
template <> __device__ __forceinline__ double cheb_at<double>(const Inst& I, int t) { return I.cheb[t]; }
template <> __device__ __forceinline__ ff cheb_at<ff>(const Inst& I, int t) {
  const float2 v = I.cheb_ff[t];
  return ff(v.x, v.y);
}

// Dot products of two matrix rows r0, r1 with one column x (stride s) over len terms.  FP64:
// one chain per row, in index order (the order of k_mode).  Float-float: each row's sum is
// split over even and odd indices, four independent chains, because a float-float FMA is a
// chain of ~12 dependent FP32 operations whose latency one chain per row would expose.
template <class A>
__device__ __forceinline__ void dot2(const A* r0, const A* r1, const A* x, int s, int len, A& a0, A& a1) {
  if constexpr (std::is_same<A, ff>::value) {
    A p0 = A(0.0), p1 = A(0.0), q0 = A(0.0), q1 = A(0.0);
    int j = 0;
    for (; j + 1 < len; j += 2) {
      const A x0 = x[j * s], x1 = x[(j + 1) * s];
      p0 = fma(r0[j], x0, p0);
      p1 = fma(r1[j], x0, p1);
      q0 = fma(r0[j + 1], x1, q0);
      q1 = fma(r1[j + 1], x1, q1);
    }
    if (j < len) {
      const A x0 = x[j * s];
      p0 = fma(r0[j], x0, p0);
      p1 = fma(r1[j], x0, p1);
    }
    a0 = a0 + (p0 + q0);
    a1 = a1 + (p1 + q1);
  } else {
    for (int j = 0; j < len; ++j) {
      const A x0 = x[j * s];
      a0 = fma(r0[j], x0, a0);
      a1 = fma(r1[j], x0, a1);
    }
  }
}

// One chain in index order: a += r[j] x[j s] for j < len (dot2's chain for a row without a
// partner).
template <class A>
__device__ __forceinline__ void dot1(const A* r, const A* x, int s, int len, A& a) {
  for (int j = 0; j < len; ++j) a = fma(r[j], x[j * s], a);
}
// The two chains of one synthesis row side by side, each in index order: e over len terms of
// the even-class row re and column xe, o over len - 1 terms of the odd-class row ro and xo.
template <class A>
__device__ __forceinline__ void dot_eo(const A* re, const A* ro, const A* xe, const A* xo, int s, int len, A& e,
                                       A& o) {
  for (int j = 0; j + 1 < len; ++j) {
    e = fma(re[j], xe[j * s], e);
    o = fma(ro[j], xo[j * s], o);
  }
  e = fma(re[len - 1], xe[(len - 1) * s], e);
}

// Per-instance flags of a group in shared memory: live[i] = instance takes part in this
// launch (active; in the dummy-dynamics step the mask already holds this step's J < tol).
__device__ __forceinline__ void group_flags(const GroupLaunch& gl, int first, int nI, int* live) {
  if (threadIdx.x < nI) live[threadIdx.x] = inst_active(gl.insts[first + threadIdx.x]) ? 1 : 0;
}

// A: arithmetic of the Chebyshev dot products (double, or ff in the float-float form).
// Five resident CTAs per SM (48 registers): with one mode per CTA a 32x33x32 batch of 8 has
// 7.5 CTAs per SM, one and a half waves at five and two at four.
template <class A>
__global__ void __launch_bounds__(kAnalysisMaxThreads, 4) k_yanalysis(GroupLaunch gl, int op, int mt) {
  extern __shared__ double sm[];
  __shared__ int live[kMaxGroup];
  int local;
  const int2 grp = gl.groups[find_group(gl, blockIdx.x, &local)];
  const int first = grp.x, nI = grp.y;
  const Inst& I0 = gl.insts[first];
  const int N = I0.N, H = N / 2 + 1, Mh = H, L2 = 2 * H, ny = I0.ny, nm = I0.nmodes, half = N / 2;
  const int nrun = run_modes(gl, I0);
  const int tile = local / 3, c = local - 3 * tile, m0 = tile * mt;
  // columns: (mode m0 + mm, instance i, part) = mm SP + 2 i + part, SPt = SP mt <= 32
  const int SP = col_pad(nI), SPt = SP * mt, XS = SPt + 1, RW = 32 / SPt;
  const ChebLayout CL(N);
  A* Ae = reinterpret_cast<A*>(sm);  // [H][H]
  A* Ao = Ae + H * H;                // [H][H] (rows < H-1 used)
  A* VP = Ao + H * H;                // [H][XS]    P_j = V_j + V_{N-j} (j < N/2), V_{N/2}
  A* VQ = VP + H * XS;               // [half][XS] Q_j = V_j - V_{N-j}
  group_flags(gl, first, nI, live);
  for (int t = threadIdx.x; t < 2 * H * H; t += blockDim.x) Ae[t] = cheb_at<A>(I0, CL.Ae() + t);
  for (int t = threadIdx.x; t < H * SPt / 2; t += blockDim.x) {
    const int pr = t % (SPt / 2), j = t / (SPt / 2), mm = pr / (SP / 2), i = pr - mm * (SP / 2);
    const int m = m0 + mm;
    double2 a = make_double2(0.0, 0.0), b = a;
    if (i < nI && m < nrun) {
      const double2* xz = gl.insts[first + i].xz + (size_t)c * ny * nm + m;
      a = xz[(size_t)j * nm];
      if (j < half) b = xz[(size_t)(N - j) * nm];
    }
    A* p = VP + j * XS + 2 * pr;
    if (j < half) {
      p[0] = A(a.x + b.x);
      p[1] = A(a.y + b.y);
      A* q = VQ + j * XS + 2 * pr;
      q[0] = A(a.x - b.x);
      q[1] = A(a.y - b.y);
    } else {
      p[0] = A(a.x);
      p[1] = A(a.y);
    }
  }
  __syncthreads();
  const double inv_step = op == MODE_PHI ? I0.inv_dt : I0.inv_dtau_hat, inv_nu = I0.inv_nu;
  // row pairs (k, k + hE) of the even coefficients n = 2k (k < H, from P), then pairs
  // (k, k + hO) of the odd coefficients n = 2k+1 (k < N/2, from Q).  A class with an odd
  // number of rows leaves its middle row with a dead partner.  In FP64, when that pair would
  // start a warp of its own (hE - 1 or hO - 1 a multiple of RW, the pairs per warp), the row
  // instead takes one single-chain task per column, in whole warps after the pairs: half a
  // pair warp's work.  At most one class has an odd count (H = N/2 + 1).
  const int hE = (H + 1) / 2, hO = (half + 1) / 2;
  const bool dbl = std::is_same<A, double>::value;
  const bool loneE = dbl && (H & 1) && (hE - 1) % RW == 0, loneO = dbl && (half & 1) && (hO - 1) % RW == 0;
  const int pE = hE - (loneE ? 1 : 0), pO = hO - (loneO ? 1 : 0);
  const int ER = round_up(pE, RW), OR = round_up(pO, RW), PT = (ER + OR) * SPt;
  const int ntask = PT + (loneE || loneO ? SPt : 0);
  auto task = [&](int t, auto single_c) {
    constexpr bool single = decltype(single_c)::value;
    const int sc = single ? t - PT : t % SPt, rs = t / SPt, mm = sc / SP, m = m0 + mm;
    const bool even = single ? loneE : rs < ER;
    const int nrow = even ? H : half, hh = even ? hE : hO, pp = even ? pE : pO;
    const int k0 = single ? hh - 1 : (even ? rs : rs - ER), k1 = k0 + hh;
    const bool v0 = single || k0 < pp, v1 = !single && v0 && k1 < nrow;
    const int i = (sc - mm * SP) >> 1, part = sc & 1;
    const bool out = i < nI && m < nrun && live[i];
    const double* st = nullptr;
    double u0a = 0.0, u0b = 0.0;
    if (out) {
      const Inst& I = gl.insts[first + i];
      st = reinterpret_cast<const double*>((op == MODE_PHI ? I.uhat : I.rhat) + ((size_t)c * nm + m) * ny) + part;
      if (v0) u0a = st[2 * (even ? 2 * k0 : 2 * k0 + 1)];
      if (v1) u0b = st[2 * (even ? 2 * k1 : 2 * k1 + 1)];
    }
    const A* row0 = (even ? Ae : Ao) + (v0 ? k0 : 0) * H;
    const A* row1 = (even ? Ae : Ao) + (v1 ? k1 : 0) * H;
    const A* v = (even ? VP : VQ) + sc;
    const int len = even ? H : half;  // P_j for j < H, Q_j for j < N/2
    A a0 = A(0.0), a1 = A(0.0);
    if constexpr (single) dot1(row0, v, XS, len, a0);
    else dot2(row0, row1, v, XS, len, a0, a1);
    if (!out) return;
    double* fr = gl.insts[first + i].frg + ((size_t)m * 3 + c) * 2 * L2 + part * L2;
    if (v0) fr[even ? k0 : Mh + k0] = fma(u0a, inv_step, to_double(a0)) * inv_nu;
    if (v1) fr[even ? k1 : Mh + k1] = fma(u0b, inv_step, to_double(a1)) * inv_nu;
  };
  for (int t = threadIdx.x; t < ntask; t += blockDim.x) {
    if (t < PT) task(t, std::false_type());
    else task(t, std::true_type());
  }
}

// ---------------------------------------------------------------- norm of r1
// J = ||r1|| of every active instance from the plane sums of the adjoint product kernel
// (same order of operations as norm_from_parts), its history entry, and the convergence
// mask (J < tol: the instance stops before this step's update).  One CTA per instance;
// ny <= 257 (the split kernels serve grids with dense operators, ny <= 129).
__global__ void __launch_bounds__(128) k_jnorm(const Inst* insts, int step_index) {
  __shared__ double part[3 * 257];
  __shared__ double w[257];
  const Inst& I = insts[blockIdx.x];
  if (!inst_active(I)) return;
  const int ny = I.ny;
  for (int t = threadIdx.x; t < 3 * ny; t += blockDim.x) part[t] = I.normpart[t];
  for (int t = threadIdx.x; t < ny; t += blockDim.x) w[t] = I.ccw[t];
  __syncthreads();
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int j = 0; j < ny; ++j) s = fma(w[j], part[j] + part[ny + j] + part[2 * ny + j], s);
  const double J = sqrt(0.5 * I.inv_nxnz * s);
  if (I.hist) I.hist[(size_t)step_index * I.hist_stride] = J;
  if (I.tol > 0.0 && J < I.tol && I.active) *I.active = 0;
}

// ---------------------------------------------------------------- Stokes solve
__device__ __forceinline__ void cp_async8(double* dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(double* dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct SolveItem {
  int first, nI, m, g;
};
__device__ __forceinline__ SolveItem solve_item(const GroupLaunch& gl, int item) {
  int local;
  const int2 grp = gl.groups[find_group(gl, item, &local)];
  return SolveItem{grp.x, grp.y, local >> 1, local & 1};
}

// Stage the operator blocks Av, Ag and Eh of (mode m, parity group g) and the class-split
// right-hand sides of the group's instances at mode m (6 (N+2) doubles each) into buf.
__device__ __forceinline__ void solve_stage(const GroupLaunch& gl, const SolveItem& it, int sig, double* buf) {
  const Inst& I0 = gl.insts[it.first];
  const int N = I0.N, Mh = N / 2 + 1, per = 6 * (N + 2);
  const DenseLayout DL(N);
  const int MM = Mh * Mh, n3p = (3 * MM + 1) & ~1;
  const double* src = I0.dense[sig] + (size_t)it.m * DL.per_mode() + DL.block(it.g, 0);
  for (int t = threadIdx.x; t < 3 * MM; t += blockDim.x) cp_async8(buf + t, src + t);
  double* fr = buf + n3p;
  const int hp = per / 2;
  for (int t = threadIdx.x; t < it.nI * hp; t += blockDim.x) {
    const int i = t / hp, k = t - i * hp;
    cp_async16(fr + i * per + 2 * k, gl.insts[it.first + i].frg + (size_t)it.m * per + 2 * k);
  }
}

// Persistent: CTA b takes the items b, b + gridDim.x, ...; the operands of the next item are
// copied asynchronously while the current one is computed.  bufsz: doubles per stage buffer;
// scratch after the two buffers: six [Mh][SP + 1] arrays for the largest grid of the launch.
__global__ void __launch_bounds__(kSolveThreads) k_ysolve(GroupLaunch gl, int op, int nitems, int bufsz, int scr_rows) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int live[kMaxGroup];
  __shared__ double ik2_sh;
  const int sig = op == MODE_PHI ? 0 : 1;
  int item = blockIdx.x;
  if (item >= nitems) return;
  SolveItem cur = solve_item(gl, item);
  solve_stage(gl, cur, sig, sm);
  cp_commit();
  for (int k = 0; item < nitems; ++k, item += gridDim.x) {
    double* buf = sm + (size_t)(k & 1) * bufsz;
    const int nxt = item + gridDim.x;
    SolveItem nx = cur;
    if (nxt < nitems) {
      nx = solve_item(gl, nxt);
      solve_stage(gl, nx, sig, sm + (size_t)((k + 1) & 1) * bufsz);
    }
    cp_commit();
    cp_wait_prev();
    const int first = cur.first, nI = cur.nI, m = cur.m, g = cur.g;
    const Inst& I0 = gl.insts[first];
    if (threadIdx.x < nI) live[threadIdx.x] = inst_active(gl.insts[first + threadIdx.x]) ? 1 : 0;
    if (threadIdx.x == 32) {
      // 1/k^2 of the mode, once per item (an FP64 division costs the pipe per lane-instruction)
      const int Mz0 = I0.Mz, ix0 = m / Mz0;
      const double kx0 = I0.kx[ix0], kz0 = I0.kz[m - ix0 * Mz0];
      ik2_sh = (kx0 == 0.0 && kz0 == 0.0) ? 0.0 : 1.0 / (kx0 * kx0 + kz0 * kz0);
    }
    const int N = I0.N, Mh = N / 2 + 1, L2 = 2 * Mh, ny = I0.ny, nm = I0.nmodes, Mz = I0.Mz;
    const int SP = col_pad(nI), XS = SP + 1, RW = 32 / SP;
    const int pv = g, pP = 1 - g, McV = (N - pv) / 2 + 1, McP = (N - pP) / 2 + 1;
    const int ix = m / Mz, p = m - ix * Mz;
    const double kx = I0.kx[ix], kz = I0.kz[p];
    const bool mean = kx == 0.0 && kz == 0.0;
    const int MM = Mh * Mh, per = 6 * L2;
    const double* D = buf;                          // [3][Mh][Mh] blocks Av, Ag, Eh of group g
    const double* FR = buf + ((3 * MM + 1) & ~1);   // [nI][3][2][L2] right-hand sides
    double* FV = sm + 2 * (size_t)bufsz;            // [Mh][XS] f_v (class g); mean mode: f_u (class g)
    double* GG = FV + scr_rows * XS;                // [Mh][XS] g (class 1-g);   mean mode: f_w (class g)
    double* HH = GG + scr_rows * XS;                // [Mh][XS] h (class 1-g)
    double* OV = HH + scr_rows * XS;                // [Mh][XS] v (class g);     mean mode: u
    double* OX = OV + scr_rows * XS;                // [Mh][XS] xi (class 1-g);  mean mode: w
    double* OE = OX + scr_rows * XS;                // [Mh][XS] eta (class 1-g)
    __syncthreads();
    // right-hand sides: column s = 2 i + rho (instance i, real/imaginary part rho)
    for (int t = threadIdx.x; t < Mh * SP; t += blockDim.x) {
      const int s = t % SP, j = t / SP, i = s >> 1, rho = s & 1;
      double fv = 0.0, gg = 0.0, hh = 0.0;
      if (i < nI) {
        const double* fr = FR + i * per;
        if (mean) {
          const int Mc = (N - g) / 2 + 1;
          if (j < Mc) {
            fv = fr[(0 * 2 + rho) * L2 + g * Mh + j];
            gg = fr[(2 * 2 + rho) * L2 + g * Mh + j];
          }
        } else {
          if (j < McV) fv = fr[(1 * 2 + rho) * L2 + pv * Mh + j];
          if (j < McP) {
            const double fu = fr[(0 * 2 + (1 - rho)) * L2 + pP * Mh + j];
            const double fw = fr[(2 * 2 + (1 - rho)) * L2 + pP * Mh + j];
            const double sgn = rho == 0 ? -1.0 : 1.0;  // Re(i a) = -Im a, Im(i a) = Re a
            gg = sgn * fma(kx, fu, kz * fw);
            hh = sgn * fma(kz, fu, -kx * fw);
          }
        }
      }
      FV[j * XS + s] = fv;
      GG[j * XS + s] = gg;
      HH[j * XS + s] = hh;
    }
    const int nV = mean ? (N - g) / 2 + 1 : McV;
    const int nU = mean ? nV : McP;
    const int nout = nV + 2 * nU;
    __syncthreads();
    // v = Av f_v + Ag g (row list A), eta = Eh h (row list B); mean mode: u = Eh f_u,
    // w = Eh f_w (list A), no list B.  A task is one row of list A (McV + McP terms) or two
    // rows of list B (McP terms each), so the tasks carry about the same work; warps hold RW
    // rows of one list.  Each row is one fma chain in increasing j (the order of the single
    // per-mode kernel, so the bits agree).  xi = -dv/dy follows from v below.
    {
      const int Mc0 = (N - g) / 2 + 1;
      const int nA = mean ? 2 * Mc0 : McV, nB = mean ? 0 : McP;
      const int hB = (nB + 1) / 2;
      const int PA = round_up(nA, RW), PB = round_up(hB, RW);
      for (int t = threadIdx.x; t < (PA + PB) * SP; t += blockDim.x) {
        const int sc = t % SP, rs = t / SP;
        if (rs < PA) {
          if (rs >= nA) continue;
          double a = 0.0;
          double* out;
          if (mean) {
            // rows < Mc0: u from f_u; rows >= Mc0: w from f_w (both with Eh)
            const bool isu = rs < Mc0;
            const int r = isu ? rs : rs - Mc0;
            const double* col = D + 2 * MM + r;
            const double* X = (isu ? FV : GG) + sc;
            for (int j = 0; j < Mc0; ++j) a = fma(col[j * Mh], X[j * XS], a);
            out = (isu ? OV : OX) + r * XS + sc;
          } else {
            const double* cA = D + rs;       // Av
            for (int j = 0; j < McV; ++j) a = fma(cA[j * Mh], FV[j * XS + sc], a);
            const double* cG = cA + MM;      // Ag
            for (int j = 0; j < McP; ++j) a = fma(cG[j * Mh], GG[j * XS + sc], a);
            out = OV + rs * XS + sc;
          }
          *out = a;
        } else {
          const int q = rs - PA;
          const bool v0 = q < hB, v1 = v0 && q + hB < nB;
          const int r0 = v0 ? q : 0, r1 = v1 ? q + hB : 0;
          const double* c0 = D + 2 * MM + r0;
          const double* c1 = D + 2 * MM + r1;
          double a0 = 0.0, a1 = 0.0;
          for (int j = 0; j < McP; ++j) {
            const double x = HH[j * XS + sc];
            a0 = fma(c0[j * Mh], x, a0);
            a1 = fma(c1[j * Mh], x, a1);
          }
          if (v0) OE[r0 * XS + sc] = a0;
          if (v1) OE[r1 * XS + sc] = a1;
        }
      }
    }
    __syncthreads();
    if (!mean) {  // xi = -dv/dy (class 1-g), one column per thread
      for (int s = threadIdx.x; s < SP; s += blockDim.x)
        xi_from_v(N, pv, OV + s, XS, OX + s, XS, I0.rco + RcoLayout(N).off(pv, 4));
      __syncthreads();
    }
    // assembly and output: v (class g) and u, w (class 1-g); mean mode: u, v = 0, w (class g)
    const double inv_step = op == MODE_PHI ? I0.inv_dt : I0.inv_dtau_hat;
    const double ik2 = ik2_sh;
    for (int t = threadIdx.x; t < nI * nout; t += blockDim.x) {
      const int i = t / nout, kk = t - i * nout;
      if (!live[i]) continue;
      int comp, row, n;
      double vr, vi;
      if (kk < nV) {
        comp = 1;
        row = kk;
        n = (mean ? g : pv) + 2 * row;
        vr = mean ? 0.0 : OV[row * XS + 2 * i];
        vi = mean ? 0.0 : OV[row * XS + 2 * i + 1];
      } else {
        const bool isu = kk < nV + nU;
        comp = isu ? 0 : 2;
        row = kk - nV - (isu ? 0 : nU);
        n = (mean ? g : pP) + 2 * row;
        if (mean) {
          const double* src = isu ? OV : OX;
          vr = src[row * XS + 2 * i];
          vi = src[row * XS + 2 * i + 1];
        } else {
          const double xr = OX[row * XS + 2 * i], xi = OX[row * XS + 2 * i + 1];
          const double er = OE[row * XS + 2 * i], ei = OE[row * XS + 2 * i + 1];
          if (isu) {
            vr = fma(kx, xi, kz * ei) * ik2;
            vi = -fma(kx, xr, kz * er) * ik2;
          } else {
            vr = fma(kz, xi, -kx * ei) * ik2;
            vi = fma(-kz, xr, kx * er) * ik2;
          }
        }
      }
      const Inst& I = gl.insts[first + i];
      const size_t gidx = ((size_t)comp * nm + m) * ny + n;
      if (op == MODE_PHI) {
        const double2 u0 = I.uhat[gidx];
        I.rhat[gidx] = make_double2((vr - u0.x) * inv_step, (vi - u0.y) * inv_step);
      } else {
        const double2 q0 = I.rhat[gidx], u0 = I.uhat[gidx];
        const double fr = -(vr - q0.x) * inv_step;
        const double fi = -(vi - q0.y) * inv_step;
        I.uhat[gidx] = make_double2(fma(I.dtau, fr, u0.x), fma(I.dtau, fi, u0.y));
      }
    }
    __syncthreads();  // buffer and scratch are reused by the next item
    cur = nx;
  }
}

// slot 0: synthesis of uhat, slot 1: of rhat.  q = 0..4: V_u V_v V_w W_u W_w.  Ten resident
// CTAs per SM (48 registers): one mode per CTA gives a 32x33x32 batch of 8 12.5 CTAs per SM.
// In a reduced launch (modes m >= 0 only), the y-value slot of mode -m that mirrors part
// `part` of mode m (flattened index m = i Mz + p, 0 < i <= Kx) of field qf (velocity
// component c), and the sign of the s2 relation a_{-m} = e2_c (-1)^m conj(a_m), e2 = (+1, +1, -1)
// (the conjugate flips the imaginary part).  Null for m = 0 or a full launch.
template <bool RED>
__device__ __forceinline__ double* mirror_dst(const GroupLaunch& gl, const Inst& I0, double2* yv, int slot, int qf,
                                              int c, int m, int part, double* sgn) {
  if (!RED) return nullptr;
  const int ix = m / I0.Mz;
  if (ix == 0) return nullptr;
  *sgn = ((ix & 1) ? -1.0 : 1.0) * (c == 2 ? -1.0 : 1.0) * (part ? -1.0 : 1.0);
  const int mm = (I0.Mx - ix) * I0.Mz + (m - ix * I0.Mz);
  return reinterpret_cast<double*>(yv + ((size_t)slot * kFieldsY + qf) * I0.ny * I0.nmodes + mm) + part;
}

template <class A, bool RED>
// RED: a reduced launch (gl.reduced), which also writes the mirrored y-values of mode -m
// (a separate instantiation, so that the full launch keeps its register budget).
__global__ void __launch_bounds__(kSynthMaxThreads, 5) k_ysynth(GroupLaunch gl, int slot, int check_active, int mt) {
  extern __shared__ double sm[];
  __shared__ int live[kMaxGroup];
  int local;
  const int2 grp = gl.groups[find_group(gl, blockIdx.x, &local)];
  const int first = grp.x, nI = grp.y;
  const Inst& I0 = gl.insts[first];
  const int N = I0.N, H = N / 2 + 1, ny = I0.ny, nm = I0.nmodes, half = N / 2;
  const int nrun = run_modes(gl, I0);
  const int tile = local / kFieldsY, qf = local - kFieldsY * tile, m0 = tile * mt;
  const int c = qf < 3 ? qf : (qf == 3 ? 0 : 2);
  const bool deriv = qf >= 3;
  // columns: (mode m0 + mm, instance i, part) = mm SP + 2 i + part, SPt = SP mt <= 32
  const int SP = col_pad(nI), SPt = SP * mt, XS = SPt + 1, RW = 32 / SPt;
  const ChebLayout CL(N);
  A* ME = reinterpret_cast<A*>(sm);  // [H][H] Ce or De
  A* MO = ME + H * H;                // [H][H] Co or Do (columns < H-1 used)
  A* AE = MO + H * H;                // [H][XS] even coefficients a_{2k}
  A* AO = AE + H * XS;               // [H-1][XS] odd coefficients a_{2k+1}
  if (threadIdx.x < nI) live[threadIdx.x] = (!check_active || inst_active(gl.insts[first + threadIdx.x])) ? 1 : 0;
  const int tabE = deriv ? CL.De() : CL.Ce(), tabO = deriv ? CL.Do() : CL.Co();
  for (int t = threadIdx.x; t < H * H; t += blockDim.x) {
    ME[t] = cheb_at<A>(I0, tabE + t);
    MO[t] = cheb_at<A>(I0, tabO + t);
  }
  for (int t = threadIdx.x; t < ny * (SPt / 2); t += blockDim.x) {
    const int n = t % ny, pr = t / ny, mm = pr / (SP / 2), i = pr - mm * (SP / 2), m = m0 + mm;
    double2 v = make_double2(0.0, 0.0);
    if (i < nI && m < nrun)
      v = (slot == 0 ? gl.insts[first + i].uhat : gl.insts[first + i].rhat)[((size_t)c * nm + m) * ny + n];
    A* d = ((n & 1) ? AO : AE) + (n >> 1) * XS + 2 * pr;
    d[0] = A(v.x);
    d[1] = A(v.y);
  }
  __syncthreads();
  // rows j and j + hJ of the output (hJ = H/2 rounded up), values at y_j and y_{N-j}.  An odd
  // H leaves the middle row hJ - 1 with a dead partner.  In FP64, when that pair would start a
  // warp of its own, each of the row's columns instead takes one thread that runs the row's
  // even and odd chains side by side, in whole warps after the pairs: half a pair warp's work.
  const int hJ = (H + 1) / 2;
  const bool lone = std::is_same<A, double>::value && (H & 1) && (hJ - 1) % RW == 0;
  const int np = hJ - (lone ? 1 : 0), PT = round_up(np, RW) * SPt;
  const int ntask = PT + (lone ? SPt : 0);
  for (int t = threadIdx.x; t < ntask; t += blockDim.x) {
    if (t >= PT) {
      const int sc = t - PT, j = hJ - 1, mm = sc / SP, m = m0 + mm;
      A e = A(0.0), o = A(0.0);
      dot_eo(ME + j * H, MO + j * H, AE + sc, AO + sc, XS, H, e, o);
      const int i = (sc - mm * SP) >> 1, part = sc & 1;
      if (i >= nI || m >= nrun || !live[i]) continue;
      double* dst = reinterpret_cast<double*>(gl.insts[first + i].yv + ((size_t)slot * kFieldsY + qf) * ny * nm + m) + part;
      double sgn;
      double* dsm = mirror_dst<RED>(gl, I0, gl.insts[first + i].yv, slot, qf, c, m, part, &sgn);
      const double v0_ = to_double(e + o);
      dst[(size_t)j * nm * 2] = v0_;
      if (dsm) dsm[(size_t)j * nm * 2] = sgn * v0_;
      if (j < half) {
        const double v1_ = to_double(deriv ? o - e : e - o);
        dst[(size_t)(N - j) * nm * 2] = v1_;
        if (dsm) dsm[(size_t)(N - j) * nm * 2] = sgn * v1_;
      }
      continue;
    }
    const int sc = t % SPt, j0 = t / SPt, j1 = j0 + hJ, mm = sc / SP, m = m0 + mm;
    const bool v0 = j0 < np, v1 = v0 && j1 < H;
    const A* re0 = ME + (v0 ? j0 : 0) * H;
    const A* ro0 = MO + (v0 ? j0 : 0) * H;
    const A* re1 = ME + (v1 ? j1 : 0) * H;
    const A* ro1 = MO + (v1 ? j1 : 0) * H;
    A e0 = A(0.0), o0 = A(0.0), e1 = A(0.0), o1 = A(0.0);
    dot2(re0, re1, AE + sc, XS, H, e0, e1);
    dot2(ro0, ro1, AO + sc, XS, H - 1, o0, o1);
    const int i = (sc - mm * SP) >> 1, part = sc & 1;
    if (!v0 || i >= nI || m >= nrun || !live[i]) continue;
    double* dst = reinterpret_cast<double*>(gl.insts[first + i].yv + ((size_t)slot * kFieldsY + qf) * ny * nm + m) + part;
    double sgn;
    double* dsm = mirror_dst<RED>(gl, I0, gl.insts[first + i].yv, slot, qf, c, m, part, &sgn);
    // T_{2k} even, T_{2k+1} odd in y; T'_{2k} odd, T'_{2k+1} even
    const double a0 = to_double(e0 + o0);
    dst[(size_t)j0 * nm * 2] = a0;
    if (dsm) dsm[(size_t)j0 * nm * 2] = sgn * a0;
    if (j0 < half) {
      const double b0 = to_double(deriv ? o0 - e0 : e0 - o0);
      dst[(size_t)(N - j0) * nm * 2] = b0;
      if (dsm) dsm[(size_t)(N - j0) * nm * 2] = sgn * b0;
    }
    if (v1) {
      const double a1 = to_double(e1 + o1);
      dst[(size_t)j1 * nm * 2] = a1;
      if (dsm) dsm[(size_t)j1 * nm * 2] = sgn * a1;
      if (j1 < half) {
        const double b1 = to_double(deriv ? o1 - e1 : e1 - o1);
        dst[(size_t)(N - j1) * nm * 2] = b1;
        if (dsm) dsm[(size_t)(N - j1) * nm * 2] = sgn * b1;
      }
    }
  }
}

int split_ctas_per_group(int kind, int nmodes, int mt) {
  const int tiles = (nmodes + mt - 1) / mt;
  return kind == 0 ? 3 * tiles : kind == 1 ? 2 * nmodes : kFieldsY * tiles;
}
// Largest group on a grid: kMaxGroup (every loop of the split kernels strides over its
// tasks; shared memory is checked where the groups are set).
int split_max_group(int) { return kMaxGroup; }
static size_t col_pad_host(int G) {
  size_t sp = 2;
  while (sp < 2 * (size_t)G) sp <<= 1;
  return sp;
}
int split_col_pad(int G) { return (int)col_pad_host(G); }
// ---------------------------------------------------------------- fused per-mode half-step
// CTA = (instance group, mode m): the whole per-mode work of one half-step of the descent
// (PHI: the NSE Stokes step and r1; PSI_UPDATE: the dummy-dynamics Stokes step, f and the
// update) for the group's instances, with every intermediate in shared memory:
//   analysis (3 components) -> Stokes solve (parity groups 0, 1) -> epilogue (r1 or the new
//   u, to global memory and to shared memory) -> synthesis (V_u V_v V_w W_u W_w of r1 or u).
// The lane mappings, and the operations of every output, are those of k_yanalysis, k_ysolve
// and k_ysynth, so the results are bit-identical to the split kernels.
constexpr int kStepThreads = 256;

struct StepLayout {
  int cheb, dense, v, fr, st, uh, sc, out, total;  // offsets in doubles
};
__host__ __device__ inline StepLayout step_layout(int N, int SP) {
  const int H = N / 2 + 1, ny = N + 1, XS = SP + 1, L2 = 2 * H;
  StepLayout L;
  L.cheb = 0;
  L.dense = L.cheb + ((6 * H * H + 1) & ~1);
  L.v = L.dense + ((6 * H * H + 1) & ~1);
  L.fr = L.v + 3 * 2 * H * XS;
  L.st = L.fr + (SP / 2) * 6 * L2;
  L.uh = L.st + 3 * ny * XS;
  L.sc = L.uh + 3 * ny * XS;
  L.out = L.sc + 6 * H * XS;
  L.total = L.out + 3 * 2 * H * XS;
  return L;
}

__global__ void __launch_bounds__(kStepThreads) k_ystep(GroupLaunch gl, int op) {
  extern __shared__ __align__(16) double sm[];
  __shared__ int live[kMaxGroup];
  __shared__ double ik2_sh;
  int m;
  const int2 grp = gl.groups[find_group(gl, blockIdx.x, &m)];
  const int first = grp.x, nI = grp.y;
  const Inst& I0 = gl.insts[first];
  const int N = I0.N, H = N / 2 + 1, Mh = H, L2 = 2 * H, ny = I0.ny, nm = I0.nmodes, Mz = I0.Mz, half = N / 2;
  const int SP = col_pad(nI), XS = SP + 1, RW = 32 / SP;
  const bool phi = op == MODE_PHI;
  const int sig = phi ? 0 : 1;
  const DenseLayout DL(N);
  const ChebLayout CL(N);
  const StepLayout SL = step_layout(N, SP);
  double* CH = sm + SL.cheb;   // Chebyshev tables (Ce Co De Do Ae Ao)
  double* D = sm + SL.dense;   // the 6 operator blocks of mode m (3 per parity group)
  double* V = sm + SL.v;       // [3][2H][XS] folded product values: P rows 0..H-1, Q rows H..H+N/2-1
  double* FR = sm + SL.fr;     // [SP/2][3][2][L2] right-hand sides (class-split)
  double* ST = sm + SL.st;     // [3][ny][XS] state of the step (uhat for PHI, rhat = r1 for PSI)
  double* UH = sm + SL.uh;     // [3][ny][XS] uhat (PSI)
  double* SC = sm + SL.sc;     // [6][Mh][XS] solve scratch
  double* OUT = sm + SL.out;   // [3][2H][XS] new coefficients, class-split rows (even 0..H-1, odd H..)
  // read-only tables, asynchronously
  {
    const double* src = I0.dense[sig] + (size_t)m * DL.per_mode();
    for (int t = threadIdx.x; t < DL.per_mode(); t += blockDim.x) cp_async8(D + t, src + t);
    for (int t = threadIdx.x; t < CL.total(); t += blockDim.x) cp_async8(CH + t, I0.cheb + t);
    cp_commit();
  }
  if (threadIdx.x < nI) live[threadIdx.x] = inst_active(gl.insts[first + threadIdx.x]) ? 1 : 0;
  if (threadIdx.x == 32) {
    const int ix0 = m / Mz;
    const double kx0 = I0.kx[ix0], kz0 = I0.kz[m - ix0 * Mz];
    ik2_sh = (kx0 == 0.0 && kz0 == 0.0) ? 0.0 : 1.0 / (kx0 * kx0 + kz0 * kz0);
  }
  // state columns and folded product values (column s = 2 i + part; padding columns zero)
  for (int t = threadIdx.x; t < 3 * ny * (SP / 2); t += blockDim.x) {
    const int n = t % ny, r = t / ny, i = r % (SP / 2), c = r / (SP / 2);
    double2 a = make_double2(0.0, 0.0), u = a;
    if (i < nI) {
      const Inst& I = gl.insts[first + i];
      const size_t gi = ((size_t)c * nm + m) * ny + n;
      a = (phi ? I.uhat : I.rhat)[gi];
      if (!phi) u = I.uhat[gi];
    }
    double* d = ST + (c * ny + n) * XS + 2 * i;
    d[0] = a.x;
    d[1] = a.y;
    if (!phi) {
      double* e = UH + (c * ny + n) * XS + 2 * i;
      e[0] = u.x;
      e[1] = u.y;
    }
  }
  for (int t = threadIdx.x; t < 3 * H * (SP / 2); t += blockDim.x) {
    const int i = t % (SP / 2), r = t / (SP / 2), j = r % H, c = r / H;
    double2 a = make_double2(0.0, 0.0), b = a;
    if (i < nI) {
      const double2* xz = gl.insts[first + i].xz + (size_t)c * ny * nm + m;
      a = xz[(size_t)j * nm];
      if (j < half) b = xz[(size_t)(N - j) * nm];
    }
    double* Vc = V + c * 2 * H * XS;
    double* p = Vc + j * XS + 2 * i;
    if (j < half) {
      p[0] = a.x + b.x;
      p[1] = a.y + b.y;
      double* q = Vc + (H + j) * XS + 2 * i;
      q[0] = a.x - b.x;
      q[1] = a.y - b.y;
    } else {
      p[0] = a.x;
      p[1] = a.y;
    }
  }
  cp_wait_all();
  __syncthreads();
  const double inv_step = phi ? I0.inv_dt : I0.inv_dtau_hat, inv_nu = I0.inv_nu;
  // ---- analysis: F = (state/step + Chebyshev coefficients of the products)/nu (class-split)
  {
    const int hE = (H + 1) / 2, hO = (half + 1) / 2;
    const int ER = round_up(hE, RW), OR = round_up(hO, RW), per = ER + OR;
    const double* Ae = CH + CL.Ae();
    const double* Ao = CH + CL.Ao();
    for (int t = threadIdx.x; t < 3 * per * SP; t += blockDim.x) {
      const int sc = t % SP, rr = t / SP, c = rr / per, rs = rr - c * per;
      const bool even = rs < ER;
      const int nrow = even ? H : half, hh = even ? hE : hO;
      const int k0 = even ? rs : rs - ER, k1 = k0 + hh;
      const bool v0 = k0 < hh, v1 = v0 && k1 < nrow;
      const double* row0 = (even ? Ae : Ao) + (v0 ? k0 : 0) * H;
      const double* row1 = (even ? Ae : Ao) + (v1 ? k1 : 0) * H;
      const double* v = V + c * 2 * H * XS + (even ? 0 : H) * XS + sc;
      const int len = even ? H : half;
      double a0 = 0.0, a1 = 0.0;
      for (int j = 0; j < len; ++j) {
        const double x = v[j * XS];
        a0 = fma(row0[j], x, a0);
        a1 = fma(row1[j], x, a1);
      }
      const int i = sc >> 1, part = sc & 1;
      if (i >= nI) continue;
      double* fr = FR + (i * 3 + c) * 2 * L2 + part * L2;
      const double* st = ST + c * ny * XS + sc;
      if (v0) fr[even ? k0 : Mh + k0] = fma(st[(even ? 2 * k0 : 2 * k0 + 1) * XS], inv_step, a0) * inv_nu;
      if (v1) fr[even ? k1 : Mh + k1] = fma(st[(even ? 2 * k1 : 2 * k1 + 1) * XS], inv_step, a1) * inv_nu;
    }
  }
  __syncthreads();
  // ---- Stokes solve per parity group g, epilogue into global memory and OUT
  const int ix = m / Mz, p = m - ix * Mz;
  const double kx = I0.kx[ix], kz = I0.kz[p];
  const bool mean = kx == 0.0 && kz == 0.0;
  const double ik2 = ik2_sh;
  const int MM = Mh * Mh, per6 = 6 * L2;
  double* FV = SC;
  double* GG = FV + Mh * XS;
  double* HV = GG + Mh * XS;
  double* OV = HV + Mh * XS;
  double* OX = OV + Mh * XS;
  double* OE = OX + Mh * XS;
  for (int g = 0; g < 2; ++g) {
    const int pv = g, pP = 1 - g, McV = (N - pv) / 2 + 1, McP = (N - pP) / 2 + 1;
    const double* Dg = D + DL.block(g, 0);
    for (int t = threadIdx.x; t < Mh * SP; t += blockDim.x) {
      const int s = t % SP, j = t / SP, i = s >> 1, rho = s & 1;
      double fv = 0.0, gg = 0.0, hh = 0.0;
      if (i < nI) {
        const double* fr = FR + i * per6;
        if (mean) {
          const int Mc = (N - g) / 2 + 1;
          if (j < Mc) {
            fv = fr[(0 * 2 + rho) * L2 + g * Mh + j];
            gg = fr[(2 * 2 + rho) * L2 + g * Mh + j];
          }
        } else {
          if (j < McV) fv = fr[(1 * 2 + rho) * L2 + pv * Mh + j];
          if (j < McP) {
            const double fu = fr[(0 * 2 + (1 - rho)) * L2 + pP * Mh + j];
            const double fw = fr[(2 * 2 + (1 - rho)) * L2 + pP * Mh + j];
            const double sgn = rho == 0 ? -1.0 : 1.0;  // Re(i a) = -Im a, Im(i a) = Re a
            gg = sgn * fma(kx, fu, kz * fw);
            hh = sgn * fma(kz, fu, -kx * fw);
          }
        }
      }
      FV[j * XS + s] = fv;
      GG[j * XS + s] = gg;
      HV[j * XS + s] = hh;
    }
    __syncthreads();
    {
      // list A: v rows (Av f_v + Ag g; xi = -dv/dy follows below); mean mode: u and w rows
      const int Mc0 = (N - g) / 2 + 1;
      const int nA = mean ? 2 * Mc0 : McV, nB = mean ? 0 : McP;
      const int hA = (nA + 1) / 2, hB = (nB + 1) / 2;
      const int PA = round_up(hA, RW), PB = round_up(hB, RW);
      for (int t = threadIdx.x; t < (PA + PB) * SP; t += blockDim.x) {
        const int sc = t % SP, rs = t / SP;
        double a0 = 0.0, a1 = 0.0;
        double *out0, *out1;
        bool v0, v1;
        if (rs < PA) {
          v0 = rs < hA;
          v1 = v0 && rs + hA < nA;
          const int r0 = v0 ? rs : 0, r1 = v1 ? rs + hA : 0;
          if (mean) {
            const double* col0 = Dg + 2 * MM + r0;  // Eh
            const double* col1 = Dg + 2 * MM + (v1 ? r1 - Mc0 : 0);
            for (int j = 0; j < Mc0; ++j) {
              a0 = fma(col0[j * Mh], FV[j * XS + sc], a0);
              a1 = fma(col1[j * Mh], GG[j * XS + sc], a1);
            }
            out0 = OV + r0 * XS + sc;
            out1 = OX + (v1 ? r1 - Mc0 : 0) * XS + sc;
          } else {
            const double* cA0 = Dg + r0;  // Av
            const double* cA1 = Dg + r1;
            for (int j = 0; j < McV; ++j) {
              const double x = FV[j * XS + sc];
              a0 = fma(cA0[j * Mh], x, a0);
              a1 = fma(cA1[j * Mh], x, a1);
            }
            const double* cG0 = cA0 + MM;  // Ag
            const double* cG1 = cA1 + MM;
            for (int j = 0; j < McP; ++j) {
              const double x = GG[j * XS + sc];
              a0 = fma(cG0[j * Mh], x, a0);
              a1 = fma(cG1[j * Mh], x, a1);
            }
            out0 = OV + r0 * XS + sc;
            out1 = OV + r1 * XS + sc;
          }
        } else {
          const int q = rs - PA;
          v0 = q < hB;
          v1 = v0 && q + hB < nB;
          const int r0 = v0 ? q : 0, r1 = v1 ? q + hB : 0;
          const double* c0 = Dg + 2 * MM + r0;  // Eh
          const double* c1 = Dg + 2 * MM + r1;
          for (int j = 0; j < McP; ++j) {
            const double x = HV[j * XS + sc];
            a0 = fma(c0[j * Mh], x, a0);
            a1 = fma(c1[j * Mh], x, a1);
          }
          out0 = OE + r0 * XS + sc;
          out1 = OE + r1 * XS + sc;
        }
        if (v0) *out0 = a0;
        if (v1) *out1 = a1;
      }
    }
    __syncthreads();
    if (!mean) {  // xi = -dv/dy (class 1-g), one column per thread
      for (int s = threadIdx.x; s < SP; s += blockDim.x)
        xi_from_v(N, pv, OV + s, XS, OX + s, XS, I0.rco + RcoLayout(N).off(pv, 4));
      __syncthreads();
    }
    // assembly: v (class g) and u, w (class 1-g); mean mode: u, v = 0, w (class g)
    const int nV = mean ? (N - g) / 2 + 1 : McV;
    const int nU = mean ? nV : McP;
    const int nout = nV + 2 * nU;
    for (int t = threadIdx.x; t < nI * nout; t += blockDim.x) {
      const int i = t / nout, kk = t - i * nout;
      if (!live[i]) continue;
      int comp, row, n;
      double vr, vi;
      if (kk < nV) {
        comp = 1;
        row = kk;
        n = (mean ? g : pv) + 2 * row;
        vr = mean ? 0.0 : OV[row * XS + 2 * i];
        vi = mean ? 0.0 : OV[row * XS + 2 * i + 1];
      } else {
        const bool isu = kk < nV + nU;
        comp = isu ? 0 : 2;
        row = kk - nV - (isu ? 0 : nU);
        n = (mean ? g : pP) + 2 * row;
        if (mean) {
          const double* src = isu ? OV : OX;
          vr = src[row * XS + 2 * i];
          vi = src[row * XS + 2 * i + 1];
        } else {
          const double xr = OX[row * XS + 2 * i], xi = OX[row * XS + 2 * i + 1];
          const double er = OE[row * XS + 2 * i], ei = OE[row * XS + 2 * i + 1];
          if (isu) {
            vr = fma(kx, xi, kz * ei) * ik2;
            vi = -fma(kx, xr, kz * er) * ik2;
          } else {
            vr = fma(kz, xi, -kx * ei) * ik2;
            vi = fma(-kz, xr, kx * er) * ik2;
          }
        }
      }
      const Inst& I = gl.insts[first + i];
      const size_t gidx = ((size_t)comp * nm + m) * ny + n;
      const double* st = ST + (comp * ny + n) * XS + 2 * i;
      double nr, ni;
      if (phi) {
        nr = (vr - st[0]) * inv_step;
        ni = (vi - st[1]) * inv_step;
        I.rhat[gidx] = make_double2(nr, ni);
      } else {
        const double* uo = UH + (comp * ny + n) * XS + 2 * i;
        const double fr = -(vr - st[0]) * inv_step;
        const double fi = -(vi - st[1]) * inv_step;
        nr = fma(I.dtau, fr, uo[0]);
        ni = fma(I.dtau, fi, uo[1]);
        I.uhat[gidx] = make_double2(nr, ni);
      }
      double* o = OUT + (comp * 2 * H + (n & 1) * H + (n >> 1)) * XS + 2 * i;
      o[0] = nr;
      o[1] = ni;
    }
    // the next group's right-hand sides do not touch OV/OX/OE; its products wait at the barrier
  }
  __syncthreads();
  // ---- synthesis of the new coefficients: V_c (values) and W_c (y-derivative values)
  {
    const int hJ = (H + 1) / 2, JR = round_up(hJ, RW);
    const int slot = phi ? 1 : 0;
    for (int t = threadIdx.x; t < kFieldsY * JR * SP; t += blockDim.x) {
      const int sc = t % SP, rr = t / SP, qf = rr / JR, j0 = rr - qf * JR, j1 = j0 + hJ;
      const int c = qf < 3 ? qf : (qf == 3 ? 0 : 2);
      const bool deriv = qf >= 3;
      const bool v0 = j0 < hJ, v1 = v0 && j1 < H;
      const double* ME = CH + (deriv ? CL.De() : CL.Ce());
      const double* MO = CH + (deriv ? CL.Do() : CL.Co());
      const double* re0 = ME + (v0 ? j0 : 0) * H;
      const double* ro0 = MO + (v0 ? j0 : 0) * H;
      const double* re1 = ME + (v1 ? j1 : 0) * H;
      const double* ro1 = MO + (v1 ? j1 : 0) * H;
      const double* AE = OUT + c * 2 * H * XS + sc;
      const double* AO = AE + H * XS;
      double e0 = 0.0, o0 = 0.0, e1 = 0.0, o1 = 0.0;
      for (int k = 0; k < H; ++k) {
        const double x = AE[k * XS];
        e0 = fma(re0[k], x, e0);
        e1 = fma(re1[k], x, e1);
      }
      for (int k = 0; k < H - 1; ++k) {
        const double x = AO[k * XS];
        o0 = fma(ro0[k], x, o0);
        o1 = fma(ro1[k], x, o1);
      }
      const int i = sc >> 1, part = sc & 1;
      if (!v0 || i >= nI || !live[i]) continue;
      double* dst = reinterpret_cast<double*>(gl.insts[first + i].yv + ((size_t)slot * kFieldsY + qf) * ny * nm + m) + part;
      dst[(size_t)j0 * nm * 2] = e0 + o0;
      if (j0 < half) dst[(size_t)(N - j0) * nm * 2] = deriv ? o0 - e0 : e0 - o0;
      if (v1) {
        dst[(size_t)j1 * nm * 2] = e1 + o1;
        if (j1 < half) dst[(size_t)(N - j1) * nm * 2] = deriv ? o1 - e1 : e1 - o1;
      }
    }
  }
}

size_t smem_ystep(int N, int G) { return sizeof(double) * (size_t)step_layout(N, (int)col_pad_host(G)).total; }
void launch_ystep(int ctas, size_t smem, cudaStream_t s, GroupLaunch gl, int op) {
  k_ystep<<<ctas, kStepThreads, smem, s>>>(gl, op);
}
cudaError_t set_ystep_smem(size_t smem) {
  return raise_smem_limit((const void*)k_ystep, smem);
}

size_t smem_yanalysis(int N, int G, int mt) {
  const size_t H = N / 2 + 1, XS = col_pad_host(G) * mt + 1;
  return sizeof(double) * (2 * H * H + (2 * H) * XS);
}
// Stage buffer of the persistent solve (doubles): operator blocks + right-hand sides of G instances.
size_t ysolve_buffer(int N, int G) {
  const size_t Mh = N / 2 + 1, n3p = (3 * Mh * Mh + 1) & ~(size_t)1;
  return n3p + (size_t)G * 6 * (N + 2);
}
size_t smem_ysolve(int N, int G) {
  const size_t Mh = N / 2 + 1, XS = col_pad_host(G) + 1;
  return sizeof(double) * (2 * ysolve_buffer(N, G) + 6 * Mh * XS);
}
size_t smem_ysynth(int N, int G, int mt) {
  const size_t H = N / 2 + 1, XS = col_pad_host(G) * mt + 1;
  return sizeof(double) * (2 * H * H + (2 * H) * XS);
}
// Row tasks of one CTA, as the kernels count them (pairs of rows per lane in whole warps,
// then the lone middle row's single-chain tasks in FP64), and the threads for one pass.
static int tasks_ru(int a, int b) { return (a + b - 1) / b * b; }
int split_yanalysis_threads(int N, int G, int mt, bool fp64) {
  const int H = N / 2 + 1, half = N / 2, SPt = (int)col_pad_host(G) * mt, RW = 32 / SPt;
  const int hE = (H + 1) / 2, hO = (half + 1) / 2;
  const bool loneE = fp64 && (H & 1) && (hE - 1) % RW == 0, loneO = fp64 && (half & 1) && (hO - 1) % RW == 0;
  const int pE = hE - (loneE ? 1 : 0), pO = hO - (loneO ? 1 : 0);
  const int ntask = (tasks_ru(pE, RW) + tasks_ru(pO, RW)) * SPt + (loneE || loneO ? SPt : 0);
  return std::max(64, std::min(kAnalysisMaxThreads, tasks_ru(ntask, 32)));
}
int split_ysynth_threads(int N, int G, int mt, bool fp64) {
  const int H = N / 2 + 1, SPt = (int)col_pad_host(G) * mt, RW = 32 / SPt, hJ = (H + 1) / 2;
  const bool lone = fp64 && (H & 1) && (hJ - 1) % RW == 0;
  const int ntask = tasks_ru(hJ - (lone ? 1 : 0), RW) * SPt + (lone ? SPt : 0);
  return std::max(64, std::min(kSynthMaxThreads, tasks_ru(ntask, 32)));
}
void launch_yanalysis(int ctas, int threads, size_t smem, cudaStream_t s, GroupLaunch gl, int op, bool ff_arith,
                      int mt) {
  if (ff_arith) k_yanalysis<ff><<<ctas, threads, smem, s>>>(gl, op, mt);
  else k_yanalysis<double><<<ctas, threads, smem, s>>>(gl, op, mt);
}
void launch_ysolve(int ctas, int nitems, int bufsz, int scr_rows, size_t smem, cudaStream_t s, GroupLaunch gl,
                   int op) {
  k_ysolve<<<ctas, kSolveThreads, smem, s>>>(gl, op, nitems, bufsz, scr_rows);
}
void launch_jnorm(int ninst, cudaStream_t s, const Inst* insts, int step_index) {
  k_jnorm<<<ninst, 128, 0, s>>>(insts, step_index);
}
int ysolve_ctas_per_sm(size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ysolve, kSolveThreads, smem) != cudaSuccess) return 0;
  return n;
}
void launch_ysynth_split(int ctas, int threads, size_t smem, cudaStream_t s, GroupLaunch gl, int slot,
                         int check_active, bool ff_arith, int mt) {
  if (gl.reduced) {
    if (ff_arith) k_ysynth<ff, true><<<ctas, threads, smem, s>>>(gl, slot, check_active, mt);
    else k_ysynth<double, true><<<ctas, threads, smem, s>>>(gl, slot, check_active, mt);
  } else {
    if (ff_arith) k_ysynth<ff, false><<<ctas, threads, smem, s>>>(gl, slot, check_active, mt);
    else k_ysynth<double, false><<<ctas, threads, smem, s>>>(gl, slot, check_active, mt);
  }
}
cudaError_t set_split_smem(size_t analysis, size_t solve, size_t synth) {
  cudaError_t e;
  if ((e = raise_smem_limit((const void*)k_yanalysis<double>, analysis))) return e;
  if ((e = raise_smem_limit((const void*)k_yanalysis<ff>, analysis))) return e;
  if ((e = raise_smem_limit((const void*)k_ysolve, solve))) return e;
  if ((e = raise_smem_limit((const void*)k_ysynth<double, false>, synth))) return e;
  if ((e = raise_smem_limit((const void*)k_ysynth<double, true>, synth))) return e;
  if ((e = raise_smem_limit((const void*)k_ysynth<ff, true>, synth))) return e;
  return raise_smem_limit((const void*)k_ysynth<ff, false>, synth);
}

}  // namespace pcf
