// CUDA kernels (sm_103a) of one adjoint-descent step for plane Couette flow.
//
// Data flow of one descent step (paper §4, steps 1-5), per instance:
//   k_mode(SYNTH)      uhat -> y-values of u and du/dy at the Gauss-Lobatto points
//   k_xzsynth(slot 0)  -> 11 physical fields u, grad u on each y-plane (inverse FFT in x, z)
//   k_prod_M           -> M(u) per plane, forward FFT in z, x, 2/3 truncation
//   k_mode(PHI)        -> Chebyshev analysis, Stokes step (step 1), r1 (step 2), synthesis of r1
//   k_xzsynth(slot 1)  -> 11 physical fields r1, grad r1
//   k_prod_N           -> N(r1) per plane (+ plane sums of r1^2 for J), forward FFT
//   k_mode(PSI_UPDATE) -> analysis, Stokes step of the dummy dynamics (step 3), f (step 4),
//                         u += dtau f (step 5), synthesis of the new u for the next step
// The mode kernels work on Chebyshev columns of a few Fourier modes per CTA; the plane
// kernels on one y-plane of one field (or product component) per CTA.  All arithmetic is
// FP64; the FP64 pipe is the bound on GB300, so the transforms are radix-4/2/3 Stockham
// FFTs in shared memory (x, z) and parity-folded dense Chebyshev matrices (y).
#include "pcf_kernels.cuh"

namespace pcf {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ int find_inst(const LaunchInfo& li, int cta, int* local) {
  int lo = 0, hi = li.ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (li.prefix[mid] <= cta) lo = mid; else hi = mid - 1;
  }
  *local = cta - li.prefix[lo];
  return lo;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// x-storage index i (m = i for i <= Kx, m = i - Mx otherwise) -> FFT bin
__device__ __forceinline__ int xbin(int i, int Kx, int Mx, int nx) { return i <= Kx ? i : nx - (Mx - i); }

// ------------------------------------------------------------------ Stockham FFT in shared memory
template <int R>
__device__ __forceinline__ void butterfly(double2* v, bool inv);

template <>
__device__ __forceinline__ void butterfly<2>(double2* v, bool) {
  const double2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void butterfly<4>(double2* v, bool inv) {
  const double2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  const double2 t2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
  // t3 = -i d (forward) or +i d (inverse)
  const double2 t3 = inv ? make_double2(-d.y, d.x) : make_double2(d.y, -d.x);
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}

template <>
__device__ __forceinline__ void butterfly<3>(double2* v, bool inv) {
  const double h = 0.86602540378443864676;  // sin(2 pi/3)
  const double2 s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
  const double2 y0 = cadd(v[0], s);
  const double2 m = make_double2(fma(-0.5, s.x, v[0].x), fma(-0.5, s.y, v[0].y));
  const double2 t = make_double2(h * d.x, h * d.y);
  // forward: y1 = m - i t, y2 = m + i t
  const double2 it = make_double2(-t.y, t.x);
  v[0] = y0;
  v[1] = inv ? cadd(m, it) : csub(m, it);
  v[2] = inv ? csub(m, it) : cadd(m, it);
}

// One radix-R pass over nb contiguous batches of length L (Stockham autosort).
template <int R>
__device__ __forceinline__ void stockham_pass(const double2* __restrict__ a, double2* __restrict__ b, int L, int nb,
                                              int Ns, const double2* __restrict__ tw, bool inv) {
  const int nq = L / R;
  const int total = nq * nb;
  const int twstep = L / (Ns * R);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int bi = t / nq;
    const int j = t - bi * nq;
    const int k = j % Ns;
    const double2* ab = a + bi * L;
    double2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ab[j + r * nq];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        double2 w = tw[r * k * twstep];
        if (inv) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    butterfly<R>(v, inv);
    const int idx = (j / Ns) * Ns * R + k;
    double2* bb = b + bi * L;
#pragma unroll
    for (int r = 0; r < R; ++r) bb[idx + r * Ns] = v[r];
  }
}

// Full transform of nb batches; a holds the input; returns the buffer with the result.
__device__ double2* fft_run(double2* a, double2* b, int L, int nb, const int* radix, int nr, const double2* tw,
                            bool inv) {
  int Ns = 1;
  for (int s = 0; s < nr; ++s) {
    const int R = radix[s];
    if (R == 4) stockham_pass<4>(a, b, L, nb, Ns, tw, inv);
    else if (R == 2) stockham_pass<2>(a, b, L, nb, Ns, tw, inv);
    else stockham_pass<3>(a, b, L, nb, Ns, tw, inv);
    __syncthreads();
    double2* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

__device__ __forceinline__ void load_twiddles(const Inst& I, double2* twx, double2* twz) {
  for (int t = threadIdx.x; t < I.nx; t += blockDim.x) twx[t] = I.twx[t];
  for (int t = threadIdx.x; t < I.nz; t += blockDim.x) twz[t] = I.twz[t];
}

__host__ __device__ inline size_t plane_buf_elems(const Inst& I) {
  const size_t a = (size_t)I.Mz * I.nx, b = (size_t)(I.nx / 2) * I.nz;
  return a > b ? a : b;
}
size_t smem_xzsynth(const Inst& I) { return sizeof(double2) * (2 * plane_buf_elems(I) + I.nx + I.nz); }
size_t smem_prod(const Inst& I) { return sizeof(double2) * (2 * plane_buf_elems(I) + I.nx + I.nz) + 8 * 32; }

__device__ __forceinline__ bool inst_active(const Inst& I) { return I.active == nullptr || *I.active != 0; }

// ------------------------------------------------------------------ plane synthesis
// CTA = (instance, y-plane j, field f).  Field f of slot: 0 u, 1 v, 2 w, 3 u_x, 4 u_y,
// 5 u_z, 6 v_x, 7 v_z, 8 w_x, 9 w_y, 10 w_z, made from the y-values V0 V1 V2 W0 W2.
__constant__ int c_src[kFieldsSynth] = {0, 1, 2, 0, 3, 0, 1, 1, 2, 4, 2};
__constant__ int c_fac[kFieldsSynth] = {0, 0, 0, 1, 0, 2, 1, 2, 1, 0, 2};

__global__ void __launch_bounds__(128) k_xzsynth(LaunchInfo li, int slot, int nfields) {
  extern __shared__ double2 sm[];
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  if (!inst_active(I)) return;
  const int f = local % nfields, j = local / nfields;
  const int nx = I.nx, nz = I.nz, Mx = I.Mx, Mz = I.Mz, Kx = I.Kx, Kz = I.Kz;
  const size_t PB = plane_buf_elems(I);
  double2* B0 = sm;
  double2* B1 = sm + PB;
  double2* twx = sm + 2 * PB;
  double2* twz = twx + nx;
  load_twiddles(I, twx, twz);
  for (int t = threadIdx.x; t < Mz * nx; t += blockDim.x) B0[t] = make_double2(0.0, 0.0);
  __syncthreads();
  const double2* src = I.yv + (((size_t)slot * kFieldsY + c_src[f]) * I.ny + j) * (size_t)I.nmodes;
  const int fac = c_fac[f];
  for (int t = threadIdx.x; t < I.nmodes; t += blockDim.x) {
    const int i = t / Mz, p = t - i * Mz;
    double2 s = src[t];
    if (fac == 1) { const double k = I.kx[i]; s = make_double2(-k * s.y, k * s.x); }
    else if (fac == 2) { const double k = I.kz[p]; s = make_double2(-k * s.y, k * s.x); }
    B0[p * nx + xbin(i, Kx, Mx, nx)] = s;
  }
  __syncthreads();
  double2* G = fft_run(B0, B1, nx, Mz, I.rx, I.nrx, twx, true);
  double2* Hb = (G == B0) ? B1 : B0;
  const int nr = nx / 2;
  for (int t = threadIdx.x; t < nr * nz; t += blockDim.x) {
    const int r = t / nz, z = t - r * nz;
    const int x1 = 2 * r, x2 = x1 + 1;
    double2 h = make_double2(0.0, 0.0);
    if (z == 0) {
      h = make_double2(G[x1].x, G[x2].x);
    } else if (z <= Kz) {
      const double2 g1 = G[z * nx + x1], g2 = G[z * nx + x2];
      h = make_double2(g1.x - g2.y, g1.y + g2.x);
    } else if (z >= nz - Kz) {
      const int p = nz - z;
      const double2 g1 = G[p * nx + x1], g2 = G[p * nx + x2];
      h = make_double2(g1.x + g2.y, g2.x - g1.y);
    }
    Hb[t] = h;
  }
  __syncthreads();
  double2* Rz = fft_run(Hb, G, nz, nr, I.rz, I.nrz, twz, true);
  double* out = I.phys + (((size_t)slot * kFieldsSynth + f) * I.ny + j) * (size_t)nx * nz;
  for (int t = threadIdx.x; t < nr * nz; t += blockDim.x) {
    const int r = t / nz, z = t - r * nz;
    const double2 h = Rz[t];
    out[(2 * r) * nz + z] = h.x;
    out[(2 * r + 1) * nz + z] = h.y;
  }
}

// ------------------------------------------------------------------ products + analysis
// Field pointer of slot s, field f, plane j.
__device__ __forceinline__ const double* fplane(const Inst& I, int s, int f, int j) {
  return I.phys + (((size_t)s * kFieldsSynth + f) * I.ny + j) * (size_t)I.nx * I.nz;
}

// gradient component d_d (d = 0 x, 1 y, 2 z) of velocity component c at point e of plane j
__device__ __forceinline__ double grad_at(const double* const* F, int c, int d, int e) {
  // fields: 3 u_x, 4 u_y, 5 u_z, 6 v_x, 7 v_z, 8 w_x, 9 w_y, 10 w_z; v_y = -u_x - w_z
  if (c == 0) return F[3 + d][e];
  if (c == 2) return F[8 + d][e];
  if (d == 0) return F[6][e];
  if (d == 2) return F[7][e];
  return -(F[3][e] + F[10][e]);
}

// Forward 2D transform of the product plane held in Hb as pairs of rows, 2/3 truncation.
__device__ void analyse_plane(const Inst& I, double2* Hb, double2* Ob, const double2* twx, const double2* twz,
                              double2* dst) {
  const int nx = I.nx, nz = I.nz, Mx = I.Mx, Mz = I.Mz, Kx = I.Kx;
  const int nr = nx / 2;
  double2* R = fft_run(Hb, Ob, nz, nr, I.rz, I.nrz, twz, false);
  double2* X = (R == Hb) ? Ob : Hb;
  for (int t = threadIdx.x; t < nr * Mz; t += blockDim.x) {
    const int r = t / Mz, p = t - r * Mz;
    const double2 hp = R[r * nz + p];
    const double2 hm = R[r * nz + (p == 0 ? 0 : nz - p)];
    const double2 g1 = make_double2(0.5 * (hp.x + hm.x), 0.5 * (hp.y - hm.y));
    const double2 g2 = make_double2(0.5 * (hp.y + hm.y), -0.5 * (hp.x - hm.x));
    X[p * nx + 2 * r] = g1;
    X[p * nx + 2 * r + 1] = g2;
  }
  __syncthreads();
  double2* Y = fft_run(X, R, nx, Mz, I.rx, I.nrx, twx, false);
  const double s = I.inv_nxnz;
  for (int t = threadIdx.x; t < I.nmodes; t += blockDim.x) {
    const int i = t / Mz, p = t - i * Mz;
    const double2 v = Y[p * nx + xbin(i, Kx, Mx, nx)];
    dst[t] = make_double2(v.x * s, v.y * s);
  }
}

// CTA = (instance, plane j, component c): M_c = -y d_x u_c - v [c=x] - (u.grad) u_c.
__global__ void __launch_bounds__(128) k_prod_M(LaunchInfo li) {
  extern __shared__ double2 sm[];
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  if (!inst_active(I)) return;
  const int c = local % 3, j = local / 3;
  const int nx = I.nx, nz = I.nz;
  const size_t PB = plane_buf_elems(I);
  double2* B0 = sm;
  double2* B1 = sm + PB;
  double2* twx = sm + 2 * PB;
  double2* twz = twx + nx;
  load_twiddles(I, twx, twz);
  const double* F[kFieldsSynth];
#pragma unroll
  for (int f = 0; f < kFieldsSynth; ++f) F[f] = fplane(I, 0, f, j);
  const double y = I.ygrid[j];
  const int nr = nx / 2;
  for (int t = threadIdx.x; t < nr * nz; t += blockDim.x) {
    const int r = t / nz, z = t - r * nz;
    double m[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = (2 * r + h) * nz + z;
      const double u = F[0][e], v = F[1][e], w = F[2][e];
      const double gx = grad_at(F, c, 0, e), gy = grad_at(F, c, 1, e), gz = grad_at(F, c, 2, e);
      double val = -fma(y + u, gx, fma(v, gy, w * gz));
      if (c == 0) val -= v;
      m[h] = val;
    }
    B0[t] = make_double2(m[0], m[1]);
  }
  __syncthreads();
  analyse_plane(I, B0, B1, twx, twz, I.xz + ((size_t)c * I.ny + j) * I.nmodes);
}

// CTA = (instance, plane j, component c):
// N_c = (U.grad) q_c - q_j d_c U_j with U = (y + u, v, w), plus sum over the plane of q_c^2.
__global__ void __launch_bounds__(128) k_prod_N(LaunchInfo li) {
  extern __shared__ double2 sm[];
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  if (!inst_active(I)) return;
  const int c = local % 3, j = local / 3;
  const int nx = I.nx, nz = I.nz;
  const size_t PB = plane_buf_elems(I);
  double2* B0 = sm;
  double2* B1 = sm + PB;
  double2* twx = sm + 2 * PB;
  double2* twz = twx + nx;
  double* red = reinterpret_cast<double*>(twz + nz);
  load_twiddles(I, twx, twz);
  const double* U[kFieldsSynth];
  const double* Q[kFieldsSynth];
#pragma unroll
  for (int f = 0; f < kFieldsSynth; ++f) {
    U[f] = fplane(I, 0, f, j);
    Q[f] = fplane(I, 1, f, j);
  }
  const double y = I.ygrid[j];
  const int nr = nx / 2;
  double sq = 0.0;
  for (int t = threadIdx.x; t < nr * nz; t += blockDim.x) {
    const int r = t / nz, z = t - r * nz;
    double m[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int e = (2 * r + h) * nz + z;
      const double u = U[0][e], v = U[1][e], w = U[2][e];
      const double q0 = Q[0][e], q1 = Q[1][e], q2 = Q[2][e];
      const double qc = Q[c][e];
      sq = fma(qc, qc, sq);
      const double adv = fma(y + u, grad_at(Q, c, 0, e), fma(v, grad_at(Q, c, 1, e), w * grad_at(Q, c, 2, e)));
      const double tr = fma(q0, grad_at(U, 0, c, e), fma(q1, grad_at(U, 1, c, e), q2 * grad_at(U, 2, c, e)));
      double val = adv - tr;
      if (c == 1) val -= q0;
      m[h] = val;
    }
    B0[t] = make_double2(m[0], m[1]);
  }
  // deterministic block reduction of sum q_c^2
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    I.normpart[(size_t)c * I.ny + j] = s;
  }
  analyse_plane(I, B0, B1, twx, twz, I.xz + ((size_t)c * I.ny + j) * I.nmodes);
}

// CTA = (instance, plane j, component c): sum over the plane of q_c^2 (slot 1, field c).
__global__ void __launch_bounds__(128) k_norm_planes(LaunchInfo li) {
  __shared__ double red[32];
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  const int c = local % 3, j = local / 3;
  const double* q = fplane(I, 1, c, j);
  double sq = 0.0;
  for (int t = threadIdx.x; t < I.nx * I.nz; t += blockDim.x) sq = fma(q[t], q[t], sq);
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    I.normpart[(size_t)c * I.ny + j] = s;
  }
}

// J = sqrt(0.5 * sum_j w_j * mean_{x,z} |q|^2) from the plane sums (fixed order).
__device__ double norm_from_parts(const Inst& I) {
  double s = 0.0;
  for (int j = 0; j < I.ny; ++j) {
    const double pj = I.normpart[j] + I.normpart[I.ny + j] + I.normpart[2 * I.ny + j];
    s = fma(I.ccw[j], pj, s);
  }
  return sqrt(0.5 * I.inv_nxnz * s);
}

__global__ void k_norm_final(LaunchInfo li, double* out) {
  for (int b = threadIdx.x; b < li.ninst; b += blockDim.x) out[b] = norm_from_parts(li.insts[b]);
}

// ------------------------------------------------------------------ per-mode kernel
size_t smem_mode(const Inst& I, int mpc) {
  // cheb + rco + per mode: solver table, Fr/U0/Out ([3][2][L2] each), chain scratch [4][6][Mh]
  const int N = I.N, Mh = N / 2 + 1, H = Mh, L2 = 2 * Mh;
  const TabLayout TL(N);
  size_t d = 6 * (size_t)H * H + 10 * (size_t)Mh;
  d += (size_t)mpc * (TL.per_mode() + 18 * (size_t)L2 + 24 * (size_t)Mh);
  return d * sizeof(double);
}

__global__ void __launch_bounds__(128) k_mode(LaunchInfo li, int op, int sig, int mpc_arg, int step_index) {
  extern __shared__ double smd[];
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  const int mpc = I.mpc > 0 ? I.mpc : mpc_arg;
  const int N = I.N, Mh = N / 2 + 1, H = Mh, L2 = 2 * Mh, ny = I.ny;
  const int nm = I.nmodes, Mz = I.Mz;
  const int m0 = local * mpc;
  const int nmod = min(mpc, nm - m0);
  const TabLayout TL(N);
  const RcoLayout RL(N);
  const ChebLayout CL(N);
  const bool solve = (op != MODE_SYNTH_ONLY);

  // descent: norm of r1 (computed by k_prod_N), history and convergence decision
  if (op == MODE_PSI_UPDATE) {
    if (!inst_active(I)) return;
    const double J = norm_from_parts(I);
    if (local == 0 && threadIdx.x == 0 && I.hist) I.hist[(size_t)step_index * I.hist_stride] = J;
    if (I.tol > 0.0 && J < I.tol) {
      if (local == 0 && threadIdx.x == 0 && I.active) *I.active = 0;
      return;
    }
  } else if (op != MODE_SOLVE && op != MODE_SYNTH_ONLY && !inst_active(I)) {
    return;
  }

  double* cheb = smd;
  double* rco = cheb + CL.total();
  double* tabs = rco + RL.total();
  const int PM = TL.per_mode();
  double* Fr = tabs + (size_t)mpc * PM;          // [mpc][3][2][L2]
  double* U0 = Fr + (size_t)mpc * 6 * L2;        // [mpc][3][2][L2]
  double* Out = U0 + (size_t)mpc * 6 * L2;       // [mpc][3][2][L2] (also y-values input)
  double* Ch = Out + (size_t)mpc * 6 * L2;       // [mpc][4][6][Mh]

  for (int t = threadIdx.x; t < CL.total(); t += blockDim.x) cheb[t] = I.cheb[t];
  for (int t = threadIdx.x; t < RL.total(); t += blockDim.x) rco[t] = I.rco[t];
  const double* tabg = solve ? I.tab[sig] : nullptr;
  if (solve && !I.dense[sig])
    for (int t = threadIdx.x; t < nmod * PM; t += blockDim.x) tabs[t] = tabg[(size_t)m0 * PM + t];

  // state coefficients of the input (u for PHI/SYNTH, r1 for PSI, rhs for SOLVE), class-split
  const double2* insrc = (op == MODE_PHI || (op == MODE_SYNTH_ONLY && sig == 0)) ? I.uhat : I.rhat;
  for (int t = threadIdx.x; t < nmod * 3 * ny; t += blockDim.x) {
    const int n = t % ny, mc = t / ny, c = mc % 3, mm = mc / 3;
    const double2 v = insrc[((size_t)c * nm + m0 + mm) * ny + n];
    double* dst = U0 + ((size_t)mm * 3 + c) * 2 * L2 + (n & 1) * Mh + (n >> 1);
    dst[0] = v.x;
    dst[L2] = v.y;
  }
  // y-values of the products at this CTA's modes
  if (op == MODE_PHI || op == MODE_PSI_UPDATE || op == MODE_PSI_GRAD) {
    for (int t = threadIdx.x; t < nmod * 3 * ny; t += blockDim.x) {
      const int mm = t % nmod, cj = t / nmod, j = cj % ny, c = cj / ny;
      const double2 v = I.xz[((size_t)c * ny + j) * nm + m0 + mm];
      double* dst = Out + ((size_t)mm * 3 + c) * 2 * L2 + j;
      dst[0] = v.x;
      dst[L2] = v.y;
    }
  }
  __syncthreads();

  const double step = sig == 0 ? I.dt : I.dtau_hat;
  const double inv_step = 1.0 / step;
  const double inv_nu = 1.0 / I.nu;
  const int half = N / 2;
  if (solve) {
    if (op != MODE_SOLVE) {
      // fold y-values: P_j = V_j + V_{N-j} (at j), Q_j = V_j - V_{N-j} (at N-j), j < N/2
      for (int t = threadIdx.x; t < nmod * 6 * half; t += blockDim.x) {
        const int j = t % half, a = t / half;
        double* v = Out + (size_t)a * L2;
        const double p = v[j], q = v[N - j];
        v[j] = p + q;
        v[N - j] = p - q;
      }
      __syncthreads();
      // Chebyshev analysis + right-hand side F = (state/step + product)/nu
      const double* Ae = cheb + CL.Ae();
      const double* Ao = cheb + CL.Ao();
      for (int t = threadIdx.x; t < nmod * 3 * (2 * H - 1); t += blockDim.x) {
        const int k2 = t % (2 * H - 1), mc = t / (2 * H - 1);
        const double* v = Out + (size_t)mc * 2 * L2;
        double ar = 0.0, ai = 0.0;
        int pos;
        if (k2 < H) {
          const double* row = Ae + k2 * H;
          for (int j = 0; j < H; ++j) { ar = fma(row[j], v[j], ar); ai = fma(row[j], v[L2 + j], ai); }
          pos = k2;
        } else {
          const int k = k2 - H;
          const double* row = Ao + k * H;
          for (int j = 0; j < half; ++j) { ar = fma(row[j], v[N - j], ar); ai = fma(row[j], v[L2 + N - j], ai); }
          pos = Mh + k;
        }
        const double* u0 = U0 + (size_t)mc * 2 * L2;
        double* fr = Fr + (size_t)mc * 2 * L2;
        fr[pos] = fma(u0[pos], inv_step, ar) * inv_nu;
        fr[L2 + pos] = fma(u0[L2 + pos], inv_step, ai) * inv_nu;
      }
    } else {
      for (int t = threadIdx.x; t < nmod * 6 * L2; t += blockDim.x) Fr[t] = U0[t] * inv_nu;
    }
    __syncthreads();

    const double sigma = I.sigma[sig];
    const double* dn = I.dense[sig];
    if (dn) {
      // Stokes step with the dense per-mode operators: inputs g, h per (mode, group, part)
      const DenseLayout DL(N);
      for (int t = threadIdx.x; t < nmod * 4 * Mh; t += blockDim.x) {
        const int i = t % Mh, c4 = t / Mh, mm = c4 >> 2, g = (c4 >> 1) & 1, rho = c4 & 1;
        const int pP = 1 - g, McP = (N - pP) / 2 + 1;
        const int m = m0 + mm, ix = m / Mz, p = m - ix * Mz;
        const double kx = I.kx[ix], kz = I.kz[p];
        if (i >= McP || (kx == 0.0 && kz == 0.0)) continue;
        const double* fr = Fr + (size_t)mm * 6 * L2;
        const double fu = fr[(0 * 2 + (1 - rho)) * L2 + pP * Mh + i];
        const double fw = fr[(2 * 2 + (1 - rho)) * L2 + pP * Mh + i];
        const double sgn = rho == 0 ? -1.0 : 1.0;
        double* sc = Ch + ((size_t)mm * 4 + g * 2 + rho) * 6 * Mh;
        sc[i] = sgn * fma(kx, fu, kz * fw);
        sc[Mh + i] = sgn * fma(kz, fu, -kx * fw);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < nmod * 4 * 3 * Mh; t += blockDim.x) {
        const int r = t % Mh, q = t / Mh, which = q % 3, c4 = q / 3, mm = c4 >> 2, g = (c4 >> 1) & 1,
                  rho = c4 & 1;
        const int pv = g, pP = 1 - g, McV = (N - pv) / 2 + 1, McP = (N - pP) / 2 + 1;
        const int m = m0 + mm, ix = m / Mz, p = m - ix * Mz;
        const double kx = I.kx[ix], kz = I.kz[p];
        const double* D = dn + (size_t)m * DL.per_mode();
        const double* fr = Fr + (size_t)mm * 6 * L2;
        double* sc = Ch + ((size_t)mm * 4 + g * 2 + rho) * 6 * Mh;
        if (kx == 0.0 && kz == 0.0) {
          // mean mode: u (which 0) and w (which 1) of class g
          const int Mc = (N - g) / 2 + 1;
          if (which == 2 || r >= Mc) continue;
          const double* row = D + DL.block(g, 4) + r * Mh;
          const double* f = fr + ((which == 0 ? 0 : 2) * 2 + rho) * L2 + g * Mh;
          double a = 0.0;
          for (int j = 0; j < Mc; ++j) a = fma(__ldg(row + j), f[j], a);
          sc[(which == 0 ? 0 : Mh) + r] = a;
          continue;
        }
        const double* fv = fr + (1 * 2 + rho) * L2 + pv * Mh;
        if (which == 0) {
          if (r >= McV) continue;
          const double* ra = D + DL.block(g, 0) + r * Mh;
          const double* rg = D + DL.block(g, 1) + r * Mh;
          double a = 0.0;
          for (int j = 0; j < McV; ++j) a = fma(__ldg(ra + j), fv[j], a);
          for (int j = 0; j < McP; ++j) a = fma(__ldg(rg + j), sc[j], a);
          sc[2 * Mh + r] = a;
        } else if (which == 1) {
          if (r >= McP) continue;
          const double* ra = D + DL.block(g, 2) + r * Mh;
          const double* rg = D + DL.block(g, 3) + r * Mh;
          double a = 0.0;
          for (int j = 0; j < McV; ++j) a = fma(__ldg(ra + j), fv[j], a);
          for (int j = 0; j < McP; ++j) a = fma(__ldg(rg + j), sc[j], a);
          sc[3 * Mh + r] = a;
        } else {
          if (r >= McP) continue;
          const double* re = D + DL.block(g, 4) + r * Mh;
          double a = 0.0;
          for (int j = 0; j < McP; ++j) a = fma(__ldg(re + j), sc[Mh + j], a);
          sc[4 * Mh + r] = a;
        }
      }
    } else {
    // Stokes step: 4 chains per mode (group x part)
      for (int t = threadIdx.x; t < nmod * 4; t += blockDim.x) {
        const int mm = t >> 2, g = (t >> 1) & 1, rho = t & 1;
        const int m = m0 + mm, i = m / Mz, p = m - i * Mz;
        const double kx = I.kx[i], kz = I.kz[p];
        const double k2 = kx * kx + kz * kz;
        const double* tab = tabs + (size_t)mm * PM;
        const double* fr = Fr + (size_t)mm * 6 * L2;
        double* sc = Ch + ((size_t)mm * 4 + g * 2 + rho) * 6 * Mh;
        if (k2 == 0.0) {
          // mean mode: v = 0, Dirichlet Helmholtz problems for u and w (class g, part rho)
          const int Mc = (N - g) / 2 + 1;
          const double* s = tab + TL.solver(1, g);
          for (int c = 0; c < 3; c += 2) {
            tau_solve(Mc, s, s + Mh, s + 2 * Mh, s + 3 * Mh, s[4 * Mh], rco + RL.off(g, 0), rco + RL.off(g, 1),
                      rco + RL.off(g, 2), fr + (c * 2 + rho) * L2 + g * Mh, 0.0, sc + (c == 0 ? 0 : Mh));
          }
        } else {
          mode_chain(N, g, rho, kx, kz, sigma + k2, tab, rco, fr, L2, sc);
        }
      }
    }
    __syncthreads();
    // assemble u, v, w (class-split) from v, xi, eta
    for (int t = threadIdx.x; t < nmod * L2; t += blockDim.x) {
      const int mm = t / L2, pos = t - mm * L2;
      const int par = pos >= Mh ? 1 : 0, i = pos - par * Mh;
      const int Mc = (N - par) / 2 + 1;
      double* o = Out + (size_t)mm * 6 * L2;
      if (i >= Mc) {
        for (int a = 0; a < 6; ++a) o[a * L2 + pos] = 0.0;
        continue;
      }
      const int m = m0 + mm, ix = m / Mz, p = m - ix * Mz;
      const double kx = I.kx[ix], kz = I.kz[p];
      const double k2 = kx * kx + kz * kz;
      const double* chv_re = Ch + ((size_t)mm * 4 + par * 2 + 0) * 6 * Mh;
      const double* chv_im = Ch + ((size_t)mm * 4 + par * 2 + 1) * 6 * Mh;
      if (k2 == 0.0) {
        o[0 * L2 + pos] = chv_re[i];
        o[1 * L2 + pos] = chv_im[i];
        o[2 * L2 + pos] = 0.0;
        o[3 * L2 + pos] = 0.0;
        o[4 * L2 + pos] = chv_re[Mh + i];
        o[5 * L2 + pos] = chv_im[Mh + i];
        continue;
      }
      const double* cxe_re = Ch + ((size_t)mm * 4 + (1 - par) * 2 + 0) * 6 * Mh;
      const double* cxe_im = Ch + ((size_t)mm * 4 + (1 - par) * 2 + 1) * 6 * Mh;
      const double xr = cxe_re[3 * Mh + i], xi = cxe_im[3 * Mh + i];
      const double er = cxe_re[4 * Mh + i], ei = cxe_im[4 * Mh + i];
      const double ik2 = 1.0 / k2;
      o[0 * L2 + pos] = fma(kx, xi, kz * ei) * ik2;
      o[1 * L2 + pos] = -fma(kx, xr, kz * er) * ik2;
      o[2 * L2 + pos] = chv_re[2 * Mh + i];
      o[3 * L2 + pos] = chv_im[2 * Mh + i];
      o[4 * L2 + pos] = fma(kz, xi, -kx * ei) * ik2;
      o[5 * L2 + pos] = fma(-kz, xr, kx * er) * ik2;
    }
    __syncthreads();
  }

  // outputs and the field to synthesise (class-split, in Fr)
  double2* gout = nullptr;
  double scale = 0.0;
  int slot = -1;
  if (op == MODE_PHI) { gout = I.rhat; scale = 1.0 / I.dt; slot = 1; }
  if (op == MODE_PSI_UPDATE) { slot = 0; }
  if (op == MODE_PSI_GRAD) { gout = I.fhat; }
  if (op == MODE_SOLVE) { gout = I.fhat; }
  if (op == MODE_SYNTH_ONLY) { slot = sig; }
  for (int t = threadIdx.x; t < nmod * 3 * ny; t += blockDim.x) {
    const int n = t % ny, mc = t / ny, c = mc % 3, mm = mc / 3;
    const int pos = (n & 1) * Mh + (n >> 1);
    const size_t base = ((size_t)mm * 3 + c) * 2 * L2 + pos;
    const size_t gidx = ((size_t)c * nm + m0 + mm) * ny + n;
    double vr, vi;
    if (op == MODE_PHI) {
      vr = (Out[base] - U0[base]) * scale;
      vi = (Out[base + L2] - U0[base + L2]) * scale;
      gout[gidx] = make_double2(vr, vi);
    } else if (op == MODE_PSI_UPDATE || op == MODE_PSI_GRAD) {
      const double fr = -(Out[base] - U0[base]) * inv_step;
      const double fi = -(Out[base + L2] - U0[base + L2]) * inv_step;
      if (op == MODE_PSI_GRAD) {
        gout[gidx] = make_double2(fr, fi);
        continue;
      }
      const double2 u = I.uhat[gidx];
      vr = fma(I.dtau, fr, u.x);
      vi = fma(I.dtau, fi, u.y);
      I.uhat[gidx] = make_double2(vr, vi);
    } else if (op == MODE_SOLVE) {
      gout[gidx] = make_double2(Out[base], Out[base + L2]);
      continue;
    } else {
      vr = U0[base];
      vi = U0[base + L2];
    }
    Fr[base] = vr;
    Fr[base + L2] = vi;
  }
  if (slot < 0) return;
  __syncthreads();

  // Chebyshev synthesis: V_c (values) and W_c (y-derivative values) for c = u, v, w (W_v unused)
  const double* Ce = cheb + CL.Ce();
  const double* Co = cheb + CL.Co();
  const double* De = cheb + CL.De();
  const double* Do = cheb + CL.Do();
  double2* yv = I.yv + (size_t)slot * kFieldsY * ny * nm;
  for (int t = threadIdx.x; t < nmod * kFieldsY * H; t += blockDim.x) {
    const int mm = t % nmod, rest = t / nmod, j = rest % H, q = rest / H;
    const int c = q < 3 ? q : (q == 3 ? 0 : 2);
    const bool deriv = q >= 3;
    const double* a = Fr + ((size_t)mm * 3 + c) * 2 * L2;
    const double* re = deriv ? De + j * H : Ce + j * H;
    const double* ro = deriv ? Do + j * H : Co + j * H;
    double er = 0.0, ei = 0.0, orr = 0.0, oi = 0.0;
    for (int k = 0; k < H; ++k) { er = fma(re[k], a[k], er); ei = fma(re[k], a[L2 + k], ei); }
    for (int k = 0; k < H - 1; ++k) { orr = fma(ro[k], a[Mh + k], orr); oi = fma(ro[k], a[L2 + Mh + k], oi); }
    double2* dst = yv + (size_t)q * ny * nm + m0 + mm;
    if (!deriv) {
      dst[(size_t)j * nm] = make_double2(er + orr, ei + oi);
      if (j < half) dst[(size_t)(N - j) * nm] = make_double2(er - orr, ei - oi);
    } else {
      // T'_{2k} is odd, T'_{2k+1} even in y
      dst[(size_t)j * nm] = make_double2(er + orr, ei + oi);
      if (j < half) dst[(size_t)(N - j) * nm] = make_double2(orr - er, oi - ei);
    }
  }
}

// ------------------------------------------------------------------ FP64 throughput probe
__global__ void k_fp64_probe(double* out, int iters) {
  double a0 = threadIdx.x * 1e-9, a1 = a0 + 1e-9, a2 = a0 + 2e-9, a3 = a0 + 3e-9;
  double a4 = a0 + 4e-9, a5 = a0 + 5e-9, a6 = a0 + 6e-9, a7 = a0 + 7e-9;
  const double m = 0.999999999, c = 1e-12;
  for (int i = 0; i < iters; ++i) {
    a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
    a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
  }
  const double s = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  if (s == 12345.678) out[blockIdx.x] = s;  // keeps the loop alive
}

}  // namespace pcf
