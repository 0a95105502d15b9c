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
#include <map>
#include <mutex>
#include <utility>

#include "pcf_ff.cuh"
#include "pcf_kernels.cuh"
#include "pcf_plane_common.cuh"

namespace pcf {

cudaError_t raise_smem_limit(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> limit;  // (kernel, device) -> bytes set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[std::make_pair(func, dev)];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}


// One radix-R pass over nb batches of length L, batch b at b LS (Stockham autosort).  The
// plane kernels use LS = L + 1: a warp that walks down a column of a batch array then meets
// 32 different banks.
template <int R, class C, class TW>
__device__ __forceinline__ void stockham_pass(const C* __restrict__ a, C* __restrict__ b, int L, int LS, int nb,
                                              int Ns, const TW& tw, bool inv) {
  const int nq = L / R;
  const int total = nq * nb;
  const int twstep = L / (Ns * R);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int bi = t / nq;
    const int j = t - bi * nq;
    const int k = j % Ns;
    const C* ab = a + bi * LS;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ab[j + r * nq];
    if (Ns > 1) tw_butterfly<R>(v, tw, k, twstep, L, inv);
    else butterfly<R, C>(v, inv);
    const int idx = (j / Ns) * Ns * R + k;
    C* bb = b + bi * LS;
#pragma unroll
    for (int r = 0; r < R; ++r) bb[idx + r * Ns] = v[r];
  }
}

// Full transform of nb batches (stride LS); a holds the input; returns the buffer with the result.
template <class C, class TW>
__device__ C* fft_run(C* a, C* b, int L, int LS, int nb, const int* radix, int nr, const TW& tw, bool inv) {
  int Ns = 1;
  for (int s = 0; s < nr; ++s) {
    const int R = radix[s];
    if (R == 4) stockham_pass<4, C>(a, b, L, LS, nb, Ns, tw, inv);
    else if (R == 2) stockham_pass<2, C>(a, b, L, LS, nb, Ns, tw, inv);
    else stockham_pass<3, C>(a, b, L, LS, nb, Ns, tw, inv);
    __syncthreads();
    C* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// The same pass with its inputs read through ld(b, i) (element i of batch b) and its outputs
// written through st(b, i, v), so that a transform's first pass can read its input where it
// lies (and build it on the fly) and its last pass can write the result where it is needed,
// without shared-memory round trips and barriers of their own.  Same arithmetic as
// stockham_pass.
template <int R, class C, class TW, class LD, class ST>
__device__ __forceinline__ void stockham_pass_io(int L, int nb, int Ns, const TW& tw, bool inv, const LD& ld,
                                                 const ST& st) {
  const int nq = L / R;
  const int total = nq * nb;
  const int twstep = L / (Ns * R);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int bi = t / nq;
    const int j = t - bi * nq;
    const int k = j % Ns;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ld(bi, j + r * nq);
    if (Ns > 1) tw_butterfly<R>(v, tw, k, twstep, L, inv);
    else butterfly<R, C>(v, inv);
    const int idx = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) st(bi, idx + r * Ns, v[r]);
  }
}

template <class C>
struct SmemLd {
  const C* p;
  int LS;
  __device__ __forceinline__ C operator()(int b, int i) const { return p[b * LS + i]; }
};
template <class C>
struct SmemSt {
  C* p;
  int LS;
  __device__ __forceinline__ void operator()(int b, int i, C v) const { p[b * LS + i] = v; }
};

template <class C, class TW, class LD, class ST>
__device__ __forceinline__ void pass_r(int R, int L, int nb, int Ns, const TW& tw, bool inv, const LD& ld,
                                       const ST& st) {
  if (R == 4) stockham_pass_io<4, C>(L, nb, Ns, tw, inv, ld, st);
  else if (R == 2) stockham_pass_io<2, C>(L, nb, Ns, tw, inv, ld, st);
  else stockham_pass_io<3, C>(L, nb, Ns, tw, inv, ld, st);
}

// Full transform of nb batches whose first pass reads through ld.  The later passes
// ping-pong between a and b (stride LS), the first pass writing a.  With OUT_ST the last
// pass writes through st (returns null); otherwise the result stays in shared memory and
// the buffer holding it is returned.  A barrier follows every pass but the last.
template <bool OUT_ST, class C, class TW, class LD, class ST>
__device__ C* fft_run_io(C* a, C* b, int L, int LS, int nb, const int* radix, int nr, const TW& tw, bool inv,
                         const LD& ld, const ST& st) {
  int Ns = 1;
  C* cur = nullptr;
  C* out = a;
  for (int s = 0; s < nr; ++s) {
    const int R = radix[s];
    const bool first = s == 0, last = s == nr - 1 && OUT_ST;
    if (first && last) pass_r<C>(R, L, nb, Ns, tw, inv, ld, st);
    else if (first) pass_r<C>(R, L, nb, Ns, tw, inv, ld, SmemSt<C>{out, LS});
    else if (last) pass_r<C>(R, L, nb, Ns, tw, inv, SmemLd<C>{cur, LS}, st);
    else pass_r<C>(R, L, nb, Ns, tw, inv, SmemLd<C>{cur, LS}, SmemSt<C>{out, LS});
    Ns *= R;
    if (s < nr - 1) __syncthreads();
    cur = out;
    out = (out == a) ? b : a;
  }
  return OUT_ST ? nullptr : cur;
}

// Twiddles of the plane kernels in shared memory: the standard tables (FP32, float-float), or
// for FP64 the tangent-form entries of the transform's direction (inv: the inverse
// transform) and their rotation flags.  PlaneTw<T>::type is the pass functions' view.
template <class T>
struct PlaneTw {
  using C = typename Cx<T>::c;
  using type = TwStd<C>;
  static __device__ __forceinline__ type view(C* tw, unsigned char*) { return type{tw}; }
  static __device__ __forceinline__ void load(const Inst& I, C* twx, C* twz, unsigned char*, unsigned char*, bool) {
    const typename Sto<T>::c* sx = twx_of<T>(I);
    const typename Sto<T>::c* sz = twz_of<T>(I);
    for (int t = threadIdx.x; t < I.nx; t += blockDim.x) twx[t] = load_c<T>(sx[t]);
    for (int t = threadIdx.x; t < I.nz; t += blockDim.x) twz[t] = load_c<T>(sz[t]);
  }
};
template <>
struct PlaneTw<double> {
  using type = TwTan;
  static __device__ __forceinline__ type view(double2* tw, unsigned char* rot) { return type{tw, rot}; }
  static __device__ __forceinline__ void load(const Inst& I, double2* twx, double2* twz, unsigned char* rx,
                                              unsigned char* rz, bool inv) {
    const double2* sx = I.tanx + (inv ? I.nx : 0);
    const double2* sz = I.tanz + (inv ? I.nz : 0);
    for (int t = threadIdx.x; t < I.nx; t += blockDim.x) {
      twx[t] = sx[t];
      rx[t] = I.rotx[t];
    }
    for (int t = threadIdx.x; t < I.nz; t += blockDim.x) {
      twz[t] = sz[t];
      rz[t] = I.rotz[t];
    }
  }
};

// Shared-memory plan of a plane transform: two buffers of PB complex values; x-stage
// batches (one per retained z mode) have stride LX = nx + 1, z-stage batches (one per row
// pair) stride LZ = nz + 1.  The z stage handles `chunk` row pairs at a time: all of them
// when both stages fit the budget, else as many as fit (two ping-pong buffers) inside the
// partner of the x-stage buffer.
struct PlanePlan {
  int PB, chunk, LX, LZ;
};
__host__ __device__ inline PlanePlan plane_plan(const Inst& I, int elem) {
  PlanePlan pp;
  pp.LX = I.nx + 1;
  pp.LZ = I.nz + 1;
  const int a = I.Mz * pp.LX, b = (I.nx / 2) * pp.LZ;
  if ((size_t)2 * (a > b ? a : b) * elem <= 100 * 1024) {
    pp.PB = a > b ? a : b;
    pp.chunk = I.nx / 2;
  } else {
    pp.PB = a;
    pp.chunk = a / (2 * pp.LZ);
    if (pp.chunk < 1) pp.chunk = 1;
  }
  return pp;
}
// [B0 | B1 | twx (nx) | twz (nz) | 32 doubles of reduction | rotation flags of twx, twz]
size_t smem_plane(const Inst& I, int elem) {
  const PlanePlan pp = plane_plan(I, elem);
  return (size_t)elem * (2 * (size_t)pp.PB + I.nx + I.nz) + 8 * 32 + (size_t)((I.nx + I.nz + 15) & ~15);
}
size_t smem_xzsynth(const Inst& I) { return smem_plane(I, sizeof(double2)); }
size_t smem_prod(const Inst& I) { return smem_plane(I, sizeof(double2)); }


// ------------------------------------------------------------------ plane synthesis
// CTA = (instance, y-plane j, field f).  Field f of slot: 0 u, 1 v, 2 w, 3 u_x, 4 u_y,
// 5 u_z, 6 v_x, 7 v_z, 8 w_x, 9 w_y, 10 w_z, made from the y-values V0 V1 V2 W0 W2.
__constant__ int c_src[kFieldsSynth] = {0, 1, 2, 0, 3, 0, 1, 1, 2, 4, 2};
__constant__ int c_fac[kFieldsSynth] = {0, 0, 0, 1, 0, 2, 1, 2, 1, 0, 2};

// Resident CTAs per SM the synthesis kernel is compiled for (register budget).
#ifndef PCF_XZ_MINB
#define PCF_XZ_MINB 8
#endif

template <class T>
__global__ void __launch_bounds__(128, PCF_XZ_MINB) k_xzsynth_t(LaunchInfo li, int slot, int nfields) {
  using C = typename Cx<T>::c;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  if (!inst_active(I)) return;
  const int f = local % nfields, j = local / nfields;
  const int nx = I.nx, nz = I.nz, Mx = I.Mx, Mz = I.Mz, Kx = I.Kx, Kz = I.Kz;
  const PlanePlan pp = plane_plan(I, sizeof(C));
  C* B0 = sm;
  C* B1 = sm + pp.PB;
  C* twx = sm + 2 * pp.PB;
  C* twz = twx + nx;
  unsigned char* rtx = reinterpret_cast<unsigned char*>(twz + nz) + 8 * 32;
  unsigned char* rtz = rtx + nx;
  PlaneTw<T>::load(I, twx, twz, rtx, rtz, true);  // first used after the first pass's barrier
  const typename PlaneTw<T>::type tx = PlaneTw<T>::view(twx, rtx), tz = PlaneTw<T>::view(twz, rtz);
  const int LX = pp.LX, LZ = pp.LZ;
  const typename Sto<T>::c* src = yv_of<T>(I) + (((size_t)slot * kFieldsY + c_src[f]) * I.ny + j) * (size_t)I.nmodes;
  const int fac = c_fac[f];
  // x stage: batch p (retained z mode), element = x bin; the input is the y-values (times
  // i kx or i kz for the x and z derivatives); bins outside |m| <= Kx are zero
  const auto scaled = [&](C s, int i, int p) -> C {
    if (fac == 1) { const T k = (T)I.kx[i]; s = Cx<T>::mk(-k * s.y, k * s.x); }
    else if (fac == 2) { const T k = (T)I.kz[p]; s = Cx<T>::mk(-k * s.y, k * s.x); }
    return s;
  };
  // the y-values, converted and scaled once per mode in a coalesced loop, at their bins in B0
  // (the other bins are never read: the first pass returns zero for them)
  for (int t = threadIdx.x; t < I.nmodes; t += blockDim.x) {
    const int i = t / Mz, p = t - i * Mz;
    B0[p * LX + xbin(i, Kx, Mx, nx)] = scaled(load_c<T>(src[t]), i, p);
  }
  __syncthreads();
  const auto ldx = [&](int p, int bin) -> C {
    return (bin <= Kx || bin >= nx - Kx) ? B0[p * LX + bin] : Cx<T>::mk(0, 0);
  };
  C* G = fft_run_io<false, C>(B1, B0, nx, LX, Mz, I.rx, I.nrx, tx, true, ldx, SmemSt<C>{nullptr, 0});
  __syncthreads();
  C* Zb = (G == B0) ? B1 : B0;
  const int nr = nx / 2;
  T* out = phys_of<T>(I) + (((size_t)slot * kFieldsSynth + f) * I.ny + j) * (size_t)nx * nz;
  for (int r0 = 0; r0 < nr; r0 += pp.chunk) {
    const int nrc = min(pp.chunk, nr - r0);
    C* Z0 = Zb;
    C* Z1 = (pp.chunk == nr) ? G : Zb + pp.chunk * LZ;
    // Row pair (x1, x2) -> one complex row whose inverse z transform gives row x1 in the
    // real part and row x2 in the imaginary part: h_z = G_z[x1] + i G_z[x2] with
    // G_{-p} = conj(G_p) (p = 0: real parts only; |p| > Kz: zero), built as the first z
    // pass reads it.  Branch-free, so that a warp issues each multiply-add once for all its
    // lanes: s = +-1 picks the conjugate, and the multiply-adds by +-1 and 0 are exact.
    const auto ldz = [&](int r, int z) -> C {
      const int x1 = 2 * (r0 + r), x2 = x1 + 1;
      const bool lo = z <= Kz, hi = z >= nz - Kz;
      const int p = lo ? z : nz - z;
      C g1 = Cx<T>::mk(0, 0), g2 = g1;
      if (lo || hi) {
        g1 = G[p * LX + x1];
        g2 = G[p * LX + x2];
      }
      if (z == 0) g1.y = g2.y = T(0.0);
      const T sg = lo ? T(1.0) : T(-1.0);
      return Cx<T>::mk(fma(-sg, g2.y, g1.x), fma(sg, g1.y, g2.x));
    };
    // the last z pass writes rows x1 (real part) and x2 (imaginary part) of the plane
    const auto stz = [&](int r, int z, C h) {
      out[(2 * (r0 + r)) * nz + z] = h.x;
      out[(2 * (r0 + r) + 1) * nz + z] = h.y;
    };
    fft_run_io<true, C>(Z0, Z1, nz, LZ, nrc, I.rz, I.nrz, tz, true, ldz, stz);
    if (r0 + pp.chunk < nr) __syncthreads();  // the next chunk rewrites Z0
  }
}

// ------------------------------------------------------------------ products + analysis
template <class T>
__device__ __forceinline__ const T* fplane(const Inst& I, int s, int f, int j) {
  return phys_of<T>(I) + (((size_t)s * kFieldsSynth + f) * I.ny + j) * (size_t)I.nx * I.nz;
}

// The 11 field planes of a slot at one y-plane: field f at p + f fs (one base pointer and a
// stride instead of 11 pointers held in registers).
template <class T>
struct PlaneSet {
  const T* p;
  int fs;
  __device__ __forceinline__ const T* operator[](int f) const { return p + f * fs; }
};

// gradient component d_d (d = 0 x, 1 y, 2 z) of velocity component c at point e of plane j
template <class T>
__device__ __forceinline__ T grad_at(const PlaneSet<T>& F, int c, int d, int e) {
  // fields: 3 u_x, 4 u_y, 5 u_z, 6 v_x, 7 v_z, 8 w_x, 9 w_y, 10 w_z; v_y = -u_x - w_z
  if (c == 0) return F[3 + d][e];
  if (c == 2) return F[8 + d][e];
  if (d == 0) return F[6][e];
  if (d == 2) return F[7][e];
  return -(F[3][e] + F[10][e]);
}

// Pointwise products of the plane, row pairs packed as complex values.
// Ub, dUb: the base-flow profile U(y_j) and U'(y_j) of the plane; Vb: the base flow's
// constant wall-normal velocity (u_b = (U(y), Vb, 0)), added to the advecting v only when VB
// (so that the flows without suction keep their instruction count).
template <class T, bool ADJ, bool VB>
__device__ __forceinline__ void product_pair(const Inst& I, const PlaneSet<T>& U, const PlaneSet<T>& Q, int c, T Ub,
                                             T dUb, T Vb, int e0, int e1, T* m, typename Acc<T>::type* sq) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int e = h == 0 ? e0 : e1;
    const T u = U[0][e], v = U[1][e], w = U[2][e];
    const T va = VB ? v + Vb : v;  // wall-normal velocity of u_b + u
    if (!ADJ) {
      const T gx = grad_at<T>(U, c, 0, e), gy = grad_at<T>(U, c, 1, e), gz = grad_at<T>(U, c, 2, e);
      T val = -fma(Ub + u, gx, fma(va, gy, w * gz));
      if (c == 0) val -= dUb * v;
      m[h] = val;
    } else {
      const T q0 = Q[0][e], q1 = Q[1][e], q2 = Q[2][e];
      const T qc = Q[c][e];
      acc_sq(sq, qc);
      const T adv = fma(Ub + u, grad_at<T>(Q, c, 0, e), fma(va, grad_at<T>(Q, c, 1, e), w * grad_at<T>(Q, c, 2, e)));
      const T tr = fma(q0, grad_at<T>(U, 0, c, e), fma(q1, grad_at<T>(U, 1, c, e), q2 * grad_at<T>(U, 2, c, e)));
      T val = adv - tr;
      if (c == 1) val -= dUb * q0;
      m[h] = val;
    }
  }
}

// Products of the rows r0 .. r0 + nrc - 1 of a plane for component CC (a compile-time
// constant, so that the field indices fold).
template <class T, bool ADJ, int CC, bool VB>
__device__ __forceinline__ void product_rows(const Inst& I, const PlaneSet<T>& U, const PlaneSet<T>& Q, T Ub, T dUb,
                                             T Vb, int r0, int nrc, int nz, int LZ, typename Cx<T>::c* Z0,
                                             typename Acc<T>::type* sq) {
  for (int t = threadIdx.x; t < nrc * nz; t += blockDim.x) {
    const int r = t / nz, z = t - r * nz;
    const int e0 = (2 * (r0 + r)) * nz + z, e1 = e0 + nz;
    T m[2];
    product_pair<T, ADJ, VB>(I, U, Q, CC, Ub, dUb, Vb, e0, e1, m, sq);
    Z0[r * LZ + z] = Cx<T>::mk(m[0], m[1]);
  }
}

// product_rows for component c (uniform in the CTA)
template <class T, bool ADJ, bool VB>
__device__ __forceinline__ void product_rows_c(int c, const Inst& I, const PlaneSet<T>& U, const PlaneSet<T>& Q,
                                               T Ub, T dUb, T Vb, int r0, int nrc, int nz, int LZ,
                                               typename Cx<T>::c* Z0, typename Acc<T>::type* sq) {
  if (c == 0) product_rows<T, ADJ, 0, VB>(I, U, Q, Ub, dUb, Vb, r0, nrc, nz, LZ, Z0, sq);
  else if (c == 1) product_rows<T, ADJ, 1, VB>(I, U, Q, Ub, dUb, Vb, r0, nrc, nz, LZ, Z0, sq);
  else product_rows<T, ADJ, 2, VB>(I, U, Q, Ub, dUb, Vb, r0, nrc, nz, LZ, Z0, sq);
}

// CTA = (instance, plane j, component c): product component c on the plane (M(u) or
// N(q) with W = u_b + u = (U(y) + u, Vb + v, w)), forward FFT in z then x, 2/3
// truncation.  ADJ also sums q_c^2 over the plane (in FP64) for J.
// Register budgets: eight resident CTAs per SM for M(u); six for N(q), which holds both
// fields' plane pointers (at 8 x 32x33x32 its 792 CTAs then fit one wave of 152 SMs).
// VB: some instance of the launch has a base flow with suction (its own instantiation, so
// that the flows without suction keep their register allocation).
template <class T, bool ADJ, bool VB>
__global__ void __launch_bounds__(128, ADJ ? 6 : 8) k_prod_t(LaunchInfo li, int step_index) {
  using C = typename Cx<T>::c;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  if (!inst_active(I)) return;
  const int c = local % 3, j = local / 3;
  const int nx = I.nx, nz = I.nz, Mx = I.Mx, Mz = I.Mz, Kx = I.Kx;
  const PlanePlan pp = plane_plan(I, sizeof(C));
  C* B0 = sm;
  C* B1 = sm + pp.PB;
  C* twx = sm + 2 * pp.PB;
  C* twz = twx + nx;
  double* red = reinterpret_cast<double*>(twz + nz);
  unsigned char* rtx = reinterpret_cast<unsigned char*>(red + 32);
  unsigned char* rtz = rtx + nx;
  PlaneTw<T>::load(I, twx, twz, rtx, rtz, false);
  const typename PlaneTw<T>::type tx = PlaneTw<T>::view(twx, rtx), tz = PlaneTw<T>::view(twz, rtz);
  const int fs = I.ny * nx * nz;  // between the fields of a slot
  const PlaneSet<T> U{fplane<T>(I, 0, 0, j), fs};
  const PlaneSet<T> Q{ADJ ? fplane<T>(I, 1, 0, j) : nullptr, fs};
  const T Ub = (T)I.ubase[j], dUb = (T)I.ubase[I.ny + j];
  const T Vb = VB ? (T)I.ubase[2 * I.ny + j] : (T)0.0;  // suction velocity of the base flow
  const int nr = nx / 2, LX = pp.LX, LZ = pp.LZ;
  const bool whole = pp.chunk == nr;
  // the x-stage input X[p][x] lives in B0 when chunked (z chunks use B1), else decided below
  C* X = B0;
  typename Acc<T>::type sq = 0.0;
  __syncthreads();
  for (int r0 = 0; r0 < nr; r0 += pp.chunk) {
    const int nrc = min(pp.chunk, nr - r0);
    C* Z0 = whole ? B0 : B1;
    C* Z1 = whole ? B1 : B1 + pp.chunk * LZ;
    product_rows_c<T, ADJ, VB>(c, I, U, Q, Ub, dUb, Vb, r0, nrc, nz, LZ, Z0, &sq);
    __syncthreads();
    C* R = fft_run<C>(Z0, Z1, nz, LZ, nrc, I.rz, I.nrz, tz, false);
    if (whole) X = (R == B0) ? B1 : B0;
    for (int t = threadIdx.x; t < nrc * Mz; t += blockDim.x) {
      const int r = t / Mz, p = t - r * Mz;
      const C hp = R[r * LZ + p];
      const C hm = R[r * LZ + (p == 0 ? 0 : nz - p)];
      const T half = (T)0.5;
      X[p * LX + 2 * (r0 + r)] = Cx<T>::mk(half * (hp.x + hm.x), half * (hp.y - hm.y));
      X[p * LX + 2 * (r0 + r) + 1] = Cx<T>::mk(half * (hp.y + hm.y), -half * (hp.x - hm.x));
    }
    __syncthreads();
  }
  if (ADJ) {
    double sqd = acc_value(sq);
    for (int o = 16; o > 0; o >>= 1) sqd += __shfl_down_sync(0xffffffffu, sqd, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sqd;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      I.normpart[(size_t)c * I.ny + j] = s;
    }
  }
  C* Y = fft_run<C>(X, X == B0 ? B1 : B0, nx, LX, Mz, I.rx, I.nrx, tx, false);
  const T sc = (T)I.inv_nxnz;
  typename Sto<T>::c* dst = xz_of<T>(I) + ((size_t)c * I.ny + j) * I.nmodes;
  for (int t = threadIdx.x; t < I.nmodes; t += blockDim.x) {
    const int i = t / Mz, p = t - i * Mz;
    const C v = Y[p * LX + xbin(i, Kx, Mx, nx)];
    dst[t] = store_c<T>(Cx<T>::mk(v.x * sc, v.y * sc));
  }
  if (ADJ && step_index >= 0) {
    // J = ||r1|| once all 3 ny plane sums of the instance are written: the CTA that counts
    // last computes it (the chain of norm_from_parts, so the bits match the other paths),
    // writes the history entry, clears the mask when J < tol (the instance stops before this
    // step's update) and resets the counter for the next launch.
    __shared__ int last;
    if (threadIdx.x == 0) {
      __threadfence();
      last = atomicAdd(I.jcount, 1) == 3 * I.ny - 1;
    }
    __syncthreads();
    if (last) {  // uniform in the CTA
      // the plane buffers are free now: stage the per-plane sums and the weights
      const int ny = I.ny;
      const double* P = I.normpart;
      double* ps = reinterpret_cast<double*>(smraw);
      for (int q = threadIdx.x; q < ny; q += blockDim.x) {
        ps[q] = __ldcg(P + q) + __ldcg(P + ny + q) + __ldcg(P + 2 * ny + q);
        ps[ny + q] = I.ccw[q];
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < ny; ++q) s = fma(ps[ny + q], ps[q], s);
        const double J = sqrt(0.5 * I.inv_nxnz * s);
        if (I.hist) I.hist[(size_t)step_index * I.hist_stride] = J;
        if (I.tol > 0.0 && J < I.tol && I.active) *I.active = 0;
        *I.jcount = 0;
      }
    }
  }
}

// CTA = (instance, plane j, component c): sum over the plane of the squared velocity
// component c of a slot (0: u, 1: q).
template <class T>
__global__ void __launch_bounds__(128) k_norm_planes_t(LaunchInfo li, int slot) {
  __shared__ double red[32];
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  const int c = local % 3, j = local / 3;
  const T* q = fplane<T>(I, slot, c, j);
  typename Acc<T>::type sa = 0.0;
  for (int t = threadIdx.x; t < I.nx * I.nz; t += blockDim.x) acc_sq(&sa, q[t]);
  double sq = acc_value(sa);
  for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    I.normpart[(size_t)c * I.ny + j] = s;
  }
}

// host launchers (the kernel templates are instantiated in this translation unit only)
// plane arithmetic: 0 FP64, 1 FP32 (mixed form), 2 float-float
void launch_xzsynth(int kind, int ctas, size_t smem, cudaStream_t s, LaunchInfo li, int slot, int nf) {
  if (kind == 1) k_xzsynth_t<float><<<ctas, 128, smem, s>>>(li, slot, nf);
  else if (kind == 2) k_xzsynth_t<ff><<<ctas, 128, smem, s>>>(li, slot, nf);
  else k_xzsynth_t<double><<<ctas, 128, smem, s>>>(li, slot, nf);
}
template <class T, bool VB>
static void launch_prod_t(bool adj, int ctas, size_t smem, cudaStream_t s, LaunchInfo li, int step_index) {
  if (adj) k_prod_t<T, true, VB><<<ctas, 128, smem, s>>>(li, step_index);
  else k_prod_t<T, false, VB><<<ctas, 128, smem, s>>>(li, -1);
}
void launch_prod(int kind, bool adj, bool suction, int ctas, size_t smem, cudaStream_t s, LaunchInfo li,
                 int step_index) {
  if (kind == 1) {
    if (suction) launch_prod_t<float, true>(adj, ctas, smem, s, li, step_index);
    else launch_prod_t<float, false>(adj, ctas, smem, s, li, step_index);
  } else if (kind == 2) {
    if (suction) launch_prod_t<ff, true>(adj, ctas, smem, s, li, step_index);
    else launch_prod_t<ff, false>(adj, ctas, smem, s, li, step_index);
  } else {
    if (suction) launch_prod_t<double, true>(adj, ctas, smem, s, li, step_index);
    else launch_prod_t<double, false>(adj, ctas, smem, s, li, step_index);
  }
}
void launch_norm_planes(int kind, int ctas, cudaStream_t s, LaunchInfo li, int slot) {
  if (kind == 1) k_norm_planes_t<float><<<ctas, 128, 0, s>>>(li, slot);
  else if (kind == 2) k_norm_planes_t<ff><<<ctas, 128, 0, s>>>(li, slot);
  else k_norm_planes_t<double><<<ctas, 128, 0, s>>>(li, slot);
}
template <class T>
static cudaError_t set_plane_smem_t(size_t synth, size_t prod) {
  cudaError_t e;
  if ((e = raise_smem_limit((const void*)k_xzsynth_t<T>, synth))) return e;
  if ((e = raise_smem_limit((const void*)k_prod_t<T, false, false>, prod))) return e;
  if ((e = raise_smem_limit((const void*)k_prod_t<T, false, true>, prod))) return e;
  if ((e = raise_smem_limit((const void*)k_prod_t<T, true, true>, prod))) return e;
  return raise_smem_limit((const void*)k_prod_t<T, true, false>, prod);
}
cudaError_t set_plane_smem(int kind, size_t synth, size_t prod) {
  if (kind == 1) return set_plane_smem_t<float>(synth, prod);
  if (kind == 2) return set_plane_smem_t<ff>(synth, prod);
  return set_plane_smem_t<double>(synth, prod);
}

__global__ void k_norm_final(LaunchInfo li, double* out) {
  for (int b = threadIdx.x; b < li.ninst; b += blockDim.x) out[b] = norm_from_parts(li.insts[b]);
}

// ------------------------------------------------------------------ per-mode kernel
size_t smem_mode(const Inst& I, int mpc) {
  // [cheb (FP64 form only)] + rco + per mode: [solver table (sweep solve only)],
  // Fr/U0/Out ([3][2][L2] each), chain scratch [4][6][Mh], 1/k^2
  const int N = I.N, Mh = N / 2 + 1, H = Mh, L2 = 2 * Mh;
  const TabLayout TL(N);
  size_t d = (I.mixed ? 0 : 6 * (size_t)H * H) + 10 * (size_t)Mh;
  d += (size_t)mpc * ((I.dense[0] ? 0 : TL.per_mode()) + 18 * (size_t)L2 + 24 * (size_t)Mh + 1);
  return d * sizeof(double);
}

// a0 += sum_j col[j stride] x0[j] and a1 += sum_j col[j stride] x1[j] over j < n, each chain in
// index order; the operator column is read through the read-only cache eight elements ahead of
// the FMAs, so that a thread keeps eight loads in flight (the dense operators of a large grid
// come from HBM, and one outstanding load per thread left the solve waiting on latency).
__device__ __forceinline__ void dot2_ldg(const double* col, int stride, const double* x0, const double* x1, int n,
                                         double& a0, double& a1) {
  int j = 0;
  for (; j + 8 <= n; j += 8) {
    double d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) d[k] = __ldg(col + (j + k) * stride);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      a0 = fma(d[k], x0[j + k], a0);
      a1 = fma(d[k], x1[j + k], a1);
    }
  }
  for (; j < n; ++j) {
    const double d = __ldg(col + j * stride);
    a0 = fma(d, x0[j], a0);
    a1 = fma(d, x1[j], a1);
  }
}

__global__ void __launch_bounds__(320) k_mode(LaunchInfo li, int op, int sig, int mpc_arg, int step_index) {
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

  // descent: J = ||r1|| from the plane sums of k_prod<N>, its history entry and the
  // convergence decision; step_index < 0: the product kernel has taken them already (the
  // instance's mask then holds this step's J < tol)
  if (op == MODE_PSI_UPDATE) {
    if (!inst_active(I)) return;
    if (step_index >= 0) {
      const double J = norm_from_parts(I);
      if (local == 0 && threadIdx.x == 0 && I.hist) I.hist[(size_t)step_index * I.hist_stride] = J;
      if (I.tol > 0.0 && J < I.tol) {
        if (local == 0 && threadIdx.x == 0 && I.active) *I.active = 0;
        return;
      }
    }
  } else if (op != MODE_SOLVE && op != MODE_SYNTH_ONLY && !inst_active(I)) {
    return;
  }

  const bool need_cheb = !I.mixed, need_tabs = !I.dense[0];
  double* cheb = smd;
  double* rco = cheb + (need_cheb ? CL.total() : 0);
  double* tabs = rco + RL.total();
  const int PM = TL.per_mode();
  double* Fr = tabs + (need_tabs ? (size_t)mpc * PM : 0);  // [mpc][3][2][L2]
  double* U0 = Fr + (size_t)mpc * 6 * L2;        // [mpc][3][2][L2]
  double* Out = U0 + (size_t)mpc * 6 * L2;       // [mpc][3][2][L2] (also y-values input)
  double* Ch = Out + (size_t)mpc * 6 * L2;       // [mpc][4][6][Mh]
  double* IK2 = Ch + (size_t)mpc * 24 * Mh;      // [mpc] 1/k^2 (0 for the mean mode)

  // 1/k^2 once per mode: an FP64 division costs the pipe per lane-instruction
  for (int t = threadIdx.x; t < nmod; t += blockDim.x) {
    const int m = m0 + t, ix = m / Mz, p = m - ix * Mz;
    const double kx = I.kx[ix], kz = I.kz[p];
    const double k2 = kx * kx + kz * kz;
    IK2[t] = m == 0 ? 0.0 : 1.0 / k2;
  }

  if (need_cheb)
    for (int t = threadIdx.x; t < CL.total(); t += blockDim.x) cheb[t] = I.cheb[t];
  for (int t = threadIdx.x; t < RL.total(); t += blockDim.x) rco[t] = I.rco[t];
  const double* tabg = solve ? I.tab[sig] : nullptr;
  if (solve && need_tabs)
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
  if (!I.mixed && (op == MODE_PHI || op == MODE_PSI_UPDATE || op == MODE_PSI_GRAD)) {
    for (int t = threadIdx.x; t < nmod * 3 * ny; t += blockDim.x) {
      const int mm = t % nmod, cj = t / nmod, j = cj % ny, c = cj / ny;
      const double2 v = I.xz[((size_t)c * ny + j) * nm + m0 + mm];
      double* dst = Out + ((size_t)mm * 3 + c) * 2 * L2 + j;
      dst[0] = v.x;
      dst[L2] = v.y;
    }
  }
  __syncthreads();

  const double inv_step = sig == 0 ? I.inv_dt : I.inv_dtau_hat;  // 1 / the step size
  const double inv_nu = I.inv_nu;
  const int half = N / 2;
  if (solve) {
    if (I.mixed && op != MODE_SOLVE) {
      // mixed form: Chebyshev coefficients of the products come from the tensor-core kernel
      for (int t = threadIdx.x; t < nmod * 3 * ny; t += blockDim.x) {
        const int mm = t % nmod, cn = t / nmod, n = cn % ny, c = cn / ny;
        const float2 v = I.xzc[((size_t)c * ny + n) * nm + m0 + mm];
        const int pos = (n & 1) * Mh + (n >> 1);
        const double* u0 = U0 + ((size_t)mm * 3 + c) * 2 * L2;
        double* fr = Fr + ((size_t)mm * 3 + c) * 2 * L2;
        fr[pos] = fma(u0[pos], inv_step, (double)v.x) * inv_nu;
        fr[L2 + pos] = fma(u0[L2 + pos], inv_step, (double)v.y) * inv_nu;
      }
    } else if (op != MODE_SOLVE) {
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
        if (i >= McP || m == 0) continue;  // m == 0: the mean mode
        const double* fr = Fr + (size_t)mm * 6 * L2;
        const double fu = fr[(0 * 2 + (1 - rho)) * L2 + pP * Mh + i];
        const double fw = fr[(2 * 2 + (1 - rho)) * L2 + pP * Mh + i];
        const double sgn = rho == 0 ? -1.0 : 1.0;
        double* sc = Ch + ((size_t)mm * 4 + g * 2 + rho) * 6 * Mh;
        sc[i] = sgn * fma(kx, fu, kz * fw);
        sc[Mh + i] = sgn * fma(kz, fu, -kx * fw);
      }
      __syncthreads();
      // Two task lists, so that a warp's lanes carry chains of one length: list A, one v row
      // (Av f_v + Ag g: McV + McP terms) per task; list B, two eta rows (Eh h: McP terms
      // each) per task.  A task runs both parts' chains (real and imaginary right-hand
      // sides), which share each operator load; every chain keeps the index order of the
      // other kernel organisations.  Mean mode: list A holds the u rows, list B the w rows.
      // Every task is two operator segments run by the same code (a v row continues its chain
      // into the second segment; an eta pair stores the first row and starts the second), so
      // the warp that holds the last tasks of list A and the first of list B runs one pass.
      const int HB = (Mh + 1) / 2, nA = nmod * 2 * Mh, nB = nmod * 2 * HB;
      const int S1 = 6 * Mh;  // the imaginary part's chain scratch follows the real part's
      for (int t = threadIdx.x; t < nA + nB; t += blockDim.x) {
        const bool isA = t < nA;
        const int tt = isA ? t : t - nA, per = isA ? Mh : HB;
        const int r = tt % per, q = tt / per, g = q & 1, mm = q >> 1;
        const int pv = g, pP = 1 - g, McV = (N - pv) / 2 + 1, McP = (N - pP) / 2 + 1;
        const int m = m0 + mm;
        const double* D = dn + (size_t)m * DL.per_mode();
        const double* fr = Fr + (size_t)mm * 6 * L2;
        double* s0 = Ch + ((size_t)mm * 4 + g * 2) * 6 * Mh;  // real part's chain scratch
        const double *c1 = D, *c2 = D;
        const double *x10 = s0, *x11 = s0, *x20 = s0, *x21 = s0;  // segment inputs, real / imaginary
        int n1 = 0, n2 = 0;
        double *o1 = nullptr, *o2 = nullptr;  // real-part outputs (imaginary at + S1)
        if (m == 0) {  // the mean mode: Eh of class g applied to f_u (list A) or f_w (list B)
          const int Mc = (N - g) / 2 + 1;
          const double* f0 = fr + (isA ? 0 : 4) * L2 + g * Mh;
          x10 = x20 = f0;
          x11 = x21 = f0 + L2;
          if (r < Mc) { c1 = D + DL.at(g, DL.kEh, r, 0); n1 = Mc; o1 = s0 + (isA ? 0 : Mh) + r; }
          if (!isA && r + HB < Mc) { c2 = D + DL.at(g, DL.kEh, r + HB, 0); n2 = Mc; o2 = s0 + Mh + r + HB; }
        } else if (isA) {  // v = Av f_v + Ag g, one chain over both segments
          if (r < McV) {
            c1 = D + DL.at(g, DL.kAv, r, 0);
            x10 = fr + 2 * L2 + pv * Mh;
            x11 = x10 + L2;
            n1 = McV;
            c2 = D + DL.at(g, DL.kAg, r, 0);
            x20 = s0;
            x21 = s0 + S1;
            n2 = McP;
            o2 = s0 + 2 * Mh + r;
          }
        } else {  // eta = Eh h, rows r and r + HB
          x10 = x20 = s0 + Mh;
          x11 = x21 = s0 + Mh + S1;
          if (r < McP) { c1 = D + DL.at(g, DL.kEh, r, 0); n1 = McP; o1 = s0 + 4 * Mh + r; }
          if (r + HB < McP) { c2 = D + DL.at(g, DL.kEh, r + HB, 0); n2 = McP; o2 = s0 + 4 * Mh + r + HB; }
        }
        double a0 = 0.0, a1 = 0.0;
        dot2_ldg(c1, Mh, x10, x11, n1, a0, a1);
        if (o1) {
          o1[0] = a0;
          o1[S1] = a1;
          a0 = a1 = 0.0;
        }
        dot2_ldg(c2, Mh, x20, x21, n2, a0, a1);
        if (o2) {
          o2[0] = a0;
          o2[S1] = a1;
        }
      }
      __syncthreads();
      // xi = -dv/dy (class 1-g) of every (mode, group, part) chain but the mean mode's
      for (int t = threadIdx.x; t < nmod * 4; t += blockDim.x) {
        const int mm = t >> 2, g = (t >> 1) & 1, rho = t & 1;
        const int m = m0 + mm, ix = m / Mz, p = m - ix * Mz;
        if (m == 0) continue;
        double* sc = Ch + ((size_t)mm * 4 + g * 2 + rho) * 6 * Mh;
        xi_from_v(N, g, sc + 2 * Mh, 1, sc + 3 * Mh, 1, rco + RL.off(g, 4));
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
      const double* chv_re = Ch + ((size_t)mm * 4 + par * 2 + 0) * 6 * Mh;
      const double* chv_im = Ch + ((size_t)mm * 4 + par * 2 + 1) * 6 * Mh;
      if (m == 0) {  // the mean mode
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
      const double ik2 = IK2[mm];
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
  if (op == MODE_PHI) { gout = I.rhat; scale = I.inv_dt; slot = 1; }
  if (op == MODE_PSI_UPDATE) { slot = 0; }
  if (op == MODE_PSI_GRAD) { gout = I.fhat; }
  if (op == MODE_SOLVE) { gout = I.fhat; }
  if (op == MODE_SYNTH_ONLY) { slot = sig; }
  if (I.mixed) slot = -1;  // the tensor-core kernel synthesises from the FP64 state
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
