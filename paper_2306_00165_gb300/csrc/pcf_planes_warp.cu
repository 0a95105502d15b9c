// Plane kernels of the FP32 (mixed-precision) form with the x and z transforms in warp
// registers: the synthesis of the 11 physical fields of a y-plane and the products M(u),
// N(q) with their forward transforms and 2/3 truncation (paper §4, steps 1 and 3).
//
// In FP32 the plane kernels move many bytes per flop: a 128 x 128 plane of one field is
// 64 KB, while its transforms are ~0.5 MFLOP.  Their bound is HBM bandwidth, and the
// shared-memory Stockham kernels, whose passes are separated by CTA barriers and which
// hold two plane buffers per CTA, leave it far from reached: few warps per SM, each pass
// waiting for the slowest warp.  Here one warp transforms one row of length L = 32 E
// (E = 1..4 complex values per lane) with no barrier: an E-point DFT in registers, a
// twiddle, and a 32-point DFT across the lanes (five radix-2 stages exchanged by xor
// shuffles, then the bit reversal as one shuffle).  Only the x-stage result of a plane
// (the retained z modes, Mz rows) is held in shared memory between the x and z stages.
//
// Index maps (L = 32 E, lane l, register e or s):
//   decimation in frequency: in x[l + 32 e]  ->  out X[E l + s]  (cyclic in, blocked out)
//   decimation in time:      in x[E l + r]  ->  out X[l + 32 s]  (blocked in, cyclic out)
// so every global access is to E consecutive elements per lane (vector loads and stores)
// and every shared-memory column walk has an odd stride.
//
// The 32-point stage is branch-free: the lower lane of a pair computes p + v and the upper
// lane (p - v) w, both as (p + sg v) w' with sg = +-1 and w' = 1 on the lower lane (a
// multiply by exactly 1), so that a warp issues each instruction once for all its lanes.
#include "pcf_kernels.cuh"
#include "pcf_plane_common.cuh"

namespace pcf {

constexpr int kWarpPlaneThreads = 256;

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float2 cshfl(float2 v, int s) {
  return make_float2(__shfl_sync(kFull, v.x, s), __shfl_sync(kFull, v.y, s));
}
__device__ __forceinline__ float2 cshflx(float2 v, int m) {
  return make_float2(__shfl_xor_sync(kFull, v.x, m), __shfl_xor_sync(kFull, v.y, m));
}
__device__ __forceinline__ double2 cshfl(double2 v, int s) {
  return make_double2(__shfl_sync(kFull, v.x, s), __shfl_sync(kFull, v.y, s));
}
__device__ __forceinline__ double2 cshflx(double2 v, int m) {
  return make_double2(__shfl_xor_sync(kFull, v.x, m), __shfl_xor_sync(kFull, v.y, m));
}

// Twiddles of the 32-point stage of lane `lane`, forward sign: stage s (pair distance
// h = 16 >> s) multiplies the upper lane's difference by W_32^{(lane mod h) 16/h}; tw is a
// length-32E table of W_L^k, so W_32^m = tw[m E].  Stage 4 (h = 1) has no twiddle.
template <class C>
__device__ __forceinline__ void net_twiddles(C* w, const C* tw, int E, int lane) {
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int h = 16 >> s;
    w[s] = tw[((lane & (h - 1)) * (16 / h)) * E];
  }
}

// 32-point DFT across the lanes, one complex value per lane, natural order in and out.
template <class C>
__device__ __forceinline__ C dft32(C v, const C* w, bool inv, int lane) {
  using R = decltype(v.x);
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int h = 16 >> s;
    const C p = cshflx(v, h);
    const bool up = (lane & h) != 0;
    const R sg = up ? R(-1) : R(1);
    C d;
    d.x = fma(sg, v.x, p.x);
    d.y = fma(sg, v.y, p.y);
    if (s < 4) {
      C t = w[s];
      if (inv) t.y = -t.y;
      C one;
      one.x = R(1);
      one.y = R(0);
      d = cmul(d, up ? t : one);
    }
    v = d;
  }
  return cshfl(v, (int)(__brev((unsigned)lane) >> 27));
}

template <class C>
__device__ __forceinline__ void dft_small(C* x, int E, bool inv) {
  if (E == 2) butterfly<2, C>(x, inv);
  else if (E == 3) butterfly<3, C>(x, inv);
  else if (E == 4) butterfly<4, C>(x, inv);
}

// Decimation in frequency: x[e] = element lane + 32 e on entry, x[s] = X[E lane + s] on return.
template <class C>
__device__ __forceinline__ void fft_dif(C* x, int E, const C* tw, const C* w32, bool inv, int lane) {
  dft_small(x, E, inv);
#pragma unroll
  for (int s = 1; s < 4; ++s)
    if (s < E) {
      C t = tw[lane * s];
      if (inv) t.y = -t.y;
      x[s] = cmul(x[s], t);
    }
#pragma unroll
  for (int s = 0; s < 4; ++s)
    if (s < E) x[s] = dft32(x[s], w32, inv, lane);
}

// Decimation in time: x[r] = element E lane + r on entry, x[s] = X[lane + 32 s] on return.
template <class C>
__device__ __forceinline__ void fft_dit(C* x, int E, const C* tw, const C* w32, bool inv, int lane) {
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (r < E) x[r] = dft32(x[r], w32, inv, lane);
#pragma unroll
  for (int r = 1; r < 4; ++r)
    if (r < E) {
      C t = tw[lane * r];
      if (inv) t.y = -t.y;
      x[r] = cmul(x[r], t);
    }
  dft_small(x, E, inv);
}

// h[k] for a run-time k < 4 by selects (a dynamic register index would move h to local memory)
template <class C>
__device__ __forceinline__ C pick(const C* h, int k) {
  return k == 0 ? h[0] : (k == 1 ? h[1] : (k == 2 ? h[2] : h[3]));
}

// E consecutive reals starting at p (vector loads for E = 2, 4; p is E-aligned)
__device__ __forceinline__ void load_seg(const float* p, int E, float* v) {
  if (E == 4) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else if (E == 2) {
    const float2 a = *reinterpret_cast<const float2*>(p);
    v[0] = a.x; v[1] = a.y;
  } else {
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (q < E) v[q] = p[q];
  }
}
__device__ __forceinline__ void store_seg(float* p, int E, const float* v) {
  if (E == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else if (E == 2) *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  else {
#pragma unroll
    for (int q = 0; q < 3; ++q)
      if (q < E) p[q] = v[q];
  }
}

// Two adjacent complex values as one 16-byte shared-memory access (float2 pairs; p is
// 16-byte aligned), else two accesses.
__device__ __forceinline__ void st_pair(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void ld_pair(const float2* p, float2& a, float2& b) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
template <class C>
__device__ __forceinline__ void st_pair(C* p, C a, C b) {
  p[0] = a;
  p[1] = b;
}
template <class C>
__device__ __forceinline__ void ld_pair(const C* p, C& a, C& b) {
  a = p[0];
  b = p[1];
}

// Shared-memory plan: staged spectral values S[Mx][SP] (SP = Mz rounded up to odd), x-stage
// rows G[Mz][LG] (LG = nx + 2: 16-byte aligned rows and conflict-free 16-byte column
// walks), then the twiddles of x and z and a reduction scratch.
struct WarpPlan {
  int SP, LG;
  size_t S, G, twx, twz, red, total;  // offsets in complex values, total in bytes
};
__host__ __device__ inline WarpPlan warp_plan(const Inst& I, int elem) {
  WarpPlan w;
  w.SP = I.Mz | 1;
  w.LG = I.nx + 2;
  w.S = 0;
  w.G = (w.S + (size_t)I.Mx * w.SP + 1) & ~(size_t)1;  // even: 16-byte aligned pairs of float2
  w.twx = w.G + (size_t)I.Mz * w.LG;
  w.twz = w.twx + I.nx;
  w.red = w.twz + I.nz;
  w.total = w.red * elem + 8 * 32;
  return w;
}

template <class T>
__device__ __forceinline__ void load_twiddles_w(const Inst& I, typename Cx<T>::c* twx, typename Cx<T>::c* twz) {
  const typename Sto<T>::c* sx = twx_of<T>(I);
  const typename Sto<T>::c* sz = twz_of<T>(I);
  for (int t = threadIdx.x; t < I.nx; t += blockDim.x) twx[t] = load_c<T>(sx[t]);
  for (int t = threadIdx.x; t < I.nz; t += blockDim.x) twz[t] = load_c<T>(sz[t]);
}

__constant__ int c_src_w[kFieldsSynth] = {0, 1, 2, 0, 3, 0, 1, 1, 2, 4, 2};
__constant__ int c_fac_w[kFieldsSynth] = {0, 0, 0, 1, 0, 2, 1, 2, 1, 0, 2};

}  // namespace

bool plane_warp_ok(const Inst& I) {
  const auto ok = [](int n) { return n == 32 || n == 64 || n == 96 || n == 128; };
  return ok(I.nx) && ok(I.nz);
}
size_t smem_plane_warp(const Inst& I, int elem) { return warp_plan(I, elem).total; }

// CTA = (instance, y-plane j, field f), 8 warps.  Field f of slot: 0 u, 1 v, 2 w, 3 u_x,
// 4 u_y, 5 u_z, 6 v_x, 7 v_z, 8 w_x, 9 w_y, 10 w_z, made from the y-values V0 V1 V2 W0 W2
// (times i kx or i kz for the x and z derivatives).
template <class T>
__global__ void __launch_bounds__(kWarpPlaneThreads, 3) k_xzsynth_w(LaunchInfo li, int slot, int nfields) {
  using C = typename Cx<T>::c;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  if (!inst_active(I)) return;
  const int f = local % nfields, j = local / nfields;
  const int nx = I.nx, nz = I.nz, Mx = I.Mx, Mz = I.Mz, Kx = I.Kx, Kz = I.Kz;
  const WarpPlan wp = warp_plan(I, sizeof(C));
  const int SP = wp.SP, LG = wp.LG, EX = nx >> 5, EZ = nz >> 5;
  C* S = sm + wp.S;
  C* G = sm + wp.G;
  C* twx = sm + wp.twx;
  C* twz = sm + wp.twz;
  load_twiddles_w<T>(I, twx, twz);
  const typename Sto<T>::c* src =
      yv_of<T>(I) + (((size_t)slot * kFieldsY + c_src_w[f]) * I.ny + j) * (size_t)I.nmodes;
  const int fac = c_fac_w[f];
  for (int t = threadIdx.x; t < I.nmodes; t += blockDim.x) {
    const int i = t / Mz, p = t - i * Mz;
    C s = load_c<T>(src[t]);
    if (fac == 1) { const T k = (T)I.kx[i]; s = Cx<T>::mk(-k * s.y, k * s.x); }
    else if (fac == 2) { const T k = (T)I.kz[p]; s = Cx<T>::mk(-k * s.y, k * s.x); }
    S[i * SP + p] = s;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  C w32[4];
  net_twiddles(w32, twx, EX, lane);
  // x stage: row p (retained z mode) over the x bins, inverse transform, bins |m| > Kx zero
  for (int p = warp; p < Mz; p += nw) {
    C x[4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (e < EX) {
        const int bin = lane + 32 * e;
        C v = Cx<T>::mk(0, 0);
        if (bin <= Kx) v = S[bin * SP + p];
        else if (bin >= nx - Kx) v = S[(bin - nx + Mx) * SP + p];
        x[e] = v;
      }
    fft_dif(x, EX, twx, w32, true, lane);
    C* g = G + (size_t)p * LG + EX * lane;
    if (EX == 4) {
      st_pair(g, x[0], x[1]);
      st_pair(g + 2, x[2], x[3]);
    } else if (EX == 2) {
      st_pair(g, x[0], x[1]);
    } else {
#pragma unroll
      for (int s = 0; s < 3; ++s)
        if (s < EX) g[s] = x[s];
    }
  }
  __syncthreads();
  // z stage: row pair (x1, x2) -> one complex row h_z = G_z[x1] + i G_z[x2] with
  // G_{-p} = conj(G_p) (p = 0: real parts only; |p| > Kz: zero); its inverse transform holds
  // row x1 in the real part and row x2 in the imaginary part.
  T* out = phys_of<T>(I) + (((size_t)slot * kFieldsSynth + f) * I.ny + j) * (size_t)nx * nz;
  for (int r = warp; r < nx / 2; r += nw) {
    const int x1 = 2 * r;
    C h[4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (e < EZ) {
        const int z = lane + 32 * e;
        const bool lo = z <= Kz, hi = z >= nz - Kz;
        const int p = lo ? z : nz - z;
        C g1 = Cx<T>::mk(0, 0), g2 = g1;
        if (lo || hi) {
          ld_pair(G + (size_t)p * LG + x1, g1, g2);
        }
        if (z == 0) g1.y = g2.y = T(0.0);
        const T sg = lo ? T(1.0) : T(-1.0);
        h[e] = Cx<T>::mk(fma(-sg, g2.y, g1.x), fma(sg, g1.y, g2.x));
      }
    fft_dif(h, EZ, twz, w32, true, lane);
    T re[4], im[4];
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (s < EZ) {
        re[s] = h[s].x;
        im[s] = h[s].y;
      }
    store_seg(out + (size_t)x1 * nz + EZ * lane, EZ, re);
    store_seg(out + (size_t)(x1 + 1) * nz + EZ * lane, EZ, im);
  }
}

namespace {

// Values at the E consecutive points z0.. of row x of field f (plane j, slot s); field 11
// stands for v_y = -u_x - w_z (incompressibility).
template <class T, int F>
__device__ __forceinline__ void seg(const T* plane, int fstride, int off, int E, T* v) {
  if (F < kFieldsSynth) {
    load_seg(plane + F * fstride + off, E, v);
  } else {
    T a[4], c[4];
    load_seg(plane + 3 * fstride + off, E, a);
    load_seg(plane + 10 * fstride + off, E, c);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = -(a[q] + c[q]);
  }
}

// Fields of d_d u_c (d = 0 x, 1 y, 2 z): 3 u_x 4 u_y 5 u_z, 6 v_x 11 v_y 7 v_z, 8 w_x 9 w_y 10 w_z
template <int CC, int D>
struct GradField {
  static constexpr int f = CC == 0 ? 3 + D : (CC == 2 ? 8 + D : (D == 0 ? 6 : (D == 2 ? 7 : 11)));
};

// Product component CC at the E points z0.. of row x: M(u) (ADJ false) or N(q) (ADJ true)
// in the convective forms of §4, with the association order of product_pair (the last
// term first), streamed so that only two fields are live at a time; ADJ also sums q_CC^2.
template <class T, bool ADJ, int CC>
__device__ __forceinline__ void product_seg(const T* U, const T* Q, int fstride, int off, int E, T Ub, T dUb, T Vb,
                                            T* m, double* sq) {
  T a[4], g[4], acc[4];
  if (!ADJ) {
    seg<T, 2>(U, fstride, off, E, a);
    seg<T, GradField<CC, 2>::f>(U, fstride, off, E, g);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = a[q] * g[q];
    T vv[4];
    seg<T, 1>(U, fstride, off, E, vv);
    seg<T, GradField<CC, 1>::f>(U, fstride, off, E, g);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fma(vv[q] + Vb, g[q], acc[q]);  // v of u_b + u
    seg<T, 0>(U, fstride, off, E, a);
    seg<T, GradField<CC, 0>::f>(U, fstride, off, E, g);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      T val = -fma(Ub + a[q], g[q], acc[q]);
      if (CC == 0) val -= dUb * vv[q];
      m[q] = val;
    }
  } else {
    // adv = (U + u) d_x q_c + v d_y q_c + w d_z q_c
    seg<T, 2>(U, fstride, off, E, a);
    seg<T, GradField<CC, 2>::f>(Q, fstride, off, E, g);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = a[q] * g[q];
    seg<T, 1>(U, fstride, off, E, a);
    seg<T, GradField<CC, 1>::f>(Q, fstride, off, E, g);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = fma(a[q] + Vb, g[q], acc[q]);
    seg<T, 0>(U, fstride, off, E, a);
    seg<T, GradField<CC, 0>::f>(Q, fstride, off, E, g);
    T adv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) adv[q] = fma(Ub + a[q], g[q], acc[q]);
    // tr = q_0 d_c u_0 + q_1 d_c u_1 + q_2 d_c u_2
    seg<T, 2>(Q, fstride, off, E, a);
    seg<T, GradField<2, CC>::f>(U, fstride, off, E, g);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      acc[q] = a[q] * g[q];
      if (CC == 2 && q < E) *sq = fma((double)a[q], (double)a[q], *sq);
    }
    seg<T, 1>(Q, fstride, off, E, a);
    seg<T, GradField<1, CC>::f>(U, fstride, off, E, g);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      acc[q] = fma(a[q], g[q], acc[q]);
      if (CC == 1 && q < E) *sq = fma((double)a[q], (double)a[q], *sq);
    }
    seg<T, 0>(Q, fstride, off, E, a);
    seg<T, GradField<0, CC>::f>(U, fstride, off, E, g);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (CC == 0 && q < E) *sq = fma((double)a[q], (double)a[q], *sq);
      T val = adv[q] - fma(a[q], g[q], acc[q]);
      if (CC == 1) val -= dUb * a[q];
      m[q] = val;
    }
  }
}

// z stage of one row pair: products at rows x1, x1 + 1 packed as one complex row, forward
// DIT transform, two-for-one unpacking of the retained z modes into X[p][x1], X[p][x1 + 1].
template <class T, bool ADJ, int CC>
__device__ __forceinline__ void prod_row_pair(const Inst& I, const T* U, const T* Q, int fstride, int x1, T Ub,
                                              T dUb, T Vb, int EZ, const typename Cx<T>::c* twz,
                                              const typename Cx<T>::c* w32, typename Cx<T>::c* X, int LG, int lane,
                                              double* sq) {
  using C = typename Cx<T>::c;
  const int nz = I.nz, Kz = I.Kz, z0 = EZ * lane;
  // the two rows one after the other (not interleaved), so that only one row's fields are
  // live in registers at a time
  C h[4];
#pragma unroll 1
  for (int row = 0; row < 2; ++row) {
    T m[4];
    product_seg<T, ADJ, CC>(U, Q, fstride, (x1 + row) * nz + z0, EZ, Ub, dUb, Vb, m, sq);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (row == 0) h[q].x = m[q];
      else h[q].y = m[q];
    }
  }
  fft_dit(h, EZ, twz, w32, false, lane);
  // h[s] = H[lane + 32 s]; its partner H[(nz - p) mod nz] sits in lane (32 - lane) mod 32,
  // register EZ - 1 - s, except on lane 0, which holds it itself (H[0], or H[32 (EZ - s)])
  const T half = (T)0.5;
#pragma unroll
  for (int s = 0; s < 4; ++s)
    if (s < EZ) {
      C hm = cshfl(pick(h, EZ - 1 - s), (32 - lane) & 31);
      if (lane == 0) hm = pick(h, s == 0 ? 0 : EZ - s);
      const int p = lane + 32 * s;
      if (p <= Kz) {
        const C hp = h[s];
        st_pair(X + (size_t)p * LG + x1, Cx<T>::mk(half * (hp.x + hm.x), half * (hp.y - hm.y)),
                Cx<T>::mk(half * (hp.y + hm.y), -half * (hp.x - hm.x)));
      }
    }
}

}  // namespace

// CTA = (instance, plane j, component c), 8 warps: product component c on the plane (M(u),
// or N(q) with W = u_b + u), forward transforms in z then x, 2/3 truncation; the adjoint
// products also sum q_c^2 over the plane (FP64) and, with step_index >= 0, the CTA that
// finishes last for an instance computes J as the Stockham kernel does.
template <class T, bool ADJ>
__global__ void __launch_bounds__(kWarpPlaneThreads, 2) k_prod_w(LaunchInfo li, int step_index) {
  using C = typename Cx<T>::c;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* sm = reinterpret_cast<C*>(smraw);
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  if (!inst_active(I)) return;
  const int c = local % 3, j = local / 3;
  const int nx = I.nx, Mx = I.Mx, Mz = I.Mz, Kx = I.Kx;
  const WarpPlan wp = warp_plan(I, sizeof(C));
  const int SP = wp.SP, LG = wp.LG, EX = nx >> 5, EZ = I.nz >> 5;
  C* O = sm + wp.S;  // truncated output [Mx][SP]
  C* X = sm + wp.G;  // z-transformed rows [Mz][LG]
  C* twx = sm + wp.twx;
  C* twz = sm + wp.twz;
  double* red = reinterpret_cast<double*>(sm + wp.red);
  load_twiddles_w<T>(I, twx, twz);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  C w32[4];
  net_twiddles(w32, twz, EZ, lane);
  const T Ub = (T)I.ubase[j], dUb = (T)I.ubase[I.ny + j], Vb = (T)I.ubase[2 * I.ny + j];
  double sq = 0.0;
  const int fstride = I.ny * nx * I.nz;  // between the fields of a slot
  const T* U = phys_of<T>(I) + (size_t)j * nx * I.nz;
  const T* Q = ADJ ? U + (size_t)kFieldsSynth * fstride : nullptr;
  for (int r = warp; r < nx / 2; r += nw) {
    if (c == 0) prod_row_pair<T, ADJ, 0>(I, U, Q, fstride, 2 * r, Ub, dUb, Vb, EZ, twz, w32, X, LG, lane, &sq);
    else if (c == 1) prod_row_pair<T, ADJ, 1>(I, U, Q, fstride, 2 * r, Ub, dUb, Vb, EZ, twz, w32, X, LG, lane, &sq);
    else prod_row_pair<T, ADJ, 2>(I, U, Q, fstride, 2 * r, Ub, dUb, Vb, EZ, twz, w32, X, LG, lane, &sq);
  }
  if (ADJ) {
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(kFull, sq, o);
    if (lane == 0) red[warp] = sq;
  }
  __syncthreads();
  if (ADJ && threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    I.normpart[(size_t)c * I.ny + j] = s;
  }
  // x stage: retained z mode p over x, forward DIF, the retained bins scaled into O[i][p]
  const T sc = (T)I.inv_nxnz;
  for (int p = warp; p < Mz; p += nw) {
    C x[4];
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (e < EX) x[e] = X[(size_t)p * LG + lane + 32 * e];
    fft_dif(x, EX, twx, w32, false, lane);
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (s < EX) {
        const int bin = EX * lane + s;
        int i = -1;
        if (bin <= Kx) i = bin;
        else if (bin >= nx - Kx) i = bin - nx + Mx;
        if (i >= 0) O[i * SP + p] = Cx<T>::mk(x[s].x * sc, x[s].y * sc);
      }
  }
  __syncthreads();
  typename Sto<T>::c* dst = xz_of<T>(I) + ((size_t)c * I.ny + j) * I.nmodes;
  for (int t = threadIdx.x; t < I.nmodes; t += blockDim.x) {
    const int i = t / Mz, p = t - i * Mz;
    dst[t] = store_c<T>(O[i * SP + p]);
  }
  if (ADJ && step_index >= 0) {
    // J = ||r1|| once all 3 ny plane sums of the instance are written (the chain of
    // norm_from_parts, as in the Stockham kernel)
    __shared__ int last;
    if (threadIdx.x == 0) {
      __threadfence();
      last = atomicAdd(I.jcount, 1) == 3 * I.ny - 1;
    }
    __syncthreads();
    if (last) {
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

void launch_xzsynth_warp(int ctas, size_t smem, cudaStream_t s, LaunchInfo li, int slot, int nf) {
  k_xzsynth_w<float><<<ctas, kWarpPlaneThreads, smem, s>>>(li, slot, nf);
}
void launch_prod_warp(bool adj, int ctas, size_t smem, cudaStream_t s, LaunchInfo li, int step_index) {
  if (adj) k_prod_w<float, true><<<ctas, kWarpPlaneThreads, smem, s>>>(li, step_index);
  else k_prod_w<float, false><<<ctas, kWarpPlaneThreads, smem, s>>>(li, -1);
}
cudaError_t set_plane_warp_smem(size_t synth, size_t prod) {
  cudaError_t e;
  if ((e = raise_smem_limit((const void*)k_xzsynth_w<float>, synth))) return e;
  if ((e = raise_smem_limit((const void*)k_prod_w<float, false>, prod))) return e;
  return raise_smem_limit((const void*)k_prod_w<float, true>, prod);
}

}  // namespace pcf
