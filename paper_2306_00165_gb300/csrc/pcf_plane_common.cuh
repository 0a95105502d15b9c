// Complex arithmetic in the three plane arithmetics (FP64, FP32, float-float), typed views
// of an instance's plane buffers and twiddle tables, and the small DFT butterflies shared by
// the shared-memory Stockham plane kernels (pcf_kernels.cu) and the warp-register plane
// kernels (pcf_planes_warp.cu).
#pragma once
#include "pcf_ff.cuh"
#include "pcf_kernels.cuh"

namespace pcf {

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// x-storage index i (m = i for i <= Kx, m = i - Mx otherwise) -> FFT bin
__device__ __forceinline__ int xbin(int i, int Kx, int Mx, int nx) { return i <= Kx ? i : nx - (Mx - i); }

// ------------------------------------------------------------------ complex helpers (FP64 / FP32)
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

__device__ __forceinline__ ff2 cmul(ff2 a, ff2 b) { return ff2{fma(a.x, b.x, -(a.y * b.y)), fma(a.x, b.y, a.y * b.x)}; }
__device__ __forceinline__ ff2 cadd(ff2 a, ff2 b) { return ff2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ ff2 csub(ff2 a, ff2 b) { return ff2{a.x - b.x, a.y - b.y}; }

template <class T> struct Cx;
template <> struct Cx<double> {
  using c = double2;
  static __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
};
template <> struct Cx<float> {
  using c = float2;
  static __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
};
template <> struct Cx<ff> {
  using c = ff2;
  static __device__ __forceinline__ ff2 mk(ff a, ff b) { return ff2{a, b}; }
};

// Element type of the y-values, the transformed products and the twiddle tables in memory:
// the compute type's complex, except in the float-float form, whose plane kernels read and
// write the FP64 arrays of the y transforms and convert at the boundary.
template <class T> struct Sto { using c = typename Cx<T>::c; };
template <> struct Sto<ff> { using c = double2; };
template <class T> __device__ __forceinline__ typename Cx<T>::c load_c(const typename Sto<T>::c& v) { return v; }
template <> __device__ __forceinline__ ff2 load_c<ff>(const double2& v) { return ff2{ff(v.x), ff(v.y)}; }
template <class T> __device__ __forceinline__ typename Sto<T>::c store_c(const typename Cx<T>::c& v) { return v; }
template <> __device__ __forceinline__ double2 store_c<ff>(const ff2& v) {
  return make_double2(to_double(v.x), to_double(v.y));
}

// Accumulator of the plane sums of q^2 (FP64; float-float in the float-float form)
template <class T> struct Acc { using type = double; };
template <> struct Acc<ff> { using type = ff; };
__device__ __forceinline__ void acc_sq(double* s, double q) { *s = fma(q, q, *s); }
__device__ __forceinline__ void acc_sq(double* s, float q) { *s = fma((double)q, (double)q, *s); }
__device__ __forceinline__ void acc_sq(ff* s, ff q) { *s = fma(q, q, *s); }
__device__ __forceinline__ double acc_value(double s) { return s; }
__device__ __forceinline__ double acc_value(ff s) { return to_double(s); }

// typed views of an instance's plane buffers and twiddles
template <class T> __device__ __forceinline__ T* phys_of(const Inst& I);
template <> __device__ __forceinline__ double* phys_of<double>(const Inst& I) { return I.phys; }
template <> __device__ __forceinline__ float* phys_of<float>(const Inst& I) { return I.physf; }
template <> __device__ __forceinline__ ff* phys_of<ff>(const Inst& I) { return reinterpret_cast<ff*>(I.phys); }
template <class T> __device__ __forceinline__ const typename Sto<T>::c* yv_of(const Inst& I);
template <> __device__ __forceinline__ const double2* yv_of<double>(const Inst& I) { return I.yv; }
template <> __device__ __forceinline__ const float2* yv_of<float>(const Inst& I) { return I.yvf; }
template <> __device__ __forceinline__ const double2* yv_of<ff>(const Inst& I) { return I.yv; }
template <class T> __device__ __forceinline__ typename Sto<T>::c* xz_of(const Inst& I);
template <> __device__ __forceinline__ double2* xz_of<double>(const Inst& I) { return I.xz; }
template <> __device__ __forceinline__ float2* xz_of<float>(const Inst& I) { return I.xzf; }
template <> __device__ __forceinline__ double2* xz_of<ff>(const Inst& I) { return I.xz; }
template <class T> __device__ __forceinline__ const typename Sto<T>::c* twx_of(const Inst& I);
template <> __device__ __forceinline__ const double2* twx_of<double>(const Inst& I) { return I.twx; }
template <> __device__ __forceinline__ const float2* twx_of<float>(const Inst& I) { return I.twxf; }
template <> __device__ __forceinline__ const double2* twx_of<ff>(const Inst& I) { return I.twx; }
template <class T> __device__ __forceinline__ const typename Sto<T>::c* twz_of(const Inst& I);
template <> __device__ __forceinline__ const double2* twz_of<double>(const Inst& I) { return I.twz; }
template <> __device__ __forceinline__ const float2* twz_of<float>(const Inst& I) { return I.twzf; }
template <> __device__ __forceinline__ const double2* twz_of<ff>(const Inst& I) { return I.twz; }

// ------------------------------------------------------------------ Stockham FFT in shared memory
template <int R, class C>
__device__ __forceinline__ void butterfly(C* v, bool inv);

template <>
__device__ __forceinline__ void butterfly<2, double2>(double2* v, bool) {
  const double2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <>
__device__ __forceinline__ void butterfly<2, float2>(float2* v, bool) {
  const float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <int R, class C>
__device__ __forceinline__ void butterfly4(C* v, bool inv) {
  const C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  const C t2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
  // t3 = -i d (forward) or +i d (inverse)
  C t3;
  if (inv) { t3.x = -d.y; t3.y = d.x; } else { t3.x = d.y; t3.y = -d.x; }
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}
template <>
__device__ __forceinline__ void butterfly<2, ff2>(ff2* v, bool) {
  const ff2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}
template <>
__device__ __forceinline__ void butterfly<4, double2>(double2* v, bool inv) { butterfly4<4, double2>(v, inv); }
template <>
__device__ __forceinline__ void butterfly<4, ff2>(ff2* v, bool inv) { butterfly4<4, ff2>(v, inv); }
template <>
__device__ __forceinline__ void butterfly<4, float2>(float2* v, bool inv) { butterfly4<4, float2>(v, inv); }

template <class C>
__device__ __forceinline__ void butterfly3(C* v, bool inv) {
  using R = decltype(v[0].x);
  const R h = (R)0.86602540378443864676;  // sin(2 pi/3)
  const C s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
  const C y0 = cadd(v[0], s);
  C m, it;
  m.x = fma((R)-0.5, s.x, v[0].x);
  m.y = fma((R)-0.5, s.y, v[0].y);
  // forward: y1 = m - i t, y2 = m + i t with t = h d
  it.x = -h * d.y;
  it.y = h * d.x;
  v[0] = y0;
  v[1] = inv ? cadd(m, it) : csub(m, it);
  v[2] = inv ? csub(m, it) : cadd(m, it);
}
template <>
__device__ __forceinline__ void butterfly<3, double2>(double2* v, bool inv) { butterfly3(v, inv); }
template <>
__device__ __forceinline__ void butterfly<3, float2>(float2* v, bool inv) { butterfly3(v, inv); }
template <>
__device__ __forceinline__ void butterfly<3, ff2>(ff2* v, bool inv) { butterfly3(v, inv); }

// ------------------------------------------------------------------ twiddled butterflies
// A Stockham pass of radix R with Ns > 1 multiplies input r of butterfly k by w^(r q1),
// q1 = k * twstep, w = exp(-2 pi i/L) (its conjugate for the inverse transform), then applies
// the radix-R DFT.  Two twiddle representations:
//
// TwStd: the table tw[q] = w^q; a complex multiply per twiddled input, then the butterfly
// (radix 4 with three twiddles: 28 FP64 operations; radix 2: 8).
//
// TwTan (FP64): every twiddle in the tangent form of Linzer and Feig (FMA-based FFT
// butterflies, IEEE Trans. Signal Process. 1993): w^q = m (rot ? i : 1)(1 + i t) with |t| <= 1, so that
// x +- w^q y costs six fused multiply-adds: z = y (1 + i t) takes two, x +- m z four (a factor
// i swaps the parts of z, done with selects on the integer pipe).  A radix-4 butterfly is
// four such pairs, using w^(3 q1) y3 +- ... = w^q1 (y1 +- w^(2 q1) y3) and -i w^q1 = w^(q1 + L/4):
// 24 FMAs.  Radix 2: one pair, 6 FMAs.  The entries e[q] = (t, m) and rot[q] are built on
// the host for the transform's direction (conjugated for the inverse).
template <class C>
struct TwStd {
  const C* tw;
};
struct TwTan {
  const double2* e;
  const unsigned char* rot;
};

// (x + w y, x - w y) for the tangent-form twiddle (e, rot)
__device__ __forceinline__ void tan_pm(double2 x, double2 y, double2 e, bool rot, double2* P, double2* Q) {
  const double zr = fma(-e.x, y.y, y.x), zi = fma(e.x, y.x, y.y);
  const double u = rot ? zi : zr, v = rot ? zr : zi;
  const double rp = fma(e.y, u, x.x), rm = fma(-e.y, u, x.x);
  const double ip = fma(e.y, v, x.y), im = fma(-e.y, v, x.y);
  *P = make_double2(rot ? rm : rp, ip);
  *Q = make_double2(rot ? rp : rm, im);
}

// The twiddled radix-R butterfly of a pass (Ns > 1), input r of butterfly k at v[r].
template <int R, class C>
__device__ __forceinline__ void tw_butterfly(C* v, const TwStd<C>& T, int k, int twstep, int L, bool inv) {
#pragma unroll
  for (int r = 1; r < R; ++r) {
    C w = T.tw[r * k * twstep];
    if (inv) w.y = -w.y;
    v[r] = cmul(v[r], w);
  }
  butterfly<R, C>(v, inv);
}
template <int R>
__device__ __forceinline__ void tw_butterfly(double2* v, const TwTan& T, int k, int twstep, int L, bool inv) {
  const int q1 = k * twstep;
  if (R == 2) {
    tan_pm(v[0], v[1], T.e[q1], T.rot[q1], &v[0], &v[1]);
  } else if (R == 4) {
    const int q2 = 2 * q1, q3 = q1 + L / 4;
    const double2 e2 = T.e[q2];
    const bool r2 = T.rot[q2];
    double2 t0, t1, P, Q;
    tan_pm(v[0], v[2], e2, r2, &t0, &t1);
    tan_pm(v[1], v[3], e2, r2, &P, &Q);
    tan_pm(t0, P, T.e[q1], T.rot[q1], &v[0], &v[2]);
    tan_pm(t1, Q, T.e[q3], T.rot[q3], &v[1], &v[3]);
  } else {
    // radix 3: rebuild w^(r q1) = (m, m t) or (-m t, m) and multiply
#pragma unroll
    for (int r = 1; r < R; ++r) {
      const int q = r * q1;
      const double2 e = T.e[q];
      const double mt = e.y * e.x;
      const double2 w = T.rot[q] ? make_double2(-mt, e.y) : make_double2(e.y, mt);
      v[r] = cmul(v[r], w);
    }
    butterfly<R, double2>(v, inv);
  }
}


}  // namespace pcf
