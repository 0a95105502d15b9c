// Host side of the pcfadj library: per-grid tables, context, launch sequences, C ABI.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <thread>
#include <vector>

#include "pcf_kernels.cuh"

using namespace pcf;

namespace {

constexpr double kPi = 3.14159265358979323846;

thread_local char g_last_error[256] = "";

#define PCF_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      snprintf(g_last_error, sizeof(g_last_error), "%s: %s", #call, cudaGetErrorString(e_)); \
      return PCF_ECUDA;                                                                    \
    }                                                                                      \
  } while (0)

bool grid_ok(int nx, int ny, int nz) {
  auto ok_fft = [](int n) {
    if (n < 16 || n > 128 || (n % 2)) return false;
    int m = n;
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    return m == 1;
  };
  return ok_fft(nx) && ok_fft(nz) && ny >= 9 && ny <= 129 && (ny % 2 == 1);
}

void radix_plan(int L, int* r, int* nr) {
  int n = 0;
  while (L % 4 == 0) { r[n++] = 4; L /= 4; }
  while (L % 2 == 0) { r[n++] = 2; L /= 2; }
  while (L % 3 == 0) { r[n++] = 3; L /= 3; }
  *nr = n;
}

// cos(pi a / N) with the argument reduced exactly in integers
double cospi_frac(long long a, int N) {
  long long m = a % (2LL * N);
  if (m < 0) m += 2LL * N;
  return std::cos(kPi * (double)m / (double)N);
}

// T'_n(cos(pi j/N))
double cheb_dvalue(int n, int j, int N) {
  if (j == 0) return (double)n * n;
  if (j == N) return ((n + 1) % 2 ? -1.0 : 1.0) * (double)n * n;
  const double th = kPi * (double)j / (double)N;
  long long m = ((long long)n * j) % (2LL * N);
  return (double)n * std::sin(kPi * (double)m / (double)N) / std::sin(th);
}

// Cinv_{n j}: coefficient n of the interpolant of the values at y_j (DCT-I inverse).
double cinv(int n, int j, int N) {
  const double cn = (n == 0 || n == N) ? 2.0 : 1.0;
  const double cj = (j == 0 || j == N) ? 2.0 : 1.0;
  return 2.0 / ((double)N * cn * cj) * cospi_frac((long long)n * j, N);
}

std::vector<double> make_cheb(int N) {
  const ChebLayout CL(N);
  const int H = CL.H;
  std::vector<double> t(CL.total(), 0.0);
  for (int j = 0; j < H; ++j)
    for (int k = 0; k < H; ++k) {
      t[CL.Ce() + j * H + k] = cospi_frac((long long)j * (2 * k), N);
      t[CL.De() + j * H + k] = cheb_dvalue(2 * k, j, N);
      if (k < H - 1) {
        t[CL.Co() + j * H + k] = cospi_frac((long long)j * (2 * k + 1), N);
        t[CL.Do() + j * H + k] = cheb_dvalue(2 * k + 1, j, N);
      }
    }
  for (int k = 0; k < H; ++k)
    for (int j = 0; j < H; ++j) {
      t[CL.Ae() + k * H + j] = cinv(2 * k, j, N);
      if (k < H - 1) t[CL.Ao() + k * H + j] = cinv(2 * k + 1, j, N);
    }
  return t;
}

std::vector<double> make_rco(int N) {
  const RcoLayout RL(N);
  const int Mh = N / 2 + 1;
  std::vector<double> t(RL.total(), 0.0);
  for (int par = 0; par < 2; ++par) {
    const int Mc = (N - par) / 2 + 1;
    for (int i = 0; i < Mc; ++i) {
      const int n = par + 2 * i;
      const double dn = n;
      if (i >= 1) {
        const double cm2 = (n - 2 == 0) ? 2.0 : 1.0;
        t[RL.off(par, 0) + i] = -cm2 / (4.0 * dn * (dn - 1.0));
        t[RL.off(par, 1) + i] = (n <= N - 2) ? 1.0 / (2.0 * (dn * dn - 1.0)) : 0.0;
        t[RL.off(par, 2) + i] = (n + 2 <= N - 2) ? -1.0 / (4.0 * dn * (dn + 1.0)) : 0.0;
      }
      t[RL.off(par, 3) + i] = dn * dn;
      t[RL.off(par, 4) + i] = 2.0 * dn;
    }
    (void)Mh;
  }
  return t;
}

// Sweep coefficients of the quasi-tridiagonal tau system (lambda, par), see tau_solve.
void solver_coefs(int N, int par, double lam, const std::vector<double>& rco, double* dst) {
  const RcoLayout RL(N);
  const int Mh = N / 2 + 1;
  const int Mc = (N - par) / 2 + 1;
  double* c = dst;
  double* inv = dst + Mh;
  double* beta = dst + 2 * Mh;
  double* B = dst + 3 * Mh;
  for (int i = 0; i < 4 * Mh + 2; ++i) dst[i] = 0.0;
  const double* ra = rco.data() + RL.off(par, 0);
  const double* rb = rco.data() + RL.off(par, 1);
  const double* rc = rco.data() + RL.off(par, 2);
  double bnext = 0.0;
  for (int i = Mc - 1; i >= 1; --i) {
    const double a = lam * ra[i], bb = 1.0 + lam * rb[i], cc = lam * rc[i];
    const double den = bb + cc * bnext;
    c[i] = cc;
    inv[i] = 1.0 / den;
    beta[i] = -a / den;
    bnext = beta[i];
  }
  B[0] = 1.0;
  double sum = 1.0;
  for (int i = 1; i < Mc; ++i) {
    B[i] = beta[i] * B[i - 1];
    sum += B[i];
  }
  dst[4 * Mh] = 1.0 / sum;
}

// Homogeneous responses and 2x2 influence matrix of group g (see mode_chain).
void group_tables(int N, int g, double k2, double sigma, const double* tab, const std::vector<double>& rco,
                  double* dst) {
  const TabLayout TL(N);
  const RcoLayout RL(N);
  const int Mh = N / 2 + 1;
  const int pv = g, pP = 1 - g;
  const int McP = (N - pP) / 2 + 1, McV = (N - pv) / 2 + 1;
  const double lamH = sigma + k2;
  std::vector<double> P(Mh), T(Mh), V(Mh), R(Mh), unit(Mh);
  double F1[2], F2[2];
  std::vector<double> vh[2];
  for (int h = 0; h < 2; ++h) {
    std::fill(R.begin(), R.end(), 0.0);
    double bc = 0.0;
    if (h == 0) {
      bc = 1.0;  // Dirichlet value of the pressure class
    } else {
      std::fill(unit.begin(), unit.end(), 0.0);
      unit[McV - 1] = 1.0;  // T_N (g = 0) or T_{N-1} (g = 1)
      class_deriv(N, pv, unit.data(), rco.data() + RL.off(pv, 4), T.data());
      for (int i = 0; i < McP; ++i) R[i] = -T[i];
    }
    const double* s = tab + TL.solver(0, pP);
    tau_solve(McP, s, s + Mh, s + 2 * Mh, s + 3 * Mh, s[4 * Mh], rco.data() + RL.off(pP, 0),
              rco.data() + RL.off(pP, 1), rco.data() + RL.off(pP, 2), R.data(), bc, P.data());
    class_deriv(N, pP, P.data(), rco.data() + RL.off(pP, 4), T.data());
    for (int i = 0; i < McV; ++i) R[i] = -T[i];
    s = tab + TL.solver(1, pv);
    tau_solve(McV, s, s + Mh, s + 2 * Mh, s + 3 * Mh, s[4 * Mh], rco.data() + RL.off(pv, 0),
              rco.data() + RL.off(pv, 1), rco.data() + RL.off(pv, 2), R.data(), 0.0, V.data());
    double f1 = 0.0;
    for (int i = 0; i < McV; ++i) f1 += rco[RL.off(pv, 3) + i] * V[i];
    double f2 = lamH * V[McV - 1];
    if (g == 1) f2 += 2.0 * N * P[McP - 1];
    if (h == 1) f2 -= 1.0;
    F1[h] = f1;
    F2[h] = f2;
    vh[h] = V;
  }
  for (int i = 0; i < 2 * Mh + 4; ++i) dst[i] = 0.0;
  for (int i = 0; i < McV; ++i) {
    dst[i] = vh[0][i];
    dst[Mh + i] = vh[1][i];
  }
  const double det = F1[0] * F2[1] - F1[1] * F2[0];
  dst[2 * Mh + 0] = F2[1] / det;
  dst[2 * Mh + 1] = -F1[1] / det;
  dst[2 * Mh + 2] = -F2[0] / det;
  dst[2 * Mh + 3] = F1[0] / det;
}

std::vector<double> make_mode_tables(int N, const std::vector<double>& kx, const std::vector<double>& kz,
                                     double sigma, const std::vector<double>& rco) {
  const TabLayout TL(N);
  const int Mx = (int)kx.size(), Mz = (int)kz.size();
  const int PM = TL.per_mode();
  std::vector<double> t((size_t)Mx * Mz * PM, 0.0);
  for (int i = 0; i < Mx; ++i)
    for (int p = 0; p < Mz; ++p) {
      double* d = t.data() + ((size_t)i * Mz + p) * PM;
      const double k2 = kx[i] * kx[i] + kz[p] * kz[p];
      for (int par = 0; par < 2; ++par) {
        solver_coefs(N, par, k2, rco, d + TL.solver(0, par));
        solver_coefs(N, par, sigma + k2, rco, d + TL.solver(1, par));
      }
      if (k2 > 0.0)
        for (int g = 0; g < 2; ++g) group_tables(N, g, k2, sigma, d, rco, d + TL.group(g));
    }
  return t;
}

// Dense per-mode operators: the chain of mode_chain applied to unit inputs (no correction
// shortcut: the same arithmetic as the sweep path, one column at a time).
std::vector<double> make_dense_tables(int N, const std::vector<double>& kx, const std::vector<double>& kz,
                                      double sigma, const std::vector<double>& rco, const std::vector<double>& tabs) {
  const TabLayout TL(N);
  const RcoLayout RL(N);
  const DenseLayout DL(N);
  const int Mx = (int)kx.size(), Mz = (int)kz.size(), Mh = N / 2 + 1, L2 = 2 * Mh;
  std::vector<double> out((size_t)Mx * Mz * DL.per_mode(), 0.0);
  auto work = [&](int i0, int i1) {
  std::vector<double> Fr(6 * L2), sc(6 * Mh);
  for (int i = i0; i < i1; ++i)
    for (int p = 0; p < Mz; ++p) {
      const size_t m = (size_t)i * Mz + p;
      const double* tab = tabs.data() + m * TL.per_mode();
      double* d = out.data() + m * DL.per_mode();
      const double k2 = kx[i] * kx[i] + kz[p] * kz[p];
      for (int g = 0; g < 2; ++g) {
        const int pv = g, pP = 1 - g;
        const int McV = (N - pv) / 2 + 1, McP = (N - pP) / 2 + 1;
        if (k2 == 0.0) {
          const int Mc = (N - g) / 2 + 1;
          const double* s = tab + TL.solver(1, g);
          std::vector<double> e(Mh), y(Mh);
          for (int j = 0; j < Mc; ++j) {
            std::fill(e.begin(), e.end(), 0.0);
            e[j] = 1.0;
            tau_solve(Mc, s, s + Mh, s + 2 * Mh, s + 3 * Mh, s[4 * Mh], rco.data() + RL.off(g, 0),
                      rco.data() + RL.off(g, 1), rco.data() + RL.off(g, 2), e.data(), 0.0, y.data());
            for (int r = 0; r < Mc; ++r) d[DL.at(g, DL.kEh, r, j)] = y[r];
          }
          continue;
        }
        // columns for f_v (class pv) and g (class pP), taken through the real-part chain
        // (rho = 0, where g enters as -(kx f_u + kz f_w) built from the imaginary parts)
        for (int src = 0; src < 2; ++src) {
          const int nc = src == 0 ? McV : McP;
          for (int j = 0; j < nc; ++j) {
            std::fill(Fr.begin(), Fr.end(), 0.0);
            if (src == 0) {
              Fr[(1 * 2 + 0) * L2 + pv * Mh + j] = 1.0;
            } else {
              // rho = 0: g_re = -(kx Im f_u + kz Im f_w); choose Im f_u so that g_re = e_j
              if (kx[i] != 0.0) Fr[(0 * 2 + 1) * L2 + pP * Mh + j] = -1.0 / kx[i];
              else Fr[(2 * 2 + 1) * L2 + pP * Mh + j] = -1.0 / kz[p];
            }
            std::fill(sc.begin(), sc.end(), 0.0);
            mode_chain(N, g, 0, kx[i], kz[p], sigma + k2, tab, rco.data(), Fr.data(), L2, sc.data());
            for (int r = 0; r < McV; ++r) d[DL.at(g, src == 0 ? DL.kAv : DL.kAg, r, j)] = sc[2 * Mh + r];
          }
        }
        // eta: inverse Helmholtz of class pP
        const double* s = tab + TL.solver(1, pP);
        std::vector<double> e(Mh), y(Mh);
        for (int j = 0; j < McP; ++j) {
          std::fill(e.begin(), e.end(), 0.0);
          e[j] = 1.0;
          tau_solve(McP, s, s + Mh, s + 2 * Mh, s + 3 * Mh, s[4 * Mh], rco.data() + RL.off(pP, 0),
                    rco.data() + RL.off(pP, 1), rco.data() + RL.off(pP, 2), e.data(), 0.0, y.data());
          for (int r = 0; r < McP; ++r) d[DL.at(g, DL.kEh, r, j)] = y[r];
        }
      }
    }
  };
  // x-mode rows are independent: split them over host threads
  const int nt = std::max(1, std::min<int>(Mx, (int)std::thread::hardware_concurrency()));
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) pool.emplace_back(work, Mx * t / nt, Mx * (t + 1) / nt);
  for (auto& th : pool) th.join();
  return out;
}

// Interpolatory (Clenshaw-Curtis) weights: w_j = sum_n Cinv_{n j} int_{-1}^{1} T_n dy.
std::vector<double> make_ccw(int N) {
  std::vector<double> w(N + 1, 0.0);
  for (int j = 0; j <= N; ++j) {
    double s = 0.0;
    for (int n = 0; n <= N; n += 2) s += cinv(n, j, N) * (2.0 / (1.0 - (double)n * n));
    w[j] = s;
  }
  return w;
}

uint16_t f2bf(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
float bf2f(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

// Split-BF16 copies of the full Chebyshev matrices for the tensor-core transforms:
// [C hi, C lo, C' hi, C' lo, Cinv hi, Cinv lo], each P x P row-major, zero padded.
std::vector<uint16_t> make_tc_matrices(int N) {
  const int ny = N + 1, P = (ny + 15) & ~15;
  std::vector<uint16_t> t((size_t)6 * P * P, 0);
  auto put = [&](int mat, int r, int c, double v) {
    const float f = (float)v;
    const uint16_t hi = f2bf(f);
    t[((size_t)2 * mat) * P * P + (size_t)r * P + c] = hi;
    t[((size_t)2 * mat + 1) * P * P + (size_t)r * P + c] = f2bf(f - bf2f(hi));
  };
  for (int j = 0; j < ny; ++j)
    for (int n = 0; n < ny; ++n) {
      put(0, j, n, cospi_frac((long long)j * n, N));
      put(1, j, n, cheb_dvalue(n, j, N));
      put(2, n, j, cinv(n, j, N));
    }
  return t;
}

// The tcgen05 contraction's operands as byte images of its shared-memory A region: for each
// matrix and part (hi, lo) of make_tc_matrices, 128 rows (rows >= P zero) x P K elements in
// the no-swizzle K-major core-matrix layout, where the chunk of row r and K elements
// 8kc..8kc+7 starts at element ((kc * 16 + r / 8) * 64 + (r % 8) * 8).  One bulk copy then
// fills the region.  Empty when P > 128 (the kernel is not used there).
std::vector<uint16_t> make_tc05_images(const std::vector<uint16_t>& t, int P) {
  if (P > 128) return {};
  const size_t img = (size_t)128 * P;
  std::vector<uint16_t> o(6 * img, 0);
  for (int a = 0; a < 6; ++a)
    for (int r = 0; r < P; ++r)
      for (int kc = 0; kc < P / 8; ++kc)
        for (int e = 0; e < 8; ++e)
          o[a * img + ((size_t)kc * 16 + r / 8) * 64 + (r % 8) * 8 + e] = t[(size_t)a * P * P + (size_t)r * P + 8 * kc + e];
  return o;
}

std::vector<float2> to_float2(const std::vector<double2>& v) {
  std::vector<float2> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = make_float2((float)v[i].x, (float)v[i].y);
  return o;
}

std::vector<double2> make_twiddles(int L) {
  std::vector<double2> w(L);
  for (int k = 0; k < L; ++k) {
    const double a = -2.0 * kPi * (double)k / (double)L;
    w[k] = make_double2(std::cos(a), std::sin(a));
  }
  return w;
}

// Tangent form of the twiddles w^q = c + i s (w = e^{-2 pi i/L}) for the FMA butterflies:
// w^q = m (1 + i t) with t = s/c, m = c where |c| >= |s|; else w^q = m i (1 + i t) with
// m = s, t = -c/s (rot = 1).  |t| <= 1 either way.  rot[q] = 1 exactly where the angle's
// distance to the nearest multiple of pi exceeds pi/4: 2q mod L in (L/4, 3L/4), decided in
// integers.  tan[0, L): w^q; tan[L, 2L): its conjugate c - i s (t -> -t, and m -> -m where
// rot = 1).
void make_tangent_twiddles(int L, std::vector<double2>* tan, std::vector<unsigned char>* rot) {
  tan->assign(2 * (size_t)L, make_double2(0.0, 0.0));
  rot->assign(L, 0);
  for (int q = 0; q < L; ++q) {
    const double a = -2.0 * kPi * (double)q / (double)L;
    const double c = std::cos(a), s = std::sin(a);
    const int r2 = (2 * q) % L;
    const bool r = 4 * r2 > L && 4 * r2 < 3 * L;
    (*rot)[q] = r ? 1 : 0;
    if (!r) {
      (*tan)[q] = make_double2(s / c, c);
      (*tan)[L + q] = make_double2(-s / c, c);
    } else {
      (*tan)[q] = make_double2(-c / s, s);
      (*tan)[L + q] = make_double2(c / s, -s);
    }
  }
}

template <class T>
cudaError_t upload(const std::vector<T>& h, T** d) {
  cudaError_t e = cudaMalloc((void**)d, h.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

#include "pcf_ctx.h"

namespace {

template <class T>
cudaError_t ctx_alloc(pcf_ctx* c, T** p, size_t n) {
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e == cudaSuccess) c->allocs.push_back((void*)*p);
  return e;
}

pcf_status push_descriptors(pcf_ctx* c) {
  PCF_CUDA(cudaMemcpyAsync(c->dinst, c->hinst.data(), sizeof(Inst) * c->hinst.size(), cudaMemcpyHostToDevice, c->cs));
  return PCF_OK;
}

LaunchInfo li_of(pcf_ctx* c, const int* pre) { return LaunchInfo{c->dinst, pre, c->B}; }

// kernel launch with optional per-class event timing
template <class F>
pcf_status timed(pcf_ctx* c, int cls, F&& launch) {
  if (!c->timing) {
    launch();
    return PCF_OK;
  }
  cudaEvent_t a, b;
  PCF_CUDA(cudaEventCreate(&a));
  PCF_CUDA(cudaEventCreate(&b));
  PCF_CUDA(cudaEventRecord(a, c->cs));
  launch();
  PCF_CUDA(cudaEventRecord(b, c->cs));
  PCF_CUDA(cudaEventSynchronize(b));
  float ms = 0.f;
  PCF_CUDA(cudaEventElapsedTime(&ms, a, b));
  c->kms[cls] += ms;
  c->kcount[cls] += 1;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return PCF_OK;
}

pcf_status launch_mode(pcf_ctx* c, int op, int sig, int step_index) {
  return timed(c, op == MODE_PHI ? 3 : (op == MODE_SYNTH_ONLY ? 0 : 6), [&] {
    k_mode<<<c->cta_mode, c->mode_thr, c->sm_mode, c->cs>>>(li_of(c, c->pre_mode), op, sig, c->mpc, step_index);
  });
}
pcf_status launch_synth(pcf_ctx* c, int slot, int nf) {
  const int* pre = nf == kFieldsSynth ? c->pre_synth11 : c->pre_synth3;
  const int ctas = nf == kFieldsSynth ? c->cta_synth11 : c->cta_synth3;
  return timed(c, slot == 0 ? 1 : 4, [&] {
    if (c->plane_warp) launch_xzsynth_warp(ctas, c->sm_synth, c->cs, li_of(c, pre), slot, nf);
    else launch_xzsynth(c->plane_kind, ctas, c->sm_synth, c->cs, li_of(c, pre), slot, nf);
  });
}
pcf_status launch_prodM(pcf_ctx* c) {
  return timed(c, 2, [&] {
    if (c->plane_warp) launch_prod_warp(false, c->cta_prod, c->sm_prod, c->cs, li_of(c, c->pre_prod), -1);
    else launch_prod(c->plane_kind, false, c->suction, c->cta_prod, c->sm_prod, c->cs, li_of(c, c->pre_prod));
  });
}
pcf_status launch_prodN(pcf_ctx* c, int step_index = -1) {
  return timed(c, 5, [&] {
    if (c->plane_warp) launch_prod_warp(true, c->cta_prod, c->sm_prod, c->cs, li_of(c, c->pre_prod), step_index);
    else
      launch_prod(c->plane_kind, true, c->suction, c->cta_prod, c->sm_prod, c->cs, li_of(c, c->pre_prod),
                  step_index);
  });
}

pcf_status launch_tc_synth(pcf_ctx* c, int slot) {
  return timed(c, 12, [&] {
    if (c->tc05) launch_cheb_synth_tc05(c->cta_tcs, c->sm_tc, c->cs, li_of(c, c->pre_tcs), slot);
    else launch_cheb_synth_tc(c->cta_tcs, c->sm_tc, c->cs, li_of(c, c->pre_tcs), slot);
  });
}
pcf_status launch_tc_analysis(pcf_ctx* c) {
  return timed(c, 13, [&] {
    if (c->tc05) launch_cheb_analysis_tc05(c->cta_tca, c->sm_tc, c->cs, li_of(c, c->pre_tca));
    else launch_cheb_analysis_tc(c->cta_tca, c->sm_tc, c->cs, li_of(c, c->pre_tca));
  });
}
// split mode kernels of the FP64 descent step
GroupLaunch gl_of(pcf_ctx* c, const int* pre, int red = 0) {
  return GroupLaunch{c->dinst, pre, c->d_groups, c->ngroups, red};
}
// red: the reduced launch of a symmetric descent step (modes m >= 0 only)
pcf_status launch_split_analysis(pcf_ctx* c, int op, bool red = false) {
  return timed(c, 7, [&] {
    launch_yanalysis(red ? c->cta_ya_r : c->cta_ya, c->thr_ya, c->sm_ya, c->cs,
                     gl_of(c, red ? c->pre_ya_r : c->pre_ya, red), op, c->plane_kind == 2, c->smt);
  });
}
GroupLaunch gl_solve(pcf_ctx* c, bool red = false) {
  return GroupLaunch{c->dinst, red ? c->pre_ys_r : c->pre_ys, c->d_groups_s, c->ngroups_s, red ? 1 : 0};
}
pcf_status launch_split_solve(pcf_ctx* c, int op, bool red = false) {
  if (c->sweep)
    return timed(c, op == MODE_PHI ? 3 : 6, [&] {
      launch_sweep(red ? c->cta_sw_r : c->cta_sw, c->thr_sw, c->sm_sw, c->cs,
                   LaunchInfo{c->dinst, red ? c->pre_sw_r : c->pre_sw, c->B}, op, red ? 1 : 0);
    });
  return timed(c, op == MODE_PHI ? 3 : 6, [&] {
    launch_ysolve(red ? c->grid_ys_r : c->grid_ys, red ? c->cta_ys_r : c->cta_ys, c->buf_ys, c->rows_ys, c->sm_ys,
                  c->cs, gl_solve(c, red), op);
  });
}
pcf_status launch_fused_step(pcf_ctx* c, int op) {
  return timed(c, op == MODE_PHI ? 3 : 6,
               [&] { launch_ystep(c->cta_yf, c->sm_yf, c->cs, gl_of(c, c->pre_yf), op); });
}
pcf_status launch_split_jnorm(pcf_ctx* c, int step_index) {
  return timed(c, 9, [&] { launch_jnorm(c->B, c->cs, c->dinst, step_index); });
}
pcf_status launch_split_synth(pcf_ctx* c, int slot, int in_step, bool red = false) {
  return timed(c, in_step ? 8 : 0, [&] {
    launch_ysynth_split(red ? c->cta_yy_r : c->cta_yy, c->thr_yy, c->sm_yy, c->cs,
                        gl_of(c, red ? c->pre_yy_r : c->pre_yy, red), slot, in_step, c->plane_kind == 2, c->smt_y);
  });
}

// y-synthesis of the state (slot 0) or of r1 (slot 1) in either form
pcf_status launch_ysynth(pcf_ctx* c, int slot) {
  if (c->mixed) return launch_tc_synth(c, slot);
  if (c->split) return launch_split_synth(c, slot, 0);
  return launch_mode(c, MODE_SYNTH_ONLY, slot, 0);
}

// projection onto the symmetric subspace: each instance's own mask (mask_override < 0) or mask
pcf_status launch_sym(pcf_ctx* c, int mask_override, bool red = false) {
  return timed(c, 10, [&] { launch_symmetrize(c->sym_ctas, c->B, c->cs, c->dinst, mask_override, red ? 1 : 0); });
}

pcf_status check_launch() {
  PCF_CUDA(cudaGetLastError());
  return PCF_OK;
}

#define PCF_TRY(x)              \
  do {                          \
    pcf_status s_ = (x);        \
    if (s_ != PCF_OK) return s_; \
  } while (0)

pcf_status enter(pcf_ctx* c) {
  PCF_CUDA(cudaEventRecord(c->ev_in, c->user));
  PCF_CUDA(cudaStreamWaitEvent(c->cs, c->ev_in, 0));
  return PCF_OK;
}
pcf_status leave(pcf_ctx* c) {
  PCF_CUDA(cudaEventRecord(c->ev_out, c->cs));
  PCF_CUDA(cudaStreamWaitEvent(c->user, c->ev_out, 0));
  return PCF_OK;
}

void set_pointers(pcf_ctx* c, const double* u, const double* r, double* f) {
  for (int b = 0; b < c->B; ++b) {
    Inst& I = c->hinst[b];
    I.uhat = u ? (double2*)u + c->state_off[b] : nullptr;
    I.rhat = r ? (double2*)r + c->state_off[b] : nullptr;
    I.fhat = f ? (double2*)f + c->state_off[b] : nullptr;
    I.hist = nullptr;
    I.active = nullptr;
    I.tol = 0.0;
  }
}

pcf_status step_body(pcf_ctx* c, int s) {
  if (c->mixed) {
    if (s > 0) PCF_TRY(launch_tc_synth(c, 0));
    PCF_TRY(launch_synth(c, 0, kFieldsSynth));
    PCF_TRY(launch_prodM(c));
    PCF_TRY(launch_tc_analysis(c));
    PCF_TRY(launch_mode(c, MODE_PHI, 0, s));
    PCF_TRY(launch_tc_synth(c, 1));
    PCF_TRY(launch_synth(c, 1, kFieldsSynth));
    PCF_TRY(launch_prodN(c, s));  // with J, its history entry and the convergence mask
    PCF_TRY(launch_tc_analysis(c));
    PCF_TRY(launch_mode(c, MODE_PSI_UPDATE, 1, -1));
    if (c->any_sym) PCF_TRY(launch_sym(c, -1));  // the next step's synthesis reads the projected state
    return PCF_OK;
  }
  if (c->split && c->fused) {
    PCF_TRY(launch_synth(c, 0, kFieldsSynth));
    PCF_TRY(launch_prodM(c));
    PCF_TRY(launch_fused_step(c, MODE_PHI));
    PCF_TRY(launch_synth(c, 1, kFieldsSynth));
    PCF_TRY(launch_prodN(c));
    PCF_TRY(launch_split_jnorm(c, s));
    PCF_TRY(launch_fused_step(c, MODE_PSI_UPDATE));
    if (c->any_sym) {
      PCF_TRY(launch_sym(c, -1));
      PCF_TRY(launch_ysynth(c, 0));
    }
    return PCF_OK;
  }
  if (c->split) {
    // in the symmetric subspace of s2 the per-mode work covers the modes m >= 0; the
    // synthesis mirrors their y-values to -m, and the projection after the update rebuilds
    // the state's modes -m
    const bool red = c->reduced;
    // the y-values of the state the previous step updated (the call's first step reads the
    // synthesis done at the call's start)
    if (s > 0) PCF_TRY(launch_split_synth(c, 0, 1, red));
    PCF_TRY(launch_synth(c, 0, kFieldsSynth));
    PCF_TRY(launch_prodM(c));
    PCF_TRY(launch_split_analysis(c, MODE_PHI, red));
    PCF_TRY(launch_split_solve(c, MODE_PHI, red));
    PCF_TRY(launch_split_synth(c, 1, 1, red));
    PCF_TRY(launch_synth(c, 1, kFieldsSynth));
    PCF_TRY(launch_prodN(c, s));  // with J, its history entry and the convergence mask
    PCF_TRY(launch_split_analysis(c, MODE_PSI_UPDATE, red));
    PCF_TRY(launch_split_solve(c, MODE_PSI_UPDATE, red));
    if (c->any_sym) PCF_TRY(launch_sym(c, -1, red));
    return PCF_OK;
  }
  PCF_TRY(launch_synth(c, 0, kFieldsSynth));
  PCF_TRY(launch_prodM(c));
  PCF_TRY(launch_mode(c, MODE_PHI, 0, s));
  PCF_TRY(launch_synth(c, 1, kFieldsSynth));
  PCF_TRY(launch_prodN(c, s));  // with J, its history entry and the convergence mask
  PCF_TRY(launch_mode(c, MODE_PSI_UPDATE, 1, -1));
  if (c->any_sym) {
    PCF_TRY(launch_sym(c, -1));
    PCF_TRY(launch_ysynth(c, 0));
  }
  return PCF_OK;
}

// One DNS step u <- u + dt r1 (pcf_dns): ||u|| and the extremum capture of the previous
// step, M(u), the Stokes step of §4 step 1 (writing r1), the update, and the y-synthesis of
// the new state for the next step.
pcf_status dns_body(pcf_ctx* c) {
  PCF_TRY(launch_synth(c, 0, kFieldsSynth));
  PCF_TRY(timed(c, 11, [&] {
    launch_norm_planes(c->plane_kind, c->cta_synth3, c->cs, li_of(c, c->pre_synth3), 0);
    launch_dns_norm(c->B, c->cs, c->dinst, c->d_dns);
    launch_dns_capture(c->dns_ctas, c->B, c->cs, c->dinst, c->d_dns);
  }));
  PCF_TRY(launch_prodM(c));
  if (c->mixed) {
    PCF_TRY(launch_tc_analysis(c));
    PCF_TRY(launch_mode(c, MODE_PHI, 0, 0));
  } else if (c->split && c->fused) {
    PCF_TRY(launch_fused_step(c, MODE_PHI));
  } else if (c->split) {
    PCF_TRY(launch_split_analysis(c, MODE_PHI));
    PCF_TRY(launch_split_solve(c, MODE_PHI));
  } else {
    PCF_TRY(launch_mode(c, MODE_PHI, 0, 0));
  }
  PCF_TRY(timed(c, 11, [&] { launch_dns_update(c->dns_ctas, c->B, c->cs, c->dinst, c->d_dns); }));
  if (c->any_sym) PCF_TRY(launch_sym(c, -1));
  return launch_ysynth(c, 0);
}

}  // namespace

// ------------------------------------------------------------------ ABI
extern "C" {

int pcf_abi_version(void) { return PCF_ABI_VERSION; }

const char* pcf_status_str(pcf_status s) {
  switch (s) {
    case PCF_OK: return "ok";
    case PCF_EINVAL: return "invalid argument";
    case PCF_ECUDA: return g_last_error[0] ? g_last_error : "CUDA error";
    case PCF_ENOMEM: return "out of memory";
    case PCF_ENAN: return "non-finite residual norm";
    case PCF_ETIMEOUT: return "bounded device wait timed out";
    case PCF_ENOTCONV: return "not converged";
    case PCF_ENOTSUP: return "not supported by this build";
  }
  return "unknown status";
}

long long pcf_state_len(int nx, int ny, int nz) {
  if (!grid_ok(nx, ny, nz)) return 0;
  const int Kx = nx / 3 - 1, Kz = nz / 3 - 1;
  return 3LL * (2 * Kx + 1) * (Kz + 1) * ny;
}

long long pcf_psi_len(int nx, int ny, int nz) {
  if (nx < 6 || nz < 6 || ny < 5) return 0;
  const int Kx = nx / 3 - 1, Kz = nz / 3 - 1;
  const long long indep = ((long long)(2 * Kx + 1) * (2 * Kz + 1) - 1) / 2;
  return indep * (2LL * (ny - 4) + 2LL * (ny - 2)) + 2LL * (ny - 2);
}

static bool params_ok(const pcf_params* prm) {
  return grid_ok(prm->nx, prm->ny, prm->nz) && prm->batch >= 1 && prm->Re > 0 && prm->dt > 0 &&
         prm->dtau_hat > 0 && prm->Lx > 0 && prm->Lz > 0 && prm->solve_kind >= 0 && prm->solve_kind <= 5 &&
         prm->modes_per_block >= 0 &&
         (prm->base_flow == PCF_COUETTE || prm->base_flow == PCF_POISEUILLE ||
          (prm->base_flow == PCF_ASBL && prm->suction_length > 0 && std::isfinite(prm->suction_length))) &&
         prm->symmetry >= 0 && prm->symmetry <= 3 && prm->plane_kernel >= 0 && prm->plane_kernel <= 1 &&
         prm->contraction_kernel >= 0 && prm->contraction_kernel <= 1 &&
         !((prm->symmetry & PCF_SYM_S1) && prm->base_flow != PCF_COUETTE);
}

// Device tables of one grid (shared by every instance on that grid).
struct GridTables {
  double *cheb, *rco, *ccw, *kx, *kz, *y, *ub, *tab0, *tab1, *dense0, *dense1;
  float2* cheb_ff = nullptr;
  double2 *twx, *twz, *tanx, *tanz;
  unsigned char *rotx, *rotz;
  float2 *twxf = nullptr, *twzf = nullptr;
  uint16_t* tcA = nullptr;
  uint16_t* tcA5 = nullptr;
  double sig[2];
};

static pcf_status build_tables(pcf_ctx* c, const pcf_params* prm, GridTables* g) {
  const int N = prm->ny - 1, nx = prm->nx, ny = prm->ny, nz = prm->nz;
  const int Kx = nx / 3 - 1, Kz = nz / 3 - 1, Mx = 2 * Kx + 1, Mz = Kz + 1;
  const double nu = 1.0 / prm->Re;
  std::vector<double> kx(Mx), kz(Mz), yg(ny);
  for (int i = 0; i < Mx; ++i) kx[i] = 2.0 * kPi * (i <= Kx ? i : i - Mx) / prm->Lx;
  for (int p = 0; p < Mz; ++p) kz[p] = 2.0 * kPi * p / prm->Lz;
  for (int j = 0; j < ny; ++j) yg[j] = cospi_frac(j, N);
  // base-flow profile U(y_j), U'(y_j) and the constant wall-normal velocity V (one explicit
  // fma, so every host rounds alike; the suction profile goes through the host's exp)
  std::vector<double> ub(3 * (size_t)ny, 0.0);
  for (int j = 0; j < ny; ++j) {
    const double y = yg[j];
    if (prm->base_flow == PCF_POISEUILLE) {
      ub[j] = std::fma(-y, y, 1.0);
      ub[ny + j] = -2.0 * y;
    } else if (prm->base_flow == PCF_ASBL) {
      const double d = prm->suction_length, e = std::exp(-(1.0 + y) / d);
      ub[j] = 1.0 - e;
      ub[ny + j] = e / d;
      ub[2 * ny + j] = -nu / d;
    } else {
      ub[j] = y;
      ub[ny + j] = 1.0;
    }
  }
  const std::vector<double> cheb = make_cheb(N), rco = make_rco(N), ccw = make_ccw(N);
  g->sig[0] = 1.0 / (nu * prm->dt);
  g->sig[1] = 1.0 / (nu * prm->dtau_hat);
  const std::vector<double> tab0 = make_mode_tables(N, kx, kz, g->sig[0], rco);
  const std::vector<double2> twx = make_twiddles(nx), twz = make_twiddles(nz);
  std::vector<double2> tanx, tanz;
  std::vector<unsigned char> rotx, rotz;
  make_tangent_twiddles(nx, &tanx, &rotx);
  make_tangent_twiddles(nz, &tanz, &rotz);
  if (upload(cheb, &g->cheb) || upload(rco, &g->rco) || upload(ccw, &g->ccw) || upload(kx, &g->kx) ||
      upload(kz, &g->kz) || upload(yg, &g->y) || upload(ub, &g->ub) || upload(twx, &g->twx) ||
      upload(twz, &g->twz) || upload(tab0, &g->tab0) || upload(tanx, &g->tanx) || upload(tanz, &g->tanz) ||
      upload(rotx, &g->rotx) || upload(rotz, &g->rotz))
    return PCF_ECUDA;
  for (void* p : {(void*)g->cheb, (void*)g->rco, (void*)g->ccw, (void*)g->kx, (void*)g->kz, (void*)g->y,
                  (void*)g->ub, (void*)g->twx, (void*)g->twz, (void*)g->tab0, (void*)g->tanx, (void*)g->tanz,
                  (void*)g->rotx, (void*)g->rotz})
    c->allocs.push_back(p);
  std::vector<double> tab1;
  if (prm->dtau_hat == prm->dt) {
    g->tab1 = g->tab0;
  } else {
    tab1 = make_mode_tables(N, kx, kz, g->sig[1], rco);
    if (upload(tab1, &g->tab1)) return PCF_ECUDA;
    c->allocs.push_back(g->tab1);
  }
  if (prm->precision == PCF_FLOAT_FLOAT) {
    // nearest float-float pairs: hi = fl(x), lo = fl(x - hi)
    std::vector<float2> cf(cheb.size());
    for (size_t i = 0; i < cheb.size(); ++i) {
      const float hi = static_cast<float>(cheb[i]);
      cf[i] = make_float2(hi, static_cast<float>(cheb[i] - (double)hi));
    }
    if (upload(cf, &g->cheb_ff)) return PCF_ECUDA;
    c->allocs.push_back(g->cheb_ff);
  }
  if (prm->precision == PCF_MIXED) {
    const std::vector<uint16_t> tcm = make_tc_matrices(N);
    if (upload(to_float2(twx), &g->twxf) || upload(to_float2(twz), &g->twzf) || upload(tcm, &g->tcA))
      return PCF_ECUDA;
    c->allocs.push_back(g->twxf);
    c->allocs.push_back(g->twzf);
    c->allocs.push_back(g->tcA);
    const std::vector<uint16_t> img = make_tc05_images(tcm, (ny + 15) & ~15);
    if (!img.empty()) {
      if (upload(img, &g->tcA5)) return PCF_ECUDA;
      c->allocs.push_back(g->tcA5);
    }
  }
  g->dense0 = g->dense1 = nullptr;
  const bool dense = N <= kDenseMaxN && prm->solve_kind != 1;
  if (dense) {
    if (upload(make_dense_tables(N, kx, kz, g->sig[0], rco, tab0), &g->dense0)) return PCF_ECUDA;
    c->allocs.push_back(g->dense0);
    if (prm->dtau_hat == prm->dt) {
      g->dense1 = g->dense0;
    } else {
      if (upload(make_dense_tables(N, kx, kz, g->sig[1], rco, tab1), &g->dense1)) return PCF_ECUDA;
      c->allocs.push_back(g->dense1);
    }
  }
  return PCF_OK;
}

static pcf_status upload_prefix(pcf_ctx* c, const std::vector<int>& per, int** dst, int* total) {
  std::vector<int> pre(per.size() + 1, 0);
  for (size_t b = 0; b < per.size(); ++b) pre[b + 1] = pre[b] + per[b];
  *total = pre.back();
  if (*dst) {
    PCF_CUDA(cudaMemcpy(*dst, pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice));
    return PCF_OK;
  }
  PCF_CUDA(upload(pre, dst));
  c->allocs.push_back(*dst);
  return PCF_OK;
}

// Mode tile of every instance (capped so the mode kernel's shared memory stays near 110 KB)
// and the derived launch geometry.
static pcf_status set_mode_tiles(pcf_ctx* c, int want) {
  std::vector<int> per(c->B);
  size_t sm = 0;
  for (int b = 0; b < c->B; ++b) {
    Inst& I = c->hinst[b];
    int mpc = want;
    while (mpc > 1 && smem_mode(I, mpc) > 110 * 1024) --mpc;
    if (smem_mode(I, mpc) > 227 * 1024) return PCF_ENOTSUP;
    I.mpc = mpc;
    per[b] = (I.nmodes + mpc - 1) / mpc;
    sm = std::max(sm, smem_mode(I, mpc));
  }
  c->mpc = want;
  c->sm_mode = sm;
  // threads per CTA: with the dense operators, one warp-padded pass over the solve's tasks
  // (two v rows, or two pairs of eta rows, per mode and parity group), 128 to 320 (the
  // kernel's launch bound)
  int thr = 128;
  for (int b = 0; b < c->B; ++b) {
    const Inst& I = c->hinst[b];
    if (!I.dense[0]) continue;
    const int Mh = I.N / 2 + 1, tasks = I.mpc * (2 * Mh + 2 * ((Mh + 1) / 2));
    thr = std::max(thr, std::min(320, (tasks + 31) / 32 * 32));
  }
  c->mode_thr = thr;
  PCF_TRY(upload_prefix(c, per, &c->pre_mode, &c->cta_mode));
  PCF_CUDA(raise_smem_limit((const void*)k_mode, c->sm_mode));
  return PCF_OK;
}

// Instance groups of the split mode kernels: runs of consecutive instances on the same grid,
// at most G per group, and the derived launch geometry.
// Consecutive instances that share grid and tables, at most G per group.
static std::vector<int2> make_groups(const pcf_ctx* c, int G) {
  std::vector<int2> groups;
  for (int b = 0; b < c->B; ++b) {
    const Inst& I = c->hinst[b];
    bool fresh = groups.empty() || groups.back().y == G;
    if (!fresh) {
      const Inst& P = c->hinst[b - 1];
      fresh = I.dense[0] != P.dense[0] || I.dense[1] != P.dense[1] || I.cheb != P.cheb || I.nmodes != P.nmodes;
    }
    if (fresh) groups.push_back(make_int2(b, 1)); else groups.back().y += 1;
  }
  return groups;
}

// Geometry of the split step's sweep solve with `threads` lanes per CTA (32 or 64): CTA
// prefixes over the instances for the full and the reduced launch, shared memory.
static pcf_status set_sweep(pcf_ctx* c, int threads) {
  std::vector<int> per(c->B), perr(c->B);
  int Nmax = 0;
  for (int b = 0; b < c->B; ++b) {
    const Inst& I = c->hinst[b];
    Nmax = std::max(Nmax, I.N);
    per[b] = sweep_ctas(I.nmodes, threads);
    perr[b] = sweep_ctas((I.Kx + 1) * I.Mz, threads);
  }
  const size_t sm = smem_sweep(Nmax, threads);
  if (sm > 227 * 1024) return PCF_ENOTSUP;
  PCF_TRY(upload_prefix(c, per, &c->pre_sw, &c->cta_sw));
  PCF_TRY(upload_prefix(c, perr, &c->pre_sw_r, &c->cta_sw_r));
  PCF_CUDA(set_sweep_smem(sm));
  c->thr_sw = threads;
  c->sm_sw = sm;
  return PCF_OK;
}

// Instance groups of the persistent Stokes solve (at most G instances each): items, prefix,
// shared-memory layout and grid.
static pcf_status set_solve_groups(pcf_ctx* c, int G) {
  int Nmax = 0;
  for (const Inst& I : c->hinst) Nmax = std::max(Nmax, I.N);
  G = std::max(1, std::min(G, split_max_group(Nmax)));
  while (G > 1 && smem_ysolve(Nmax, G) > 227 * 1024) --G;
  const std::vector<int2> groups = make_groups(c, G);
  const int ng = (int)groups.size();
  int gmax = 1;
  for (const int2& gq : groups) gmax = std::max(gmax, gq.y);
  std::vector<int> ps(ng + 1, 0), psr(ng + 1, 0);
  for (int q = 0; q < ng; ++q) {
    const Inst& I = c->hinst[groups[q].x];
    ps[q + 1] = ps[q] + split_ctas_per_group(1, I.nmodes, 1);
    psr[q + 1] = psr[q] + split_ctas_per_group(1, (I.Kx + 1) * I.Mz, 1);  // modes m >= 0
  }
  // the persistent solve lays out every item in buffers sized for the largest grid and group
  const size_t ss = smem_ysolve(Nmax, gmax);
  if (ss > 227 * 1024) return PCF_ENOTSUP;
  if (!c->d_groups_s) {
    if (ctx_alloc(c, &c->d_groups_s, (size_t)c->B) || ctx_alloc(c, &c->pre_ys, (size_t)c->B + 1) ||
        ctx_alloc(c, &c->pre_ys_r, (size_t)c->B + 1))
      return PCF_ENOMEM;
  }
  PCF_CUDA(cudaMemcpy(c->d_groups_s, groups.data(), sizeof(int2) * ng, cudaMemcpyHostToDevice));
  PCF_CUDA(cudaMemcpy(c->pre_ys, ps.data(), sizeof(int) * (ng + 1), cudaMemcpyHostToDevice));
  PCF_CUDA(cudaMemcpy(c->pre_ys_r, psr.data(), sizeof(int) * (ng + 1), cudaMemcpyHostToDevice));
  c->cta_ys_r = psr[ng];
  c->sgrp_s = G;
  c->ngroups_s = ng;
  c->cta_ys = ps[ng];
  c->sm_ys = ss;
  c->buf_ys = (int)ysolve_buffer(Nmax, gmax);
  c->rows_ys = Nmax / 2 + 1;
  PCF_CUDA(set_split_smem(c->sm_ya, ss, c->sm_yy));
  int dev = 0, nsm = 0;
  PCF_CUDA(cudaGetDevice(&dev));
  PCF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int per_sm = std::max(1, ysolve_ctas_per_sm(ss));
  c->grid_ys = std::min(c->cta_ys, nsm * per_sm);
  c->grid_ys_r = std::min(c->cta_ys_r, nsm * per_sm);
  return PCF_OK;
}

// Instance groups of the split analysis and synthesis (at most G instances each) with mt_a and
// mt_y consecutive modes per CTA (mt_y < 1: the same as mt_a); also resets the solve's groups.
static pcf_status set_split_groups(pcf_ctx* c, int G, int mt = 1, int mt_y = 0) {
  int Nmax = 0;
  for (const Inst& I : c->hinst) Nmax = std::max(Nmax, I.N);
  G = std::max(1, std::min(G, split_max_group(Nmax)));
  while (G > 1 && smem_ysolve(Nmax, G) > 227 * 1024) --G;
  std::vector<int2> groups = make_groups(c, G);
  const int ng = (int)groups.size();
  int gmax = 1;
  for (const int2& gq : groups) gmax = std::max(gmax, gq.y);
  mt = std::max(1, mt);
  while (mt > 1 && split_col_pad(gmax) * mt > 32) mt >>= 1;
  mt_y = mt_y < 1 ? mt : mt_y;
  while (mt_y > 1 && split_col_pad(gmax) * mt_y > 32) mt_y >>= 1;
  std::vector<int> pa(ng + 1, 0), py(ng + 1, 0), pf(ng + 1, 0), par(ng + 1, 0), pyr(ng + 1, 0);
  size_t sa = 0, sy = 0;
  int thr_a = 64, thr_y = 64;  // threads per CTA: one pass over the row tasks of any group
  for (int q = 0; q < ng; ++q) {
    const Inst& I = c->hinst[groups[q].x];
    const int nrun = (I.Kx + 1) * I.Mz;  // the reduced launches: modes m >= 0
    pf[q + 1] = pf[q] + I.nmodes;
    pa[q + 1] = pa[q] + split_ctas_per_group(0, I.nmodes, mt);
    py[q + 1] = py[q] + split_ctas_per_group(2, I.nmodes, mt_y);
    par[q + 1] = par[q] + split_ctas_per_group(0, nrun, mt);
    pyr[q + 1] = pyr[q] + split_ctas_per_group(2, nrun, mt_y);
    sa = std::max(sa, smem_yanalysis(I.N, groups[q].y, mt));
    sy = std::max(sy, smem_ysynth(I.N, groups[q].y, mt_y));
    const bool fp64 = c->plane_kind != 2;
    thr_a = std::max(thr_a, split_yanalysis_threads(I.N, groups[q].y, mt, fp64));
    thr_y = std::max(thr_y, split_ysynth_threads(I.N, groups[q].y, mt_y, fp64));
  }
  if (std::max(sa, sy) > 227 * 1024) return PCF_ENOTSUP;
  if (!c->d_groups) {
    if (ctx_alloc(c, &c->d_groups, (size_t)c->B) || ctx_alloc(c, &c->pre_ya, (size_t)c->B + 1) ||
        ctx_alloc(c, &c->pre_yy, (size_t)c->B + 1) || ctx_alloc(c, &c->pre_yf, (size_t)c->B + 1) ||
        ctx_alloc(c, &c->pre_ya_r, (size_t)c->B + 1) || ctx_alloc(c, &c->pre_yy_r, (size_t)c->B + 1))
      return PCF_ENOMEM;
  }
  PCF_CUDA(cudaMemcpy(c->pre_ya_r, par.data(), sizeof(int) * (ng + 1), cudaMemcpyHostToDevice));
  PCF_CUDA(cudaMemcpy(c->pre_yy_r, pyr.data(), sizeof(int) * (ng + 1), cudaMemcpyHostToDevice));
  c->cta_ya_r = par[ng];
  c->cta_yy_r = pyr[ng];
  PCF_CUDA(cudaMemcpy(c->pre_yf, pf.data(), sizeof(int) * (ng + 1), cudaMemcpyHostToDevice));
  c->cta_yf = pf[ng];
  c->sm_yf = smem_ystep(Nmax, gmax);
  PCF_CUDA(cudaMemcpy(c->d_groups, groups.data(), sizeof(int2) * ng, cudaMemcpyHostToDevice));
  PCF_CUDA(cudaMemcpy(c->pre_ya, pa.data(), sizeof(int) * (ng + 1), cudaMemcpyHostToDevice));
  PCF_CUDA(cudaMemcpy(c->pre_yy, py.data(), sizeof(int) * (ng + 1), cudaMemcpyHostToDevice));
  c->sgrp = G;
  c->smt = mt;
  c->smt_y = mt_y;
  c->ngroups = ng;
  c->cta_ya = pa[ng];
  c->cta_yy = py[ng];
  c->sm_ya = sa;
  c->sm_yy = sy;
  c->thr_ya = thr_a;
  c->thr_yy = thr_y;
  if (c->sm_yf <= 227 * 1024) PCF_CUDA(set_ystep_smem(c->sm_yf));
  // the solve follows the same group size unless tuned on its own (autotune_split)
  return set_solve_groups(c, G);
}

// Autotuner of the split mode kernels: time the per-mode work of a whole step (analysis,
// solve and synthesis of both half-steps, or the fused kernel twice and the norm kernel) on
// the batch for each candidate group size, mode tile and organisation, and keep the fastest.
static pcf_status autotune_split(pcf_ctx* c) {
  const int cand[] = {1, 2, 4, 6, 8};
  cudaEvent_t a, b;
  PCF_CUDA(cudaEventCreate(&a));
  PCF_CUDA(cudaEventCreate(&b));
  int best = 2, best_mt = 1;
  bool best_fused = false;
  float best_ms = 1e30f;
  int last = 0;
  for (int G0 : cand) {
    const int G = std::min(G0, c->B);
    if (G == last) continue;
    last = G;
    for (int mt = 1; mt <= 16 && split_col_pad(G) * mt <= 32; mt *= 2) {
      if (set_split_groups(c, G, mt) != PCF_OK || c->sgrp != G || c->smt != mt) continue;
      for (int fuse = 0; fuse < 2; ++fuse) {
        if (fuse && (mt > 1 || c->sm_yf > 227 * 1024)) continue;  // the fused kernel has no mode tile
        if (((c->prm.solve_kind == 3 || c->prm.solve_kind == 5) && fuse) || (c->prm.solve_kind == 4 && !fuse))
          continue;
        // the per-mode work of a whole step in each organisation (both half-steps; the fused
        // path also launches the separate norm kernel)
        auto seq = [&] {
          if (fuse) {
            launch_ystep(c->cta_yf, c->sm_yf, c->cs, gl_of(c, c->pre_yf), MODE_PHI);
            launch_jnorm(c->B, c->cs, c->dinst, 0);
            launch_ystep(c->cta_yf, c->sm_yf, c->cs, gl_of(c, c->pre_yf), MODE_PSI_UPDATE);
            return;
          }
          for (int op : {(int)MODE_PHI, (int)MODE_PSI_UPDATE}) {
            launch_yanalysis(c->cta_ya, c->thr_ya, c->sm_ya, c->cs, gl_of(c, c->pre_ya), op, c->plane_kind == 2,
                             c->smt);
            launch_ysolve(c->grid_ys, c->cta_ys, c->buf_ys, c->rows_ys, c->sm_ys, c->cs, gl_solve(c), op);
            launch_ysynth_split(c->cta_yy, c->thr_yy, c->sm_yy, c->cs, gl_of(c, c->pre_yy), op == MODE_PHI ? 1 : 0, 1,
                                c->plane_kind == 2, c->smt_y);
          }
        };
        seq();
        PCF_CUDA(cudaEventRecord(a, c->cs));
        for (int r = 0; r < 3; ++r) seq();
        PCF_CUDA(cudaEventRecord(b, c->cs));
        PCF_CUDA(cudaEventSynchronize(b));
        float ms = 0.f;
        PCF_CUDA(cudaEventElapsedTime(&ms, a, b));
        if (ms < best_ms) {
          best_ms = ms;
          best = G;
          best_mt = mt;
          best_fused = fuse != 0;
        }
      }
    }
  }
  c->tuned_split_ms = best_ms / 3.0;
  pcf_status st = set_split_groups(c, best, best_mt);
  c->fused = st == PCF_OK && best_fused;
  if (st == PCF_OK && !c->fused) {
    // analysis and synthesis mode tiles, each timed alone
    auto time5 = [&](auto&& launch, float* ms) -> pcf_status {
      launch();
      PCF_CUDA(cudaEventRecord(a, c->cs));
      for (int r = 0; r < 5; ++r) launch();
      PCF_CUDA(cudaEventRecord(b, c->cs));
      PCF_CUDA(cudaEventSynchronize(b));
      PCF_CUDA(cudaEventElapsedTime(ms, a, b));
      return PCF_OK;
    };
    int mt_a = best_mt, mt_y = best_mt;
    float ba = 1e30f, by = 1e30f;
    for (int mt = 1; mt <= 16 && split_col_pad(best) * mt <= 32; mt *= 2) {
      if (set_split_groups(c, best, mt, mt) != PCF_OK || c->smt != mt || c->smt_y != mt) continue;
      float ms = 0.f;
      PCF_TRY(time5([&] {
        launch_yanalysis(c->cta_ya, c->thr_ya, c->sm_ya, c->cs, gl_of(c, c->pre_ya), MODE_PHI, c->plane_kind == 2,
                         c->smt);
      }, &ms));
      if (ms < ba) { ba = ms; mt_a = mt; }
      PCF_TRY(time5([&] {
        launch_ysynth_split(c->cta_yy, c->thr_yy, c->sm_yy, c->cs, gl_of(c, c->pre_yy), 1, 1, c->plane_kind == 2,
                            c->smt_y);
      }, &ms));
      if (ms < by) { by = ms; mt_y = mt; }
    }
    st = set_split_groups(c, best, mt_a, mt_y);
  }
  float solve_ms = 1e30f;  // five dense solves in the chosen groups
  if (st == PCF_OK && !c->fused) {
    // the solve alone over its own group sizes
    int best_s = c->sgrp_s;
    float best_s_ms = 1e30f;
    last = 0;
    for (int G0 : {1, 2, 4, 8}) {
      const int G = std::min(G0, c->B);
      if (G == last) continue;
      last = G;
      if (set_solve_groups(c, G) != PCF_OK || c->sgrp_s != G) continue;
      auto seq = [&] {
        launch_ysolve(c->grid_ys, c->cta_ys, c->buf_ys, c->rows_ys, c->sm_ys, c->cs, gl_solve(c), MODE_PHI);
      };
      seq();
      PCF_CUDA(cudaEventRecord(a, c->cs));
      for (int r = 0; r < 5; ++r) seq();
      PCF_CUDA(cudaEventRecord(b, c->cs));
      PCF_CUDA(cudaEventSynchronize(b));
      float ms = 0.f;
      PCF_CUDA(cudaEventElapsedTime(&ms, a, b));
      if (ms < best_s_ms) {
        best_s_ms = ms;
        best_s = G;
      }
    }
    st = set_solve_groups(c, best_s);
    solve_ms = best_s_ms;
  }
  c->sweep = false;
  if (st == PCF_OK && !c->fused && c->prm.solve_kind != 3) {
    // the banded sweeps, one thread per chain, against the dense solve (solve_kind 5: always)
    int best_t = 0;
    float best_t_ms = c->prm.solve_kind == 5 ? 1e30f : solve_ms;
    for (int thr : {32, 64}) {
      if (set_sweep(c, thr) != PCF_OK) continue;
      auto seq = [&] {
        launch_sweep(c->cta_sw, c->thr_sw, c->sm_sw, c->cs, LaunchInfo{c->dinst, c->pre_sw, c->B}, MODE_PHI, 0);
      };
      seq();
      PCF_CUDA(cudaEventRecord(a, c->cs));
      for (int r = 0; r < 5; ++r) seq();
      PCF_CUDA(cudaEventRecord(b, c->cs));
      PCF_CUDA(cudaEventSynchronize(b));
      float ms = 0.f;
      PCF_CUDA(cudaEventElapsedTime(&ms, a, b));
      if (ms < best_t_ms) {
        best_t_ms = ms;
        best_t = thr;
      }
    }
    if (best_t > 0) {
      st = set_sweep(c, best_t);
      c->sweep = st == PCF_OK;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return st;
}

// Time the Stokes-step mode kernel on the batch for each candidate tile; keep the fastest.
static pcf_status time_mode_tiles(pcf_ctx* c, cudaEvent_t a, cudaEvent_t b, int* best, float* best_ms) {
  const int cand[] = {1, 2, 3, 4, 6, 8};
  *best = 4;
  *best_ms = 1e30f;
  for (int mpc : cand) {
    if (set_mode_tiles(c, mpc) != PCF_OK) continue;
    PCF_TRY(push_descriptors(c));
    k_mode<<<c->cta_mode, c->mode_thr, c->sm_mode, c->cs>>>(li_of(c, c->pre_mode), MODE_PHI, 0, mpc, 0);
    PCF_CUDA(cudaEventRecord(a, c->cs));
    for (int r = 0; r < 3; ++r)
      k_mode<<<c->cta_mode, c->mode_thr, c->sm_mode, c->cs>>>(li_of(c, c->pre_mode), MODE_PHI, 0, mpc, 0);
    PCF_CUDA(cudaEventRecord(b, c->cs));
    PCF_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    PCF_CUDA(cudaEventElapsedTime(&ms, a, b));
    if (ms < *best_ms) {
      *best_ms = ms;
      *best = mpc;
    }
  }
  return PCF_OK;
}

// Autotuner (laminar input): the mode tile and, for the mixed-precision form, the Stokes
// solve variant.  The dense per-mode operators keep the FP64 pipe full; the banded sweeps
// need ~20x fewer FP64 operations but run as sequential chains and no operator tables stream
// from memory; which one is faster depends on the grid and the batch, so both are timed.
static pcf_status autotune_tiles(pcf_ctx* c) {
  double2* z = nullptr;
  PCF_CUDA(cudaMalloc(&z, sizeof(double2) * (size_t)c->total_state));
  PCF_CUDA(cudaMemset(z, 0, sizeof(double2) * (size_t)c->total_state));
  set_pointers(c, (const double*)z, (const double*)c->r_int, nullptr);
  PCF_TRY(push_descriptors(c));
  cudaEvent_t a, b;
  PCF_CUDA(cudaEventCreate(&a));
  PCF_CUDA(cudaEventCreate(&b));
  int best = 4;
  float best_ms = 1e30f;
  PCF_TRY(time_mode_tiles(c, a, b, &best, &best_ms));
  if (c->mixed && c->hinst[0].dense[0]) {
    std::vector<const double*> saved;
    for (Inst& I : c->hinst) {
      saved.push_back(I.dense[0]);
      saved.push_back(I.dense[1]);
      I.dense[0] = I.dense[1] = nullptr;
    }
    int best2 = 4;
    float ms2 = 1e30f;
    PCF_TRY(time_mode_tiles(c, a, b, &best2, &ms2));
    if (ms2 < best_ms) {
      best = best2;
      best_ms = ms2;
    } else {
      for (size_t i = 0; i < c->hinst.size(); ++i) {
        c->hinst[i].dense[0] = saved[2 * i];
        c->hinst[i].dense[1] = saved[2 * i + 1];
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  c->tuned_ms = best_ms / 3.0;
  pcf_status st = set_mode_tiles(c, best);
  if (st == PCF_OK && c->split) {
    st = push_descriptors(c);
    if (st == PCF_OK) st = autotune_split(c);
  }
  if (cudaStreamSynchronize(c->cs) != cudaSuccess && st == PCF_OK) st = PCF_ECUDA;
  cudaFree(z);
  return st;
}

static pcf_status create_batch(const pcf_params* list, int nlist, void* stream, pcf_ctx** out) {
  if (!list || nlist < 1 || !out) return PCF_EINVAL;
  int B = 0;
  for (int k = 0; k < nlist; ++k) {
    if (!params_ok(&list[k])) return PCF_EINVAL;
    if (list[k].precision != PCF_FP64 && list[k].precision != PCF_MIXED && list[k].precision != PCF_FLOAT_FLOAT)
      return PCF_ENOTSUP;
    if (list[k].precision != list[0].precision) return PCF_EINVAL;
    if (list[k].precision == PCF_MIXED && list[k].ny > 113) return PCF_ENOTSUP;
    B += list[k].batch;
  }
  pcf_ctx* c = new pcf_ctx();
  c->prm = list[0];
  c->prm.batch = B;
  c->N = list[0].ny - 1;
  c->Kx = list[0].nx / 3 - 1;
  c->Kz = list[0].nz / 3 - 1;
  c->Mx = 2 * c->Kx + 1;
  c->Mz = c->Kz + 1;
  c->nm = c->Mx * c->Mz;
  c->B = B;
  c->state_len = 3LL * c->nm * list[0].ny;
  c->user = (cudaStream_t)stream;
  c->mixed = list[0].precision == PCF_MIXED;
  c->plane_kind = c->mixed ? 1 : list[0].precision == PCF_FLOAT_FLOAT ? 2 : 0;
  auto fail = [&](pcf_status s) {
    pcf_destroy(c);
    return s;
  };
  if (cudaStreamCreateWithFlags(&c->cs, cudaStreamNonBlocking) != cudaSuccess) return fail(PCF_ECUDA);
  if (cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) != cudaSuccess) return fail(PCF_ECUDA);
  if (cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess) return fail(PCF_ECUDA);

  // one table set per distinct problem
  std::vector<GridTables> gts;
  std::vector<int> grid_of(nlist);
  c->uniform = true;
  for (int k = 0; k < nlist; ++k) c->suction = c->suction || list[k].base_flow == PCF_ASBL;
  for (int k = 0; k < nlist; ++k) {
    int found = -1;
    for (int q = 0; q < k; ++q) {
      const pcf_params &a = list[k], &p = list[q];
      if (a.nx == p.nx && a.ny == p.ny && a.nz == p.nz && a.Lx == p.Lx && a.Lz == p.Lz && a.Re == p.Re &&
          a.dt == p.dt && a.dtau_hat == p.dtau_hat && a.solve_kind == p.solve_kind && a.base_flow == p.base_flow &&
          (a.base_flow != PCF_ASBL || a.suction_length == p.suction_length)) {
        found = grid_of[q];
        break;
      }
    }
    if (found < 0) {
      GridTables g;
      pcf_status st = build_tables(c, &list[k], &g);
      if (st != PCF_OK) return fail(st);
      gts.push_back(g);
      found = (int)gts.size() - 1;
    }
    grid_of[k] = found;
    if (found != 0) c->uniform = false;
  }

  // per-instance workspace, one allocation per buffer kind
  size_t n_yv = 0, n_ph = 0, n_xz = 0, n_np = 0, n_fr = 0;
  c->state_off.assign(B + 1, 0);
  {
    int b = 0;
    for (int k = 0; k < nlist; ++k)
      for (int r = 0; r < list[k].batch; ++r, ++b) {
        const pcf_params& p = list[k];
        const long long nm = (long long)(2 * (p.nx / 3 - 1) + 1) * (p.nz / 3);
        n_yv += 2ULL * kFieldsY * p.ny * nm;
        n_ph += 2ULL * kFieldsSynth * p.ny * p.nx * p.nz;
        n_xz += 3ULL * p.ny * nm;
        n_np += 3ULL * p.ny;
        n_fr += 6ULL * (p.ny + 1) * nm;
        c->state_off[b + 1] = c->state_off[b] + 3LL * nm * p.ny;
      }
  }
  c->total_state = c->state_off[B];
  double2 *yv = nullptr, *xz = nullptr;
  double *ph = nullptr, *np = nullptr, *fr = nullptr;
  float2 *yvf = nullptr, *xzf = nullptr, *xzc = nullptr;
  float* phf = nullptr;
  int* jc = nullptr;
  if (ctx_alloc(c, &np, n_np) || ctx_alloc(c, &c->r_int, (size_t)c->total_state) ||
      ctx_alloc(c, &c->active, (size_t)B) || ctx_alloc(c, &jc, (size_t)B))
    return fail(PCF_ENOMEM);
  if (cudaMemset(jc, 0, sizeof(int) * B) != cudaSuccess) return fail(PCF_ECUDA);
  if (c->mixed) {
    if (ctx_alloc(c, &yvf, n_yv) || ctx_alloc(c, &phf, n_ph) || ctx_alloc(c, &xzf, n_xz) || ctx_alloc(c, &xzc, n_xz))
      return fail(PCF_ENOMEM);
  } else {
    if (ctx_alloc(c, &yv, n_yv) || ctx_alloc(c, &ph, n_ph) || ctx_alloc(c, &xz, n_xz) || ctx_alloc(c, &fr, n_fr))
      return fail(PCF_ENOMEM);
  }
  c->hinst.resize(B);
  std::vector<int> per11(B), per3(B), per1(B, 1), per_tcs(B), per_tca(B);
  size_t o_yv = 0, o_ph = 0, o_xz = 0, o_np = 0, o_fr = 0;
  c->split = !c->mixed;
  // the FP32 form's plane kernels keep their transforms in warp registers wherever every
  // instance's nx and nz allow it (unless the caller asks for the shared-memory kernels)
  c->plane_warp = c->mixed && list[0].plane_kernel != 1;
  // the tcgen05 contraction holds the whole padded matrix in one 128-row MMA tile (the mixed
  // form's ny <= 113 keeps it there)
  c->tc05 = c->mixed && list[0].contraction_kernel != 1;
  for (int k = 0; k < nlist; ++k)
    if (((list[k].ny + 15) & ~15) > 128) c->tc05 = false;
  // symmetric descent on the modes m >= 0 when every instance enforces s2 (split kernels)
  c->reduced = true;
  for (int k = 0; k < nlist; ++k)
    if (!(list[k].symmetry & PCF_SYM_S2)) c->reduced = false;
  int b = 0;
  for (int k = 0; k < nlist; ++k)
    for (int r = 0; r < list[k].batch; ++r, ++b) {
      const pcf_params& p = list[k];
      const GridTables& g = gts[grid_of[k]];
      Inst& I = c->hinst[b];
      memset(&I, 0, sizeof(I));
      I.nx = p.nx; I.ny = p.ny; I.nz = p.nz; I.N = p.ny - 1;
      I.Kx = p.nx / 3 - 1; I.Kz = p.nz / 3 - 1; I.Mx = 2 * I.Kx + 1; I.Mz = I.Kz + 1;
      I.nmodes = I.Mx * I.Mz;
      radix_plan(p.nx, I.rx, &I.nrx);
      radix_plan(p.nz, I.rz, &I.nrz);
      I.nu = 1.0 / p.Re; I.dt = p.dt; I.dtau_hat = p.dtau_hat; I.dtau = 0.0;
      I.inv_nu = 1.0 / I.nu; I.inv_dt = 1.0 / I.dt; I.inv_dtau_hat = 1.0 / I.dtau_hat;
      I.inv_nxnz = 1.0 / ((double)p.nx * p.nz);
      I.cheb = g.cheb; I.cheb_ff = g.cheb_ff; I.rco = g.rco; I.ygrid = g.y; I.ubase = g.ub; I.ccw = g.ccw;
      I.kx = g.kx; I.kz = g.kz;
      I.twx = g.twx; I.twz = g.twz;
      I.tanx = g.tanx; I.tanz = g.tanz; I.rotx = g.rotx; I.rotz = g.rotz;
      I.tab[0] = g.tab0; I.tab[1] = g.tab1;
      I.dense[0] = g.dense0; I.dense[1] = g.dense1;
      I.sigma[0] = g.sig[0]; I.sigma[1] = g.sig[1];
      I.normpart = np + o_np;
      I.jcount = jc + b;
      if (c->mixed) {
        I.yvf = yvf + o_yv; I.physf = phf + o_ph; I.xzf = xzf + o_xz; I.xzc = xzc + o_xz;
        I.twxf = g.twxf; I.twzf = g.twzf; I.tcA = g.tcA; I.tcA5 = g.tcA5; I.mixed = 1;
      } else {
        I.yv = yv + o_yv; I.phys = ph + o_ph; I.xz = xz + o_xz; I.frg = fr + o_fr;
      }
      if (!I.dense[0] || !I.dense[1] || p.solve_kind == 2 || smem_ysolve(I.N, 1) > 227 * 1024) c->split = false;
      o_yv += 2ULL * kFieldsY * p.ny * I.nmodes;
      o_ph += 2ULL * kFieldsSynth * p.ny * p.nx * p.nz;
      o_xz += 3ULL * p.ny * I.nmodes;
      o_np += 3ULL * p.ny;
      o_fr += 6ULL * (p.ny + 1) * I.nmodes;
      I.hist_stride = B;
      I.sym = p.symmetry;
      if (p.symmetry) c->any_sym = true;
      c->sym_ctas = std::max(c->sym_ctas, symmetrize_ctas(I));
      c->dns_ctas = std::max(c->dns_ctas, dns_ctas(I));
      per11[b] = kFieldsSynth * p.ny;
      per3[b] = 3 * p.ny;
      per_tcs[b] = kFieldsY * cheb_tc_tiles(I.nmodes);
      per_tca[b] = 3 * cheb_tc_tiles(I.nmodes);
      const int elem = c->mixed ? (int)sizeof(float2) : (int)sizeof(double2);
      if (!plane_warp_ok(I)) c->plane_warp = false;
      c->sm_synth = std::max(c->sm_synth, smem_plane(I, elem));
      c->sm_prod = std::max(c->sm_prod, smem_plane(I, elem));
      c->sm_warp = std::max(c->sm_warp, smem_plane_warp(I, elem));
      if (c->mixed) c->sm_tc = std::max(c->sm_tc, c->tc05 ? smem_cheb_tc05(p.ny) : smem_cheb_tc(p.ny));
    }
  if (ctx_alloc(c, &c->dinst, (size_t)B)) return fail(PCF_ENOMEM);
  int dummy;
  pcf_status st;
  if ((st = upload_prefix(c, per11, &c->pre_synth11, &c->cta_synth11)) != PCF_OK ||
      (st = upload_prefix(c, per3, &c->pre_synth3, &c->cta_synth3)) != PCF_OK ||
      (st = upload_prefix(c, per3, &c->pre_prod, &c->cta_prod)) != PCF_OK ||
      (st = upload_prefix(c, per1, &c->pre_inst, &dummy)) != PCF_OK ||
      (st = upload_prefix(c, per_tcs, &c->pre_tcs, &c->cta_tcs)) != PCF_OK ||
      (st = upload_prefix(c, per_tca, &c->pre_tca, &c->cta_tca)) != PCF_OK)
    return fail(st);
  if (c->mixed && (c->tc05 ? set_cheb_tc05_smem(c->sm_tc) : set_cheb_tc_smem(c->sm_tc))) return fail(PCF_ECUDA);
  if (c->plane_warp) {
    c->sm_synth = c->sm_prod = c->sm_warp;
    if (set_plane_warp_smem(c->sm_synth, c->sm_prod)) return fail(PCF_ECUDA);
  } else if (set_plane_smem(c->plane_kind, c->sm_synth, c->sm_prod)) {
    return fail(PCF_ECUDA);
  }
  const int want = list[0].modes_per_block;
  st = want > 0 ? set_mode_tiles(c, want) : autotune_tiles(c);
  if (st == PCF_OK && want > 0 && c->split) {
    st = set_split_groups(c, want);
    c->fused = st == PCF_OK && c->prm.solve_kind == 4 && c->sm_yf <= 227 * 1024;
    if (st == PCF_OK && c->prm.solve_kind == 5) {
      st = set_sweep(c, 32);
      c->sweep = st == PCF_OK;
    }
  }
  if (st != PCF_OK) return fail(st);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(PCF_ECUDA);
  *out = c;
  return PCF_OK;
}

pcf_status pcf_create(const pcf_params* prm, void* stream, pcf_ctx** out) {
  if (!prm || !out) return PCF_EINVAL;
  return create_batch(prm, 1, stream, out);
}

pcf_status pcf_batch_create(const pcf_params* list, int n, void* stream, pcf_ctx** out) {
  return create_batch(list, n, stream, out);
}

long long pcf_state_offset(const pcf_ctx* c, int instance) {
  if (!c || instance < 0 || instance > c->B) return -1;
  return c->state_off[instance];
}

int pcf_mode_tile(const pcf_ctx* c) { return c ? (c->split ? c->sgrp : c->mpc) : 0; }

int pcf_plane_variant(const pcf_ctx* c) { return c ? (c->plane_warp ? 1 : 0) : -1; }

int pcf_contraction_variant(const pcf_ctx* c) { return c ? (c->tc05 ? 1 : 0) : -1; }

int pcf_symmetric_modes(const pcf_ctx* c) {
  if (!c) return -1;
  return c->reduced && c->split && !c->fused ? (c->Kx + 1) * c->Mz : c->Mx * c->Mz;
}

int pcf_solve_variant(const pcf_ctx* c) {
  if (!c) return -1;
  if (c->split) return c->fused ? 3 : (c->sweep ? 4 : 2);
  return c->hinst[0].dense[0] ? 1 : 0;
}

void pcf_destroy(pcf_ctx* c) {
  if (!c) return;
  if (c->cs) cudaStreamSynchronize(c->cs);
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  for (auto& kv : c->dns_graphs) cudaGraphExecDestroy(kv.second);
  for (void* p : c->allocs) cudaFree(p);
  if (c->u_dev) cudaFree(c->u_dev);
  if (c->hist_dev) cudaFree(c->hist_dev);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->cs) cudaStreamDestroy(c->cs);
  delete c;
}

pcf_status pcf_residual(pcf_ctx* c, const double* u, double* r, double* rnorm) {
  if (!c || !u || !r) return PCF_EINVAL;
  set_pointers(c, u, r, nullptr);
  PCF_TRY(enter(c));
  PCF_TRY(push_descriptors(c));
  PCF_TRY(launch_ysynth(c, 0));
  PCF_TRY(launch_synth(c, 0, kFieldsSynth));
  PCF_TRY(launch_prodM(c));
  if (c->mixed) PCF_TRY(launch_tc_analysis(c));
  PCF_TRY(launch_mode(c, MODE_PHI, 0, 0));
  if (rnorm) {
    if (c->mixed) PCF_TRY(launch_tc_synth(c, 1));
    PCF_TRY(launch_synth(c, 1, 3));
    launch_norm_planes(c->plane_kind, c->cta_synth3, c->cs, li_of(c, c->pre_synth3), 1);
    k_norm_final<<<1, 32, 0, c->cs>>>(li_of(c, c->pre_inst), rnorm);
  }
  PCF_TRY(check_launch());
  return leave(c);
}

pcf_status pcf_adjoint_gradient(pcf_ctx* c, const double* u, const double* r, double* f) {
  if (!c || !u || !r || !f) return PCF_EINVAL;
  set_pointers(c, u, r, f);
  PCF_TRY(enter(c));
  PCF_TRY(push_descriptors(c));
  PCF_TRY(launch_ysynth(c, 0));
  PCF_TRY(launch_ysynth(c, 1));
  PCF_TRY(launch_synth(c, 0, kFieldsSynth));
  PCF_TRY(launch_synth(c, 1, kFieldsSynth));
  PCF_TRY(launch_prodN(c));
  if (c->mixed) PCF_TRY(launch_tc_analysis(c));
  PCF_TRY(launch_mode(c, MODE_PSI_GRAD, 1, 0));
  PCF_TRY(check_launch());
  return leave(c);
}

pcf_status pcf_influence_matrix_solve(pcf_ctx* c, const double* rhs, double* out, double step) {
  if (!c || !rhs || !out) return PCF_EINVAL;
  int sig;
  if (step == c->prm.dt) sig = 0;
  else if (step == c->prm.dtau_hat) sig = 1;
  else return PCF_EINVAL;
  set_pointers(c, nullptr, rhs, out);
  PCF_TRY(enter(c));
  PCF_TRY(push_descriptors(c));
  PCF_TRY(launch_mode(c, MODE_SOLVE, sig, 0));
  PCF_TRY(check_launch());
  return leave(c);
}

static pcf_status descent_internal(pcf_ctx* c, double* u, double dtau, int nsteps, double* hist, double tol) {
  if (!c || !u || nsteps < 0 || !(dtau >= 0)) return PCF_EINVAL;
  if (nsteps == 0) return PCF_OK;
  set_pointers(c, u, (const double*)c->r_int, nullptr);
  for (int b = 0; b < c->B; ++b) {
    c->hinst[b].dtau = dtau;
    c->hinst[b].hist = hist ? hist + b : nullptr;
    if (tol > 0.0) {
      c->hinst[b].tol = tol;
      c->hinst[b].active = c->active + b;
    }
  }
  PCF_TRY(enter(c));
  PCF_TRY(push_descriptors(c));
  if (c->any_sym) PCF_TRY(launch_sym(c, -1));  // the run starts in the symmetric subspace
  if (c->timing) {
    PCF_TRY(launch_ysynth(c, 0));
    for (int s = 0; s < nsteps; ++s) PCF_TRY(step_body(c, s));
    PCF_TRY(check_launch());
    return leave(c);
  }
  auto it = c->graphs.find(nsteps);
  if (it == c->graphs.end()) {
    cudaGraph_t g;
    PCF_CUDA(cudaStreamBeginCapture(c->cs, cudaStreamCaptureModeThreadLocal));
    pcf_status st = launch_ysynth(c, 0);
    for (int s = 0; s < nsteps && st == PCF_OK; ++s) st = step_body(c, s);
    cudaError_t e = cudaStreamEndCapture(c->cs, &g);
    if (st != PCF_OK) return st;
    PCF_CUDA(e);
    cudaGraphExec_t ex;
    PCF_CUDA(cudaGraphInstantiate(&ex, g, 0));
    cudaGraphDestroy(g);
    it = c->graphs.emplace(nsteps, ex).first;
  }
  PCF_CUDA(cudaGraphLaunch(it->second, c->cs));
  return leave(c);
}

pcf_status pcf_descent_step(pcf_ctx* c, double* u, double dtau, int nsteps, double* hist) {
  return descent_internal(c, u, dtau, nsteps, hist, 0.0);
}

// Descent in chunks with convergence masks and the DMD schedule of §6.2 (see pcf_run_schedule).
static pcf_status run_schedule(pcf_ctx* c, double* u, double dtau, int max_steps, double tol,
                               const pcf_dmd_schedule* sc, int* steps_out, double* j_out, int* dmd_jumps) {
  if (!c || !u || max_steps < 1 || !(tol > 0) || !(dtau > 0)) return PCF_EINVAL;
  const bool dmd = sc != nullptr;
  if (dmd && (sc->snapshots < 3 || sc->spacing < 1 || sc->gap < 0 || !(sc->rank_tol > 0) || std::isnan(sc->j_start)))
    return PCF_EINVAL;
  if (dmd && !c->uniform) return PCF_ENOTSUP;
  const int B = c->B;
  const int chunk = dmd ? sc->spacing : 100;
  const int S = dmd ? sc->snapshots : 0;
  const int gap_chunks = dmd ? (sc->gap + chunk - 1) / chunk : 0;
  const long long plen = pcf_psi_len(c->prm.nx, c->prm.ny, c->prm.nz);
  const int sub = std::min(chunk, 256);  // steps per captured graph
  double *ring = nullptr, *tmp = nullptr, *ordered = nullptr, *hist = nullptr;
  auto release = [&] {
    if (hist) cudaFree(hist);
    if (ring) cudaFree(ring);
    if (tmp) cudaFree(tmp);
    if (ordered) cudaFree(ordered);
  };
  if (cudaMalloc(&hist, sizeof(double) * (size_t)chunk * B) != cudaSuccess) return PCF_ENOMEM;
  if (dmd && (cudaMalloc(&ring, sizeof(double) * (size_t)S * B * plen) != cudaSuccess ||
              cudaMalloc(&tmp, sizeof(double) * (size_t)B * plen) != cudaSuccess ||
              cudaMalloc(&ordered, sizeof(double) * (size_t)S * plen) != cudaSuccess)) {
    release();
    return PCF_ENOMEM;
  }
  enum { FIRST = 0, COLLECT = 1, GAP = 2 };
  std::vector<int> ones(B, 1), steps(B, 0), done(B, 0), phase(B, FIRST), wait(B, 0), filled(B, 0), next(B, 0);
  std::vector<double> J(B, NAN), hh((size_t)chunk * B);
  int jumps = 0;
  auto finish = [&](pcf_status st) {
    cudaStreamSynchronize(c->user);
    release();
    for (int b = 0; b < B; ++b) {
      if (steps_out) steps_out[b] = done[b] == 1 ? steps[b] : -1;
      if (j_out) j_out[b] = J[b];
    }
    if (dmd_jumps) *dmd_jumps = jumps;
    return st;
  };
  if (cudaMemcpyAsync(c->active, ones.data(), sizeof(int) * B, cudaMemcpyHostToDevice, c->user) != cudaSuccess)
    return finish(PCF_ECUDA);
  const size_t pbytes = sizeof(double) * (size_t)plen;
  int taken = 0;
  while (taken < max_steps) {
    const int n = std::min(chunk, max_steps - taken);
    for (int o = 0; o < n; o += sub) {
      const pcf_status st = descent_internal(c, u, dtau, std::min(sub, n - o), hist + (size_t)o * B, tol);
      if (st != PCF_OK) return finish(st);
    }
    if (cudaMemcpyAsync(hh.data(), hist, sizeof(double) * (size_t)n * B, cudaMemcpyDeviceToHost, c->user) !=
            cudaSuccess ||
        cudaStreamSynchronize(c->user) != cudaSuccess)
      return finish(PCF_ECUDA);
    int alive = 0;
    for (int b = 0; b < B; ++b) {
      if (done[b]) continue;
      for (int s = 0; s < n; ++s) {
        const double v = hh[(size_t)s * B + b];
        J[b] = v;
        if (!std::isfinite(v)) { done[b] = 2; break; }
        if (v < tol) { done[b] = 1; steps[b] = taken + s; break; }
      }
      if (!done[b]) ++alive;
    }
    taken += n;
    if (!alive) break;
    if (!dmd) continue;
    bool snap = false;
    for (int b = 0; b < B; ++b) snap = snap || (!done[b] && phase[b] != GAP);
    if (snap) {
      const pcf_status st = pcf_snapshot(c, u, tmp);
      if (st != PCF_OK) return finish(st);
    }
    for (int b = 0; b < B; ++b) {
      if (done[b]) continue;
      if (phase[b] == GAP) {
        if (--wait[b] <= 0) phase[b] = COLLECT;
        continue;
      }
      // snapshot of instance b into its ring slot (a sliding window before the first jump)
      double* slot = ring + ((size_t)next[b] * B + b) * plen;
      if (cudaMemcpyAsync(slot, tmp + (size_t)b * plen, pbytes, cudaMemcpyDeviceToDevice, c->user) != cudaSuccess)
        return finish(PCF_ECUDA);
      next[b] = (next[b] + 1) % S;
      filled[b] = std::min(filled[b] + 1, S);
      if (filled[b] < S || (phase[b] == FIRST && !(J[b] < sc->j_start))) continue;
      // the window in time order (oldest at slot next[b])
      for (int k = 0; k < S; ++k)
        if (cudaMemcpyAsync(ordered + (size_t)k * plen, ring + ((size_t)((next[b] + k) % S) * B + b) * plen, pbytes,
                            cudaMemcpyDeviceToDevice, c->user) != cudaSuccess)
          return finish(PCF_ECUDA);
      int r = 0;
      double jr = 0;
      const pcf_status sd =
          pcf_dmd_extrapolate(c, ordered, plen, S - 1, sc->rank_tol, u + 2 * (size_t)c->state_off[b], &r, &jr);
      if (sd == PCF_OK) ++jumps;
      else if (sd != PCF_ENAN) return finish(sd);
      filled[b] = 0;
      next[b] = 0;
      phase[b] = gap_chunks > 0 ? GAP : COLLECT;
      wait[b] = gap_chunks;
    }
  }
  for (int b = 0; b < B; ++b)
    if (done[b] == 2) return finish(PCF_ENAN);
  return finish(PCF_OK);
}

pcf_status pcf_run(pcf_ctx* c, double* u, double dtau, int max_steps, double tol, int dmd_period, int dmd_snapshots,
                   double rank_tol, int* steps_out, double* j_out, int* dmd_jumps) {
  if (dmd_period < 0) return PCF_EINVAL;
  if (dmd_period == 0) return run_schedule(c, u, dtau, max_steps, tol, nullptr, steps_out, j_out, dmd_jumps);
  if (dmd_snapshots < 3 || dmd_period % dmd_snapshots) return PCF_EINVAL;
  pcf_dmd_schedule sc;
  sc.snapshots = dmd_snapshots;
  sc.spacing = dmd_period / dmd_snapshots;
  sc.gap = 0;
  sc.j_start = INFINITY;
  sc.rank_tol = rank_tol;
  return run_schedule(c, u, dtau, max_steps, tol, &sc, steps_out, j_out, dmd_jumps);
}

pcf_status pcf_run_schedule(pcf_ctx* c, double* u, double dtau, int max_steps, double tol,
                            const pcf_dmd_schedule* schedule, int* steps_out, double* j_out, int* dmd_jumps) {
  return run_schedule(c, u, dtau, max_steps, tol, schedule, steps_out, j_out, dmd_jumps);
}

pcf_status pcf_descent_step_host(pcf_ctx* c, double* u_host, double dtau, int nsteps, double* hist_host) {
  if (!c || !u_host || nsteps < 0) return PCF_EINVAL;
  const size_t bytes = sizeof(double2) * (size_t)c->total_state;
  if (!c->u_dev) PCF_CUDA(cudaMalloc(&c->u_dev, bytes));
  if (hist_host && c->hist_cap < nsteps) {
    if (c->hist_dev) cudaFree(c->hist_dev);
    c->hist_dev = nullptr;
    PCF_CUDA(cudaMalloc(&c->hist_dev, sizeof(double) * (size_t)nsteps * c->B));
    c->hist_cap = nsteps;
  }
  PCF_CUDA(cudaMemcpyAsync(c->u_dev, u_host, bytes, cudaMemcpyHostToDevice, c->user));
  PCF_TRY(pcf_descent_step(c, (double*)c->u_dev, dtau, nsteps, hist_host ? c->hist_dev : nullptr));
  PCF_CUDA(cudaMemcpyAsync(u_host, c->u_dev, bytes, cudaMemcpyDeviceToHost, c->user));
  if (hist_host)
    PCF_CUDA(cudaMemcpyAsync(hist_host, c->hist_dev, sizeof(double) * (size_t)nsteps * c->B,
                             cudaMemcpyDeviceToHost, c->user));
  PCF_CUDA(cudaStreamSynchronize(c->user));
  return PCF_OK;
}

pcf_status pcf_set_kernel_timing(pcf_ctx* c, int enable) {
  if (!c) return PCF_EINVAL;
  c->timing = enable ? 1 : 0;
  for (int i = 0; i < kNumKernelClasses; ++i) {
    c->kms[i] = 0.0;
    c->kcount[i] = 0;
  }
  return PCF_OK;
}

pcf_status pcf_kernel_times(pcf_ctx* c, double* ms, long long* launches, int n) {
  if (!c || n < 0) return PCF_EINVAL;
  for (int i = 0; i < n && i < kNumKernelClasses; ++i) {
    if (ms) ms[i] = c->kms[i];
    if (launches) launches[i] = c->kcount[i];
  }
  return PCF_OK;
}

int pcf_launches_per_step(pcf_ctx* c) {
  if (!c) return 0;
  const int base = c->split ? (c->fused ? 7 : 10) : c->mixed ? 10 : 6;
  // symmetric subspace: the projection, plus a separate synthesis where the update kernel
  // synthesises the state itself (fused and single per-mode kernels)
  return base + (c->any_sym ? ((c->split && !c->fused) || c->mixed ? 1 : 2) : 0);
}

pcf_status pcf_norm(pcf_ctx* c, const double* u, double* out) {
  if (!c || !u || !out) return PCF_EINVAL;
  set_pointers(c, u, nullptr, nullptr);
  PCF_TRY(enter(c));
  PCF_TRY(push_descriptors(c));
  PCF_TRY(launch_ysynth(c, 0));
  PCF_TRY(launch_synth(c, 0, 3));
  launch_norm_planes(c->plane_kind, c->cta_synth3, c->cs, li_of(c, c->pre_synth3), 0);
  k_norm_final<<<1, 32, 0, c->cs>>>(li_of(c, c->pre_inst), out);
  PCF_TRY(check_launch());
  return leave(c);
}

pcf_status pcf_split_config(const pcf_ctx* c, int* cfg) {
  if (!c || !cfg) return PCF_EINVAL;
  cfg[0] = c->split ? c->sgrp : 0;
  cfg[1] = c->split ? c->smt : 0;
  cfg[2] = c->split ? c->smt_y : 0;
  cfg[3] = c->split && !c->fused ? c->sgrp_s : 0;
  return PCF_OK;
}

long long pcf_launches_per_call(pcf_ctx* c, int nsteps) {
  if (!c || nsteps < 0) return -1;
  if (nsteps == 0) return 0;
  // the entry projection and synthesis, then the steps; the split step synthesises the state
  // at its start, which the first step takes from the entry synthesis
  const long long entry = 1 + (c->any_sym ? 1 : 0);
  return entry + (long long)nsteps * pcf_launches_per_step(c) - (c->split && !c->fused ? 1 : 0);
}

pcf_status pcf_symmetrize(pcf_ctx* c, double* u, int mask) {
  if (!c || !u || mask < 0 || mask > 3) return PCF_EINVAL;
  if (mask == 0) return PCF_OK;
  set_pointers(c, u, nullptr, nullptr);
  PCF_TRY(enter(c));
  PCF_TRY(push_descriptors(c));
  PCF_TRY(launch_sym(c, mask));
  PCF_TRY(check_launch());
  return leave(c);
}

pcf_status pcf_dns(pcf_ctx* c, double* u, int nsteps, double* hist, double* guesses, int max_guesses,
                   int* n_guesses) {
  if (!c || !u || nsteps < 0 || max_guesses < 0 || (max_guesses > 0 && !guesses)) return PCF_EINVAL;
  const int B = c->B;
  if (!c->d_dns) {
    if (ctx_alloc(c, &c->d_dns, (size_t)B) || ctx_alloc(c, &c->uprev, (size_t)c->total_state) ||
        ctx_alloc(c, &c->dns_count, (size_t)B))
      return PCF_ENOMEM;
  }
  set_pointers(c, u, (const double*)c->r_int, nullptr);
  int* count = n_guesses ? n_guesses : c->dns_count;
  std::vector<DnsInst> hd(B);
  for (int b = 0; b < B; ++b) {
    DnsInst& D = hd[b];
    D.hist = hist ? hist + b : nullptr;
    D.hist_stride = B;
    D.uprev = c->uprev + c->state_off[b];
    D.guess = guesses ? (double2*)guesses + c->state_off[b] : nullptr;
    D.gstride = c->total_state;
    D.gmax = max_guesses;
    D.count = count + b;
    D.step = 0;
    D.slot = -1;
    D.h1 = D.h2 = 0.0;
  }
  PCF_TRY(enter(c));
  PCF_TRY(push_descriptors(c));
  PCF_CUDA(cudaMemcpyAsync(c->d_dns, hd.data(), sizeof(DnsInst) * B, cudaMemcpyHostToDevice, c->cs));
  PCF_CUDA(cudaMemsetAsync(count, 0, sizeof(int) * B, c->cs));
  if (nsteps == 0) return leave(c);
  if (c->any_sym) PCF_TRY(launch_sym(c, -1));
  PCF_TRY(launch_ysynth(c, 0));
  if (c->timing) {
    for (int s = 0; s < nsteps; ++s) PCF_TRY(dns_body(c));
    PCF_TRY(check_launch());
    return leave(c);
  }
  // graphs of up to 64 steps (the step counter lives on the device, so one graph serves
  // every chunk)
  const int chunk = 64;
  for (int done = 0; done < nsteps;) {
    const int n = std::min(chunk, nsteps - done);
    auto it = c->dns_graphs.find(n);
    if (it == c->dns_graphs.end()) {
      cudaGraph_t g;
      PCF_CUDA(cudaStreamBeginCapture(c->cs, cudaStreamCaptureModeThreadLocal));
      pcf_status st = PCF_OK;
      for (int s = 0; s < n && st == PCF_OK; ++s) st = dns_body(c);
      cudaError_t e = cudaStreamEndCapture(c->cs, &g);
      if (st != PCF_OK) return st;
      PCF_CUDA(e);
      cudaGraphExec_t ex;
      PCF_CUDA(cudaGraphInstantiate(&ex, g, 0));
      cudaGraphDestroy(g);
      it = c->dns_graphs.emplace(n, ex).first;
    }
    PCF_CUDA(cudaGraphLaunch(it->second, c->cs));
    done += n;
  }
  return leave(c);
}

pcf_status pcf_probe_fp64_peak(void* stream, double* gflops) {
  if (!gflops) return PCF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, nsm = 0;
  PCF_CUDA(cudaGetDevice(&dev));
  PCF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  double* d;
  PCF_CUDA(cudaMalloc(&d, sizeof(double) * 4096));
  const int blocks = nsm * 8, threads = 256, iters = 4096;
  k_fp64_probe<<<blocks, threads, 0, s>>>(d, iters);  // warm-up
  cudaEvent_t a, b;
  PCF_CUDA(cudaEventCreate(&a));
  PCF_CUDA(cudaEventCreate(&b));
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    PCF_CUDA(cudaEventRecord(a, s));
    k_fp64_probe<<<blocks, threads, 0, s>>>(d, iters);
    PCF_CUDA(cudaEventRecord(b, s));
    PCF_CUDA(cudaEventSynchronize(b));
    float ms;
    PCF_CUDA(cudaEventElapsedTime(&ms, a, b));
    best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(d);
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  *gflops = flops / (best * 1e-3) / 1e9;
  return PCF_OK;
}


}  // extern "C"
