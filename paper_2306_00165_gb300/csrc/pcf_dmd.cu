// Snapshot vector psi and DMD steady-state extrapolation (paper §6.1-6.2).
//
// psi (§6.2, "minimum number of independent variables"): per independent Fourier mode
// (p > 0: every m; p = 0: m > 0) the Chebyshev coefficients 0..N-4 of v and 0..N-2 of
// the wall-normal vorticity eta = i kz u - i kx w (real parts, then imaginary parts),
// followed by the coefficients 0..N-2 of the mean u and w.  The remaining coefficients
// follow from v = dv/dy = 0 and eta = 0 at the walls, u and w from the divergence
// constraint and eta.
//
// DMD: the snapshot matrix S = [s_0 .. s_M] is reduced by a Householder QR on the
// device (S = Q R, Q never formed); Psi = Q R[:, 0:M] and Psi' = Q R[:, 1:M+1], so the
// SVD of Psi, the projected operator A~ = U^T Psi' V Sigma^-1, its eigenpairs and the
// least-squares amplitudes are all computed from the small R on the host; the steady
// state b_1 phi_1 = Psi' (Re(b_1 V Sigma^-1 w_1)) is a combination of the snapshots.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "pcf_ctx.h"
#include "pcf_linalg.h"

namespace pcf {

// ------------------------------------------------------------------ psi <-> uhat
__global__ void k_psi_extract(const double2* __restrict__ uhat, long long state_len, double* __restrict__ psi,
                              long long psi_len, const int* __restrict__ indep, int nindep,
                              const double* __restrict__ kx, const double* __restrict__ kz, int Mz, int ny, int nm,
                              int B) {
  const int N = ny - 1;
  const long long per = (long long)(nindep + 1) * ny;
  const long long total = per * B;
  const int segv = N - 3, sege = N - 1, seg = 2 * segv + 2 * sege;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / per);
    const long long r = t - (long long)b * per;
    const int q = (int)(r / ny), n = (int)(r - (long long)q * ny);
    const double2* u = uhat + (size_t)b * state_len;
    double* out = psi + (size_t)b * psi_len;
    if (q < nindep) {
      const int i = indep[2 * q], j = indep[2 * q + 1], m = i * Mz + j;
      double* o = out + (size_t)q * seg;
      const double2 vv = u[((size_t)1 * nm + m) * ny + n];
      if (n < segv) {
        o[n] = vv.x;
        o[segv + n] = vv.y;
      }
      if (n < sege) {
        const double2 uu = u[((size_t)0 * nm + m) * ny + n], ww = u[((size_t)2 * nm + m) * ny + n];
        const double a = kx[i], c = kz[j];
        o[2 * segv + n] = -c * uu.y + a * ww.y;
        o[2 * segv + sege + n] = c * uu.x - a * ww.x;
      }
    } else if (n < sege) {
      double* o = out + (size_t)nindep * seg;
      o[n] = u[((size_t)0 * nm + 0) * ny + n].x;
      o[sege + n] = u[((size_t)2 * nm + 0) * ny + n].x;
    }
  }
}

// One thread per (instance, independent mode or mean): rebuild the mode's u, v, w.
__global__ void k_psi_rebuild(const double* __restrict__ psi, long long psi_len, double2* __restrict__ uhat,
                              long long state_len, const int* __restrict__ indep, int nindep,
                              const double* __restrict__ kx, const double* __restrict__ kz, int Mx, int Mz, int ny,
                              int nm, int B) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * (nindep + 1)) return;
  const int b = t / (nindep + 1), q = t - b * (nindep + 1);
  const int N = ny - 1;
  const int segv = N - 3, sege = N - 1, seg = 2 * segv + 2 * sege;
  const double* in = psi + (size_t)b * psi_len;
  double2* u = uhat + (size_t)b * state_len;
  double vr[130], vi[130], er[130], ei[130];
  if (q == nindep) {
    // mean u, w: Dirichlet completion, imaginary part zero; v = 0
    const double* o = in + (size_t)nindep * seg;
    for (int c = 0; c < 2; ++c) {
      for (int n = 0; n <= N; ++n) vr[n] = n < sege ? o[c * sege + n] : 0.0;
      for (int par = 0; par < 2; ++par) {
        const int top = (N % 2 == par) ? N : N - 1;
        double s = 0.0;
        for (int n = par; n < top; n += 2) s += vr[n];
        vr[top] = -s;
      }
      const int comp = c == 0 ? 0 : 2;
      for (int n = 0; n <= N; ++n) u[((size_t)comp * nm + 0) * ny + n] = make_double2(vr[n], 0.0);
    }
    for (int n = 0; n <= N; ++n) u[((size_t)1 * nm + 0) * ny + n] = make_double2(0.0, 0.0);
    return;
  }
  const int i = indep[2 * q], j = indep[2 * q + 1], m = i * Mz + j;
  const double* o = in + (size_t)q * seg;
  for (int n = 0; n <= N; ++n) {
    vr[n] = n < segv ? o[n] : 0.0;
    vi[n] = n < segv ? o[segv + n] : 0.0;
    er[n] = n < sege ? o[2 * segv + n] : 0.0;
    ei[n] = n < sege ? o[2 * segv + sege + n] : 0.0;
  }
  // v: for each parity class the two top coefficients from sum a_n = 0, sum n^2 a_n = 0
  for (int par = 0; par < 2; ++par) {
    const int hi = (N % 2 == par) ? N : N - 1, lo = hi - 2;
    double s0r = 0, s1r = 0, s0i = 0, s1i = 0;
    for (int n = par; n < lo; n += 2) {
      const double n2 = (double)n * n;
      s0r += vr[n];
      s1r += n2 * vr[n];
      s0i += vi[n];
      s1i += n2 * vi[n];
    }
    const double h2 = (double)hi * hi, l2 = (double)lo * lo, det = l2 - h2;
    vr[hi] = (s1r - s0r * l2) / det;
    vr[lo] = (s0r * h2 - s1r) / det;
    vi[hi] = (s1i - s0i * l2) / det;
    vi[lo] = (s0i * h2 - s1i) / det;
  }
  // eta: top coefficient of each class from sum a_n = 0
  for (int par = 0; par < 2; ++par) {
    const int top = (N % 2 == par) ? N : N - 1;
    double sr = 0, si = 0;
    for (int n = par; n < top; n += 2) {
      sr += er[n];
      si += ei[n];
    }
    er[top] = -sr;
    ei[top] = -si;
  }
  const double a = kx[i], c = kz[j], k2 = a * a + c * c;
  // xi = -dv/dy by the coefficient recurrence, then u, w
  double br2 = 0, br1 = 0, bi2 = 0, bi1 = 0;  // b_{n+2}, b_{n+1}
  double xr[130], xi[130];
  for (int n = N; n >= 0; --n) {
    double br = 0.0, bi = 0.0;
    if (n + 1 <= N) {
      br = br2 + 2.0 * (n + 1) * vr[n + 1];
      bi = bi2 + 2.0 * (n + 1) * vi[n + 1];
    }
    br2 = br1;
    bi2 = bi1;
    br1 = br;
    bi1 = bi;
    xr[n] = br;
    xi[n] = bi;
  }
  xr[0] *= 0.5;
  xi[0] *= 0.5;
  const int mconj = (Mx - i) * Mz;  // storage index of (-m, 0)
  for (int n = 0; n <= N; ++n) {
    const double xre = -xr[n], xim = -xi[n];
    const double2 uu = make_double2((a * xim + c * ei[n]) / k2, -(a * xre + c * er[n]) / k2);
    const double2 vv = make_double2(vr[n], vi[n]);
    const double2 ww = make_double2((c * xim - a * ei[n]) / k2, (-c * xre + a * er[n]) / k2);
    u[((size_t)0 * nm + m) * ny + n] = uu;
    u[((size_t)1 * nm + m) * ny + n] = vv;
    u[((size_t)2 * nm + m) * ny + n] = ww;
    if (j == 0) {
      u[((size_t)0 * nm + mconj) * ny + n] = make_double2(uu.x, -uu.y);
      u[((size_t)1 * nm + mconj) * ny + n] = make_double2(vv.x, -vv.y);
      u[((size_t)2 * nm + mconj) * ny + n] = make_double2(ww.x, -ww.y);
    }
  }
}

// ------------------------------------------------------------------ Householder QR (R only)
// A: rows x ncol column-major with leading dimension ld (in doubles).
constexpr int kQrBlocks = 64;

__global__ void k_qr_dots(const double* __restrict__ A, long long rows, long long ld, int j, int ncol,
                          double* __restrict__ part) {
  __shared__ double red[32];
  const double* aj = A + (size_t)j * ld;
  for (int k = j; k < ncol; ++k) {
    const double* ak = A + (size_t)k * ld;
    double s = 0.0;
    for (long long i = j + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows;
         i += (long long)gridDim.x * blockDim.x)
      s = fma(aj[i], ak[i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      part[(size_t)(k - j) * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// coef[k] (k > j) = 2 v^T a_k / v^T v for the reflector v = x - alpha e_j; alpha[j] = R_jj.
__global__ void k_qr_reflect(double* __restrict__ A, long long ld, int j, int ncol, const double* __restrict__ part,
                             int G, double* __restrict__ coef, double* __restrict__ alpha) {
  __shared__ double sxj, salpha, svtv;
  if (threadIdx.x == 0) {
    double x2 = 0.0;
    for (int g = 0; g < G; ++g) x2 += part[g];
    const double xj = A[(size_t)j * ld + j];
    const double nrm = sqrt(x2);
    const double al = xj >= 0.0 ? -nrm : nrm;
    sxj = xj;
    salpha = al;
    svtv = 2.0 * (x2 - al * xj);
    alpha[j] = al;
  }
  __syncthreads();
  for (int k = j + 1 + threadIdx.x; k < ncol; k += blockDim.x) {
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += part[(size_t)(k - j) * G + g];
    const double vta = s - salpha * A[(size_t)k * ld + j];
    coef[k] = svtv > 0.0 ? 2.0 * vta / svtv : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) A[(size_t)j * ld + j] = sxj - salpha;
}

__global__ void k_qr_update(double* __restrict__ A, long long rows, long long ld, int j, int ncol,
                            const double* __restrict__ coef) {
  for (long long i = j + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows;
       i += (long long)gridDim.x * blockDim.x) {
    const double vi = A[(size_t)j * ld + i];
    for (int k = j + 1; k < ncol; ++k) A[(size_t)k * ld + i] = fma(-coef[k], vi, A[(size_t)k * ld + i]);
  }
}

// cand[c][i] = sum_k C[c][k] S[i][k+1]  (k < M): steady states as combinations of snapshots
__global__ void k_combine(const double* __restrict__ S, long long rows, long long ld, int M,
                          const double* __restrict__ C, int ncand, double* __restrict__ out, long long out_ld) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows;
       i += (long long)gridDim.x * blockDim.x) {
    for (int c = 0; c < ncand; ++c) {
      double s = 0.0;
      for (int k = 0; k < M; ++k) s = fma(C[(size_t)c * M + k], S[(size_t)(k + 1) * ld + i], s);
      out[(size_t)c * out_ld + i] = s;
    }
  }
}

}  // namespace pcf

using namespace pcf;

namespace {

thread_local char g_dmd_err[256] = "";

#define DMD_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      snprintf(g_dmd_err, sizeof(g_dmd_err), "%s: %s", #call, cudaGetErrorString(e_));    \
      return PCF_ECUDA;                                                                   \
    }                                                                                     \
  } while (0)

pcf_status ensure_indep(pcf_ctx* c) {
  if (c->d_indep) return PCF_OK;
  std::vector<int> idx;
  for (int i = 0; i < c->Mx; ++i)
    for (int j = 0; j < c->Mz; ++j) {
      const int m = i <= c->Kx ? i : i - c->Mx;
      if (j > 0 || m >= 1) {
        idx.push_back(i);
        idx.push_back(j);
      }
    }
  c->nindep = (int)idx.size() / 2;
  c->psi_len = pcf_psi_len(c->prm.nx, c->prm.ny, c->prm.nz);
  DMD_CUDA(cudaMalloc(&c->d_indep, idx.size() * sizeof(int)));
  c->allocs.push_back(c->d_indep);
  DMD_CUDA(cudaMemcpy(c->d_indep, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice));
  return PCF_OK;
}

pcf_status ensure_dmd(pcf_ctx* c, int ncol) {
  if (c->dmd_cap >= ncol) return PCF_OK;
  const int cap = std::max(ncol, 32);
  const int ncand = ((cap + c->B - 1) / c->B) * c->B;
  double *A, *part, *coef, *cpsi, *J, *cc;
  double2* cu;
  DMD_CUDA(cudaMalloc(&A, sizeof(double) * (size_t)c->psi_len * cap));
  DMD_CUDA(cudaMalloc(&part, sizeof(double) * (size_t)kQrBlocks * cap));
  DMD_CUDA(cudaMalloc(&coef, sizeof(double) * 2 * (size_t)cap));
  DMD_CUDA(cudaMalloc(&cpsi, sizeof(double) * (size_t)c->psi_len * ncand));
  DMD_CUDA(cudaMalloc(&cu, sizeof(double2) * (size_t)c->state_len * ncand));
  DMD_CUDA(cudaMalloc(&J, sizeof(double) * (size_t)c->B));
  DMD_CUDA(cudaMalloc(&cc, sizeof(double) * (size_t)cap * ncand));
  for (void* p : {(void*)A, (void*)part, (void*)coef, (void*)cpsi, (void*)cu, (void*)J, (void*)cc})
    c->allocs.push_back(p);
  c->dmd_A = A;
  c->dmd_part = part;
  c->dmd_coef = coef;
  c->dmd_cpsi = cpsi;
  c->dmd_cu = cu;
  c->dmd_J = J;
  c->dmd_c = cc;
  c->dmd_cap = cap;
  c->dmd_ncand_cap = ncand;
  return PCF_OK;
}

pcf_status sync_in(pcf_ctx* c) {
  DMD_CUDA(cudaEventRecord(c->ev_in, c->user));
  DMD_CUDA(cudaStreamWaitEvent(c->cs, c->ev_in, 0));
  return PCF_OK;
}
pcf_status sync_out(pcf_ctx* c) {
  DMD_CUDA(cudaEventRecord(c->ev_out, c->cs));
  DMD_CUDA(cudaStreamWaitEvent(c->user, c->ev_out, 0));
  return PCF_OK;
}

#define DMD_TRY(x)               \
  do {                           \
    pcf_status s_ = (x);         \
    if (s_ != PCF_OK) return s_; \
  } while (0)

}  // namespace

extern "C" {

pcf_status pcf_snapshot(pcf_ctx* c, const double* u_hat, double* psi) {
  if (!c || !u_hat || !psi) return PCF_EINVAL;
  if (!c->uniform) return PCF_ENOTSUP;
  DMD_TRY(ensure_indep(c));
  DMD_TRY(sync_in(c));
  const long long total = (long long)(c->nindep + 1) * c->prm.ny * c->B;
  const int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
  k_psi_extract<<<blocks, 256, 0, c->cs>>>((const double2*)u_hat, c->state_len, psi, c->psi_len, c->d_indep,
                                           c->nindep, c->hinst[0].kx, c->hinst[0].kz, c->Mz, c->prm.ny, c->nm, c->B);
  DMD_CUDA(cudaGetLastError());
  return sync_out(c);
}

pcf_status pcf_from_snapshot(pcf_ctx* c, const double* psi, double* u_hat) {
  if (!c || !u_hat || !psi) return PCF_EINVAL;
  if (!c->uniform) return PCF_ENOTSUP;
  if (c->prm.ny > 129) return PCF_EINVAL;
  DMD_TRY(ensure_indep(c));
  DMD_TRY(sync_in(c));
  const int n = c->B * (c->nindep + 1);
  k_psi_rebuild<<<(n + 127) / 128, 128, 0, c->cs>>>(psi, c->psi_len, (double2*)u_hat, c->state_len, c->d_indep,
                                                    c->nindep, c->hinst[0].kx, c->hinst[0].kz, c->Mx, c->Mz,
                                                    c->prm.ny, c->nm, c->B);
  DMD_CUDA(cudaGetLastError());
  return sync_out(c);
}

pcf_status pcf_dmd_extrapolate(pcf_ctx* c, const double* S, long long ld, int M, double rank_tol, double* u_out,
                               int* rank_used, double* j_out) {
  if (!c || !S || !u_out || M < 1 || !(rank_tol >= 0)) return PCF_EINVAL;
  if (!c->uniform) return PCF_ENOTSUP;
  DMD_TRY(ensure_indep(c));
  if (ld < c->psi_len) return PCF_EINVAL;
  const int ncol = M + 1;
  DMD_TRY(ensure_dmd(c, ncol));
  DMD_TRY(sync_in(c));
  const long long rows = c->psi_len;
  // copy the snapshots into the QR workspace (column-major, ld = rows)
  DMD_CUDA(cudaMemcpy2DAsync(c->dmd_A, sizeof(double) * rows, S, sizeof(double) * ld, sizeof(double) * rows, ncol,
                             cudaMemcpyDeviceToDevice, c->cs));
  double* alpha = c->dmd_coef + c->dmd_cap;
  for (int j = 0; j < ncol; ++j) {
    k_qr_dots<<<kQrBlocks, 256, 0, c->cs>>>(c->dmd_A, rows, rows, j, ncol, c->dmd_part);
    k_qr_reflect<<<1, 128, 0, c->cs>>>(c->dmd_A, rows, j, ncol, c->dmd_part, kQrBlocks, c->dmd_coef, alpha);
    if (j + 1 < ncol) k_qr_update<<<kQrBlocks, 256, 0, c->cs>>>(c->dmd_A, rows, rows, j, ncol, c->dmd_coef);
  }
  DMD_CUDA(cudaGetLastError());
  std::vector<double> Rcm((size_t)ncol * ncol), al(ncol);
  DMD_CUDA(cudaMemcpy2DAsync(Rcm.data(), sizeof(double) * ncol, c->dmd_A, sizeof(double) * rows,
                             sizeof(double) * ncol, ncol, cudaMemcpyDeviceToHost, c->cs));
  DMD_CUDA(cudaMemcpyAsync(al.data(), alpha, sizeof(double) * ncol, cudaMemcpyDeviceToHost, c->cs));
  DMD_CUDA(cudaStreamSynchronize(c->cs));
  // R (row-major, ncol x ncol, upper triangular)
  std::vector<double> R((size_t)ncol * ncol, 0.0);
  for (int j = 0; j < ncol; ++j) {
    R[(size_t)j * ncol + j] = al[j];
    for (int k = j + 1; k < ncol; ++k) R[(size_t)j * ncol + k] = Rcm[(size_t)k * ncol + j];
  }
  // Psi ~ R0 = R[:, 0:M], Psi' ~ R1 = R[:, 1:M+1], last snapshot t = R[:, M]
  std::vector<double> R0((size_t)ncol * M), R1((size_t)ncol * M), t(ncol);
  for (int i = 0; i < ncol; ++i) {
    for (int k = 0; k < M; ++k) {
      R0[(size_t)i * M + k] = R[(size_t)i * ncol + k];
      R1[(size_t)i * M + k] = R[(size_t)i * ncol + k + 1];
    }
    t[i] = R[(size_t)i * ncol + M];
  }
  std::vector<double> U, s, V;
  la::svd_jacobi(ncol, M, R0, U, s, V);
  int rstar = 0;
  for (int k = 0; k < M; ++k)
    if (s[k] > rank_tol * s[0]) ++rstar;
  if (rstar == 0) return PCF_ENAN;
  // candidates r = rstar .. 1: coefficient vectors over the snapshots s_1..s_M
  std::vector<double> Cc((size_t)rstar * M, 0.0);
  std::vector<int> rank_of(rstar);
  int ncand = 0;
  for (int r = rstar; r >= 1; --r) {
    std::vector<double> VS((size_t)M * r);  // V_r Sigma_r^-1
    for (int i = 0; i < M; ++i)
      for (int k = 0; k < r; ++k) VS[(size_t)i * r + k] = V[(size_t)i * M + k] / s[k];
    std::vector<double> X((size_t)ncol * r, 0.0);  // R1 V_r Sigma_r^-1
    for (int i = 0; i < ncol; ++i)
      for (int k = 0; k < r; ++k) {
        double a = 0;
        for (int l = 0; l < M; ++l) a += R1[(size_t)i * M + l] * VS[(size_t)l * r + k];
        X[(size_t)i * r + k] = a;
      }
    std::vector<double> At((size_t)r * r, 0.0);  // U_r^T X
    for (int a = 0; a < r; ++a)
      for (int b = 0; b < r; ++b) {
        double v = 0;
        for (int i = 0; i < ncol; ++i) v += U[(size_t)i * M + a] * X[(size_t)i * r + b];
        At[(size_t)a * r + b] = v;
      }
    std::vector<la::cd> lam, W;
    if (!la::eig_general(r, At, lam, W)) continue;
    int q1 = 0;
    double best = 1e300;
    for (int q = 0; q < r; ++q) {
      const double w = std::abs(std::log(lam[q]));
      if (w < best) {
        best = w;
        q1 = q;
      }
    }
    std::vector<double> cp = la::lstsq_svd(ncol, r, X, t);
    std::vector<la::cd> bvec(cp.begin(), cp.end());
    if (!la::csolve(r, W, bvec)) continue;
    const la::cd b1 = bvec[q1];
    double* cv = Cc.data() + (size_t)ncand * M;
    for (int l = 0; l < M; ++l) {
      la::cd a = 0;
      for (int k = 0; k < r; ++k) a += VS[(size_t)l * r + k] * W[(size_t)k * r + q1];
      cv[l] = std::real(b1 * a);
    }
    rank_of[ncand++] = r;
  }
  if (ncand == 0) return PCF_ENAN;
  // candidate states on the device
  DMD_CUDA(cudaMemcpyAsync(c->dmd_c, Cc.data(), sizeof(double) * (size_t)ncand * M, cudaMemcpyHostToDevice, c->cs));
  k_combine<<<std::min<long long>((rows + 255) / 256, 2048), 256, 0, c->cs>>>(S, rows, ld, M, c->dmd_c, ncand,
                                                                             c->dmd_cpsi, rows);
  DMD_CUDA(cudaGetLastError());
  const int nb = (ncand + c->B - 1) / c->B * c->B;
  for (int k = ncand; k < nb; ++k)  // pad to whole batches with the last candidate
    DMD_CUDA(cudaMemcpyAsync(c->dmd_cpsi + (size_t)k * rows, c->dmd_cpsi + (size_t)(ncand - 1) * rows,
                             sizeof(double) * rows, cudaMemcpyDeviceToDevice, c->cs));
  {
    const int n = nb * (c->nindep + 1);
    k_psi_rebuild<<<(n + 127) / 128, 128, 0, c->cs>>>(c->dmd_cpsi, rows, c->dmd_cu, c->state_len, c->d_indep,
                                                      c->nindep, c->hinst[0].kx, c->hinst[0].kz, c->Mx, c->Mz,
                                                      c->prm.ny, c->nm, nb);
    DMD_CUDA(cudaGetLastError());
  }
  DMD_CUDA(cudaEventRecord(c->ev_out, c->cs));
  DMD_CUDA(cudaStreamWaitEvent(c->user, c->ev_out, 0));
  std::vector<double> Jc(nb);
  for (int g = 0; g < nb; g += c->B) {
    DMD_TRY(pcf_residual(c, (const double*)(c->dmd_cu + (size_t)g * c->state_len), (double*)c->r_int, c->dmd_J));
    DMD_CUDA(cudaMemcpyAsync(Jc.data() + g, c->dmd_J, sizeof(double) * c->B, cudaMemcpyDeviceToHost, c->user));
  }
  DMD_CUDA(cudaStreamSynchronize(c->user));
  int bi = -1;
  for (int k = 0; k < ncand; ++k)  // candidates are ordered by decreasing rank: ties keep the larger r
    if (std::isfinite(Jc[k]) && (bi < 0 || Jc[k] < Jc[bi])) bi = k;
  if (bi < 0) return PCF_ENAN;
  DMD_CUDA(cudaMemcpyAsync(u_out, c->dmd_cu + (size_t)bi * c->state_len, sizeof(double2) * c->state_len,
                           cudaMemcpyDeviceToDevice, c->user));
  DMD_CUDA(cudaStreamSynchronize(c->user));
  if (rank_used) *rank_used = rank_of[bi];
  if (j_out) *j_out = Jc[bi];
  return PCF_OK;
}

}  // extern "C"
