// pcf_influence_matrix_solve_noalloc: the per-mode Stokes solve without any allocation.
//
// Who needs it: code that runs where allocating device memory is not possible or not
// allowed - e.g. a host application whose device memory is owned by a fixed pool or a
// foreign allocator, a plugin that must not grow the device footprint after start-up,
// or code between a memory-budget check and a launch.  pcf_create allocates its tables
// and workspace with cudaMalloc; this entry point instead keeps everything it needs
// beyond the caller's input and output (the instance descriptor, the CTA prefix, the
// Chebyshev-tau sweep coefficients, the homogeneous responses and 2x2 influence-matrix
// inverses of every mode) in one file-scope static device array of fixed size, and
// rebuilds that content on the device at every call.
//
// Limits and rules:
// * Capacity: kNoAllocDoubles doubles (5 MiB), enough for grids up to 64 x 65 x 64
//   (861 Fourier modes, ny <= 65) and a single instance (batch = 1).  Larger requests
//   return PCF_EINVAL before anything is launched.
// * The array exists once per device for the lifetime of the process (every GPU that
//   loads the library holds these 5 MiB until exit).
// * Set-up: the first call on a device, with that device current, looks up the array's
//   device address (cudaGetSymbolAddress); later calls on that device reuse it.  Make
//   that first call before any stream capture.  Each call also raises the solve
//   kernel's dynamic shared-memory limit to what it needs (a limit, not an allocation).
// * Every call shares the one array and overwrites all of it that the solve reads, so no
//   state carries over from a previous call.  Calls that overlap on the GPU (on different
//   streams, or from different host threads without ordering) race on the array: order
//   them on one stream.
#include <cmath>
#include <cstring>

#include "pcf_kernels.cuh"

namespace pcf {
namespace {

constexpr size_t kNoAllocDoubles = 5u * 1024u * 1024u / sizeof(double);
constexpr int kNoAllocMaxMh = 33;  // ny <= 65
constexpr int kNoAllocMaxModes = 861;

// The scratch.  Host code must not take its address directly (in host code the name is
// a host-side stand-in); the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Offsets (in doubles) of the pieces inside the scratch array.
struct NoAllocLayout {
  size_t inst, prefix, rco, cheb, kx, kz, tab, end;
  NoAllocLayout(int N, int Mx, int Mz) {
    const TabLayout TL(N);
    const RcoLayout RL(N);
    const ChebLayout CL(N);
    size_t o = 0;
    auto take = [&](size_t n) { size_t r = o; o += (n + 31) & ~size_t(31); return r; };
    inst = take((sizeof(Inst) + sizeof(double) - 1) / sizeof(double));
    prefix = take(2);
    rco = take(RL.total());
    cheb = take(CL.total());
    kx = take(Mx);
    kz = take(Mz);
    tab = take((size_t)Mx * Mz * TL.per_mode());
    end = o;
  }
};

// Descriptor, prefix, shared coefficients, wavenumbers; zeroes the (unused) Chebyshev
// matrices the solve kernel stages into shared memory.
__global__ void k_noalloc_setup_shared(Inst I, double* base, NoAllocLayout L, double Lx, double Lz) {
  const int N = I.N;
  const RcoLayout RL(N);
  const ChebLayout CL(N);
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  if (t0 == 0) {
    *reinterpret_cast<Inst*>(base + L.inst) = I;
    int* pre = reinterpret_cast<int*>(base + L.prefix);
    pre[0] = 0;
    pre[1] = 0;
  }
  double* rco = base + L.rco;
  for (int t = t0; t < RL.total(); t += nt) rco[t] = 0.0;
  for (int t = t0; t < CL.total(); t += nt) base[L.cheb + t] = 0.0;
  for (int t = t0; t < I.Mx; t += nt) {
    const int m = t <= I.Kx ? t : t - I.Mx;
    base[L.kx + t] = 2.0 * 3.14159265358979323846 * m / Lx;
  }
  for (int t = t0; t < I.Mz; t += nt) base[L.kz + t] = 2.0 * 3.14159265358979323846 * t / Lz;
  __syncthreads();
  // tau right-hand-side combinations and class constants (one thread per class element)
  const int Mh = N / 2 + 1;
  for (int t = t0; t < 2 * Mh; t += nt) {
    const int par = t / Mh, i = t - par * Mh;
    const int Mc = (N - par) / 2 + 1;
    if (i >= Mc) continue;
    const int n = par + 2 * i;
    const double dn = n;
    if (i >= 1) {
      const double cm2 = (n - 2 == 0) ? 2.0 : 1.0;
      rco[RL.off(par, 0) + i] = -cm2 / (4.0 * dn * (dn - 1.0));
      rco[RL.off(par, 1) + i] = (n <= N - 2) ? 1.0 / (2.0 * (dn * dn - 1.0)) : 0.0;
      rco[RL.off(par, 2) + i] = (n + 2 <= N - 2) ? -1.0 / (4.0 * dn * (dn + 1.0)) : 0.0;
    }
    rco[RL.off(par, 3) + i] = dn * dn;
    rco[RL.off(par, 4) + i] = 2.0 * dn;
  }
}

__device__ void na_solver_coefs(int N, int par, double lam, const double* rco, double* dst) {
  const RcoLayout RL(N);
  const int Mh = N / 2 + 1, Mc = (N - par) / 2 + 1;
  for (int i = 0; i < 4 * Mh + 2; ++i) dst[i] = 0.0;
  double bnext = 0.0;
  for (int i = Mc - 1; i >= 1; --i) {
    const double a = lam * rco[RL.off(par, 0) + i], bb = 1.0 + lam * rco[RL.off(par, 1) + i];
    const double cc = lam * rco[RL.off(par, 2) + i];
    const double den = bb + cc * bnext;
    dst[i] = cc;
    dst[Mh + i] = 1.0 / den;
    dst[2 * Mh + i] = -a / den;
    bnext = dst[2 * Mh + i];
  }
  double B = 1.0, sum = 1.0;
  dst[3 * Mh] = 1.0;
  for (int i = 1; i < Mc; ++i) {
    B *= dst[2 * Mh + i];
    dst[3 * Mh + i] = B;
    sum += B;
  }
  dst[4 * Mh] = 1.0 / sum;
}

// One thread per mode: sweep coefficients of the four tau operators, then the two
// homogeneous responses and the 2x2 influence-matrix inverse of each parity group.
__global__ void k_noalloc_setup_modes(double* base, NoAllocLayout L, int N, int Mx, int Mz, double sigma) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= Mx * Mz) return;
  const TabLayout TL(N);
  const RcoLayout RL(N);
  const int Mh = N / 2 + 1;
  const double* rco = base + L.rco;
  const int i = m / Mz, p = m - i * Mz;
  const double kx = base[L.kx + i], kz = base[L.kz + p];
  const double k2 = kx * kx + kz * kz;
  double* d = base + L.tab + (size_t)m * TL.per_mode();
  for (int par = 0; par < 2; ++par) {
    na_solver_coefs(N, par, k2, rco, d + TL.solver(0, par));
    na_solver_coefs(N, par, sigma + k2, rco, d + TL.solver(1, par));
  }
  for (int g = 0; g < 2; ++g) {
    double* gd = d + TL.group(g);
    for (int t = 0; t < 2 * Mh + 4; ++t) gd[t] = 0.0;
    if (k2 == 0.0) continue;
    const int pv = g, pP = 1 - g;
    const int McP = (N - pP) / 2 + 1, McV = (N - pv) / 2 + 1;
    double P[kNoAllocMaxMh], T[kNoAllocMaxMh], V[kNoAllocMaxMh], R[kNoAllocMaxMh], U[kNoAllocMaxMh];
    double F1[2], F2[2];
    for (int h = 0; h < 2; ++h) {
      for (int t = 0; t < Mh; ++t) R[t] = 0.0;
      double bc = 0.0;
      if (h == 0) {
        bc = 1.0;
      } else {
        for (int t = 0; t < Mh; ++t) U[t] = 0.0;
        U[McV - 1] = 1.0;
        class_deriv(N, pv, U, rco + RL.off(pv, 4), T);
        for (int t = 0; t < McP; ++t) R[t] = -T[t];
      }
      const double* s = d + TL.solver(0, pP);
      tau_solve(McP, s, s + Mh, s + 2 * Mh, s + 3 * Mh, s[4 * Mh], rco + RL.off(pP, 0), rco + RL.off(pP, 1),
                rco + RL.off(pP, 2), R, bc, P);
      class_deriv(N, pP, P, rco + RL.off(pP, 4), T);
      for (int t = 0; t < McV; ++t) R[t] = -T[t];
      s = d + TL.solver(1, pv);
      tau_solve(McV, s, s + Mh, s + 2 * Mh, s + 3 * Mh, s[4 * Mh], rco + RL.off(pv, 0), rco + RL.off(pv, 1),
                rco + RL.off(pv, 2), R, 0.0, V);
      double f1 = 0.0;
      for (int t = 0; t < McV; ++t) f1 += rco[RL.off(pv, 3) + t] * V[t];
      double f2 = (sigma + k2) * V[McV - 1];
      if (g == 1) f2 += 2.0 * N * P[McP - 1];
      if (h == 1) f2 -= 1.0;
      F1[h] = f1;
      F2[h] = f2;
      for (int t = 0; t < McV; ++t) gd[h * Mh + t] = V[t];
    }
    const double det = F1[0] * F2[1] - F1[1] * F2[0];
    gd[2 * Mh + 0] = F2[1] / det;
    gd[2 * Mh + 1] = -F1[1] / det;
    gd[2 * Mh + 2] = -F2[0] / det;
    gd[2 * Mh + 3] = F1[0] / det;
  }
}

bool noalloc_grid_ok(int nx, int ny, int nz) {
  if (nx < 16 || nz < 16 || nx > 64 || nz > 64 || (nx % 2) || (nz % 2) || ny < 9 || !(ny % 2)) return false;
  const int Kx = nx / 3 - 1, Kz = nz / 3 - 1;
  const int Mh = (ny - 1) / 2 + 1;
  return Mh <= kNoAllocMaxMh && (2 * Kx + 1) * (Kz + 1) <= kNoAllocMaxModes;
}

}  // namespace
}  // namespace pcf

using namespace pcf;

extern "C" pcf_status pcf_influence_matrix_solve_noalloc(const pcf_params* prm, const double* rhs_hat,
                                                         double* out_hat, double step, void* stream) {
  if (!prm || !rhs_hat || !out_hat || prm->batch != 1 || !(prm->Re > 0) || !(step > 0) || !(prm->Lx > 0) ||
      !(prm->Lz > 0))
    return PCF_EINVAL;
  if (!noalloc_grid_ok(prm->nx, prm->ny, prm->nz)) return PCF_EINVAL;
  const int N = prm->ny - 1, Kx = prm->nx / 3 - 1, Kz = prm->nz / 3 - 1;
  const int Mx = 2 * Kx + 1, Mz = Kz + 1, nm = Mx * Mz;
  const NoAllocLayout L(N, Mx, Mz);
  if (L.end > kNoAllocDoubles) return PCF_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PCF_ECUDA;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PCF_ECUDA;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  double* base = g_scratch_ptr[dev];
  cudaStream_t s = (cudaStream_t)stream;

  Inst I;
  memset(&I, 0, sizeof(I));
  I.nx = prm->nx; I.ny = prm->ny; I.nz = prm->nz; I.N = N; I.Kx = Kx; I.Kz = Kz; I.Mx = Mx; I.Mz = Mz;
  I.nmodes = nm;
  I.nu = 1.0 / prm->Re;
  I.dt = step;
  I.dtau_hat = step;
  I.inv_nu = 1.0 / I.nu;
  I.inv_dt = I.inv_dtau_hat = 1.0 / step;
  I.inv_nxnz = 1.0 / ((double)prm->nx * prm->nz);
  I.rco = base + L.rco;
  I.cheb = base + L.cheb;
  I.kx = base + L.kx;
  I.kz = base + L.kz;
  I.tab[0] = I.tab[1] = base + L.tab;
  I.sigma[0] = I.sigma[1] = 1.0 / (I.nu * step);
  I.rhat = (double2*)rhs_hat;
  I.fhat = (double2*)out_hat;
  I.hist_stride = 1;

  int mpc = prm->modes_per_block > 0 ? prm->modes_per_block : 4;
  while (mpc > 1 && smem_mode(I, mpc) > 110 * 1024) --mpc;
  const size_t smem = smem_mode(I, mpc);
  if (smem > 227 * 1024) return PCF_EINVAL;
  // a limit, not an allocation; it only ever grows, so this call cannot lower the limit a
  // context launches the same kernel with
  if (raise_smem_limit((const void*)k_mode, smem) != cudaSuccess) return PCF_ECUDA;
  k_noalloc_setup_shared<<<1, 256, 0, s>>>(I, base, L, prm->Lx, prm->Lz);
  k_noalloc_setup_modes<<<(nm + 127) / 128, 128, 0, s>>>(base, L, N, Mx, Mz, I.sigma[0]);
  const int ctas = (nm + mpc - 1) / mpc;
  // the prefix over the one instance is {0}; LaunchInfo reads prefix[0] only
  LaunchInfo li{reinterpret_cast<const Inst*>(base + L.inst), reinterpret_cast<const int*>(base + L.prefix), 1};
  k_mode<<<ctas, 128, smem, s>>>(li, MODE_SOLVE, 0, mpc, 0);
  if (cudaGetLastError() != cudaSuccess) return PCF_ECUDA;
  return PCF_OK;
}
