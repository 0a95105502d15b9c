// Stokes step of the descent (§4 steps 1 and 4: the Stokes operator with the influence-matrix
// correction) by banded Chebyshev-tau sweeps, one thread per chain.
//
// A chain is (instance, parity group g, Fourier mode m, part rho): the Poisson problem for the
// pressure, the Helmholtz problem for v with the 2x2 influence-matrix correction, xi = -dv/dy,
// and the Helmholtz problem for eta, each a quasi-tridiagonal tau system solved by one
// backward and one forward sweep (the same sequence as the per-mode kernel's banded variant).
// A sweep is a serial chain of FP64 operations, but the chains are independent: lanes 2k and
// 2k+1 of a warp hold the two parts of one (g, m), and a warp holds 16 consecutive modes of
// one group, so all 32 lanes run the same instruction sequence.  Per element of a chain about
// 38 FP64 operations are issued, against 12 Mh multiply-adds per row of the dense per-mode
// operators.
//
// Each lane's scratch (four class arrays of Mh doubles) lives in shared memory as columns of a
// [Mh][T] array (element i of lane l at i T + l), so the lanes of a warp touch consecutive
// words.  The right-hand sides are read where the analysis kernel left them (class-split,
// [3][2][N+2] per mode), the per-mode sweep coefficients from the mode table of the step
// size, and the results are assembled into r1 (Stokes step of the NSE) or into the update of
// u (Stokes step of the dummy dynamics), as the dense solve kernel does.
#include "pcf_kernels.cuh"

namespace pcf {

namespace {

// Quasi-tridiagonal tau solve of one class (see tau_solve): r read at stride RS, y written
// at stride YS.  The multiply-adds are written out as fma so that every lane and every build
// rounds the same way.
template <int RS, int YS>
__device__ __forceinline__ void sweep_tau(int Mc, const double* __restrict__ s, int Mh,
                                          const double* __restrict__ ra, const double* __restrict__ rb,
                                          const double* __restrict__ rc, const double* r, double* y) {
  const double* c = s;
  const double* inv = s + Mh;
  const double* beta = s + 2 * Mh;
  const double* B = s + 3 * Mh;
  const double invSumB = s[4 * Mh];
  double alpha = 0.0;
  // i = Mc - 1 has no r[i + 1] term (Mc >= 4 on every accepted grid)
  if (Mc > 1) {
    const int i = Mc - 1;
    const double rhs = fma(rb[i], r[i * RS], ra[i] * r[(i - 1) * RS]);
    alpha = fma(-c[i], alpha, rhs) * inv[i];
    y[i * YS] = alpha;
  }
#pragma unroll 4
  for (int i = Mc - 2; i >= 1; --i) {
    const double rhs = fma(rc[i], r[(i + 1) * RS], fma(rb[i], r[i * RS], ra[i] * r[(i - 1) * RS]));
    alpha = fma(-c[i], alpha, rhs) * inv[i];
    y[i * YS] = alpha;
  }
  double A = 0.0, sumA = 0.0;
#pragma unroll 4
  for (int i = 1; i < Mc; ++i) {
    A = fma(beta[i], A, y[i * YS]);
    y[i * YS] = A;
    sumA += A;
  }
  const double y0 = -sumA * invSumB;  // boundary row: the class sums to zero
  y[0] = y0;
#pragma unroll 4
  for (int i = 1; i < Mc; ++i) y[i * YS] = fma(B[i], y0, y[i * YS]);
}

// Derivative of the class array a (parity q, stride AS) into the class array d (parity 1 - q,
// stride DS), as class_deriv; NEG stores -(D a) (the sign carried in the accumulator).
template <int AS, int DS, bool NEG>
__device__ __forceinline__ void sweep_deriv(int N, int q, const double* a, const double* __restrict__ two_n,
                                            double* d) {
  const int p = 1 - q;
  const int Md = (N - p) / 2 + 1;
  double acc = 0.0;
  int j = Md - 1;
  if (p + 2 * j + 1 > N) {  // the top element of the class of D a has no a_{n+1}
    d[j * DS] = 0.0;
    --j;
  }
#pragma unroll 4
  for (; j >= 0; --j) {
    acc = fma(NEG ? -two_n[j + p] : two_n[j + p], a[(j + p) * AS], acc);  // a_{n+1}, n = p + 2j
    d[j * DS] = acc;
  }
  if (p == 0) d[0] = acc * 0.5;
}

template <int T, int OP>
__global__ void __launch_bounds__(T) k_sweep(LaunchInfo li, int red) {
  extern __shared__ double sw[];
  int local;
  const int b = find_inst(li, blockIdx.x, &local);
  const Inst& I = li.insts[b];
  if (!inst_active(I)) return;
  const int lane = threadIdx.x;
  const int N = I.N, Mh = N / 2 + 1, L2 = 2 * Mh, ny = I.ny, nm = I.nmodes, Mz = I.Mz;
  const int nr = red ? (I.Kx + 1) * Mz : nm;  // reduced launch: the modes m >= 0
  const int q = local * T + lane;
  const bool valid = q < 4 * nr;
  const int rho = q & 1, gm = valid ? q >> 1 : 0, g = gm / nr, m = gm - g * nr;
  const int pv = g, pP = 1 - g, McV = (N - pv) / 2 + 1, McP = (N - pP) / 2 + 1;
  const int sig = OP == MODE_PHI ? 0 : 1;
  const TabLayout TL(N);
  const RcoLayout RL(N);
  // scratch columns of this lane: R2, T (later xi), P (later eta), V
  double* R2 = sw + lane;
  double* Tx = R2 + Mh * T;
  double* Pe = Tx + Mh * T;
  double* V = Pe + Mh * T;
  const int ix = m / Mz, p = m - ix * Mz;
  const double kx = I.kx[ix], kz = I.kz[p];
  const bool mean = m == 0;
  const double* tab = I.tab[sig] + (size_t)m * TL.per_mode();
  const double* rco = I.rco;
  const double* Fr = I.frg + (size_t)m * 6 * L2;
  if (valid) {
    if (mean) {
      // mean mode: v = 0; Dirichlet Helmholtz problems for u (into P) and w (into V), class g
      const int Mc = (N - g) / 2 + 1;
      const double* s = tab + TL.solver(1, g);
      sweep_tau<1, T>(Mc, s, Mh, rco + RL.off(g, 0), rco + RL.off(g, 1), rco + RL.off(g, 2),
                      Fr + (0 * 2 + rho) * L2 + g * Mh, Pe);
      sweep_tau<1, T>(Mc, s, Mh, rco + RL.off(g, 0), rco + RL.off(g, 1), rco + RL.off(g, 2),
                      Fr + (2 * 2 + rho) * L2 + g * Mh, V);
    } else {
      const double* fu_o = Fr + (0 * 2 + (1 - rho)) * L2 + pP * Mh;  // other part of f_u, class pP
      const double* fw_o = Fr + (2 * 2 + (1 - rho)) * L2 + pP * Mh;
      const double* fv = Fr + (1 * 2 + rho) * L2 + pv * Mh;          // this part of f_v, class pv
      const double sgn = rho == 0 ? -1.0 : 1.0;                       // Re(i a) = -Im a, Im(i a) = Re a
      // Poisson: D^2 P - k^2 P = -(D f_v + i kx f_u + i kz f_w), class pP
      sweep_deriv<1, T, false>(N, pv, fv, rco + RL.off(pv, 4), Tx);
      for (int i = 0; i < McP; ++i) R2[i * T] = -(Tx[i * T] + sgn * fma(kx, fu_o[i], kz * fw_o[i]));
      const double* s = tab + TL.solver(0, pP);
      sweep_tau<T, T>(McP, s, Mh, rco + RL.off(pP, 0), rco + RL.off(pP, 1), rco + RL.off(pP, 2), R2, Pe);
      // v: (sigma + k^2 - D^2) v = f_v - D P, v(+-1) = 0
      sweep_deriv<T, T, false>(N, pP, Pe, rco + RL.off(pP, 4), Tx);
      for (int i = 0; i < McV; ++i) R2[i * T] = fv[i] - Tx[i * T];
      s = tab + TL.solver(1, pv);
      sweep_tau<T, T>(McV, s, Mh, rco + RL.off(pv, 0), rco + RL.off(pv, 1), rco + RL.off(pv, 2), R2, V);
      // influence matrix: dv/dy(+-1) = 0 and the tau consistency of the v equation
      const double* nsq = rco + RL.off(pv, 3);
      double F1 = 0.0;
      for (int i = 0; i < McV; ++i) F1 = fma(nsq[i], V[i * T], F1);
      const double lamH = I.sigma[sig] + (kx * kx + kz * kz);
      double F2 = fma(lamH, V[(McV - 1) * T], -fv[McV - 1]);
      if (g == 1) F2 = fma(2.0 * N, Pe[(McP - 1) * T], F2);
      const double* gt = tab + TL.group(g);
      const double* Zi = gt + 2 * Mh;
      const double c1 = -fma(Zi[0], F1, Zi[1] * F2);
      const double c2 = -fma(Zi[2], F1, Zi[3] * F2);
      for (int i = 0; i < McV; ++i) V[i * T] = fma(c1, gt[i], fma(c2, gt[Mh + i], V[i * T]));
      // xi = -dv/dy (class pP), into T's column
      sweep_deriv<T, T, true>(N, pv, V, rco + RL.off(pv, 4), Tx);
      // eta: (sigma + k^2 - D^2) eta = i kz f_u - i kx f_w, eta(+-1) = 0, into P's column
      for (int i = 0; i < McP; ++i) R2[i * T] = sgn * fma(kz, fu_o[i], -kx * fw_o[i]);
      s = tab + TL.solver(1, pP);
      sweep_tau<T, T>(McP, s, Mh, rco + RL.off(pP, 0), rco + RL.off(pP, 1), rco + RL.off(pP, 2), R2, Pe);
    }
  }
  __syncwarp();  // the partner lane's xi and eta
  if (!valid) return;
  const double inv_step = OP == MODE_PHI ? I.inv_dt : I.inv_dtau_hat;
  const auto put = [&](int comp, int n, double val) {
    const size_t gidx = ((size_t)comp * nm + m) * ny + n;
    double* rh = reinterpret_cast<double*>(I.rhat + gidx) + rho;
    double* uh = reinterpret_cast<double*>(I.uhat + gidx) + rho;
    if (OP == MODE_PHI) {
      *rh = (val - *uh) * inv_step;
    } else {
      const double f = -(val - *rh) * inv_step;
      *uh = fma(I.dtau, f, *uh);
    }
  };
  if (mean) {
    const int Mc = (N - g) / 2 + 1;
    for (int i = 0; i < Mc; ++i) {
      const int n = g + 2 * i;
      put(0, n, Pe[i * T]);
      put(1, n, 0.0);
      put(2, n, V[i * T]);
    }
    return;
  }
  for (int i = 0; i < McV; ++i) put(1, pv + 2 * i, V[i * T]);
  // u and w of class pP from the other part's xi and eta, as the dense solve assembles them
  const double ik2 = 1.0 / (kx * kx + kz * kz);
  const double* Xo = Tx + (rho == 0 ? 1 : -1);
  const double* Eo = Pe + (rho == 0 ? 1 : -1);
  for (int i = 0; i < McP; ++i) {
    const double xo = Xo[i * T], eo = Eo[i * T];
    double uu, ww;
    if (rho == 0) {
      uu = fma(kx, xo, kz * eo) * ik2;
      ww = fma(kz, xo, -kx * eo) * ik2;
    } else {
      uu = -fma(kx, xo, kz * eo) * ik2;
      ww = fma(-kz, xo, kx * eo) * ik2;
    }
    put(0, pP + 2 * i, uu);
    put(2, pP + 2 * i, ww);
  }
}

}  // namespace

// four scratch columns per lane
size_t smem_sweep(int N, int threads) { return sizeof(double) * 4 * (size_t)(N / 2 + 1) * threads; }

int sweep_ctas(int nmodes_run, int threads) { return (4 * nmodes_run + threads - 1) / threads; }

void launch_sweep(int ctas, int threads, size_t smem, cudaStream_t s, LaunchInfo li, int op, int red) {
  const bool phi = op == MODE_PHI;
  if (threads == 64) {
    if (phi) k_sweep<64, MODE_PHI><<<ctas, 64, smem, s>>>(li, red);
    else k_sweep<64, MODE_PSI_UPDATE><<<ctas, 64, smem, s>>>(li, red);
  } else {
    if (phi) k_sweep<32, MODE_PHI><<<ctas, 32, smem, s>>>(li, red);
    else k_sweep<32, MODE_PSI_UPDATE><<<ctas, 32, smem, s>>>(li, red);
  }
}

cudaError_t set_sweep_smem(size_t smem) {
  cudaError_t e;
  if ((e = raise_smem_limit((const void*)k_sweep<32, MODE_PHI>, smem))) return e;
  if ((e = raise_smem_limit((const void*)k_sweep<32, MODE_PSI_UPDATE>, smem))) return e;
  if ((e = raise_smem_limit((const void*)k_sweep<64, MODE_PHI>, smem))) return e;
  return raise_smem_limit((const void*)k_sweep<64, MODE_PSI_UPDATE>, smem);
}

}  // namespace pcf
