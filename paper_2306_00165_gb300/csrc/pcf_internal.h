// Internal declarations of the pcfadj library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pcfadj.h"

#define PCF_HD __host__ __device__ __forceinline__

namespace pcf {

constexpr int kMaxRadix = 8;     // max number of FFT stages
constexpr int kFieldsSynth = 11; // u v w u_x u_y u_z v_x v_z w_x w_y w_z (v_y = -u_x - w_z)
constexpr int kFieldsY = 5;      // y-values V_u V_v V_w and y-derivative values W_u W_w
constexpr int kNumKernelClasses = 14;

// ------------------------------------------------------------------ table layout
// Chebyshev index n runs 0..N (N = ny - 1, even).  A parity class par holds the
// coefficients n = par + 2i, i = 0..Mc(par)-1, Mc(0) = N/2 + 1, Mc(1) = N/2.
// Per-mode solver table (one per step size sigma), doubles:
//   for op in {0: Poisson (lambda = k^2), 1: Helmholtz (lambda = sigma + k^2)}
//     for par in {0, 1}: c[Mh], inv[Mh], beta[Mh], B[Mh], invSumB, pad
//   for group g in {0: A (v even, tau at T_N), 1: B (v odd, tau at T_{N-1})}
//     vh1[Mh], vh2[Mh], Zinv[4]
// Mh = N/2 + 1.
struct TabLayout {
  int N, Mh;
  PCF_HD TabLayout(int N_) : N(N_), Mh(N_ / 2 + 1) {}
  PCF_HD int solver(int op, int par) const { return (op * 2 + par) * (4 * Mh + 2); }
  PCF_HD int group(int g) const { return 4 * (4 * Mh + 2) + g * (2 * Mh + 4); }
  PCF_HD int per_mode() const { return 4 * (4 * Mh + 2) + 2 * (2 * Mh + 4); }
};

// Dense form of the same per-mode solve (used for N <= kDenseMaxN): for each parity group g
// three Mh x Mh column-major blocks (element (r, j) at block + j Mh + r, so that threads
// computing consecutive rows read consecutive addresses) mapping the group's inputs to its outputs,
//   v  = Av f_v + Ag g,   eta = Eh h,
// with f_v the v right-hand side (class g), g = Re/Im part of i(kx f_u + kz f_w) and
// h = Re/Im part of i(kz f_u - kx f_w) (class 1-g).  For the mean mode, Eh of group g is
// the inverse Dirichlet Helmholtz operator of class g (applied to f_u and f_w).
// xi = -dv/dy follows from v by the derivative recurrence (xi_from_v), the step of the
// banded sweeps.
constexpr int kDenseMaxN = 128;
struct DenseLayout {
  int Mh;
  enum { kAv = 0, kAg = 1, kEh = 2 };
  PCF_HD DenseLayout(int N) : Mh(N / 2 + 1) {}
  PCF_HD int block(int g, int k) const { return (g * 3 + k) * Mh * Mh; }
  PCF_HD int at(int g, int k, int r, int j) const { return block(g, k) + j * Mh + r; }
  PCF_HD int per_mode() const { return 6 * Mh * Mh; }
};

// Shared (N-dependent) coefficient table, doubles, each array of length Mh:
//   for par: ra, rb, rc (tau right-hand-side combination), nsq (n^2 of the class
//   element), two_n (2 n of the class element)
struct RcoLayout {
  int Mh;
  PCF_HD RcoLayout(int N) : Mh(N / 2 + 1) {}
  PCF_HD int off(int par, int k) const { return (par * 5 + k) * Mh; }
  PCF_HD int total() const { return 10 * Mh; }
};

// Parity-folded Chebyshev matrices (doubles), H = N/2 + 1 rows (j = 0..N/2):
//   Ce[j][k] = T_{2k}(y_j)        k < H         (values from even coefficients)
//   Co[j][k] = T_{2k+1}(y_j)      k < H-1
//   De[j][k] = T'_{2k}(y_j)       k < H
//   Do[j][k] = T'_{2k+1}(y_j)     k < H-1
//   Ae[k][j] = Cinv_{2k, j}        j < H  (coefficients from folded sums P_j)
//   Ao[k][j] = Cinv_{2k+1, j}      j < H  (coefficients from folded differences Q_j)
struct ChebLayout {
  int H;
  PCF_HD ChebLayout(int N) : H(N / 2 + 1) {}
  PCF_HD int Ce() const { return 0; }
  PCF_HD int Co() const { return H * H; }
  PCF_HD int De() const { return 2 * H * H; }
  PCF_HD int Do() const { return 3 * H * H; }
  PCF_HD int Ae() const { return 4 * H * H; }
  PCF_HD int Ao() const { return 5 * H * H; }
  PCF_HD int total() const { return 6 * H * H; }
};

// ------------------------------------------------------------------ instance descriptor
struct Inst {
  int nx, ny, nz, N, Kx, Kz, Mx, Mz, nmodes;
  int mpc;  // Fourier modes per CTA of the mode kernel (0: use the launch argument)
  int nrx, nrz;
  int rx[kMaxRadix], rz[kMaxRadix];
  double nu, dt, dtau_hat, dtau, inv_nxnz, tol;
  double inv_nu, inv_dt, inv_dtau_hat;  // 1/nu, 1/dt, 1/dtau_hat (IEEE quotients, set on the host)
  // tables (device)
  const double* cheb;
  const float2* cheb_ff;  // the same table as float-float pairs (hi, lo), for the float-float form
  const double* rco;
  const double* ygrid;
  const double* ubase;  // [3][ny]: base-flow profile U(y_j), U'(y_j) and the constant V
  const double* ccw;
  const double* kx;   // [Mx]
  const double* kz;   // [Mz]
  const double2* twx; // e^{-2 pi i k/nx}, k < nx
  const double2* twz; // e^{-2 pi i k/nz}, k < nz
  const double2* tanx;        // [2][nx] tangent-form twiddles (t, m) of the FP64 plane FFTs:
  const double2* tanz;        //   forward, then inverse; see TwTan
  const unsigned char* rotx;  // [nx] their rotation flags (|sin| > |cos|)
  const unsigned char* rotz;  // [nz]
  const float2* twxf; // FP32 copies for the mixed-precision form
  const float2* twzf;
  const double* tab[2];  // per-mode solver tables: [0] sigma = 1/(nu dt), [1] sigma = 1/(nu dtau_hat)
  const double* dense[2];  // per-mode dense solve operators (DenseLayout) or null
  double sigma[2];
  // buffers (device), uhat layout unless noted
  double2* uhat;
  double2* rhat;
  double2* fhat;
  double2* yv;        // [2][5][ny][Mx][Mz]: slot 0 for u, slot 1 for q
  double* phys;       // [2][11][ny][nx][nz]: slot 0 for u, slot 1 for q
  double2* xz;        // [3][ny][Mx][Mz]
  double* normpart;   // [3][ny]
  double* frg;        // [nmodes][3][2][N + 2]: class-split Stokes right-hand sides (FP64 split mode kernels)
  // mixed-precision form: FP32 plane data and Chebyshev coefficients of the products
  float* physf;       // [2][11][ny][nx][nz]
  float2* yvf;        // [2][5][ny][Mx][Mz]
  float2* xzf;        // [3][ny][Mx][Mz]
  float2* xzc;        // [3][ny][Mx][Mz]: Chebyshev coefficients of xzf (n in place of j)
  int mixed;          // 1: the mode kernel reads xzc and leaves the synthesis to the tensor-core kernel
  const void* tcA;    // bf16 [6][P][P], P = ny rounded up to 16: C hi/lo, C' hi/lo, Cinv hi/lo
  const void* tcA5;   // the same as [6] shared-memory images of the tcgen05 kernel's A region
                      // (128 x P, core-matrix layout); null when P > 128
  double* hist;       // J history base (may be null)
  int hist_stride;
  int* active;        // 1 = keep updating
  int sym;            // symmetry mask enforced on this instance (pcf_symmetry bits)
  int* jcount;        // CTAs of the adjoint product kernel done with their plane sums (zero between launches)
};

// ------------------------------------------------------------------ quasi-tridiagonal tau solver
// Solves (lambda - D^2) y = r on Chebyshev rows 0..N-2 for the parity class par, with
// the class boundary row sum_{class} y_n = bc, using the precomputed sweep
// coefficients of (lambda, par).  r and y are class arrays (element i <-> n = par+2i);
// r is read at i-1, i, i+1.  y may alias scratch but not r.
// Row i >= 1 (n = par + 2i) is the Chebyshev identity
//   y_n = c_{n-2} z_{n-2}/(4n(n-1)) - e_n z_n/(2(n^2-1)) + e_{n+2} z_{n+2}/(4n(n+1)),
// z = D^2 y = lambda y - r on rows <= N-2 (e_m = [m <= N-2]).
PCF_HD void tau_solve(int Mc, const double* __restrict__ c, const double* __restrict__ inv,
                      const double* __restrict__ beta, const double* __restrict__ B, double invSumB,
                      const double* __restrict__ ra, const double* __restrict__ rb,
                      const double* __restrict__ rc, const double* r, double bc, double* y) {
  // backward sweep: alpha_i = (rhs_i - c_i alpha_{i+1}) inv_i, stored in y[i]
  double alpha = 0.0;
  for (int i = Mc - 1; i >= 1; --i) {
    double rhs = ra[i] * r[i - 1] + rb[i] * r[i];
    if (i + 1 < Mc) rhs += rc[i] * r[i + 1];
    alpha = (rhs - c[i] * alpha) * inv[i];
    y[i] = alpha;
  }
  // forward: A_i = alpha_i + beta_i A_{i-1}
  double A = 0.0, sumA = 0.0;
  for (int i = 1; i < Mc; ++i) {
    A = y[i] + beta[i] * A;
    y[i] = A;
    sumA += A;
  }
  const double y0 = (bc - sumA) * invSumB;
  y[0] = y0;
  for (int i = 1; i < Mc; ++i) y[i] += B[i] * y0;
}

// Derivative of a class array a (parity q) into class array d (parity 1-q):
// (D a)_n = (D a)_{n+2} + 2 (n+1) a_{n+1}; (D a)_0 halved.  two_n holds 2n for a's
// class elements (n = q + 2i).  Degree of D a is N-1: for q = 0 the top of the odd
// class (n = N-1) is 2N a_N; for q = 1 the even class top (n = N) is 0.
PCF_HD void class_deriv(int N, int q, const double* __restrict__ a, const double* __restrict__ two_n,
                        double* __restrict__ d) {
  // d's class parity p = 1 - q; element j <-> n = p + 2j; needs a_{n+1} -> a index (n+1-q)/2
  const int p = 1 - q;
  const int Md = (N - p) / 2 + 1;
  double acc = 0.0;
  for (int j = Md - 1; j >= 0; --j) {
    const int n = p + 2 * j;
    if (n + 1 <= N) acc += two_n[(n + 1 - q) / 2] * a[(n + 1 - q) / 2];
    d[j] = acc;
  }
  if (p == 0) d[0] *= 0.5;
}

// xi = -dv/dy from the class array v (parity pv, stride vs) into the class array xi (parity
// 1 - pv, stride xs): class_deriv's recurrence with the sign carried in the accumulator,
// nacc = -acc (fma(-c, v, nacc) = -fma(c, v, acc) exactly), so that each step is one FMA on
// the dependent chain; two_n holds 2n for v's class elements (RcoLayout off(pv, 4)).  The
// results are those of class_deriv followed by the sign.
PCF_HD void xi_from_v(int N, int pv, const double* __restrict__ v, int vs, double* __restrict__ xi, int xs,
                      const double* __restrict__ two_n) {
  const int p = 1 - pv;
  const int Md = (N - p) / 2 + 1;
  double nacc = 0.0;
  for (int j = Md - 1; j >= 0; --j) {
    const int n = p + 2 * j;
    if (n + 1 <= N) {
      const int i = (n + 1 - pv) / 2;
      nacc = fma(-two_n[i], v[i * vs], nacc);
    }
    xi[j * xs] = nacc;
  }
  if (p == 0) xi[0] = nacc * 0.5;
}

// One chain of the per-mode Stokes solve: group g (v parity g), real (rho = 0) or
// imaginary (rho = 1) part.  Fr: mode right-hand side [3][2][L2] class-split.
// Writes V (class g, v), XI = -dv/dy and ETA (class 1-g) into scratch.
PCF_HD void mode_chain(int N, int g, int rho, double kx, double kz, double lamH, const double* tab,
                           const double* rco, const double* Fr, int L2, double* scratch) {
  const int Mh = N / 2 + 1;
  const TabLayout TL(N);
  const RcoLayout RL(N);
  const int pv = g, pP = 1 - g;
  const int McP = (N - pP) / 2 + 1, McV = (N - pv) / 2 + 1;
  double* P = scratch;
  double* T = scratch + Mh;
  double* V = scratch + 2 * Mh;
  double* XI = scratch + 3 * Mh;
  double* ETA = scratch + 4 * Mh;
  double* R2 = scratch + 5 * Mh;
  const double* fu_o = Fr + (0 * 2 + (1 - rho)) * L2 + pP * Mh;  // other part of f_u, class pP
  const double* fw_o = Fr + (2 * 2 + (1 - rho)) * L2 + pP * Mh;
  const double* fv = Fr + (1 * 2 + rho) * L2 + pv * Mh;          // this part of f_v, class pv
  // Poisson right-hand side -(D f_v + i kx f_u + i kz f_w), this part, class pP
  class_deriv(N, pv, fv, rco + RL.off(pv, 4), T);
  const double sgn = rho == 0 ? -1.0 : 1.0;  // Re(i a) = -Im a, Im(i a) = Re a
  for (int i = 0; i < McP; ++i) R2[i] = -(T[i] + sgn * fma(kx, fu_o[i], kz * fw_o[i]));
  const double* s = tab + TL.solver(0, pP);
  tau_solve(McP, s, s + Mh, s + 2 * Mh, s + 3 * Mh, s[4 * Mh], rco + RL.off(pP, 0), rco + RL.off(pP, 1),
            rco + RL.off(pP, 2), R2, 0.0, P);
  // v: (sigma + k^2 - D^2) v = f_v - D P, v(+-1) = 0
  class_deriv(N, pP, P, rco + RL.off(pP, 4), T);
  for (int i = 0; i < McV; ++i) R2[i] = fv[i] - T[i];
  s = tab + TL.solver(1, pv);
  tau_solve(McV, s, s + Mh, s + 2 * Mh, s + 3 * Mh, s[4 * Mh], rco + RL.off(pv, 0), rco + RL.off(pv, 1),
            rco + RL.off(pv, 2), R2, 0.0, V);
  // influence-matrix conditions: dv/dy(1) = 0 and the tau consistency of the v equation
  const double* nsq = rco + RL.off(pv, 3);
  double F1 = 0.0;
  for (int i = 0; i < McV; ++i) F1 = fma(nsq[i], V[i], F1);
  double F2 = lamH * V[McV - 1] - fv[McV - 1];
  if (g == 1) F2 += 2.0 * N * P[McP - 1];
  const double* gt = tab + TL.group(g);
  const double* Zi = gt + 2 * Mh;
  const double c1 = -fma(Zi[0], F1, Zi[1] * F2);
  const double c2 = -fma(Zi[2], F1, Zi[3] * F2);
  for (int i = 0; i < McV; ++i) V[i] = fma(c1, gt[i], fma(c2, gt[Mh + i], V[i]));
  // xi = -dv/dy (class pP)
  class_deriv(N, pv, V, rco + RL.off(pv, 4), XI);
  for (int i = 0; i < McP; ++i) XI[i] = -XI[i];
  // eta = i kz u - i kx w: (sigma + k^2 - D^2) eta = i kz f_u - i kx f_w, eta(+-1) = 0
  for (int i = 0; i < McP; ++i) R2[i] = sgn * fma(kz, fu_o[i], -kx * fw_o[i]);
  s = tab + TL.solver(1, pP);
  tau_solve(McP, s, s + Mh, s + 2 * Mh, s + 3 * Mh, s[4 * Mh], rco + RL.off(pP, 0), rco + RL.off(pP, 1),
            rco + RL.off(pP, 2), R2, 0.0, ETA);
}

}  // namespace pcf
