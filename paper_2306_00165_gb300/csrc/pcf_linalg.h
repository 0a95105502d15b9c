// Small dense linear algebra on the host for the DMD projected problem (r <= ~100).
//
// * svd_jacobi: one-sided (Hestenes) Jacobi SVD of an m x n real matrix, m >= n.
// * eig_general: eigenvalues and right eigenvectors of a real n x n matrix via complex
//   Householder reduction to Hessenberg form, single-shift QR iterations with Wilkinson
//   shifts and deflation (complex Schur form), and back substitution on the triangle.
// * lstsq_svd: minimum-norm least squares through svd_jacobi.
// All matrices are row-major std::vector<double> / std::vector<cd>.
#pragma once
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace pcf {
namespace la {

using cd = std::complex<double>;

// A = U diag(s) V^T; U: m x n (overwrites a copy of A), V: n x n, s sorted descending.
inline void svd_jacobi(int m, int n, const std::vector<double>& A, std::vector<double>& U, std::vector<double>& s,
                       std::vector<double>& V) {
  U = A;
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  const double eps = 1e-15;
  for (int sweep = 0; sweep < 80; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double a = 0, b = 0, c = 0;
        for (int i = 0; i < m; ++i) {
          const double up = U[(size_t)i * n + p], uq = U[(size_t)i * n + q];
          a += up * up;
          b += uq * uq;
          c += up * uq;
        }
        if (a == 0.0 || b == 0.0) continue;
        const double rel = std::fabs(c) / std::sqrt(a * b);
        off = std::max(off, rel);
        if (rel < eps) continue;
        const double zeta = (b - a) / (2.0 * c);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = cs * t;
        for (int i = 0; i < m; ++i) {
          const double up = U[(size_t)i * n + p], uq = U[(size_t)i * n + q];
          U[(size_t)i * n + p] = cs * up - sn * uq;
          U[(size_t)i * n + q] = sn * up + cs * uq;
        }
        for (int i = 0; i < n; ++i) {
          const double vp = V[(size_t)i * n + p], vq = V[(size_t)i * n + q];
          V[(size_t)i * n + p] = cs * vp - sn * vq;
          V[(size_t)i * n + q] = sn * vp + cs * vq;
        }
      }
    if (off < eps) break;
  }
  s.assign(n, 0.0);
  for (int j = 0; j < n; ++j) {
    double nn = 0;
    for (int i = 0; i < m; ++i) nn += U[(size_t)i * n + j] * U[(size_t)i * n + j];
    s[j] = std::sqrt(nn);
    if (s[j] > 0)
      for (int i = 0; i < m; ++i) U[(size_t)i * n + j] /= s[j];
  }
  // sort descending
  std::vector<int> idx(n);
  for (int j = 0; j < n; ++j) idx[j] = j;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return s[a] > s[b]; });
  std::vector<double> U2(U.size()), V2(V.size()), s2(n);
  for (int k = 0; k < n; ++k) {
    const int j = idx[k];
    s2[k] = s[j];
    for (int i = 0; i < m; ++i) U2[(size_t)i * n + k] = U[(size_t)i * n + j];
    for (int i = 0; i < n; ++i) V2[(size_t)i * n + k] = V[(size_t)i * n + j];
  }
  U.swap(U2);
  V.swap(V2);
  s.swap(s2);
}

// x = argmin |A x - b| (minimum norm), A: m x n.
inline std::vector<double> lstsq_svd(int m, int n, const std::vector<double>& A, const std::vector<double>& b) {
  std::vector<double> U, s, V;
  svd_jacobi(m, n, A, U, s, V);
  const double cut = (s.empty() ? 0.0 : s[0]) * 1e-14 * std::max(m, n);
  std::vector<double> y(n, 0.0), x(n, 0.0);
  for (int k = 0; k < n; ++k) {
    if (s[k] <= cut) continue;
    double d = 0;
    for (int i = 0; i < m; ++i) d += U[(size_t)i * n + k] * b[i];
    y[k] = d / s[k];
  }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) x[i] += V[(size_t)i * n + k] * y[k];
  return x;
}

// Eigen-decomposition of a real n x n matrix A: lam[k], W[:, k] (row-major n x n, unit columns).
inline bool eig_general(int n, const std::vector<double>& A, std::vector<cd>& lam, std::vector<cd>& W) {
  std::vector<cd> H((size_t)n * n), Z((size_t)n * n, cd(0.0));
  for (size_t i = 0; i < H.size(); ++i) H[i] = A[i];
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
  auto h = [&](int i, int j) -> cd& { return H[(size_t)i * n + j]; };
  auto z = [&](int i, int j) -> cd& { return Z[(size_t)i * n + j]; };
  // Householder reduction to upper Hessenberg form: H <- P H P, Z <- Z P
  for (int k = 0; k + 2 < n; ++k) {
    double xn = 0;
    for (int i = k + 1; i < n; ++i) xn += std::norm(h(i, k));
    xn = std::sqrt(xn);
    if (xn == 0.0) continue;
    const cd x0 = h(k + 1, k);
    const cd ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1.0);
    std::vector<cd> v(n, 0.0);
    for (int i = k + 1; i < n; ++i) v[i] = h(i, k);
    v[k + 1] += ph * xn;
    double vn = 0;
    for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
    if (vn == 0.0) continue;
    // P = I - 2 v v^H / (v^H v)
    for (int j = 0; j < n; ++j) {  // H <- P H
      cd d = 0;
      for (int i = k + 1; i < n; ++i) d += std::conj(v[i]) * h(i, j);
      d *= 2.0 / vn;
      for (int i = k + 1; i < n; ++i) h(i, j) -= v[i] * d;
    }
    for (int i = 0; i < n; ++i) {  // H <- H P, Z <- Z P
      cd d = 0, e = 0;
      for (int j = k + 1; j < n; ++j) {
        d += h(i, j) * v[j];
        e += z(i, j) * v[j];
      }
      d *= 2.0 / vn;
      e *= 2.0 / vn;
      for (int j = k + 1; j < n; ++j) {
        h(i, j) -= d * std::conj(v[j]);
        z(i, j) -= e * std::conj(v[j]);
      }
    }
    for (int i = k + 2; i < n; ++i) h(i, k) = 0.0;
  }
  // shifted QR iterations on the Hessenberg matrix
  int hi = n - 1, iter = 0;
  const double eps = 2.2e-16;
  while (hi > 0) {
    if (++iter > 100 * n) return false;
    int lo = hi;
    while (lo > 0) {
      const double sc = std::abs(h(lo, lo)) + std::abs(h(lo - 1, lo - 1));
      if (std::abs(h(lo, lo - 1)) <= eps * (sc > 0 ? sc : 1.0)) {
        h(lo, lo - 1) = 0.0;
        break;
      }
      --lo;
    }
    if (lo == hi) {
      --hi;
      iter = 0;
      continue;
    }
    // Wilkinson shift from the trailing 2x2 of the active block
    const cd a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
    const cd tr = a + d, det = a * d - b * c;
    const cd disc = std::sqrt(tr * tr - 4.0 * det);
    cd mu1 = 0.5 * (tr + disc), mu2 = 0.5 * (tr - disc);
    cd mu = std::abs(mu1 - d) < std::abs(mu2 - d) ? mu1 : mu2;
    if (iter % 11 == 10) mu = d + cd(std::abs(h(hi, hi - 1)), 0.0);  // exceptional shift
    // QR step on rows/cols lo..hi with Givens rotations
    std::vector<cd> cs(n), sn(n);
    for (int i = lo; i <= hi; ++i) h(i, i) -= mu;
    for (int k = lo; k < hi; ++k) {
      const cd x = h(k, k), y = h(k + 1, k);
      const double r = std::sqrt(std::norm(x) + std::norm(y));
      cd c_, s_;
      if (r == 0.0) { c_ = 1.0; s_ = 0.0; }
      else { c_ = x / r; s_ = y / r; }
      cs[k] = c_;
      sn[k] = s_;
      // rows k, k+1 <- G^H [row k; row k+1], G = [c -conj(s); s conj(c)]
      for (int j = k; j < n; ++j) {
        const cd hk = h(k, j), hk1 = h(k + 1, j);
        h(k, j) = std::conj(c_) * hk + std::conj(s_) * hk1;
        h(k + 1, j) = -s_ * hk + c_ * hk1;
      }
    }
    for (int k = lo; k < hi; ++k) {
      const cd c_ = cs[k], s_ = sn[k];
      // columns k, k+1 <- [col k, col k+1] G
      for (int i = 0; i <= std::min(hi, k + 2); ++i) {
        const cd hk = h(i, k), hk1 = h(i, k + 1);
        h(i, k) = hk * c_ + hk1 * s_;
        h(i, k + 1) = -hk * std::conj(s_) + hk1 * std::conj(c_);
      }
      for (int i = 0; i < n; ++i) {
        const cd zk = z(i, k), zk1 = z(i, k + 1);
        z(i, k) = zk * c_ + zk1 * s_;
        z(i, k + 1) = -zk * std::conj(s_) + zk1 * std::conj(c_);
      }
    }
    for (int i = lo; i <= hi; ++i) h(i, i) += mu;
  }
  // the rows above the active window were not rotated on the right beyond k+2; finish
  // the upper triangle consistently by recomputing T = Z^H A Z
  std::vector<cd> T((size_t)n * n, 0.0), AZ((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const double aik = A[(size_t)i * n + k];
      if (aik == 0.0) continue;
      for (int j = 0; j < n; ++j) AZ[(size_t)i * n + j] += aik * z(k, j);
    }
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const cd zc = std::conj(z(k, i));
      for (int j = i; j < n; ++j) T[(size_t)i * n + j] += zc * AZ[(size_t)k * n + j];
    }
  lam.assign(n, 0.0);
  for (int i = 0; i < n; ++i) lam[i] = T[(size_t)i * n + i];
  // eigenvectors of the triangle by back substitution, then W = Z Y
  std::vector<cd> Y((size_t)n * n, 0.0);
  double tnorm = 0;
  for (const cd& t : T) tnorm = std::max(tnorm, std::abs(t));
  const double small = eps * (tnorm > 0 ? tnorm : 1.0);
  for (int k = 0; k < n; ++k) {
    Y[(size_t)k * n + k] = 1.0;
    for (int i = k - 1; i >= 0; --i) {
      cd s = 0;
      for (int j = i + 1; j <= k; ++j) s += T[(size_t)i * n + j] * Y[(size_t)j * n + k];
      cd den = T[(size_t)i * n + i] - lam[k];
      if (std::abs(den) < small) den = small;
      Y[(size_t)i * n + k] = -s / den;
    }
  }
  W.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      cd s = 0;
      for (int j = 0; j <= k; ++j) s += z(i, j) * Y[(size_t)j * n + k];
      W[(size_t)i * n + k] = s;
    }
  for (int k = 0; k < n; ++k) {
    double nn = 0;
    for (int i = 0; i < n; ++i) nn += std::norm(W[(size_t)i * n + k]);
    nn = std::sqrt(nn);
    if (nn > 0)
      for (int i = 0; i < n; ++i) W[(size_t)i * n + k] /= nn;
  }
  return true;
}

// Solve the complex n x n system M x = b by Gaussian elimination with partial pivoting.
inline bool csolve(int n, std::vector<cd> M, std::vector<cd>& b) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::abs(M[(size_t)i * n + k]) > std::abs(M[(size_t)piv * n + k])) piv = i;
    if (std::abs(M[(size_t)piv * n + k]) == 0.0) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(M[(size_t)k * n + j], M[(size_t)piv * n + j]);
      std::swap(b[k], b[piv]);
    }
    for (int i = k + 1; i < n; ++i) {
      const cd f = M[(size_t)i * n + k] / M[(size_t)k * n + k];
      for (int j = k; j < n; ++j) M[(size_t)i * n + j] -= f * M[(size_t)k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    cd s = b[i];
    for (int j = i + 1; j < n; ++j) s -= M[(size_t)i * n + j] * b[j];
    b[i] = s / M[(size_t)i * n + i];
  }
  return true;
}

}  // namespace la
}  // namespace pcf
