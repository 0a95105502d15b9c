// Symmetric-subspace projection (§5.1) and the helper kernels of the direct numerical
// simulation that produces guesses (§5.2).
#include "pcf_kernels.cuh"

namespace pcf {

// ------------------------------------------------------------------ symmetric subspace
// Group average over the symmetries of mask (bit 0: s1, bit 1: s2) of §5.1,
//   s1 [u,v,w](x,y,z) = [-u,-v,w](-x + Lx/2, -y, z + Lz/2),
//   s2 [u,v,w](x,y,z) = [u,v,-w](x + Lx/2, y, -z).
// On the coefficients of component c at x-mode m, z-mode p, Chebyshev index n (x -> -x maps
// m to -m, y -> -y multiplies T_n by (-1)^n, a shift by L/2 multiplies mode m by (-1)^m,
// z -> -z maps p to -p, i.e. to the conjugate of mode -m):
//   (s1 a)_{m,p,n}    = e1_c (-1)^(m+p+n) a_{-m,p,n},   e1 = (-1, -1, +1)
//   (s2 a)_{m,p,n}    = e2_c (-1)^m conj(a_{-m,p,n}),   e2 = (+1, +1, -1)
//   (s1 s2 a)_{m,p,n} = -(-1)^(p+n) conj(a_{m,p,n}).
// One thread per (c, m >= 0, p, n) reads modes m and -m and writes both, in place.
// mask_override >= 0 replaces every instance's own mask (I.sym); inactive instances
// (converged, I.active == 0) are left alone.
// reduced (every mask contains s2; the descent updated the modes m >= 0 only): mode -m is
// rebuilt from mode m by the s2 relation instead of averaged with it, and with s1 as well
// mode m is first projected by its own s1 s2 relation, a <- (a + s1 s2 a)/2.
__global__ void __launch_bounds__(256) k_symmetrize(const Inst* insts, int mask_override, int reduced) {
  const Inst& I = insts[blockIdx.y];
  const int mask = mask_override >= 0 ? mask_override : I.sym;
  if (mask == 0 || !inst_active(I)) return;
  const int ny = I.ny, Mz = I.Mz, Mx = I.Mx;
  const int per_i = Mz * ny, per_c = (I.Kx + 1) * per_i;
  const double scale = mask == 3 ? 0.25 : 0.5;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * per_c; t += gridDim.x * blockDim.x) {
    const int c = t / per_c;
    int r = t - c * per_c;
    const int i = r / per_i;  // storage index of m = i (0 <= m <= Kx)
    r -= i * per_i;
    const int p = r / ny, n = r - p * ny;
    const int im = i == 0 ? 0 : Mx - i;  // storage index of -m
    double2* base = I.uhat + (size_t)c * Mx * per_i;
    const size_t ka = (size_t)i * per_i + (size_t)p * ny + n;
    const size_t kb = (size_t)im * per_i + (size_t)p * ny + n;
    const double2 a = base[ka], b = base[kb];
    const double sm = (i & 1) ? -1.0 : 1.0;           // (-1)^m
    const double spn = ((p + n) & 1) ? -1.0 : 1.0;    // (-1)^(p+n)
    const double e1 = c == 2 ? 1.0 : -1.0, e2 = -e1;
    const double f1 = e1 * sm * spn, f2 = e2 * sm;
    double2 oa, ob;
    if (reduced && i > 0) {
      if (mask == 3) oa = make_double2(0.5 * (a.x - spn * a.x), 0.5 * (a.y + spn * a.y));
      else oa = a;
      base[ka] = oa;
      base[kb] = make_double2(f2 * oa.x, -f2 * oa.y);
      continue;
    }
    if (mask == 1) {
      oa = make_double2(a.x + f1 * b.x, a.y + f1 * b.y);
      ob = make_double2(b.x + f1 * a.x, b.y + f1 * a.y);
    } else if (mask == 2) {
      oa = make_double2(a.x + f2 * b.x, a.y - f2 * b.y);
      ob = make_double2(b.x + f2 * a.x, b.y - f2 * a.y);
    } else {
      oa = make_double2((a.x + f1 * b.x) + (f2 * b.x - spn * a.x), (a.y + f1 * b.y) + (spn * a.y - f2 * b.y));
      ob = make_double2((b.x + f1 * a.x) + (f2 * a.x - spn * b.x), (b.y + f1 * a.y) + (spn * b.y - f2 * a.y));
    }
    base[ka] = make_double2(scale * oa.x, scale * oa.y);
    if (kb != ka) base[kb] = make_double2(scale * ob.x, scale * ob.y);
  }
}

int symmetrize_ctas(const Inst& I) {
  const int n = 3 * (I.Kx + 1) * I.Mz * I.ny;
  return (n + 255) / 256;
}

void launch_symmetrize(int ctas_x, int ninst, cudaStream_t s, const Inst* insts, int mask_override, int reduced) {
  k_symmetrize<<<dim3(ctas_x, ninst), 256, 0, s>>>(insts, mask_override, reduced);
}

// ------------------------------------------------------------------ DNS with the Stokes step
// h_s = ||u_s|| from the plane sums of u^2 (same arithmetic as the norm of r1), its history
// entry, and the discrete-extremum test of the previous step:
//   (h_{s-1} - h_{s-2}) (h_s - h_{s-1}) < 0  ->  u_{s-1} (held in uprev) is a guess.
// One CTA per instance; D.step counts the steps of the current call.
__global__ void __launch_bounds__(128) k_dns_norm(const Inst* insts, DnsInst* dns) {
  __shared__ double part[3 * 257];
  __shared__ double w[257];
  const Inst& I = insts[blockIdx.x];
  DnsInst& D = dns[blockIdx.x];
  const int ny = I.ny;
  for (int t = threadIdx.x; t < 3 * ny; t += blockDim.x) part[t] = I.normpart[t];
  for (int t = threadIdx.x; t < ny; t += blockDim.x) w[t] = I.ccw[t];
  __syncthreads();
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int j = 0; j < ny; ++j) s = fma(w[j], part[j] + part[ny + j] + part[2 * ny + j], s);
  const double h = sqrt(0.5 * I.inv_nxnz * s);
  const int step = D.step;
  if (D.hist) D.hist[(size_t)step * D.hist_stride] = h;
  int slot = -1;
  if (step >= 2 && (D.h1 - D.h2) * (h - D.h1) < 0.0) {
    const int k = *D.count;
    if (k < D.gmax) slot = k;
    *D.count = k + 1;
  }
  D.slot = slot;
  D.h2 = D.h1;
  D.h1 = h;
  D.step = step + 1;
}

// Copy uprev (u_{s-1}) into the instance's guess slot chosen by k_dns_norm.
__global__ void __launch_bounds__(256) k_dns_capture(const Inst* insts, const DnsInst* dns) {
  const DnsInst& D = dns[blockIdx.y];
  if (D.slot < 0 || !D.guess) return;
  const Inst& I = insts[blockIdx.y];
  const int n = 3 * I.nmodes * I.ny;
  double2* dst = D.guess + (size_t)D.slot * D.gstride;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) dst[t] = D.uprev[t];
}

// uprev <- u, then u <- u + dt r1 = u^dt (the Stokes step of §4 step 1 as a time stepper).
__global__ void __launch_bounds__(256) k_dns_update(const Inst* insts, const DnsInst* dns) {
  const Inst& I = insts[blockIdx.y];
  const DnsInst& D = dns[blockIdx.y];
  const int n = 3 * I.nmodes * I.ny;
  const double dt = I.dt;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const double2 u = I.uhat[t], r = I.rhat[t];
    D.uprev[t] = u;
    I.uhat[t] = make_double2(fma(dt, r.x, u.x), fma(dt, r.y, u.y));
  }
}

int dns_ctas(const Inst& I) {
  const int n = 3 * I.nmodes * I.ny;
  return (n + 255) / 256;
}

void launch_dns_norm(int ninst, cudaStream_t s, const Inst* insts, DnsInst* dns) {
  k_dns_norm<<<ninst, 128, 0, s>>>(insts, dns);
}
void launch_dns_capture(int ctas_x, int ninst, cudaStream_t s, const Inst* insts, const DnsInst* dns) {
  k_dns_capture<<<dim3(ctas_x, ninst), 256, 0, s>>>(insts, dns);
}
void launch_dns_update(int ctas_x, int ninst, cudaStream_t s, const Inst* insts, const DnsInst* dns) {
  k_dns_update<<<dim3(ctas_x, ninst), 256, 0, s>>>(insts, dns);
}

}  // namespace pcf
