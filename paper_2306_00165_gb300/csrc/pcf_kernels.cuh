// Kernel entry points of the pcfadj library (declared for the host launcher).
#pragma once
#include "pcf_internal.h"

namespace pcf {

// Operation of the per-mode kernel.
enum ModeOp : int {
  MODE_SYNTH_ONLY = 0,   // y-synthesis (no solve): sig 0 reads uhat into slot 0, sig 1 rhat into slot 1
  MODE_PHI = 1,          // Stokes step of the NSE, r1 = (u+ - u)/dt, synthesis of r1
  MODE_PSI_UPDATE = 2,   // Stokes step of the dummy dynamics, f, u += dtau f, synthesis of u
  MODE_PSI_GRAD = 3,     // same as MODE_PSI_UPDATE but only writes f
  MODE_SOLVE = 4,        // Stokes step from a coefficient right-hand side (rhat), output fhat
};

struct LaunchInfo {
  const Inst* insts;
  const int* prefix;   // CTA prefix over instances (length ninst + 1)
  int ninst;
};

// Launch over groups of consecutive instances that share one grid.
struct GroupLaunch {
  const Inst* insts;
  const int* prefix;   // CTA prefix over groups (length ngroups + 1)
  const int2* groups;  // (first instance, instance count) per group
  int ngroups;
  // 1: the modes m >= 0 only (storage indices i <= Kx, the first (Kx + 1) Mz modes); the
  // synthesis also writes the y-values of mode -m from those of m by the s2 relation
  // a_{-m} = e2_c (-1)^m conj(a_m), which every state in an s2-invariant subspace satisfies
  int reduced;
};

// Number of (Fourier) modes a launch over instance I processes.
__device__ __forceinline__ int run_modes(const GroupLaunch& gl, const Inst& I) {
  return gl.reduced ? (I.Kx + 1) * I.Mz : I.nmodes;
}

__device__ __forceinline__ int find_inst(const LaunchInfo& li, int cta, int* local) {
  int lo = 0, hi = li.ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (li.prefix[mid] <= cta) lo = mid; else hi = mid - 1;
  }
  *local = cta - li.prefix[lo];
  return lo;
}

__device__ __forceinline__ bool inst_active(const Inst& I) { return I.active == nullptr || *I.active != 0; }

// Per-instance state of the DNS that produces guesses (pcf_dns), on the device.
struct DnsInst {
  double* hist;        // ||u_s|| history base (may be null), stride hist_stride
  int hist_stride;
  double2* uprev;      // the state before the current update
  double2* guess;      // guess base (may be null); guess k at guess + k * gstride
  long long gstride;
  int gmax;
  int* count;          // extrema found so far
  int step, slot;      // steps taken in this call; guess slot of this step's capture (-1: none)
  double h1, h2;       // ||u|| of the previous two steps
};

// J = sqrt(0.5 * sum_j w_j * mean_{x,z} |q|^2) from the plane sums (fixed order).
__device__ __forceinline__ double norm_from_parts(const Inst& I) {
  double s = 0.0;
  for (int j = 0; j < I.ny; ++j) {
    const double pj = I.normpart[j] + I.normpart[I.ny + j] + I.normpart[2 * I.ny + j];
    s = fma(I.ccw[j], pj, s);
  }
  return sqrt(0.5 * I.inv_nxnz * s);
}

// Raise the maximum dynamic shared memory of kernel func on the current device to at least
// bytes.  The attribute belongs to the function, not to a context, so it only ever grows: a
// context that needs less must not lower the limit another context launches with.
cudaError_t raise_smem_limit(const void* func, size_t bytes);

// Stokes step by banded tau sweeps, one thread per chain (pcf_sweep.cu): shared memory per
// CTA of `threads` lanes, CTAs for an instance whose launch covers nmodes_run modes, launch
// over a CTA prefix per instance (red: the modes m >= 0 only), and the shared-memory limit.
size_t smem_sweep(int N, int threads);
int sweep_ctas(int nmodes_run, int threads);
void launch_sweep(int ctas, int threads, size_t smem, cudaStream_t s, LaunchInfo li, int op, int red);
cudaError_t set_sweep_smem(size_t smem);

// kind: plane arithmetic, 0 FP64, 1 FP32 (mixed form), 2 float-float
void launch_xzsynth(int kind, int ctas, size_t smem, cudaStream_t s, LaunchInfo li, int slot, int nf);
// step_index >= 0 (adjoint product only): the last CTA of each instance also computes J from
// the plane sums, its history entry and the convergence mask (in place of launch_jnorm)
// suction: some instance of the launch has a base flow with a wall-normal velocity (ASBL)
void launch_prod(int kind, bool adj, bool suction, int ctas, size_t smem, cudaStream_t s, LaunchInfo li,
                 int step_index = -1);
void launch_norm_planes(int kind, int ctas, cudaStream_t s, LaunchInfo li, int slot);
cudaError_t set_plane_smem(int kind, size_t synth, size_t prod);
// Plane kernels of the FP32 form with the x, z transforms in warp registers
// (pcf_planes_warp.cu): nx, nz in {32, 64, 96, 128}.
bool plane_warp_ok(const Inst& I);
size_t smem_plane_warp(const Inst& I, int elem_bytes);
void launch_xzsynth_warp(int ctas, size_t smem, cudaStream_t s, LaunchInfo li, int slot, int nf);
void launch_prod_warp(bool adj, int ctas, size_t smem, cudaStream_t s, LaunchInfo li, int step_index);
cudaError_t set_plane_warp_smem(size_t synth, size_t prod);
__global__ void k_mode(LaunchInfo li, int op, int sig, int mpc, int step_index);
__global__ void k_norm_final(LaunchInfo li, double* out);
__global__ void k_fp64_probe(double* out, int iters);

size_t smem_plane(const Inst& I, int elem_bytes);
size_t smem_xzsynth(const Inst& I);
size_t smem_prod(const Inst& I);
size_t smem_mode(const Inst& I, int mpc);
size_t smem_cheb_tc(int ny);
void launch_cheb_synth_tc(int ctas, size_t smem, cudaStream_t s, LaunchInfo li, int slot);
void launch_cheb_analysis_tc(int ctas, size_t smem, cudaStream_t s, LaunchInfo li);
cudaError_t set_cheb_tc_smem(size_t smem);
// The same contractions on the 5th-generation tensor cores (tcgen05, TMEM accumulator;
// pcf_cheb_tc05.cu), same CTA map.
size_t smem_cheb_tc05(int ny);
void launch_cheb_synth_tc05(int ctas, size_t smem, cudaStream_t s, LaunchInfo li, int slot);
void launch_cheb_analysis_tc05(int ctas, size_t smem, cudaStream_t s, LaunchInfo li);
cudaError_t set_cheb_tc05_smem(size_t smem);
int cheb_tc_tiles(int nmodes);

// Split mode kernels of the FP64 descent step (Chebyshev analysis, dense Stokes solve,
// Chebyshev synthesis) over groups of instances on the same grid (at most
// split_max_group() instances; G below is the largest group of a launch).
// kind: 0 analysis, 1 solve, 2 synthesis.
// The solve kernel is persistent (ctas <= nitems CTAs loop over the (group, mode, parity)
// items, double-buffering each item's operands in shared memory).
int split_ctas_per_group(int kind, int nmodes, int mt);
int split_col_pad(int G);  // columns of a group of G instances (2 G rounded up to a power of two)
int split_max_group(int N);
size_t smem_yanalysis(int N, int G, int mt);
size_t ysolve_buffer(int N, int G);
size_t smem_ysolve(int N, int G);
size_t smem_ysynth(int N, int G, int mt);
// ff_arith: the Chebyshev dot products in float-float arithmetic (float-float form)
// mt: consecutive modes per CTA of the analysis and synthesis kernels (col_pad(G) mt <= 32)
void launch_yanalysis(int ctas, int threads, size_t smem, cudaStream_t s, GroupLaunch gl, int op, bool ff_arith,
                      int mt);
void launch_ysolve(int ctas, int nitems, int bufsz, int scr_rows, size_t smem, cudaStream_t s, GroupLaunch gl,
                   int op);
void launch_jnorm(int ninst, cudaStream_t s, const Inst* insts, int step_index);
int ysolve_ctas_per_sm(size_t smem);
void launch_ysynth_split(int ctas, int threads, size_t smem, cudaStream_t s, GroupLaunch gl, int slot,
                         int check_active, bool ff_arith, int mt);
// threads per CTA of the split analysis / synthesis: one pass over a CTA's row tasks
int split_yanalysis_threads(int N, int G, int mt, bool fp64);
int split_ysynth_threads(int N, int G, int mt, bool fp64);
cudaError_t set_split_smem(size_t analysis, size_t solve, size_t synth);
// The fused per-mode half-step (analysis + solve + synthesis), one CTA per (group, mode).
size_t smem_ystep(int N, int G);
void launch_ystep(int ctas, size_t smem, cudaStream_t s, GroupLaunch gl, int op);
cudaError_t set_ystep_smem(size_t smem);

// Symmetric-subspace projection and the DNS helpers (pcf_sym_dns.cu).
int symmetrize_ctas(const Inst& I);
void launch_symmetrize(int ctas_x, int ninst, cudaStream_t s, const Inst* insts, int mask_override,
                       int reduced = 0);
int dns_ctas(const Inst& I);
void launch_dns_norm(int ninst, cudaStream_t s, const Inst* insts, DnsInst* dns);
void launch_dns_capture(int ctas_x, int ninst, cudaStream_t s, const Inst* insts, const DnsInst* dns);
void launch_dns_update(int ctas_x, int ninst, cudaStream_t s, const Inst* insts, const DnsInst* dns);

}  // namespace pcf
