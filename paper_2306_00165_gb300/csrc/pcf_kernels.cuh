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

__device__ __forceinline__ int find_inst(const LaunchInfo& li, int cta, int* local) {
  int lo = 0, hi = li.ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (li.prefix[mid] <= cta) lo = mid; else hi = mid - 1;
  }
  *local = cta - li.prefix[lo];
  return lo;
}

void launch_xzsynth(bool f32, int ctas, size_t smem, cudaStream_t s, LaunchInfo li, int slot, int nf);
void launch_prod(bool f32, bool adj, int ctas, size_t smem, cudaStream_t s, LaunchInfo li);
void launch_norm_planes(bool f32, int ctas, cudaStream_t s, LaunchInfo li);
cudaError_t set_plane_smem(bool f32, size_t synth, size_t prod);
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
int cheb_tc_tiles(int nmodes);

}  // namespace pcf
