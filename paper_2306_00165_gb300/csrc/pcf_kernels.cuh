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

__global__ void k_xzsynth(LaunchInfo li, int slot, int nfields);
__global__ void k_prod_M(LaunchInfo li);
__global__ void k_prod_N(LaunchInfo li);
__global__ void k_norm_planes(LaunchInfo li);
__global__ void k_mode(LaunchInfo li, int op, int sig, int mpc, int step_index);
__global__ void k_norm_final(LaunchInfo li, double* out);
__global__ void k_fp64_probe(double* out, int iters);

size_t smem_xzsynth(const Inst& I);
size_t smem_prod(const Inst& I);
size_t smem_mode(const Inst& I, int mpc);

}  // namespace pcf
