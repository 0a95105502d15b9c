// Context of the pcfadj library (internal; shared by the host translation units).
#pragma once
#include <map>
#include <vector>

#include "pcf_kernels.cuh"

struct pcf_ctx {
  pcf_params prm;
  int N, Kx, Kz, Mx, Mz, nm, B, mpc;
  long long state_len;  // complex values per instance (instance 0; all instances when uniform)
  std::vector<long long> state_off;  // complex offset of each instance's state, [B+1]
  long long total_state = 0;
  bool uniform = true;   // every instance on the same problem
  bool suction = false;  // some instance has a base flow with suction (PCF_ASBL)
  int mode_thr = 128;    // threads per CTA of the single per-mode kernel
  int thr_ya = 256, thr_yy = 128;  // threads per CTA of the split analysis and synthesis
  bool mixed = false;    // mixed-precision form (FP32 planes, split-BF16 Chebyshev, FP64 solves)
  int plane_kind = 0;    // arithmetic of the x-z plane kernels: 0 FP64, 1 FP32, 2 float-float
  bool plane_warp = false;  // FP32 plane kernels with the transforms in warp registers
  bool tc05 = false;        // Chebyshev contractions of the mixed form on tcgen05 (else mma.sync)
  // descent steps in the symmetric subspace run the per-mode kernels on the modes m >= 0 only
  // (every instance enforces s2; split FP64 or float-float kernels); the reduced CTA maps:
  bool reduced = false;
  int* pre_ya_r = nullptr;
  int* pre_yy_r = nullptr;
  int* pre_ys_r = nullptr;
  int cta_ya_r = 0, cta_yy_r = 0, cta_ys_r = 0, grid_ys_r = 0;
  double tuned_ms = 0.0; // autotuner: time of the chosen mode-kernel launch
  cudaStream_t user = nullptr, cs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<void*> allocs;
  std::vector<pcf::Inst> hinst;
  pcf::Inst* dinst = nullptr;
  // prefix arrays
  int* pre_synth11 = nullptr;
  int* pre_synth3 = nullptr;
  int* pre_prod = nullptr;
  int* pre_mode = nullptr;
  int* pre_inst = nullptr;
  int* pre_tcs = nullptr;   // tensor-core synthesis (mixed form)
  int* pre_tca = nullptr;   // tensor-core analysis (mixed form)
  int cta_synth11 = 0, cta_synth3 = 0, cta_prod = 0, cta_mode = 0, cta_tcs = 0, cta_tca = 0;
  size_t sm_synth = 0, sm_prod = 0, sm_mode = 0, sm_tc = 0, sm_warp = 0;
  // split mode kernels (FP64 form with dense operators): instance groups and geometry
  bool split = false;
  int sgrp = 0;                 // largest instances per group
  int smt = 1;                  // consecutive modes per CTA of the split analysis
  int smt_y = 1;                // ... and of the split synthesis (tuned separately)
  int ngroups = 0;
  int2* d_groups = nullptr;     // [B] (first, count)
  int* pre_ya = nullptr;        // CTA prefixes over groups [B + 1]
  int* pre_ys = nullptr;
  int* pre_yy = nullptr;
  int cta_ya = 0, cta_ys = 0, cta_yy = 0;
  int grid_ys = 0, buf_ys = 0, rows_ys = 0;  // persistent solve: CTAs, stage buffer, scratch rows
  // the solve's own instance groups (its right-hand sides are per instance, so its grouping
  // is independent of the analysis and synthesis kernels'); tuned separately
  int sgrp_s = 0, ngroups_s = 0;
  // the split step's Stokes solve by banded sweeps, one thread per chain (k_sweep), in place
  // of the dense solve: CTA prefixes per instance (full and reduced launches) and geometry
  bool sweep = false;
  int* pre_sw = nullptr;
  int* pre_sw_r = nullptr;
  int cta_sw = 0, cta_sw_r = 0, thr_sw = 32;
  size_t sm_sw = 0;
  int2* d_groups_s = nullptr;
  bool fused = false;           // the step runs the fused per-mode kernel (k_ystep)
  int* pre_yf = nullptr;        // its CTA prefix over groups [B + 1]
  int cta_yf = 0;
  size_t sm_yf = 0;
  size_t sm_ya = 0, sm_ys = 0, sm_yy = 0;
  double tuned_split_ms = 0.0;
  double2* r_int = nullptr;    // internal r1 buffer for descent
  double2* u_dev = nullptr;    // device state for the *_host entry point
  double* hist_dev = nullptr;
  int hist_cap = 0;
  int* active = nullptr;
  std::map<int, cudaGraphExec_t> graphs;
  // symmetric subspace and DNS
  bool any_sym = false;         // some instance enforces a symmetry
  int sym_ctas = 0, dns_ctas = 0;
  pcf::DnsInst* d_dns = nullptr;
  double2* uprev = nullptr;
  int* dns_count = nullptr;
  std::map<int, cudaGraphExec_t> dns_graphs;
  // timing
  int timing = 0;
  double kms[pcf::kNumKernelClasses] = {0};
  long long kcount[pcf::kNumKernelClasses] = {0};
  std::vector<cudaEvent_t> evpool;
  // snapshot vector (psi) and DMD workspace, allocated on first use
  int* d_indep = nullptr;   // (i, j) storage indices of the independent modes
  int nindep = 0;
  long long psi_len = 0;
  double* dmd_A = nullptr;      // Householder QR workspace, psi_len x cap
  double* dmd_part = nullptr;   // partial sums
  double* dmd_coef = nullptr;   // per-column reflector data
  double* dmd_cpsi = nullptr;   // candidate snapshot vectors
  double2* dmd_cu = nullptr;    // candidate states
  double* dmd_J = nullptr;      // candidate norms (batch)
  double* dmd_c = nullptr;      // candidate coefficient vectors (device)
  int dmd_cap = 0;              // columns the DMD workspace holds
  int dmd_ncand_cap = 0;
};

