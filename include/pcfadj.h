/*
 * pcfadj.h - C ABI of the GB300 (sm_103a) adjoint-descent solver for equilibria of
 * plane Couette flow (Ashtari & Schneider, arXiv 2306.00165).
 *
 * The library advances the constrained adjoint-descent dynamics of §3.4,
 * Eq. (adjoint_evolution_divergence_free), with the five-step scheme of §4:
 * (1) an influence-matrix Stokes step of the Navier-Stokes equations, Eq. (u_trick),
 * (2) the finite-difference residual r1, Eq. (r1_approximation), (3) a Stokes step of
 * the dummy dynamics for r1, Eq. (g_trick), (4) the finite-difference descent
 * direction f, Eq. (f_approximation), and (5) the Euler update, Eq. (forward_Euler_update).
 * DMD extrapolation follows §6.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Spectral field ("uhat" layout): the Fourier x Chebyshev x Fourier coefficients of
 * §4, Eq. (Foureir_Chebyshev_Fourier), stored as interleaved complex doubles
 * (re, im) in the order [batch][3][Mx][Mz][Ny] with Ny (Chebyshev index n) fastest.
 * Component 0, 1, 2 = u, v, w.  x-modes are stored m = 0..Kx, -Kx..-1
 * (Mx = 2 Kx + 1, Kx = nx/3 - 1); z-modes p = 0..Kz (Mz = Kz + 1, Kz = nz/3 - 1);
 * the p < 0 half is the complex conjugate.  One instance holds 3*Mx*Mz*Ny complex
 * values (pcf_state_len).  Inputs must be admissible: divergence-free and zero at
 * y = +-1 (the state space of §3.1); the p = 0 plane conjugate-symmetric in m.
 *
 * Memory: unless an argument says "host", every pointer is a DEVICE pointer owned
 * by the caller; the library never frees it.  The context owns its workspace and
 * tables (allocated once in pcf_create).
 *
 * Streams: every call is enqueued on the stream given to pcf_create and returns
 * without synchronising, except where noted (pcf_dmd_extrapolate and the *_host
 * variants synchronise).  Errors are reported only by the return code: a call
 * that returns anything but PCF_OK has enqueued no partial update of its outputs
 * unless noted; nothing aborts the process.
 *
 * Grids: nx, nz in {16, 32, 48, 64, 96, 128} (products of 2, 3, 4), ny odd with
 * 9 <= ny <= 129; batch >= 1.
 */
#ifndef PCFADJ_H
#define PCFADJ_H

#ifdef __cplusplus
extern "C" {
#endif

#define PCF_ABI_VERSION 3

typedef enum {
  PCF_OK = 0,
  PCF_EINVAL = 1,     /* bad size, pointer or parameter */
  PCF_ECUDA = 2,      /* a CUDA runtime call failed */
  PCF_ENOMEM = 3,     /* device or host allocation failed */
  PCF_ENAN = 4,       /* a residual norm came out non-finite */
  PCF_ETIMEOUT = 5,   /* a bounded device wait gave up */
  PCF_ENOTCONV = 6,   /* no convergence within the step budget */
  PCF_ENOTSUP = 7     /* valid request this build does not provide */
} pcf_status;

typedef enum {
  PCF_FP64 = 0,         /* the plain method: FP64 throughout */
  PCF_MIXED = 1,        /* FP32 x-z transforms and products, split-BF16 tensor-core Chebyshev
                           transforms, FP64 Stokes solves, norms and state; ny <= 113
                           (PCF_ENOTSUP above) */
  PCF_FLOAT_FLOAT = 2   /* x-z transforms and products in float-float arithmetic (pairs of
                           FP32, ~48 significant bits) on the FP32 pipe; everything else FP64 */
} pcf_precision;

/* Problem description; all instances of a context share one grid.
 * Re: Reynolds number (nu = 1/Re); Lx, Lz: box lengths; dt: physical step of the
 * Navier-Stokes Stokes step (step 1 of §4); dtau_hat: step of the dummy dynamics
 * (step 3 of §4).  The paper uses Re = 400, Lx = 2 pi/1.14, Lz = 2 pi/2.5,
 * dt = dtau_hat = 0.25 (§5.1). */
typedef struct pcf_params {
  int nx, ny, nz;
  int batch;
  double Lx, Lz, Re;
  double dt, dtau_hat;
  int precision;        /* pcf_precision; PCF_FP64 for the plain method */
  int modes_per_block;  /* tile of the per-mode kernels (Fourier modes per CTA of the single
                           per-mode kernel; instances per group of the split kernels);
                           0 = autotuned */
  int solve_kind;       /* 0: dense per-mode operators when ny <= 129, else banded sweeps; the
                           autotuner picks the kernel organisation (FP64 form, ny <= 97: split
                           or fused kernels over instance groups; mixed form: dense against
                           sweeps), see pcf_solve_variant.  1: banded sweeps.  2: dense
                           operators inside the single per-mode kernel.  3: FP64 split
                           analysis / solve / synthesis kernels with the dense solve.  4: FP64
                           fused per-mode half-step kernel.  2, 3 and 4 give bit-identical
                           results.  5: FP64 split analysis and synthesis kernels with the
                           Stokes solve by banded sweeps, one thread per chain (group g, mode,
                           real or imaginary part); with 0 the autotuner times it against the
                           dense solve. */
  int base_flow;        /* pcf_base_flow: the laminar base flow u_b = (U(y), V, 0) */
  int symmetry;         /* pcf_symmetry mask enforced along the descent and the DNS (0: none).
                           s1 requires PCF_COUETTE (it maps the Poiseuille profile to its
                           negative and suction to blowing); PCF_EINVAL otherwise. */
  int plane_kernel;     /* x-z plane kernels of the mixed form (FP32): 0 = transforms in warp
                           registers when every instance has nx, nz in {32, 64, 96, 128}, else
                           the shared-memory Stockham kernels; 1 = always the Stockham kernels.
                           The FP64 and float-float forms always use the Stockham kernels.
                           pcf_plane_variant reports the choice. */
  int contraction_kernel; /* Chebyshev transforms of the mixed form (split-BF16, FP32
                           accumulation): 0 = tcgen05 MMAs with the accumulator in tensor
                           memory (the padded matrix in one 128-row MMA tile, its operand
                           moved by bulk copies on the TMA engine); 1 = warp-level
                           mma.sync.  pcf_contraction_variant reports the choice.  Ignored
                           by the other forms. */
  double suction_length; /* PCF_ASBL only: suction length delta of the boundary layer in
                           units of the half-height (> 0, finite; PCF_EINVAL otherwise).
                           Ignored by the other base flows. */
} pcf_params;

/* Base flows (§3.1 derives the method for a general laminar base flow u_b; §7 names plane
 * Poiseuille flow and the asymptotic suction boundary layer as flows where only u_b
 * changes).  The perturbation u vanishes at both walls in every case; the Poiseuille base
 * flow absorbs the fixed driving pressure gradient, so the perturbation's mean pressure
 * gradient stays zero.  The suction boundary layer sits on the wall y = -1 (lengths in units
 * of the half-height, Re = U/(nu h)): U = 1 - exp(-(1 + y)/delta) with the uniform suction
 * V = -nu/delta, which solve V U' = nu U'' without a pressure gradient; the wall y = +1 moves
 * at U(1) with the same uniform wall-normal velocity (a finite box standing in for the free
 * stream).  The suction enters M and N as advection by V (u_b + u advects). */
typedef enum {
  PCF_COUETTE = 0,     /* plane Couette flow:    U = y       (walls moving at +-1) */
  PCF_POISEUILLE = 1,  /* plane Poiseuille flow: U = 1 - y^2 (pressure-driven) */
  PCF_ASBL = 2         /* asymptotic suction boundary layer: U = 1 - exp(-(1+y)/delta),
                          V = -nu/delta (pcf_params.suction_length = delta) */
} pcf_base_flow;

/* Symmetries of §5.1 (bit mask).  s1 = shift-and-rotate, s2 = shift-and-reflect:
 *   s1 [u,v,w](x,y,z) = [-u,-v,w](-x + Lx/2, -y, z + Lz/2)
 *   s2 [u,v,w](x,y,z) = [u,v,-w](x + Lx/2, y, -z)
 * They commute and are involutions; the subspace invariant under a mask is the image of the
 * group average over {e, s1}, {e, s2} or {e, s1, s2, s1 s2} (an orthogonal projection).
 * The descent is equivariant under them (§3.4), so it preserves that subspace; enforcing it
 * (pcf_params.symmetry) projects the state at the start of every call and after every
 * update, which removes only rounding drift out of the subspace. */
typedef enum {
  PCF_SYM_NONE = 0,
  PCF_SYM_S1 = 1,
  PCF_SYM_S2 = 2
} pcf_symmetry;

typedef struct pcf_ctx pcf_ctx;

/* Version of this ABI (PCF_ABI_VERSION). */
int pcf_abi_version(void);

/* Human-readable name of a status code; never NULL. */
const char* pcf_status_str(pcf_status s);

/* Number of complex values of one instance in the uhat layout: 3*Mx*Mz*ny.
 * Returns 0 for an invalid grid. */
long long pcf_state_len(int nx, int ny, int nz);

/* Length of the real snapshot vector psi of §6.2 (minimum number of independent
 * variables of a divergence-free Fourier-Chebyshev field): per independent mode
 * 2(ny-4) + 2(ny-2) reals, plus 2(ny-2) for the mean u, w.  20218 at 32x31x32. */
long long pcf_psi_len(int nx, int ny, int nz);

/* Create a context on the current CUDA device.  stream: a cudaStream_t (NULL =
 * default stream).  Builds the per-mode influence-matrix tables of the Stokes steps
 * for dt and dtau_hat (§4) and allocates the workspace.  *out is set only on PCF_OK. */
pcf_status pcf_create(const pcf_params* params, void* stream, pcf_ctx** out);

/* Create a context over a batch of instances whose grids (and Re, box, step sizes) may
 * differ: list[k] describes list[k].batch instances (the batched form of the method:
 * many initial guesses of uneven grid sizes advanced by the same kernel launches, each
 * step captured in one CUDA graph, with per-instance convergence masks in pcf_run).
 * Instance states are stored back to back in the order given; pcf_state_offset gives
 * each one's offset.  Tables are shared between instances on the same problem.  With
 * list[0].modes_per_block = 0 an autotuner times the mode kernel for several tiles on
 * the batch and keeps the fastest (pcf_mode_tile).  DMD entry points require every
 * instance on one problem (PCF_ENOTSUP otherwise). */
pcf_status pcf_batch_create(const pcf_params* list, int n, void* stream, pcf_ctx** out);

/* Offset, in complex values, of instance `instance`'s state in the batch layout
 * (instance = batch gives the total); -1 for an invalid instance. */
long long pcf_state_offset(const pcf_ctx* ctx, int instance);

/* Fourier modes per CTA chosen for the per-mode kernels of the descent step (by the
 * autotuner or the caller). */
int pcf_mode_tile(const pcf_ctx* ctx);

/* Stokes solve the descent step uses: 0 banded tau sweeps inside the per-mode kernel,
 * 1 dense per-mode operators inside the per-mode kernel, 2 dense operators in the split
 * analysis / solve / synthesis kernels over instance groups, 3 dense operators in the fused
 * per-mode half-step kernel over instance groups, 4 banded sweeps with one thread per chain
 * between the split analysis and synthesis kernels (2, 3 and 4: FP64 and float-float forms).
 * With solve_kind 0 the FP64 form times 2 against 3 and then the chosen dense solve against
 * 4, the mixed-precision form 0 against 1, at creation, and each keeps the faster.  -1 for a
 * NULL context. */
int pcf_solve_variant(const pcf_ctx* ctx);

/* x-z plane kernels the context launches: 0 shared-memory Stockham passes, 1 transforms in
 * warp registers (FP32 form, see pcf_params.plane_kernel); -1 for a NULL context. */
int pcf_plane_variant(const pcf_ctx* ctx);

/* Tensor-core instructions of the mixed form's Chebyshev transforms: 1 tcgen05 (tensor
 * memory accumulator), 0 mma.sync, -1 for a NULL context (see pcf_params.contraction_kernel). */
int pcf_contraction_variant(const pcf_ctx* ctx);

/* Fourier modes the per-mode kernels of one descent step process per instance: Mx*Mz, or
 * (Kx+1)*Mz (the modes m >= 0) when every instance enforces s2 (pcf_params.symmetry) and the
 * step runs the split per-mode kernels.  A state invariant under s2 satisfies
 * a_{-m,p,n} = e2_c (-1)^m conj(a_{m,p,n}) with e2 = (+1, +1, -1) for (u, v, w); the step then
 * computes the modes m >= 0, mirrors their y-values, and rebuilds the modes m < 0 of the
 * updated state in its projection.  -1 for a NULL context. */
int pcf_symmetric_modes(const pcf_ctx* ctx);

/* Release a context (waits for its stream).  NULL is ignored. */
void pcf_destroy(pcf_ctx* ctx);

/* Steps 1-2 of §4: r1 = (Phi_dt(u) - u)/dt, Eq. (r1_approximation), where Phi_dt is
 * one IMEX-Euler influence-matrix Stokes step of Eq. (u_trick) with
 * M(u) = -(u_b.grad)u - (u.grad)u_b - (u.grad)u, u_b = (y, 0, 0).
 * u_hat: batch instances in the uhat layout (input).  r_hat: same layout (output).
 * r_norm: batch doubles (output, may be NULL): J = ||r1||, the volume-normalised L2
 * norm with Clenshaw-Curtis weights in y. */
pcf_status pcf_residual(pcf_ctx* ctx, const double* u_hat, double* r_hat, double* r_norm);

/* Steps 3-4 of §4: f = -(Psi_dtauhat(r1) - r1)/dtau_hat, Eq. (f_approximation), where
 * Psi is one Stokes step of the dummy dynamics Eq. (g_trick) with
 * N(r1) = (grad r1)(u_b + u) - (grad(u_b + u))^T r1 (u frozen), taken in the
 * diffusive direction of tau-hat.  u_hat, r_hat: inputs (r_hat normally from
 * pcf_residual); f_hat: output; all in the uhat layout. */
pcf_status pcf_adjoint_gradient(pcf_ctx* ctx, const double* u_hat, const double* r_hat, double* f_hat);

/* One influence-matrix Stokes step alone (the solve used by steps 1 and 3 of §4):
 * out solves (1/step - nu Lap) out + grad p = rhs, div out = 0, out(y=+-1) = 0, per
 * Fourier mode with the Chebyshev-tau method (momentum on rows 0..ny-3, divergence
 * on every row).  step must equal params.dt or params.dtau_hat (else PCF_EINVAL).
 * rhs_hat, out_hat: uhat layout. */
pcf_status pcf_influence_matrix_solve(pcf_ctx* ctx, const double* rhs_hat, double* out_hat, double step);

/* nsteps descent steps of §4 (steps 1-5 each), in place on u_hat:
 * u <- u + dtau f.  r_norm_hist: nsteps*batch doubles ([step][instance], J before
 * each step) or NULL.  Launched as a captured CUDA graph. */
pcf_status pcf_descent_step(pcf_ctx* ctx, double* u_hat, double dtau, int nsteps, double* r_norm_hist);

/* Same as pcf_descent_step with HOST buffers: copies u_hat (host, batch states) to
 * the device, runs nsteps steps, copies the updated state and the norm history
 * (host, nsteps*batch doubles, may be NULL) back, then synchronises. */
pcf_status pcf_descent_step_host(pcf_ctx* ctx, double* u_hat_host, double dtau, int nsteps, double* r_norm_hist_host);

/* Snapshot vector of §6.2 for every instance: psi[batch][pcf_psi_len] (device,
 * output) from u_hat (input).  Coordinates: Chebyshev coefficients 0..ny-5 of v and
 * 0..ny-3 of eta = i kz u - i kx w per independent mode (re, im), then the mean u,
 * w coefficients 0..ny-3. */
pcf_status pcf_snapshot(pcf_ctx* ctx, const double* u_hat, double* psi);

/* Volume-normalised L2 norm ||u|| of every instance (the norm of J, §2; Table 2 lists
 * ||u|| of the equilibria found).  norm: device double[batch]. */
pcf_status pcf_norm(pcf_ctx* ctx, const double* u_hat, double* norm);

/* Project u_hat (every instance, in place) onto the subspace invariant under the symmetries
 * of mask (pcf_symmetry bits, 0..3; 0 leaves u_hat unchanged): the group average of §5.1's
 * s1 and s2.  Admissible inputs give admissible outputs.  PCF_EINVAL for a mask outside 0..3. */
pcf_status pcf_symmetrize(pcf_ctx* ctx, double* u_hat, int mask);

/* Direct numerical simulation with the Stokes step of §4 step 1 as the time stepper (IMEX
 * Euler: implicit viscous term and pressure, explicit M, step pcf_params.dt):
 *   u <- u^dt = u + dt r1(u),  nsteps times, in place on u_hat.
 * §5.2 takes its guesses for the robustness experiment from such a run: the states where
 * ||u|| (volume-normalised L2) has a local extremum in time.
 * norm_hist: device [nsteps][batch] doubles, ||u_s|| before step s, or NULL.
 * guesses: device room for max_guesses batch states ([max_guesses][total state] complex, the
 *   uhat layout of the whole batch per guess); the state u_s of instance b at each strict
 *   discrete extremum ((h_s - h_{s-1}) (h_{s+1} - h_s) < 0, 1 <= s <= nsteps - 2) is stored
 *   at guess k = the number of earlier extrema of b, while k < max_guesses.  May be NULL
 *   when max_guesses = 0.
 * n_guesses: device int[batch], zeroed by the call, then the number of extrema found per
 *   instance (may exceed max_guesses), or NULL.
 * With pcf_params.symmetry set, the state is projected at the start and after each step.
 * The explicit advection of Euler's method needs dt <= 2 nu / max|U + u|^2 for the longest
 * waves (e.g. dt <= 0.005 at Re = 400); the dt = 0.25 of the descent is not a DNS step. */
pcf_status pcf_dns(pcf_ctx* ctx, double* u_hat, int nsteps, double* norm_hist, double* guesses, int max_guesses,
                   int* n_guesses);

/* Inverse of pcf_snapshot: completes the wall conditions and rebuilds u_hat. */
pcf_status pcf_from_snapshot(pcf_ctx* ctx, const double* psi, double* u_hat);

/* DMD steady-state extrapolation of §6 for one instance.
 * snapshots: device, (M+1) columns of pcf_psi_len doubles (column k = snapshot k,
 * oldest first) with column stride ld >= pcf_psi_len doubles; the M pairs are
 * (s_k, s_{k+1}).  Householder QR of the
 * snapshot matrix on the device; SVD, eigen-decomposition and amplitudes of the
 * small projected problem on the host; for each truncation rank r = r*..1 (r* = number
 * of singular values above rank_tol * sigma_1) the steady mode b_1 phi_1 (|ln lambda|
 * smallest) is rebuilt and its residual norm evaluated; the r with the smallest norm
 * is kept.  u_out_hat: device, one instance (output).  rank_used, j_out: host
 * (outputs, may be NULL).  Synchronises.  PCF_ENAN if no candidate has a finite norm. */
pcf_status pcf_dmd_extrapolate(pcf_ctx* ctx, const double* snapshots, long long ld, int M, double rank_tol,
                               double* u_out_hat, int* rank_used, double* j_out);

/* Runs the descent to convergence for every instance (the hot loop of §5.1 with the DMD
 * acceleration of §6): steps of pcf_descent_step with a per-instance convergence mask
 * (an instance stops updating once J = ||r1|| < tol), at most max_steps steps.  With
 * dmd_period > 0, a snapshot (pcf_snapshot) is taken every dmd_period/dmd_snapshots
 * steps and after each period every unconverged instance jumps to its DMD steady state
 * (pcf_dmd_extrapolate on the period's dmd_snapshots snapshots); a jump is skipped only
 * when no candidate has a finite residual.  dmd_period = 0 disables DMD.
 * u_hat: device, in place.  steps_out (host, batch): steps taken until J < tol, -1 if
 * not converged; j_out (host, batch): last J; dmd_jumps (host): jumps taken.  Each may
 * be NULL.  Synchronises; allocates its snapshot ring for the call.  PCF_ENAN if an
 * instance's J became non-finite. */
pcf_status pcf_run(pcf_ctx* ctx, double* u_hat, double dtau, int max_steps, double tol, int dmd_period,
                   int dmd_snapshots, double rank_tol, int* steps_out, double* j_out, int* dmd_jumps);

/* DMD schedule of §6.2.  The paper lets J fall to log J = -4.5 before the first
 * extrapolation, builds each linear model from M = 100 snapshots 200 time units apart, and
 * integrates 1.5e5 time units after each jump before it collects again.  Here:
 * snapshots are taken every `spacing` descent steps; before the first extrapolation they
 * fill a sliding window of the latest `snapshots`, and the first extrapolation happens at
 * the first snapshot point where the window is full and the last J < j_start (+INFINITY:
 * as soon as the window is full); after a jump the descent runs `gap` steps (rounded up to a
 * multiple of spacing), then collects `snapshots` fresh snapshots and jumps again.
 * pcf_run(dmd_period P, dmd_snapshots S) is this schedule with spacing P/S, gap 0 and
 * j_start = +INFINITY. */
typedef struct pcf_dmd_schedule {
  int snapshots;     /* stored snapshots per extrapolation, M + 1 >= 3 */
  int spacing;       /* descent steps between snapshots, >= 1 */
  int gap;           /* descent steps from a jump to the start of the next collection, >= 0 */
  double j_start;    /* threshold on J for the first extrapolation (not NaN) */
  double rank_tol;   /* rank threshold of pcf_dmd_extrapolate, > 0 */
} pcf_dmd_schedule;

/* pcf_run with a general DMD schedule (NULL: no DMD).  Same outputs, synchronisation and
 * errors as pcf_run; the snapshot ring holds schedule->snapshots states per instance. */
pcf_status pcf_run_schedule(pcf_ctx* ctx, double* u_hat, double dtau, int max_steps, double tol,
                            const pcf_dmd_schedule* schedule, int* steps_out, double* j_out, int* dmd_jumps);

/* The Stokes solve of pcf_influence_matrix_solve for callers that cannot allocate device
 * memory (the paper has no counterpart; this is a library service).  Such callers - an
 * application whose device memory belongs to a fixed pool or a foreign allocator, or a
 * plugin that must not grow its device footprint after start-up - cannot use
 * pcf_create, which allocates tables and workspace with cudaMalloc.  This entry point
 * needs no context and allocates nothing: everything beyond rhs_hat and out_hat (the
 * per-mode tau sweep coefficients, homogeneous responses and 2x2 influence-matrix
 * inverses, the instance descriptor) lives in one static device array of 5 MiB that the
 * library holds on every GPU it is loaded on, rebuilt on the device at every call.
 * params: grid and Re, Lx, Lz (dt, dtau_hat, precision ignored; batch must be 1);
 * limit: nx, nz <= 64 (at most 861 retained modes) and ny <= 65, else PCF_EINVAL before
 * any launch.  step: the implicit step (any positive value).  rhs_hat, out_hat: device,
 * uhat layout, one instance.  stream: cudaStream_t (NULL = default stream); asynchronous.
 * The first call on a device (with that device current) looks up the array's address;
 * make it before any stream capture.  All calls share the array: calls that overlap on the
 * GPU race and must be ordered on one stream. */
pcf_status pcf_influence_matrix_solve_noalloc(const pcf_params* params, const double* rhs_hat, double* out_hat,
                                              double step, void* stream);

/* ---- Learned proposal (the accelerated form with a neural operator) ----
 * A Fourier-space neural operator on the spectral coefficients of the state proposes the
 * state far ahead in pseudo-time; the descent judges every proposal by the residual norm
 * and keeps its own state otherwise.  Features per retained Fourier mode mp (all Mx*Mz)
 * and Chebyshev index n: (Re v, Im v, Re eta, Im eta), eta = i kz u - i kx w, or
 * (u, w, 0, 0) for the mean mode; layout float [MP][S][NY][4].
 * `scale` is a device array [MP][NY][4] of per-coefficient feature scales (e.g. inverse RMS
 * over the training states); network outputs are increments in the same scaled units.
 * Network, per retained Fourier mode mp with F = NY*4 coefficients X[mp]:
 * H0 = X[mp] E[mp]^T + bE; Z_l = H_{l-1} (R_l[mp] + L_l)^T + b_l; H_l = H_{l-1} + GELU(Z_l);
 * Y[mp] = H_L D[mp]^T + bD[mp]; loss mean((Y - T)^2).  All products run on the tensor
 * cores in BF16 with FP32 accumulation; Adam on FP32 master weights.
 * Parameter layout (float): E [MP][W][F], bE [W], D [MP][F][W], bD [MP][F], then per
 * layer R [MP][W][W], L [W][W], b [W].  All array arguments are device pointers
 * unless named *_host. */
typedef struct pcf_fno pcf_fno;
pcf_status pcf_fno_create(int MP, int NY, int width, int layers, unsigned long long seed, void* stream, pcf_fno** out);
void pcf_fno_destroy(pcf_fno* net);
long long pcf_fno_num_params(const pcf_fno* net);
pcf_status pcf_fno_set_params(pcf_fno* net, const float* params_host);
pcf_status pcf_fno_get_params(pcf_fno* net, float* params_host);
/* Y = network(X) for S samples. */
pcf_status pcf_fno_forward(pcf_fno* net, const float* X, int S, float* Y);
/* Loss and its gradient (grad: device, pcf_fno_num_params floats, may be NULL); loss on the host. */
pcf_status pcf_fno_loss_grad(pcf_fno* net, const float* X, const float* T, int S, double* loss_host, float* grad);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr; loss before the step. */
pcf_status pcf_fno_train_step(pcf_fno* net, const float* X, const float* T, int S, float lr, double* loss_host);
/* Features of every instance of a uniform context: X [nm][batch][ny][4]. */
pcf_status pcf_fno_features(pcf_ctx* ctx, const double* u_hat, float* X, const float* scale);
/* One proposal: u' = state of (features(u) + network(features(u))) / scale, completed to an
 * admissible field (walls, divergence).  With relax_steps > 0 both u and u' first take that
 * many plain descent steps of size dtau.  Instance b then takes the proposal's branch iff
 * its residual norm J is lower (ties keep the plain branch).  accepted_host,
 * J_before_host (plain branch), J_after_host (proposal branch): batch entries each (may
 * be NULL).  Synchronises. */
pcf_status pcf_fno_propose(pcf_ctx* ctx, pcf_fno* net, double* u_hat, const float* scale, int relax_steps,
                           double dtau, int* accepted_host, double* J_before_host, double* J_after_host);

/* Measures the FP64 FMA throughput of the current device with a dependent-chain-free
 * DFMA loop (used for the ALU roofline).  gflops: host output.  Synchronises. */
pcf_status pcf_probe_fp64_peak(void* stream, double* gflops);

/* Enables (1) or disables (0) per-kernel CUDA-event timing on the context stream for
 * subsequent eager (non-graph) calls; pcf_kernel_times returns the accumulated
 * milliseconds and launch counts per kernel class (host arrays of length n).
 * Kernel classes: 0 ysynth, 1 xzsynth_u, 2 prod_M, 3 mode_phi, 4 xzsynth_q,
 * 5 prod_N, 6 mode_psi, 7 yanalysis, 8 ysynth_step, 9 jnorm, 10 symmetrize, 11 dns_aux,
 * 12 cheb_synth_tc, 13 cheb_analysis_tc.
 * In the FP64 form with dense per-mode operators (ny <= 97) the per-mode work of a step
 * runs as three kernels: 7 (Chebyshev analysis + right-hand side, twice per step), 3/6
 * (Stokes solve and update of the NSE / dummy step), 8 (Chebyshev synthesis of r1 and of
 * the new u).  J, its history and the convergence mask come from the last CTA of each
 * instance in 5, except with the fused half-step kernel, where 9 computes them; without
 * dense operators 3/6 hold the whole per-mode kernel and 7, 8, 9 stay empty.  10 is the
 * projection onto the symmetric subspace, 11 the small kernels around pcf_dns; 12 and 13 are the
 * mixed form's tensor-core Chebyshev synthesis and analysis (its mode kernel, 3/6, then holds
 * only the Stokes solve). */
pcf_status pcf_set_kernel_timing(pcf_ctx* ctx, int enable);

/* Organisation the autotuner chose for the split per-mode kernels (FP64 and float-float
 * forms): cfg[0] instances per group of the analysis and synthesis kernels, cfg[1] and cfg[2]
 * consecutive modes per CTA of the analysis and of the synthesis, cfg[3] instances per group
 * of the Stokes solve.  Zeros where the context does not use those kernels (fused solve:
 * cfg[3] = 0).  cfg: host int[4]. */
pcf_status pcf_split_config(const pcf_ctx* ctx, int* cfg);

/* Kernel launches of one pcf_descent_step call of nsteps steps (the entry synthesis, and
 * projection when a symmetry is enforced, plus the steps); -1 for a bad argument. */
long long pcf_launches_per_call(pcf_ctx* ctx, int nsteps);
pcf_status pcf_kernel_times(pcf_ctx* ctx, double* ms, long long* launches, int n);

/* Number of kernel launches one descent step issues inside a multi-step call (for launch
 * accounting; pcf_launches_per_call counts a whole call). */
int pcf_launches_per_step(pcf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PCFADJ_H */
