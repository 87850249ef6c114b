/*
 * mdgp.h -- C ABI of the GB300 micro-MD + Gaussian-process library.
 *
 * The library runs the hot path of the hybrid continuum-atomistic scheme of
 * Stephenson, Kermode & Lockerby (arXiv:1603.04628): batches of independent
 * Lennard-Jones micro-elements (paper App. A; body force of Sec. 2.1
 * Eq. momentumEq; time-averaged mass flow rate of Eq. continuityEq), the
 * Gaussian-process surrogate that decides which macro sections need one
 * (Sec. 2.2, Eqs. quadraticKernelEq, d2Eq, covarianceEq, predMeanEq,
 * predVarEq), and the macro time step of Algorithm 1 (Sec. 2.4).
 *
 * Conventions for every entry point:
 *   - Units are reduced Lennard-Jones units (eps = sigma = m = 1).
 *   - Pointers are HOST pointers unless the name says _dev.  The caller owns
 *     every array it passes; the library copies what it needs and keeps no
 *     caller pointer after the call returns.
 *   - Return value: MDGP_OK (0) or a negative mdgp_status.  On failure the
 *     outputs are unspecified.  Per-element failures inside a batch do not
 *     fail the call; they are reported in mdgp_result.status.
 *   - A context is not thread-safe; use one context per host thread.
 *   - All device work runs on one GPU, on the context's stream.
 */
#ifndef MDGP_H
#define MDGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MDGP_OK = 0,
  MDGP_E_ARG = -1,       /* invalid argument (null pointer, size or geometry out of range) */
  MDGP_E_NOMEM = -2,     /* device or host allocation failed */
  MDGP_E_CUDA = -3,      /* a CUDA runtime call failed */
  MDGP_E_UNSTABLE = -4,  /* an element blew up (non-finite state or atoms far outside the box) */
  MDGP_E_NOTPD = -5,     /* GP covariance not positive definite */
  MDGP_E_TIMEOUT = -6,   /* a bounded device-side wait gave up */
  MDGP_E_STATE = -7,     /* call out of order (e.g. launch before plan) */
  MDGP_E_OVERFLOW = -8,  /* an atom had more neighbours than the list capacity */
  MDGP_E_SKIN = -9,      /* an atom moved more than half the list skin between rebuilds */
  MDGP_E_LIMIT = -10     /* a size beyond a fixed limit of an allocation-free entry point */
} mdgp_status;

typedef enum {
  MDGP_PREC_FP64 = 0,    /* FP64 pair forces and FP64 state */
  MDGP_PREC_FP32 = 1     /* FP32 pair forces; positions, velocities and tether anchors as
                            double-float pairs (two FP32 words, hi + lo, about 44 significant
                            bits: ~1e-13 sigma on a cell-relative offset); FP64 accumulators */
} mdgp_precision;

typedef struct mdgp_ctx mdgp_ctx;

/* ------------------------------------------------------------------------ */
/* Micro-element MD (paper App. A, Sec. 2.1).                                */
/* ------------------------------------------------------------------------ */

/* One micro-element: a fluid slab of height h between two FCC walls, periodic
 * in x (streamwise, length Lx) and z (spanwise, length Lz).
 * Every fluid atom feels the body force of Eq. momentumEq,
 *   F = g_ext - (m / rho) dp/dx,  rho = m * density. */
typedef struct {
  double h;          /* distance between the innermost wall planes */
  double dpdx;       /* local pressure gradient dp/dx */
  double density;    /* fluid number density n; N_fluid = round(n Lx h Lz) */
  double T;          /* target temperature (wall thermostat; initial velocities) */
  int64_t steps_eq;      /* equilibration steps (not sampled) */
  int64_t steps_sample;  /* sampling steps, split into n_blocks contiguous blocks */
  double Lx, Lz;     /* periodic lengths; each must be >= 3 r_c */
  double g_ext;      /* external force per atom F_ext (Eq. extForcing1 value at this time) */
  uint64_t seed;     /* Philox key */
  int32_t flags;     /* reserved, 0 */
  int32_t id;        /* element id: Philox counter word 2 */
  double wall_amp;   /* 0: planar walls h apart.  In [0, 1): the walls follow
                        h(x) = h (1 - wall_amp cos(2 pi x / Lx)) symmetrically about the
                        mid-plane of the widest gap h (1 + wall_amp) -- one element is then
                        a whole periodic converging-diverging channel (the full MD of
                        Sec. 3); N_fluid = round(n Lx h Lz) fills the gap at uniform
                        density, P_xx is over the fluid volume Lx h Lz.  FP32 and FP64. */
} mdgp_element;

/* Time-averaged outputs of one element. */
typedef struct {
  double q;        /* mean mass flow rate (m / Lx) sum_fluid v_x over the sampling steps */
  double q_se;     /* its standard error: std(block means, ddof 1) / sqrt(n_blocks) */
  double p;        /* mean P_xx of the fluid slab (kinetic + virial, fluid-wall pairs half) */
  double p_se;     /* its standard error, same estimator */
  double T_meas;   /* mean fluid kinetic temperature m <|v|^2> / 3 over the samples */
  double e_drift;  /* (E_end - E_start) / N_atoms, E = kinetic + LJ (shifted) + tether */
  int64_t n_fluid, n_wall;
  int32_t status;  /* MDGP_OK, or MDGP_E_UNSTABLE / _OVERFLOW / _SKIN / _TIMEOUT for this element */
  int32_t start;   /* how the run started: 0 the lattice (cold), 1 a snapshot
                      (mdgp_micro_plan_from) */
} mdgp_result;

/* Physics constants shared by all elements of a context. */
typedef struct {
  double dt;            /* time step (default 0.005) */
  double rc;            /* LJ cut-off (default 2.5); energy shifted, force truncated */
  double k_tether;      /* wall spring constant (default 150) */
  double gamma_wall;    /* Langevin friction on wall atoms, G-JF scheme (default 1) */
  double wall_density;  /* FCC wall number density (default 1) */
  double eps_wf, sig_wf;  /* wall-fluid LJ pair (default 1, 1) */
  double eps_ww, sig_ww;  /* wall-wall LJ pair (default 1, 1) */
  double fluid_margin;  /* gap between the wall plane and the fluid lattice (default 0.7) */
  double tau_T;         /* Berendsen time constant, mode 1 (default 0.5) */
  double mass;          /* atom mass (default 1) */
  int32_t n_blocks;     /* blocks for the standard error (default 10, max 64) */
  int32_t mode;         /* 0: tethered walls + Langevin wall thermostat; 1: frozen walls (no
                           wall-wall pairs) + Berendsen on the fluid's v_z with time constant tau_T
                           (paper App. A; pair it with eps_wf 0.2, sig_wf 0.75, wall_density 4,
                           rc 4, dt 0.0025, T 2.44 for the paper's parameters) */
  int32_t wall_planes;  /* FCC (100) planes per wall (default 3) */
  int32_t list_capacity;/* neighbour-list entries per atom (default 128; a batch that
                           overflows it is rerun by mdgp_micro_batch with twice as many) */
  double skin;          /* Verlet-list skin beyond r_c (default 0.4) */
  int32_t rebuild_every;/* eager paths (mdgp_micro_profile): steps between list rebuilds; 0 = from
                           the skin and T.  Graph replays rebuild when an atom has moved skin/2. */
  int32_t build_variant;/* list build: 0 or 3, the block-ballot build (one block of four warps
                           per cell, candidates culled to the cell's bounding box and then
                           its octants, lanes over candidates) -- the only one kept */
  int32_t persistent;   /* FP32 pair forces: 1 = the step loop is one persistent cooperative
                           kernel per list-rebuild interval (steps separated by a grid barrier,
                           inside a graph WHILE loop; default), 0 = one launch per step with a
                           conditional rebuild after each, 2 = the persistent
                           kernel launched by the host once per rebuild interval, without a
                           graph (a host round trip per interval: for profilers, which capture
                           ordinary launches).  FP64 pair forces always use 0.  Same results
                           every way. */
  int32_t wait_timeout_ms;  /* limit of every bounded device-side wait (the persistent step
                           loop's grid barrier), in milliseconds of the GPU's global timer
                           (default 2000; <= 0 takes the default).  A wait that runs out
                           ends the run and marks every element MDGP_E_TIMEOUT. */
  int32_t inject_barrier_skip;  /* test only (default 0): 1 makes one block of the persistent
                           step kernel leave out its first grid-barrier arrival, so that the
                           other blocks' bounded waits run out; the launch then ends with
                           MDGP_E_TIMEOUT for every element and the context stays usable. */
  int32_t threads_per_atom; /* FP32 persistent step loop: threads that share one atom's pair
                           loop, 1, 2, 4 or 8; 0 (default) = automatic: the largest that the
                           batch fills (several only for batches too small to occupy every SM
                           with one thread per atom), or, where the resident-atom kernel
                           applies (see resident), the largest from there down to two at which
                           it fits.  Results differ only by the summation order. */
  int32_t resident;     /* FP32 persistent step loop with several threads per atom and tethered
                           walls: 1 (default) = keep each atom's state and element constants in
                           registers and the block's lists in shared memory for a whole
                           list-rebuild interval (a step then reads global memory only for the
                           neighbour positions), when every block holds one chunk of atoms and
                           the shared memory fits; 0 = always the general persistent kernel.
                           The same trajectory bit for bit either way. */
} mdgp_md_params;

/* Fill *out with the defaults listed above.  Returns MDGP_E_ARG on null. */
int mdgp_md_params_default(mdgp_md_params* out);

/* Create a context on CUDA device `device` computing pair forces in
 * `precision` (mdgp_precision).  *out receives the handle; free it with
 * mdgp_destroy.  MDGP_E_CUDA if the device cannot be used. */
int mdgp_create(mdgp_ctx** out, int device, int precision);
int mdgp_destroy(mdgp_ctx* ctx);

/* Replace the physics constants (copied).  Invalidates any plan. */
int mdgp_set_md_params(mdgp_ctx* ctx, const mdgp_md_params* params);

/* Run all work of this context on `stream` (a cudaStream_t, not owned; it
 * must not be the legacy default stream, because the step loop is captured
 * into a CUDA graph).  0 selects the context's own non-blocking stream, which
 * is also the initial choice.  Invalidates any plan. */
int mdgp_set_stream(mdgp_ctx* ctx, void* stream);

/* Run n elements to completion and write n results (host arrays).  Blocking.
 * Equivalent to mdgp_micro_plan + mdgp_micro_launch + mdgp_micro_results.
 * Elements whose steps_eq + steps_sample differ run as separate sub-batches.
 * MDGP_E_ARG: n < 1, a null pointer, Lx or Lz < 3 r_c, h <= 2 fluid_margin,
 * density < 0, steps_sample < 0. */
int mdgp_micro_batch(mdgp_ctx* ctx, const mdgp_element* el, int64_t n, mdgp_result* out);

/* Plan a batch: validate, lay the atoms and cells out in device memory,
 * upload the element descriptors and capture the step loop in a CUDA graph.
 * *n_atoms (may be null) receives the total atom count.  All elements must
 * share steps_eq + steps_sample (MDGP_E_ARG otherwise). */
int mdgp_micro_plan(mdgp_ctx* ctx, const mdgp_element* el, int64_t n, int64_t* n_atoms);

/* Start state of one element: the final snapshot of an earlier run (paper
 * Sec. 2.4 and Algorithm 1: a new MD run starts from the final state of the
 * database entry most correlated with it, a cold run from a lattice with
 * zero mean velocity).  xv holds n_fluid + n_wall rows of
 * (x, y, z, vx, vy, vz), fluid first, then walls -- the order and the
 * absolute positions mdgp_micro_state gives; h, Lx, Lz are the geometry the
 * snapshot was taken in.  xv = null asks for a cold start. */
typedef struct {
  const float* xv;
  int64_t n_fluid, n_wall;
  double h, Lx, Lz;
} mdgp_start;

/* mdgp_micro_plan with start states (starts may be null: all cold; copied
 * during the call).  A snapshot taken at another h, Lx or Lz, or with
 * another wall atom count, gives a cold start (the paper starts from the
 * lattice when the database holds no entry at the channel height).
 * Otherwise the fluid and the walls start from the snapshot (positions
 * wrapped into the box in x and z).  Surplus fluid atoms are removed (those
 * with the smallest Philox key, counter (atom, 0, element id, 2)).  Missing
 * ones are inserted one at a time: the lowest-energy of 64 Philox-drawn
 * sites (counter (k, try, element id, 3)) of the slab [0.6, h - 0.6],
 * steepest descent of the new atom's shifted LJ energy (USHER, De Fabritiis
 * et al., J. Chem. Phys. 121, 12139 (2004)), then 60 steepest-descent steps
 * of it and the fluid atoms within 2 sigma (largest move 0.01 sigma a
 * step); velocities Maxwell-Boltzmann at T (counter (atom, 0, element id,
 * 4)) plus the snapshot's mean fluid velocity.  The potential energy the
 * insertions leave above the kept fluid's plus one mean per-atom energy
 * (sum over its pairs) per new atom is taken out of the fluid's peculiar
 * kinetic energy (down to a quarter at most).  A new atom left above
 * 1000 epsilon gives a cold start.  The tether anchors are the lattice
 * sites either way; mdgp_result.start reports what was used.  Elements are
 * prepared on up to 16 host threads. */
int mdgp_micro_plan_from(mdgp_ctx* ctx, const mdgp_element* el, int64_t n, const mdgp_start* starts,
                         int64_t* n_atoms);

/* The start state mdgp_micro_plan_from would give one element, computed on
 * the host (no device is touched): params may be null (the defaults);
 * *n_rows receives n_fluid + n_wall.  With xv non-null (cap >= *n_rows
 * rows of 6 doubles, else MDGP_E_ARG) *kind receives 0 for a cold start
 * (xv untouched: the lattice is built on the device) or 1 with xv filled
 * (x y z vx vy vz, fluid first, then walls). */
int mdgp_start_state(const mdgp_md_params* params, const mdgp_element* el, const mdgp_start* start, double* xv,
                     int64_t cap, int64_t* n_rows, int32_t* kind);

/* Enqueue the planned batch on the context's stream: build the elements,
 * replay the step graph, reduce the results on the device.  Asynchronous;
 * MDGP_E_STATE without a plan. */
int mdgp_micro_launch(mdgp_ctx* ctx);

/* Wait for the launched batch and copy its n results to the host. */
int mdgp_micro_results(mdgp_ctx* ctx, mdgp_result* out, int64_t n);

/* Number of kernels the last launched batch ran (graph nodes counted one by
 * one, including the neighbour-list rebuilds that ran); valid after
 * mdgp_micro_results. */
int64_t mdgp_micro_launch_count(const mdgp_ctx* ctx);

/* Which step loop the planned batch runs: 0 one launch per step (per-step
 * graphs), 1 the persistent kernel in a graph WHILE loop, 2 the persistent
 * kernel launched by the host.  MDGP_E_STATE without a plan. */
int mdgp_micro_path(const mdgp_ctx* ctx);

/* Continue the last launch's batch from where it ended: another
 * steps_eq + steps_sample steps (the plan's count) from the device state the
 * last mdgp_micro_launch or mdgp_micro_continue left, with every measurement
 * taken afresh over them (steps_eq of them unsampled, as in the plan) and the
 * energy drift measured from the continued start.  g_ext and dpdx (n
 * elements each, the plan's order; either may be NULL to keep the last
 * value) give each element's new forcing, Eq. momentumEq with the element's
 * density.  The Langevin noise continues its stream (the step counter of
 * the Philox counter runs on), so a plan of S steps continued once follows
 * the same trajectory as one of 2 S steps up to the summation order of a
 * list rebuilt at the boundary.  Used to run a full-channel MD in windows
 * with the forcing of each macro step (Sec. 3).  Enqueued on the context's
 * stream; results by mdgp_micro_results.  MDGP_E_STATE without a launch on
 * the current plan. */
int mdgp_micro_continue(mdgp_ctx* ctx, const double* g_ext, const double* dpdx);

/* Launch shape of the planned batch's persistent step kernel (FP32 pair
 * forces, persistent = 1 or 2) into out[0..4]: out[0] = blocks, out[1] =
 * threads per block, out[2] = atoms per block, out[3] = threads per atom in
 * the pair loop, out[4] = 1 when the kernel keeps the atoms resident (see
 * mdgp_md_params.resident), else 0.  MDGP_E_STATE without a plan or on the
 * per-step path. */
int mdgp_micro_launch_shape(const mdgp_ctx* ctx, int32_t* out);

/* With persistent = 2 (the host launches the persistent step kernel once
 * per list-rebuild interval): CUDA-event times of the last batch's
 * launches on the context's stream.  out[0] = total milliseconds inside
 * the persistent kernel, out[1] = the steps those launches ran, out[2] =
 * the launches, out[3] = total milliseconds of the rebuilds between them,
 * out[4] = those rebuilds.  MDGP_E_STATE unless the planned batch runs on
 * that path. */
int mdgp_micro_direct_timing(const mdgp_ctx* ctx, double* out);

/* Number of neighbour-list rebuilds the last batch ran (valid after
 * mdgp_micro_results).  A rebuild runs when some atom has moved more than
 * half the skin since the previous one. */
int64_t mdgp_micro_rebuild_count(const mdgp_ctx* ctx);

/* Copy the planned batch's current atom state to the host: positions and
 * velocities as (n_atoms x 3) row-major doubles, atoms ordered element by
 * element, fluid first then walls (either pointer may be null). */
int mdgp_micro_state(mdgp_ctx* ctx, double* x, double* v, int64_t n_atoms);

/* LJ pair forces of ONE element at the given positions (n_atoms x 3,
 * fluid then walls, as built for `el`), computed by the library's production
 * path (cell binning, cell-order sort, Verlet lists, list force kernel) in the
 * context's precision: forces (n_atoms x 3), each fluid
 * atom's x-virial share (half of x_ij F_x,ij for every pair it is in; 0 for
 * wall atoms) and per-atom shifted LJ energies (half per pair).  Any output
 * may be null. */
int mdgp_md_forces(mdgp_ctx* ctx, const mdgp_element* el, const double* x, int64_t n_atoms,
                   double* f, double* wxx, double* epot);

/* Time the planned batch's kernels one by one: rebuild the elements and run
 * the first `steps` steps without the graph, with CUDA events on the
 * context's stream around every launch.  FP64 pair forces: ms[0] = mean
 * integration kernel time, ms[1] = mean pair-force kernel time.  FP32 pair
 * forces (one fused launch per step: forces + integration): ms[0] = 0,
 * ms[1] = mean fused step time (with the frozen-wall thermostat, both of
 * its launches).  ms[2] = mean time of one whole neighbour-list rebuild (5
 * kernels); all in milliseconds; ms[3] = atoms, ms[4] = cells, ms[5] = steps
 * between rebuilds.  Leaves the batch state mid-run (launch it again for
 * results).  MDGP_E_STATE without a plan. */
int mdgp_micro_profile(mdgp_ctx* ctx, int64_t steps, double* ms);

/* ------------------------------------------------------------------------ */
/* Gaussian-process surrogate (paper Sec. 2.2), FP64 on the GPU.             */
/* ------------------------------------------------------------------------ */

typedef struct mdgp_gp mdgp_gp;

/* Hyperparameters theta = (sf2, l2, sn2) of Sec. 2.3 and the input scaling
 * of Eq. d2Eq. */
typedef struct {
  double sf2;              /* signal variance sigma_f^2 (> 0) */
  double l2;               /* length scale ell^2 in normalised input space (> 0) */
  double sn2;              /* noise variance sigma_n^2 added to the diagonal (Eq. covarianceEq, >= 0) */
  double fallback_scale;   /* scale used where the mean separation is undefined (< 2 entries or
                              zero spread); <= 0 means 1 */
  const double* fixed_scales; /* D scales to use instead of the database's mean separations, or null */
  const double* fallback_scales; /* D per-dimension fallbacks (entries <= 0 take fallback_scale),
                                    or null; copied during the call */
  double period;           /* 0: the squared-exponential kernel (Eq. quadraticKernelEq) on the scaled
                              inputs of Eq. d2Eq.  > 0: the periodic kernel of App. B
                              (Eq. periodicKernel), sf2 exp(-2 sin^2(pi |t - t'| / period) / l2),
                              on one input (D = 1, time) with no scaling; fixed_scales must be null */
  int32_t hold;            /* mdgp_gp_optimize only: bit mask of hyperparameters kept at their start
                              values (1 sf2, 2 l2, 4 sn2; App. B keeps sf2) */
  int32_t reserved;
} mdgp_gp_params;

/* Fit a GP to M database entries (Eqs. quadraticKernelEq, d2Eq,
 * covarianceEq): X is M x D row-major, y has M outputs, mu_X (nullable) the
 * prior mean at the inputs (zero in the paper; a learned mean otherwise).
 * The scale of dimension k is the mean of |x_ik - x_jk| over all pairs
 * i < j.  Builds C = K + sn2 I and its Cholesky factor and
 * alpha = C^-1 (y - mu_X) in FP64 on the device.  M = 0 gives the prior.
 * Limits: 0 <= M <= 16384, 1 <= D <= 8.  MDGP_E_NOTPD if C is not positive
 * definite.  *out is freed with mdgp_gp_free; it uses ctx's device and
 * stream and must not outlive ctx. */
int mdgp_gp_fit(mdgp_ctx* ctx, const double* X, const double* y, int64_t M, int32_t D,
                const mdgp_gp_params* params, const double* mu_X, mdgp_gp** out);

/* Factor the covariance of the inputs alone: the scales, C = K + sn2 I and
 * its Cholesky factor exactly as mdgp_gp_fit builds them, but no alpha.  The
 * posterior variance of Eq. predVarEq does not involve the outputs, so
 * Algorithm 1's gate can run on this handle before the MD results it waits
 * for exist; mdgp_gp_set_outputs adds them later on the same factor.  Until
 * then mdgp_gp_predict gives the variances and the prior mean (mu_Xs, or 0)
 * as the mean, and mdgp_gp_log_marginal fails with MDGP_E_ARG.  Arguments,
 * limits and errors as for mdgp_gp_fit. */
int mdgp_gp_fit_inputs(mdgp_ctx* ctx, const double* X, int64_t M, int32_t D, const mdgp_gp_params* params,
                       mdgp_gp** out);

/* Give a handle its M outputs y (and prior mean mu_X at the inputs,
 * nullable): solves alpha = C^-1 (y - mu_X) and the evidence terms on the
 * handle's existing factor (Eq. predMeanEq, Eq. evidenceEq).  The result is
 * the one mdgp_gp_fit gives for the same X, y, mu_X and params, bit for bit:
 * the same kernels run on the same factor.  May be called again with new
 * outputs for the same inputs.  Host arrays; blocking. */
int mdgp_gp_set_outputs(mdgp_gp* gp, const double* y, const double* mu_X);

/* Posterior at m queries Xs (m x D): mean = mu_Xs + K(Xs, X) alpha
 * (Eq. predMeanEq) and the latent variance sf2 - K(Xs, X) C^-1 K(X, Xs) on
 * the diagonal (Eq. predVarEq), clamped at 0.  mu_Xs may be null (zero prior
 * mean).  var may be null: the means alone, without the per-query
 * triangular solve the variance needs; mean may be null when var is not.
 * Host arrays; blocking. */
int mdgp_gp_predict(mdgp_gp* gp, const double* Xs, int64_t m, const double* mu_Xs, double* mean, double* var);

/* Allocation-free posterior (no counterpart in the paper: an addition for
 * callers that cannot call cudaMalloc while they run, such as applications
 * that hand all device memory to their own pool allocator up front, or
 * latency-bound loops where an allocation, which may synchronise the
 * device, is not acceptable).  Computes what mdgp_gp_fit followed by
 * mdgp_gp_predict computes, but every buffer beyond the caller's inputs and
 * outputs lives in one fixed device array inside the library (about 2 MiB,
 * held on every GPU that loads the library until the process exits); it
 * calls no allocator.
 *   X (M x D), y (M), mu_X (M, nullable), Xs (m x D), mu_Xs (m, nullable)
 *   and the outputs mean (m), var (m) are DEVICE pointers on the current
 *   device; params as for mdgp_gp_fit (fixed_scales must be null, period 0); stream is
 *   a cudaStream_t (0 = legacy default stream).
 *   Limits: 1 <= M <= 512 (MDGP_E_LIMIT beyond), 1 <= D <= 8.
 *   The first call on a device looks up the array's device address once
 *   (with that device current); make that first call before any stream
 *   capture.  Blocking: returns after the stream has finished the work, with
 *   MDGP_E_NOTPD if the covariance was not positive definite.
 *   Every call shares the one array: calls that can overlap on the GPU
 *   (from several host threads or streams) race and must be serialised by
 *   the caller.  The call clears what must start at zero itself. */
int mdgp_gp_posterior_noalloc(const double* X, const double* y, int64_t M, int32_t D,
                              const mdgp_gp_params* params, const double* mu_X, const double* Xs, int64_t m,
                              const double* mu_Xs, double* mean, double* var, void* stream);

/* The D input scales the fit used (Eq. d2Eq denominators); the period for
 * the periodic kernel. */
int mdgp_gp_scales(const mdgp_gp* gp, double* scales);

/* Log marginal likelihood of the fitted data (Eq. evidenceEq, Sec. 2.3):
 * -1/2 (y - mu)^T C^-1 (y - mu) - 1/2 log det C - M/2 log 2 pi, with the
 * fit's scales and hyperparameters; 0 for an empty database. */
int mdgp_gp_log_marginal(const mdgp_gp* gp, double* lml);

/* Hyperparameters by maximum evidence (Sec. 2.3): a pattern search over
 * (sf2, l2, sn2) from *start (its fallback and fixed scales, its kernel and
 * the values start->hold names are kept):
 * each coordinate in turn tries value x step and value / step and keeps the
 * better evidence (a gain above 1e-9 relative); a pass without a move takes
 * the square root of the step, from 4 down to 1.05, or until max_evals fits.
 * Every trial is a GPU fit.  A trial whose covariance is not positive
 * definite scores -inf.  *best receives the result and *best_lml (nullable)
 * its log marginal likelihood.  MDGP_E_ARG for M < 1. */
int mdgp_gp_optimize(mdgp_ctx* ctx, const double* X, const double* y, int64_t M, int32_t D,
                     const mdgp_gp_params* start, const double* mu_X, int32_t max_evals, mdgp_gp_params* best,
                     double* best_lml);
int mdgp_gp_free(mdgp_gp* gp);

/* ------------------------------------------------------------------------ */
/* Macro time step, Algorithm 1 (paper Sec. 2.4).                            */
/* ------------------------------------------------------------------------ */

typedef struct mdgp_hybrid mdgp_hybrid;

/* Converging-diverging periodic channel and its coupling (Sec. 2.1):
 * n_sections sections at x_j = j dx (Eq. subsEq, L = n_sections dx) with
 * h_j = h0 (1 - h_amp cos(2 pi x_j / L)); pressure p = eos_K (n - eos_n0);
 * forcing dP(t) = dP_amp sin(2 pi t / period), an inlet-outlet pressure
 * difference turned into the external force F_ext = dP / (L eos_n0) that
 * every fluid atom of the channel feels (Eq. momentumEq's F_ext); section
 * j's GP input is (h_j, G_j) with G_j = dp/dx_j - n_j F_ext (central
 * differences) and its MD element gets dpdx = G_j, i.e. the body force
 * F = F_ext - dp/dx_j / n_j (Eq. momentumEq); density update by Eq. continuityEq with
 * A_j = h_j Lz.  The MD elements are Lx x Lz x h_j at the section's density. */
typedef struct {
  int32_t n_sections;     /* >= 3 */
  int32_t sn2_from_data;  /* 1: sigma_n^2 = (mean standard error of the database runs)^2, taken
                             at the start of each step; 0: sn2 below */
  double dx, h0, Lx, Lz;
  double eos_K, eos_n0;
  double dP_amp, period, dt;  /* forcing amplitude and period; macro time step */
  double T;                   /* MD temperature */
  int64_t md_steps_eq, md_steps_sample;
  uint64_t seed;              /* MD seed; the k-th MD run of the case gets element id k */
  double sf2, l2, sn2;        /* q-GP hyperparameters (Sec. 2.3) */
  int32_t inputs;             /* q-GP inputs: 0 = (h, G); 1 = the paper's (h, n, F) with
                                 F = -G / n the force per unit mass on the fluid (Sec. 2.4) */
  int32_t factor_cache_mb;    /* device memory, in MiB, for the gate's covariance factors that a
                                 step keeps so that its means reuse them (0 = 4096; < 0 = keep
                                 none).  A factor not kept is computed again for the means, with
                                 the same result bit for bit. */
  int32_t warm_start;         /* 1: an MD run starts from the final snapshot of the database entry
                                 x_in that maximises K(x_in, x*) (Algorithm 1, Sec. 2.4), among the
                                 entries at the section's height the database held when the step
                                 began (none: the lattice), through
                                 mdgp_micro_plan_from, and equilibrates md_steps_eq_warm steps;
                                 0: every run starts from the lattice (default) */
  int32_t reserved2;
  int64_t md_steps_eq_warm;   /* equilibration steps of a warm-started run (0 = md_steps_eq / 4);
                                 with pseudo_nu > 0 the least of them */
  double pseudo_nu;           /* > 0: a warm-started run equilibrates for the start-up time t_s
                                 of mdgp_pseudo_md (Algorithm 1's pseudoMD) from x_in's force to
                                 x*'s, in MD steps, clamped to [md_steps_eq_warm, md_steps_eq];
                                 the fluid's kinematic viscosity (LJ units).  0: off (default) */
  double pseudo_slip;         /* Navier slip length of the walls for pseudoMD */
  double pseudo_eps_q;        /* pseudoMD's flow-rate tolerance (0 = sqrt(sn2) / 4) */
  double h_amp;               /* relative amplitude a of the height profile
                                 h_j = h0 (1 - a cos(2 pi x_j / L)), in [0, 1) (default 0.5; the
                                 paper's channel, Eq. heightEq, has a / mean height = 0.25) */
} mdgp_macro_params;

/* Time step statistics returned by mdgp_hybrid_step. */
typedef struct {
  int64_t step;           /* macro steps taken */
  double t;               /* macro time */
  int32_t md_runs;        /* MD runs this step */
  int32_t md_warm;        /* of which started from a snapshot (warm_start) */
  int64_t md_runs_total;
  int64_t db_size;        /* database entries after the step */
  int64_t md_atoms;       /* atoms over this step's MD runs */
  double q_mean;          /* section-averaged flow rate */
  double max_sd;          /* largest predicted standard deviation */
  double gp_seconds, md_seconds;  /* wall time in GP work and in the MD batch */
  int64_t md_steps_eq_warm;       /* equilibration steps of this step's warm-started runs (0: none) */
} mdgp_hybrid_stats;

/* Prior mean for the GP (a learned mean): fill out[0..m) at the m rows of
 * x (m x D row-major, D = 2 or 3 by mdgp_macro_params.inputs).  Return 0 on
 * success. */
typedef int (*mdgp_mean_fn)(void* user, const double* x, int64_t m, double* out);

int mdgp_macro_params_default(mdgp_macro_params* p);

/* Algorithm 1's pseudoMD (Sec. 2.4: the start-up time t_s of a new MD run
 * from a 1D Navier-Stokes solution with Navier slip), on the host.  The
 * streamwise velocity u(y, t) of a channel of height h obeys
 * du/dt = nu d2u/dy2 + g with u = slip du/dn at both walls (n into the
 * fluid); it starts at rest (from_rest = 1) or at the steady profile for
 * force g_from, and g_to drives it.  The flow rate is
 * Q(t) = q_scale * integral_0^h u dy (q_scale = m n Lz for the elements'
 * q).  *t_s receives the first time at which |Q(t) - Q_inf| <= eps_q (0
 * when it holds at t = 0).  Second-order finite differences on 64 cells
 * (the slip condition through a ghost node), implicit Euler in time with
 * steps of h^2 / (nu pi^2) / 1000, at most 10^6 of them (then
 * MDGP_E_LIMIT); Q_inf is the discrete steady state's.  A negative slip
 * places no-slip planes -slip inside each wall (the fluid between them and
 * the wall at rest): the flowing width is h + 2 slip.  MDGP_E_ARG unless
 * h, nu, q_scale, eps_q > 0 and h + 2 slip > 0. */
int mdgp_pseudo_md(double h, double nu, double slip, double g_from, double g_to, int32_t from_rest,
                   double q_scale, double eps_q, double* t_s);

/* New case: densities start at density0 (n_sections values, or eos_n0 when
 * null); empty database.  Uses ctx for the GP and MD work. */
int mdgp_hybrid_create(mdgp_ctx* ctx, const mdgp_macro_params* p, const double* density0, mdgp_hybrid** out);

/* Use fn (with user) as the GP prior mean from now on (null: zero mean).
 * mdgp_hybrid_set_mlp_mean needs the 2-input form (inputs = 0). */
int mdgp_hybrid_set_mean(mdgp_hybrid* h, mdgp_mean_fn fn, void* user);

/* One macro step with uncertainty threshold sigma_t (Algorithm 1): MD for
 * exactly the sections whose predicted standard deviation exceeds sigma_t
 * when Algorithm 1 reaches them, all of a step's MD runs in one batch.
 * sigma_t = 0 runs MD at every section without evaluating the GP (the
 * MD-everywhere reference; the database still grows).  MDGP_E_ARG for a
 * negative or NaN sigma_t. */
int mdgp_hybrid_step(mdgp_hybrid* h, double sigma_t, mdgp_hybrid_stats* stats);

/* Current per-section state (each pointer may be null; n_sections values):
 * density, flow rate of the last step, predicted standard deviation, 1 where
 * the flow rate came from MD, effective gradient G. */
int mdgp_hybrid_state(const mdgp_hybrid* h, double* density, double* q, double* sd, int32_t* from_md,
                      double* G);

/* Database: *M entries; with cap >= *M copies inputs (M x D, D = 2 or 3 by
 * mdgp_macro_params.inputs), outputs and standard errors (any may be null). */
int mdgp_hybrid_database(const mdgp_hybrid* h, double* X, double* y, double* se, int64_t cap, int64_t* M);

/* Pressure from a GP instead of the linear equation of state (the paper's
 * p-GP, Sec. 2.4): fit on M pre-simulation results, X (M x 2, row-major:
 * channel height h, density n) and measured pressures y, with hyperparameters
 * (sf2, l2, sn2) and the scales of Eq. d2Eq; every later step takes
 * p_j = its posterior mean at (h_j, n_j).  M = 0 returns to the linear law.
 * The arrays are copied.  MDGP_E_ARG on bad sizes or hyperparameters. */
int mdgp_hybrid_set_pressure(mdgp_hybrid* h, const double* X, const double* y, int64_t M, double sf2, double l2,
                             double sn2);
/* Replace the case's q database by M entries (X: M x D row-major with the
 * case's input layout; se may be null = 0); snapshots are dropped, the
 * prior mean is evaluated at the new inputs.  Sec. 3.3: a case may start
 * from the database an earlier case ended with. */
int mdgp_hybrid_set_database(mdgp_hybrid* h, const double* X, const double* y, const double* se, int64_t M);

/* Write the q database (and with with_snapshots != 0 each entry's final MD
 * snapshot, the warm-start source) to a file: "MDGPDB1\0", int32 D,
 * int32 with_snapshots, int64 M, double X[M D], y[M], se[M], then per
 * entry int64 n_fluid, n_wall, double h, g, float xv[6 (n_fluid + n_wall)]
 * (zero counts: no snapshot); little-endian host layout.  MDGP_E_ARG when
 * the file cannot be written. */
int mdgp_hybrid_save(const mdgp_hybrid* h, const char* path, int32_t with_snapshots);

/* Replace the case's q database (and snapshots, if the file has them) by a
 * file mdgp_hybrid_save wrote.  MDGP_E_ARG when the file is unreadable,
 * malformed or was written with another input dimension D; the case is
 * then unchanged. */
int mdgp_hybrid_load(mdgp_hybrid* h, const char* path);

int mdgp_hybrid_free(mdgp_hybrid* h);

/* ------------------------------------------------------------------------ */
/* Learned prior mean: MLP 2 -> 64 -> 64 -> 1 (benchmark addition; the       */
/* paper's GP has zero prior mean, Sec. 2.2 Eq. GPEq).                        */
/* ------------------------------------------------------------------------ */

typedef struct mdgp_mlp mdgp_mlp;

/* Full-batch Adam training settings. */
typedef struct {
  int32_t epochs;        /* Adam steps (default 2000) */
  int32_t eval_every;    /* holdout evaluation interval (default 20) */
  double lr, beta1, beta2, eps;  /* default 1e-3, 0.9, 0.999, 1e-8 */
  double holdout_frac;   /* rows held out for early stopping (default 0.2, in [0, 1)) */
  uint64_t seed;         /* split seed */
} mdgp_mlp_params;

int mdgp_mlp_params_default(mdgp_mlp_params* p);

/* Parameter count (4417): W1 (64 x 2), b1 (64), W2 (64 x 64), b2 (64),
 * W3 (64), b3 (1), FP32, row-major, a layer computing z = a W^T + b. */
int mdgp_mlp_num_params(void);

/* New network on ctx's device: initial parameters from init (num_params
 * floats) or, when null, uniform(+-1/sqrt(fan_in)) from `seed`. */
int mdgp_mlp_create(mdgp_ctx* ctx, const float* init, uint64_t seed, mdgp_mlp** out);
int mdgp_mlp_free(mdgp_mlp* m);

/* Train on n rows (X: n x 2 row-major, y: n): inputs and output are
 * standardised with the training rows' mean and deviation; every epoch is
 * one full-batch forward/backward (hidden layer products on the tensor cores
 * in BF16 with FP32 accumulation) and one Adam step on FP32 master weights;
 * the weights with the lowest holdout loss are kept.  Losses returned in
 * standardised units (either pointer may be null). */
int mdgp_mlp_train(mdgp_mlp* m, const double* X, const double* y, int64_t n, const mdgp_mlp_params* p,
                   double* train_loss, double* holdout_loss);

/* Network output in the original units at n rows of X (n x 2). */
int mdgp_mlp_predict(mdgp_mlp* m, const double* X, int64_t n, double* out);

/* Mean-squared-error loss and its gradient (num_params floats, may be null)
 * at the current weights for ALREADY STANDARDISED rows X (n x 2), y (n)
 * under the current standardiser (identity for a new network). */
int mdgp_mlp_loss_grad(mdgp_mlp* m, const double* X, const double* y, int64_t n, double* loss, float* grads);

/* One Adam step with the given gradient (num_params floats; null uses the
 * gradient accumulated on the device). */
int mdgp_mlp_adam_step(mdgp_mlp* m, const float* grads, const mdgp_mlp_params* p);

/* Copy the parameters (num_params floats) and the standardiser
 * (x mean[2], x std[2], y mean, y std) out of / into the network. */
int mdgp_mlp_get(const mdgp_mlp* m, float* params, double* standardiser);
int mdgp_mlp_set(mdgp_mlp* m, const float* params, const double* standardiser);

/* Use the network as the hybrid's GP prior mean (null: zero mean again). */
int mdgp_hybrid_set_mlp_mean(mdgp_hybrid* h, mdgp_mlp* m);

/* Choose the neighbour-list skin (0.3-0.6) for this batch by timing: each candidate runs the batch for probe_steps steps
 * (after one warm-up run) with CUDA events on the context's stream; the
 * fastest is kept in the context (and copied to *best, its atom-steps/s to
 * *best_rate; either may be null).  Results do not depend on the choice
 * beyond rounding. */
int mdgp_autotune(mdgp_ctx* ctx, const mdgp_element* el, int64_t n, int64_t probe_steps, mdgp_md_params* best,
                  double* best_rate);

/* Last CUDA error string seen by the context (static storage). */
const char* mdgp_last_error(const mdgp_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MDGP_H */
