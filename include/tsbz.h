/*
 * tsbz -- two-step Brillouin-zone sampling for real-time TDDFT on one GPU.
 *
 * C ABI of the propagation library.  The library advances many independent
 * sub-simulations (one shifted k-subgrid each, Sec. II.B steps 1-4 and
 * Eqs. 9-10) of the time-dependent Kohn-Sham equation (Eq. 1) with the
 * Hamiltonian of Eq. 2, and returns the density (Eq. 3) and the macroscopic
 * current (Eqs. 5-6) of each, plus their two-step average (Eq. 9).
 *
 * Conventions (all entry points):
 *  - Hartree atomic units; k and A are Cartesian (bohr^-1).
 *  - Grid arrays are [n3][n2][n1] with x (n1) fastest; orbital arrays of a
 *    sub-simulation are [n_k][n_bands][n3][n2][n1], interleaved complex
 *    (re, im) doubles; the k order is the caller's.
 *  - Every function returns a status: TSBZ_OK (0) or a negative TSBZ_E*
 *    code; tsbz_last_error() gives the text.  No C++ exception crosses the
 *    ABI.  A failed call leaves the context usable unless it returns
 *    TSBZ_ECUDA, after which only tsbz_last_error and tsbz_destroy are valid.
 *  - Input arrays are owned by the caller and are copied (host arrays) or
 *    read (device arrays) before the call returns; outputs go to caller
 *    buffers whose capacity (in doubles) is passed and checked.
 *  - The context owns its device memory.  It is obtained from the optional
 *    caller allocator (tsbz_alloc) or else from cudaMalloc, and released by
 *    tsbz_destroy.  Work is issued on the caller's stream (or the legacy
 *    default stream); calls that return host data synchronise that stream.
 *  - A context is not thread-safe; distinct contexts may be used from
 *    distinct threads.
 */
#ifndef TSBZ_H
#define TSBZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSBZ_OK 0
#define TSBZ_EINVAL (-1)     /* bad argument, size or capacity            */
#define TSBZ_ENOMEM (-2)     /* device or host allocation failed          */
#define TSBZ_ECUDA (-3)      /* a CUDA call failed                         */
#define TSBZ_ETIMEOUT (-4)   /* a bounded device wait gave up              */
#define TSBZ_ENONFINITE (-5) /* a non-finite current was produced          */
#define TSBZ_ESTATE (-6)     /* call out of order (e.g. no ground state)   */

/* Arithmetic of the propagation (a2-a5).  In every mode the density and
 * current are summed over k-points, bands and tiles in FP64 (or in float
 * two-sum pairs, which carry those sums to about 48 bits), and
 * the Hartree and XC potentials and the time integration of the observables
 * are FP64; in the single-precision modes the per-point and per-projector
 * terms themselves are formed from the float orbitals and projections in
 * float. */
#define TSBZ_FP64 0          /* everything in double                          */
#define TSBZ_FP32 1          /* stencil, Taylor and projectors in float; on
                                cells of at most 8 atoms with 16^3 grids the
                                projector contractions are factorised per axis
                                and their z contractions run on tensor cores
                                (three-product TF32, FP32 accumulate), fused
                                with the stencil in one kernel per stage      */
#define TSBZ_FP32_TC 2       /* as FP32 with dense projector GEMMs on tensor
                                cores in their own kernels (scaled split-FP16,
                                three products, FP32 accumulate)              */

/* Time step (tsbz_set_propagator). */
#define TSBZ_PROP_TAYLOR4 0  /* 4th-order Taylor with q = k + A(t_n + dt/2) and
                                v_Hxc[rho(t_n)] (the default)                 */
#define TSBZ_PROP_ETRS 1     /* enforced time-reversal symmetry: a Taylor-4
                                predictor gives rho~(t_{n+1}); then
                                T4(dt/2; A(t_{n+1}), v_Hxc[rho~])
                                T4(dt/2; A(t_n), v_Hxc[rho(t_n)])             */

#define TSBZ_HXC_SCF 0       /* v_Hxc[rho(t)] updated every step (Eq. 2)      */
#define TSBZ_HXC_FROZEN 1    /* v_Hxc kept at its loaded value                */

typedef struct tsbz_ctx tsbz_ctx;

/* Optional device allocator: alloc returns device memory of `bytes` bytes
 * aligned to at least 256 bytes, or NULL; free releases it. */
typedef struct {
  void* (*alloc)(size_t bytes, void* user);
  void (*free)(void* ptr, void* user);
  void* user;
} tsbz_alloc;

/* A cell and its synthetic norm-conserving pseudopotential (Eq. 2, Sec. III).
 *  - orthorhombic edges a[3] (bohr), grid n[3] (each fd_nd+1 .. 1024);
 *  - atoms at fractional positions atom_frac[3*n_atoms];
 *  - local part per atom: -z_ion erf(r/r_erf)/r + c_core exp(-r^2/(2 sigma_core^2)),
 *    defined through its Fourier series with the G = 0 Coulomb term removed;
 *  - projectors (if use_projectors): per atom one s and three p functions
 *    beta = N exp(-|d|^2/(2 r_proj^2)) * {1, d_x, d_y, d_z}, d the minimum-image
 *    displacement, zero unless every |d_ax|/h_ax < proj_half, each normalised
 *    to dV sum beta^2 = 1, energies e_kb_s and e_kb_p;
 *  - n_bands occupied bands with occupation occ each;
 *  - fd_nd: stencil half-width (1..6); hxc_mode: TSBZ_HXC_*;
 *  - xc: 0 none, 1 LDA Perdew-Zunger 81; hartree: 0/1. */
typedef struct {
  double a[3];
  int n[3];
  int n_atoms;
  const double* atom_frac;
  double z_ion, r_erf, c_core, sigma_core;
  double r_proj, proj_half, e_kb_s, e_kb_p;
  int use_projectors;
  int n_bands;
  double occ;
  int fd_nd;
  int hxc_mode;
  int xc;
  int hartree;
} tsbz_cell_desc;

/* Library version (major*10000 + minor*100 + patch). */
int tsbz_version(void);

/* Create a context on CUDA device `device` computing in `precision`
 * (TSBZ_FP64 / TSBZ_FP32 / TSBZ_FP32_TC).  `cuda_stream` is a cudaStream_t
 * or NULL; `alloc` may be NULL.  *out receives the context. */
int tsbz_create(tsbz_ctx** out, int device, int precision, void* cuda_stream, const tsbz_alloc* alloc);

/* Register a cell (Eq. 2's v_ion and grid); builds v_loc, the projector
 * tables and the FD weights on the host and copies them to the device. */
int tsbz_init_cell(tsbz_ctx* ctx, const tsbz_cell_desc* desc, int* cell_id);

/* Add one sub-simulation (Sec. II.B step 3): n_k k-points k_cart[n_k][3]
 * of cell `cell_id`, time step dt and a budget of max_steps steps (also the
 * capacity of its current history).  Sub-simulations of one context may
 * differ in cell, n_k, dt and budget.  Sub-simulations can only be added
 * before the first load_ground_state. */
int tsbz_add_subsim(tsbz_ctx* ctx, int cell_id, int n_k, const double* k_cart, double dt, int max_steps,
                    int* subsim_id);

/* Load the initial orbitals of a sub-simulation: psi is complex128
 * [n_k][n_bands][n3][n2][n1] (n_elems complex values), on the host
 * (psi_on_device = 0) or the device (1).  v_hxc_frozen ([n3][n2][n1] host
 * doubles) is required in TSBZ_HXC_FROZEN mode and ignored otherwise.
 * Computes rho(0), v_Hxc[rho(0)] and J(0-) (A = 0), and resets the step count.
 * A host upload is asynchronous: it is enqueued on the context stream and may
 * still be in flight when the call returns.  Page-locked host memory mapped
 * into the device's address space is read by the conversion kernel directly
 * (no staging copy); it, and a page-locked v_hxc_frozen, must stay unchanged
 * until a later call that waits for the device (tsbz_propagate,
 * tsbz_get_current, tsbz_get_density, tsbz_get_state, ...) has returned.
 * Pageable host memory is read before the call returns.  A device source is
 * copied and waited for before the call returns, so its owner may free it. */
int tsbz_load_ground_state(tsbz_ctx* ctx, int subsim_id, const double* psi, size_t n_elems, int psi_on_device,
                           const double* v_hxc_frozen);

/* Impulsive field of Eq. 11, read as A(t) = -k0 dir theta(t) (A = 0 before
 * the kick, -k0 dir from t = 0+ on).  subsim_id = -1 applies to all. */
int tsbz_set_kick(tsbz_ctx* ctx, int subsim_id, double k0, const double dir[3]);

/* General field: samples A(j dt/2), j = 0..2*n_steps, as [2 n_steps + 1][3]
 * (j = 0 is t = 0+); n_steps <= the sub-simulation's max_steps. */
int tsbz_set_field(tsbz_ctx* ctx, int subsim_id, int n_steps, const double* a_samples);

/* Advance every sub-simulation by n_steps 4th-order Taylor steps (Eq. 1 with
 * the step defined in the header of the CUDA sources): h uses
 * q = k + A(t_n + dt/2) and v_Hxc[rho(t_n)]; after the step rho, v_Hxc and
 * J(t_{n+1}) (q = k + A(t_{n+1})) are updated.  Step budgets are honoured:
 * a sub-simulation that reaches its max_steps stops there (its units skip
 * the remaining steps, decided on the device, so graph replays honour it
 * too) while the others go on; tsbz_get_step gives each one's count.
 * Returns when the work is complete; TSBZ_ENONFINITE names the first failing
 * sub-simulation. */
int tsbz_propagate(tsbz_ctx* ctx, int n_steps);

/* Current history J(t_j), j = first .. first+count-1 (j = 0 is t = 0+), as
 * [count][3], and J(0-) (nullable).  subsim_id = -1 returns the two-step
 * average (1/N_H) sum_m (J_m(t_j) - J_m(0-)) (Eq. 9, Sec. II.B step 4) and
 * J0_minus = 0; all sub-simulations then need the same dt. */
int tsbz_get_current(tsbz_ctx* ctx, int subsim_id, int first, int count, double* J, double* J0_minus);

/* The two-step mean of the current over all N_H sub-simulations (as
 * tsbz_get_current with subsim_id = -1, Eq. 9) together with its standard
 * error, the error bars of Sec. III.B (Fig. 6): the sub-simulations are N_H
 * data sets, so sigma_E(t_j) = sqrt( sum_m (dJ_m - mean)^2 / (N_H (N_H - 1)) )
 * per sample and component (0 when N_H = 1).  It is a true standard error
 * for random shifts; for Halton shifts it is the paper's indicator.  mean
 * and stderr_out are [count][3]; all sub-simulations need the same dt and at
 * least first + count - 1 steps.  FP64 on the host, fixed order. */
int tsbz_get_current_stats(tsbz_ctx* ctx, int first, int count, double* mean, double* stderr_out);

/* Density rho(r) = (1/N_k) sum_k sum_b occ |u_bk(r)|^2 (Eq. 3) of a
 * sub-simulation at its current step, [n3][n2][n1] doubles (cap >= n_pts). */
int tsbz_get_density(tsbz_ctx* ctx, int subsim_id, double* rho, size_t cap);

/* Orbital norms dV sum_r |u_bk(r)|^2 at the current step, [n_k][n_bands]. */
int tsbz_get_norms(tsbz_ctx* ctx, int subsim_id, double* norms, size_t cap);

/* Steps done by a sub-simulation. */
int tsbz_get_step(tsbz_ctx* ctx, int subsim_id, int* step);

/* Checkpoint: copy the orbitals out as complex128 (cap in complex values)
 * together with the step count; tsbz_load_state restores orbitals, step
 * count and recomputes rho and v_Hxc from them. */
int tsbz_get_state(tsbz_ctx* ctx, int subsim_id, double* psi, size_t cap, int* step);
int tsbz_load_state(tsbz_ctx* ctx, int subsim_id, const double* psi, size_t n_elems, int step);

/* The local potential and the projector normalisations of a cell as built
 * by tsbz_init_cell: vloc [n3][n2][n1] (cap >= n_pts), norms [4 n_atoms]. */
int tsbz_get_cell_tables(tsbz_ctx* ctx, int cell_id, double* vloc, size_t cap, double* proj_norms, size_t ncap);

/* Kernel launches issued by this context so far (for accounting). */
int tsbz_get_launch_count(tsbz_ctx* ctx, long long* launches);

/* Device time of the most recent tsbz_propagate (CUDA events on the
 * context stream, recorded only while profiling is on) split by kernel
 * family: times_ms[0..6] = {bra, stage, observe, finalize, hxc, field, ket}. */
int tsbz_get_timings(tsbz_ctx* ctx, double* times_ms, int n);
int tsbz_set_profiling(tsbz_ctx* ctx, int on);

/* Replay time steps from a CUDA graph (on = 1; default off).  The first
 * propagated step after enabling runs normally and is then captured once on
 * a stream the library owns; later steps replay the graph, ordered against
 * the caller's stream by events.  Profiling (tsbz_set_profiling) takes the
 * direct-launch path.  Set-up calls invalidate nothing: the graph reads the
 * step counters and field samples from device memory. */
int tsbz_set_graphs(tsbz_ctx* ctx, int on);

/* Kohn-Sham ground state on the GPU (the step before the propagation;
 * Sec. II.B step 2 starts every sub-simulation from converged orbitals): for
 * every sub-simulation, the n_bands lowest states of h_k at A = 0 on each of
 * its k-points with fixed occupations, self-consistent in rho on its own
 * k-set (frozen cells keep their v_Hxc).  Chebyshev-filtered subspace
 * iteration (filter of the given degree damping [lam + 0.1 Ha, b], lam the
 * block's largest Ritz value and b an upper bound of the spectrum; about 48
 * is a good degree; Cholesky-QR re-orthonormalisation)
 * with Pulay density mixing (history 8, mixing parameter mix) from a uniform
 * density, until dV sum |rho_out - rho_in| / N_e <= tol for every
 * sub-simulation.  The loaded orbitals are the starting block and are
 * replaced by an orthonormal basis of the converged occupied space (the
 * density, the current and every propagated observable depend on that space
 * only); rho, v_Hxc and J(0-) are then recomputed from them.  TSBZ_FP64
 * contexts, at most 256 bands per cell (TSBZ_EINVAL beyond), before the first
 * step.  Device scratch: five n_units n_b^2 complex matrices of the largest
 * cell, from the context's allocator.  *iters_out and
 * *err_out (nullable): iterations done and the last density error.  Returns
 * TSBZ_ESTATE when max_iter iterations did not converge. */
int tsbz_ground_state(tsbz_ctx* ctx, int max_iter, double tol, int degree, double mix, int* iters_out,
                      double* err_out);

/* Choose the time step (TSBZ_PROP_TAYLOR4 or TSBZ_PROP_ETRS).  The paper
 * leaves the propagator to its TDDFT code; ETRS costs three Taylor-4
 * expansions per step (predictor and two half steps) and keeps psi(t_n) and
 * v_eff(t_n) on the device during the step.  ETRS runs in TSBZ_FP64 and
 * TSBZ_FP32 (TSBZ_EINVAL in TSBZ_FP32_TC).  A captured step graph is dropped. */
int tsbz_set_propagator(tsbz_ctx* ctx, int propagator);

/* Autotuner of the batched launch (the per-cell choice of kernel variants:
 * tile shapes and schedules; the method itself is the same in every variant).
 * For each cell with more than one variant it runs, per variant, one untimed
 * step of every sub-simulation and then two windows of two timed steps (CUDA
 * events on the context stream; the faster window counts), the default
 * variant first and the others while budget_ms of device time lasts, and
 * keeps the fastest.  The trial steps are undone
 * afterwards: orbitals, projections, step counts, densities, potentials and
 * norms are restored bit for bit from a snapshot taken on the device (one
 * temporary copy of the orbitals, from the context's allocator), and no
 * current sample is exposed.  Results after tuning agree with the default
 * variant's within the arithmetic's rounding, not bit for bit.  A captured
 * step graph is dropped.  Needs loaded ground states and at least one
 * sub-simulation with steps left (TSBZ_ESTATE otherwise).  *n_tried
 * (nullable) receives the number of variants timed. */
int tsbz_autotune(tsbz_ctx* ctx, int budget_ms, int* n_tried);

/* The variant in force for a cell, the number it can run (n_variants) and the
 * ms per step the autotuner measured for each (ms[0..n_ms-1], 0 = untimed);
 * any output pointer may be NULL.  Variants: FP32 on 16^3 and 8^3 cells:
 * 0 = fused tensor-core / bulk-staged stage, 1 = z-march stage with CUDA-core
 * projections; point-parallel stage kernels (FP64, other FP32 shapes): bands
 * per staged projection chunk 8 (0), 4 (1), 16 (2). */
int tsbz_get_variant(tsbz_ctx* ctx, int cell_id, int* variant, int* n_variants, double* ms, int n_ms);

/* Force a cell's variant (0 <= variant < n_variants; TSBZ_EINVAL otherwise). */
int tsbz_set_variant(tsbz_ctx* ctx, int cell_id, int variant);

/* Self-test of failure detection without a GPU fault: one CTA on `device`
 * waits on a bulk-copy barrier with the same bounded wait the kernels use,
 * limited to `polls` polls (1 .. 2^24).  With deliver = 0 no copy is issued,
 * the wait runs out, the kernel records the timeout and returns, and the call
 * returns TSBZ_ETIMEOUT with the device still usable; with deliver = 1 the
 * 16-byte copy completes the barrier and the call returns TSBZ_OK.
 * *status_out (nullable) receives the kernel's status word. */
int tsbz_selftest_bounded_wait(int device, int polls, int deliver, int* status_out);

/* Arithmetic throughput probe (instrumentation; the paper has no counterpart):
 * the peak rate of fused multiply-adds on `device`, against which the
 * ALU-bound kernels of this library are measured.  kind 0 = FP32 FMA,
 * 1 = packed FP32x2 FMA (two FMAs per instruction), 2 = FP64 FMA.  One
 * untimed launch of a grid that fills every SM with independent FMA chains,
 * then the fastest of three timed launches (CUDA events); `iters` (1 .. 2^24)
 * sets the work per launch (64 FMAs per chain and iteration, 8 chains per
 * thread).  *flops_per_s receives 2 x FMAs / second, *ms_out (nullable) the
 * launch time.  Synchronous; uses the legacy default stream and a small
 * device allocation.  Returns TSBZ_OK, TSBZ_EINVAL, TSBZ_ENOMEM or TSBZ_ECUDA. */
int tsbz_probe_alu_peak(int device, int kind, int iters, double* flops_per_s, double* ms_out);

/* Self-test of the fifth-generation tensor-core building blocks that the
 * projector contractions use (instrumentation; the paper has no
 * counterpart): one CTA on `device` forms D = A B^T with M = 128, N = 32,
 * K = 16 as three TF32 products (A_lo B_hi + A_hi B_lo + A_hi B_hi, FP32
 * accumulation) by tcgen05.mma with A in tensor memory and B in shared memory
 * (canonical K-major layout, no swizzle), and copies D back.
 *  - a: host, row-major [128][16]; b: host, row-major [32][16] (B^T); d: host,
 *    row-major [128][32], written.  All owned by the caller.
 *  - swap_lbo_sbo: 0 = descriptor with the K-direction core-matrix stride as
 *    its leading-dimension offset (the layout the library uses), 1 = the two
 *    offsets exchanged (both stay inside the operand's buffer).
 *  - The MMA completion wait is bounded; a timeout returns TSBZ_ETIMEOUT with
 *    the tensor memory released.  *status_out (nullable): status word.
 *  - Synchronous; small device allocations.  Returns TSBZ_OK, TSBZ_EINVAL,
 *    TSBZ_ECUDA or TSBZ_ETIMEOUT. */
int tsbz_selftest_umma(int device, int swap_lbo_sbo, const float* a, const float* b, float* d, int* status_out);

const char* tsbz_last_error(tsbz_ctx* ctx);
void tsbz_destroy(tsbz_ctx* ctx);

/* ---- Host-side method helpers (no context, no GPU) ------------------------
 * k-points of the shifted Monkhorst-Pack grid of Eq. 10 (shift = 0 gives
 * Eq. 8): k = sum_j (2 n_j - N_j - 1 + 2 s_j)/(2 N_j) b_j with
 * b_j = (2 pi / a_j) e_j, each fractional coordinate wrapped into
 * [-1/2, 1/2); order n_1 fastest.  k_out has 3 * mp[0]*mp[1]*mp[2] doubles. */
int tsbz_shifted_kpoints(const double a[3], const int mp[3], const double shift[3], double* k_out, size_t cap);

/* First n points of the Halton sequence in bases 2, 3, 5 (index m = 1..n),
 * the quasi-random shifts of Sec. II.B; out has 3 n doubles. */
int tsbz_halton(int n, double* out, size_t cap);

/* Samples A(j dt/2), j = 0..2 n_steps, of the laser pulse of Eq. 15, read as
 * A(t) = -(e0/w0) dir sin^4(pi t/T) sin(w0 (t - T/2)) on (0, T), else 0. */
int tsbz_pulse_samples(double e0, double w0, double t_pulse, const double dir[3], double dt, int n_steps,
                       double* out, size_t cap);

/* ---- Allocation-free density ------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: code that runs inside another
 * framework's memory pool or a pre-sized arena, or a loop that must not hit
 * cudaMalloc's implicit device synchronisation.  It computes the density of
 * tsbz_get_density, rho(r) = (1/n_k) sum_k sum_b occ |u_bk(r)|^2, from
 * orbitals the caller already holds on the device, and allocates nothing:
 * its partial sums use a file-scope static device buffer of
 * TSBZ_NOALLOC_SCRATCH_DOUBLES doubles (2 MiB) that every GPU loading the
 * library keeps until the process exits.
 *  - psi: device, complex128 [n_k][n_bands][n3][n2][n1]; rho: device, doubles
 *    [n3][n2][n1], overwritten.  Both stay owned by the caller.
 *  - n3*n2*n1 must not exceed TSBZ_NOALLOC_SCRATCH_DOUBLES (TSBZ_EINVAL);
 *    any n_k is accepted (k-points are reduced in chunks that fit the buffer).
 *  - Work is queued on cuda_stream (NULL = legacy default stream); the call
 *    returns without synchronising.  The first call on a device looks up the
 *    buffer's device address once for that device; make that first call
 *    before any stream capture.  The address stays cached for the life of
 *    the process: after a cudaDeviceReset (or any reset of the device's
 *    primary context) the cached address is stale, so do not call this
 *    entry point again in that process.
 *  - All calls share the one buffer: calls that overlap on the GPU (other
 *    streams, other threads) race and must be serialised by the caller.
 *  - Returns TSBZ_OK, TSBZ_EINVAL or TSBZ_ECUDA. */
#define TSBZ_NOALLOC_SCRATCH_DOUBLES 262144
int tsbz_density_noalloc(const double* psi, int n_k, int n_bands, const int n[3], double occ, double* rho,
                         void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TSBZ_H */
