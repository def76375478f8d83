/*
 * md.h -- C ABI of the GB300 (sm_103a) rigid multi-site molecular dynamics
 * hot path described in "ls1 mardyn: The massively parallel molecular
 * dynamics code for large systems" (Niethammer et al., arXiv 1408.4599).
 *
 * The library computes, on one GPU, the short-range forces, torques,
 * potential energy and virial of rigid molecules made of Lennard-Jones
 * centres, point charges, point dipoles and linear point quadrupoles
 * (§2), over a linked-cell grid with a centre-of-mass cut-off and periodic
 * boundaries (§3), with the reaction field for dipoles and the isotropic
 * long-range correction for dispersion (§3), together with the cell rebuild
 * and the leapfrog translational and rotational integrator (§3, Eqs. 2-5).
 *
 * Conventions shared by every entry point
 *   - Reduced units; k_B = k_C = 1 (§2, units paragraph).
 *   - Arrays are FP64, row-major: positions r, velocities v, angular
 *     momenta j, forces F and torques tau are n x 3; quaternions q are
 *     n x 4 as (w, x, y, z), unit, rotating body-frame vectors into the
 *     space frame.  j is the space-frame angular momentum.
 *   - Leapfrog state: v and j are half-step values v(t - dt/2), j(t - dt/2)
 *     (Eqs. 2 and 4); r and q are at time t.
 *   - Pointers flagged on_device are CUDA device pointers; otherwise host
 *     pointers (pageable or pinned).  The library copies inputs; the caller
 *     keeps ownership of every pointer it passes.  The library owns the
 *     device state it allocates and frees it in md_destroy.
 *   - cuda_stream is a cudaStream_t (NULL = the legacy default stream).
 *     Calls marked "asynchronous" only enqueue work on that stream.
 *   - Every function returns md_status; no exception crosses the ABI.
 *     Arguments are validated before anything is launched.  Faults found
 *     on the device (non-finite values, capacity overflow, a bounded wait
 *     that ran out) are recorded in device flags and returned by the next
 *     synchronising call (md_energy_virial, md_get_*, md_sync).
 *   - A handle is not thread-safe: one host thread at a time per handle.
 */
#ifndef MD_H
#define MD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct md_system md_system;
typedef struct md_batch md_batch;

typedef enum {
    MD_OK = 0,
    MD_ERR_ARG = -1,         /* invalid argument (NULL, NaN, out of range, bad model) */
    MD_ERR_BOX = -2,         /* box edge < 2 rc on some axis */
    MD_ERR_STATE = -3,       /* call out of order (e.g. no molecules set) */
    MD_ERR_CUDA = -4,        /* a CUDA runtime call failed; see md_last_error */
    MD_ERR_OOM = -5,         /* device allocation failed */
    MD_ERR_NONFINITE = -6,   /* non-finite force, torque or position detected */
    MD_ERR_OVERFLOW = -7,    /* a fixed-capacity buffer would overflow */
    MD_ERR_TIMEOUT = -8,     /* a bounded device wait gave up */
    MD_ERR_UNSUPPORTED = -9  /* valid input outside what the library supports */
} md_status;

/* One rigid component (molecule type), §2 "rigid rotators".  Positions are
 * body-frame offsets from the centre of mass in the principal-axes frame
 * (the library checks that the LJ-site masses put the centre of mass at the
 * origin and make the inertia tensor diagonal).  Masses sit on LJ centres.
 * Dipole and quadrupole axes are body-frame unit vectors; quadrupoles are
 * linear, Buckingham convention (Q = Theta_zz). */
typedef struct {
    int32_t n_lj;
    const double *lj_pos;    /* n_lj x 3 */
    const int32_t *lj_type;  /* n_lj, index into md_site_types.eps/sigma */
    const double *lj_mass;   /* n_lj */
    int32_t n_chg;
    const double *chg_pos;   /* n_chg x 3 */
    const double *chg_q;     /* n_chg */
    int32_t n_dip;
    const double *dip_pos;   /* n_dip x 3 */
    const double *dip_axis;  /* n_dip x 3 */
    const double *dip_mu;    /* n_dip */
    int32_t n_quad;
    const double *quad_pos;  /* n_quad x 3 */
    const double *quad_axis; /* n_quad x 3 */
    const double *quad_Q;    /* n_quad */
} md_component;

/* LJ types (§2, Eq. 1) with Lorentz-Berthelot mixing adjusted by binary
 * parameters: eps_ab = xi_ab sqrt(eps_a eps_b), sigma_ab = eta_ab
 * (sigma_a + sigma_b)/2.  xi, eta are n_types x n_types, NULL = all 1. */
typedef struct {
    int32_t n_types;
    const double *eps;
    const double *sigma;
    const double *xi;
    const double *eta;
    int32_t n_comp;          /* exactly 1 (one component per system) */
    const md_component *comp;
} md_site_types;

typedef struct {
    double eps_rf;           /* reaction-field continuum permittivity; INFINITY allowed (§3) */
    int32_t lj_shift;        /* 1: truncated-shifted LJ (LJTS, §2) */
    int32_t lj_lrc;          /* 1: report the isotropic long-range correction (§3) */
    int32_t deterministic;   /* 1: bitwise run-to-run reproducible (full shell, no atomics, cells
                              *    assigned to warps by a fixed stride).  0: cells are handed out
                              *    from a counter, so the energy, virial and md_param_grad sums
                              *    group differently per launch (last-bit differences) */
    int32_t half_shell;      /* 1: Newton-3 half-shell cell pairs (§3 figure on cell enumeration) */
    int32_t cell_div;        /* cells per cut-off length (§3): 1 (or 0): edge >= cutoff, 27-cell
                              *    stencil; 2: edge >= cutoff / 2, 125-cell stencil (15.6 instead
                              *    of 27 cutoff^3 examined around each molecule).  Same pairs and
                              *    results; the half shell needs >= 2 cell_div + 1 cells per axis */
} md_options;

typedef struct {
    double U_pot;            /* pair energy inside the cut-off */
    double U_lrc;            /* long-range correction (0 unless lj_lrc) */
    double U_rf_self;        /* reaction-field self energy, reported apart from U_pot */
    double K_trans, K_rot;   /* kinetic energies at time t (see md_energy_virial) */
    double W;                /* molecular virial sum_{i<j} R_ij . F_ij */
    double W_lrc;            /* long-range virial correction */
    double W_xx, W_yy, W_zz; /* diagonal of the molecular virial */
    double T;                /* 2 (K_trans + K_rot) / n_dof */
    double P;                /* (2 K_trans + W + W_lrc) / (3 V) */
    double time;             /* simulated time since md_set_molecules */
    int64_t step;            /* steps since md_set_molecules */
    int64_t n_mol_pairs;     /* interacting molecule pairs (unordered) */
    int64_t n_site_pairs;    /* interacting site pairs: n_mol_pairs * (n_lj^2 + n_el^2) */
    int64_t n_examined;      /* distance-tested molecule pairs (unordered) */
    int64_t n_molecules;
} md_observables;

/* Per-kernel timing gathered with CUDA events on the calling stream while
 * profiling is enabled (md_profile). */
typedef struct {
    int64_t launches[8];     /* [0] integrate [1] bin [2] pack [3] force [4] kinetic [5] batch [6] adjoint [7] other */
    double ms[8];
} md_kernel_times;

/* Creates a system: periodic box (edge lengths, each >= 2 cutoff), centre-
 * of-mass cut-off radius (§3), site types (§2) and options.  Cells of edge
 * >= cutoff / cell_div, floor(cell_div L / cutoff) per axis (§3 linked
 * cells).  Allocates no per-molecule memory yet.  Errors: MD_ERR_ARG (also
 * cell_div not 0, 1 or 2), MD_ERR_BOX, MD_ERR_UNSUPPORTED (more than one
 * component, > 8 merged sites or LJ types).  *out is set only on MD_OK. */
md_status md_create(const double box[3], double cutoff, const md_site_types *types, const md_options *options,
                    md_system **out);

/* Replaces the molecular state with n molecules (§2 rigid rotators).
 * comp_id may be NULL (all component 0).  r (n x 3), q (n x 4) required;
 * v, j may be NULL (zero).  Positions are wrapped into [0, L); quaternions
 * are renormalised.  The step counter restarts.  Asynchronous for device
 * input; host input is copied (and validated on the device) before return.
 * Errors: MD_ERR_ARG (NULL r/q, n < 0; for host input also a non-finite
 * value or a zero quaternion, after which no molecules are set),
 * MD_ERR_OOM; invalid device input is reported as MD_ERR_NONFINITE by the
 * next synchronising call. */
md_status md_set_molecules(md_system *sys, int64_t n, const int32_t *comp_id, const double *r, const double *v,
                           const double *q, const double *j, int32_t on_device, void *cuda_stream);

/* Rebuilds the cells (counting sort, §3) and evaluates forces, torques,
 * energy and virial at the current configuration (§3 force calculation
 * and summation).  Asynchronous; results stay on the device. */
md_status md_compute_forces(md_system *sys, void *cuda_stream);

/* n_steps leapfrog steps of size dt (Eqs. 2-5): half-kick/drift/rotate
 * with the current forces, wrap, rebuild cells, recompute forces.
 * T_target <= 0: NVE.  T_target > 0: NVT by velocity rescaling (§2,
 * ensembles): after the update of each step, v and j of every molecule are
 * scaled by sqrt(T_target / T_half), T_half = 2 (K_trans + K_rot) / dof of
 * the half-step state (v, j at t + dt/2, q at t + dt; dof = 3N - 3 + N x
 * rotational dof); positions and orientations of the step are unchanged.
 * Computes forces first if they are stale.  Asynchronous (the factor is
 * computed and applied on the device).  For n_steps >= 2 (profiling off)
 * pairs of steps are captured once as a CUDA graph per cell-buffer parity,
 * dt and T_target and replayed; the result is that of n_steps single steps
 * (bitwise with the deterministic full shell).  A graph is dropped when
 * the molecules or parameters change. */
md_status md_step(md_system *sys, int32_t n_steps, double dt, double T_target, void *cuda_stream);

/* Synchronising read-back of the observables at the current time t:
 * U, W from the last force evaluation; K from v(t) = v(t-dt/2) + dt/2 F/m
 * and j(t) = j(t-dt/2) + dt/2 tau with the dt of the last md_step (0 before
 * the first step); LRC from N, V (§3).  Returns any recorded device fault. */
md_status md_energy_virial(md_system *sys, md_observables *out);

/* Copies the state back in the caller's molecule order.  Any pointer may be
 * NULL to skip it.  Synchronising. */
md_status md_get_molecules(md_system *sys, double *r, double *v, double *q, double *j, int32_t on_device,
                           void *cuda_stream);

/* Copies forces and torques of the last evaluation in the caller's order.
 * Synchronising. */
md_status md_get_forces(md_system *sys, double *F, double *tau, int32_t on_device, void *cuda_stream);

/* Force-field parameters theta, in this order: eps_t and sigma_t of each LJ
 * type (Eq. 1), then each charge q, each dipole moment mu and each
 * quadrupole moment Q of the component (§2), in the md_component order.
 * md_n_params returns their number P (-1 for a NULL handle). */
int32_t md_n_params(const md_system *sys);
md_status md_get_params(md_system *sys, double *theta /* P, host */);

/* Replaces the parameters (same order; eps >= 0, sigma > 0, finite) and
 * recompiles the mixing tables; geometry is unchanged.  Forces become stale.
 * Errors: MD_ERR_ARG (wrong count or value; the old parameters stay). */
md_status md_set_params(md_system *sys, const double *theta, int32_t n_params);

/* Sensitivities for force-field fitting: d<U>/d theta and d<W>/d theta with
 * <.> the mean over n_cfg fixed configurations, U = pair energy + LRC and
 * W = molecular virial + LRC virial (§3).  Every pair term is recomputed
 * (nothing is stored from a forward pass).  r_all: n_cfg x n x 3, q_all:
 * n_cfg x n x 4 (host or device per on_device).  dU, dW: P doubles (host);
 * means[2] = <U>, <W> (host).  Synchronising.  The system is left holding
 * the last configuration with stale forces.  Errors: MD_ERR_ARG,
 * MD_ERR_UNSUPPORTED (site signature without a compiled adjoint, or a
 * system created with cell_div = 2). */
md_status md_param_grad(md_system *sys, int32_t n_cfg, int64_t n, const double *r_all, const double *q_all,
                        int32_t on_device, double *dU, double *dW, double *means, void *cuda_stream);

/* Number of molecules currently set. */
int64_t md_n_molecules(const md_system *sys);

/* Synchronises the stream and returns any recorded device fault. */
md_status md_sync(md_system *sys, void *cuda_stream);

/* Enables (1) or disables (0) CUDA-event timing of each kernel launch on
 * the stream the launch uses; md_kernel_times_get reads the totals. */
md_status md_profile(md_system *sys, int32_t enable);
md_status md_kernel_times_get(md_system *sys, md_kernel_times *out);

/* ------------------------------------------------------------------------
 * Batched replicas: n_sys independent systems of one model and cut-off,
 * each with its own periodic box and molecules, advanced together.  One
 * launch of each kernel covers every replica; the force kernels are
 * persistent and take cells from a work queue ordered longest-first by the
 * per-cell cost estimate n_d ~ N_i/2 (N_i + sum_neigh N_j) (§4, Eq. 6).
 * Replicas with >= 3 cells per axis use the Newton-3 half stencil when
 * options->half_shell is set, smaller boxes the full stencil.
 *
 * md_batch_create: boxes n_sys x 3 (host), each edge >= 2 cutoff.
 * Errors as md_create; MD_ERR_UNSUPPORTED for options->cell_div = 2 (the
 * replicas use cells of edge >= cutoff). */
md_status md_batch_create(int32_t n_sys, const double *boxes, double cutoff, const md_site_types *types,
                          const md_options *options, md_batch **out);

/* Molecules of all replicas, concatenated in replica order: n_per_sys[k]
 * molecules of replica k (host array of n_sys); r, v, q, j as in
 * md_set_molecules, sum(n_per_sys) rows each; v, j may be NULL. */
md_status md_batch_set_molecules(md_batch *b, const int64_t *n_per_sys, const double *r, const double *v,
                                 const double *q, const double *j, int32_t on_device, void *cuda_stream);

/* Forces of every replica at the current configuration.  Asynchronous. */
md_status md_batch_compute_forces(md_batch *b, void *cuda_stream);

/* n_steps leapfrog steps of every replica (NVE, or NVT for the replicas
 * given a target by md_batch_set_thermostat).  use_graph != 0 captures
 * pairs of steps into a CUDA graph once (per buffer parity and dt) and
 * replays it; an odd last step runs eagerly.  Asynchronous. */
md_status md_batch_step(md_batch *b, int32_t n_steps, double dt, int32_t use_graph, void *cuda_stream);

/* Per-replica NVT by velocity rescaling (§2, ensembles), as md_step with
 * T_target: T_target (host, n_sys; NULL = all NVE) > 0 gives replica k the
 * target T_target[k], <= 0 leaves it NVE.  The factors are computed on the
 * device every step (one block per replica) and applied while v and j are
 * reordered, so captured graphs need no host work.  Errors: MD_ERR_ARG
 * (non-finite target).  Synchronising. */
md_status md_batch_set_thermostat(md_batch *b, const double *T_target, void *cuda_stream);

/* Observables of every replica (out: n_sys entries, host).  Synchronising. */
md_status md_batch_energy_virial(md_batch *b, md_observables *out, void *cuda_stream);

/* State / forces of all replicas in the concatenated input order. */
md_status md_batch_get_molecules(md_batch *b, double *r, double *v, double *q, double *j, int32_t on_device,
                                 void *cuda_stream);
md_status md_batch_get_forces(md_batch *b, double *F, double *tau, int32_t on_device, void *cuda_stream);

/* Tiles of the batched force evaluation (§4: the same cost model orders
 * the work; these choose how it is cut). */
typedef struct {
    int32_t chunk;        /* cells per work-queue grab: 1, 2, 4 or 8 */
    int32_t grid_pct;     /* launched share of the resident blocks: 100 or 50 */
    int32_t test_width;   /* candidates per lane per distance-test round: 4 or 8 */
    double half_min_occ;  /* replicas whose mean occupancy (molecules per cell) is below this run the full
                           * 27-cell stencil instead of the Newton-3 half stencil: 0, 2 or 6 */
    float ms;             /* batched force evaluation with the chosen tiles (mean of 3, CUDA events) */
    float default_ms;     /* the same with the defaults (chunk 2, 100%, 8, 0) */
    int32_t from_cache;   /* 1: the choice came from the tuning cache, not from timing */
    char key[160];        /* cache key: GPU name | site signature | occupancy bucket (half-octaves) */
} md_batch_tuning;

/* Autotuner: times the batched force evaluation (CUDA events on
 * cuda_stream) over work chunk x grid share x test width x shell policy
 * (48 tile sets) and keeps the fastest.  cache_path (may be NULL): a text
 * file of earlier choices keyed by out->key; a hit is applied without
 * timing, a miss is timed and stored.  The default tile set is timed too
 * (out->default_ms) for the comparison.  Captured step graphs are dropped.
 * Synchronising.  Errors: MD_ERR_ARG (NULL b or out), MD_ERR_STATE (no
 * molecules set), MD_ERR_CUDA. */
md_status md_batch_tune_tiles(md_batch *b, void *cuda_stream, const char *cache_path, md_batch_tuning *out);

/* The same without a cache; outputs may be NULL. */
md_status md_batch_tune(md_batch *b, void *cuda_stream, int32_t *best_chunk, int32_t *best_grid_pct,
                        float *best_ms);

void md_batch_destroy(md_batch *b);
const char *md_batch_last_error(const md_batch *b);

/* Kinetic energies K_out[0] = sum 1/2 m v(t)^2 and K_out[1] = sum 1/2
 * w.I w at time t from half-step state, exactly as md_energy_virial forms
 * them (v(t) = v + dt/2 F/m, j(t) = j + dt/2 tau, w = I^-1 R(q)^T j(t)),
 * but as a stand-alone call that allocates no memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate:
 * programs whose own allocator has reserved the device memory up front and
 * must account for every byte, and loops that must not incur the
 * device-wide synchronisation of cudaFree.
 *   n: molecules, at most 8,388,608 (MD_ERR_OVERFLOW beyond).
 *   v, j, F, tau: device, n x 3 FP64; q: device, n x 4 FP64 unit
 *   quaternions; mass > 0 and the principal moments I[3] (host, >= 0; a
 *   zero moment contributes nothing); dt >= 0 (0 treats v, j as full-step).
 *   K_out: device, 2 doubles, written asynchronously on cuda_stream.
 * Scratch: a fixed 64 KiB file-scope device array, held by every GPU that
 * loads the library until the process exits.  The first call on a device
 * looks up the array's device address with that device current, so make
 * that first call before any stream capture.  All calls share the scratch:
 * calls whose work overlaps on the GPU (e.g. on different streams) race.
 * The looked-up address is kept for the life of the process, so a device
 * reset (cudaDeviceReset) after the first call on that device is not
 * supported.  MD_ERR_CUDA reports a failed look-up or launch of this call
 * only; an earlier error left pending by other work is not consumed.
 * Errors: MD_ERR_ARG, MD_ERR_OVERFLOW, MD_ERR_CUDA. */
md_status md_kinetic_noalloc(int64_t n, const double *v, const double *q, const double *j, const double *F,
                             const double *tau, double mass, const double I[3], double dt, double *K_out,
                             void *cuda_stream);

/* Measured FP32 FMA throughput of the current GPU: a full-occupancy grid of
 * threads, each running eight independent FMA chains, timed with CUDA
 * events on cuda_stream (best of three launches after one warm-up, ~5 ms
 * each).  paired = 0 issues scalar fma.rn.f32; paired = 1 the paired
 * fma.rn.f32x2 (two FMAs per instruction on sm_100-class GPUs).
 * out[0] = FLOP/s (an FMA counts 2), out[1] = ms of the best launch (host,
 * 2 doubles).  The paper has no counterpart: this is the measured
 * denominator of the force kernel's FP32 roofline, beside the unit-count
 * figure SMs x 128 lanes x 2 x clock.  Allocates and frees a small sink
 * buffer; synchronising.  Errors: MD_ERR_ARG (NULL out, paired not 0/1),
 * MD_ERR_OOM, MD_ERR_CUDA. */
md_status md_fp32_peak(int32_t paired, double *out, void *cuda_stream);

void md_destroy(md_system *sys);
const char *md_status_str(md_status s);
const char *md_last_error(const md_system *sys);

#ifdef __cplusplus
}
#endif
#endif
