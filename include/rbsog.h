/*
 * rbsog.h -- C ABI of the GB300 (sm_103a) implementation of the random batch
 * sum-of-Gaussians (RBSOG) electrostatics for NPT molecular dynamics,
 * arXiv 2602.23582 (Jiang, Liang, Zhou).
 *
 * The library computes, per MD step and per system, Algorithm 1 of the paper:
 *   - the SOG short-range pair forces, energy and virial (sec. 2.2, 3.1;
 *     eqs. force_SOG, U_short, P_short) over cell lists rebuilt every step;
 *   - P Fourier modes drawn from the radial proposal by Metropolis-Hastings
 *     (App. D) and recalibrated for the non-radial target (sec. 3.2);
 *   - the structure factors rho(k) (eq. rho_k) of the distinct modes;
 *   - the random-batch force (App. B, eq. f_approx), energy and pressure
 *     estimators (eqs. P_approx_r, P_approx_nr);
 *   - a Langevin NPT integrator (eq. Langevin_NPT).
 *
 * Units are LAMMPS "real": Angstrom, fs, kcal/mol, e, g/mol, K, atm.  The
 * paper writes Coulomb in Gaussian units; every Coulomb energy, force and
 * virial is multiplied by params.ke.
 *
 * Conventions:
 *   - Every function returns an rbsog_status; rbsog_last_error() gives text.
 *     No exception crosses the ABI.
 *   - Host arrays passed in are copied; the caller keeps ownership.  Device
 *     pointers (on_device != 0) must be CUDA device memory of the current
 *     device, valid for the duration of the call; the library does not keep
 *     them.  The context owns every other device allocation.
 *   - Arrays of atoms are row-major N x 3 FP64 unless stated; atoms of all
 *     systems of a context are concatenated in system order.
 *   - The cell h is upper triangular, h = [[Lx, xy, xz], [0, Ly, yz], [0, 0, Lz]]
 *     (cell vectors as columns): box[3] are its edge lengths (Lx, Ly, Lz) and
 *     tilt[3] = (xy, xz, yz) its tilts, zero for an orthorhombic box.  A box
 *     whose perpendicular width along an axis (the edge itself when
 *     orthorhombic) is below (2 cell_sub + 1) r_c / cell_sub is rejected
 *     (RBSOG_EBOX).  A tilted (triclinic) cell is held fixed: it needs
 *     coupling RBSOG_COUPLE_FIXED, skin 0 and the paper sampler, in a context
 *     made by rbsog_create (RBSOG_EUNSUPPORTED otherwise); the Fourier modes
 *     are k = 2 pi h^{-T} m (eq. Sr) and the proposal of App. D is
 *     m* = round(h^T u) with the mass of eq. proposal.
 *   - Results depend only on (inputs, seed, rng_id, step): Philox4x64-10
 *     counters (step, purpose, index) under the key (seed, rng_id).
 */
#ifndef RBSOG_H
#define RBSOG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RBSOG_OK = 0,
    RBSOG_EINVAL = -1,        /* bad argument */
    RBSOG_ENOMEM = -2,        /* device or host allocation failed */
    RBSOG_EBOX = -3,          /* box edge < 3 r_c, or non-positive */
    RBSOG_ENONFINITE = -4,    /* non-finite force, energy or pressure */
    RBSOG_EUNSUPPORTED = -5,  /* option not supported */
    RBSOG_ETIMEOUT = -6,      /* a bounded device wait gave up */
    RBSOG_ECUDA = -7,         /* CUDA runtime error */
    RBSOG_EOVERFLOW = -8      /* a cell holds more atoms than the kernels take, or a
                                 request exceeds a fixed scratch */
} rbsog_status;

/* Sampler kinds (sec. 3.2, App. D). */
enum {
    RBSOG_SAMPLER_PAPER = 0,      /* MH radial chain (App. D) + recalibration chain */
    RBSOG_SAMPLER_IID = 1,        /* independent exact draws from P^r and P^nr */
    RBSOG_SAMPLER_IID_RECAL = 2   /* exact radial draws + recalibration chain */
};

/* Precision of the hot kernels. */
enum {
    RBSOG_FP64 = 0,               /* every step in FP64 */
    RBSOG_FP32 = 1                /* FP32 pair/sincos math, FP64 accumulation */
};

/* Pressure coupling of the barostat (eq. Langevin_NPT for a diagonal h). */
enum {
    RBSOG_COUPLE_ISO = 0,         /* one box momentum for x, y, z */
    RBSOG_COUPLE_SEMI_ISO = 1,    /* x = y coupled, z free */
    RBSOG_COUPLE_FIXED = 2        /* box held fixed (NVT) */
};

typedef struct {
    /* SOG split (sec. 2.2 / 3.1; Table 2 gives (b, sigma, omega) at r_c = 9 A,
     * sigma scales linearly with r_c) */
    double rc;              /* cutoff, A */
    double b, sigma, omega;
    int M;                  /* Gaussians of the force/pressure split (M = M~) */
    int M_energy;           /* Gaussians of the energy split, >= M */
    /* random batch (sec. 3.2) */
    int P;                  /* batch size, 1..4096 */
    int sampler;            /* RBSOG_SAMPLER_* */
    uint64_t seed;
    int precision;          /* RBSOG_FP64 or RBSOG_FP32 */
    double ke;              /* Coulomb constant, 332.06371 kcal A/(mol e^2) in real units */
    /* Langevin NPT (eq. Langevin_NPT) */
    double dt;              /* fs */
    double T;               /* K */
    double P_ext;           /* atm */
    double gamma;           /* 1/fs, particle friction */
    double gamma_box;       /* 1/fs, box friction */
    double tau_box;         /* fs, barostat period used to set the box mass */
    double compressibility; /* 1/atm, used to set the box mass */
    int coupling;           /* RBSOG_COUPLE_* */
    int cell_sub;           /* cells per cutoff length along an axis: 1 or 2; 0 = choose
                               (2 when a box edge is below 3.3 r_c, else 1) */
    int thermo_every;       /* energies (and the Coulomb/LJ split of the short-range
                               virial) are evaluated on steps whose counter is a
                               multiple of thermo_every (0: none), on the last step of
                               each rbsog_run call and by every rbsog_step; the other
                               steps compute forces and the total virial only, which is
                               all the dynamics uses.  Forces and the total virial do
                               not depend on this setting.  Default 1 (every step). */
    double skin;            /* A, FP32 build only (ignored in FP64): NPT steps keep the
                               pair lists of the last build, made with cells and a
                               candidate test at r_c + skin, while every atom's
                               displacement since that build (after the affine rescaling
                               of the box) stays below (min_a lambda_a (r_c + skin) - r_c)/2,
                               lambda_a = L_a / L_a at the build; then no pair within r_c
                               can be missing from them.  Otherwise, and on every
                               rbsog_step, the lists are rebuilt.  0: rebuilt every step.
                               The box must hold 2 cell_sub + 1 cells of (r_c + skin) /
                               cell_sub. */
    int cluster_cols;       /* FP32 build: sub-columns per cell axis of the in-cell atom
                               order that forms the pair kernel's 4-atom clusters, 1..4;
                               0 = from each system's density (about one cluster wide).
                               A launch-shape choice: results change only by FP32
                               rounding (each choice is deterministic). */
} rbsog_params;

typedef struct {
    int n_atoms;
    const double *q;        /* N charges, e */
    const double *mass;     /* N masses, g/mol */
    const int *type;        /* N LJ types in [0, ntypes) */
    const int *mol;         /* N molecule ids: atoms of a molecule contiguous; pairs
                               with equal ids are excluded from the pair sums */
    int ntypes;
    const double *lj_eps;   /* ntypes^2, kcal/mol (12-6, cut unshifted at rc) */
    const double *lj_sig;   /* ntypes^2, A */
    int n_bonds;
    const int *bonds;       /* n_bonds x 2 atom indices (within the system) */
    const double *bond_k;   /* U = k (r - r0)^2 */
    const double *bond_r0;
    int n_angles;
    const int *angles;      /* n_angles x 3, centre atom in the middle */
    const double *angle_k;  /* U = k (theta - theta0)^2 */
    const double *angle_t0;
    int n_excl;
    const int *excl;        /* n_excl x 2 intramolecular pairs whose Fourier-part
                               interaction is removed (all pairs of a molecule) */
    const double *r0;       /* N x 3 initial positions, A */
    const double *v0;       /* N x 3 initial velocities, A/fs, or NULL (zero) */
    double box[3];          /* edge lengths, A */
    uint64_t rng_id;        /* second word of this system's Philox key (seed, rng_id):
                               results do not depend on the system's place in a batch */
    double tilt[3];         /* (xy, xz, yz), A: tilts of a triclinic cell (all zero:
                               orthorhombic); see the conventions above */
} rbsog_system_desc;

/* Energies, kcal/mol: indices into rbsog_result.energy */
enum {
    RBSOG_E_COUL_SHORT = 0,  /* U^N (eq. U_short) */
    RBSOG_E_COUL_LONG = 1,   /* U^F* estimated with the radial samples */
    RBSOG_E_COUL_SELF = 2,   /* U_self (App. A) */
    RBSOG_E_COUL_EXCL = 3,   /* removed intramolecular Fourier-part energy */
    RBSOG_E_LJ = 4,
    RBSOG_E_BOND = 5,
    RBSOG_E_ANGLE = 6,
    RBSOG_E_COUL = 7,        /* short + long - self + excl */
    RBSOG_E_KIN = 8          /* kinetic energy */
};

typedef struct {
    double energy[9];        /* RBSOG_E_* */
    double virial[9];        /* total virial V P (no kinetic part), kcal/mol, row-major */
    double virial_coul_short[9];
    double virial_long_r[9]; /* V P^F,r*  (eq. P_approx_r) */
    double virial_long_nr[9];/* V P^F,nr* (eq. P_approx_nr) */
    double virial_lj[9];
    double virial_bonded[9]; /* bonds + angles + exclusion corrections */
    double pressure[9];      /* (kinetic + virial) / V, atm */
    double box[3];
    double volume;
    int n_distinct_modes;
    int n_accept_r, n_accept_nr;
    uint64_t step;
    int list_builds;         /* pair-list builds of this system so far (FP32 build) */
    double tilt[3];          /* (xy, xz, yz) of the cell */
} rbsog_result;

typedef struct rbsog_ctx rbsog_ctx;

/* Fill *p with the paper's working parameters: Table 2 row 2 (b =
 * 1.62976708826776469, omega = 1.007806979343806, sigma = 3.270345668108471
 * r_c / 9), M = M_energy = 10, P = 100, the paper MH sampler, FP32, and the
 * Langevin NPT settings of sec. 4.3 (0.1 ps / 0.5 ps, 4.5e-5 bar^-1). */
void rbsog_default_params(rbsog_params *p, double rc);

/* Create a context holding n_systems independent systems (the batched path:
 * every kernel launch covers all systems).  stream: cudaStream_t to run on
 * (NULL: a stream the context creates; it orders with the legacy stream).  Runs one force evaluation at step 0
 * so that rbsog_run can start. */
rbsog_status rbsog_create(const rbsog_params *params, int n_systems,
                          const rbsog_system_desc *systems, void *stream,
                          rbsog_ctx **out);

void rbsog_destroy(rbsog_ctx *ctx);

/* Text of the last error of ctx; with ctx == NULL, of the calling thread's
 * last failed rbsog_create. */
const char *rbsog_last_error(const rbsog_ctx *ctx);

/* Total atoms of all systems, and atom offset / count of system s. */
int rbsog_n_atoms(const rbsog_ctx *ctx);
rbsog_status rbsog_system_range(const rbsog_ctx *ctx, int s, int *atom0, int *n);

/* Replace the box of system s; rescale_positions != 0 scales its positions
 * affinely (r -> r L'/L).  A tilted cell is held fixed: RBSOG_EUNSUPPORTED. */
rbsog_status rbsog_set_box(rbsog_ctx *ctx, int s, const double box[3], int rescale_positions);

/* Copy positions (all systems, N_total x 3) in or out.  on_device: r is a
 * device pointer. */
rbsog_status rbsog_set_positions(rbsog_ctx *ctx, const double *r, int on_device);
rbsog_status rbsog_get_positions(rbsog_ctx *ctx, double *r, int on_device);
rbsog_status rbsog_get_velocities(rbsog_ctx *ctx, double *v, int on_device);

/* One force, energy and pressure evaluation of every system at the current
 * positions and boxes (Algorithm 1, steps 2-7) with Philox step counter
 * `step`.  forces (N_total x 3, kcal/(mol A)) may be NULL; results is an
 * array of n_systems entries or NULL.  The integrator state is not touched. */
rbsog_status rbsog_step(rbsog_ctx *ctx, uint64_t step, double *forces, int on_device,
                        rbsog_result *results);

/* One force-only evaluation of every system at the current positions and
 * boxes with Philox step counter `step`: the forces of eq. f_approx plus the
 * short-range, bonded and exclusion forces (sec. 2.2, 3.1), and the virial
 * tensor W of eqs. P_approx_r, P_approx_nr with the short-range and
 * molecule parts, the quantities an NPT step needs; no energies.  This is
 * the evaluation each step of rbsog_run performs (FP32 build: the cutoff
 * decided in FP32, the virial formed from the pair kernel's force sums), so
 * it costs less than rbsog_step.  forces: N_total x 3 (kcal/(mol A)), on the
 * host or (on_device = 1) the device, or NULL.  virial: n_systems x 9 doubles
 * on the host (row-major 3 x 3 per system, kcal/mol, the same tensor as
 * rbsog_result.virial), or NULL.  The integrator state is not touched.
 * Errors: as rbsog_step (RBSOG_EBOX, RBSOG_EOVERFLOW, RBSOG_ENONFINITE for a
 * system whose step failed; RBSOG_ECUDA). */
rbsog_status rbsog_step_forces(rbsog_ctx *ctx, uint64_t step, double *forces, int on_device,
                               double *virial);

/* Advance every system by nsteps Langevin NPT steps (Algorithm 1 step 8),
 * replaying a captured CUDA graph of one step.  last: n_systems results of
 * the final step, or NULL. */
rbsog_status rbsog_run(rbsog_ctx *ctx, int nsteps, rbsog_result *last);

/* Enqueue nsteps NPT steps on the context stream and return without waiting
 * or checking flags; rbsog_sync() waits and reports the flags (box too small,
 * cell overflow, non-finite results) raised since the last check. */
rbsog_status rbsog_run_async(rbsog_ctx *ctx, int nsteps);
rbsog_status rbsog_sync(rbsog_ctx *ctx);
/* Bounded wait for the steps enqueued on the context (a request loop that
 * must not block on the GPU): returns RBSOG_ETIMEOUT when they are still
 * running after timeout_ms (they keep running; call again, or rbsog_sync),
 * else what rbsog_sync returns.  The wait polls the stream (no device-side
 * wait is involved).  Errors: RBSOG_EINVAL (timeout_ms < 0 or not finite). */
rbsog_status rbsog_sync_timeout(rbsog_ctx *ctx, double timeout_ms);

/* Change thermo_every (rbsog_params) of a live context; every >= 0. */
rbsog_status rbsog_set_thermo_every(rbsog_ctx *ctx, int every);

/* The context stream (cudaStream_t) the library launches on. */
void *rbsog_stream(rbsog_ctx *ctx);

/* Checkpoint: the integrator state (positions, momenta, boxes, box momenta,
 * step counter).  buf == NULL returns the size in *len. */
rbsog_status rbsog_get_state(rbsog_ctx *ctx, void *buf, size_t *len);
rbsog_status rbsog_set_state(rbsog_ctx *ctx, const void *buf, size_t len);

/* Introspection of the last evaluation (for tests and diagnostics).
 * cells: ncell[3] and, per atom of system s, its cell index (x fastest).
 * modes: m^r (P x 3), m^nr (P x 3), distinct modes D (nD x 3) in
 * lexicographic order with multiplicities c_r, c_nr (arrays of >= P+1), the
 * normalizers S^r, S^nr and rho(k_d) (2 nD doubles, re/im interleaved). */
rbsog_status rbsog_debug_cells(rbsog_ctx *ctx, int s, int *ncell, int *cell_of_atom);
rbsog_status rbsog_debug_modes(rbsog_ctx *ctx, int s, int *mr, int *mnr, int *D, int *cr,
                               int *cnr, int *nD, double *S, double *rho);

/* Number of cudaMalloc and cudaFree calls the library has made in this
 * process so far (every thread, every context): a test shows with it that a
 * call allocates and frees nothing. */
unsigned long long rbsog_debug_device_alloc_calls(void);

/* Shared-proposal estimator of the non-radial long-range virial (sec. 3.2:
 * the P radial samples of the last evaluation reused for eq. PcoulFnr with
 * importance weights f_nr / P^r = S^r k^2 R(k), R(k) = sum_l w~_l s~_l^7
 * e^{-s~_l^2 k^2/4} / sum_l w~_l s~_l^5 e^{-s~_l^2 k^2/4}; the alternative that
 * the measure recalibration replaces).  out (host, n_systems x 9 doubles):
 * V P^F,nr,sh of every system, kcal/mol, row-major.  For comparing
 * estimators; the MD step does not use it.  Needs a previous evaluation
 * (rbsog_step, rbsog_run); runs on the context stream and synchronizes it.
 * Errors: RBSOG_EINVAL for a null argument, RBSOG_ECUDA. */
rbsog_status rbsog_virial_nr_shared(rbsog_ctx *ctx, double *out);

/* Kernel timings of the last rbsog_step / rbsog_run call with timing enabled:
 * enable != 0 records CUDA events around each kernel of one step (slower). */
rbsog_status rbsog_set_timing(rbsog_ctx *ctx, int enable);
rbsog_status rbsog_get_timing(rbsog_ctx *ctx, int max, char *names, double *ms, int *count);

/* ---- Pool of slots (the served path: many systems stepping in the same
 * kernel launches, entering and leaving at run time).
 *
 * A pool context has n_slots slots, each sized by its rbsog_slot_caps (the
 * cell grid takes boxes up to 1.15 max_box); all device memory is allocated
 * by rbsog_pool_create.  Slots start empty.  rbsog_run / rbsog_run_async
 * step every running slot together; a slot loaded with nsteps > 0 stops after
 * that many NPT steps (its state frozen, its last results kept) until it is
 * unloaded.  Each system keeps its own Philox counter (0 at its first
 * evaluation), so its trajectory does not depend on the other slots. */
typedef struct {
    int max_atoms, max_molecules, max_bonds, max_angles, max_excl, max_types;
    double max_box[3];
    double max_density;     /* atoms per A^3 a loaded system may reach (sizes the FP32 pair lists) */
} rbsog_slot_caps;

rbsog_status rbsog_pool_create(const rbsog_params *params, int n_slots, const rbsog_slot_caps *caps,
                               void *stream, rbsog_ctx **out);
/* Copy a system into an empty slot (host arrays as for rbsog_create; nsteps
 * > 0 or -1 for no limit).  Waits for the context stream.  Errors:
 * RBSOG_EINVAL (slot busy, system larger than the slot, bad system). */
rbsog_status rbsog_pool_load(rbsog_ctx *ctx, int slot, const rbsog_system_desc *sys, int nsteps);
/* Evaluate forces, energies and virial of every running slot at its current
 * counter: required after loading, before stepping (slots already running
 * recompute identical values).  Waits and checks the flags. */
rbsog_status rbsog_pool_prime(rbsog_ctx *ctx);
/* Per slot: 0 empty, 1 running, 2 finished, 3 stopped by a failure (its box
 * too small for the cell stencil, a cell overflow, non-finite results: err
 * holds the RBSOG_E* code; the other slots are not affected); step: its
 * Philox counter.  step and err may be NULL.  In a pool, rbsog_run and
 * rbsog_sync stop a failing system instead of returning its error. */
rbsog_status rbsog_pool_state(rbsog_ctx *ctx, int *state, unsigned long long *step, int *err);
/* Copy out positions (r), velocities (v) -- n x 3 host buffers of the slot's
 * system, either may be NULL -- and the results of its last step, then empty
 * the slot. */
rbsog_status rbsog_pool_unload(rbsog_ctx *ctx, int slot, double *r, double *v, rbsog_result *res);

/* ---- Request loop of the served path (rbsog_server.cpp, on the pool API).
 * rbsog_server_create sizes a pool to hbm_fraction of the free device memory
 * (at most n_slots slots, classes caps[0..n) in order).  Requests wait in
 * arrival order; each rbsog_server_pump call retires finished requests,
 * admits queued ones into free slots that fit them (first fit), primes them,
 * then advances every running slot up to max_steps NPT steps in the same
 * launches.  Step latencies (CUDA events per step) and aggregate atom-steps/s
 * over the pumped steps are kept for rbsog_server_stats.  rbsog_server_create
 * returns RBSOG_EINVAL for a null argument or hbm_fraction outside (0, 1],
 * RBSOG_ENOMEM when not even one slot fits the budget, RBSOG_ECUDA when the
 * free device memory cannot be queried, or the pool's own error. */
typedef struct rbsog_server rbsog_server;
rbsog_status rbsog_server_create(const rbsog_params *params, int n_slots, const rbsog_slot_caps *caps,
                                 double hbm_fraction, void *stream, rbsog_server **out);
void rbsog_server_destroy(rbsog_server *srv);
int rbsog_server_slots(const rbsog_server *srv);
rbsog_ctx *rbsog_server_context(rbsog_server *srv);
/* Queue a copy of `sys` for nsteps NPT steps; RBSOG_EUNSUPPORTED if it fits no slot. */
rbsog_status rbsog_server_submit(rbsog_server *srv, const rbsog_system_desc *sys, int nsteps,
                                 long long *ticket);
rbsog_status rbsog_server_pump(rbsog_server *srv, int max_steps, int *n_running, int *n_queued);
/* done = 1 once the request finished; then r, v (n x 3, may be NULL) and the
 * results of its last step.  Returns the request's own status once done
 * (RBSOG_OK, or why its system was stopped early, e.g. RBSOG_EBOX). */
rbsog_status rbsog_server_result(rbsog_server *srv, long long ticket, int *done, double *r, double *v,
                                 rbsog_result *res);
rbsog_status rbsog_server_stats(const rbsog_server *srv, double *p50_ms, double *p99_ms,
                                double *atom_steps_per_s, long long *steps, int *failed);

/* Pair-kernel trace for profiling inside a run: the next nsteps graph steps of
 * rbsog_run / rbsog_run_async record CUDA events immediately before and after
 * their pair kernel, on the context stream; rbsog_trace_pair_times waits for
 * the stream and returns the durations (ms) of the steps traced so far, in
 * order (at most max).  nsteps = 0 disarms.  Host cost: two graph-node
 * updates per traced launch; device cost: two event records. */
rbsog_status rbsog_trace_pair(rbsog_ctx *ctx, int nsteps);
rbsog_status rbsog_trace_pair_times(rbsog_ctx *ctx, int max, double *ms, int *count);

/* Stateless structure factor (eq. rho_k) on device buffers:
 *   r    device, N x 3 FP64 positions (any image)
 *   q    device, N FP64 charges
 *   m    device, nD x 3 int modes; k = 2 pi m / box
 *   rho  device, 2 nD FP64 (re, im), overwritten
 *   work device scratch of rbsog_structure_factor_workspace(N, nD) bytes
 * precision: RBSOG_FP64 or RBSOG_FP32.  Runs on `stream`. */
size_t rbsog_structure_factor_workspace(int n_atoms, int nD);
rbsog_status rbsog_structure_factor(const double *r, const double *q, int n_atoms,
                                    const double box[3], const int *m, int nD,
                                    double *rho, void *work, int precision, void *stream);

/* Allocation-free variant of rbsog_structure_factor (the paper has no
 * counterpart: this is an interface for host programs, not part of the
 * method).  Same arguments and results as rbsog_structure_factor, without
 * `work`: the scratch is a fixed 4 MiB device array inside the library, one
 * per device.  For callers that may not allocate device memory while they
 * run -- an MD engine that has handed all device memory to its own pool, or
 * that keeps work in flight on other streams, cannot let a call reach
 * cudaMalloc (which may fail mid-run) or cudaFree (which waits for the whole
 * device).  This call performs no device allocation or free.
 *   - Size limit: rbsog_structure_factor_workspace(n_atoms, nD) must not
 *     exceed 4 MiB (e.g. 100,000 atoms with up to ~1,600 modes); larger
 *     requests return RBSOG_EOVERFLOW before anything is launched, with the
 *     reason in rbsog_last_error(NULL).
 *   - The first call on a device does a one-time set-up (it looks up the
 *     scratch address with that device current); make that first call before
 *     any stream capture begins.
 *   - Calls on the same device must not overlap in time: two calls running at
 *     once on different streams share the scratch and race.
 *   - Nothing in the scratch needs clearing between calls.
 * Errors: RBSOG_EINVAL (null pointer, n_atoms < 1, nD < 1, bad precision),
 * RBSOG_EBOX (box edge <= 0), RBSOG_EOVERFLOW (too large), RBSOG_ECUDA. */
rbsog_status rbsog_structure_factor_noalloc(const double *r, const double *q, int n_atoms,
                                            const double box[3], const int *m, int nD,
                                            double *rho, int precision, void *stream);

/* ---- Autotuner (launch shapes per size class).  Times one NPT step of the
 * given systems for each candidate shape -- cell_sub in {1, 2} (where the
 * boxes hold the stencil of cells of r_c) x cluster_cols in {1, 2, 3, 4} in
 * the FP32 build; cell_sub alone in the FP64 build -- as the median of
 * `nsteps` graph steps after a warm-up, each candidate in a context of its
 * own on `stream`, and writes the fastest into *best (a copy of *params with
 * cell_sub and cluster_cols set).  times (may be NULL): ms per step of each
 * candidate, in the order cell_sub 1..2, then cluster_cols 1..4 (FP32: 8
 * entries, FP64: 2), negative for a candidate the boxes cannot take.  The
 * systems are not changed (each candidate steps its own copy).  Errors: as
 * rbsog_create; RBSOG_EINVAL when no candidate runs. */
rbsog_status rbsog_autotune(const rbsog_params *params, int n_systems, const rbsog_system_desc *systems,
                            int nsteps, void *stream, rbsog_params *best, double *times);

/* ---- Single-system decomposition over several GPUs (sec. 3.2; Algorithm 1,
 * steps 4-6): every rank draws the same modes from the same Philox key
 * (rbsog_modes), forms the partial structure factors of its own atoms
 * (rbsog_structure_factor on its slab), the partials are summed across
 * ranks by the caller (one all-reduce of 2 nD doubles), and every rank then
 * computes the long-range forces on its own atoms and the estimators from
 * the summed rho (rbsog_longrange_force) with no further exchange. */

/* Capacity the mode arrays of rbsog_modes need: P + 1 (paper and
 * recalibrated samplers) or 2 P (independent draws); 0 for a bad argument. */
int rbsog_modes_capacity(const rbsog_params *params);

/* The random batch of one evaluation, as a context with this box draws it
 * for a system keyed (params->seed, rng_id) at Philox counter `step`: the
 * App. D radial chain and the recalibration chain of sec. 3.2 (or the
 * sampler params->sampler names), reduced to the distinct modes.
 *   box  host, 3 edge lengths (orthorhombic h)
 *   D    host, >= 3 rbsog_modes_capacity(params) ints: the distinct modes m
 *        (k = 2 pi m / box) in lexicographic order, row-major nD x 3
 *   cr, cnr host, >= rbsog_modes_capacity(params) ints: multiplicities of
 *        each mode among the P radial and the P recalibrated samples
 *   nD   host, out: the number of distinct modes
 *   S    host, 2 doubles or NULL: the normalizers S^r, S^nr (eqs. Sr, Snr)
 * Runs on `stream` (cudaStream_t; NULL: the legacy stream), synchronizes it,
 * and allocates and frees a small device buffer.  Errors: RBSOG_EINVAL (null
 * argument, bad parameters), RBSOG_EBOX (box edge <= 0), RBSOG_ENOMEM,
 * RBSOG_ECUDA; the text is in rbsog_last_error(NULL). */
rbsog_status rbsog_modes(const rbsog_params *params, const double box[3], uint64_t rng_id, uint64_t step, int *D,
                         int *cr, int *cnr, int *nD, double *S, void *stream);

/* Random-batch long-range forces on n_atoms atoms from the structure factors
 * of the whole system (eq. f_approx: F_i = q_i sum_d alpha_d k_d
 * Im(e^{-i k_d . r_i} rho_d), alpha_d = -ke S^r c_r[d] / (2 P V k_d^2)), and
 * optionally the estimators of eqs. P_approx_r, P_approx_nr:
 *   r, q     device, n_atoms x 3 positions and n_atoms charges (FP64); the
 *            caller's atoms (a rank's slab), any image
 *   m, cr    device, nD x 3 modes and nD radial multiplicities (rbsog_modes)
 *   cnr      device, nD recalibrated multiplicities, or NULL (no P^F,nr*)
 *   rho      device, 2 nD FP64 (re, im): rho(k_d) summed over ALL atoms of
 *            the system (every rank's partial rbsog_structure_factor, summed)
 *   P, Sr, Snr, ke: batch size, normalizers (rbsog_modes) and Coulomb constant
 *   F        device, n_atoms x 3 FP64, overwritten (kcal/(mol A))
 *   est      host, 7 doubles or NULL: U^F* (= V tr P^F,r* / 3; kcal/mol) and
 *            V P^F,nr* (xx yy zz xy xz yz; kcal/mol).  With est the call
 *            synchronizes the stream; without, it only enqueues.
 *   work     device scratch of rbsog_longrange_force_workspace(nD) bytes
 * precision: RBSOG_FP64, or RBSOG_FP32 (FP32 phases from 32-bit fixed-point
 * fractional coordinates, FP64 sums).  Errors: RBSOG_EINVAL, RBSOG_EBOX,
 * RBSOG_ECUDA. */
size_t rbsog_longrange_force_workspace(int nD);
rbsog_status rbsog_longrange_force(const double *r, const double *q, int n_atoms, const double box[3], const int *m,
                                   const int *cr, const int *cnr, int nD, const double *rho, int P, double Sr,
                                   double Snr, double ke, double *F, double *est, void *work, int precision,
                                   void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RBSOG_H */
