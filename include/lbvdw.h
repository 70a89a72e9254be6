/*
 * lbvdw.h -- C ABI of the GB300 lattice Boltzmann library for N-component
 * van der Waals mixtures (Ridl & Wagner, "Lattice Boltzmann simulation of
 * mixtures with multicomponent van der Waals equation of state",
 * arXiv:1805.07251).
 *
 * One timestep (lb_step) performs, per node and component c, in one fused
 * CUDA kernel:
 *   1. moments rho^c = sum_i f_i^c and rho^c u^c = sum_i f_i^c v_i        (Sec. III)
 *   2. chemical potential
 *        mu^c = kT [ln(rho^c/eta) + b^c rho/eta] - sum_c' [2 a^{cc'} rho^c' + kappa^{cc'} Lap rho^c'],
 *      eta = 1 - sum_c b^c rho^c, rho = sum_c rho^c  (Eq. discreteChemicalPotential with
 *      the interaction function psi of Eqs. a-psi, kappa-psi and Sec. V folded into a
 *      lattice Laplacian)
 *   3. mean-field force gained by component c:
 *        "log" (Eq. forceMuLog):  G^{mu,c} = -gamma_mu rho^c D mu^c + theta D rho^c
 *        "nid" (Eq. forceMuId):   G^{mu,c} = -rho^c D (gamma_mu mu^c - theta ln rho^c)
 *   4. friction between components with the implicit velocity u-hat (Eq. forceFriction),
 *      solved exactly per node
 *   5. Psi correction (Eq. forceCorrectionsPsi)
 *   6. BGK collision towards the Hermite equilibrium (Eqs. BGKcollisionOperator, feq)
 *      plus the forcing populations with moments 0, G and G u + u G - Psi (Sec. III and
 *      the explicit D1Q3 update of Sec. V)
 *   7. streaming (Eq. LBequation), periodic in every direction.
 * theta = 1/3 is the lattice temperature (sound speed squared); kT is the
 * thermodynamic temperature in mu, p and F.  D is the central difference
 * (1/theta) sum_i w_i v_i phi(x + v_i), Lap the lattice Laplacian
 * (2/theta) sum_i w_i (phi(x + v_i) - phi(x)); in D1Q3 these are the central
 * difference and the three-point Laplacian of Sec. V.
 *
 * Conventions for every entry point:
 *   - Every call returns an lb_status; no C++ exception crosses this boundary.
 *   - Host arrays belong to the caller; the library copies in and out.  Device
 *     buffers of a context belong to the context until lb_destroy.
 *   - Field layouts (x fastest):  rho [c][y][x];  mom [c][d][y][x] with d = 0 (x),
 *     1 (y, D2Q9 only);  populations [c][i][y][x].
 *   - Lattice velocity order:  D1Q3: 0, +1, -1.  D2Q9: (0,0) (1,0) (0,1) (-1,0) (0,-1)
 *     (1,1) (-1,1) (-1,-1) (1,-1), weights 4/9, 1/9 x4, 1/36 x4.
 *   - Calls that read results back (lb_read_moments, lb_free_energy, lb_save_state)
 *     synchronise the context's stream and report any error the step kernels flagged
 *     since the last such call.  lb_step is asynchronous.
 *   - After LB_E_DOMAIN, LB_E_CUDA or LB_E_TIMEOUT the context is poisoned: every call
 *     but lb_init_fields*, lb_load_state, lb_last_error and lb_destroy returns LB_E_STATE
 *     until the fields are set again.
 *   - One context must not be used from two host threads at the same time.
 *   - Each call makes its context's device current while it runs and restores the
 *     calling thread's current device before returning.
 *   - Streams: NULL in lb_params.stream is CUDA's legacy default stream (a C ABI has no
 *     notion of a framework's "current" stream); the Python binding passes PyTorch's
 *     current stream when the caller names none.
 *   - Device memory of a context comes from cudaMalloc in lb_create (freed by
 *     lb_destroy); lb_free_energy_noalloc allocates nothing.
 */
#ifndef LBVDW_H
#define LBVDW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBVDW_ABI 3

typedef enum {
    LB_OK = 0,
    LB_E_INVALID = 1, /* bad argument or parameter set */
    LB_E_NOMEM = 2,   /* device or host allocation failed */
    LB_E_CUDA = 3,    /* a CUDA call failed; lb_last_error names it */
    LB_E_DOMAIN = 4,  /* rho^c <= 0, eta <= 0 or a non-finite value met in a step */
    LB_E_TIMEOUT = 5, /* a bounded device-side wait ran out */
    LB_E_STATE = 6    /* call out of order, or context poisoned */
} lb_status;

typedef enum { LB_D1Q3 = 1, LB_D2Q9 = 2 } lb_lattice;

typedef enum {
    LB_FP64 = 0,       /* populations and all arithmetic in FP64 */
    LB_FP32_MIXED = 1, /* FP32 populations stored as deviations f_i - w_i rho_ref^c;
                          FP64 in mu^c (eta, 1/eta, the logarithms -- a table-driven FP64
                          log -- and the differences of mu) and in mass sums */
    LB_FP32_DFMU = 2,  /* as LB_FP32_MIXED, with the FP64 operations of mu^c done in
                          double-float (pairs of FP32, ~44 significant bits) on the FP32
                          pipe; mass sums stay FP64 */
    LB_FP32 = 3        /* FP32 populations (deviations) and FP32 mu^c (CUDA's logf): no
                          FP64-class arithmetic in the step; measures what the FP64 mu of the
                          two modes above buys.  Single runs only (no batches, no adjoint) */
} lb_precision;

typedef enum { LB_FORCE_LOG = 0, LB_FORCE_NID = 1 } lb_force_method;

/* Organisation of the fused step kernel (the arithmetic, and so every result, is
 * the same bit for bit):
 *   LB_KERNEL_TILES   one CTA per tile_x x tile_y tile; each tile recomputes rho on a
 *                     2-node ring and mu on a 1-node ring around itself.
 *   LB_KERNEL_STRIPS  (D2Q9, FP32 storage) one CTA per column strip tile_x nodes wide
 *                     and per segment of its rows, walking down the segment tile_y
 *                     rows at a time; the populations of the rows ahead arrive in
 *                     shared memory by asynchronous bulk copies (cp.async.bulk with
 *                     mbarrier completion) while the current rows are collided.
 *                     Needs nx % tile_x == 0 and ny % tile_y == 0, with
 *                     (tile_x, tile_y) = (32, 8) for 1-2 components, (32, 4) for 3-4.
 *   LB_KERNEL_WS      (D2Q9, two components, LB_FP32_DFMU or LB_FP32, 32 x 8 tiles)
 *                     persistent warp-specialised tiles: per CTA, 4 loader warps stage
 *                     the next tile (populations, densities, momenta) in double-buffered
 *                     shared memory while 8 compute warps run mu and the collision of the
 *                     current one.  Bitwise the results of LB_KERNEL_TILES.
 *   LB_KERNEL_AUTO    tiles (measured faster on GB300 than the strips: 44.5k against
 *                     27.8k component-MLUPS for 2 components at 1024^2; the strips'
 *                     shared-memory staging leaves two CTAs, 18 warps, per SM). */
typedef enum { LB_KERNEL_AUTO = 0, LB_KERNEL_TILES = 1, LB_KERNEL_STRIPS = 2, LB_KERNEL_WS = 3 } lb_kernel_kind;

typedef struct {
    uint32_t abi;        /* must equal LBVDW_ABI */
    int32_t lattice;     /* lb_lattice */
    int32_t nx, ny;      /* nodes; ny == 1 for D1Q3; nx, ny >= 2 otherwise (nx >= 2 for D1Q3) */
    int32_t ncomp;       /* 1..4 components */
    int32_t precision;   /* lb_precision */
    int32_t force_method;/* lb_force_method */
    int32_t check_every; /* >0: lb_step synchronises and checks the error word every
                            check_every steps; 0: only calls that read back check it */
    double tau;          /* BGK relaxation time, > 1/2 */
    double kT;           /* thermodynamic temperature in mu, p, F; > 0 */
    double gamma_mu;     /* prefactor of mu in the force (Eq. forceMuNid); > 0 */
    double a[16];        /* a^{cc'} (Eq. a-psi), row major with row stride 4, symmetric */
    double kappa[16];    /* kappa^{cc'} (Eq. kappa-psi), stride 4, symmetric */
    double lambda[16];   /* friction lambda^{cc'} (Eq. forceFriction), stride 4, symmetric,
                            >= 0; diagonal ignored */
    double b[4];         /* excluded volume b^c > 0 */
    double rho_ref[4];   /* FP32 storage only: reference density of component c whose
                            rest equilibrium is subtracted before FP32 storage; 0 = use
                            the mean density set by lb_init_fields */
    int32_t device;      /* CUDA device ordinal */
    int32_t tile_x, tile_y; /* 0 = default; tiles: D2Q9 32x8, 64x4, 32x16 or 64x8,
                               D1Q3 128x1 or 256x1; strips: see lb_kernel_kind */
    int32_t kernel;      /* lb_kernel_kind */
    int32_t segments;    /* strips: row segments per strip (0 = enough CTAs to fill the
                            GPU once); ignored by tiles */
    void *stream;        /* cudaStream_t for every launch and copy; NULL = legacy default */
    /* Collision matrix of Eq. BGKcollisionOperator, diagonal in the D2Q9 Hermite moment
     * basis (D2Q9 only, tile kernel with 32 x 8 tiles; 0 = tau, i.e. BGK):
     *   tau_shear  relaxation time of the two shear moments (traceless second moment):
     *              kinematic viscosity theta (tau_shear - 1/2); 1/2 < tau_shear <= tau
     *              (larger values are unstable with the Psi correction);
     *   tau_ghost  relaxation time of the three ghost moments (third and fourth order),
     *              > 1/2.
     * The bulk moment (trace) keeps tau.  The Psi correction (Eq. forceCorrectionsPsi)
     * is taken per eigenspace: trace with tau, traceless part of G G / rho with
     * tau_shear.  With tau_shear = tau the stationary states are exactly those of BGK
     * for any tau_ghost; tau_shear < tau shifts coexisting densities by O(1e-3). */
    double tau_shear;
    double tau_ghost;
} lb_params;

typedef struct lb_ctx lb_ctx;

/* Fill *p with defaults: abi, D2Q9, 64 x 64, 2 components, FP64, "log", tau = 1,
 * kT = 1/3, gamma_mu = 1, a = 0, kappa = 0, lambda = 0, b = 0 (so callers must set
 * b before lb_create). */
void lb_default_params(lb_params *p);

/* Validate *p (symmetry of a, kappa, lambda; b > 0; tau > 1/2; sizes: nx ny <= 2^31, and
 * Q nx ny < 2^32 for the FP32 storage precisions) and create a
 * context on p->device: allocates two population buffers, a moments buffer and a
 * diagnostics scratch area with cudaMalloc (and, for the configurations whose steps
 * lb_step chains, one 32-bit completion flag per 32 x 8 tile).  No kernel runs.  On
 * success *out owns those buffers.  Errors: LB_E_INVALID, LB_E_NOMEM, LB_E_CUDA. */
lb_status lb_create(const lb_params *p, lb_ctx **out);

/* Set the state to the equilibrium (Eq. feq, at theta = 1/3) of host densities
 * rho [c][y][x] and momenta mom [c][d][y][x] (bare rho^c u^c; NULL = at rest).
 * Synchronous.  Clears the error word and the poisoned flag.  The fields are copied to
 * the device first; their check and (FP32 storage without rho_ref) their mean run there.
 * Errors: LB_E_INVALID (NULL ctx/rho), LB_E_DOMAIN (a density <= 0 or not finite, or
 * eta <= 0 at some node: the state is left unset), LB_E_CUDA. */
lb_status lb_init_fields(lb_ctx *ctx, const double *rho, const double *mom);

/* Same as lb_init_fields with device pointers (FP64, same layouts), enqueued on the
 * context stream; the caller keeps the buffers alive until the stream reaches it.
 * The domain check of the densities is deferred to the next read-back call. */
lb_status lb_init_fields_dev(lb_ctx *ctx, const double *rho_dev, const double *mom_dev);

/* Enqueue nsteps >= 0 timesteps (Eq. LBequation with the forces of Sec. III and V) on
 * the context stream.  Asynchronous unless check_every > 0.
 * Consecutive steps of one call are chained when the configuration allows it (D2Q9, two
 * components, LB_FP32_DFMU or LB_FP32, tiles of 32 x 8 with every ragged tile at least 3
 * nodes wide and high): step s + 1 launches while step s is finishing, and a tile of step
 * s + 1 that starts early waits on completion flags of the 3 x 3 tiles around it instead
 * of on the whole grid.  The results are bitwise those of one launch per step; a chain is
 * cut where check_every synchronises, a single step is always one plain launch, and steps
 * enqueued while the stream is being captured into a CUDA graph are plain launches.  A
 * chained wait is bounded (one second); one that runs out sets the error word's stall bit.
 * Errors: LB_E_STATE, LB_E_INVALID, LB_E_CUDA, LB_E_DOMAIN and LB_E_TIMEOUT (only when
 * check_every > 0). */
lb_status lb_step(lb_ctx *ctx, int64_t nsteps);

/* Copy rho^c [c][y][x] and bare momenta j^c = sum_i f_i^c v_i [c][d][y][x] of the
 * current state to host arrays (mom may be NULL).  The physical velocity of Sec. III
 * is u-hat^c = j^c/rho^c + G^c/(2 rho^c).  Synchronises; reports flagged errors. */
lb_status lb_read_moments(lb_ctx *ctx, double *rho, double *mom);

/* Device-pointer variant of lb_read_moments (FP64 outputs), enqueued on the context
 * stream; does not synchronise or check the error word. */
lb_status lb_read_moments_dev(lb_ctx *ctx, double *rho_dev, double *mom_dev);

/* Lattice free energy of Eq. discreteFreeEnergy of the current densities,
 *   F = sum_x [ sum_c kT rho^c ln(rho^c/eta) - sum_cc' a^{cc'} rho^c rho^c'
 *               - 1/2 sum_cc' kappa^{cc'} rho^c Lap rho^c' ],
 * per-component mass sum_x rho^c (mass[ncomp], may be NULL) and total momentum
 * sum_x sum_c j^c (mom_total[2], may be NULL), all reduced in FP64 in a fixed order
 * (one partial per CTA, then one CTA), so results are bitwise reproducible.
 * Synchronises; reports flagged errors. */
lb_status lb_free_energy(lb_ctx *ctx, double *F, double *mass, double *mom_total);

/* No-allocation variant of lb_free_energy for callers that cannot allocate device
 * memory (code inside another framework's memory pool or under a fixed memory budget,
 * tools handed a bare device pointer to a state, callers that must not trigger an
 * allocation in the middle of their own stream work).  The paper has no counterpart:
 * this is an interface convenience, not part of the method.
 *   p      parameters of the state (lattice, nx, ny, ncomp, precision, kT, a, kappa, b,
 *          device, stream; rho_ref must be set (> 0) for the FP32 precisions, as the
 *          stored populations are deviations from w_i rho_ref^c)
 *   f_dev  device populations [c][i][y][x] in the storage type of p->precision
 *   out_dev device output of ncomp + 4 doubles: mass[ncomp], F, sum j_x, sum j_y and an
 *          error flag (1.0 when a density or eta <= 0 or a non-finite value was met)
 * Enqueued on p->stream; returns without synchronising.  All scratch lives in one static
 * device array of 2^21 doubles (16 MiB) that every GPU loading the library holds until
 * exit; it fits ncomp * (1 + d) * nx * ny <= 2^21 - 7169 doubles (d = 1 for D1Q3, 2 for
 * D2Q9), e.g. a 512 x 512 D2Q9 lattice with two components; larger states are rejected
 * with LB_E_INVALID.  Every call shares the array and it keeps the last call's contents
 * (the error word is cleared at the start of each call); calls that overlap on the GPU
 * race, so serialise them.  Each call looks up the array's device address
 * (cudaGetSymbolAddress, which allocates nothing) with p->device current, so the address
 * stays right after a device reset; the first call on a device also loads the library's
 * module there, so make it before any stream capture.  The caller's current device is
 * restored before returning.  Calls no cudaMalloc, cudaFree or allocating library routine.
 * Errors: LB_E_INVALID, LB_E_CUDA. */
lb_status lb_free_energy_noalloc(const lb_params *p, const void *f_dev, double *out_dev);

/* ---- adjoint rollout -----------------------------------------------------------------
 * Reverse-mode gradients of a loss of the final densities with respect to the initial
 * densities and the mixture parameters a, kappa, b, through the hand-written transpose
 * of the fused timestep (Eqs. LBequation, BGKcollisionOperator, feq, forceCorrectionsPsi,
 * forceFriction, forceMuLog, discreteChemicalPotential; "log" force).  FP64 contexts get
 * an FP64 adjoint; FP32-storage contexts (LB_FP32_MIXED, LB_FP32_DFMU) an FP32 adjoint
 * whose chemical-potential recompute and Jacobian run in FP64, linearised at the FP32
 * forward trajectory.  Long rollouts keep a copy of the state every ckpt_every steps and
 * recompute each segment during the backward pass with the forward's own step kernel. */

/* Advance nsteps >= 1 timesteps from the current state (which must come from
 * lb_init_fields with mom = NULL for rho_bar_0 below to be the gradient with respect to
 * the initial densities), keeping (nsteps / ckpt_every + 1) device checkpoints in the
 * context's storage type.  Errors: LB_E_INVALID (precision LB_FP32 or the nid force),
 * LB_E_STATE, LB_E_NOMEM, LB_E_CUDA. */
lb_status lb_rollout_forward(lb_ctx *ctx, int64_t nsteps, int32_t ckpt_every);

/* Given rho_bar_T = dL/d rho at the end of the recorded rollout (host [c][y][x]), return
 * rho_bar_0 = dL/d rho_0 (host [c][y][x], may be NULL) and grad (host, may be NULL) =
 * [dL/da_cd (ncomp x ncomp, each entry taken as independent), dL/dkappa_cd (ncomp x ncomp),
 * dL/db_c (ncomp)].  For a symmetric pair a_12 = a_21 the gradient of the shared value is
 * the sum of the two entries.  Allocates ckpt_every states plus work arrays (in the
 * storage type; moments, chemical potential and gradient sums in FP64) for the duration
 * of the call; synchronises.  Errors: LB_E_INVALID, LB_E_STATE (no rollout),
 * LB_E_NOMEM, LB_E_CUDA. */
lb_status lb_rollout_backward(lb_ctx *ctx, const double *rho_bar_T, double *rho_bar_0, double *grad);

/* ---- batched independent runs (a phase-diagram sweep) --------------------------------
 * Many independent runs that share the mixture (ncomp, a, b, kappa, lambda, tau, force
 * method, precision) but differ in lattice, size, kT, gamma_mu and a kappa scale advance together on
 * one GPU.  Every run follows exactly the arithmetic of the same run advanced alone
 * through lb_create/lb_step (bitwise equal results).  D2Q9 runs: one kernel launch per
 * timestep over a flat list of tiles of all runs.  D1Q3 runs (2 <= nx <= 4096): one CTA
 * per run holds the whole run in shared memory for a chunk of timesteps.  lb_batch_step
 * replays CUDA graphs of 32-timestep chunks. */
typedef struct {
    int32_t lattice;  /* LB_D1Q3 (ny = 1, 2 <= nx <= 4096) or LB_D2Q9 (nx, ny >= 2) */
    int32_t nx, ny;
    double kT;        /* this run's thermodynamic temperature */
    double gamma_mu;  /* this run's gamma_mu */
    double kappa_scale; /* this run's kappa^{cc'} = kappa_scale * shared kappa^{cc'} (0 = 1):
                           a wider interface, the stabilisation of deep quenches (Sec. VI);
                           equilibrium bulk phases do not depend on kappa */
} lb_run_desc;

typedef struct lb_batch lb_batch;

/* Create a batch: shared->{abi, ncomp, precision, force_method, tau, a, kappa, lambda, b,
 * rho_ref, device, stream, tile_x, tile_y} apply to every run (tile: D2Q9 tile, 0 = 32x8;
 * lattice, nx, ny, kT, gamma_mu are taken from runs[]).  Allocates pooled buffers with
 * cudaMalloc.  Errors: LB_E_INVALID (bad run, D1Q3 run too long for shared memory),
 * LB_E_NOMEM, LB_E_CUDA. */
lb_status lb_batch_create(const lb_params *shared, const lb_run_desc *runs, int32_t nruns, lb_batch **out);

/* Equilibrium at rest of host densities: rho_all holds the runs one after another, each
 * in the layout [c][y][x].  Synchronous; clears the per-run error flags.
 * Errors: LB_E_INVALID, LB_E_DOMAIN (a density <= 0 or eta <= 0), LB_E_CUDA. */
lb_status lb_batch_init(lb_batch *b, const double *rho_all);

/* Enqueue nsteps timesteps of every run on the batch stream (asynchronous). */
lb_status lb_batch_step(lb_batch *b, int64_t nsteps);

/* Densities [c][y][x] and bare momenta [c][d][y][x] (may be NULL) of one run; synchronises. */
lb_status lb_batch_read(lb_batch *b, int32_t run, double *rho, double *mom);

/* Per-run error words (bit 0: a density or eta <= 0 or a non-finite value was met);
 * flags[nruns]; synchronises.  A failed run does not stop the others. */
lb_status lb_batch_errors(lb_batch *b, uint32_t *flags);

/* Select the D2Q9 tile (32x8, 64x4, 32x16 or 64x8); drops the captured graphs. */
lb_status lb_batch_set_tile(lb_batch *b, int32_t tile_x, int32_t tile_y);

/* Advance nsteps timesteps and return their device time in ms (CUDA events on the batch
 * stream; synchronises).  Used by the tile autotuner. */
lb_status lb_batch_time_steps(lb_batch *b, int32_t nsteps, double *ms);

int64_t lb_batch_step_count(const lb_batch *b);
int64_t lb_batch_launch_count(const lb_batch *b);
const char *lb_batch_last_error(const lb_batch *b);
lb_status lb_batch_destroy(lb_batch *b);

/* Size in bytes of a saved state, and save/load of the raw populations
 * ([c][i][y][x] in the storage type of the precision, plus a 64-byte header with the
 * step counter and a parameter hash).  lb_save_state synchronises; lb_load_state
 * checks the header against the context (LB_E_INVALID on mismatch). */
size_t lb_state_bytes(const lb_ctx *ctx);
lb_status lb_save_state(lb_ctx *ctx, void *host_buf, size_t bytes);
lb_status lb_load_state(lb_ctx *ctx, const void *host_buf, size_t bytes);

/* Number of timesteps taken since the state was last set (lb_init_fields,
 * lb_init_fields_dev or lb_load_state). */
int64_t lb_step_count(const lb_ctx *ctx);

/* Kernel launches enqueued by this context since creation (for launch accounting). */
int64_t lb_launch_count(const lb_ctx *ctx);

/* Whether lb_step chains consecutive steps of this context (see lb_step): the number of
 * 32 x 8 tile rows of a chained step that set completion flags for the next step, 0 when
 * the configuration is not chained, -1 for a NULL context. */
int32_t lb_chain_rows(const lb_ctx *ctx);

/* Whether the chained steps of this context load their input populations with an
 * evict-first L2 cache policy: 1 where one population buffer (N Q nx ny stored values) takes
 * at most 60 % of the device's L2, so that each step's output stays resident in the L2 for
 * the next step's reads; 0 otherwise or when not chained; -1 for a NULL context.  A cache
 * policy changes no result.  (Implementation choice of this library; the paper has no
 * counterpart.) */
int32_t lb_chain_evict_first(const lb_ctx *ctx);

/* Copy the context's parameters as resolved by lb_create (kernel organisation and
 * tile chosen for LB_KERNEL_AUTO and tile 0 x 0) into *out.  Errors: LB_E_INVALID
 * (NULL argument). */
lb_status lb_get_params(const lb_ctx *ctx, lb_params *out);

/* Release every device buffer of the context and the context itself (NULL is a no-op). */
lb_status lb_destroy(lb_ctx *ctx);

/* Static text of a status; last error message of a context (never NULL). */
const char *lb_status_str(lb_status s);
const char *lb_last_error(const lb_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* LBVDW_H */
