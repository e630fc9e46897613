/*
 * icarus.h -- C ABI of libicarus, the GB300 (sm_103a) hot path of the Icarus 3.0 dynamic
 * heliosphere model (Baratashvili et al., arXiv 2501.15923).
 *
 * What the library computes (paper references are to that article):
 *   - ideal MHD (Sect. 2, Eqs. 1-6: density, momentum, total energy, induction; p_tot =
 *     p + B^2/2, mu0 = 1, gamma given at init) in the frame co-rotating with the Sun
 *     (Sect. 2, Eqs. 2-3: F = rho (Omega x r) x Omega + 2 rho v x Omega in momentum, v.F in
 *     energy) with solar gravity (Sect. 2, g = GM/r^2, applied as an inward pull);
 *   - on a fixed spherical grid, radially stretched (dr ~ r) between r_in and r_out (Sect. 2,
 *     Sect. 3.2: stretched grid, latitude +-60 deg);
 *   - the r = r_in boundary driven by boundary maps interpolated linearly in time (Sect. 3),
 *     the same value in every ghost layer (Sect. 2.1), asymm for v_theta, v_phi, B_theta
 *     (Sect. 2.1), cone-CME injection (Sect. 3.2, "bc_icarus");
 *   - the solution sampled along moving spacecraft trajectories (Sect. 2, particle sampling).
 * The paper defers the scheme to its host framework; this library takes: limited linear
 * reconstruction of primitives (minmod / van Leer / MC), TVDLF or HLL fluxes, SSP-RK2,
 * two ghost layers, Linde-type div-B diffusion, dt = CFL / max_cells sum_d (|v_d|+c_f,d)/dx_d.
 *
 * Conventions
 *   - Every call returns 0 on success or a negative ICARUS_E* code; icarus_last_error() gives a
 *     message (thread-local). Host pointers are borrowed for the duration of the call only; the
 *     library copies what it keeps. Device memory belongs to the context (allocated at init
 *     through the allocator in icarus_options, cudaMalloc when none) and is released by
 *     icarus_destroy.
 *   - Units at the boundary of this API are SI unless a name says otherwise. Internally the
 *     library works in code units: L0 = 1 AU, v0 = 100 km/s, n0 = 1 cm^-3 (rho0 = m_p * 1e6
 *     kg/m^3), t0 = L0/v0, p0 = rho0 v0^2, B0 = sqrt(mu0 rho0) v0. State arrays exchanged by
 *     icarus_get_state / icarus_set_state are in code units.
 *   - State layout: [8][n3][n2][n1] doubles, index 1 (r) fastest; variables (rho, m_r, m_theta,
 *     m_phi, e, B_r, B_theta, B_phi). Theta is the colatitude.
 *   - icarus_step is asynchronous on the context stream. Device-side faults of the solution
 *     (non-finite state) are recorded in a sticky status word and reported by the next
 *     synchronising call (icarus_sample, icarus_get_state, icarus_status).
 */
#ifndef ICARUS_H
#define ICARUS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    ICARUS_OK = 0,
    ICARUS_EINVAL = -1,      /* bad argument (sizes, NULL pointers, unsupported option) */
    ICARUS_ESTATE = -2,      /* call made in the wrong order (e.g. step before boundary) */
    ICARUS_ENOMEM = -3,      /* device allocation failed */
    ICARUS_ECUDA = -4,       /* a CUDA runtime call failed */
    ICARUS_ENONFINITE = -5,  /* the solution became non-finite (sticky) */
    ICARUS_ETIMEOUT = -6,    /* a bounded device wait gave up (batched form, tensor-core closure) */
    ICARUS_EFLOOR = -7       /* a density or pressure floor acted while options.strict_floors is set
                                (sticky; ENONFINITE takes precedence when both occurred) */
};

enum { ICARUS_BC_PERIODIC = 0, ICARUS_BC_CONT = 1, ICARUS_BC_REFLECT = 2, ICARUS_BC_DRIVEN = 3 };
enum { ICARUS_GEOM_SPHERICAL = 0, ICARUS_GEOM_CARTESIAN = 1 };
enum { ICARUS_LIM_MINMOD = 0, ICARUS_LIM_VANLEER = 1, ICARUS_LIM_MC = 2 };
/* face fluxes: TVDLF (Rusanov), HLL, HLLD (Miyoshi & Kusano 2005; not in the fused stage or the
 * batched form) */
enum { ICARUS_FLUX_TVDLF = 0, ICARUS_FLUX_HLL = 1, ICARUS_FLUX_HLLD = 2 };
/* GLM (Dedner et al. 2002; a scheme variant, the paper names no div-B method): a scalar psi whose
 * upwind (B_n, psi) face state replaces the normal-field flux, carried with flux c_h^2 B_n*,
 * c_h = CFL dmin / dt, damped by exp(-glm_alpha c_h dt / dmin) per step; all three precision
 * forms (psi in the state's type), not the fused stage or the batched form. */
/* Powell (Powell et al. 1999; the eight-wave formulation): the source -(div B) (0, B, v.B, v) added
 * to the residual, div B of the cell from the face averages of the cell-centred field (the same
 * discrete divergence as the Linde term); all three precision forms, not the fused stage or the
 * batched form. */
enum { ICARUS_DIVB_NONE = 0, ICARUS_DIVB_LINDE = 1, ICARUS_DIVB_GLM = 2, ICARUS_DIVB_POWELL = 3 };
/* FP64: everything in double. FP32: state and arithmetic in float. MIXED: state, update
 * accumulation and the dt reduction in double; primitives, reconstruction, fluxes and sources in
 * float, except the primitive (pressure / positivity) recovery of the first four radial cells,
 * which stays in double. */
enum { ICARUS_FP64 = 0, ICARUS_FP32 = 1, ICARUS_MIXED = 2 };

typedef struct {
    int n1, n2, n3;        /* cells along r, theta, phi (x, y, z for Cartesian); each >= 1 */
    int geometry;          /* ICARUS_GEOM_* (Cartesian is for verification problems) */
    int stretch;           /* 1: r edges r_in (r_out/r_in)^(i/n1) (dr ~ r); 0: uniform */
    double x1min, x1max;   /* r range in AU (spherical) */
    double x2min, x2max;   /* colatitude range in rad (spherical; inside (0, pi)) */
    double x3min, x3max;   /* longitude range in rad, co-rotating frame (spherical) */
    int bc[6];             /* ICARUS_BC_* for (1-, 1+, 2-, 2+, 3-, 3+); DRIVEN only at 1- */
    int band_refine;       /* static refinement band (a fixed stand-in for the adaptive refinement
                              of Sect. 2): > 1 makes the radial cells band_refine times narrower
                              in [band_lo, band_hi] (in ln r when stretched) than outside, with n1
                              cells in all; 0 or 1: no band; at most 64 */
    double band_lo, band_hi;   /* the band, x1min < band_lo < band_hi < x1max (AU) */
} icarus_grid;

typedef void *(*icarus_alloc_fn)(size_t bytes, void *user);
typedef void (*icarus_free_fn)(void *ptr, void *user);

typedef struct {
    double cfl;            /* Courant number (0, 1] */
    int limiter;           /* ICARUS_LIM_* */
    int flux;              /* ICARUS_FLUX_* */
    int gravity;           /* 1: solar gravity on */
    int divb;              /* ICARUS_DIVB_* */
    double divb_coef;      /* Linde coefficient C_d */
    double rho_floor;      /* density floor, code units */
    double p_floor;        /* pressure floor, code units */
    int precision;         /* ICARUS_FP64 | ICARUS_FP32 | ICARUS_MIXED */
    int ring_capacity;     /* probe records kept on the device between drains (>= 1) */
    void *cuda_stream;     /* cudaStream_t to run on; NULL: the library creates its own */
    icarus_alloc_fn alloc; /* device allocator (NULL: cudaMalloc); must return 256-B aligned */
    icarus_free_fn free;   /* matching free (NULL: cudaFree) */
    void *alloc_user;      /* passed to alloc / free */
    int fused;             /* kernel sequence of a stage (the same arithmetic in each):
                              0: default. FP32 and MIXED with TVDLF / HLL and without GLM or the
                              tracer: theta- and phi-flux kernels, then one update kernel that
                              forms the r-face fluxes of its radial row segment in shared memory
                              (no r-flux array in HBM, one launch fewer); everything else: the
                              separate r-, theta-, phi-flux kernels and the update.
                              1: one fused stage kernel (fluxes, div B, update), FP32 and MIXED
                              only, TVDLF / HLL, Linde or no div-B control, no tracer. It keeps all
                              face fluxes on chip, but on GB300 it is about 2x slower than the
                              separate kernels: they are not bandwidth-bound, and the fused kernel
                              runs at half their occupancy and recomputes each face's neighbouring
                              slopes.
                              2: the separate kernels everywhere (the r-flux kernel too).
                              Other values: EINVAL */
    int init_vphi;         /* initial state's v_phi (Sect. 2.1 names none): ICARUS_IC_COROTATING
                              (0: at rest in the co-rotating frame) or ICARUS_IC_INERTIAL_RADIAL
                              (1: v_phi = -Omega r sin(theta), the inertially radial flow, parallel
                              to the spiral field) */
    int cme_model;         /* cone CME at the inner boundary (Sect. 3.2): ICARUS_CME_WINDOW (0): the cone
                              of the half-width over [t_on, t_on + duration); ICARUS_CME_SPHERE (1): a
                              spherical cloud of radius r_in sin(half-width) moving out along the
                              axis at the CME speed, its leading point at r_in at t_on; the footprint
                              is the part of the r_in sphere inside the cloud, for 2 R / speed (the
                              duration entry is not used) */
    int tracer;            /* 1: carry the CME tracer c (Sect. 3.2 marks inserted CME plasma): rho c is
                              conserved, moved by the mass flux with the limited upwind c, c = 1 on
                              the driven face inside the CME footprint and 0 outside, rho c clipped
                              to [0, rho] after each stage; starts at c = 0 (icarus_set_tracer).
                              Not with the fused stage kernel or the batched form. */
    double glm_alpha;      /* divb = ICARUS_DIVB_GLM: psi damping constant (>= 0; 0.1 is usual) */
    int strict_floors;     /* 1: a floor activation is an error: the step still applies the floor (and
                              counts it), and the context's sticky status becomes ICARUS_EFLOOR, which
                              the synchronising calls and later icarus_step calls return; 0: floors
                              are only counted (icarus_status) */
} icarus_options;

#define ICARUS_IC_COROTATING 0
#define ICARUS_IC_INERTIAL_RADIAL 1
#define ICARUS_CME_WINDOW 0
#define ICARUS_CME_SPHERE 1

typedef struct icarus_ctx icarus_ctx;

/* Create a solver context on the current CUDA device: uploads the grid metrics (computed on
 * the host in double), allocates the state, flux and scratch buffers.
 * gamma: adiabatic index (Sect. 2: 1.5). omega_rot: rotation rate of the frame in rad/s (Sect. 2,
 * the Sun's rotation). *out receives the context. EINVAL on bad sizes or options. */
int icarus_init(const icarus_grid *grid, double gamma, double omega_rot,
                const icarus_options *opts, icarus_ctx **out);

/* Set the inner-boundary driving (Sect. 3): n_maps >= 1 maps at times t_maps[n_maps] (s,
 * strictly increasing), maps[n_maps][5][n2][n3] in SI with fields (v_r m/s, n m^-3, p Pa,
 * B_r T, B_phi T) at the grid's angular cell centres; between map times the values are linear
 * in time, outside the table they are clamped to the first / last map. n_cme cone CMEs
 * cmes[n_cme][8] = (t_on s, duration s, lat rad, lon rad (co-rotating), half_width rad,
 * speed m/s, n m^-3, T K); inside the cone during [t_on, t_on + duration) the boundary takes
 * v_r = speed, n, p = 2 n k_B T (Sect. 3.2). The first call also sets the initial state from
 * the maps at the current time by radial expansion (Sect. 2.1) and computes the first dt.
 * Later calls replace the maps and CMEs only. The maps are copied to the device as given (one DMA
 * when the caller's array is in pinned host memory) and scaled to code units there. Synchronous. */
int icarus_set_boundary(icarus_ctx *ctx, int n_maps, const double *t_maps, const double *maps,
                        int n_cme, const double *cmes);

/* Advance n >= 0 time steps (each: dt from the CFL bound, SSP-RK2 with the boundary refilled at
 * each stage time, probes recorded at the new time). Asynchronous on the context stream; the
 * steps run as replays of a captured CUDA graph. ESTATE before the first set_boundary /
 * set_state. Returns, without synchronising, the sticky status of the steps that have completed
 * on the device (each step's last kernel copies the status word into host-mapped memory):
 * ENONFINITE or EFLOOR, and then launches nothing. Steps still in flight report at a later call;
 * icarus_set_state clears the status. */
int icarus_step(icarus_ctx *ctx, int n);

/* Advance n >= 0 time steps like icarus_step, recovering from a failed attempt. The explicit
 * scheme of Sect. 2 is stable only below a Courant limit, and a run whose flow outgrows the
 * configured number (a violent transient: colliding streams, a fast CME front) shows it as a
 * negative pressure or density (a floor activation, reported when options.strict_floors is set)
 * or a non-finite state. Before the steps the state, the CME tracer and GLM psi (when carried), the
 * time, dt, probe-ring position and floor count are copied on the device into a snapshot
 * (allocated on first use, one state's worth). The call then synchronises and reads the status:
 * on ENONFINITE or EFLOOR it restores the snapshot, halves the CFL number (dt recomputed from the
 * restored state) and runs the n steps again, at most max_retries times (0 <= max_retries <= 20).
 * A retry's probe records replace the failed attempt's. After a retry succeeds, the configured CFL
 * number is put back and the next dt recomputed with it. *halvings (may be NULL) receives the
 * halvings the returned attempt used. Returns ICARUS_OK, or, once the retries are spent, the last
 * attempt's ENONFINITE / EFLOOR with the snapshot restored (configured CFL, its dt) and that
 * status kept (sticky, as after icarus_step). The status the context already had is returned at
 * once, without stepping. Synchronous. */
int icarus_step_recover(icarus_ctx *ctx, int n, int max_retries, int *halvings);

/* Probe sampling (Sect. 2). traj[n_probes][n_knots][4] = (t s, r m, lat rad, lon rad in the
 * inertial frame, unwrapped), knots in increasing t. If traj is non-NULL it is registered for
 * the following steps and the current state is sampled once at the current time. Then the
 * records kept on the device since the last drain are copied, oldest first, into
 * out[cap][n_probes][13] = (t s, n m^-3, v_r, v_theta, v_phi (inertial) m/s, B_r, B_theta,
 * B_phi T, p Pa, |B| T, i, j, k), with (i, j, k) the lower corner of the 2x2x2 cell-centre
 * stencil used for the trilinear interpolation. *n_written receives the number of records
 * (at most cap; older records beyond the ring capacity are lost). Synchronous. */
int icarus_sample(icarus_ctx *ctx, int n_probes, int n_knots, const double *traj,
                  double *out, int cap, int *n_written);

/* Release all device memory of the context (synchronises its stream first). */
int icarus_destroy(icarus_ctx *ctx);

/* Copy the interior state [8][n3][n2][n1] (code units, double) and the time (code units) to
 * the host. Synchronous; returns ENONFINITE if the status word is set. */
int icarus_get_state(icarus_ctx *ctx, double *U, double *t);

/* Replace the interior state (code units, double) and the time (code units); recomputes dt.
 * Synchronous. Enables stepping without boundary maps when no face is DRIVEN. */
int icarus_set_state(icarus_ctx *ctx, const double *U, double t);

/* CME tracer (options.tracer = 1): set c of the interior cells from HOST doubles [n3][n2][n1]
 * (rho c = rho * c with the current rho), or copy c = rho c / rho back to the host. Synchronous.
 * EINVAL without the tracer option, ESTATE before a state exists. icarus_set_state keeps rho c
 * (so c changes with rho). */
int icarus_set_tracer(icarus_ctx *ctx, const double *c);
int icarus_get_tracer(icarus_ctx *ctx, double *c);

/* GLM div-B control (divb = ICARUS_DIVB_GLM): psi of the interior cells as HOST doubles
 * [n3][n2][n1] (code units of B times speed), set or read. Synchronous. EINVAL without GLM.
 * psi starts at 0 and is kept by icarus_set_state. */
int icarus_set_psi(icarus_ctx *ctx, const double *psi);
int icarus_get_psi(icarus_ctx *ctx, double *psi);

/* Copy the interior state into a DEVICE buffer U_dev [8][n3][n2][n1] (double, code units).
 * Synchronous. */
int icarus_copy_state(icarus_ctx *ctx, double *U_dev);

/* Cap dt so that the run stops exactly at t_stop (code units); t_stop <= 0 removes the cap. */
int icarus_set_stop_time(icarus_ctx *ctx, double t_stop);

/* Current time and the dt of the next step (code units). Synchronous. */
int icarus_time(icarus_ctx *ctx, double *t, double *dt);

/* Check of the square root and the reciprocal that the FP64 kernels use in place of the library's
 * correctly rounded ones (the fast-speed roots in the Riemann flux; the reciprocals of the face
 * densities, of the van Leer slope sums and of rho): single-precision estimates refined by two
 * Newton steps, within one ulp of the correctly rounded results. For the n host values x,
 * y[4i .. 4i + 3] receive that root of x[i], the library sqrt, that reciprocal and the library
 * 1 / x[i]. Synchronous; a temporary device buffer. EINVAL for n outside [1, 2^24] or NULL. */
int icarus_math_check(int n, const double *x, double *y);

/* Measured fused multiply-add rate of the current GPU (not part of the paper's method; the
 * denominator of the arithmetic roofline of the FP64 kernels, whose bound is the FP64 pipe):
 * blocks_per_sm x SMs blocks of 256 threads, each thread `chains` (1, 4, 8 or 16) independent
 * recurrences x <- x a + b in double (precision = ICARUS_FP64) or single (ICARUS_FP32) for `iters`
 * rounds (a multiple of 4). *tflops = 2 x threads x chains x iters / duration of the timed launch
 * (CUDA events, after one warm-up launch), *ms that duration. chains = 1 gives the dependent,
 * latency-bound rate. Synchronous; creates and destroys its own stream. */
int icarus_fma_rate(int precision, int chains, int blocks_per_sm, long long iters, double *tflops, double *ms);

/* Sticky status (0, ENONFINITE or, with options.strict_floors, EFLOOR) and the number of floor
 * activations. Synchronous. */
int icarus_status(icarus_ctx *ctx, long long *floor_hits);

/* Code-unit scales: s[0] = t0 s, s[1] = p0 Pa, s[2] = B0 T, s[3] = Omega in rad per t0,
 * s[4] = GM in code units. */
int icarus_scales(icarus_ctx *ctx, double *s);

/* Number of kernel launches one step makes (for launch accounting). */
int icarus_launches_per_step(icarus_ctx *ctx);

/* The cudaStream_t the context runs on (for events and ordering with other work). */
void *icarus_get_stream(icarus_ctx *ctx);

/* Measurement helper: run n_steps steps launching the kernels one by one (no graph) with CUDA
 * events around each launch on the context stream, and return the average duration in ms of one
 * launch of each kernel class: ms[ICARUS_KERNEL_CLASSES] = (ghost fill (3 kernels), flux r,
 * flux theta, flux phi, div B, update stage 1, update stage 2, probes, fused stage 1, fused
 * stage 2); a class the context does not launch reads 0 (the fused stage kernel replaces the
 * flux, div-B and update kernels of the FP32 and MIXED forms when options.fused = 1; with the
 * default kernel sequence of those forms the update classes time the update that forms the r-face
 * fluxes itself, and flux r reads 0). The
 * steps advance the solution like icarus_step. Synchronous. */
#define ICARUS_KERNEL_CLASSES 10
int icarus_time_kernels(icarus_ctx *ctx, int n_steps, double *ms);

/* ---- batched ensemble -------------------------------------------------------------------
 * Many independent solves (members) with their own grids, drivers, CMEs, probes, dt and t,
 * advanced together by one graph launch per ensemble step, in one of three forms
 * (icarus_batch_set_mode): the members' own step kernels as parallel graph branches (default);
 * ONE persistent, cooperatively launched kernel that runs every phase of every member's step,
 * with grid-wide barriers between phases (bounded waits: a barrier that does not complete within
 * about two seconds records ETIMEOUT and the kernel returns); or one launch per phase over all
 * members. Steps are replayed from a CUDA graph (the persistent form launches directly where the
 * driver does not allow capturing the cooperative launch). Each member is an icarus_ctx (icarus_batch_member)
 * on which icarus_set_boundary / icarus_sample / icarus_get_state / icarus_time work as usual;
 * stepping a member with icarus_step runs it alone. */
typedef struct icarus_batch icarus_batch;
#define ICARUS_BATCH_MAX_MEMBERS 1024

/* n_members (1..ICARUS_BATCH_MAX_MEMBERS) contexts with grids[n_members] and shared gamma,
 * omega_rot and options (precision included), all on one stream (opts->cuda_stream or a new one). */
int icarus_batch_init(int n_members, const icarus_grid *grids, double gamma, double omega_rot,
                      const icarus_options *opts, icarus_batch **out);

/* The member context m (owned by the batch; do not destroy it). */
int icarus_batch_member(icarus_batch *b, int m, icarus_ctx **ctx);

/* Pick the flux tile shapes by timed trials (reps launches per candidate) on the current states:
 * per member, once per distinct grid shape (cached), in the persistent mode; per direction for the
 * whole ensemble on the batched flux launches in the per-phase mode (set the mode first).
 * Synchronous. */
int icarus_batch_autotune(icarus_batch *b, int reps);

/* The chosen tile candidates of member m: cfg[0] radial (0: 128x2, 1: 64x4, 2: 32x8 threads),
 * cfg[1] theta / phi (0: 16x16, 1: 32x8). */
int icarus_batch_tiles(icarus_batch *b, int m, int *cfg);

/* How a batched step is launched. ICARUS_BATCH_PERSISTENT: ONE cooperative persistent kernel per
 * step, grid-wide barriers between the phases, flux tiles per member. ICARUS_BATCH_PHASES:
 * one launch per phase (ghost r / theta / phi, the fluxes of each direction, div B, update, twice;
 * per-member dt; probes: 18 launches per step whatever the number of members), each over the work
 * items of all members, so that every phase runs with its own register budget; one flux tile shape
 * per direction for the whole ensemble (icarus_batch_autotune times the candidates on the batched
 * launch). ICARUS_BATCH_CONCURRENT: every member's own step (the single solver's kernels, 17 per
 * member) captured into ONE graph per ensemble step as up to 16 parallel branches (members placed
 * on the least-loaded branch, largest first), so that members' kernels overlap on the GPU; the
 * default (on GB300 the fastest: each kernel keeps the single solver's register budget and reads
 * its parameters from the constant bank, while the GPU fills one member's tails with others). All
 * three replay a CUDA graph and give the same result up to the compiler's fused multiply-adds (the
 * same per-cell and per-face arithmetic). Changing the mode keeps the states. */
#define ICARUS_BATCH_PERSISTENT 0
#define ICARUS_BATCH_PHASES 1
#define ICARUS_BATCH_CONCURRENT 2
int icarus_batch_set_mode(icarus_batch *b, int mode);

/* Set the tile candidates of member m by hand (same codes as icarus_batch_tiles). */
int icarus_batch_set_tiles(icarus_batch *b, int m, int cfg_r, int cfg_t);

/* Advance every member by n steps, each member with its own dt. Asynchronous. */
int icarus_batch_step(icarus_batch *b, int n);

/* ETIMEOUT if a barrier wait gave up, else the first member's sticky status. Synchronous. */
int icarus_batch_status(icarus_batch *b);

/* Self-test of the batched form's bounded grid barrier: `blocks` small blocks (1..64) meet at one
 * barrier, block `absent` (-1: none) never arrives; the others wait at most spin_limit clock
 * ticks, then record the failure and return. ETIMEOUT when the wait gave up, OK when every block
 * arrived; the device stays usable either way. For tests of the failure path. */
int icarus_batch_barrier_selftest(int blocks, int absent, long long spin_limit);

/* info[4] = (members, blocks of the persistent launch, 1 if steps replay a CUDA graph, mode). */
int icarus_batch_info(icarus_batch *b, int *info);

/* The cudaStream_t of the batch. */
void *icarus_batch_stream(icarus_batch *b);

/* Release the batch and all member contexts. */
int icarus_batch_destroy(icarus_batch *b);

/* ---- learned closure ---------------------------------------------------------------------
 * A 4-layer 3-D convolutional network (8 -> 32 -> 32 -> 32 -> 8 channels, 3x3x3 kernels, ReLU,
 * phi circular / r and theta replicate padding) that predicts the correction of a coarse state
 * towards the restricted fine solution (not in the paper). BF16 weights and activations, FP32
 * accumulation on the 5th-generation tensor cores (tcgen05: forward, data and weight gradients),
 * FP32 Adam master weights; device memory from cudaMalloc, released by
 * icarus_closure_destroy. Every wait of the tcgen05 kernels is bounded: one that expires makes
 * the call return ETIMEOUT. */
typedef struct icarus_closure icarus_closure;

/* Network for a coarse grid n1 x n2 x n3, weights initialised from seed; runs on cuda_stream. */
int icarus_closure_create(int n1, int n2, int n3, unsigned long long seed, void *cuda_stream,
                          icarus_closure **out);
int icarus_closure_destroy(icarus_closure *c);

/* Self-test of the closure kernels' bounded barrier wait: one block waits on a shared-memory
 * barrier that expects one arrival, which it gives (arrive = 1: OK) or not (arrive = 0: the wait
 * gives up after `limit` polls and the call returns ETIMEOUT; the device stays usable). */
int icarus_closure_wait_selftest(int arrive, int limit);

/* Field-wise normalisation per radial index (host arrays [8][n1]): the input is (U - in_mean) /
 * in_scale, the network's output is multiplied by out_scale to give the correction dU. */
int icarus_closure_set_norm(icarus_closure *c, const double *in_mean, const double *in_scale,
                            const double *out_scale);

/* One Adam step (learning rate lr) on one pair: U_in and dU_target are DEVICE arrays
 * [8][n3][n2][n1] (code units); the loss is the mean squared error of the normalised correction.
 * *loss (host, may be NULL) receives the loss before the update; synchronous when loss != NULL. */
int icarus_closure_train_step(icarus_closure *c, const double *U_in, const double *dU_target, double lr,
                              double *loss);

/* Predicted correction dU_out (DEVICE [8][n3][n2][n1]) for a coarse state U_in (DEVICE). */
int icarus_closure_predict(icarus_closure *c, const double *U_in, double *dU_out);

/* Add the predicted correction to an FP64 coarse context's state in place (primitives, ghosts
 * and the next dt refreshed), on the context's stream. */
int icarus_closure_apply(icarus_closure *c, icarus_ctx *ctx);

/* Get (set = 0) or set (set = 1) the FP32 weights of one layer as host arrays w [O][27][C],
 * b [O] with the padded channel counts (C, O) = (16, 32), (32, 32), (32, 32), (32, 16). */
int icarus_closure_weights(icarus_closure *c, int layer, float *w, float *b, int set);

/* Volume-weighted 2x2x2 restriction of a fine context's state onto a coarse context whose grid is
 * half as fine in every direction (state, primitives, time and dt of the coarse context set). */
int icarus_restrict(icarus_ctx *fine, icarus_ctx *coarse);

/* One convolution layer on host FP32 arrays (channels last, x [n3][n2][n1][C], w [O][27][C],
 * b [O], g = dL/dy [n3][n2][n1][O]): y = act(conv(x) + b) and the gradients dx, dw, db, with
 * the tensor-core kernels of the closure (inputs rounded to BF16). (C, O, act) in {(16, 32, ReLU),
 * (32, 32, ReLU), (32, 16, linear)}. For checking the kernels against a reference. */
int icarus_conv3d_layer(int n1, int n2, int n3, int C, int O, int act, const float *x, const float *w,
                        const float *b, const float *g, float *y, float *dx, float *dw, float *db);

/* Largest grid (interior cells) icarus_cfl_dt_noalloc accepts: 16384 blocks of 256 cells. */
#define ICARUS_NOALLOC_MAX_CELLS 4194304LL

/* CFL time step of a caller-owned state without allocating anything. The paper has no
 * counterpart: this serves callers that cannot allocate device memory where they need a time
 * step (a framework's fixed pool, a real-time loop that forbids allocation after start-up, an
 * embedder that only owns its own buffers). It computes the same quantity as the dt that
 * icarus_set_state / icarus_time report: CFL / max over cells of sum_d (|v_d| + c_f,d) / dx_d.
 *   grid   : the grid (as for icarus_init, refined band included; a grid icarus_init rejects is
 *            rejected here with the same EINVAL message); at most ICARUS_NOALLOC_MAX_CELLS
 *            interior cells, otherwise EINVAL; nothing is launched after an EINVAL
 *   gamma  : adiabatic index; cfl: Courant number in (0, 1]
 *   U      : DEVICE pointer, interior conserved state [8][n3][n2][n1] doubles in code units
 *            (the layout of icarus_get_state)
 *   dt     : DEVICE pointer to one double that receives the time step (code units), or -1.0
 *            when any cell's signal speed is not finite (a NaN or inf in the state; there is no
 *            status word here, so the sentinel is the only signal)
 *   stream : cudaStream_t to run on (NULL: the legacy default stream); the call returns
 *            without synchronising
 * Scratch: the reduction's partial maxima and its completion counter live in one file-scope
 * __device__ array of (32 + 16384) doubles (128 KiB) that every GPU loading the library holds
 * until the process exits. The call never allocates or frees (no cudaMalloc / cudaFree, no
 * library allocator). The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress while that device is current; make that first call before any stream
 * capture. All calls on a device share the array and its counter (cleared at the start of every
 * call), so calls that overlap on the GPU (different streams, concurrently) race and must be
 * ordered by the caller. The array's first 256 bytes hold the counter and the non-finite flag; the
 * call's last block clears both again. */
int icarus_cfl_dt_noalloc(const icarus_grid *grid, double gamma, double cfl, const double *U, double *dt,
                          void *stream);

/* Message of the last failing call on this thread. */
const char *icarus_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
