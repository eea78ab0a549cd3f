/*
 * casimir.h -- C ABI of the GB300 time-domain Casimir-force library.
 *
 * The library computes Casimir forces by the time-domain stress-tensor method
 * of McCauley, Rodriguez, Joannopoulos and Johnson, "Casimir forces in the time
 * domain: Applications" (arXiv:0906.5170):
 *
 *   F_i = 2 Im int_0^inf dt g(-t) [Gamma^E_i(t) + Gamma^H_i(t)]            (Eq. (1))
 *
 * where Gamma is the stress-tensor surface functional of the field response to
 * a current J = delta(t) f_n on the stress surface S (Sec. II, Eqs. (3)-(6)),
 * summed over a cosine harmonic basis f_n on each face of S (Sec. III, Eq. (7)),
 * over source directions, polarisations and k-points (Sec. III B, III D), with
 * every simulation run in a medium of uniform conductivity sigma (Sec. II).
 * The prefactor 2 and the sign follow from the fluctuation-dissipation theorem
 * with the paper's transform convention g(-t) = (1/2pi) int_0^inf g(xi) e^{i xi t} dxi.
 *
 * Units: c = eps0 = mu0 = hbar = 1; lengths in units of the geometry's length
 * scale; the computational cell spans [0, n_a / resolution] along axis a.
 *
 * Conventions for every call:
 *   - return 0 (CASIMIR_OK) on success, CASIMIR_NOTREADY (> 0) for work still
 *     running, a negative CASIMIR_E* code on failure; nothing aborts the
 *     process; casimir_last_error() gives a message for the calling thread;
 *   - every pointer argument is a HOST pointer unless stated otherwise;
 *   - arrays passed in are copied before the call returns; the caller keeps
 *     ownership and may free them immediately;
 *   - objects returned through an out-pointer are owned by the caller and are
 *     released with the matching *_destroy call.
 */
#ifndef CASIMIR_H
#define CASIMIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define CASIMIR_OK         0
#define CASIMIR_NOTREADY   1   /* request admitted or queued, not finished yet */
#define CASIMIR_EINVAL    -1   /* malformed problem or argument */
#define CASIMIR_ENOMEM    -2   /* the plan alone exceeds the context's HBM budget, or allocation failed */
#define CASIMIR_ECUDA     -3   /* a CUDA call failed (message in casimir_last_error) */
#define CASIMIR_EBUSY     -4   /* request queue full */
#define CASIMIR_ETIMEOUT  -5   /* the device watchdog stopped the run (step or time limit) */
#define CASIMIR_ECANCELED -6   /* request cancelled */

/* ---- problem description (Sec. II and III) ---------------------------------- */
enum { CASIMIR_BC_PEC = 0, CASIMIR_BC_PML = 1, CASIMIR_BC_PERIODIC = 2 };
enum { CASIMIR_SHAPE_BOX = 0, CASIMIR_SHAPE_SPHERE = 1,
       CASIMIR_SHAPE_GRID = 2 };   /* a voxel mask over the box [lo, hi] (arbitrary geometry) */
enum { CASIMIR_MAT_PEC = 0,        /* eps = -inf (Sec. III A): tangential E vanishes */
       CASIMIR_MAT_PMC = 1,        /* mu = -inf (Sec. III A): tangential H vanishes */
       CASIMIR_MAT_DIELECTRIC = 2, /* constant eps, mu */
       CASIMIR_MAT_LORENTZ = 3 };  /* eps_inf + sum_j delta_eps_j w_j^2/(w_j^2 - w^2): undamped poles, one for
                                      the silicon model of Eq. (9), three for the silica model of
                                      Sec. III D; continued onto the contour (w^2 -> xi^2 + i sigma xi) */
#define CASIMIR_MAX_POLES 3
enum { CASIMIR_POL_TM = 1, CASIMIR_POL_TE = 2, CASIMIR_POL_TETM = 3, /* 2D, k_z = 0 */
       CASIMIR_POL_FULL = 4 };     /* all six source components (2D with k_z != 0, or 3D) */
enum { CASIMIR_G_PLAIN = 0,        /* Im g(-t) of Appendix A */
       CASIMIR_G_ZINV = 1 };       /* z-invariant PEC/vacuum kernel of Appendix A.2: a 2D (k_z = 0)
                                      TE+TM run gives the 3D force per unit length.  The kernel is
                                      g(xi) times the factor i*omega/2 stated in the text, i.e. half
                                      of the closed form printed there. */
enum { CASIMIR_FP32 = 0,           /* FP32 fields, FP64 projection and accumulation */
       CASIMIR_FP64 = 1 };         /* FP64 throughout */
enum { CASIMIR_BASIS_COSINE = 0,   /* per-face cosine series, Eq. (7) */
       CASIMIR_BASIS_POINT = 1 };  /* one source per surface pixel (Sec. II point-source method) */
enum { CASIMIR_COORDS_CARTESIAN = 0,
       CASIMIR_COORDS_CYLINDRICAL = 1 };  /* (r, z) cross-section of a rotationally symmetric
                                             geometry with fields ~ exp(i m phi) (Sec. III C and
                                             the appendix on cylindrical coordinates): axis 0 is r
                                             (the symmetry axis at r = 0, a PEC wall at r = n[0]
                                             Delta), axis 1 is z; the force is along z and sums
                                             the m sectors through the k-point weights (1 for
                                             m = 0, 2 for m > 0: the +m and -m terms). */

/* One geometric object; later objects override earlier ones where they overlap.
 * Membership is closed (boundary points belong to the object).
 *
 * CASIMIR_SHAPE_GRID: `mask` holds mask_n[0] x mask_n[1] x mask_n[2] bytes, x fastest
 * (index (k * mask_n[1] + j) * mask_n[0] + i); voxel (i, j, k) spans the box [lo, hi] cut
 * into mask_n[a] equal slabs along each axis a, and the object is the union of the closed
 * voxels whose byte is non-zero (so a mask of voxels aligned with a box reproduces that box).
 * Two-dimensional problems need mask_n[2] == 1 and ignore lo[2], hi[2].  Every used axis
 * needs hi[a] > lo[a] and mask_n[a] >= 1 (CASIMIR_EINVAL otherwise).  The planner copies
 * the mask; the caller may free it once casimir_plan returns.  Several materials: one
 * object per material, each with its own mask. */
typedef struct {
    int shape;           /* CASIMIR_SHAPE_* */
    int kind;            /* CASIMIR_MAT_* */
    double lo[3], hi[3]; /* box corners */
    double center[3];    /* sphere centre */
    double radius;       /* sphere radius */
    double eps, mu;      /* dielectric */
    double eps_inf;      /* Lorentz: eps at high frequency */
    double delta_eps[CASIMIR_MAX_POLES];  /* Lorentz pole strengths (>= 0; 0: the pole is absent) */
    double omega0[CASIMIR_MAX_POLES];     /* Lorentz pole frequencies (> 0 where delta_eps > 0); every
                                             pole needs omega0 dt < 2, and the medium eps(4/dt^2) above
                                             the lattice's (dt/2)^2 k_max^2 (CASIMIR_EINVAL otherwise) */
    const uint8_t *mask; /* CASIMIR_SHAPE_GRID: the voxel mask (NULL for other shapes) */
    int mask_n[3];       /* CASIMIR_SHAPE_GRID: voxels per axis */
    int reserved;
} casimir_object;

/* One axis-aligned face of the stress surface S: normal along `axis`, outward
 * sign `sign` (+1/-1), at coordinate `pos`; extent [lo[b], hi[b]] along each
 * tangential axis b (entries along `axis` are ignored).  Each tangential extent
 * must be an integer number of cells. */
typedef struct {
    int axis, sign;
    double pos;
    double lo[3], hi[3];
} casimir_face;

/* A k-point (Bloch k_x, k_y; or k_z for a 2D cross-section) and its weight in
 * the force sum (quadrature weight times the measure, e.g. 1/pi for k_z).  In
 * cylindrical coordinates k must be zero and m is the azimuthal order. */
typedef struct {
    double k[3];
    double weight;
    int m;               /* cylindrical coordinates: fields ~ exp(i m phi) */
    int reserved;
} casimir_kpoint;

typedef struct {
    int dims;            /* 2 or 3 */
    int n[3];            /* cells; n[2] == 1 when dims == 2 */
    double resolution;   /* cells per unit length: Delta = 1/resolution */
    double courant;      /* Delta_t = courant * Delta */
    int n_steps;         /* T, samples t_n = n Delta_t, n = 1..T */
    double sigma;        /* contour conductivity (Sec. II), >= 0 */
    double bg_eps, bg_mu;
    int n_objects;
    const casimir_object *objects;
    int bc[3];           /* CASIMIR_BC_* per axis; PEC and PML axes are closed by a PEC wall at 0 == L */
    int pml_cells[3];    /* CPML thickness per PML axis */
    int n_faces;
    const casimir_face *faces;
    int n_harm;          /* cosine harmonics per tangential axis and face (capped at the pixel count) */
    int polarization;    /* CASIMIR_POL_* */
    int n_kpoints;
    const casimir_kpoint *kpoints;
    int force_axis;      /* 0, 1 or 2 */
    int g_variant;       /* CASIMIR_G_* */
    int precision;       /* CASIMIR_FP32 / CASIMIR_FP64 */
    int basis;           /* CASIMIR_BASIS_* */
    int coords;          /* CASIMIR_COORDS_*.  Cylindrical problems: dims 2, polarization FULL,
                            bc[0] PEC (the wall at r = R), no PML, no Lorentz media, k = 0 and
                            courant < 2 / sqrt(max(9, 8 + 4 m^2)) for every k-point (the i m / r
                            terms next to the axis bound the time step); else CASIMIR_EINVAL. */
} casimir_problem;

/* ---- opaque handles ----------------------------------------------------------- */
typedef struct casimir_ctx casimir_ctx_t;
typedef struct casimir_plan casimir_plan_t;
typedef struct casimir_request *casimir_ticket;

typedef struct {
    int64_t n_sims;            /* source simulations in the plan (after exact pruning) */
    int64_t n_cells;           /* sum of grid cells over the sims */
    int64_t cell_updates;      /* n_cells * n_steps */
    int64_t device_bytes;      /* device memory the plan needs while running */
    int64_t bytes_per_update;  /* algorithmic bytes per cell-update of the dominant kernel */
    int64_t upload_bytes;      /* host-to-device bytes copied when the plan is first admitted */
    int64_t bytes_per_step;    /* algorithmic bytes of one time step over all simulations: every
                                  stored field, CPML auxiliary and Lorentz (P, P_prev per present
                                  pole) value read and written once, plus the material ids */
    int64_t launches;          /* launch indices one request of the plan takes: ceil(n_steps / k)
                                  for the k time steps its kernels fuse into one launch (2D TM/TE
                                  runs k = steps_per_launch; cylindrical runs and FP32 Cartesian
                                  six-component runs with at most one Lorentz pole per material
                                  k = 2 when steps_per_launch >= 2; other runs k = 1) */
} casimir_plan_info;

typedef struct {
    double queue_ms;           /* submit -> admission */
    double device_ms;          /* admission -> device completion */
    double total_ms;           /* submit -> result available */
    int64_t cell_updates;
    int64_t kernel_launches;   /* kernels of this library launched for the request */
} casimir_stats;

/* ---- context ----------------------------------------------------------------- */
/* Create a context on CUDA device `device`; plans are admitted while the device
 * memory they need fits in `hbm_budget_bytes` (0: 90% of free memory).  The
 * context owns its device memory, its streams and the request executor. */
int casimir_ctx_create(int device, uint64_t hbm_budget_bytes, casimir_ctx_t **out);
void casimir_ctx_destroy(casimir_ctx_t *ctx);

/* Run all device work of this context on `stream` (a cudaStream_t, or NULL for
 * the context's own stream).  Lets a caller bracket the work with its own events. */
int casimir_ctx_set_stream(casimir_ctx_t *ctx, void *cuda_stream);

/* Route the context's device allocations through caller callbacks (e.g. a
 * framework's caching allocator).  alloc returns a device pointer or NULL. */
typedef void *(*casimir_alloc_fn)(size_t bytes, void *user);
typedef void (*casimir_free_fn)(void *ptr, void *user);
int casimir_ctx_set_allocator(casimir_ctx_t *ctx, casimir_alloc_fn alloc, casimir_free_fn free_, void *user);

/* Watchdog: a request stops with CASIMIR_ETIMEOUT once it has been running for
 * `max_ms` milliseconds (0: no limit).  Checked between chunks of time steps, so
 * no device code ever waits on it. */
int casimir_ctx_set_watchdog(casimir_ctx_t *ctx, double max_ms);

/* Run simulations in waves whose field memory totals at most `bytes` (0, the
 * default: all simulations of an admitted request at once; the environment
 * variable CASIMIR_WAVE_BYTES sets the initial value).  Waves bound the number
 * of simulations in flight, e.g. to keep their fields in the L2 cache.  Applies
 * to requests admitted after the call. */
int casimir_ctx_set_wave_bytes(casimir_ctx_t *ctx, int64_t bytes);

/* Device time of the batched time-step kernels since the last reset, measured
 * with CUDA events on the context's stream: total milliseconds, number of step
 * launches and cell-updates performed.  reset != 0 zeroes the counters. */
int casimir_ctx_kernel_stats(casimir_ctx_t *ctx, double *step_ms, int64_t *launches,
                             int64_t *cell_updates, int reset);

/* ---- plan: host-side set-up of one force computation (Sec. III) -------------- */
/* Rasterise the geometry onto the Yee grid, build the face pixels, harmonic
 * basis, interpolation stencils, g(-t) weights and the simulation list.  The
 * problem's arrays are copied.  ctx == NULL builds a host-only plan that can be
 * inspected but not run (no device needed).  Errors: CASIMIR_EINVAL (malformed
 * problem), CASIMIR_ENOMEM (the plan alone needs more device memory than the budget). */
int casimir_plan(casimir_ctx_t *ctx, const casimir_problem *problem, casimir_plan_t **out);
int casimir_plan_get_info(const casimir_plan_t *plan, casimir_plan_info *info);

/* Introspection of the rasterised geometry (step a0 of the method, Sec. III): for k-point
 * `kpoint` and the field array storing component `comp` (0..2) of E (field 0) or H
 * (field 1), out[(k * n[1] + j) * n[0] + i] receives the coefficient at that array's
 * site of cell (i, j, k): 1/eps (E; 1/eps_inf in a Lorentz medium) or 1/mu (H), and 0
 * where the site is masked (E on PEC, on a closed wall or, in cylindrical runs, on the
 * axis where the component vanishes; H on PMC or the axis).  off[3] receives the site's
 * position within the cell in units of Delta ((i + off[0]) Delta, ...); the TE family of
 * two-dimensional runs lives on the lattice shifted by half a cell, so its offsets differ
 * from the standard Yee ones.  `out` holds n[0] n[1] n[2] doubles; works on host-only
 * plans.  CASIMIR_EINVAL if the plan's polarisation has no such array or kpoint is out of
 * range. */
int casimir_plan_site_coefs(const casimir_plan_t *plan, int kpoint, int field, int comp,
                            double off[3], double *out);

/* Introspection of the rasterised Lorentz media (Eq. (9), the silica model of Sec. III D):
 * for k-point `kpoint`, E component `comp` and pole slot `pole` (0 .. CASIMIR_MAX_POLES - 1),
 * de[cell] and w0[cell] receive that slot's strength and frequency at the component's site of
 * every cell (same indexing as casimir_plan_site_coefs).  The poles present at a site fill
 * the first slots; empty slots and masked sites (PEC, closed walls) hold 0.  Six-component
 * plans only (CASIMIR_EINVAL otherwise, or for an index out of range). */
int casimir_plan_site_poles(const casimir_plan_t *plan, int kpoint, int comp, int pole,
                            double *de, double *w0);

/* Introspection of the CPML coefficients (Sec. III B; polynomial grading of order 3,
 * reflection 1e-8, kappa = 1, frequency shift falling linearly from 0.05 to 0 at the wall):
 * for PML axis `axis` and sites on integer (half = 0) or half-integer (half = 1) positions
 * along it, b[i], c[i] and inv_kappa[i] for i < n[axis], in the update psi <- b psi + c dF
 * and the stretched derivative inv_kappa dF + psi.  CASIMIR_EINVAL if the axis is not a PML
 * axis of the plan. */
int casimir_plan_pml(const casimir_plan_t *plan, int axis, int half, double *b, double *c,
                     double *inv_kappa);

/* Execution options of a plan (how the leapfrog of Sec. III A is scheduled; the computed
 * force does not depend on them beyond rounding).  0 in a field selects the default. */
typedef struct {
    int steps_per_launch;   /* time steps fused into one pass over memory: 2D TM/TE runs 1, 2 or 3
                               (default 3 for FP32 runs, 2 for FP64 runs); cylindrical runs 1 or 2
                               (any value >= 2 fuses two; the default fuses two); other 2D
                               six-component runs in FP32 whose materials have at most one
                               Lorentz pole 1 or 2 (any value >= 2 fuses two; the default fuses
                               two); all other six-component runs take one step per launch */
    int march_rows;         /* 2D six-component and cylindrical runs: rows per strip tile, 16, 32 or 64 (default 32) */
    int kernel_3d;          /* 3D runs: 3 = column march, both half steps per pass (the default without
                               CPML); 1 = x-line kernel, one half step per pass (the default with
                               CPML); 2 = one-thread-per-cell kernel */
    int reserved;
} casimir_plan_options;

/* casimir_plan with explicit options (NULL: defaults).  CASIMIR_EINVAL for values out of range. */
int casimir_plan_ex(casimir_ctx_t *ctx, const casimir_problem *problem, const casimir_plan_options *opts,
                    casimir_plan_t **out);
/* The options a plan was prepared with (after defaults and autotuning). */
int casimir_plan_get_options(const casimir_plan_t *plan, casimir_plan_options *opts);

/* Autotuning (on != 0): casimir_plan then picks the options itself.  For the first problem of
 * each class (dimension, polarisation family, precision, coordinates, CPML and Lorentz media,
 * complex fields, grid size to a factor of two) it runs every candidate option set on a copy of
 * the problem cut to 128 steps, times the step kernels with CUDA events and keeps the fastest;
 * later problems of the class reuse the choice.  Trials run only while the context is idle
 * (otherwise the defaults apply and nothing is cached).  Off by default. */
int casimir_ctx_set_autotune(casimir_ctx_t *ctx, int on);
/* Release a plan; blocks until the plan's queued or running requests have finished. */
void casimir_plan_destroy(casimir_plan_t *plan);

/* ---- requests ------------------------------------------------------------------ */
/* Queue one force computation of `plan` (non-blocking).  The plan must stay
 * alive until the request has finished.  CASIMIR_EBUSY when the queue is full. */
int casimir_submit(casimir_plan_t *plan, uint64_t user_tag, casimir_ticket *out);

/* Wait up to `wait_ms` (0: poll, < 0: forever) for the result.  On success F[3]
 * holds the force (only F[force_axis] is non-zero), *err_est (may be NULL) an
 * estimate of the truncation error of the time integral, *st (may be NULL)
 * timings.  Returns CASIMIR_NOTREADY while running; CASIMIR_ETIMEOUT or
 * CASIMIR_ECANCELED for a request the watchdog stopped or the caller cancelled; for
 * a request that failed on the device, the failing call's code (CASIMIR_ECUDA,
 * CASIMIR_ENOMEM), with that call's message in casimir_last_error() of the calling
 * thread.  After a return other than CASIMIR_NOTREADY the ticket is released. */
int casimir_force(casimir_ticket ticket, int wait_ms, double F[3], double *err_est, casimir_stats *st);

/* Cancel a queued or running request (its ticket is still released by casimir_force). */
int casimir_cancel(casimir_ticket ticket);

/* Run one request of `plan` to completion on the context's stream, synchronously:
 * F[3] as above; per_sim (may be NULL, else n_sims doubles) receives every
 * simulation's FP64 contribution in plan order. */
int casimir_run(casimir_plan_t *plan, double F[3], double *per_sim, casimir_stats *st);

/* The same computation without batching, as a point of comparison for the
 * batched executor: one run at a time (the simulations of one k-point, harmonic
 * and polarisation family), each time step issuing that run's field-update
 * launches and a separate projection launch, and no CUDA graph.  Arguments and
 * results as for casimir_run. */
int casimir_run_plain(casimir_plan_t *plan, double F[3], double *per_sim, casimir_stats *st);

/* Per-simulation description in plan order (for per-simulation parity):
 * desc[6*s + 0..5] = k-point, face, harmonic n1, harmonic n2, source kind (0 J, 1 K),
 * source component. */
int casimir_plan_sims(const casimir_plan_t *plan, int32_t *desc, int64_t n);

/* Introspection of simulation `sim` (plan order) of a plan, steps a2 and a8 of the method
 * (Sec. II, Eqs. (3)-(6); Sec. III A): which = 0 gives its source, the stored field values
 * right after the impulse (E = D/eps or H = B/mu at each site, masked sites dropped to 0);
 * which = 1 its measurement functional, s(n) = sum_e weight_e * field_e (the stress-tensor
 * projection of the harmonic f_n with dA and eps_S or mu_S).  Entry e: comp[e] = 3 * field +
 * component (field 0 E, 1 H), idx[e] = the site's cell index (k * n[1] + j) * n[0] + i on
 * that array's lattice (casimir_plan_site_coefs gives the offsets), val[2e], val[2e + 1] =
 * real and imaginary part, with the sign of the stored array (the TE family stores -E).
 * Returns the number of entries (writes at most cap of them; cap 0 only counts), or
 * CASIMIR_EINVAL for a bad simulation index, `which` or buffer.  Works on host-only plans. */
int64_t casimir_plan_sim_entries(const casimir_plan_t *plan, int64_t sim, int which, int32_t *comp,
                                 int64_t *idx, double *val, int64_t cap);

/* The time weights w_n = 2 Delta_t Im g(-n Delta_t), n = 1..n_steps, of Eq. (1)
 * (rectangle rule); w must hold n_steps doubles. */
int casimir_plan_weights(const casimir_plan_t *plan, double *w, int64_t n);

/* Allocation-free run of a plan (no counterpart in the paper; an entry point for
 * embedding the library).  Some callers cannot let a library allocate device memory:
 * a host that has already handed nearly all of the GPU's memory to its own pool, so
 * that a cudaMalloc would fail or fragment that pool; an embedder whose memory
 * manager must not be re-entered from inside one of its own callbacks; and
 * latency-bound loops that cannot absorb the device-wide synchronisation that
 * cudaFree implies.  This call performs no cudaMalloc, cudaFree or other allocating
 * routine: every intermediate (fields, simulation and tile tables, the plan's copied
 * tables, the launch counter) lives in one static device array of 64 MiB per device,
 * which every GPU that loads the library holds until the process exits.
 *   plan       any plan of two-dimensional (TM/TE) simulations, including a
 *              host-only plan built with ctx == NULL;
 *   d_per_sim  DEVICE pointer to n_sims doubles; receives every simulation's
 *              contribution sum_n w_n s(n) in plan order, before the k-point
 *              weight (all work is queued on `cuda_stream`; synchronise it
 *              before reading);
 *   cuda_stream a cudaStream_t, or NULL for the default stream.
 * The first call on a device does the set-up: with that device current it looks up
 * the array's device address (and, under lazy module loading, its first launches
 * load the kernels); make that first call, and let it complete, before any stream
 * capture begins.  Every call reuses the same array, which keeps the previous
 * call's contents (the call clears what must start at zero); calls whose work
 * overlaps on the GPU race on the array and must be serialised by the caller.
 * The tables reach the device through ordinary asynchronous copies from host
 * memory owned by the call.  Returns CASIMIR_ENOMEM, with the required size in
 * casimir_last_error(), when the plan does not fit in the array, and
 * CASIMIR_EINVAL for non-2D plans. */
int casimir_run_noalloc(const casimir_plan_t *plan, double *d_per_sim, void *cuda_stream);

/* Thread-local message describing the last error of the calling thread. */
const char *casimir_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CASIMIR_H */
