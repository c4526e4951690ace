/*
 * ugks.h -- C ABI of the GB300 unified gas-kinetic scheme (UGKS) library.
 *
 * One explicit UGKS time step on an unstructured physical mesh times a
 * discrete velocity space, as defined in Zhang, Wei, Long, Xu, "An efficiency
 * and memory-saving programming paradigm for the unified gas-kinetic scheme"
 * (arXiv:2412.06546): BGK-Shakhov model with reduced distributions h, b
 * (Sec. 2.1-2.2), finite-volume update of f and W (Sec. 2.3, Eq.
 * microscopicFlux, macroscopicUpdata, macroscopicFlux), the time-integrated
 * interface solution (Sec. 2.4, Eq. fullSolution), ghost far field and Maxwell
 * isothermal walls (Sec. 2.5, Eq. maxWalldes), the trapezoid source term
 * (Sec. 2.6) and the two-stage update of Algorithm 1 (Sec. 3.2, Eq. microS1,
 * microS2).  Every step of the path runs in the library's CUDA kernels.
 *
 * Units: gas constant R = 1, reference density and temperature 1, velocities
 * in sqrt(R T_ref).  Monatomic gas (argon, K = 0 internal degrees of freedom):
 * 2D cases store h and b per velocity, 3D cases store h only (b = 0).
 *
 * Conventions for every entry point:
 *  - Every call returns a ugks_status; no exception or abort crosses the ABI.
 *    On failure ugks_last_error() returns a thread-local message.
 *  - Input arrays are host pointers, copied by the call; the caller keeps
 *    ownership.  Output arrays are caller-owned host buffers unless the name
 *    says "device".
 *  - A case handle is used from one host thread at a time.
 *  - Device memory comes from the ugks_alloc callbacks (NULL: cudaMalloc /
 *    cudaFree) and work is issued on the stream given at creation.
 */
#ifndef UGKS_H
#define UGKS_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    UGKS_OK = 0,
    UGKS_EINVAL = 1,        /* invalid argument (message says which) */
    UGKS_ENOMEM = 2,        /* device or host allocation failed */
    UGKS_ECUDA = 3,         /* a CUDA runtime call failed */
    UGKS_ENUMERIC = 4,      /* non-finite or non-positive density/temperature */
    UGKS_ENOTCONVERGED = 5, /* a served case hit its step limit */
    UGKS_EBUSY = 6,         /* server cannot admit the request now */
    UGKS_ETIMEOUT = 7,      /* bounded wait ran out */
    UGKS_ENOTFOUND = 8      /* unknown ticket */
} ugks_status;

/* face types (Sec. 2.5; PERIODIC is an addition for closed test domains) */
enum { UGKS_FACE_INTERIOR = 0, UGKS_FACE_WALL = 1, UGKS_FACE_FARFIELD = 2, UGKS_FACE_PERIODIC = 3 };

/* precision of the stored distribution and the per-velocity arithmetic.
 * UGKS_FP64: everything in FP64 (the plain method).
 * UGKS_FP32: f stored and streamed in FP32, per-velocity products in FP32,
 * and every velocity-moment sum accumulated in FP64: the face sums (interface
 * W0, the moments of g0) from FP32 partials of at most 16 terms per GPU lane
 * (512 per warp), the wall density and the heat flux from Kahan-compensated
 * FP32 lane sums, the moments of the flux residual that update W from
 * double-float (about 44-bit) lane and warp sums; W, the equilibrium
 * parameters (rho, U, lambda), the heat flux and the collision coefficients
 * dt/(2 tau) and 1/(1 + dt/(2 tau)) are formed in FP64. */
enum { UGKS_FP64 = 0, UGKS_FP32 = 1 };

/* Unstructured physical mesh (Sec. 2.3): cells Omega_i and faces S_ij. */
typedef struct {
    int32_t dim;              /* 2 or 3 */
    int64_t n_cells, n_faces;
    const double *cell_xc;    /* [n_cells][dim] centroids */
    const double *cell_vol;   /* [n_cells] |Omega_i| > 0 */
    const int64_t *face_cells;/* [n_faces][2] owner, neighbour; -1 on wall / far field */
    const double *face_n;     /* [n_faces][dim] unit normal, owner -> neighbour (outward at boundaries) */
    const double *face_S;     /* [n_faces] face area S_ij > 0 */
    const double *face_xc;    /* [n_faces][dim] face centre, as seen from the owner */
    const int32_t *face_type; /* [n_faces] UGKS_FACE_* */
    const int32_t *face_tag;  /* [n_faces] wall index (0 <= tag < n_walls) for WALL faces */
    const double *face_shift; /* [n_faces][dim] or NULL: PERIODIC faces, vector added to the
                                 neighbour centroid to bring its image next to the owner */
} ugks_mesh;

/* Discrete velocity space (Sec. 2.3): int Q du = sum_k Q_k V_k */
typedef struct {
    int32_t dim;
    int64_t nv;
    const double *u;          /* [nv][dim] velocities u_k */
    const double *w;          /* [nv] cell volumes V_k (quadrature weights) */
    int32_t cart_n[3];        /* > 0 for a tensor grid (informational) */
} ugks_vgrid;

/* Gas, boundary and numerical parameters */
typedef struct {
    double Kn;        /* Knudsen number (mean free path / L_ref); +inf: collisionless */
    double L_ref;     /* reference length of Kn (e.g. the cylinder diameter) */
    double Pr;        /* Prandtl number of the Shakhov model (1: BGK) */
    double omega;     /* viscosity exponent, mu = mu_ref T^omega */
    double cfl;       /* dt = cfl * min_i h_i / max_k |u_k| unless dt > 0 */
    double dt;        /* fixed time step if > 0 */
    int32_t limiter;  /* 1: Venkatakrishnan limiter on micro and macro slopes */
    double venkat_K;  /* limiter constant K, eps^2 = (K h_i)^3 */
    int32_t n_walls;
    const double *wall_T;   /* [n_walls] wall temperature */
    const double *wall_U;   /* [n_walls][3] wall velocity */
    double inf_rho, inf_U[3], inf_T; /* far-field state */
    int32_t precision;      /* UGKS_FP64 or UGKS_FP32 */
    const double *prim_init;/* [n_cells][dim+2] initial (rho, U, T), or NULL: far-field state */
    int32_t patch_cells;    /* gather tiling: cells per patch (0: autotuned by timing the gather
                               kernel on this case, cached per case shape) */
    int32_t vtile;          /* gather tiling: velocities per tile, 32, 64 or 128 (0: automatic) */
    int32_t gather_threads; /* gather tiling: threads per CTA, 256 or 512 (512 only for UGKS_FP32 with
                               vtile <= 64; 0: automatic, 256 unless the autotuner picks 512) */
    int32_t gather_tile_group; /* gather grid order: the grid sweeps the patches once per group of this
                               many velocity tiles, the tiles of a patch adjacent, so that a patch's
                               face data are read once per group (1 .. 1024, larger values are
                               clamped to the number of tiles; 0: chosen by the autotuner when
                               patch_cells is 0, else 1) */
    int32_t w0_analytic;    /* interface equilibrium W0 (Sec. 2.4) from: 0 the discrete half-range
                               sums over the velocity set (default), 1 the analytic half-range
                               moments of the face-state Maxwellians over the continuous velocity
                               space (erfc); the slopes of g0 use the discrete moments either way */
} ugks_params;

/* Device allocator.  alloc returns a device pointer of at least `bytes`
 * (256-byte aligned) usable on `stream`, or NULL; free releases it.  Blocks
 * are freed by ugks_destroy and by ugks_create when the autotuner replaces a
 * tiling's patch arrays, in both cases after the case stream has finished the
 * work that reads them. */
typedef struct {
    void *ctx;
    void *(*alloc)(void *ctx, size_t bytes, void *stream);
    void (*free)(void *ctx, void *ptr, size_t bytes, void *stream);
} ugks_alloc;

typedef struct ugks_case ugks_case;

typedef struct {
    int32_t dim, ncomp, precision;
    int64_t n_cells, n_faces, nv, nv_pad;
    double dt;
    int64_t step;              /* steps taken so far */
    size_t device_bytes;       /* device memory held by the case */
    size_t f_bytes;            /* bytes of one copy of f */
    int32_t n_patches, patch_cells, vtile;  /* gather tiling in use */
    int64_t kernel_launches_per_step;
    int64_t n_wall_faces;               /* faces of type UGKS_FACE_WALL */
    int32_t gather_threads;             /* threads per CTA of the gather pass in use */
    int32_t gather_tile_group;          /* velocity tiles per group of the gather grid in use */
} ugks_info_t;

/* Create a case: validates and copies the inputs, orders cells for locality,
 * builds least-squares coefficients and gather patches, allocates device state
 * and initialises f^0 = Maxwellian(W^0) (Sec. 3.1).  `stream` is a cudaStream_t
 * (NULL: the legacy default stream).  On success *out owns the device memory. */
ugks_status ugks_create(const ugks_mesh *mesh, const ugks_vgrid *vgrid, const ugks_params *params,
                        const ugks_alloc *alloc, void *stream, ugks_case **out);

/* Advance `nsteps` time steps (Algorithm 1 each).  Asynchronous on the case
 * stream; errors of the launches are reported, numeric checks are not (see
 * ugks_check). */
ugks_status ugks_step(ugks_case *c, int32_t nsteps);

/* Wait for the case stream and report UGKS_ENUMERIC if the state holds a
 * non-finite value or a non-positive density or temperature. */
ugks_status ugks_check(ugks_case *c);

/* Smallest and largest density of the current state over the own cells (all
 * cells unless ugks_set_owned limited them): range[0] = min rho, range[1] =
 * max rho (host buffer of 2 doubles); a non-positive or non-finite density
 * counts as 0, and both are 0 for a case without own cells.  The ratio
 * range[0] / range[1] bounds where the FP32-storage form holds its accuracy:
 * the flux terms of a cell far thinner than its surroundings are of the
 * surrounding gas's size, and the FP32 rounding of the stored f there is an
 * absolute error of about 6e-8 times that size.  On an impulsive Mach-5
 * cylinder start (a near-vacuum wake) the temperature error of the thinnest
 * cell stayed below 5e-9 / ratio down to ratios of 5e-9, and the state was
 * lost at 1.5e-9: a ratio of at least 5e-6 keeps that error below 1e-3, of
 * 5e-5 below 1e-4.  A case below its bound moves to FP64 storage through
 * ugks_get_state / ugks_set_state (exact).
 * Synchronises the case stream. */
ugks_status ugks_density_range(ugks_case *c, double *range);

/* Macroscopic fields of the current state into host buffers (any may be NULL):
 * rho[C], U[C][dim], T[C], q[C][dim] (heat flux of f, Sec. 2.1).  Cell order is
 * the caller's mesh order.  Synchronises the case stream. */
ugks_status ugks_moments(ugks_case *c, double *rho, double *U, double *T, double *q);

/* Residual of the last step, res[m] = |W^{n+1}_m - W^n_m|_2 / |W^n_m|_2, m < dim+2. */
ugks_status ugks_residual(ugks_case *c, double *res);

/* Copy the state to host buffers: f[C][ncomp][nv] (FP64, caller cell order) and
 * W[C][dim+2] (conserved variables); either may be NULL.  Synchronises. */
ugks_status ugks_get_state(ugks_case *c, double *f, double *W);

/* Surface quantities of the last step at every wall face (Sec. 2.5), in the
 * caller's face order: face[i] is the face id; with F_w the macroscopic wall
 * flux of Eq. macroscopicFlux over the step, F_mw its momentum part and n_w
 * the face normal (out of the fluid cell, into the wall), p[i] = F_mw . n_w,
 * sigma[i] = |F_mw - p[i] n_w| and q[i] = F_w4 (energy), each divided by dt
 * (the time average over the step).  The arrays hold n_wall_faces entries
 * (ugks_info); any may be NULL.  Zero before the first step.  Synchronises.
 * Pressure, shear and heat flux coefficients follow by dividing by
 * rho_inf U_inf^2 / 2 (p, sigma) and rho_inf U_inf^3 / 2 (q). */
ugks_status ugks_wall_quantities(ugks_case *c, int64_t *face, double *p, double *sigma, double *q);

/* The state of selected cells only: for i < n, f[i][ncomp][nv] (FP64) and
 * W[i][dim+2] of caller cell cells[i] (either output may be NULL; ids may
 * repeat).  Serves sampled checks of cases whose whole distribution would not
 * fit host memory.  n <= n_cells.  UGKS_EINVAL for NULL cells, n out of range
 * or an id outside [0, n_cells).  Uses the case's per-step scratch as staging
 * (between steps only); synchronises. */
ugks_status ugks_get_cells(ugks_case *c, const int64_t *cells, int64_t n, double *f, double *W);

/* Replace the state from host buffers (same layout); either may be NULL.
 * The heat flux is recomputed from the new f.  The call returns once the
 * copies and kernels are queued: f is copied in chunks on a stream of the case
 * that overlaps the reordering of earlier chunks on the case stream, and the
 * case stream waits for every chunk.  Page-locked host buffers must stay
 * unchanged until the case stream has passed the upload (any synchronising
 * call, e.g. ugks_moments or ugks_check); pageable ones are read before the
 * call returns. */
ugks_status ugks_set_state(ugks_case *c, const double *f, const double *W);

/* ugks_get_state and ugks_set_state with f in single precision:
 * f[C][ncomp][nv] FP32 in caller cell order, W still FP64.  For a UGKS_FP32
 * case they move the stored values exactly with half the bytes of the FP64
 * calls; for a UGKS_FP64 case f is rounded to nearest on the way out and
 * widened exactly on the way in.  Same synchronisation as the FP64 calls. */
ugks_status ugks_get_state_f32(ugks_case *c, float *f, double *W);
ugks_status ugks_set_state_f32(ugks_case *c, const float *f, const double *W);

/* Kernel-group timing.  After ugks_profile_begin(c, max_steps) the next
 * max_steps calls of ugks_step record CUDA events on the case stream around
 * each kernel group (no host synchronisation); ugks_profile_end synchronises
 * and writes the summed milliseconds per group into ms[0..n-1] (groups in
 * launch order: 0 cell prep + macro slopes, 1 face equilibrium pass,
 * 2 wall density pass, 3 gather pass (slopes, fluxes, stage 1), 4 W update,
 * 5 collision (stage 2) + heat flux) and the number of profiled steps into
 * *steps.  Not part of the method; used by the benchmark. */
ugks_status ugks_profile_begin(ugks_case *c, int32_t max_steps);
ugks_status ugks_profile_end(ugks_case *c, double *ms, int32_t n, int32_t *steps);

/* Batched stepping of several cases (one GPU).  The cases must share the
 * dimension and precision.  Each batch step runs every case's gather pass in
 * one persistent kernel per (velocity-tile width, block size) present in the
 * batch, which walks a (case, patch, velocity tile) work list, and each of the
 * step's other kernels once for all cases (block offsets per case), so a
 * step is about a dozen launches whatever the number of cases.  The whole
 * step is captured once as a CUDA graph on `stream` (cudaStream_t, NULL: a
 * stream of the batch's own) and replayed.  Results are bit-identical to
 * stepping each case alone with ugks_step.  The cases stay owned by the
 * caller and must outlive the batch; ugks_batch_step advances each case's
 * step counter. */
typedef struct ugks_batch ugks_batch;
ugks_status ugks_batch_create(ugks_case *const *cases, int32_t n, void *stream, ugks_batch **out);
ugks_status ugks_batch_step(ugks_batch *b, int32_t nsteps);
void ugks_batch_destroy(ugks_batch *b);

/* ---- Serving loop (continuous batching of independent cases) ----
 * Requests arrive (at a time on the server clock); every ugks_server_tick
 * admits arrived requests, first fit in arrival order, while a slot is free
 * and the request's estimated device footprint (two copies of f plus the
 * O(cells + faces) arrays) fits the remaining budget; steps every running case
 * steps_per_tick times in batches (ugks_batch: one launch per kernel of the step
 * for all cases, CUDA-graph replay); then reads each running case's residual and retires
 * the converged ones (max_m r_m < tol), those at max_steps (status
 * UGKS_ENOTCONVERGED) and those with a numeric failure, keeping their rho, U,
 * T, q on the host and freeing their device memory.  The server is
 * thread-safe (one mutex); its inputs are copied at submission. */
enum { UGKS_REQ_QUEUED = 0, UGKS_REQ_RUNNING = 1, UGKS_REQ_DONE = 2, UGKS_REQ_FAILED = 3 };

typedef struct {
    int32_t state;            /* UGKS_REQ_* */
    int32_t status;           /* UGKS_OK, UGKS_ENOTCONVERGED, or the failing call's status */
    int64_t steps;            /* steps taken */
    double residual[5];       /* residual of the last step (dim+2 used) */
    double t_arrive, t_admit, t_done;   /* server clock, seconds; -1 if not yet */
    size_t footprint_bytes;   /* admission estimate */
    size_t device_bytes;      /* bytes the case actually held */
    int64_t n_cells, nv;
} ugks_result;

typedef struct {
    size_t device_budget, device_used;
    int32_t n_running, n_queued;
    int64_t total_cvu;        /* cell-velocity updates executed so far */
    double clock;             /* server clock now, seconds */
} ugks_server_stats_t;

typedef struct ugks_server ugks_server;

/* device_budget_bytes: device memory the admitted cases may hold in total;
 * max_slots: cases running at once; steps_per_tick: batched steps between
 * residual checks; stream: cudaStream_t (NULL: the server's own). */
ugks_status ugks_server_create(size_t device_budget_bytes, int32_t max_slots, int32_t steps_per_tick, void *stream,
                               ugks_server **out);
/* Queue a case (inputs copied).  t_arrive >= 0: arrival time on the server
 * clock (the request is not admitted before it); < 0: now.  Returns a ticket. */
ugks_status ugks_server_submit(ugks_server *s, const ugks_mesh *mesh, const ugks_vgrid *vgrid,
                               const ugks_params *params, double tol, int64_t max_steps, double t_arrive,
                               uint64_t *ticket);
/* One round: admit, step, retire.  Reports the running and queued counts. */
ugks_status ugks_server_tick(ugks_server *s, int32_t *n_running, int32_t *n_queued);
ugks_status ugks_server_poll(ugks_server *s, uint64_t ticket, ugks_result *out);
/* rho[C], U[C][dim], T[C], q[C][dim] of a finished request (caller order). */
ugks_status ugks_server_moments(ugks_server *s, uint64_t ticket, double *rho, double *U, double *T, double *q);
ugks_status ugks_server_stats(ugks_server *s, ugks_server_stats_t *out);
void ugks_server_destroy(ugks_server *s);

/* ---- Domain decomposition (Sec. 3.3, Algorithm 2) ----
 * A mesh is split into subdomains, each a case of its own (one per GPU, or
 * several on one GPU).  A subdomain's mesh lists its own cells first, then a
 * halo of two face rings around them (the cells one explicit step reads:
 * slopes of the face neighbours, whose limited gradients read the second
 * ring), with every face of its own cells and of the first ring.  One step of
 * the subdomain updates its own cells exactly as a step of the whole mesh
 * would, given the same time step; the halo's values come out wrong and are
 * replaced before the next step by the owners' values (f^{n+1}, W^{n+1} and the
 * heat flux q^{n+1}): pack the cells another subdomain needs into a device
 * buffer, move the buffer (a device copy on one GPU, NCCL send/receive or a
 * peer copy into the receiver's own buffer across GPUs), unpack it into the
 * receiving subdomain's halo cells.  The paper overlaps this exchange with the
 * interior update by non-blocking MPI (Algorithm 2); here the buffers move
 * between steps on the case streams. */

/* dt = cfl * min_i 2|Omega_i| / sum_f S_f(i) / max_k |u_k| over the first
 * n_cells cells of the mesh (the CFL step of Algorithm 1, as ugks_create
 * computes it over all cells).  A subdomain's own cells hold all their faces,
 * so the minimum of this value over the subdomains (their own cells first) is
 * the whole mesh's time step; pass it as ugks_params.dt to every subdomain.
 * Host computation; *dt receives the step. */
ugks_status ugks_cfl_dt(const ugks_mesh *mesh, const ugks_vgrid *vgrid, double cfl, int64_t n_cells, double *dt);

/* Mark the first n_owned cells (caller order) as the case's own cells: the
 * residual sums of later steps count only them.  Default: every cell. */
ugks_status ugks_set_owned(ugks_case *c, int64_t n_owned);

/* Residual sums of the last step over the own cells: sums[m] =
 * sum_i (W^{n+1}_im - W^n_im)^2 and sums[D+2+m] = sum_i (W^n_im)^2, m < dim+2
 * (host buffer of 2(dim+2) doubles; zeros before the first step).  Adding the
 * sums of all subdomains (an all-reduce) and taking sqrt(sums[m]) /
 * sqrt(sums[D+2+m]) gives ugks_residual of the whole mesh.  Synchronises. */
ugks_status ugks_residual_sums(ugks_case *c, double *sums);

/* Bytes of one halo row: f of a cell in the storage precision ([ncomp][nv],
 * FP32 or FP64, padded to 8 bytes), then W [dim+2] and q [dim] in FP64. */
ugks_status ugks_halo_row_bytes(const ugks_case *c, size_t *bytes);

/* Register halo list `slot` (0 <= slot < 4096): the caller cells cells[0..n)
 * whose rows ugks_halo_pack writes to, or ugks_halo_unpack reads from, a
 * buffer in this order.  The list is copied to the device; setting a slot
 * again replaces it (after the case stream has finished using the old one).
 * UGKS_EINVAL for an id outside [0, n_cells). */
ugks_status ugks_halo_set(ugks_case *c, int32_t slot, const int64_t *cells, int64_t n);

/* Write the rows of slot's cells (the current f, W and q) to device_buf
 * (n x row bytes, 8-byte aligned, caller-owned device memory), or overwrite
 * slot's cells from such a buffer.  Asynchronous on the case stream. */
ugks_status ugks_halo_pack(ugks_case *c, int32_t slot, void *device_buf);
ugks_status ugks_halo_unpack(ugks_case *c, int32_t slot, const void *device_buf);

/* Sizes and tiling of a case. */
ugks_status ugks_info(const ugks_case *c, ugks_info_t *info);

/* Release the device memory of a case (NULL is ignored). */
void ugks_destroy(ugks_case *c);

/* Residual of two conserved-variable states held on the device, computed
 * without allocating any device memory.  For callers that cannot call
 * cudaMalloc: code running under an external memory manager that has already
 * reserved the device memory, a serving loop that admits work against a fixed
 * device budget, or a monitoring hook that must not synchronise the device.
 * The paper has no counterpart; it returns the same quantity as ugks_residual.
 *   W_old, W_new: device pointers, [n_cells][dim+2] conserved variables, the
 *                 same cell order in both; read only.
 *   res:          device pointer to dim+2 doubles (caller-owned), receives
 *                 |W_new_m - W_old_m|_2 / |W_old_m|_2 per component.
 *   stream:       cudaStream_t the two kernels are issued on (NULL: legacy
 *                 default stream); the call is asynchronous.
 * Limit: n_cells <= 2,097,152 (UGKS_EINVAL above it).  The block partial sums
 * live in a fixed 655 KB file-scope device array that every device which loads
 * the library holds until the process exits.  The first call on a device looks
 * up that array's device address (with that device current), and so does the
 * first call after the device's context changed (cudaDeviceReset, or a primary
 * context released and created again); make the first call on each device, and
 * the first after such a change, before any stream capture.  All calls share
 * the array: calls whose kernels overlap on the GPU race and give wrong
 * results.  Each call writes every partial it reads, so nothing carries over
 * from an earlier call.  No cudaMalloc, cudaFree or allocating routine is
 * called. */
ugks_status ugks_residual_noalloc(const double *W_old, const double *W_new, int64_t n_cells, int32_t dim,
                                  double *res, void *stream);

/* Message of the last failed call on this thread ("" if none). */
const char *ugks_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* UGKS_H */
