/*
 * dect.h -- C ABI of libdect, the GB300 (sm_103a) hot path of sparse-view
 * dual-energy CT reconstruction and image-domain decomposition:
 *
 *   Li, Cai, Wang, Yan et al., "Efficient Image Reconstruction and Practical
 *   Decomposition for Dual-energy Computed Tomography" (arXiv:1607.01650).
 *
 * Stage 1 reconstructs the high- and low-energy images x_h, x_l from their
 * sinograms m_h, m_l by the alternating direction method (ADM) on the
 * TV-regularised least-squares model of Eq. (4) (Sec. 2.2).  Stage 2
 * decomposes the two images into two basis-material maps u_1, u_2 by the
 * penalised least-squares (PLS) estimate of Eq. (13) (Sec. 2.3).
 *
 * Conventions (all entry points):
 *   - Arrays are FP32, row-major, contiguous, in DEVICE memory of the plan's
 *     device, allocated and owned by the caller, unless stated otherwise.
 *   - Image of n x n pixels: index row * n + col, row = y, col = x; pixel
 *     (0, 0) has its centre at (-(n-1) px / 2, -(n-1) px / 2) mm; the image is
 *     centred on the rotation axis.  Units: mm, 1/mm, rad.
 *   - Sinogram: [view][bin], n_views x n_bins.  Ray (v, b) goes from the
 *     source S_v = SOD (cos t_v, sin t_v), t_v = start + v * (arc / n_views),
 *     to the centre of bin b of a flat detector, at
 *     (SOD - SDD)(cos t_v, sin t_v) + u_b (-sin t_v, cos t_v),
 *     u_b = (b - (n_bins - 1) / 2) pitch + det_offset (Sec. 2.1, Fig. 1).
 *   - Every call is ordered on `stream` (a cudaStream_t; NULL = legacy
 *     default stream) and returns once its work is enqueued, except where a
 *     call says that it synchronises.
 *   - Arguments are checked on the host before anything is enqueued; a bad
 *     argument returns DECT_ERR_INVALID_ARG and enqueues nothing.  CUDA
 *     errors are returned as DECT_ERR_CUDA; dect_last_error() gives the text.
 *   - There is no CPU fallback: without a usable sm_103a device every call
 *     that needs one returns DECT_ERR_CUDA.
 */
#ifndef DECT_H
#define DECT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DECT_OK = 0,
    DECT_ERR_INVALID_ARG = 1,
    DECT_ERR_CUDA = 2,
    DECT_ERR_OOM = 3,
    DECT_ERR_TIMEOUT = 4,
    DECT_ERR_NONFINITE = 5,
    DECT_ERR_NOT_CONVERGED = 6,
    DECT_ERR_INDEX = 7          /* an index check of the checked build failed */
} dect_status;

/* Opaque CUDA stream (binary-compatible with cudaStream_t). */
typedef struct CUstream_st *dect_stream;

/* Fan-beam slice geometry: the centre slice of the cone-beam system of
 * Sec. 2.1 / Fig. 1 and Sec. 3 (flat 1-D detector, circular source orbit). */
typedef struct {
    int n;               /* image is n x n pixels, 1 <= n <= 8192            */
    double pixel_mm;     /* pixel side (> 0)                                  */
    int n_views;         /* views, >= 1                                       */
    int n_bins;          /* detector bins, >= 1                               */
    double pitch_mm;     /* bin pitch (> 0)                                   */
    double sod_mm;       /* source to rotation axis (> image half-diagonal)   */
    double sdd_mm;       /* source to detector (> sod_mm)                     */
    double start_rad;    /* angle of view 0                                   */
    double arc_rad;      /* angular range of the n_views views (> 0)          */
    double det_offset_mm;/* detector shift along its axis                     */
} dect_geometry;

/* Opaque plan: one geometry, its Siddon system matrix A of Eq. (1) stored on
 * the device twice -- ray-major (for A x) and pixel-major (for A^T y). */
typedef struct dect_plan dect_plan;

typedef struct {
    int64_t n_pixels;     /* N = n * n                                        */
    int64_t n_rays;       /* M = n_views * n_bins                             */
    int64_t nnz;          /* (ray, pixel) intersections of A                  */
    int64_t table_bytes;  /* device bytes held by both tables                 */
    int64_t n_grid_aligned; /* rays within 1e-9 mm of running along a grid line */
} dect_plan_info;

/*
 * Build the plan of `geom` on CUDA device `device` (Eq. (1) and Siddon's
 * method, ref. [42] of the paper): each ray's pieces between consecutive
 * crossings of pixel-grid lines inside the image box, each given to the pixel
 * that holds the piece's midpoint, crossing parameters in FP64, lengths
 * stored as FP32 mm.  Zero-length pieces are dropped.  Synchronises `stream`.
 * *out receives the plan (owned by the caller; free with dect_plan_destroy).
 * Errors: DECT_ERR_INVALID_ARG for a bad geometry or NULL out;
 * DECT_ERR_OOM when the tables do not fit; DECT_ERR_CUDA otherwise.
 */
dect_status dect_plan_create(const dect_geometry *geom, int device, dect_stream stream,
                             dect_plan **out);

/*
 * Cone-beam geometry (Sec. 2.1, Fig. 1 with a flat 2-D detector; the
 * paper's scan, Sec. 3): the source turns in the plane z = 0; view v at
 * t_v = start + v * (arc / n_views), source SOD (cos t, sin t, 0); detector
 * centred at (SOD - SDD)(cos t, sin t, 0) with axes (-sin t, cos t, 0)
 * (columns) and (0, 0, 1) (rows); cell (row r, column c) at
 * u_c = (c - (n_cols - 1) / 2) pitch_u + offset_u,
 * z_r = (r - (n_rows - 1) / 2) pitch_v + offset_v.  Volume of n x n x nz
 * voxels of pixel_mm x pixel_mm x slice_mm centred on the origin, index
 * (k n + i) n + j (k along z, i = row = y, j = column = x); projections
 * [view][row][column].
 */
typedef struct {
    int n, nz;
    double pixel_mm, slice_mm;
    int n_views, n_rows, n_cols;
    double pitch_u_mm, pitch_v_mm;
    double sod_mm, sdd_mm, start_rad, arc_rad, offset_u_mm, offset_v_mm;
} dect_cone_geometry;

/*
 * Build the plan of a cone-beam geometry: the Siddon system matrix in 3-D
 * (crossings of the x, y and z grid planes, each piece given to the voxel
 * holding its midpoint, FP64 crossing parameters, FP32 lengths), ray-major
 * and voxel-major, as dect_plan_create does in 2-D.  The plan serves
 * dect_project, dect_backproject, dect_plan_get_info (n_pixels = voxels,
 * n_rays = cells x views) and dect_plan_copy_table; the fan-beam solvers
 * and the on-the-fly projector refuse it (DECT_ERR_INVALID_ARG).
 * Errors: DECT_ERR_INVALID_ARG (bad geometry: sizes < 1, non-positive
 * sizes or pitches, SOD not beyond the volume's half diagonal, SDD <= SOD,
 * more than 2^30 rays or voxels), DECT_ERR_OOM, DECT_ERR_CUDA.
 */
dect_status dect_plan_create_cone(const dect_cone_geometry *geom, int device, dect_stream stream,
                                  dect_plan **out);

/* Free a plan and its device tables (NULL is a no-op). Synchronises the device. */
dect_status dect_plan_destroy(dect_plan *plan);

/* Sizes of a plan (host struct written by the call). */
dect_status dect_plan_get_info(const dect_plan *plan, dect_plan_info *info);

/*
 * Copy the ray-major table of A to HOST memory: rowptr[n_rays + 1] (int64),
 * pix[nnz] (int32 pixel index), len[nnz] (FP32, mm); row r = v * n_bins + b,
 * entries of a row in the order the ray meets them.  Any pointer may be NULL
 * to skip it.  Synchronises `stream`.  For tests and inspection.
 */
dect_status dect_plan_copy_table(const dect_plan *plan, int64_t *rowptr, int32_t *pix,
                                 float *len, dect_stream stream);

/*
 * y = A x, Eq. (1), for `batch` images: x [batch][n][n] -> y [batch][n_views][n_bins].
 * The batch runs in passes of up to 64 images: each pass copies its images
 * into a pixel-major interleaved scratch ([pixel][64]), streams the ray-major
 * table once, and copies the sums out.  FP32 multiply-add in a fixed order;
 * deterministic.  The scratch (about 4 (N + M) min(batch, 64) bytes) is
 * taken from the stream-ordered allocator and returned before the call ends.
 * Errors: DECT_ERR_INVALID_ARG (NULL plan/pointer, batch < 0), DECT_ERR_OOM,
 * DECT_ERR_CUDA.  batch = 0 is a no-op.
 */
dect_status dect_project(const dect_plan *plan, const float *x, float *y, int batch,
                         dect_stream stream);

/*
 * x = A^T y, the exact transpose used by the gradient G_f of Eq. (9), for
 * `batch` sinograms: y [batch][n_views][n_bins] -> x [batch][n][n].
 * Gather form over the pixel-major table (rays increasing inside a pixel),
 * in passes of up to 64 sinograms interleaved as for dect_project, pixels
 * taken in 8 x 8 tiles; every pixel sums its rays in a fixed order; no
 * atomics, bitwise reproducible.  Scratch and errors as dect_project.
 */
dect_status dect_backproject(const dect_plan *plan, const float *y, float *x, int batch,
                             dect_stream stream);

/*
 * Fan-beam filtered backprojection of `batch` sinograms, the analytic
 * reconstruction the paper compares against (Sec. 2.4) and shows for its
 * real data (Sec. 3); here an initial image for dect_adm_tv (warm_start = 1).
 * Textbook algorithm for an equally spaced flat detector: bins moved to the
 * isocentre, cosine pre-weight SOD / sqrt(SOD^2 + s^2), Ram-Lak ramp filter
 * at the isocentre bin spacing, back-projection with the (SOD / L)^2 weight,
 * linear interpolation between bins, 1/2 for the double coverage of 360 deg.
 * m: [batch][n_views][n_bins] line integrals; x: [batch][n][n] (1/mm).
 * Device scratch (filtered sinograms) is taken from the stream-ordered
 * allocator and returned before the call ends.  The filter and the geometry
 * run in FP64 (the ramp filter cancels the projections' mean), the
 * back-projection sums in FP32; deterministic.
 * Errors: DECT_ERR_INVALID_ARG (NULL plan/pointer, batch < 0, a plan whose
 * arc is not 2 pi, fewer than 2 bins), DECT_ERR_OOM, DECT_ERR_CUDA.
 * batch = 0 is a no-op.
 */
dect_status dect_fbp(const dect_plan *plan, const float *m, float *x, int batch, dect_stream stream);

/* Step rules for the f-subproblem (Eq. (9)); c(G) = |G|^2/(mu|AG|^2 + rho|grad G|^2). */
enum { DECT_STEP_BB1 = 0,     /* alpha^k = c(G^{k-1}), alpha^0 = c(G^0) (lagged, BB-like) */
       DECT_STEP_CAUCHY = 1   /* alpha^k = c(G^k) (exact line search along -G)           */ };

typedef struct {
    double mu;          /* data weight of Eq. (4), > 0                                  */
    double rho;         /* penalty of Eq. (6), > 0                                      */
    double xi;          /* multiplier step of Eq. (7); <= 0 means xi = rho              */
    double beta[2];     /* Eq. (3) weights: beta[0] on x_h (energy 0), beta[1] on x_l   */
    int step_rule;      /* DECT_STEP_BB1 or DECT_STEP_CAUCHY                            */
    int max_iter;       /* iterations, >= 0                                             */
    double rel_obj_tol; /* stop a channel once |Phi_k - Phi_{k-1}| / Phi_{k-1} < tol;
                           <= 0: always run max_iter                                    */
    int check_every;    /* host checks "all channels stopped" (and whether the batch
                           can narrow) every this many iterations, rounded up to an
                           even number (>= 1; 0 = 10); used when rel_obj_tol > 0       */
    int warm_start;     /* 0: start from x = 0; 1: start from the x passed in           */
    int nonneg;         /* 1: project f onto f >= 0 after every f-step (x in R_+^N,
                           Eq. (1)); costs one extra A per iteration to rebuild the
                           residual.  0: the unconstrained steps of Eq. (7)-(10)        */
    int joint_tv;       /* 0: TV per energy channel (the stacked problem splits);
                           1: one TV over the stacked image: at each pixel the norm of
                           both energies' gradients (4-vector), one step and one
                           stopping test per slice, reports carry the slice's joint
                           objective on both channels                                  */
} dect_adm_params;

typedef struct {
    int iters;          /* iterations done (f^iters is the result)                      */
    int converged;      /* 1 if the relative-objective test fired                       */
    double objective;   /* Phi = |grad f|_TV + mu/2 |A f - g|^2 at the result (f = beta x) */
    double rel_change;  /* last relative objective change                               */
    double primal_res;  /* |A f - g| at the result, recomputed from f at the end of the
                           call (FP32 projection, FP64 norm)                             */
    double resid_drift; /* |r - (A f - g)|: how far the residual r carried through the
                           iterations by r <- r - alpha A G (Eq. (9) by linearity) has
                           moved from the recomputed one; `objective` and the stopping
                           test use the carried r                                         */
} dect_adm_report;

/*
 * ADM-TV reconstruction, Eq. (3)-(10), of `n_slices` dual-energy slices that
 * share `plan`.  m: [n_slices][2][n_views][n_bins] measured line integrals
 * (energy 0 = high kVp, 1 = low).  x: [n_slices][2][n][n]; on input the warm
 * start (read only when params->warm_start = 1), on output the images x_h, x_l.
 *
 * Each channel c runs the iteration of Eq. (10) on f = beta_c x against
 * g = beta_c m (the stacked system of Eq. (3) separates per channel because
 * the TV of Eq. (4) is taken per channel):
 *   z     = shrink(grad f - lambda/rho, 1/rho)                         Eq. (8)
 *   G     = mu A^T (A f - g) + rho grad^T(grad f - z) - grad^T lambda  Eq. (9)
 *   f    <- f - alpha G   (alpha from the step rule)                   Eq. (9)
 *   lambda <- lambda - xi (grad f - z)                                 Eq. (7)
 * with grad the backward differences of Eq. (2) and Phi the objective of
 * Eq. (4).  Bulk arithmetic is FP32; the norms that give alpha and Phi are
 * accumulated in FP64 across warps and blocks.
 * Up to 64 channels (32 slices) share one pass over the system matrix.  With
 * rel_obj_tol > 0, once no more than half of such a batch is still running,
 * the running channels continue in a batch half as wide (the same iterates;
 * only the order of the FP64 cross-block sums changes).  Calls of more than
 * 32 slices run their chunks of 32 two at a time, from two host threads on
 * streams of their own ordered after `stream`, after autotuning every batch
 * width on the calling thread; each chunk's result is that of the chunk
 * alone.
 * reports: HOST array [n_slices * 2] (may be NULL).  Synchronises `stream`.
 * Device scratch is taken from the stream-ordered allocator and returned
 * before the call ends.
 * Errors: DECT_ERR_INVALID_ARG, DECT_ERR_OOM, DECT_ERR_CUDA;
 * DECT_ERR_NONFINITE when an objective was not finite; DECT_ERR_TIMEOUT when
 * a bounded wait inside the TV step (variant 1, dect_plan_get_tv_tuning) ran
 * out (the images are then not valid).
 */
dect_status dect_adm_tv(const dect_plan *plan, const float *m, float *x, int n_slices,
                        const dect_adm_params *params, dect_adm_report *reports,
                        dect_stream stream);

/* One group of a mixed-geometry batch: slices that share `plan`. */
typedef struct {
    const dect_plan *plan;
    const float *m;            /* [n_slices][2][n_views][n_bins], device           */
    float *x;                  /* [n_slices][2][n][n], device (in: warm start)     */
    int n_slices;
    dect_adm_report *reports;  /* HOST [n_slices * 2] or NULL                       */
} dect_adm_group;

/*
 * ADM-TV of a batch of slices of uneven size and view count, Eq. (3)-(10):
 * each group is reconstructed as dect_adm_tv would (all its slices'
 * channels interleaved per table pass), and the groups run concurrently,
 * each on its own stream ordered after `stream`, from up to `workers` host
 * threads (0 = min(n_groups, 8)).  Plans must differ between groups.
 * Synchronises `stream`.  Returns the first error of any group.
 */
dect_status dect_adm_tv_groups(const dect_adm_group *groups, int n_groups,
                               const dect_adm_params *params, int workers, dect_stream stream);

/*
 * ADM-TV, Eq. (3)-(10), of slices of uneven size and view count, each
 * group's slices sharing its plan (plans may repeat), all slices of all
 * groups advanced together: one launch per ADM phase covers every running
 * slice (per-slice steps, stopping tests and reports as dect_adm_tv; each
 * slice's two energies interleaved), and slices whose channels have all
 * stopped leave the launches at the next host check (every check_every
 * iterations).  The projector is computed on the fly (no stored table):
 * a_ij is the length of ray i inside pixel j, the overlap of the ray's two
 * slabs of that pixel, from FP32 crossing parameters measured from the
 * ray's point nearest the rotation axis; A x walks each ray through its
 * pixels, A^T y takes each pixel and, per view, the bins whose rays can
 * cross it, and both evaluate a_ij by the same function, so A^T is the
 * exact transpose of A (results agree with the stored-table path to FP32
 * rounding of the lengths).  Plans with rays along a grid line
 * (dect_plan_info.n_grid_aligned > 0) are rejected (the two paths assign
 * such rays differently): use dect_adm_tv for them.
 * Each group: m [n_slices][2][n_views][n_bins], x [n_slices][2][n][n]
 * (device, as for dect_adm_tv), reports HOST [n_slices * 2] or NULL.
 * Device scratch from the stream-ordered allocator; synchronises `stream`.
 * Errors: DECT_ERR_INVALID_ARG, DECT_ERR_OOM, DECT_ERR_CUDA,
 * DECT_ERR_NONFINITE.
 */
dect_status dect_adm_tv_batch(const dect_adm_group *groups, int n_groups, const dect_adm_params *params,
                              dect_stream stream);

/* Projector forms of dect_adm_tv_batch_ex. */
#define DECT_PROJ_TABLE 0 /* the plans' stored Siddon tables (Eq. (1), ref. [42]) */
#define DECT_PROJ_OTF 1   /* computed on the fly, as dect_adm_tv_batch          */

/*
 * dect_adm_tv_batch with a choice of projector.  DECT_PROJ_TABLE streams
 * each slice's stored tables, the ones dect_adm_tv uses (A x: a warp per ray
 * of the ray-major table; A^T y: a warp per pixel of the pixel-major table,
 * deterministic, no atomics), so every slice runs the iteration of
 * dect_adm_tv on its plan, with the same launches per ADM phase over all
 * slices as dect_adm_tv_batch; plans with rays along grid lines are
 * accepted.  DECT_PROJ_OTF is dect_adm_tv_batch.  Arguments, layouts,
 * reports and errors as dect_adm_tv_batch; DECT_ERR_INVALID_ARG for another
 * `projector`.
 */
dect_status dect_adm_tv_batch_ex(const dect_adm_group *groups, int n_groups, const dect_adm_params *params,
                                 int projector, dect_stream stream);

/*
 * A x and A^T y as dect_project / dect_backproject, with the on-the-fly
 * projector of dect_adm_tv_batch (no table is read; the plan's ray and view
 * parameters, 32 bytes per ray, are built on the first call and kept with
 * the plan).  Images are processed two at a time.  Scratch from the
 * stream-ordered allocator.  Errors as dect_project.
 */
dect_status dect_project_otf(const dect_plan *plan, const float *x, float *y, int batch, dect_stream stream);
dect_status dect_backproject_otf(const dect_plan *plan, const float *y, float *x, int batch,
                                 dect_stream stream);

typedef struct {
    double eta[2][2];   /* eta[material][energy]: attenuation (1/mm) of basis material
                           1 / 2 at energy 0 (high) / 1 (low); D of Eq. (12)            */
    double gamma;       /* smoothness weight of Eq. (13), >= 0                           */
    double edge_tau;    /* edge threshold on the max-normalised Prewitt magnitude        */
    double edge_eps;    /* e_ik for pairs touching an edge pixel (Eq. (14)), >= 0        */
    int max_iter;       /* PCG iterations, >= 0                                          */
    double tol;         /* stop when |r| / |b| < tol (<= 0: run max_iter)                */
} dect_pls_params;

typedef struct {
    int iters[2];       /* PCG iterations per material                                  */
    double relres[2];   /* final |r| / |b| per material                                 */
} dect_pls_report;

/*
 * PLS decomposition, Eq. (11)-(15), of `batch` slices of n x n pixels:
 *   d = D^{-1} x per pixel (2x2 closed form in FP64), Eq. (11)-(12);
 *   edge map: 3x3 Prewitt magnitude of x_h and of x_l (replicate padding),
 *   each divided by its own maximum, edge where either exceeds edge_tau
 *   (decided in FP32, as dect_pls_edge_mask returns it);
 *   e_ik = edge_eps if pixel i or k is an edge, else 1, Eq. (14);
 *   solve (I + gamma L_e) u_m = d_m for m = 1, 2, (L_e u)_i = sum over the
 *   4-neighbours k inside the image of e_ik (u_i - u_k) -- Eq. (15), whose
 *   Hessian of R is 2 L_e -- by Jacobi-preconditioned CG from u = d.
 * x: [batch][2][n][n] (x_h, x_l per slice: the layout dect_adm_tv writes);
 * u: [batch][2][n][n] output (u_1, u_2 per slice).  x and u must not overlap.
 * reports: HOST array [batch] (may be NULL).  Synchronises `stream`.
 * Device scratch is taken from the stream-ordered allocator and returned
 * before the call ends.
 */
dect_status dect_pls_decompose(const float *x, int n, int batch, const dect_pls_params *params,
                               float *u, dect_pls_report *reports, dect_stream stream);

/*
 * The edge map of Eq. (14) (Sec. 2.3) that dect_pls_decompose uses, for
 * `batch` slices: for each of x_h and x_l the 3x3 Prewitt magnitude
 * (replicate padding) divided by that image's largest magnitude; a pixel is
 * an edge (1) when either ratio exceeds edge_tau, else 0.  Magnitudes,
 * maxima and the division are FP32 (the precision of the images), so the
 * result can differ from an FP64 decision only at pixels whose ratio lies
 * within FP32 rounding of edge_tau.
 * x: [batch][2][n][n] device (x_h, x_l per slice); mask: [batch][n][n] uint8,
 * device, written.  Device scratch (the magnitudes) is taken from the
 * stream-ordered allocator and returned before the call ends; the call does
 * not synchronise.
 * Errors: DECT_ERR_INVALID_ARG (NULL pointer, n outside 1..16384, batch < 0
 * or > 65535, non-finite edge_tau), DECT_ERR_CUDA.  batch = 0 is a no-op.
 */
dect_status dect_pls_edge_mask(const float *x, int n, int batch, double edge_tau, uint8_t *mask,
                               dect_stream stream);

/*
 * PLS decomposition of `batch` cone-beam volumes of nz slices of n x n
 * voxels (x: [batch][2][nz][n][n], u the same), Eq. (11)-(15) with the
 * 6 face neighbours of a voxel inside the volume as N_i of Eq. (14) and the
 * 3-D Prewitt magnitude for the edge map (each component the difference of
 * the two neighbours along its axis summed over the 3 x 3 neighbourhood of
 * the other two axes, replicate padding, FP32).  Otherwise as
 * dect_pls_decompose (which is this call with nz = 1 and the 2-D Prewitt).
 * Errors: as dect_pls_decompose; nz outside 1..4096 is DECT_ERR_INVALID_ARG.
 */
dect_status dect_pls_decompose_cone(const float *x, int n, int nz, int batch, const dect_pls_params *params,
                                    float *u, dect_pls_report *reports, dect_stream stream);

/* The edge map of dect_pls_decompose_cone: mask [batch][nz][n][n]. */
dect_status dect_pls_edge_mask_cone(const float *x, int n, int nz, int batch, double edge_tau, uint8_t *mask,
                                    dect_stream stream);

/*
 * dect_pls_decompose without any device allocation.  (The paper has no
 * counterpart: this is a service of the library, not a step of the method.)
 *
 * Who needs it: callers that must not allocate device memory while they
 * run -- e.g. an inline reconstruction service that reserves the whole
 * device pool at start-up and keeps its footprint fixed, or a plug-in inside
 * a process whose own allocator owns the GPU.  This variant computes exactly
 * what dect_pls_decompose computes (same kernels, same arguments, same
 * results) but takes its scratch from one fixed array compiled into the
 * library, of DECT_PLS_NOALLOC_SCRATCH_BYTES bytes, which every device that
 * loads the library holds until the process exits.  It calls no cudaMalloc,
 * cudaFree or other allocating routine, creates no stream, event or graph and
 * pins no host memory; the caller still passes x and u.
 *
 * Limits: batch * n * n <= DECT_PLS_NOALLOC_MAX_PIXELS and
 * batch <= DECT_PLS_NOALLOC_MAX_BATCH; larger work returns
 * DECT_ERR_INVALID_ARG (dect_last_error() says why) -- use
 * dect_pls_decompose for it.
 *
 * Shared state: every call on a device uses the same array, which keeps the
 * previous call's contents (the call clears what must start at zero).  Calls
 * whose work overlaps on the GPU -- e.g. on two streams without an ordering
 * between them, or from two host threads -- race on it and give wrong
 * results; order them on one stream or serialise them.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture on that device.  Synchronises
 * `stream`.
 */
#define DECT_PLS_NOALLOC_MAX_PIXELS 262144
#define DECT_PLS_NOALLOC_MAX_BATCH 64
#define DECT_PLS_NOALLOC_SCRATCH_BYTES (14u << 20)
dect_status dect_pls_decompose_noalloc(const float *x, int n, int batch, const dect_pls_params *params,
                                       float *u, dect_pls_report *reports, dect_stream stream);

/* Kernel timing of one dect_adm_tv_ex call, from CUDA events recorded
 * around the launches of the two table kernels of one iteration in each
 * launched iteration graph (the middle one of each block of check_every
 * iterations, and each single iteration): launch counts and totals cover
 * those sampled launches. */
typedef struct {
    double fwd_ms_total;   /* q = A G launches (ray-major table)      */
    double bwd_ms_total;   /* G = mu A^T r + ... (pixel-major table)  */
    int64_t fwd_launches;
    int64_t bwd_launches;
    int64_t table_bytes_fwd;  /* algorithmic bytes per fwd launch (mean over the
                                 launches timed: narrowed batches move fewer) */
    int64_t table_bytes_bwd;  /* the same for the bwd launches            */
} dect_adm_profile;

/*
 * dect_adm_tv with optional kernel timing (prof may be NULL, which makes it
 * identical to dect_adm_tv).  With prof != NULL, events are recorded around
 * the A G and A^T r launches of the middle iteration of each block of
 * check_every iterations (an event pair per launch would add a few
 * microseconds to every iteration) and read back after each block; the
 * totals cover all chunks of the call.
 */
dect_status dect_adm_tv_ex(const dect_plan *plan, const float *m, float *x, int n_slices,
                           const dect_adm_params *params, dect_adm_report *reports,
                           dect_adm_profile *prof, dect_stream stream);

/*
 * Autotuner record of a plan: the A^T variant that dect_adm_tv chose for a
 * batch of `images` interleaved channels (2, 4, 8, 16, 32 or 64; a call with
 * c channels uses the next of these widths >= min(c, 64)), and the measured
 * median time of each variant in microseconds (-1 = not available):
 *   0-2 L1-cached gather with 4x4 / 8x8 / 16x16 pixel tiles per 256-thread block,
 *   3   shared-memory sinogram windows (cp.async staged),
 *   4-5 L1-cached gather, one 1024-thread block per SM, tiles of two / four
 *       block steps (8x8 / 16x8 pixels at 32 and 64 channels, 8x16 / 16x16 below),
 *   6-7 (16, 32 or 64 channels; otherwise 4 is used) each lane gathers 8
 *       channels of an entry (two 16-byte loads), so fewer lanes receive
 *       each entry's (index, length): 6 with the lanes and tiles of 4, 7 with
 *       16 lanes per pixel over 8x8 tiles.
 * *choice = -1 until an ADM call with that width has run.  Host memory:
 * us has DECT_BWD_VARIANTS elements.
 */
#define DECT_BWD_VARIANTS 8
dect_status dect_plan_get_tuning(const dect_plan *plan, int images, int *choice,
                                 float us[DECT_BWD_VARIANTS]);

/* Fix the A^T variant used for batch width `images` (skipping the timing),
 * or pass choice = -1 to let the next ADM call time the candidates again.
 * Variant 3 falls back to 1 where the windows do not fit shared memory. */
dect_status dect_plan_set_tuning(dect_plan *plan, int images, int choice);

/*
 * Autotuner record of the forward projector A G inside dect_adm_tv, as
 * dect_plan_get_tuning gives it for A^T: the variant chosen for batch width
 * `images` and the measured median time of each (microseconds; -1 = not
 * timed).  All variants run one 1024-thread block per SM and a warp per ray:
 *   0 each lane gathers 4 channels of an entry (one 16-byte load); the row's
 *     table entries are loaded by the warp together and handed to the lanes
 *     by shuffles,
 *   1 each lane gathers 8 channels of an entry (two 16-byte loads), so fewer
 *     lanes receive each entry's (index, length), four entries per lane in
 *     flight; 16, 32 or 64 channels only (otherwise 0 is used),
 *   2 as 1 with two entries per lane in flight.
 * Timed on the set-up projection r = A f - beta m of the first ADM call
 * with that width.  Host memory: us has DECT_FWD_VARIANTS elements.
 */
#define DECT_FWD_VARIANTS 3
dect_status dect_plan_get_fwd_tuning(const dect_plan *plan, int images, int *choice,
                                     float us[DECT_FWD_VARIANTS]);

/* Fix the A variant for batch width `images`, or -1 to time the candidates
 * again on the next ADM call with that width. */
dect_status dect_plan_set_fwd_tuning(dect_plan *plan, int images, int choice);

/*
 * Autotuner record of the TV step inside dect_adm_tv (the f and r step, the
 * multiplier step of Eq. (7), the z-shrink of Eq. (8) and p, with the TV
 * norm and |r|^2), as dect_plan_get_tuning gives it for A^T: the variant
 * chosen for batch width `images` and the measured median time of each
 * (microseconds; -1 = not timed).
 *   0 blocks claim tiles of 16 rows from a counter and walk down their
 *     columns; the updated row is exchanged through shared memory, one
 *     block barrier per row,
 *   1 each block takes an equal range of (strip, row) pairs; one warp
 *     streams the rows (f, G, the multiplier) into a ring of four
 *     shared-memory stages with 1-D bulk copies (TMA) completing on
 *     mbarriers, the other warps compute from shared memory, no block
 *     barrier per row; 4 or more channels only (otherwise 0 is used).
 * Both give the same images (the same per-pixel arithmetic); the FP32
 * partial sums of the two norms are taken in a different order.  Timed
 * before the first iteration of the first ADM call with that width, where
 * the step changes nothing.  Host memory: us has DECT_TV_VARIANTS elements.
 */
#define DECT_TV_VARIANTS 2
dect_status dect_plan_get_tv_tuning(const dect_plan *plan, int images, int *choice,
                                    float us[DECT_TV_VARIANTS]);

/* Fix the TV-step variant for batch width `images`, or -1 to time the
 * candidates again on the next ADM call with that width. */
dect_status dect_plan_set_tv_tuning(dect_plan *plan, int images, int choice);

/* Number of kernels libdect has launched in this process so far (kernel
 * launches plus the kernel nodes of every graph launch). */
int64_t dect_kernel_launches(void);

/*
 * Self-test of the bounded device waits (failure detection without a GPU
 * fault): a kernel waits on a barrier that nothing completes, for at most
 * `polls` polls, and returns.  Returns DECT_ERR_TIMEOUT when the wait ran out
 * (the expected result), DECT_OK otherwise.  Synchronises `stream`.
 */
dect_status dect_selftest_bounded_wait(unsigned polls, dect_stream stream);

/* ------------------------------------------------------------------------ */
/* CNN warm start (not part of the paper's method: the learned part of the   */
/* workload).  A 3-level encoder-decoder (32/64/128 channels, 3x3            */
/* convolutions + ReLU, 2x2 average pooling, nearest up-sampling, skip       */
/* concatenation, 1x1 head) maps a short ADM reconstruction x to             */
/* x + s * net(x / s), an estimate of the converged image from which ADM     */
/* continues.  BF16 activations and weights on the tensor cores, FP32        */
/* accumulation, FP32 master weights, gradients and Adam state.  Parameter   */
/* vector (host FP32): per layer W[Cout][Cin][3][3] then b[Cout], layers     */
/* (Cin, Cout) = (1,32) (32,32) (32,64) (64,64) (64,128) (128,128) (192,64)  */
/* (64,64) (96,32) (32,32); then the head Wh[32] and bh.                     */
/* Images: FP32 [batch][h][w] device arrays, h and w multiples of 4,         */
/* batch * h * w <= the max_pixels given at creation.                        */
/* ------------------------------------------------------------------------ */
typedef struct dect_cnn dect_cnn;

int64_t dect_cnn_num_params(void);
dect_status dect_cnn_create(int device, int max_pixels, dect_cnn **out);
dect_status dect_cnn_destroy(dect_cnn *net);
/* Copy the parameter vector in (host FP32); resets the Adam state. */
dect_status dect_cnn_set_params(dect_cnn *net, const float *params);
dect_status dect_cnn_get_params(const dect_cnn *net, float *params);
/* out = x + s * net(x / s). */
dect_status dect_cnn_forward(dect_cnn *net, const float *x, float *out, int batch, int h, int w,
                             float scale, dect_stream stream);
/* Loss L = mean over all pixels of (out - target)^2 and its gradient with
 * respect to the parameters (kept on the device for dect_cnn_adam_step;
 * copied to grad if grad != NULL, host FP32).  Synchronises `stream`. */
dect_status dect_cnn_loss_grad(dect_cnn *net, const float *x, const float *target, int batch, int h,
                               int w, float scale, float *loss, float *grad, dect_stream stream);
/* One Adam step on the last gradient. */
dect_status dect_cnn_adam_step(dect_cnn *net, float lr, float beta1, float beta2, float eps,
                               dect_stream stream);

/*
 * Kernel of the 3x3 convolutions (forward and input gradient).
 * DECT_CNN_CONV_TCGEN05 (the default): a persistent implicit GEMM on the
 * 5th-generation tensor cores, accumulating in tensor memory; TMA copies the
 * weights once per block and, per 32 input channels, three column-shifted
 * halo patches of each 8 x 16 pixel tile.  DECT_CNN_CONV_MMA_SYNC: the
 * warp-level mma.sync implicit GEMM, kept for comparison.  Both compute the
 * same sums (BF16 products, FP32 accumulation) in different orders.
 * Returns DECT_ERR_INVALID_ARG for any other value.
 */
#define DECT_CNN_CONV_TCGEN05 0
#define DECT_CNN_CONV_MMA_SYNC 1
dect_status dect_cnn_set_conv_path(dect_cnn *net, int path);
int dect_cnn_get_conv_path(const dect_cnn *net); /* -1 for a NULL net */
/* Resident blocks per SM of the tensor-memory convolution: 2 (the default;
 * each block keeps the deepest operand ring that fits in half the SM's
 * shared memory, where that is at least two stages, else one block) or 1
 * (one block per SM with the deepest ring).  Any other value:
 * DECT_ERR_INVALID_ARG.  Changes speed only, not results. */
dect_status dect_cnn_set_conv_tuning(dect_cnn *net, int blocks_per_sm);

/*
 * Synchronises the device and reads the network's error word.  Returns
 * DECT_ERR_TIMEOUT (and clears the word) when a bounded wait inside a
 * tensor-memory convolution ran out since the last check: the outputs of
 * the calls since then are not valid.  dect_cnn_loss_grad runs this check
 * itself before it returns; after dect_cnn_forward the caller runs it.
 */
dect_status dect_cnn_check(dect_cnn *net);

/*
 * Checked build.  libdect_checked.so is the same library compiled with
 * index checks (DECT_CHECKED): before each table-driven gather, stencil
 * neighbour, on-the-fly ray or pixel and FBP bin access, the index is
 * checked against its array; an index outside it is not used (a safe index
 * is substituted) and the first such failure is recorded on the device.
 * dect_check_status() synchronises the device, then returns DECT_OK, or
 * DECT_ERR_INDEX with the site and index in dect_last_error(), clearing
 * the record.  In the plain library no check is compiled and
 * dect_check_status() returns DECT_OK.  dect_checked_build() returns 1 in
 * the checked library, 0 otherwise.
 */
int dect_checked_build(void);
dect_status dect_check_status(void);

/*
 * Self-test of the index checks: a kernel reads element `index` of an
 * 8-element device array through a check.  In the checked library an index
 * outside 0..7 is caught (not read) and the call returns DECT_ERR_INDEX; in
 * the plain library such an index is refused on the host
 * (DECT_ERR_INVALID_ARG).  Synchronises `stream`.
 */
dect_status dect_selftest_index(int index, dect_stream stream);

/* Text of a status code (static storage). */
const char *dect_status_string(dect_status s);

/* Text of the last CUDA error seen by this thread (static per thread). */
const char *dect_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int dect_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DECT_H */
