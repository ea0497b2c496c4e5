/*
 * fblisa.h -- C ABI of the GB300 (sm_103a) FB-LISA hot path.
 *
 * FB-LISA solves the CT problem of eq. (2.1),
 *     argmin_x  1/2 ||A x - b||^2 + mu ||x||_1 + indicator{x >= 0},
 * with Algorithm 1: mini-batches N_k of whole 2D projections (eq. (2.5)), a
 * forward-backward step x_bar = prox_{alpha R}(x - alpha grad f_N(x)) and the
 * sufficient-decrease line search (2.3).  This header exposes the operator
 * A_N, its exact transpose, the fused objective and prox reductions, and the
 * solver itself.
 *
 * Conventions shared by every call
 * --------------------------------
 * Geometry (the paper delegates the discretisation to a library, Sec. 3;
 * this is the library's own definition):
 *   view i has angle angles[i] (or 2*pi*i/n_views); source
 *   s = SOD*(cos, sin, 0); detector centre -(SDD-SOD)*(cos, sin, 0); detector
 *   axes e_u = (-sin, cos, 0), e_v = (0, 0, 1); pixel (iu, iv) centre
 *   c + (iu-(nu-1)/2)*du*e_u + (iv-(nv-1)/2)*dv*e_v, one ray per pixel.
 *   Voxel (i, j, k) centre ((i-(nx-1)/2)*vx, (j-(ny-1)/2)*vy, (k-(nz-1)/2)*vz).
 *   A is Joseph-type: along the dominant axis a of the ray direction d (ties
 *   to the lower axis) every voxel plane is crossed once, the crossing is
 *   interpolated bilinearly with zero outside the volume, and the row weight
 *   is v_a*|d|/|d_a|.
 * Layouts: volumes are [nz][ny][nx] (x fastest); sinograms are
 *   [view][nv][nu] (u fastest).  A call's "views" list selects which views,
 *   in which order; the k-th listed view fills slice k of a batch sinogram.
 * Pointers: every volume or sinogram pointer may be device memory (the fast
 *   path) or host memory (pageable or pinned); host data are staged through
 *   device buffers on the call's stream.  View lists and scalar outputs are
 *   always host pointers.  All buffers are owned by the caller.
 * Streams: "stream" is a cudaStream_t (NULL = the legacy default stream).
 *   project/backproject enqueue work and return; calls with host outputs
 *   (scalars or host volumes) return after the results are on the host.
 * Device: objects are bound to the CUDA device current at creation; calls
 *   must be made with that device current.
 * Errors: calls return a status and never throw; the message of the last
 *   failure on the calling thread is fbl_last_error().  On error no output
 *   that was passed in is partially updated by a solver step (the trial
 *   point lives in library scratch until it is accepted).
 * There is no CPU fallback: without a usable sm_103a device every call that
 *   computes returns FBL_E_CUDA.
 */
#ifndef FBLISA_H
#define FBLISA_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FBL_API __attribute__((visibility("default")))
#else
#define FBL_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FBL_OK = 0,
    FBL_E_INVAL = 1,        /* bad argument (null pointer, size, view index, dtype) */
    FBL_E_NOMEM = 2,        /* device or host allocation failed */
    FBL_E_CUDA = 3,         /* CUDA runtime error (message has the CUDA error string) */
    FBL_E_UNSUPPORTED = 4,  /* geometry outside what the kernels handle */
    FBL_E_LINESEARCH = 5,   /* no step passed (2.3) within max_backtracks */
    FBL_E_NONFINITE = 6,    /* NaN/Inf in an objective or reduction */
    FBL_E_TIMEOUT = 7       /* a bounded device wait ran out */
} fbl_status;

/* Storage types of volumes and sinograms.  Arithmetic is FP32 along rays and
 * voxel sums, FP64 in the line-search reductions, whatever the storage. */
typedef enum { FBL_F32 = 0, FBL_BF16 = 1, FBL_F16 = 2 } fbl_dtype;

typedef struct fbl_geometry fbl_geometry; /* opaque, library-owned */
typedef struct fbl_solver fbl_solver;     /* opaque, library-owned */

/* Circular cone-beam geometry; lengths in mm, angles in radians. */
typedef struct {
    int32_t nx, ny, nz;       /* volume size in voxels */
    double vx, vy, vz;        /* voxel size */
    int32_t n_views;          /* n_theta, number of views */
    const double *angles;     /* n_views angles, or NULL for 2*pi*i/n_views (copied) */
    double sod, sdd;          /* source-origin and source-detector distances */
    int32_t nu, nv;           /* detector pixels */
    double du, dv;            /* detector pixel size */
} fbl_geometry_desc;

/* The regulariser R of eq. (2.1).  FB-LISA allows any proper convex lower
 * semicontinuous R whose prox is computable (Sec. 2.1); the paper runs the l1
 * one.  Both choices here include the box 0 <= x <= x_max (x_max = +inf: the
 * paper's nonnegativity). */
typedef enum {
    FBL_REG_L1 = 0,   /* R = mu ||x||_1 + box; prox min(max(v - alpha mu, 0), x_max) */
    FBL_REG_TV = 1    /* R = mu TV(x) + box, TV isotropic with forward differences (zero at
                         each axis's last index, unit grid spacing); prox by FGP iterations
                         on the dual (see prox_tv) */
} fbl_reg;

/* Hyperparameters of Algorithm 1 (names as in the paper, Sec. 2.2 and Sec. 3). */
typedef struct {
    double alpha0;            /* initial step alpha_0 (Sec. 3: 1e-3) */
    double beta;              /* backtracking factor beta in (0, 1) */
    double mu;                /* l1 weight mu of eq. (2.1) */
    double C;                 /* C of Step 1 (Sec. 3: M = 1) */
    double eps_base;          /* eps_k = eps_base^k (Sec. 3: 0.99) */
    int32_t N0;               /* initial mini-batch size N_0 (Sec. 3: 8) */
    int32_t n_max;            /* largest mini-batch, 0 = n_views */
    int32_t max_backtracks;   /* cap on step reductions per iteration */
    int32_t proposal;         /* 0: reset alpha to alpha_0 (Step 2d); 1: learned proposal
                                 (set the network with fblisa_set_proposal) */
    uint64_t seed;            /* mini-batch permutation seed */
    int32_t x_dtype;          /* fbl_dtype of the caller's x and the solver's iterates */
    int32_t b_dtype;          /* fbl_dtype of the caller's b */
    int32_t use_graph;        /* 1: run each iteration, backtracking included, as one CUDA graph
                                 whose WHILE node repeats the trial until (2.3) holds */
    int32_t force_reject;     /* test hook: every trial fails (2.3) */
    int32_t autotune;         /* 1: time the kernels' launch configurations at creation */
    int32_t fixed_step;       /* 1: forward-backward with the constant step alpha0 and no line
                                 search (the deterministic FB baseline of Sec. 3 when
                                 N0 = n_max = n_views): no trial objective is evaluated,
                                 f_xbar and margin are reported as NaN; use_graph and
                                 proposal are ignored */
    int32_t reg;              /* fbl_reg; FBL_REG_TV needs use_graph 0 and no batch */
    int32_t tv_iters;         /* FGP iterations per TV prox (each trial of the line search) */
    int32_t tv_warm;          /* 1: each TV prox starts from the dual the previous one ended
                                 with (across trials and iterations); 0: from zero */
    double x_max;             /* upper bound of the box in R (+inf: none, the paper's R) */
} fbl_params;

/* Record of one iteration of Algorithm 1. */
typedef struct {
    int64_t k;                /* iteration index (0-based) */
    int32_t epoch;            /* t (1-based) */
    int32_t N_t;              /* mini-batch size */
    int32_t backtracks;       /* step reductions before acceptance */
    int32_t status;           /* fbl_status of the iteration */
    double alpha;             /* accepted step alpha_k */
    double alpha_init;        /* first trial step of the line search */
    double rho0;              /* ||A_N x - b_N||^2 */
    double f_x;               /* f_N(x) = n_theta/(2 N_t) rho0, eq. (2.5) */
    double f_xbar;            /* f_N(x_bar) at the accepted step */
    double gTd;               /* grad f_N(x)^T (x_bar - x) */
    double dnorm2;            /* ||x_bar - x||^2 */
    double margin;            /* rhs of (2.3) minus f_N(x_bar), >= 0 when accepted */
    double grad_norm2;        /* ||grad f_N(x)||^2 */
    int32_t j_start;          /* first trial was alpha_0 * beta^j_start (0 without proposal) */
    float pred;               /* the proposal network's output (0 without proposal) */
    float features[8];        /* the proposal's inputs at this iteration (always recorded) */
} fbl_step_stats;

/* Defaults: alpha0 1e-3, beta 0.5, mu 1, C 1, eps_base 0.99, N0 8, n_max 0,
 * max_backtracks 60, proposal 0, seed 0, F32 storage, no graph, no hook,
 * no autotuning, line search on (fixed_step 0), reg FBL_REG_L1, tv_iters 20,
 * tv_warm 1, x_max +inf. */
FBL_API void fbl_params_default(fbl_params *p);

/*
 * geometry_create -- validate a cone-beam geometry and build its device
 * tables on the current device.  The geometry is that of A in eq. (2.1),
 * n = n_p * n_theta rows (Sec. 2.1).
 * Errors: FBL_E_INVAL for non-positive sizes or distances;
 * FBL_E_UNSUPPORTED if the volume is not strictly between source and
 * detector, if a ray is dominated by its z component, or if a padded volume
 * would exceed 2^31 elements.
 */
FBL_API fbl_status geometry_create(const fbl_geometry_desc *desc, fbl_geometry **out);
FBL_API void geometry_destroy(fbl_geometry *g);

/* Launch configurations tried by the autotuner and their measured times. */
typedef struct {
    float k1_ms[5];     /* projector, (cols, k1_split) = (8,1), (8,0), (4,1), (4,0), (8,2) */
    float k2_ms[6];     /* backprojector, k2_vpl = 4, 2, 8, 16, 24, 28 (geometry_set_launch) */
    int32_t k1_cols, k1_split, k2_vpl;  /* the chosen configuration */
} fbl_tune_report;

/*
 * geometry_autotune -- time the projector and backprojector launch
 * configurations on this geometry (n_sel views spread over the orbit, storage
 * x_dtype) and keep the fastest for later calls on g.  Results do not depend
 * on the configuration beyond FP32 summation order.  Not safe to call while
 * other calls use g.  report may be NULL.
 */
FBL_API fbl_status geometry_autotune(fbl_geometry *g, int32_t x_dtype, int32_t n_sel, void *stream,
                                     fbl_tune_report *report);

/* Set the launch configuration by hand: k1_cols in {4, 8}; k1_split = the
 * projector's plane loop: 0 plain, 1 with each sample's loads issued one
 * sample ahead in the residual and objective modes (the store mode always
 * does), 2 the volume staged through shared memory by TMA brick copies (8 columns per
 * block whatever k1_cols; its bounded waits report FBL_E_TIMEOUT from the next
 * synchronous call on the geometry, the results stay correct); k2_vpl = the
 * backprojector's work per warp: 2, 4, 8 or 16 consecutive voxels per lane of
 * one voxel column, or 24 / 28 for a 2x2 group of voxel columns with 4 / 8
 * voxels per lane in each (a detector column's z-profile in a plane is then
 * formed once for its two in-plane neighbours; the sums are the same);
 * FBL_E_INVAL otherwise.  The batched solver runs k1_split 2 volumes with the
 * loads-ahead loop. */
FBL_API fbl_status geometry_set_launch(fbl_geometry *g, int32_t k1_cols, int32_t k1_split,
                                       int32_t k2_vpl);

/*
 * project -- y = A_N x (eq. (2.5)'s restricted operator) for the n_sel views
 * listed in views[] (host int32).  x: [nz][ny][nx] of x_dtype; y:
 * [n_sel][nv][nu] of y_dtype, overwritten (may be NULL when n_sel == 0).
 */
FBL_API fbl_status project(const fbl_geometry *g, const void *x, int32_t x_dtype, const int32_t *views,
                   int32_t n_sel, void *y, int32_t y_dtype, void *stream);

/*
 * backproject -- x = A_N^T y (or x += A_N^T y when accumulate != 0), the
 * exact transpose of project, needed by grad f_N in Step 2b of Algorithm 1.
 * y: [n_sel][nv][nu] of y_dtype (may be NULL when n_sel == 0); x: [nz][ny][nx]
 * float32 (zeroed when n_sel == 0 and accumulate == 0).
 */
FBL_API fbl_status backproject(const fbl_geometry *g, const void *y, int32_t y_dtype,
                       const int32_t *views, int32_t n_sel, float *x, int32_t accumulate,
                       void *stream);

/*
 * fdk -- the FDK reconstruction (Feldkamp-Davis-Kress), the analytic method
 * the paper compares with and uses to make its reference volumes (Sec. 3,
 * "Dataset" and the comparison methods), for the circular orbit and flat
 * detector of g, on the virtual detector through the rotation axis
 * (m = sod/sdd): cosine weighting sod / sqrt(sod^2 + a^2 + b^2) of each pixel
 * (a, b = its coordinates times m), Ram-Lak filtering of each detector row
 * (spatial kernel of spacing t = du m: h(0) = 1/(4 t^2), h(k t) =
 * -1/(pi^2 k^2 t^2) for odd k, 0 else; zero outside the detector), and the
 * weighted backprojection sum over views of (dtheta/2) q(eta/U, z/U) / U^2,
 * U = (sod - xi)/sod, bilinear on the detector and zero outside it; dtheta of
 * a view is half the circular gaps to its neighbours among the listed views.
 * y: [n_sel][nv][nu] of y_dtype, the projections of views[] (host int32);
 * x: [nz][ny][nx] float32, overwritten (zero when n_sel == 0).  Host or device
 * buffers; the library allocates its scratch (filtered projections of up to
 * 256 views, one volume).  FP32 filtering and interpolation, detector
 * coordinates from FP64 per voxel column.  The row filter keeps 8 detector
 * rows in shared memory: detectors wider than 3370 columns fail with
 * FBL_E_CUDA (the launch is refused).
 */
FBL_API fbl_status fdk(const fbl_geometry *g, const void *y, int32_t y_dtype, const int32_t *views,
                       int32_t n_sel, float *x, void *stream);

/*
 * residual_norm -- rho = ||A_N x - b_N||^2 in FP64 (the mini-batch fidelity
 * of eq. (2.5) up to the factor n_theta/(2 N_t)), without storing A_N x.
 * b: the full sinogram [n_views][nv][nu] of b_dtype; the listed views are
 * read from it.  *rho_host is written before the call returns.
 */
FBL_API fbl_status residual_norm(const fbl_geometry *g, const void *x, int32_t x_dtype,
                         const int32_t *views, int32_t n_sel, const void *b, int32_t b_dtype,
                         double *rho_host, void *stream);

/*
 * prox_reduce -- the forward-backward point of Step 2c,
 *   x_bar = prox_{alpha R}(x - alpha g) = max(x - alpha g - alpha mu, 0),
 * R = mu||.||_1 + indicator{x >= 0} (eq. (2.1)), stored in x_dtype, and the
 * FP64 reductions the test (2.3) needs, taken over the stored x_bar:
 *   out3_host[0] = g^T (x_bar - x), out3_host[1] = ||x_bar - x||^2,
 *   out3_host[2] = ||x_bar||_1.
 * x, x_bar: n elements of x_dtype (x_bar must not alias x); g: n float32.
 * n = 0 writes three zeros and touches no buffer (which may then be NULL).
 */
FBL_API fbl_status prox_reduce(const void *x, int32_t x_dtype, const float *g, int64_t n, double alpha,
                       double mu, void *xbar, double *out3_host, void *stream);

/*
 * evaluate -- the full objective of eq. (2.1) over all n_views views and the
 * relative error used in Sec. 3 ("Similarity measures"):
 *   out3_host[0] = F(x) = 1/2 ||A x - b||^2 + mu ||x||_1   (x >= 0 assumed),
 *   out3_host[1] = 1/2 ||A x - b||^2,
 *   out3_host[2] = RE = ||x - x_true|| / ||x_true||   (0 when x_true is NULL).
 * x, x_true: [nz][ny][nx] of x_dtype; b: the full sinogram of b_dtype.  FP32
 * projection, FP64 sums.  Returns after the values are on the host.  With
 * R = mu TV (FBL_REG_TV) the objective is out3_host[1] + mu * tv_norm(x).
 */
FBL_API fbl_status evaluate(const fbl_geometry *g, const void *x, int32_t x_dtype, const void *b,
                            int32_t b_dtype, double mu, const void *x_true, double *out3_host,
                            void *stream);

/*
 * prox_tv -- the prox of the TV regulariser (FBL_REG_TV) on one volume:
 *     x = argmin_{0 <= z <= x_max} 1/2 ||z - v||^2 + lambda TV(z),
 * TV(z) = sum over voxels of the Euclidean norm of the forward differences
 * along x, y and z (a zero difference at each axis's last index).  The paper
 * has no counterpart: FB-LISA admits any convex R with a computable prox
 * (Sec. 2.1), and this one has no closed form.  It runs `iters` iterations of
 * the fast gradient projection on the dual (Beck and Teboulle, 2009): with a
 * dual field q of unit vectors, x(q) = clip(v - lambda K^T q, 0, x_max), step
 * q <- P_ball(r + K x(r) / (12 lambda)) with momentum r from the sequence
 * t_1 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2, starting from q (q_in = 1,
 * a warm start; components without a difference are zeroed) or from zero;
 * x = x(q) of the last q.  lambda = 0 gives clip(v, 0, x_max).
 * dims = {nx, ny, nz}; v, x: [nz][ny][nx] float32, x must not alias v (nor q);
 * q: NULL, or 3 * nx*ny*nz float32 [3][nz][ny][nx] (components along x, y, z),
 * read when q_in = 1 and holding the last dual on return.  Host or device
 * pointers (host ones are staged).  Needs ny, nz <= 65535, lambda >= 0,
 * x_max > 0 (+inf allowed), 0 <= iters <= 100000: else FBL_E_INVAL.  FP32
 * arithmetic.  Device scratch of 10 volumes (13 when q is on the host or NULL),
 * stream-ordered: the dual pair alternates between two buffers.  Synchronous with
 * host buffers, else asynchronous on `stream`.
 */
FBL_API fbl_status prox_tv(const int32_t dims[3], const float *v, double lambda, double x_max, int32_t iters,
                           float *q, int32_t q_in, float *x, void *stream);

/*
 * tv_norm -- TV(x) as prox_tv defines it, an FP64 sum of FP32 per-voxel norms
 * in a fixed order.  dims = {nx, ny, nz}, x [nz][ny][nx] float32 (host or
 * device); *out_host receives the value.  Synchronous.
 */
FBL_API fbl_status tv_norm(const int32_t dims[3], const float *x, double *out_host, void *stream);

/*
 * prox_reduce_static -- the same computation and outputs as prox_reduce, for
 * callers that must not allocate device memory: code that runs under a
 * fixed memory budget reserved up front, host applications or plugins whose
 * device memory is owned by someone else, and latency-critical loops where
 * an allocation call could block or synchronize the device.  (The paper has
 * no counterpart; this is a library-level variant.)
 * It allocates nothing: the per-block partial sums and the three results
 * live in one fixed device array of 57 KiB inside the library, which every
 * GPU that loads the library keeps until the process exits.  It launches the
 * same kernels on the same grid as prox_reduce, so x_bar and the three sums
 * are identical to prox_reduce's.
 *   - x, g and x_bar must be device memory of the current device (no host
 *     staging is possible without allocating); otherwise FBL_E_INVAL.  Other
 *     arguments as for prox_reduce (n = 0 included).
 *   - n <= 134217728 (2^27, a 512^3 volume); larger n returns FBL_E_INVAL.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it; make that first call before any
 *     stream capture begins.  The cached address is not valid after a
 *     cudaDeviceReset.
 *   - The call is synchronous: it returns once the three sums are on the host.
 *   - All calls share the one array, and it keeps the last call's contents:
 *     calls whose work overlaps on the GPU (other streams, other threads)
 *     race with each other and must be serialised by the caller.
 */
FBL_API fbl_status prox_reduce_static(const void *x, int32_t x_dtype, const float *g, int64_t n,
                                      double alpha, double mu, void *xbar, double *out3_host,
                                      void *stream);

/*
 * The learned step proposal's network (no counterpart in the paper, which
 * resets the step to alpha_0 at every iteration, Step 2d): a perceptron
 * 8 -> 64 -> 64 -> 1 with tanh hidden units, FP32, parameters packed as
 * W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3 (FBL_MLP_PARAMS floats).
 * Loss: 1/(2n) sum_s (y_s - t_s)^2.  All arrays are device memory; X is
 * [n][8].  mlp_gradient writes the full-batch gradient and *loss_host;
 * mlp_train runs `epochs` passes of Adam (beta1 0.9, beta2 0.999, eps 1e-8)
 * over consecutive minibatches of `batch` samples, updating params, the
 * moment arrays and the device step counter *adam_step.
 */
enum { FBL_MLP_INPUTS = 8, FBL_MLP_HIDDEN = 64, FBL_MLP_PARAMS = 4801 };
FBL_API fbl_status mlp_forward(const float *params, const float *X, int32_t n, float *y, void *stream);
FBL_API fbl_status mlp_gradient(const float *params, const float *X, const float *t, int32_t n,
                                float *grad, double *loss_host, void *stream);
FBL_API fbl_status mlp_train(float *params, float *adam_m, float *adam_v, int32_t *adam_step,
                             const float *X, const float *t, int32_t n, int32_t batch,
                             int32_t epochs, float lr, double *last_loss_host, void *stream);

/*
 * fblisa_create -- a solver for Algorithm 1 on geometry g with the given
 * hyperparameters; owns its scratch (gradient, trial point, residual,
 * reduction slots) and its schedule/mini-batch state (Step 1, Step 2a).
 * The geometry must outlive the solver.
 */
FBL_API fbl_status fblisa_create(const fbl_geometry *g, const fbl_params *p, fbl_solver **out);
FBL_API void fblisa_destroy(fbl_solver *s);

/*
 * fblisa_step -- one iteration k of Algorithm 1 (Steps 2a-2d, plus Step 1
 * and Step 3 at epoch boundaries): draw N_k, compute f_N(x) and grad f_N(x),
 * backtrack alpha until (2.3) holds, set x <- x_bar.
 * x: [nz][ny][nx] of x_dtype, updated in place on acceptance; b: full
 * sinogram [n_views][nv][nu] of b_dtype.  *stats (may be NULL) is filled.
 * Returns after the iteration's scalars are on the host.  On
 * FBL_E_LINESEARCH / FBL_E_NONFINITE x is unchanged and the iteration
 * counter does not advance.
 */
FBL_API fbl_status fblisa_step(fbl_solver *s, void *x, const void *b, fbl_step_stats *stats,
                       void *stream);

/*
 * fblisa_run -- `epochs` epochs of Algorithm 1 from the solver's current
 * position.  trace (may be NULL) receives up to trace_cap records;
 * *n_steps (may be NULL) the number of iterations done.
 */
FBL_API fbl_status fblisa_run(fbl_solver *s, void *x, const void *b, int32_t epochs,
                      fbl_step_stats *trace, int64_t trace_cap, int64_t *n_steps, void *stream);

/*
 * fblisa_set_proposal -- install the step-proposal network (FBL_MLP_PARAMS
 * floats, host or device, copied) and switch the proposal on or off.  With
 * the proposal on, the first trial of each iteration is alpha_0 * beta^j with
 * j = clamp(floor(j_prev + net(features) + 1/2 - margin), 0, max_backtracks),
 * j_prev the grid index of the previous accepted step (0 at the first
 * iteration): a point of the plain rule's own step grid, chosen by the
 * network trained to predict how the index the plain rule needs changes from
 * one iteration to the next.  The test (2.3) and the backtracking are
 * unchanged.  Features (fbl_step_stats.features), with f = f_N(x),
 * g = grad f_N(x) and the curvature index c = log2(alpha_0 |g|^2 / (2 f)):
 * c/10 at the first iteration (0 afterwards), log(f/f_prev),
 * log(|g|/|g_prev|), (c - c_prev)/10, N_t/n_theta, log(1+k)/10, 1 if there is
 * a previous iteration, (j_prev - j_prevprev)/4 -- only relative quantities
 * once there is a previous iteration, so that a network trained on small
 * volumes transfers to large ones.  margin (finite; 0.25 recommended) trades
 * extra first trials (larger margin) against steps below the plain rule's
 * (smaller margin).  Copies params before returning; FBL_E_INVAL on a null
 * solver or a non-finite margin.
 */
FBL_API fbl_status fblisa_set_proposal(fbl_solver *s, const float *params, float margin,
                                       int32_t enable);

/*
 * Per-kernel device time of a solver, for performance reporting: with
 * profiling enabled the solver brackets each of its kernel launches with
 * CUDA events on the launching stream.  Classes: 0 residual projection
 * (Step 2b), 1 trial-objective projection (Step 2c), 2 gradient
 * backprojection, 3 prox + reductions, 4 final FP64 reductions and device
 * line-search control, 5 volume layout conversion.  Launch counts are kept
 * whether or not timing is enabled; in graph mode (use_graph) kernels run
 * inside one graph per iteration and only their counts are kept.
 */
enum { FBL_PROF_CLASSES = 6 };
typedef struct {
    double ms[FBL_PROF_CLASSES];        /* summed device time */
    int64_t launches[FBL_PROF_CLASSES]; /* kernel launches */
} fbl_profile;

/* Enable (1) or disable (0) event timing; if out is non-NULL, copy the
 * counters accumulated so far into it and reset them. */
FBL_API fbl_status fblisa_profile(fbl_solver *s, int32_t enable, fbl_profile *out);

/* The views of the most recent iteration's mini-batch N_k (host copy). */
FBL_API fbl_status fblisa_last_batch(const fbl_solver *s, int32_t *views, int32_t cap, int32_t *n);

/*
 * Batched FB-LISA over several independent volumes (no counterpart in the
 * paper, which reconstructs one volume): each volume v runs its own
 * Algorithm 1 -- geometry geoms[v], parameters params[v] (its own N_0,
 * schedule, seed, mu, ...), line search (2.3) and step proposal -- and one
 * call of fblisa_batch_step advances every volume by one iteration.  On the
 * GPU each phase of that iteration (residual projection, gradient, and, per
 * trial, prox + trial objective + decision) is ONE persistent launch over the
 * tiles of all volumes, and the whole iteration including every volume's
 * backtracking is one CUDA graph (a WHILE node that repeats while any volume
 * is still searching).  A volume's iterates are bit-identical to those of a
 * single-volume solver with the same geometry, parameters and launch
 * configuration.
 *
 * fblisa_batch_create -- n_vol in [1, 1024]; every geometry on one device;
 *   all params[v] with the same x_dtype and b_dtype, and b_dtype == x_dtype
 *   (FBL_E_UNSUPPORTED otherwise).  Launch configuration: the projector's
 *   columns per block (k1_cols) is the largest volume's, for all; every
 *   volume keeps its own geometry's plane-loop form (k1_split) and voxels per
 *   lane (k2_vpl), as set by geometry_autotune / geometry_set_launch.
 *   params[v].autotune and use_graph are ignored.  Copies what it needs; the
 *   geometries must outlive the batch.
 * fblisa_batch_set_proposal -- one network (FBL_MLP_PARAMS floats, host or
 *   device, copied) and margin for every volume, as fblisa_set_proposal;
 *   enable switches the proposal on or off for every volume.
 * fblisa_batch_step -- x[v]: [nz][ny][nx] of x_dtype, in and out (device or
 *   host); b[v]: the full sinogram [n_views][nv][nu] of b_dtype (device or
 *   host); stats: n_vol records or NULL.  Returns FBL_OK when every volume
 *   accepted a step; otherwise the status of the first volume that did not
 *   (FBL_E_LINESEARCH / FBL_E_NONFINITE, also in its stats record): that
 *   volume's x and schedule position are unchanged, the others advanced.
 * fblisa_batch_run -- `iterations` batched steps with x loaded and stored
 *   once; trace (nullable): trace_cap rows of n_vol records; *n_steps = steps
 *   completed (a failing step stops the run).
 * fblisa_batch_info -- launch_cfg[4] = {k1_cols, k1_split and k2_vpl of the
 *   largest volume, the batch's tap count} (nullable); *launches = kernels
 *   launched by its iterations so far.
 * fblisa_batch_last_batch -- fblisa_last_batch of volume v.
 */
typedef struct fbl_batch fbl_batch;  /* opaque, library-owned */
FBL_API fbl_status fblisa_batch_create(const fbl_geometry *const *geoms, const fbl_params *params,
                                       int32_t n_vol, fbl_batch **out);
FBL_API void fblisa_batch_destroy(fbl_batch *bt);
FBL_API fbl_status fblisa_batch_set_proposal(fbl_batch *bt, const float *params, float margin,
                                             int32_t enable);
FBL_API fbl_status fblisa_batch_step(fbl_batch *bt, void *const *x, const void *const *b,
                                     fbl_step_stats *stats, void *stream);
FBL_API fbl_status fblisa_batch_run(fbl_batch *bt, void *const *x, const void *const *b,
                                    int32_t iterations, fbl_step_stats *trace, int64_t trace_cap,
                                    int64_t *n_steps, void *stream);
FBL_API fbl_status fblisa_batch_info(const fbl_batch *bt, int32_t *launch_cfg, int64_t *launches);
FBL_API fbl_status fblisa_batch_last_batch(const fbl_batch *bt, int32_t v, int32_t *views, int32_t cap,
                                           int32_t *n);

/* Message of the last failed call on this thread ("" if none). */
FBL_API const char *fbl_last_error(void);

/*
 * Host-only helpers (no device needed).
 * fbl_schedule -- Step 1 of Algorithm 1 for t = 1..epochs:
 *   N_t = min{n_max, max{ceil(C / eps_{k_hat + ceil(n/N_{t-1})}), N_0}},
 *   eps_k = eps_base^k, N_{t-1} = N_0 at t = 1, iters_t = ceil(n/N_t).
 * fbl_epoch_batches -- the mini-batches of epoch t (Step 2a): a Fisher-Yates
 *   permutation of 0..n_theta-1 from SplitMix64 (seed XOR t*0xD1B54A32D192ED03;
 *   draw i swaps entry i with i + floor(u_i (n-i)), u_i = top 53 bits), cut
 *   into slices of N_t; a short last slice is padded from the front of the
 *   permutation.  views_out holds ceil(n_theta/N_t)*N_t entries.
 */
FBL_API fbl_status fbl_schedule(int32_t n_theta, int32_t N0, int32_t n_max, double C, double eps_base,
                        int32_t epochs, int32_t *N_out, int32_t *iters_out);
FBL_API fbl_status fbl_epoch_batches(uint64_t seed, int32_t epoch, int32_t n_theta, int32_t N_t,
                             int32_t *views_out);

#ifdef __cplusplus
}
#endif

#endif /* FBLISA_H */
