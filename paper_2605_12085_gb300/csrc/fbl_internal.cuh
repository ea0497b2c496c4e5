// Internal declarations shared by the C-ABI layer and the sm_103a kernels of
// the FB-LISA hot path.  Nothing here is exported.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fblisa.h"

namespace fbl {

// ---------------------------------------------------------------------------
// Storage types.  Arithmetic is always FP32 (FP64 for the line-search sums).
// ---------------------------------------------------------------------------
__host__ __device__ inline int dtype_size(int dt) { return dt == FBL_F32 ? 4 : 2; }

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }

template <typename T> __device__ __forceinline__ T from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }

// Read-only load through the non-coherent path, converted to FP32.
template <typename T> __device__ __forceinline__ float ldg_f32(const T *p) { return to_f32(__ldg(p)); }

// ---------------------------------------------------------------------------
// Volume layout used inside the library (z innermost, zero border).
//
//     V[j + 1][i + 1][k + PL]   (j in [-1, ny], i in [-1, nx], k in [-PL, pitch-PL))
//
// Everything outside the volume (i or j at -1 or n, k < 0, k >= nz) is zero.
// A ray of family f crosses the planes m of its dominant axis (m = i for
// x-planes, m = j for y-planes) and moves in-plane along the other horizontal
// axis b and along z; both families read this one copy, with the plane and
// in-plane strides swapped.  The detector rows of one column (a warp of K1)
// sample consecutive k.  A bilinear footprint with -1 < q_b < Nb and
// -1 < q_z < nz reads in bounds and sees the zero boundary without a branch.
// PL = 16 bytes of elements (at least 2) keeps each row's interior 16-byte
// aligned; pitch is a multiple of PL with at least two zeros after the last
// element, so a bilinear footprint whose z row is clamped to [-2, nz] reads
// only zeros outside the volume.
// The gradient uses the unpadded z-innermost order [j][i][k].
// ---------------------------------------------------------------------------
struct ZLayout {
    int nx, ny, nz;
    int PL;      // left pad along k, elements
    int pitch;   // row length, elements
    __host__ __device__ int64_t elems() const { return (int64_t)(ny + 2) * (nx + 2) * pitch; }
    __host__ __device__ int64_t index(int i, int j, int k) const {
        return ((int64_t)(j + 1) * (nx + 2) + (i + 1)) * pitch + k + PL;
    }
    // strides of a family: y-planes (plane j, in-plane i) or x-planes (plane i, in-plane j)
    __host__ __device__ int plane_stride(bool famY) const { return famY ? (nx + 2) * pitch : pitch; }
    __host__ __device__ int inplane_stride(bool famY) const { return famY ? pitch : (nx + 2) * pitch; }
};

inline ZLayout make_layout(int nx, int ny, int nz, int esize) {
    ZLayout L;
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    L.PL = 16 / esize;
    const int need = L.PL + nz + 2;
    L.pitch = (need + L.PL - 1) / L.PL * L.PL;
    return L;
}

// Transposed residual / weighted sinogram: rt[s][iu][RT_PAD + iv], rows of
// nv + 2*RT_PAD floats whose RT_PAD leading and trailing entries are zero.
constexpr int RT_PAD = 8;
__host__ __device__ inline int rt_pitch(int nv) { return nv + 2 * RT_PAD; }

// ---------------------------------------------------------------------------
// Geometry tables on the device.
//
// For view v and detector column iu (all rays of a column share the
// horizontal direction because e_v is vertical) the host computes in FP64:
//   fam   family: 0 if |d_x| >= |d_y| (x-planes), else 1 (y-planes)
//   qb0, qb1  q_b(m) = qb0 + m*qb1, continuous in-plane index at plane m
//   zc0, zc1  Zc(m) = zc0 + m*zc1 = t(m)/vz, so q_z = w*Zc(m) + cz with
//             w = (iv - cv)*dv the vertical pixel offset
//   wa, h2    row weight v_a*|d|/|d_a| = wa*sqrt(h2 + w^2)
// ---------------------------------------------------------------------------
// Crossing positions are exact fixed-point numbers with FX_BITS fractional
// bits held in int64 (Q.40): stepping from plane to plane adds an integer, so
// every crossing equals its closed form exactly, K1 and K2 compute the same
// positions, and the bilinear weights carry full FP32 precision whatever the
// volume size (an FP32 coordinate near 512 would only resolve 3e-5 voxel).
constexpr int FX_BITS = 40;
constexpr double FX_ONE = 1099511627776.0;  // 2^40

__host__ __device__ __forceinline__ int fx_floor(long long q) { return (int)(q >> FX_BITS); }
// Fractional part in [0, 1) to 23 bits, as an FP32 number.
__device__ __forceinline__ float fx_frac(long long q) {
    const unsigned bits = (unsigned)((unsigned long long)q >> (FX_BITS - 23)) & 0x7FFFFFu;
    return __uint_as_float(bits | 0x3F800000u) - 1.0f;
}

// The projector's per-sample vertical crossing steps in Q.32: one ray's
// Q.40 start and step rounded once to 32 fractional bits (so the position
// after j planes is within (1 + j) 2^-33 voxel of the Q.40 one), whose
// integer part is the high word and whose fraction is one funnel shift.
__host__ __device__ __forceinline__ long long fx40_to_32(long long q) { return (q + (1LL << 7)) >> 8; }
__device__ __forceinline__ int fx32_floor(long long q) { return (int)(q >> 32); }
__device__ __forceinline__ float fx32_frac(long long q) {
    // the low word's top 23 bits as the mantissa of a number in [1, 2)
    return __uint_as_float(__funnelshift_r((unsigned)(unsigned long long)q, 0x7Fu, 9)) - 1.0f;
}

// Fixed-point column constants: q_b(m) = qb0 + m*qb1 and, for the detector
// row iv with n = 2*iv - (nv-1) (so that w = n*dv/2),
// q_z(m) = n*(h0 + m*h1) + cz, all in Q.40.
struct FxCol {
    long long qb0, qb1, h0, h1;
};

struct DevGeom {
    int nx, ny, nz, nu, nv, n_views;
    float cu, cv, du, dv;        // detector centre (index units) and pixel size
    float cx, cy, cz;            // volume centre in index units
    float vx, vy, vz;            // voxel size
    float sod, sdd, inv_du;
    float hwu;                   // half width, in columns, of a voxel's column footprint
    int ntap;                    // detector rows that can touch one voxel in one column
    // launch configuration (chosen by the autotuner; defaults 8 / 1 / 4)
    int k1_cols;                 // projector: detector columns per block (4 or 8)
    int k1_split;                // projector plane loop: 0 plain, 1 loads one sample ahead, 2 TMA-staged bricks
    int k2_vpl;                  // backprojector: consecutive voxels per lane (2, 4, 8 or 16)
    long long cz_fx;             // cz in Q.40
    const float4 *colA;          // [n_views][nu] (qb0, qb1, zc0, zc1) in FP32, for range estimates
    const FxCol *colF;           // [n_views][nu] exact fixed-point constants
    const float4 *colB;          // [n_views][nu] (wa, h2, fam, 0)
    const float2 *trig;          // [n_views] (cos, sin)
    int *err;                    // device status word: FBL_E_TIMEOUT after a bounded wait gave up
};

enum ProjMode { PROJ_STORE = 0, PROJ_RESID = 1, PROJ_NORM = 2 };

// Kernel launchers (each returns the launch error, if any).

// Natural [nz][ny][nx] volume -> the library layout (interior only).
cudaError_t launch_pack(const void *x, int x_dtype, void *vol, ZLayout L, cudaStream_t st);
// Library layout -> natural [nz][ny][nx] (same dtype).
cudaError_t launch_unpack(const void *vol, ZLayout L, int dtype, void *x, cudaStream_t st);
// Gradient order [j][i][k] (float) -> natural [nz][ny][nx] float, = or +=.
cudaError_t launch_zi_to_natural(const float *gzi, float *x, int nx, int ny, int nz, int accumulate,
                                 cudaStream_t st);

// mode STORE: out[s][iv][iu] = A_{views[s]} x  (out_dtype)
// mode RESID: out = rt[s][iu][RT_PAD + iv] = W * (A x - b) as float32, partials += r^2
// mode NORM:  partials += (A x - b)^2 only
// b_views: device list mapping slot s to the view index inside b (NULL: b is
// already the batch, slot s at index s).  b is [view][nv][nu].
cudaError_t launch_project(int mode, const DevGeom &g, const void *vol, ZLayout L, int x_dtype,
                           const int32_t *views,
                           int n_sel, const void *b, int b_dtype, const int32_t *b_views,
                           void *out, int out_dtype, double *partials, int *n_partials,
                           cudaStream_t st);
int project_num_partials(const DevGeom &g, int n_sel);

// rt[s][iu][RT_PAD + iv] = W(ray) * y[s][iv][iu] (the row weight folded in for K2);
// the pad entries are left untouched (the caller zeroes them once).
cudaError_t launch_weight(const DevGeom &g, const void *y, int y_dtype, const int32_t *views,
                          int n_sel, float *rt, cudaStream_t st);

// gzi[j][i][k] = scale * sum over listed views of the transpose taps of rt;
// with g2_partials, also the per-block sums of gzi^2 (backproject_num_partials).
cudaError_t launch_backproject(const DevGeom &g, const float *rt, const int32_t *views,
                               int n_sel, float scale, float *gzi, cudaStream_t st,
                               double *g2_partials = nullptr);
int backproject_num_partials(const DevGeom &g);

// x_bar = min(max(x - alpha*g - alpha*mu, 0), xmax) on the solver's state:
// reads vol (current x) and gzi, writes trial; partials[3][nblk] =
// (g^T d, d^T d, |x_bar|_1) per block.
cudaError_t launch_prox_zi(const void *vol, ZLayout L, const float *gzi, float alpha, float amu, float xmax,
                           void *trial, int dtype, double *partials, int *n_partials,
                           cudaStream_t st);
int prox_zi_num_partials(int nx, int ny, int nz);

// Total variation (k_tv.cu).  Volumes in a memory order (n0 fastest, n1, n2),
// dual fields as 3 such volumes; the dual pair (q, r) alternates between
// (q[0], r[0]) and (q[1], r[1]), *cur naming the pair in use.  tv_prox:
// x = prox of lam TV + indicator of [0, xmax] at v by `iters` FGP iterations
// from q_start (NULL: zero), written to pair *cur first; *cur ends at the pair
// holding the last dual; y is scratch (1 volume).
bool tv_dims_ok(int n0, int n1, int n2);
cudaError_t launch_tv_prox(const float *v, int n0, int n1, int n2, float lam, float xmax, int iters,
                           const float *q_start, float *const q[2], float *const r[2], float *y, float *x, int *cur,
                           cudaStream_t st);
int tv_norm_num_partials(int n0, int n1, int n2);
cudaError_t launch_tv_norm(const float *x, int n0, int n1, int n2, double *partials, cudaStream_t st);
// The solver's TV trial point: b = x - alpha g ([j][i][k]), FGP from the
// dual in pair *cur (warm) or zero, started in the other pair, then
// x_bar = P_C(b - lam K^T q) into trial with the three partial sums of
// launch_prox_zi (same block count); *cur ends at the last dual's pair.
cudaError_t launch_tv_prox_zi(const void *vol, ZLayout L, const float *gzi, float alpha, float lam, float xmax,
                              int iters, int warm, float *b, float *const q[2], float *const r[2], int *cur,
                              float *y, void *trial, int dtype, double *partials, int *n_partials, cudaStream_t st);

// Flat prox on n elements (public prox_reduce).
cudaError_t launch_prox_flat(const void *x, const float *gr, int64_t n, float alpha, float amu,
                             void *xbar, int dtype, double *partials, int *n_partials,
                             cudaStream_t st);
int prox_flat_num_partials(int64_t n);

// The flat prox kernel on an explicit grid of nb blocks (256 threads each):
// partials[3][nb] receives the per-block sums.
cudaError_t launch_prox_flat_grid(const void *x, const float *gr, int64_t n, float alpha, float amu,
                                  void *xbar, int dtype, int nb, double *partials,
                                  cudaStream_t st);

// partials[3][nb]: sum |x|, sum (x - xr)^2, sum xr^2 (xr may be NULL).
cudaError_t launch_norms(const void *x, const void *xr, int dtype, int64_t n, double *partials,
                         int *n_partials, cudaStream_t st);

// The step-proposal network (k_mlp.cu): 8 -> 64 -> 64 -> 1, tanh, FP32.
constexpr int MLP_IN = 8;
constexpr int MLP_HIDDEN = 64;
constexpr int MLP_PARAMS = MLP_HIDDEN * MLP_IN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN +
                           MLP_HIDDEN + 1;  // 4801
constexpr int MLP_PARAMS_PAD = (MLP_PARAMS + 3) / 4 * 4;
size_t mlp_train_smem();
cudaError_t launch_mlp_forward(const float *params, const float *X, int n, float *y, cudaStream_t st);
// mode 0: full-batch gradient and loss; mode 1: Adam epochs over minibatches.
cudaError_t launch_mlp_train(float *params, float *adam_m, float *adam_v, const float *X,
                             const float *T, int n, int batch, int epochs, float lr, int mode,
                             float *grad_out, double *loss_out, int *step_io, cudaStream_t st);

// Line-search state of one iteration (device memory).
struct LSState {
    double alpha_init, alpha, beta, mu, scale;  // scale = n_theta / N_t
    double x_max;               // upper bound of the box in R (+inf: none)
    double rho0, gTd, dd, rho1, f_x, f_xbar, rhs, g2;
    int trials, max_backtracks, accepted, status, force_reject;
    int j_start;                // first trial = alpha0 * beta^j_start
    int N_t, n_theta;
    float pred;                 // network output (backtracks predicted)
    float feat[MLP_IN];         // the proposal's input features
};

// Statistics carried from one accepted iteration to the next (device memory).
struct PropState {
    double f_prev, g2_prev;
    long long k;
    int j_prev, have_prev, dj_prev, have_dj;
};

// Features of this iteration from sc[0] = rho0 and sc[5] = ||grad f_N||^2,
// then (params != NULL) the network's prediction and the first trial step
// alpha0 * beta^j; without params the first trial is alpha0 (Step 2d).
cudaError_t launch_propose(LSState *ls, const PropState *ps, const double *sc, const float *params,
                           float margin, cudaStream_t st);
cudaError_t launch_ls_init(LSState *ls, cudaStream_t st);
// Evaluate (2.3) on sc = [rho0, gTd, dd, l1, rho1]; accept (and record the
// iteration in ps), or shrink the step and request another trial (the WHILE
// condition), or stop with a status.
cudaError_t launch_ls_decide(LSState *ls, PropState *ps, const double *sc,
                             cudaGraphConditionalHandle cond, cudaStream_t st);
// launch_prox_zi with alpha and mu read from the line-search state.
cudaError_t launch_prox_zi_dev(const void *vol, ZLayout L, const float *gzi, const LSState *ls,
                               void *trial, int dtype, double *partials, int *n_partials,
                               cudaStream_t st);

// ---------------------------------------------------------------------------
// Batched iteration over several volumes (persistent launches).
//
// One FB-LISA iteration of every volume of a batch runs as one launch per
// phase: each phase's work is a list of tiles (the single-volume kernel's
// blocks, per volume), volumes laid out largest first; a grid sized to fill
// the GPU takes tiles from an atomic counter until none is left (no waits).
// Everything that changes between iterations -- the iterate / trial buffers
// (swapped on acceptance by the decision kernel), the view lists, N_t and the
// tile counts -- lives in the device descriptors below, so one captured graph
// serves every iteration.

// One volume of the batch (device memory; the host rewrites it each iteration).
struct BatchVol {
    DevGeom g;
    ZLayout L;
    void *x_cur, *x_trial;        // current iterate and trial point (library layout)
    const void *b;                // data: [n_views][nv][nu] (b_views != NULL) or the batch's views
    const int32_t *b_views;       // slot s -> view index inside b, or NULL
    const int32_t *views;         // this iteration's views (N_t)
    float *rt;                    // weighted residual rt[s][iu][RT_PAD + iv]
    float *grad;                  // gradient [j][i][k]
    double *partials;             // per-tile partial sums
    double *sc;                   // [8] scalars (rho0, gTd, dd, l1, rho1, g2)
    LSState *ls;                  // line-search state
    PropState *ps;                // proposal statistics (persistent)
    float scale;                  // n_theta / N_t
    int N_t;
    int proposal;                 // 1: learned first trial, 0: alpha_0
    int tiles[3];                 // K1, K2, K3 tiles of this volume this iteration
    int first[3];                 // first tile index of this volume in each phase
    int rfirst[2];                // this trial round: first K1 / K3 tile (searching volumes only)
};

struct BatchHdr {
    int n_vol;
    int total[3];                 // K1, K2, K3 tiles over all volumes
    int rtotal[2];                // this trial round: K1 / K3 tiles of the searching volumes
};

// Index of the volume that owns tile t, given each volume's first tile
// (non-decreasing over the array; a volume without tiles this time repeats
// its successor's first index, so the last volume with first <= t owns t).
template <class F>
__device__ __forceinline__ int batch_find_by(int n_vol, int t, F first) {
    int lo = 0, hi = n_vol - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first(mid) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int batch_find(const BatchHdr &h, const BatchVol *v, int ph, int t) {
    return batch_find_by(h.n_vol, t, [&](int q) { return v[q].first[ph]; });
}
// Trial rounds: r = 0 for the objective projection (K1), 1 for the prox (K3).
__device__ __forceinline__ int batch_find_round(const BatchHdr &h, const BatchVol *v, int r, int t) {
    return batch_find_by(h.n_vol, t, [&](int q) { return v[q].rfirst[r]; });
}

// Copy bytes (a multiple of 4, 4-byte aligned) from global to shared memory
// with nthreads threads; the caller synchronises the block afterwards.
__device__ __forceinline__ void stage_words(void *dst, const void *src, size_t bytes, int tid,
                                            int nthreads) {
    const int n = (int)(bytes / 4);
    for (int q = tid; q < n; q += nthreads) ((int *)dst)[q] = ((const int *)src)[q];
}

// A volume still inside its line search (neither accepted nor stopped).
__device__ __forceinline__ bool batch_searching(const LSState &ls) {
    return ls.accepted == 0 && ls.status == 0;
}

// ctr: two ints per launch site, zero before the launch and left zero after it.
// mode RESID reads x_cur and writes rt; mode NORM reads x_trial of the volumes
// still searching.  cols: detector columns per block, common to the batch;
// each volume keeps its own plane-loop form (g.k1_split).
cudaError_t launch_batch_project(int mode, const BatchHdr *hdr, BatchVol *vols, int x_dtype,
                                 int b_dtype, int cols, int *ctr, cudaStream_t st);
// Gradient of every volume (scale and views from the descriptor), with the
// per-tile sums of the squared gradient; each volume keeps its own voxels per
// lane (g.k2_vpl); ntap >= every volume's g.ntap.
cudaError_t launch_batch_backproject(const BatchHdr *hdr, BatchVol *vols, int ntap, int *ctr,
                                     cudaStream_t st);
// Prox + (2.3) sums of the volumes still searching, alpha from their state.
cudaError_t launch_batch_prox(const BatchHdr *hdr, BatchVol *vols, int x_dtype, int *ctr,
                              cudaStream_t st);
// sc[slot + c] of every volume (or only those still searching) = the fixed-order
// sum of its partials[c * tiles + 0 .. tiles) of phase ph, c < ncomp.
cudaError_t launch_batch_reduce(const BatchHdr *hdr, BatchVol *vols, int n_vol, int ph, int ncomp,
                                int slot, int searching_only, cudaStream_t st);
cudaError_t launch_batch_propose(BatchVol *vols, int n_vol, const float *params, float margin,
                                 cudaStream_t st);
// Line-search init of every volume, and the first trial round's tile offsets.
cudaError_t launch_batch_ls_init(BatchHdr *hdr, BatchVol *vols, int n_vol, cudaStream_t st);
// (2.3) for every volume still searching; on acceptance the volume's x_cur and
// x_trial are swapped; the next round's tile offsets cover the volumes still
// searching, and the WHILE condition is set while any volume searches.
cudaError_t launch_batch_decide(BatchHdr *hdr, BatchVol *vols, int n_vol,
                                cudaGraphConditionalHandle cond, cudaStream_t st);

// FDK (k_fdk.cu): weighted, ramp-filtered projections of n_sel views written
// transposed with a zero border, qt[s][iu + 1][iv + 1] (rows of nv + 2);
// then the weighted backprojection of them into gzi[j][i][k] (= or +=).
// view_csw: n_sel x (cos, sin, dtheta / 2) in FP64.
size_t fdk_filtered_elems(int n_sel, int nu, int nv);
cudaError_t launch_fdk_filter(const void *y, int y_dtype, int n_sel, int nu, int nv, double sod, double sdd,
                              double du, double dv, float *qt, cudaStream_t st);
cudaError_t launch_fdk_bp(const float *qt, const double *view_csw, int n_sel, int nx, int ny, int nz, int nu,
                          int nv, double vx, double vy, double vz, double sod, double sdd, double du, double dv,
                          int accumulate, float *gzi, cudaStream_t st);

// Record the message returned by fbl_last_error() on this thread.
void set_last_error(const char *msg);

// out[c] = sum of partials[c*stride + 0 .. n) in a fixed order, for c < ncomp.
cudaError_t launch_reduce(const double *partials, int n, int stride, int ncomp, double *out,
                          cudaStream_t st);

}  // namespace fbl
