// Device-side control of the backtracking line search (Algorithm 1, Step 2c)
// for the graph-captured iteration: the prox kernel reads the trial step from
// device memory, and after each trial a one-thread kernel evaluates the
// sufficient-decrease test (2.3) in FP64 and sets the condition of the
// graph's WHILE node.  The arithmetic is the host loop's, operation by
// operation, with explicitly rounded FP64 intrinsics (no contraction into
// FMA), so both modes take identical decisions.
#include <math.h>

#include "fbl_internal.cuh"
#include "fbl_reduce.cuh"

namespace fbl {
namespace {

__global__ void k_ls_init(LSState *ls) {
    ls->alpha = ls->alpha_init;
    ls->trials = 0;
    ls->accepted = 0;
    ls->status = FBL_OK;
}

// Input features of the step proposal, from this iteration's f = f_N(x) and
// g2 = ||grad f_N(x)||^2 and the previous accepted iterations.  With the
// curvature index c = log2(alpha_0 g2 / (2 f)) (g2 / (2 f) <= L), only relative
// quantities enter once there is a previous iteration, so that a network
// trained on small volumes transfers to large ones:
//   0: c/10 at the first iteration (0 afterwards), 1: log(f / f_prev),
//   2: log(|g| / |g_prev|), 3: (c - c_prev)/10, 4: N_t / n_theta,
//   5: log(1 + k)/10, 6: 1 if there is a previous iteration,
//   7: (j_prev - j_prevprev)/4, the last change of the accepted grid index.
__device__ void proposal_features(const LSState &ls, const PropState &ps, double f, double g2,
                                  float *feat) {
    const bool have = ps.have_prev != 0;
    const double c = log2(fmax(ls.alpha_init * g2 / fmax(2.0 * f, 1e-300), 1e-300));
    const double c_prev = log2(fmax(ls.alpha_init * ps.g2_prev / fmax(2.0 * ps.f_prev, 1e-300), 1e-300));
    feat[0] = have ? 0.f : (float)(0.1 * c);
    feat[1] = have ? (float)log(fmax(f, 1e-300) / fmax(ps.f_prev, 1e-300)) : 0.f;
    feat[2] = have ? (float)(0.5 * log(fmax(g2, 1e-300) / fmax(ps.g2_prev, 1e-300))) : 0.f;
    feat[3] = have ? (float)(0.1 * (c - c_prev)) : 0.f;
    feat[4] = (float)ls.N_t / (float)ls.n_theta;
    feat[5] = (float)(0.1 * log(1.0 + (double)ps.k));
    feat[6] = have ? 1.f : 0.f;
    feat[7] = ps.have_dj ? 0.25f * (float)ps.dj_prev : 0.f;
}

// One warp: features, the network (hidden units l and l+32 per lane), the
// first trial step.  ls->alpha_init holds alpha_0 on entry.
__device__ __forceinline__ void propose_warp(LSState *ls, const PropState *ps, const double *sc,
                                             const float *params, float margin) {
    __shared__ float x[MLP_IN], h1[MLP_HIDDEN];
    const int lane = threadIdx.x & 31;
    const double rho0 = sc[0], g2 = sc[5];
    const double f = __dmul_rn(__dmul_rn(0.5, ls->scale), rho0);
    if (lane == 0) proposal_features(*ls, *ps, f, g2, x);
    __syncwarp();
    float pred = 0.f;
    if (params) {
        constexpr int NI = MLP_IN, NH = MLP_HIDDEN;
        constexpr int OB1 = NH * NI, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH;
        float z[2];
        for (int h = 0; h < 2; ++h) {
            const int u = lane + 32 * h;
            float a = params[OB1 + u];
            for (int q = 0; q < NI; ++q) a = fmaf(params[u * NI + q], x[q], a);
            z[h] = tanhf(a);
        }
        h1[lane] = z[0];
        h1[lane + 32] = z[1];
        __syncwarp();
        float part = 0.f;
        for (int h = 0; h < 2; ++h) {
            const int u = lane + 32 * h;
            float a = params[OB2 + u];
            for (int v = 0; v < NH; ++v) a = fmaf(params[OW2 + u * NH + v], h1[v], a);
            part = fmaf(params[OW3 + u], tanhf(a), part);
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        pred = part + params[OB3];
    }
    if (lane == 0) {
        // the network predicts the change of the grid index from the previous
        // accepted one; rounding down (margin) prefers one extra trial to a
        // halved step
        int j = 0;
        if (params && isfinite(pred)) {
            const float base = ps->have_prev ? (float)ps->j_prev : 0.f;
            j = min(max((int)floorf(base + pred + 0.5f - margin), 0), ls->max_backtracks);
        }
        double a = ls->alpha_init;
        for (int q = 0; q < j; ++q) a = __dmul_rn(a, ls->beta);  // the plain rule's step grid
        ls->alpha_init = a;
        ls->j_start = j;
        ls->pred = pred;
        ls->g2 = g2;
        for (int q = 0; q < MLP_IN; ++q) ls->feat[q] = x[q];
    }
}

__global__ void k_propose(LSState *ls, const PropState *ps, const double *sc, const float *params,
                          float margin) {
    propose_warp(ls, ps, sc, params, margin);
}

// One block of 32 threads per volume of a batch.
__global__ void kb_propose(const BatchVol *vols, const float *params, float margin) {
    const BatchVol &bv = vols[blockIdx.x];
    propose_warp(bv.ls, bv.ps, bv.sc, bv.proposal ? params : nullptr, margin);
}

// Tile offsets of the next trial round over the volumes still searching
// (thread 0, after the block has updated every volume's state).
__device__ void batch_round_offsets(BatchHdr *hdr, BatchVol *vols, int n_vol) {
    int acc[2] = {0, 0};
    for (int v = 0; v < n_vol; ++v) {
        BatchVol &bv = vols[v];
        const bool on = batch_searching(*bv.ls);
        bv.rfirst[0] = acc[0];
        bv.rfirst[1] = acc[1];
        if (on) {
            acc[0] += bv.tiles[0];
            acc[1] += bv.tiles[2];
        }
    }
    hdr->rtotal[0] = acc[0];
    hdr->rtotal[1] = acc[1];
}

// One block, one thread per volume.
__global__ void kb_ls_init(BatchHdr *hdr, BatchVol *vols, int n_vol) {
    const int v = threadIdx.x;
    if (v < n_vol) {
        LSState *ls = vols[v].ls;
        ls->alpha = ls->alpha_init;
        ls->trials = 0;
        ls->accepted = 0;
        ls->status = FBL_OK;
    }
    __syncthreads();
    if (threadIdx.x == 0) batch_round_offsets(hdr, vols, n_vol);
}

// sc: [rho0, gTd, dd, l1, rho1] as reduced by the preceding kernels.  Returns
// 1 when another trial is needed.
__device__ __forceinline__ unsigned int ls_decide_one(LSState *ls, PropState *ps, const double *sc) {
    const double rho0 = sc[0], gTd = sc[1], dd = sc[2], rho1 = sc[4];
    const double alpha = ls->alpha;
    const double half_scale = __dmul_rn(0.5, ls->scale);
    const double f_x = __dmul_rn(half_scale, rho0);
    const double f_xb = __dmul_rn(half_scale, rho1);
    const double rhs = __dadd_rn(__dadd_rn(f_x, gTd), __ddiv_rn(dd, __dmul_rn(2.0, alpha)));
    ls->rho0 = rho0;
    ls->gTd = gTd;
    ls->dd = dd;
    ls->rho1 = rho1;
    ls->f_x = f_x;
    ls->f_xbar = f_xb;
    ls->rhs = rhs;
    unsigned int more = 0;
    if (!isfinite(f_x) || !isfinite(f_xb) || !isfinite(rhs)) {
        ls->status = FBL_E_NONFINITE;
    } else if (!ls->force_reject && f_xb <= rhs) {
        ls->accepted = 1;
        ps->f_prev = f_x;
        ps->g2_prev = ls->g2;
        const int j_acc = ls->j_start + ls->trials;
        ps->dj_prev = j_acc - ps->j_prev;
        ps->have_dj = ps->have_prev;
        ps->j_prev = j_acc;
        ps->have_prev = 1;
        ps->k += 1;
    } else if (ls->trials >= ls->max_backtracks) {
        ls->status = FBL_E_LINESEARCH;
    } else {
        ls->trials += 1;
        ls->alpha = __dmul_rn(alpha, ls->beta);
        more = 1;
    }
    return more;
}

__global__ void k_ls_decide(LSState *ls, PropState *ps, const double *sc,
                            cudaGraphConditionalHandle cond) {
    cudaGraphSetConditional(cond, ls_decide_one(ls, ps, sc));
}

// One thread per volume of a batch (a single block): (2.3) for the volumes
// still searching; an accepted volume's trial point becomes its iterate.
__global__ void kb_decide(BatchHdr *hdr, BatchVol *vols, int n_vol, cudaGraphConditionalHandle cond) {
    const int v = threadIdx.x;
    unsigned int more = 0;
    if (v < n_vol) {
        BatchVol &bv = vols[v];
        if (batch_searching(*bv.ls)) {
            more = ls_decide_one(bv.ls, bv.ps, bv.sc);
            if (bv.ls->accepted) {
                void *t = bv.x_cur;
                bv.x_cur = bv.x_trial;
                bv.x_trial = t;
            }
        }
    }
    const int any = __syncthreads_or(more);
    if (threadIdx.x == 0) {
        batch_round_offsets(hdr, vols, n_vol);
        cudaGraphSetConditional(cond, any ? 1u : 0u);
    }
}

// Prox + reductions with the step taken from the line-search state.
constexpr int PZ_TX = 64;
constexpr int PZ_TY = 4;

// One block's rows (PZ_TY (i, j) columns from blk * PZ_TY) of the prox, with
// its three sums written to partials[c * nblk + blk].  Called by every thread.
template <typename T>
__device__ __forceinline__ void prox_tile(const T *__restrict__ vol, const ZLayout &L,
                                          const float *__restrict__ gzi, const LSState *ls,
                                          T *__restrict__ trial, double *__restrict__ partials,
                                          int blk, int nblk) {
    const double a = ls->alpha;
    const float alpha = (float)a, amu = (float)(a * ls->mu), xmax = (float)ls->x_max;
    const int row = blk * PZ_TY + threadIdx.y;
    float sums[3] = {0.f, 0.f, 0.f};
    if (row < L.nx * L.ny) {
        const int j = row / L.nx, i = row - j * L.nx;
        const int64_t base = L.index(i, j, 0);
        const T *src = vol + base;
        T *dst = trial + base;
        const float *gr = gzi + (size_t)row * L.nz;
        for (int k = threadIdx.x; k < L.nz; k += PZ_TX) {
            const float x = to_f32(src[k]);
            const float gg = gr[k];
            const float xb = fminf(fmaxf(fmaf(-alpha, gg, x) - amu, 0.f), xmax);
            const T xs = from_f32<T>(xb);
            const float xr = to_f32(xs);
            dst[k] = xs;
            const float d = xr - x;
            sums[0] = fmaf(gg, d, sums[0]);
            sums[1] = fmaf(d, d, sums[1]);
            sums[2] += xr;
        }
    }
    double out[3];
    block_sum_f64<PZ_TX * PZ_TY, 3>(sums, out);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        partials[blk] = out[0];
        partials[(size_t)nblk + blk] = out[1];
        partials[2 * (size_t)nblk + blk] = out[2];
    }
}

template <typename T>
__global__ void __launch_bounds__(PZ_TX *PZ_TY) k_prox_zi_dev(const T *__restrict__ vol, ZLayout L,
                                                              const float *__restrict__ gzi,
                                                              const LSState *ls, T *__restrict__ trial,
                                                              double *__restrict__ partials) {
    prox_tile<T>(vol, L, gzi, ls, trial, partials, blockIdx.x, gridDim.x);
}

// Persistent batched prox over the volumes still searching.
template <typename T>
__global__ void __launch_bounds__(PZ_TX *PZ_TY) kb_prox(const BatchHdr *hdr, const BatchVol *vols,
                                                        int *ctr) {
    __shared__ int s_tile;
    const int tid = threadIdx.x + PZ_TX * threadIdx.y;
    const int total = hdr->rtotal[1];
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(ctr, 1);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= total) break;
        const BatchVol &bv = vols[batch_find_round(*hdr, vols, 1, t)];
        const int local = t - bv.rfirst[1];
        prox_tile<T>((const T *)bv.x_cur, bv.L, bv.grad, bv.ls, (T *)bv.x_trial, bv.partials, local,
                     bv.tiles[2]);
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(ctr + 1, 1) == (int)gridDim.x - 1) {
            ctr[0] = 0;
            ctr[1] = 0;
            __threadfence();
        }
    }
}

}  // namespace

cudaError_t launch_batch_propose(BatchVol *vols, int n_vol, const float *params, float margin,
                                 cudaStream_t st) {
    kb_propose<<<n_vol, 32, 0, st>>>(vols, params, margin);
    return cudaGetLastError();
}

cudaError_t launch_batch_ls_init(BatchHdr *hdr, BatchVol *vols, int n_vol, cudaStream_t st) {
    if (n_vol < 1 || n_vol > 1024) return cudaErrorInvalidValue;
    kb_ls_init<<<1, (n_vol + 31) / 32 * 32, 0, st>>>(hdr, vols, n_vol);
    return cudaGetLastError();
}

cudaError_t launch_batch_decide(BatchHdr *hdr, BatchVol *vols, int n_vol, cudaGraphConditionalHandle cond,
                                cudaStream_t st) {
    if (n_vol < 1 || n_vol > 1024) return cudaErrorInvalidValue;
    kb_decide<<<1, (n_vol + 31) / 32 * 32, 0, st>>>(hdr, vols, n_vol, cond);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_kb_prox(const BatchHdr *hdr, BatchVol *vols, int *ctr, cudaStream_t st) {
    static const int grid = [] {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_prox<T>, PZ_TX * PZ_TY, 0);
        return (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    }();
    kb_prox<T><<<grid, dim3(PZ_TX, PZ_TY), 0, st>>>(hdr, vols, ctr);
    return cudaGetLastError();
}

cudaError_t launch_batch_prox(const BatchHdr *hdr, BatchVol *vols, int x_dtype, int *ctr,
                              cudaStream_t st) {
    switch (x_dtype) {
        case FBL_BF16: return launch_kb_prox<__nv_bfloat16>(hdr, vols, ctr, st);
        case FBL_F16: return launch_kb_prox<__half>(hdr, vols, ctr, st);
        default: return launch_kb_prox<float>(hdr, vols, ctr, st);
    }
}

cudaError_t launch_ls_init(LSState *ls, cudaStream_t st) {
    k_ls_init<<<1, 1, 0, st>>>(ls);
    return cudaGetLastError();
}

cudaError_t launch_ls_decide(LSState *ls, PropState *ps, const double *sc,
                             cudaGraphConditionalHandle cond, cudaStream_t st) {
    k_ls_decide<<<1, 1, 0, st>>>(ls, ps, sc, cond);
    return cudaGetLastError();
}

cudaError_t launch_propose(LSState *ls, const PropState *ps, const double *sc, const float *params,
                           float margin, cudaStream_t st) {
    k_propose<<<1, 32, 0, st>>>(ls, ps, sc, params, margin);
    return cudaGetLastError();
}

cudaError_t launch_prox_zi_dev(const void *vol, ZLayout L, const float *gzi, const LSState *ls,
                               void *trial, int dtype, double *partials, int *n_partials,
                               cudaStream_t st) {
    const int nb = prox_zi_num_partials(L.nx, L.ny, L.nz);
    if (n_partials) *n_partials = nb;
    dim3 block(PZ_TX, PZ_TY);
    switch (dtype) {
        case FBL_BF16:
            k_prox_zi_dev<<<nb, block, 0, st>>>((const __nv_bfloat16 *)vol, L, gzi, ls,
                                                (__nv_bfloat16 *)trial, partials);
            break;
        case FBL_F16:
            k_prox_zi_dev<<<nb, block, 0, st>>>((const __half *)vol, L, gzi, ls, (__half *)trial,
                                                partials);
            break;
        default:
            k_prox_zi_dev<<<nb, block, 0, st>>>((const float *)vol, L, gzi, ls, (float *)trial,
                                                partials);
            break;
    }
    return cudaGetLastError();
}

}  // namespace fbl
