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
__global__ void k_propose(LSState *ls, const PropState *ps, const double *sc, const float *params,
                          float margin) {
    __shared__ float x[MLP_IN], h1[MLP_HIDDEN];
    const int lane = threadIdx.x;
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

// sc: [rho0, gTd, dd, l1, rho1] as reduced by the preceding kernels.
__global__ void k_ls_decide(LSState *ls, PropState *ps, const double *sc,
                            cudaGraphConditionalHandle cond) {
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
    cudaGraphSetConditional(cond, more);
}

// Prox + reductions with the step taken from the line-search state.
constexpr int PZ_TX = 64;
constexpr int PZ_TY = 4;

template <typename T>
__global__ void __launch_bounds__(PZ_TX *PZ_TY) k_prox_zi_dev(const T *__restrict__ vol, ZLayout L,
                                                              const float *__restrict__ gzi,
                                                              const LSState *ls, T *__restrict__ trial,
                                                              double *__restrict__ partials) {
    const double a = ls->alpha;
    const float alpha = (float)a, amu = (float)(a * ls->mu);
    const int row = blockIdx.x * PZ_TY + threadIdx.y;
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
            const float xb = fmaxf(fmaf(-alpha, gg, x) - amu, 0.f);
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
        const size_t nblk = gridDim.x;
        partials[blockIdx.x] = out[0];
        partials[nblk + blockIdx.x] = out[1];
        partials[2 * nblk + blockIdx.x] = out[2];
    }
}

}  // namespace

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
