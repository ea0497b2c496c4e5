// The learned step proposal's network: a 3-layer perceptron
//     h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),  y = W3 . h2 + b3
// with 8 inputs, two hidden layers of 64 units and one output, FP32, and its
// hand-written inference, gradient and Adam training kernels.  Parameters
// are one contiguous float array: W1[64][8], b1[64], W2[64][64], b2[64],
// W3[64], b3[1] (4801 values).  The loss is 1/(2n) sum (y - t)^2.
//
// A warp evaluates one sample at a time with each lane owning hidden units
// l and l + 32; layer inputs are exchanged through a per-warp shared-memory
// row.  For training, each warp accumulates its samples' gradients into its
// own shared-memory copy of the parameter gradient (rows of W2 belong to one
// lane, so no atomics), the copies are added in warp order, and Adam updates
// the parameters -- all inside one block, one launch per call.
#include <math.h>

#include "fbl_internal.cuh"

namespace fbl {
namespace {

constexpr int NI = MLP_IN, NH = MLP_HIDDEN;
constexpr int OW1 = 0, OB1 = OW1 + NH * NI, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH;
static_assert(OB3 + 1 == MLP_PARAMS, "parameter layout");
constexpr int TW = 8;  // warps per training block

struct WarpScratch {
    float x[NI];
    float h1[NH];
    float h2[NH];
    float dz2[NH];
};

// Forward pass of one sample by one warp; returns y (valid in every lane) and
// leaves h1, h2 in the warp's scratch.
__device__ __forceinline__ float warp_forward(const float *__restrict__ P, WarpScratch &w, int lane) {
    float z[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int u = lane + 32 * h;
        float a = P[OB1 + u];
#pragma unroll
        for (int i = 0; i < NI; ++i) a = fmaf(P[OW1 + u * NI + i], w.x[i], a);
        z[h] = tanhf(a);
    }
    w.h1[lane] = z[0];
    w.h1[lane + 32] = z[1];
    __syncwarp();
    float part = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int u = lane + 32 * h;
        float a = P[OB2 + u];
        for (int v = 0; v < NH; ++v) a = fmaf(P[OW2 + u * NH + v], w.h1[v], a);
        const float t = tanhf(a);
        w.h2[u] = t;
        part = fmaf(P[OW3 + u], t, part);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    __syncwarp();
    return part + P[OB3];
}

// Backward pass of one sample (forward state in w), dy = dL/dy; adds the
// parameter gradient into G (this warp's copy).
__device__ __forceinline__ void warp_backward(const float *__restrict__ P, WarpScratch &w, int lane,
                                              float dy, float *__restrict__ G) {
    if (lane == 0) G[OB3] += dy;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int u = lane + 32 * h;
        const float h2 = w.h2[u];
        G[OW3 + u] += dy * h2;
        const float d2 = dy * P[OW3 + u] * (1.f - h2 * h2);
        w.dz2[u] = d2;
        G[OB2 + u] += d2;
        float *row = G + OW2 + u * NH;
        for (int v = 0; v < NH; ++v) row[v] = fmaf(d2, w.h1[v], row[v]);
    }
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int v = lane + 32 * h;
        float dh1 = 0.f;
        for (int u = 0; u < NH; ++u) dh1 = fmaf(P[OW2 + u * NH + v], w.dz2[u], dh1);
        const float h1 = w.h1[v];
        const float d1 = dh1 * (1.f - h1 * h1);
        G[OB1 + v] += d1;
#pragma unroll
        for (int i = 0; i < NI; ++i) G[OW1 + v * NI + i] += d1 * w.x[i];
    }
    __syncwarp();
}

__global__ void __launch_bounds__(256) k_mlp_forward(const float *__restrict__ params,
                                                     const float *__restrict__ X, int n,
                                                     float *__restrict__ y) {
    __shared__ float P[MLP_PARAMS];
    __shared__ WarpScratch ws[8];
    for (int q = threadIdx.x; q < MLP_PARAMS; q += blockDim.x) P[q] = params[q];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * 8 + warp, nw = gridDim.x * 8;
    for (int s = gw; s < n; s += nw) {
        if (lane < NI) ws[warp].x[lane] = X[(size_t)s * NI + lane];
        __syncwarp();
        const float out = warp_forward(P, ws[warp], lane);
        if (lane == 0) y[s] = out;
        __syncwarp();
    }
}

// One block.  mode 0: full-batch gradient of the loss over all n samples into
// grad_out (and the loss into loss_out); mode 1: `epochs` passes of Adam over
// minibatches of `batch` consecutive samples.
__global__ void __launch_bounds__(TW * 32) k_mlp_train(float *__restrict__ params,
                                                       float *__restrict__ adam_m,
                                                       float *__restrict__ adam_v,
                                                       const float *__restrict__ X,
                                                       const float *__restrict__ T, int n, int batch,
                                                       int epochs, float lr, int mode,
                                                       float *__restrict__ grad_out,
                                                       double *__restrict__ loss_out,
                                                       int *__restrict__ step_io) {
    extern __shared__ float smem[];
    float *P = smem;                       // parameters
    float *G = smem + MLP_PARAMS_PAD;      // TW gradient copies
    __shared__ WarpScratch ws[TW];
    __shared__ double lsum[TW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = threadIdx.x; q < MLP_PARAMS; q += blockDim.x) P[q] = params[q];
    const int nb = mode == 0 ? 1 : (n + batch - 1) / batch;
    const int passes = mode == 0 ? 1 : epochs;
    int step = step_io ? *step_io : 0;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int e = 0; e < passes; ++e) {
        for (int bi = 0; bi < nb; ++bi) {
            const int s0 = mode == 0 ? 0 : bi * batch;
            const int s1 = mode == 0 ? n : min(n, s0 + batch);
            const float inv = 1.f / (float)(s1 - s0);
            for (int q = threadIdx.x; q < TW * MLP_PARAMS_PAD; q += blockDim.x) G[q] = 0.f;
            __syncthreads();
            float *Gw = G + warp * MLP_PARAMS_PAD;
            double lw = 0.0;
            for (int s = s0 + warp; s < s1; s += TW) {
                if (lane < NI) ws[warp].x[lane] = X[(size_t)s * NI + lane];
                __syncwarp();
                const float yv = warp_forward(P, ws[warp], lane);
                const float r = yv - T[s];
                lw += 0.5 * (double)r * (double)r;
                warp_backward(P, ws[warp], lane, r * inv, Gw);
            }
            if (lane == 0) lsum[warp] = lw;
            __syncthreads();
            // add the warps' copies in warp order; then write out or take an Adam step
            if (mode == 0) {
                for (int q = threadIdx.x; q < MLP_PARAMS; q += blockDim.x) {
                    float g = 0.f;
                    for (int w = 0; w < TW; ++w) g += G[w * MLP_PARAMS_PAD + q];
                    grad_out[q] = g;
                }
                if (threadIdx.x == 0) {
                    double l = 0.0;
                    for (int w = 0; w < TW; ++w) l += lsum[w];
                    *loss_out = l / (double)(s1 - s0);
                }
            } else {
                ++step;
                const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
                for (int q = threadIdx.x; q < MLP_PARAMS; q += blockDim.x) {
                    float g = 0.f;
                    for (int w = 0; w < TW; ++w) g += G[w * MLP_PARAMS_PAD + q];
                    const float m = b1 * adam_m[q] + (1.f - b1) * g;
                    const float v = b2 * adam_v[q] + (1.f - b2) * g * g;
                    adam_m[q] = m;
                    adam_v[q] = v;
                    P[q] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
                }
                if (threadIdx.x == 0 && loss_out) {
                    double l = 0.0;
                    for (int w = 0; w < TW; ++w) l += lsum[w];
                    loss_out[0] = l / (double)(s1 - s0);  // loss of the last minibatch
                }
            }
            __syncthreads();
        }
    }
    if (mode == 1) {
        for (int q = threadIdx.x; q < MLP_PARAMS; q += blockDim.x) params[q] = P[q];
        if (threadIdx.x == 0 && step_io) *step_io = step;
    }
}

}  // namespace

size_t mlp_train_smem() { return (size_t)(MLP_PARAMS_PAD * (1 + TW)) * sizeof(float); }

cudaError_t launch_mlp_forward(const float *params, const float *X, int n, float *y, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int blocks = (n + 7) / 8;
    if (blocks > 1024) blocks = 1024;
    k_mlp_forward<<<blocks, 256, 0, st>>>(params, X, n, y);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train(float *params, float *adam_m, float *adam_v, const float *X,
                             const float *T, int n, int batch, int epochs, float lr, int mode,
                             float *grad_out, double *loss_out, int *step_io, cudaStream_t st) {
    const size_t smem = mlp_train_smem();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_mlp_train<<<1, TW * 32, smem, st>>>(params, adam_m, adam_v, X, T, n, batch, epochs, lr, mode,
                                          grad_out, loss_out, step_io);
    return cudaGetLastError();
}

}  // namespace fbl
