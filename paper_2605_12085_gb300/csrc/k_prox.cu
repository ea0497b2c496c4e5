// K3 -- the forward-backward point of Step 2c of Algorithm 1,
//     x_bar = prox_{alpha R}(x - alpha g) = max(x - alpha g - alpha mu, 0),
// R = mu||.||_1 + indicator{x >= 0} (eq. (2.1)), fused with the reductions the
// test (2.3) needs: g^T (x_bar - x), ||x_bar - x||^2 (and ||x_bar||_1 for the
// objective F), all taken over the stored (rounded) x_bar.  Memory-bound:
// per voxel it reads x and g once and writes x_bar in the two padded layouts
// the projector reads (the transposed one through a shared-memory tile).
//
// Also here: the pack kernel that builds the two padded layouts from a
// caller's volume, the flat prox for the public prox_reduce call, and the
// fixed-order FP64 reduction of per-block partial sums.
#include "fbl_internal.cuh"
#include "fbl_reduce.cuh"

namespace fbl {
namespace {

constexpr int TB = 32;        // tile edge
constexpr int TR = 8;         // tile rows per pass
constexpr int P_NT = TB * TR; // threads per block

// Natural [nz][ny][nx] volume -> padded Y layout (same orientation) and
// padded X layout (i and j swapped inside each z-slice).
template <typename T>
__global__ void __launch_bounds__(P_NT) k_pack(const T *__restrict__ x, int nx, int ny, int nz,
                                               T *__restrict__ padY, PadLayout LY,
                                               T *__restrict__ padX, PadLayout LX) {
    __shared__ T tile[TB][TB + 1];
    const int i0 = blockIdx.x * TB, j0 = blockIdx.y * TB, k = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int r = 0; r < TB / TR; ++r) {
        const int j = j0 + ty + TR * r, i = i0 + tx;
        if (i < nx && j < ny) {
            const T v = x[((size_t)k * ny + j) * nx + i];
            padY[LY.index(i, j, k)] = v;
            tile[ty + TR * r][tx] = v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TB / TR; ++r) {
        const int i = i0 + ty + TR * r, j = j0 + tx;
        if (i < nx && j < ny) padX[LX.index(j, i, k)] = tile[tx][ty + TR * r];
    }
}

template <typename T>
__global__ void __launch_bounds__(P_NT) k_prox_padded(const T *__restrict__ padY, PadLayout LY,
                                                      const float *__restrict__ gr, float alpha,
                                                      float amu, T *__restrict__ trialY,
                                                      T *__restrict__ trialX, PadLayout LX,
                                                      int nx, int ny, int nz,
                                                      double *__restrict__ partials) {
    __shared__ T tile[TB][TB + 1];
    const int i0 = blockIdx.x * TB, j0 = blockIdx.y * TB, k = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
    float sums[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int r = 0; r < TB / TR; ++r) {
        const int j = j0 + ty + TR * r, i = i0 + tx;
        if (i < nx && j < ny) {
            const int64_t py = LY.index(i, j, k);
            const float x = to_f32(padY[py]);
            const float gg = gr[((size_t)k * ny + j) * nx + i];
            const float xb = fmaxf(fmaf(-alpha, gg, x) - amu, 0.f);
            const T xs = from_f32<T>(xb);
            const float xr = to_f32(xs);
            trialY[py] = xs;
            tile[ty + TR * r][tx] = xs;
            const float d = xr - x;
            sums[0] = fmaf(gg, d, sums[0]);
            sums[1] = fmaf(d, d, sums[1]);
            sums[2] += xr;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TB / TR; ++r) {
        const int i = i0 + ty + TR * r, j = j0 + tx;
        if (i < nx && j < ny) trialX[LX.index(j, i, k)] = tile[tx][ty + TR * r];
    }
    double out[3];
    block_sum_f64<P_NT, 3>(sums, out);
    if (tx == 0 && ty == 0) {
        const size_t nblk = (size_t)gridDim.x * gridDim.y * gridDim.z;
        const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[blk] = out[0];
        partials[nblk + blk] = out[1];
        partials[2 * nblk + blk] = out[2];
    }
}

constexpr int F_NT = 256;
constexpr int F_PER = 8;  // elements per thread per grid pass

int flat_blocks(int64_t n) {
    int64_t b = (n + (int64_t)F_NT * F_PER - 1) / ((int64_t)F_NT * F_PER);
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

template <typename T>
__global__ void __launch_bounds__(F_NT) k_prox_flat(const T *__restrict__ x,
                                                    const float *__restrict__ gr, int64_t n,
                                                    float alpha, float amu, T *__restrict__ xbar,
                                                    double *__restrict__ partials) {
    float sums[3] = {0.f, 0.f, 0.f};
    const int64_t stride = (int64_t)gridDim.x * F_NT;
    for (int64_t e = (int64_t)blockIdx.x * F_NT + threadIdx.x; e < n; e += stride) {
        const float xv = to_f32(x[e]);
        const float gg = gr[e];
        const float xb = fmaxf(fmaf(-alpha, gg, xv) - amu, 0.f);
        const T xs = from_f32<T>(xb);
        const float xr = to_f32(xs);
        xbar[e] = xs;
        const float d = xr - xv;
        sums[0] = fmaf(gg, d, sums[0]);
        sums[1] = fmaf(d, d, sums[1]);
        sums[2] += xr;
    }
    double out[3];
    block_sum_f64<F_NT, 3>(sums, out);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = out[0];
        partials[gridDim.x + blockIdx.x] = out[1];
        partials[2 * gridDim.x + blockIdx.x] = out[2];
    }
}

constexpr int R_NT = 1024;

__global__ void __launch_bounds__(R_NT) k_reduce(const double *__restrict__ partials, int n,
                                                 int stride, double *__restrict__ out) {
    __shared__ double sm[R_NT];
    const int c = blockIdx.x;
    const double *p = partials + (size_t)c * stride;
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += R_NT) s += p[q];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = R_NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sm[0];
}

}  // namespace

cudaError_t launch_pack(const void *x, int x_dtype, int nx, int ny, int nz, void *padY,
                        PadLayout LY, void *padX, PadLayout LX, cudaStream_t st) {
    dim3 block(TB, TR);
    dim3 grid((nx + TB - 1) / TB, (ny + TB - 1) / TB, nz);
    switch (x_dtype) {
        case FBL_BF16:
            k_pack<<<grid, block, 0, st>>>((const __nv_bfloat16 *)x, nx, ny, nz,
                                           (__nv_bfloat16 *)padY, LY, (__nv_bfloat16 *)padX, LX);
            break;
        case FBL_F16:
            k_pack<<<grid, block, 0, st>>>((const __half *)x, nx, ny, nz, (__half *)padY, LY,
                                           (__half *)padX, LX);
            break;
        default:
            k_pack<<<grid, block, 0, st>>>((const float *)x, nx, ny, nz, (float *)padY, LY,
                                           (float *)padX, LX);
            break;
    }
    return cudaGetLastError();
}

int prox_padded_num_partials(int nx, int ny, int nz) {
    return ((nx + TB - 1) / TB) * ((ny + TB - 1) / TB) * nz;
}

cudaError_t launch_prox_padded(const void *padY, PadLayout LY, const float *gr, float alpha,
                               float amu, void *trialY, void *trialX, PadLayout LX, int dtype,
                               int nx, int ny, int nz, double *partials, int *n_partials,
                               cudaStream_t st) {
    dim3 block(TB, TR);
    dim3 grid((nx + TB - 1) / TB, (ny + TB - 1) / TB, nz);
    if (n_partials) *n_partials = prox_padded_num_partials(nx, ny, nz);
    switch (dtype) {
        case FBL_BF16:
            k_prox_padded<<<grid, block, 0, st>>>((const __nv_bfloat16 *)padY, LY, gr, alpha, amu,
                                                  (__nv_bfloat16 *)trialY, (__nv_bfloat16 *)trialX,
                                                  LX, nx, ny, nz, partials);
            break;
        case FBL_F16:
            k_prox_padded<<<grid, block, 0, st>>>((const __half *)padY, LY, gr, alpha, amu,
                                                  (__half *)trialY, (__half *)trialX, LX, nx, ny,
                                                  nz, partials);
            break;
        default:
            k_prox_padded<<<grid, block, 0, st>>>((const float *)padY, LY, gr, alpha, amu,
                                                  (float *)trialY, (float *)trialX, LX, nx, ny, nz,
                                                  partials);
            break;
    }
    return cudaGetLastError();
}

int prox_flat_num_partials(int64_t n) { return flat_blocks(n); }

cudaError_t launch_prox_flat(const void *x, const float *gr, int64_t n, float alpha, float amu,
                             void *xbar, int dtype, double *partials, int *n_partials,
                             cudaStream_t st) {
    const int nb = flat_blocks(n);
    if (n_partials) *n_partials = nb;
    switch (dtype) {
        case FBL_BF16:
            k_prox_flat<<<nb, F_NT, 0, st>>>((const __nv_bfloat16 *)x, gr, n, alpha, amu,
                                             (__nv_bfloat16 *)xbar, partials);
            break;
        case FBL_F16:
            k_prox_flat<<<nb, F_NT, 0, st>>>((const __half *)x, gr, n, alpha, amu, (__half *)xbar,
                                             partials);
            break;
        default:
            k_prox_flat<<<nb, F_NT, 0, st>>>((const float *)x, gr, n, alpha, amu, (float *)xbar,
                                             partials);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_prox_flat_grid(const void *x, const float *gr, int64_t n, float alpha, float amu,
                                  void *xbar, int dtype, int nb, double *partials,
                                  cudaStream_t st) {
    switch (dtype) {
        case FBL_BF16:
            k_prox_flat<<<nb, F_NT, 0, st>>>((const __nv_bfloat16 *)x, gr, n, alpha, amu,
                                             (__nv_bfloat16 *)xbar, partials);
            break;
        case FBL_F16:
            k_prox_flat<<<nb, F_NT, 0, st>>>((const __half *)x, gr, n, alpha, amu, (__half *)xbar,
                                             partials);
            break;
        default:
            k_prox_flat<<<nb, F_NT, 0, st>>>((const float *)x, gr, n, alpha, amu, (float *)xbar,
                                             partials);
            break;
    }
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double *partials, int n, int stride, int ncomp, double *out,
                          cudaStream_t st) {
    k_reduce<<<ncomp, R_NT, 0, st>>>(partials, n, stride, out);
    return cudaGetLastError();
}

cudaError_t copy_unpad(const void *padY, PadLayout LY, int esize, void *x, int nx, int ny, int nz,
                       cudaStream_t st) {
    const char *src = (const char *)padY + LY.index(0, 0, 0) * esize;
    return cudaMemcpy2DAsync(x, (size_t)nx * esize, src, (size_t)LY.pitch * esize,
                             (size_t)nx * esize, (size_t)ny * nz, cudaMemcpyDeviceToDevice, st);
}

}  // namespace fbl
