// K3 -- the forward-backward point of Step 2c of Algorithm 1,
//     x_bar = prox_{alpha R}(x - alpha g) = min(max(x - alpha g - alpha mu, 0), x_max),
// R = mu||.||_1 + indicator{0 <= x <= x_max} (eq. (2.1) with x_max = +inf, the
// paper's R; a finite x_max adds the box), fused with the reductions the
// test (2.3) needs: g^T (x_bar - x), ||x_bar - x||^2 (and ||x_bar||_1 for the
// objective F), all taken over the stored (rounded) x_bar.  Memory-bound:
// per voxel it reads x and g once and writes x_bar once, in the z-innermost
// layout the projector reads; every stream is contiguous along z.
//
// Also here: the kernels that convert between the caller's [nz][ny][nx]
// volumes and the library's z-innermost layouts, the flat prox for the public
// prox_reduce call, and the fixed-order FP64 reduction of per-block sums.
#include "fbl_internal.cuh"
#include "fbl_reduce.cuh"

namespace fbl {
namespace {

constexpr int TB = 32;        // tile edge
constexpr int TR = 8;         // tile rows per pass
constexpr int P_NT = TB * TR; // threads per block

// Natural [nz][ny][nx] volume -> the library layout.  For each j, a
// 32 x 32 (k, i) tile is read along i and written along k.
template <typename T>
__global__ void __launch_bounds__(P_NT) k_pack(const T *__restrict__ x, T *__restrict__ vol,
                                               ZLayout L) {
    __shared__ T tile[TB][TB + 1];  // [k][i]
    const int i0 = blockIdx.x * TB, k0 = blockIdx.y * TB, j = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int r = 0; r < TB / TR; ++r) {
        const int k = k0 + ty + TR * r, i = i0 + tx;
        if (i < L.nx && k < L.nz) tile[ty + TR * r][tx] = x[((size_t)k * L.ny + j) * L.nx + i];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TB / TR; ++r) {
        const int i = i0 + ty + TR * r, k = k0 + tx;
        if (i < L.nx && k < L.nz) vol[L.index(i, j, k)] = tile[tx][ty + TR * r];
    }
}

// Library layout -> natural [nz][ny][nx].
template <typename T>
__global__ void __launch_bounds__(P_NT) k_unpack(const T *__restrict__ vol, ZLayout L,
                                                 T *__restrict__ x) {
    __shared__ T tile[TB][TB + 1];  // [i][k]
    const int i0 = blockIdx.x * TB, k0 = blockIdx.y * TB, j = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int r = 0; r < TB / TR; ++r) {
        const int i = i0 + ty + TR * r, k = k0 + tx;
        if (i < L.nx && k < L.nz) tile[ty + TR * r][tx] = vol[L.index(i, j, k)];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TB / TR; ++r) {
        const int k = k0 + ty + TR * r, i = i0 + tx;
        if (i < L.nx && k < L.nz) x[((size_t)k * L.ny + j) * L.nx + i] = tile[tx][ty + TR * r];
    }
}

// Gradient order [j][i][k] -> natural [nz][ny][nx] (= or +=).
__global__ void __launch_bounds__(P_NT) k_zi_to_natural(const float *__restrict__ gzi,
                                                        float *__restrict__ x, int nx, int ny,
                                                        int nz, int accumulate) {
    __shared__ float tile[TB][TB + 1];  // [i][k]
    const int i0 = blockIdx.x * TB, k0 = blockIdx.y * TB, j = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int r = 0; r < TB / TR; ++r) {
        const int i = i0 + ty + TR * r, k = k0 + tx;
        if (i < nx && k < nz) tile[ty + TR * r][tx] = gzi[((size_t)j * nx + i) * nz + k];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < TB / TR; ++r) {
        const int k = k0 + ty + TR * r, i = i0 + tx;
        if (i < nx && k < nz) {
            float *p = x + ((size_t)k * ny + j) * nx + i;
            const float v = tile[tx][ty + TR * r];
            *p = accumulate ? *p + v : v;
        }
    }
}

// Prox + reductions, streaming along z: a block owns 4 (i, j) rows of the
// z-innermost volumes; every read and write is contiguous along k.
constexpr int PZ_TX = 64;
constexpr int PZ_TY = 4;

template <typename T>
__global__ void __launch_bounds__(PZ_TX *PZ_TY) k_prox_zi(const T *__restrict__ vol, ZLayout L,
                                                          const float *__restrict__ gzi, float alpha,
                                                          float amu, float xmax, T *__restrict__ trial,
                                                          double *__restrict__ partials) {
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
        const size_t nblk = gridDim.x;
        partials[blockIdx.x] = out[0];
        partials[nblk + blockIdx.x] = out[1];
        partials[2 * nblk + blockIdx.x] = out[2];
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

// sum |x|, sum (x - xr)^2, sum xr^2 (xr may be NULL: the last two are 0)
template <typename T>
__global__ void __launch_bounds__(F_NT) k_norms(const T *__restrict__ x, const T *__restrict__ xr,
                                                int64_t n, double *__restrict__ partials) {
    float sums[3] = {0.f, 0.f, 0.f};
    const int64_t stride = (int64_t)gridDim.x * F_NT;
    for (int64_t e = (int64_t)blockIdx.x * F_NT + threadIdx.x; e < n; e += stride) {
        const float v = to_f32(x[e]);
        sums[0] += fabsf(v);
        if (xr) {
            const float r = to_f32(xr[e]);
            const float d = v - r;
            sums[1] = fmaf(d, d, sums[1]);
            sums[2] = fmaf(r, r, sums[2]);
        }
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

// Fixed-order FP64 sum of p[0 .. n) by one block of R_NT threads; the result
// is valid in thread 0.
__device__ __forceinline__ double block_reduce_fixed(const double *__restrict__ p, int n) {
    __shared__ double sm[R_NT];
    double s = 0.0;
    for (int q = threadIdx.x; q < n; q += R_NT) s += p[q];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = R_NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    return sm[0];
}

__global__ void __launch_bounds__(R_NT) k_reduce(const double *__restrict__ partials, int n,
                                                 int stride, double *__restrict__ out) {
    const int c = blockIdx.x;
    const double s = block_reduce_fixed(partials + (size_t)c * stride, n);
    if (threadIdx.x == 0) out[c] = s;
}

// One block per (volume, component): the same fixed order as k_reduce over the
// volume's tiles of phase ph (stride = its tile count).
__global__ void __launch_bounds__(R_NT) kb_reduce(const BatchVol *vols, int ph, int ncomp, int slot,
                                                  int searching_only) {
    const int v = blockIdx.x / ncomp, c = blockIdx.x % ncomp;
    const BatchVol &bv = vols[v];
    if (searching_only && !batch_searching(*bv.ls)) return;  // block-uniform
    const int n = bv.tiles[ph];
    const double s = block_reduce_fixed(bv.partials + (size_t)c * n, n);
    if (threadIdx.x == 0) bv.sc[slot + c] = s;
}

}  // namespace

cudaError_t launch_pack(const void *x, int x_dtype, void *vol, ZLayout L, cudaStream_t st) {
    dim3 block(TB, TR);
    dim3 grid((L.nx + TB - 1) / TB, (L.nz + TB - 1) / TB, L.ny);
    switch (x_dtype) {
        case FBL_BF16:
            k_pack<<<grid, block, 0, st>>>((const __nv_bfloat16 *)x, (__nv_bfloat16 *)vol, L);
            break;
        case FBL_F16: k_pack<<<grid, block, 0, st>>>((const __half *)x, (__half *)vol, L); break;
        default: k_pack<<<grid, block, 0, st>>>((const float *)x, (float *)vol, L); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_unpack(const void *vol, ZLayout L, int dtype, void *x, cudaStream_t st) {
    dim3 block(TB, TR);
    dim3 grid((L.nx + TB - 1) / TB, (L.nz + TB - 1) / TB, L.ny);
    switch (dtype) {
        case FBL_BF16:
            k_unpack<<<grid, block, 0, st>>>((const __nv_bfloat16 *)vol, L, (__nv_bfloat16 *)x);
            break;
        case FBL_F16: k_unpack<<<grid, block, 0, st>>>((const __half *)vol, L, (__half *)x); break;
        default: k_unpack<<<grid, block, 0, st>>>((const float *)vol, L, (float *)x); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_zi_to_natural(const float *gzi, float *x, int nx, int ny, int nz, int accumulate,
                                 cudaStream_t st) {
    dim3 block(TB, TR);
    dim3 grid((nx + TB - 1) / TB, (nz + TB - 1) / TB, ny);
    k_zi_to_natural<<<grid, block, 0, st>>>(gzi, x, nx, ny, nz, accumulate);
    return cudaGetLastError();
}

int prox_zi_num_partials(int nx, int ny, int nz) {
    (void)nz;
    return (nx * ny + PZ_TY - 1) / PZ_TY;
}

cudaError_t launch_prox_zi(const void *vol, ZLayout L, const float *gzi, float alpha, float amu, float xmax,
                           void *trial, int dtype, double *partials, int *n_partials,
                           cudaStream_t st) {
    const int nb = prox_zi_num_partials(L.nx, L.ny, L.nz);
    if (n_partials) *n_partials = nb;
    dim3 block(PZ_TX, PZ_TY);
    switch (dtype) {
        case FBL_BF16:
            k_prox_zi<<<nb, block, 0, st>>>((const __nv_bfloat16 *)vol, L, gzi, alpha, amu, xmax,
                                            (__nv_bfloat16 *)trial, partials);
            break;
        case FBL_F16:
            k_prox_zi<<<nb, block, 0, st>>>((const __half *)vol, L, gzi, alpha, amu, xmax, (__half *)trial,
                                            partials);
            break;
        default:
            k_prox_zi<<<nb, block, 0, st>>>((const float *)vol, L, gzi, alpha, amu, xmax, (float *)trial,
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

cudaError_t launch_norms(const void *x, const void *xr, int dtype, int64_t n, double *partials,
                         int *n_partials, cudaStream_t st) {
    const int nb = flat_blocks(n);
    if (n_partials) *n_partials = nb;
    switch (dtype) {
        case FBL_BF16:
            k_norms<<<nb, F_NT, 0, st>>>((const __nv_bfloat16 *)x, (const __nv_bfloat16 *)xr, n, partials);
            break;
        case FBL_F16:
            k_norms<<<nb, F_NT, 0, st>>>((const __half *)x, (const __half *)xr, n, partials);
            break;
        default: k_norms<<<nb, F_NT, 0, st>>>((const float *)x, (const float *)xr, n, partials); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_reduce(const BatchHdr *hdr, BatchVol *vols, int n_vol, int ph, int ncomp,
                                int slot, int searching_only, cudaStream_t st) {
    (void)hdr;
    kb_reduce<<<n_vol * ncomp, R_NT, 0, st>>>(vols, ph, ncomp, slot, searching_only);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double *partials, int n, int stride, int ncomp, double *out,
                          cudaStream_t st) {
    k_reduce<<<ncomp, R_NT, 0, st>>>(partials, n, stride, out);
    return cudaGetLastError();
}

}  // namespace fbl
