// Total variation for FB-LISA's other regulariser, R = mu TV(x) + indicator of
// [0, x_max] (FB-LISA allows any convex R with a computable prox, Sec. 2.1):
// TV(x) = sum over voxels of ||(K x)_v||_2, K the forward differences along the
// three axes with a zero difference at each axis's last index.  Its prox,
//
//     argmin_{x in C} 1/2 ||x - b||^2 + lambda TV(x),   lambda = alpha mu,
//
// is computed by the fast gradient projection on the dual of Beck and
// Teboulle (2009): per inner iteration
//
//     y = P_C(b - lambda K^T r)                               (k_tv_primal)
//     q' = P_ball(r + K y / (12 lambda)),  r = q' + theta (q' - q),  q = q'  (k_tv_dual)
//
// and the result P_C(b - lambda K^T q).  Both kernels stream the volumes once
// (memory-bound: 20 and 52 bytes per voxel).  The dual pair (q, r) alternates
// between two buffers: k_tv_dual reads one pair and writes the other.  (Updated
// in place -- every thread storing to the six lines it had just loaded -- the
// same kernel ran 8x slower, its loads waiting ~20 us with DRAM 8% busy.)
// Volumes are in any memory order given
// by (n0 fastest, n1, n2); a dual field is 3 volumes, component c along axis c
// of that order (the isotropic norm does not depend on the order).  The
// solver's volumes are in gradient order [j][i][k] (n0 = nz, n1 = nx, n2 = ny);
// its right-hand side b = x - alpha g and its final step, which also forms
// the sums of the test (2.3) with the same blocks as the l1 prox, read the
// z-innermost iterate layout.
#include <cmath>

#include "fbl_internal.cuh"
#include "fbl_reduce.cuh"

namespace fbl {
namespace {

constexpr int TV_NT = 256;

struct Dims {
    int n0, n1, n2;
    __host__ __device__ size_t N() const { return (size_t)n0 * n1 * n2; }
};

// (K^T p)(v) from the three components at v and at v - e_c.
__device__ __forceinline__ float kt_at(const float *__restrict__ p0, const float *__restrict__ p1,
                                       const float *__restrict__ p2, size_t e, int a0, int a1, int a2,
                                       const Dims &d) {
    const size_t s1 = d.n0, s2 = (size_t)d.n0 * d.n1;
    float v = 0.f;
    if (a0 < d.n0 - 1) v -= p0[e];
    if (a0 > 0) v += p0[e - 1];
    if (a1 < d.n1 - 1) v -= p1[e];
    if (a1 > 0) v += p1[e - s1];
    if (a2 < d.n2 - 1) v -= p2[e];
    if (a2 > 0) v += p2[e - s2];
    return v;
}

__global__ void __launch_bounds__(TV_NT) k_tv_primal(const float *__restrict__ b, const float *__restrict__ r,
                                                     Dims d, float lam, float xmax, float *__restrict__ y) {
    const int a0 = blockIdx.x * TV_NT + threadIdx.x, a1 = blockIdx.y, a2 = blockIdx.z;
    if (a0 >= d.n0) return;
    const size_t N = d.N(), e = ((size_t)a2 * d.n1 + a1) * d.n0 + a0;
    const float kt = kt_at(r, r + N, r + 2 * N, e, a0, a1, a2, d);
    y[e] = fminf(fmaxf(fmaf(-lam, kt, b[e]), 0.f), xmax);
}

__global__ void __launch_bounds__(TV_NT) k_tv_dual(const float *__restrict__ y, Dims d, float inv12lam,
                                                   float theta, const float *__restrict__ q,
                                                   const float *__restrict__ r, float *__restrict__ qo,
                                                   float *__restrict__ ro) {
    const int a0 = blockIdx.x * TV_NT + threadIdx.x, a1 = blockIdx.y, a2 = blockIdx.z;
    if (a0 >= d.n0) return;
    const size_t N = d.N(), e = ((size_t)a2 * d.n1 + a1) * d.n0 + a0;
    const size_t s1 = d.n0, s2 = (size_t)d.n0 * d.n1;
    const float yv = y[e];
    // components whose difference does not exist stay zero
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    const bool h0 = a0 < d.n0 - 1, h1 = a1 < d.n1 - 1, h2 = a2 < d.n2 - 1;
    if (h0) g0 = fmaf(inv12lam, y[e + 1] - yv, r[e]);
    if (h1) g1 = fmaf(inv12lam, y[e + s1] - yv, r[N + e]);
    if (h2) g2 = fmaf(inv12lam, y[e + s2] - yv, r[2 * N + e]);
    const float nrm = sqrtf(fmaf(g0, g0, fmaf(g1, g1, g2 * g2)));
    const float sc = 1.f / fmaxf(nrm, 1.f);
    g0 *= sc;
    g1 *= sc;
    g2 *= sc;
    const float o0 = q[e], o1 = q[N + e], o2 = q[2 * N + e];
    qo[e] = g0;
    qo[N + e] = g1;
    qo[2 * N + e] = g2;
    ro[e] = fmaf(theta, g0 - o0, g0);
    ro[N + e] = fmaf(theta, g1 - o1, g1);
    ro[2 * N + e] = fmaf(theta, g2 - o2, g2);
}

// The starting pair (qo, ro) = (q, q) with q's components without a
// difference set to zero (q = NULL: both zero).
__global__ void __launch_bounds__(TV_NT) k_tv_start(Dims d, const float *__restrict__ q, float *__restrict__ qo,
                                                    float *__restrict__ ro) {
    const int a0 = blockIdx.x * TV_NT + threadIdx.x, a1 = blockIdx.y, a2 = blockIdx.z;
    if (a0 >= d.n0) return;
    const size_t N = d.N(), e = ((size_t)a2 * d.n1 + a1) * d.n0 + a0;
    const bool h[3] = {a0 < d.n0 - 1, a1 < d.n1 - 1, a2 < d.n2 - 1};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float v = (!q || !h[c]) ? 0.f : q[c * N + e];
        qo[c * N + e] = v;
        ro[c * N + e] = v;
    }
}

// Per-block FP64 sums of ||(K x)_v||_2.
__global__ void __launch_bounds__(TV_NT) k_tv_norm(const float *__restrict__ x, Dims d,
                                                   double *__restrict__ partials) {
    const int a0 = blockIdx.x * TV_NT + threadIdx.x, a1 = blockIdx.y, a2 = blockIdx.z;
    float s[1] = {0.f};
    if (a0 < d.n0) {
        const size_t e = ((size_t)a2 * d.n1 + a1) * d.n0 + a0;
        const size_t s1 = d.n0, s2 = (size_t)d.n0 * d.n1;
        const float xv = x[e];
        const float g0 = a0 < d.n0 - 1 ? x[e + 1] - xv : 0.f;
        const float g1 = a1 < d.n1 - 1 ? x[e + s1] - xv : 0.f;
        const float g2 = a2 < d.n2 - 1 ? x[e + s2] - xv : 0.f;
        s[0] = sqrtf(fmaf(g0, g0, fmaf(g1, g1, g2 * g2)));
    }
    double out[1];
    block_sum_f64<TV_NT, 1>(s, out);
    if (threadIdx.x == 0)
        partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = out[0];
}

// The solver's rows: a block owns TV_TY (i, j) rows of the z-innermost
// iterate, as the l1 prox does (same block count, same partial sums).
constexpr int TV_TX = 64;
constexpr int TV_TY = 4;

template <typename T>
__global__ void __launch_bounds__(TV_TX *TV_TY) k_tv_rhs_zi(const T *__restrict__ vol, ZLayout L,
                                                            const float *__restrict__ gzi, float alpha,
                                                            float *__restrict__ b) {
    const int row = blockIdx.x * TV_TY + threadIdx.y;
    if (row >= L.nx * L.ny) return;
    const int j = row / L.nx, i = row - j * L.nx;
    const T *src = vol + L.index(i, j, 0);
    const size_t o = (size_t)row * L.nz;
    for (int k = threadIdx.x; k < L.nz; k += TV_TX) b[o + k] = fmaf(-alpha, gzi[o + k], to_f32(src[k]));
}

template <typename T>
__global__ void __launch_bounds__(TV_TX *TV_TY) k_tv_final_zi(const T *__restrict__ vol, ZLayout L,
                                                              const float *__restrict__ gzi,
                                                              const float *__restrict__ b,
                                                              const float *__restrict__ q, float lam,
                                                              float xmax, T *__restrict__ trial,
                                                              double *__restrict__ partials) {
    const int row = blockIdx.x * TV_TY + threadIdx.y;
    float sums[3] = {0.f, 0.f, 0.f};
    if (row < L.nx * L.ny) {
        const int j = row / L.nx, i = row - j * L.nx;
        const Dims d{L.nz, L.nx, L.ny};  // gradient order [j][i][k]
        const size_t N = d.N();
        const T *src = vol + L.index(i, j, 0);
        T *dst = trial + L.index(i, j, 0);
        const size_t o = (size_t)row * L.nz;
        for (int k = threadIdx.x; k < L.nz; k += TV_TX) {
            const float kt = kt_at(q, q + N, q + 2 * N, o + k, k, i, j, d);
            const float xb = fminf(fmaxf(fmaf(-lam, kt, b[o + k]), 0.f), xmax);
            const T xs = from_f32<T>(xb);
            const float xr = to_f32(xs), x = to_f32(src[k]), gg = gzi[o + k];
            dst[k] = xs;
            const float dv = xr - x;
            sums[0] = fmaf(gg, dv, sums[0]);
            sums[1] = fmaf(dv, dv, sums[1]);
            sums[2] += xr;
        }
    }
    double out[3];
    block_sum_f64<TV_TX * TV_TY, 3>(sums, out);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const size_t nblk = gridDim.x;
        partials[blockIdx.x] = out[0];
        partials[nblk + blockIdx.x] = out[1];
        partials[2 * nblk + blockIdx.x] = out[2];
    }
}

dim3 tv_grid(const Dims &d) { return dim3((d.n0 + TV_NT - 1) / TV_NT, d.n1, d.n2); }

// FGP iterations from the pair (q[*cur], r[*cur]), alternating between the
// two pairs; *cur ends at the pair holding the last dual.  theta_k from
// t_1 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2.
cudaError_t fgp_iterations(const float *b, const Dims &d, float lam, float xmax, int iters, float *y,
                           float *const q[2], float *const r[2], int *cur, cudaStream_t st) {
    const dim3 grid = tv_grid(d);
    const float inv12 = (float)(1.0 / (12.0 * (double)lam));
    double t = 1.0;
    int c = *cur;
    for (int it = 0; it < iters; ++it) {
        const double tn = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
        k_tv_primal<<<grid, TV_NT, 0, st>>>(b, r[c], d, lam, xmax, y);
        k_tv_dual<<<grid, TV_NT, 0, st>>>(y, d, inv12, (float)((t - 1.0) / tn), q[c], r[c], q[1 - c], r[1 - c]);
        c = 1 - c;
        t = tn;
    }
    *cur = c;
    return cudaGetLastError();
}

}  // namespace

bool tv_dims_ok(int n0, int n1, int n2) { return n0 > 0 && n1 > 0 && n2 > 0 && n1 <= 65535 && n2 <= 65535; }

cudaError_t launch_tv_prox(const float *v, int n0, int n1, int n2, float lam, float xmax, int iters,
                           const float *q_start, float *const q[2], float *const r[2], float *y, float *x, int *cur,
                           cudaStream_t st) {
    const Dims d{n0, n1, n2};
    const dim3 grid = tv_grid(d);
    k_tv_start<<<grid, TV_NT, 0, st>>>(d, q_start, q[*cur], r[*cur]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (lam > 0.f && (e = fgp_iterations(v, d, lam, xmax, iters, y, q, r, cur, st)) != cudaSuccess) return e;
    // result P_C(v - lam K^T q): the primal kernel on q (lam = 0 gives P_C(v))
    k_tv_primal<<<grid, TV_NT, 0, st>>>(v, q[*cur], d, lam > 0.f ? lam : 0.f, xmax, x);
    return cudaGetLastError();
}

int tv_norm_num_partials(int n0, int n1, int n2) { return ((n0 + TV_NT - 1) / TV_NT) * n1 * n2; }

cudaError_t launch_tv_norm(const float *x, int n0, int n1, int n2, double *partials, cudaStream_t st) {
    const Dims d{n0, n1, n2};
    k_tv_norm<<<tv_grid(d), TV_NT, 0, st>>>(x, d, partials);
    return cudaGetLastError();
}

cudaError_t launch_tv_prox_zi(const void *vol, ZLayout L, const float *gzi, float alpha, float lam, float xmax,
                              int iters, int warm, float *b, float *const q[2], float *const r[2], int *cur,
                              float *y, void *trial, int dtype, double *partials, int *n_partials, cudaStream_t st) {
    const int nb = (L.nx * L.ny + TV_TY - 1) / TV_TY;
    if (nb != prox_zi_num_partials(L.nx, L.ny, L.nz)) return cudaErrorInvalidConfiguration;
    const dim3 blk(TV_TX, TV_TY);
    const Dims d{L.nz, L.nx, L.ny};
    switch (dtype) {
        case FBL_BF16: k_tv_rhs_zi<<<nb, blk, 0, st>>>((const __nv_bfloat16 *)vol, L, gzi, alpha, b); break;
        case FBL_F16: k_tv_rhs_zi<<<nb, blk, 0, st>>>((const __half *)vol, L, gzi, alpha, b); break;
        default: k_tv_rhs_zi<<<nb, blk, 0, st>>>((const float *)vol, L, gzi, alpha, b); break;
    }
    // the start goes to the other pair (from the last dual when warm)
    const int c0 = *cur;
    k_tv_start<<<tv_grid(d), TV_NT, 0, st>>>(d, warm ? q[c0] : nullptr, q[1 - c0], r[1 - c0]);
    *cur = 1 - c0;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (lam > 0.f && (e = fgp_iterations(b, d, lam, xmax, iters, y, q, r, cur, st)) != cudaSuccess) return e;
    const float lm = lam > 0.f ? lam : 0.f;
    const float *qf = q[*cur];
    switch (dtype) {
        case FBL_BF16:
            k_tv_final_zi<<<nb, blk, 0, st>>>((const __nv_bfloat16 *)vol, L, gzi, b, qf, lm, xmax,
                                              (__nv_bfloat16 *)trial, partials);
            break;
        case FBL_F16:
            k_tv_final_zi<<<nb, blk, 0, st>>>((const __half *)vol, L, gzi, b, qf, lm, xmax, (__half *)trial,
                                              partials);
            break;
        default:
            k_tv_final_zi<<<nb, blk, 0, st>>>((const float *)vol, L, gzi, b, qf, lm, xmax, (float *)trial,
                                              partials);
            break;
    }
    *n_partials = nb;
    return cudaGetLastError();
}

}  // namespace fbl
