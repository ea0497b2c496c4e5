// FDK reconstruction (the analytic baseline of Sec. 3) on sm_103a: cosine
// weighting and Ram-Lak ramp filtering of every detector row, then a
// weighted gather backprojection.  Everything is written on the virtual
// detector through the rotation axis (scale m = SOD/SDD):
//
//   q(a_i, b) = t * sum_n h(a_i - a_n) p(a_n, b) SOD / sqrt(SOD^2 + a_n^2 + b^2),
//       t = du m, h(0) = 1/(4 t^2), h(k t) = -1/(pi^2 k^2 t^2) for odd k, 0 else;
//   f(x) = sum_views (dtheta/2) q(eta/U, z/U) / U^2,
//       U = (SOD - xi)/SOD, xi = x cos + y sin, eta = -x sin + y cos.
//
// k_fdk_filter: a block takes FDK_ROWS consecutive detector rows of one view,
// stages the weighted rows in shared memory and every thread forms the
// filtered values of its columns for all of them (the odd-tap coefficients
// are shared by the rows).  It writes q transposed, zero-bordered:
// qt[s][iu + 1][iv + 1] with rows of nv + 2, so the backprojection reads
// consecutive detector rows along z and needs no bounds test at the edges.
// k_fdk_bp (= or += over chunks of views): a warp owns one (i, j) voxel column and 32 * FDK_KPL voxels along
// z (lane l: k0 + l + 32 t); the per-view geometry of the column (detector
// column, its weight, the vertical map k -> v) is computed once per warp in
// FP64, each lane interpolates bilinearly.  Output in [j][i][k] order.
#include <math.h>

#include "fbl_internal.cuh"

namespace fbl {
namespace {

constexpr int FDK_ROWS = 8;    // detector rows per filter block
constexpr int FDK_FT = 256;    // filter block threads
constexpr int FDK_KPL = 8;     // voxels per lane along z in the backprojection
constexpr int FDK_WARPS = 8;   // voxel columns (consecutive i) per backprojection block

template <typename TY>
__global__ void __launch_bounds__(FDK_FT) k_fdk_filter(const TY *__restrict__ y, int nu, int nv,
                                                       double sod, double du_m, double dv_m, double cu,
                                                       double cv, float *__restrict__ qt) {
    extern __shared__ float fsm[];
    float *P = fsm;                       // [FDK_ROWS][nu] weighted rows
    float *C = fsm + FDK_ROWS * nu;       // [nu/2 + 1] t * h((2j+1) t)
    const int s = blockIdx.y, r0 = blockIdx.x * FDK_ROWS;
    const double t = du_m;
    const int nodd = nu / 2 + 1;
    for (int j = threadIdx.x; j < nodd; j += FDK_FT) {
        const double k = 2.0 * j + 1.0;
        C[j] = (float)(-1.0 / (M_PI * M_PI * k * k * t));
    }
    for (int e = threadIdx.x; e < FDK_ROWS * nu; e += FDK_FT) {
        const int r = e / nu, iu = e - r * nu, iv = r0 + r;
        float val = 0.f;
        if (iv < nv) {
            const double a = (iu - cu) * du_m, b = (iv - cv) * dv_m;
            const double w = sod / sqrt(sod * sod + a * a + b * b);
            val = (float)w * to_f32(y[((size_t)s * nv + iv) * nu + iu]);
        }
        P[r * nu + iu] = val;
    }
    __syncthreads();
    const float c0 = (float)(1.0 / (4.0 * t));
    for (int iu = threadIdx.x; iu < nu; iu += FDK_FT) {
        float acc[FDK_ROWS];
#pragma unroll
        for (int r = 0; r < FDK_ROWS; ++r) acc[r] = c0 * P[r * nu + iu];
        for (int j = 0; 2 * j + 1 < nu; ++j) {
            const int k = 2 * j + 1;
            const int lft = iu - k, rgt = iu + k;
            const float c = C[j];
#pragma unroll
            for (int r = 0; r < FDK_ROWS; ++r) {
                const float pl = lft >= 0 ? P[r * nu + lft] : 0.f;
                const float pr = rgt < nu ? P[r * nu + rgt] : 0.f;
                acc[r] = fmaf(c, pl + pr, acc[r]);
            }
        }
        float *out = qt + ((size_t)s * (nu + 2) + iu + 1) * (nv + 2) + 1 + r0;
#pragma unroll
        for (int r = 0; r < FDK_ROWS; ++r)
            if (r0 + r < nv) out[r] = acc[r];
    }
}

struct FdkView {
    double c, s, w;  // cos, sin, dtheta / 2
};

__global__ void __launch_bounds__(32 * FDK_WARPS) k_fdk_bp(const float *__restrict__ qt, const FdkView *views,
                                                           int n_sel, int nx, int ny, int nz, int nu, int nv,
                                                           double vx, double vy, double vz, double sod,
                                                           double du_m, double dv_m, double cu, double cv,
                                                           int accumulate, float *__restrict__ gzi) {
    const int lane = threadIdx.x, i = blockIdx.x * FDK_WARPS + threadIdx.y, j = blockIdx.y;
    const int k0 = blockIdx.z * 32 * FDK_KPL;
    if (i >= nx) return;  // whole warp
    const double x = (i - 0.5 * (nx - 1)) * vx, yy = (j - 0.5 * (ny - 1)) * vy;
    const double czk = 0.5 * (nz - 1);
    float acc[FDK_KPL];
#pragma unroll
    for (int q = 0; q < FDK_KPL; ++q) acc[q] = 0.f;
    const size_t vstride = (size_t)(nu + 2) * (nv + 2);
    for (int s = 0; s < n_sel; ++s) {
        const FdkView v = views[s];
        const double xi = x * v.c + yy * v.s, eta = -x * v.s + yy * v.c;
        const double invU = sod / (sod - xi);
        const double fu = eta * invU / du_m + cu;
        if (!(fu > -1.0 && fu < (double)nu)) continue;  // the column projects off the detector
        const double fl = floor(fu);
        const int iu0 = (int)fl;
        const float tu = (float)(fu - fl);
        const float w = (float)(v.w * invU * invU);
        // detector row of voxel k: fv = fv0 + k * dfv, as an exact FP64 base per
        // 32 voxels (warp-uniform) plus a small FP32 offset per lane
        const double dfv = vz * invU / dv_m;
        const double fv0 = cv - czk * dfv;
        const float dfv_f = (float)dfv;
        const float *c0 = qt + (size_t)s * vstride + (size_t)(iu0 + 1) * (nv + 2) + 1;
        const float *c1 = c0 + (nv + 2);
#pragma unroll
        for (int q = 0; q < FDK_KPL; ++q) {
            const int k = k0 + lane + 32 * q;
            const double bq = fv0 + (double)(k0 + 32 * q) * dfv;
            const double bi = floor(bq);
            const float fl = (float)(bq - bi) + (float)lane * dfv_f;  // |.| <= 1 + 31 dfv
            const float fll = floorf(fl);
            const int iv0 = (int)bi + (int)fll;
            if (k < nz && iv0 >= -1 && iv0 <= nv - 1) {
                const float tv = fl - fll;
                const float a0 = __ldg(c0 + iv0), a1 = __ldg(c0 + iv0 + 1);
                const float b0 = __ldg(c1 + iv0), b1 = __ldg(c1 + iv0 + 1);
                const float lo = fmaf(tv, a1 - a0, a0), hi = fmaf(tv, b1 - b0, b0);
                acc[q] = fmaf(w, fmaf(tu, hi - lo, lo), acc[q]);
            }
        }
    }
    float *out = gzi + ((size_t)j * nx + i) * nz;
#pragma unroll
    for (int q = 0; q < FDK_KPL; ++q) {
        const int k = k0 + lane + 32 * q;
        if (k < nz) out[k] = accumulate ? out[k] + acc[q] : acc[q];
    }
}

}  // namespace

size_t fdk_filtered_elems(int n_sel, int nu, int nv) { return (size_t)n_sel * (nu + 2) * (nv + 2); }

cudaError_t launch_fdk_filter(const void *y, int y_dtype, int n_sel, int nu, int nv, double sod, double sdd,
                              double du, double dv, float *qt, cudaStream_t st) {
    if (n_sel <= 0) return cudaSuccess;
    const double m = sod / sdd;
    const size_t smem = ((size_t)FDK_ROWS * nu + nu / 2 + 1) * sizeof(float);
    dim3 grid((nv + FDK_ROWS - 1) / FDK_ROWS, n_sel);
    const double cu = 0.5 * (nu - 1), cv = 0.5 * (nv - 1);
    cudaError_t e = cudaSuccess;
    switch (y_dtype) {
        case FBL_BF16:
            e = cudaFuncSetAttribute(k_fdk_filter<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e == cudaSuccess)
                k_fdk_filter<<<grid, FDK_FT, smem, st>>>((const __nv_bfloat16 *)y, nu, nv, sod, du * m, dv * m,
                                                         cu, cv, qt);
            break;
        case FBL_F16:
            e = cudaFuncSetAttribute(k_fdk_filter<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                k_fdk_filter<<<grid, FDK_FT, smem, st>>>((const __half *)y, nu, nv, sod, du * m, dv * m, cu, cv,
                                                         qt);
            break;
        default:
            e = cudaFuncSetAttribute(k_fdk_filter<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                k_fdk_filter<<<grid, FDK_FT, smem, st>>>((const float *)y, nu, nv, sod, du * m, dv * m, cu, cv,
                                                         qt);
            break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_fdk_bp(const float *qt, const double *view_csw, int n_sel, int nx, int ny, int nz, int nu,
                          int nv, double vx, double vy, double vz, double sod, double sdd, double du, double dv,
                          int accumulate, float *gzi, cudaStream_t st) {
    const double m = sod / sdd;
    dim3 block(32, FDK_WARPS);
    dim3 grid((nx + FDK_WARPS - 1) / FDK_WARPS, ny, (nz + 32 * FDK_KPL - 1) / (32 * FDK_KPL));
    k_fdk_bp<<<grid, block, 0, st>>>(qt, (const FdkView *)view_csw, n_sel, nx, ny, nz, nu, nv, vx, vy, vz, sod,
                                     du * m, dv * m, 0.5 * (nu - 1), 0.5 * (nv - 1), accumulate, gzi);
    return cudaGetLastError();
}

}  // namespace fbl
