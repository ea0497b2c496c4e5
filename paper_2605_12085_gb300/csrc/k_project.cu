// K1 -- mini-batch cone-beam forward projection A_N x (eq. (2.5)) on sm_103a,
// with the residual and the FP64 objective reduction of Step 2b / Step 2c
// fused into its epilogue.
//
// One thread follows one ray (view s, column iu, row iv) through every plane
// m of its dominant axis that its bilinear footprint touches.  A block is a
// 32 x 8 tile of the detector of one view; the grid runs the detector rows
// slowest, so the blocks resident at one time cover every view of the batch
// for one band of rows and share a z-slab of the volume in L2.
//
// Per-ray constants come from the geometry's column tables (FP64 on the host,
// rounded once to Q.40 fixed point): q_b(m) = qb0 + m*qb1 and
// q_z(m) = n*(h0 + m*h1) + cz.  Stepping from plane to plane adds an integer,
// so every crossing equals its closed form exactly and the gather
// backprojector reproduces it bit for bit.  The plane interval [m0, m1] is the
// exact set of planes on which the crossing lies inside (-1, Nb) x (-1, nz)
// (an interval, the maps being affine in m), and the padded volume layout
// supplies the zero border, so the inner loop has no branch.
#include "fbl_internal.cuh"
#include "fbl_reduce.cuh"

namespace fbl {
namespace {

constexpr int K1_BX = 32;
constexpr int K1_BY = 8;
constexpr int K1_NT = K1_BX * K1_BY;

struct ProjArgs {
    DevGeom g;
    const void *padX;
    PadLayout LX;
    const void *padY;
    PadLayout LY;
    const int32_t *views;
    const void *b;
    const int32_t *b_views;
    void *out;
    double *partials;
};

// Intersect [mlo, mhi] with the real interval where lo < c0 + m*c1 < hi.
__device__ __forceinline__ void clip_affine(float c0, float c1, float lo, float hi, float &mlo,
                                            float &mhi) {
    if (c1 > 0.f) {
        mlo = fmaxf(mlo, (lo - c0) / c1);
        mhi = fminf(mhi, (hi - c0) / c1);
    } else if (c1 < 0.f) {
        mlo = fmaxf(mlo, (hi - c0) / c1);
        mhi = fminf(mhi, (lo - c0) / c1);
    } else if (!(c0 > lo && c0 < hi)) {
        mlo = 1.f;
        mhi = 0.f;
    }
}

// One ray: FP32 constants for the plane-range estimate, exact Q.40 constants
// for the crossings q_b(m) = qb0 + m*qb1 and q_z(m) = qz0 + m*qz1.
struct RayConst {
    float fqb0, fqb1, fzc0, fzc1, w, cz, Nb, Nz;
    long long qb0, qb1, qz0, qz1;
    long long hi_b, hi_z;  // Nb and nz in Q.40 (the lower bound is -1)
    __device__ __forceinline__ bool inside(int m) const {
        const long long qb = qb0 + (long long)m * qb1;
        const long long qz = qz0 + (long long)m * qz1;
        constexpr long long lo = -(1LL << FX_BITS);
        return qb > lo && qb < hi_b && qz > lo && qz < hi_z;
    }
};

// Joseph sum of one ray over its planes (without the row weight).
template <typename TX>
__device__ __forceinline__ float ray_sum(const RayConst &rc, const TX *__restrict__ vol,
                                         const PadLayout &L) {
    float mlo = 0.f, mhi = (float)(L.Na - 1);
    clip_affine(rc.fqb0, rc.fqb1, -1.f, rc.Nb, mlo, mhi);
    clip_affine(fmaf(rc.w, rc.fzc0, rc.cz), rc.w * rc.fzc1, -1.f, rc.Nz, mlo, mhi);
    if (!(mlo <= mhi + 2.f)) return 0.f;
    int m0 = max(0, (int)floorf(mlo) - 1);
    int m1 = min(L.Na - 1, (int)ceilf(mhi) + 1);
    // exact interval: the crossings are affine in m, so "inside" holds on an interval
    while (m0 <= m1 && !rc.inside(m0)) ++m0;
    while (m1 >= m0 && !rc.inside(m1)) --m1;
    if (m0 > m1) return 0.f;
    while (m0 > 0 && rc.inside(m0 - 1)) --m0;
    while (m1 < L.Na - 1 && rc.inside(m1 + 1)) ++m1;
    const int sK = L.Na * L.pitch;
    const TX *row = vol + ((size_t)sK + L.PL + (size_t)m0 * L.pitch);  // (b = 0, m = m0, k = 0)
    long long qb = rc.qb0 + (long long)m0 * rc.qb1;
    long long qz = rc.qz0 + (long long)m0 * rc.qz1;
    float acc0 = 0.f, acc1 = 0.f;
    int m = m0;
    for (; m + 1 <= m1; m += 2) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int b0 = fx_floor(qb), k0 = fx_floor(qz);
            const float fb = fx_frac(qb), fz = fx_frac(qz);
            const TX *p = row + (k0 * sK + b0);
            const float v00 = ldg_f32(p), v01 = ldg_f32(p + 1);
            const float v10 = ldg_f32(p + sK), v11 = ldg_f32(p + sK + 1);
            const float lo = fmaf(fb, v01 - v00, v00);
            const float hi = fmaf(fb, v11 - v10, v10);
            const float val = fmaf(fz, hi - lo, lo);
            if (h == 0) acc0 += val; else acc1 += val;
            qb += rc.qb1;
            qz += rc.qz1;
            row += L.pitch;
        }
    }
    if (m <= m1) {
        const int b0 = fx_floor(qb), k0 = fx_floor(qz);
        const float fb = fx_frac(qb), fz = fx_frac(qz);
        const TX *p = row + (k0 * sK + b0);
        const float v00 = ldg_f32(p), v01 = ldg_f32(p + 1);
        const float v10 = ldg_f32(p + sK), v11 = ldg_f32(p + sK + 1);
        const float lo = fmaf(fb, v01 - v00, v00);
        const float hi = fmaf(fb, v11 - v10, v10);
        acc0 += fmaf(fz, hi - lo, lo);
    }
    return acc0 + acc1;
}

template <typename TX, typename TB, typename TO, int MODE>
__global__ void __launch_bounds__(K1_NT) k1_project(const ProjArgs a) {
    const DevGeom &g = a.g;
    const int iu = blockIdx.x * K1_BX + threadIdx.x;
    const int s = blockIdx.y;
    const int iv = blockIdx.z * K1_BY + threadIdx.y;
    float r2 = 0.f;
    if (iu < g.nu && iv < g.nv) {
        const int v = a.views[s];
        const size_t col = (size_t)v * g.nu + iu;
        const float4 cA = g.colA[col];
        const float4 cB = g.colB[col];
        const FxCol cF = g.colF[col];
        const bool famY = cB.z != 0.f;
        const PadLayout &L = famY ? a.LY : a.LX;
        const TX *vol = (const TX *)(famY ? a.padY : a.padX);
        const int n = 2 * iv - (g.nv - 1);  // w = n * dv / 2
        RayConst rc;
        rc.fqb0 = cA.x;
        rc.fqb1 = cA.y;
        rc.fzc0 = cA.z;
        rc.fzc1 = cA.w;
        rc.w = (float)n * (0.5f * g.dv);
        rc.cz = g.cz;
        rc.Nb = (float)L.Nb;
        rc.Nz = (float)g.nz;
        rc.qb0 = cF.qb0;
        rc.qb1 = cF.qb1;
        rc.qz0 = (long long)n * cF.h0 + g.cz_fx;
        rc.qz1 = (long long)n * cF.h1;
        rc.hi_b = (long long)L.Nb << FX_BITS;
        rc.hi_z = (long long)g.nz << FX_BITS;
        const float sum = ray_sum<TX>(rc, vol, L);
        const float W = cB.x * sqrtf(fmaf(rc.w, rc.w, cB.y));
        const float ax = W * sum;
        const size_t o = ((size_t)s * g.nv + iv) * g.nu + iu;
        if (MODE == PROJ_STORE) {
            ((TO *)a.out)[o] = from_f32<TO>(ax);
        } else {
            const int bv = a.b_views ? a.b_views[s] : s;
            const float bval = ldg_f32((const TB *)a.b + ((size_t)bv * g.nv + iv) * g.nu + iu);
            const float r = ax - bval;
            if (MODE == PROJ_RESID) ((float *)a.out)[o] = W * r;
            r2 = r * r;
        }
    }
    if (MODE != PROJ_STORE) {
        float v[1] = {r2};
        double out[1];
        block_sum_f64<K1_NT, 1>(v, out);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
            a.partials[blk] = out[0];
        }
    }
}

// rt[s][iv][iu] = W(ray) * y[s][iv][iu]
template <typename TY>
__global__ void k_weight(const DevGeom g, const TY *__restrict__ y, const int32_t *views,
                         float *__restrict__ rt) {
    const int iu = blockIdx.x * blockDim.x + threadIdx.x;
    const int iv = blockIdx.y;
    const int s = blockIdx.z;
    if (iu >= g.nu) return;
    const int v = views[s];
    const float4 cB = g.colB[(size_t)v * g.nu + iu];
    const float w = (float)(2 * iv - (g.nv - 1)) * (0.5f * g.dv);
    const float W = cB.x * sqrtf(fmaf(w, w, cB.y));
    const size_t o = ((size_t)s * g.nv + iv) * g.nu + iu;
    rt[o] = W * to_f32(y[o]);
}

template <typename TX, typename TB, typename TO, int MODE>
cudaError_t launch_t(const ProjArgs &a, int n_sel, cudaStream_t st) {
    dim3 block(K1_BX, K1_BY);
    dim3 grid((a.g.nu + K1_BX - 1) / K1_BX, n_sel, (a.g.nv + K1_BY - 1) / K1_BY);
    k1_project<TX, TB, TO, MODE><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename TX, typename TB>
cudaError_t launch_mode(int mode, int out_dtype, const ProjArgs &a, int n_sel, cudaStream_t st) {
    if (mode == PROJ_RESID) return launch_t<TX, TB, float, PROJ_RESID>(a, n_sel, st);
    if (mode == PROJ_NORM) return launch_t<TX, TB, float, PROJ_NORM>(a, n_sel, st);
    switch (out_dtype) {
        case FBL_BF16: return launch_t<TX, TB, __nv_bfloat16, PROJ_STORE>(a, n_sel, st);
        case FBL_F16: return launch_t<TX, TB, __half, PROJ_STORE>(a, n_sel, st);
        default: return launch_t<TX, TB, float, PROJ_STORE>(a, n_sel, st);
    }
}

template <typename TX>
cudaError_t launch_bdt(int mode, int b_dtype, int out_dtype, const ProjArgs &a, int n_sel,
                       cudaStream_t st) {
    if (mode == PROJ_STORE) return launch_mode<TX, float>(mode, out_dtype, a, n_sel, st);
    switch (b_dtype) {
        case FBL_BF16: return launch_mode<TX, __nv_bfloat16>(mode, out_dtype, a, n_sel, st);
        case FBL_F16: return launch_mode<TX, __half>(mode, out_dtype, a, n_sel, st);
        default: return launch_mode<TX, float>(mode, out_dtype, a, n_sel, st);
    }
}

}  // namespace

int project_num_partials(const DevGeom &g, int n_sel) {
    return ((g.nu + K1_BX - 1) / K1_BX) * n_sel * ((g.nv + K1_BY - 1) / K1_BY);
}

cudaError_t launch_project(int mode, const DevGeom &g, const void *padX, PadLayout LX,
                           const void *padY, PadLayout LY, int x_dtype, const int32_t *views,
                           int n_sel, const void *b, int b_dtype, const int32_t *b_views,
                           void *out, int out_dtype, double *partials, int *n_partials,
                           cudaStream_t st) {
    if (n_sel <= 0) {
        if (n_partials) *n_partials = 0;
        return cudaSuccess;
    }
    ProjArgs a;
    a.g = g;
    a.padX = padX;
    a.LX = LX;
    a.padY = padY;
    a.LY = LY;
    a.views = views;
    a.b = b;
    a.b_views = b_views;
    a.out = out;
    a.partials = partials;
    if (n_partials) *n_partials = project_num_partials(g, n_sel);
    switch (x_dtype) {
        case FBL_BF16: return launch_bdt<__nv_bfloat16>(mode, b_dtype, out_dtype, a, n_sel, st);
        case FBL_F16: return launch_bdt<__half>(mode, b_dtype, out_dtype, a, n_sel, st);
        default: return launch_bdt<float>(mode, b_dtype, out_dtype, a, n_sel, st);
    }
}

cudaError_t launch_weight(const DevGeom &g, const void *y, int y_dtype, const int32_t *views,
                          int n_sel, float *rt, cudaStream_t st) {
    if (n_sel <= 0) return cudaSuccess;
    dim3 block(128);
    dim3 grid((g.nu + 127) / 128, g.nv, n_sel);
    switch (y_dtype) {
        case FBL_BF16: k_weight<<<grid, block, 0, st>>>(g, (const __nv_bfloat16 *)y, views, rt); break;
        case FBL_F16: k_weight<<<grid, block, 0, st>>>(g, (const __half *)y, views, rt); break;
        default: k_weight<<<grid, block, 0, st>>>(g, (const float *)y, views, rt); break;
    }
    return cudaGetLastError();
}

}  // namespace fbl
