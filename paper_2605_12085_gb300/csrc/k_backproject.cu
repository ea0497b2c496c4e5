// K2 -- exact transpose A_N^T of the mini-batch projector (Step 2b's
// grad f_N = (n_theta/N_t) A_N^T (A_N x - b_N), eq. (2.5)) on sm_103a, in
// gather form: every voxel collects the taps that K1 would have given it.
//
// A ray of family f touches voxel (i, j, k) only on the plane m of its
// dominant axis that contains the voxel (m = i for x-planes, m = j for
// y-planes), with weight wb * wz: wb from the in-plane crossing q_b(m) of its
// column and wz from the vertical crossing q_z(m).  Both crossings are the
// exact Q.40 fixed-point numbers K1 steps through, so the two kernels use the
// same weights bit for bit.  The gather enumerates
//   * the detector columns iu within hwu of the voxel centre's projection
//     (a geometry-wide bound on the footprint, computed on the host), and for
//     each its family, plane m and in-plane weight wb; zero-weight columns are
//     skipped exactly;
//   * for each voxel of the thread's z-segment, the detector rows iv inside
//     the vertical footprint, whose width follows from the column's dq_z/div.
// The input rt already carries K1's row weight W (rt = W * r), so a tap is
// one FMA.  A thread owns a z-segment of one voxel column (i, j) and keeps the
// segment's sums in registers; lanes of a warp are consecutive i, so the
// gradient is written coalesced.  No atomics are used.
#include "fbl_internal.cuh"

namespace fbl {
namespace {

constexpr int K2_BX = 32;
constexpr int K2_BY = 4;
constexpr int K2_KS = 8;  // voxels per thread along z

struct BpArgs {
    DevGeom g;
    const float *rt;
    const int32_t *views;
    int n_sel;
    float scale;
    float *gout;
    int accumulate;
};

__global__ void __launch_bounds__(K2_BX *K2_BY) k2_backproject(const BpArgs a) {
    const DevGeom &g = a.g;
    const int i = blockIdx.x * K2_BX + threadIdx.x;
    const int j = blockIdx.y * K2_BY + threadIdx.y;
    const int k0 = blockIdx.z * K2_KS;
    if (i >= g.nx || j >= g.ny) return;
    float acc[K2_KS];
#pragma unroll
    for (int q = 0; q < K2_KS; ++q) acc[q] = 0.f;
    const float xc = ((float)i - g.cx) * g.vx;
    const float yc = ((float)j - g.cy) * g.vy;
    const size_t view_elems = (size_t)g.nv * g.nu;
    for (int s = 0; s < a.n_sel; ++s) {
        const int v = a.views[s];
        const float2 cs = g.trig[v];
        const float xi = xc * cs.x + yc * cs.y;
        const float eta = -xc * cs.y + yc * cs.x;
        const float iuc = eta * (g.sdd / (g.sod - xi)) * g.inv_du + g.cu;
        const int iu_lo = max(0, (int)ceilf(iuc - g.hwu));
        const int iu_hi = min(g.nu - 1, (int)floorf(iuc + g.hwu));
        const float *rview = a.rt + (size_t)s * view_elems;
        for (int iu = iu_lo; iu <= iu_hi; ++iu) {
            const size_t col = (size_t)v * g.nu + iu;
            const FxCol cF = g.colF[col];
            const bool famY = g.colB[col].z != 0.f;
            const int m = famY ? j : i;
            const int bb = famY ? i : j;
            // in-plane weight, from exactly K1's crossing q_b(m)
            const long long qb = cF.qb0 + (long long)m * cF.qb1;
            const int b0 = fx_floor(qb);
            const float fb = fx_frac(qb);
            const float wb = (b0 == bb) ? 1.f - fb : ((b0 + 1 == bb) ? fb : 0.f);
            if (wb == 0.f) continue;
            // q_z = n*Z + cz for row iv with n = 2*iv - (nv-1); Z > 0 because the
            // plane lies between source and detector
            const long long Z = cF.h0 + (long long)m * cF.h1;
            const float4 cA = g.colA[col];
            const float Zc = fmaf((float)m, cA.w, cA.z);
            const float inv = 1.f / (Zc * g.dv);  // detector rows per voxel along z
            const float hv = inv * 1.0001f + 1e-3f;
            const float *rcol = rview + iu;
#pragma unroll
            for (int q = 0; q < K2_KS; ++q) {
                const int k = k0 + q;
                const float ivs = fmaf((float)k - g.cz, inv, g.cv);
                const int lo = max(0, (int)ceilf(ivs - hv));
                const int hi = min(g.nv - 1, (int)floorf(ivs + hv));
                long long qz = (long long)(2 * lo - (g.nv - 1)) * Z + g.cz_fx;
                float sz = 0.f;
                for (int iv = lo; iv <= hi; ++iv) {
                    const int kz = fx_floor(qz);
                    const float fz = fx_frac(qz);
                    const float wz = (kz == k) ? 1.f - fz : ((kz + 1 == k) ? fz : 0.f);
                    sz = fmaf(wz, __ldg(rcol + (size_t)iv * g.nu), sz);
                    qz += 2 * Z;
                }
                acc[q] = fmaf(wb, sz, acc[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < K2_KS; ++q) {
        const int k = k0 + q;
        if (k < g.nz) {
            float *p = a.gout + ((size_t)k * g.ny + j) * g.nx + i;
            const float val = a.scale * acc[q];
            *p = a.accumulate ? *p + val : val;
        }
    }
}

}  // namespace

cudaError_t launch_backproject(const DevGeom &g, const float *rt, const int32_t *views,
                               int n_sel, float scale, float *gout, int accumulate,
                               cudaStream_t st) {
    BpArgs a;
    a.g = g;
    a.rt = rt;
    a.views = views;
    a.n_sel = n_sel;
    a.scale = scale;
    a.gout = gout;
    a.accumulate = accumulate;
    dim3 block(K2_BX, K2_BY);
    dim3 grid((g.nx + K2_BX - 1) / K2_BX, (g.ny + K2_BY - 1) / K2_BY, (g.nz + K2_KS - 1) / K2_KS);
    k2_backproject<<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace fbl
