// K1 -- mini-batch cone-beam forward projection A_N x (eq. (2.5)) on sm_103a,
// with the residual and the FP64 objective reduction of Step 2b / Step 2c
// fused into its epilogue.
//
// Work decomposition.  A warp follows the 32 rays of 32 consecutive detector
// rows of one detector column through every plane m of their dominant axis
// (one ray per lane).  All rays of a column share the in-plane crossing
// q_b(m) (the detector's v axis is vertical), so the warp reads, per plane,
// two adjacent rows b0, b0+1 of the z-innermost volume layout over a run of
// consecutive k: about five 32-byte sectors per load instead of one sector
// per lane.  Both ray families read the same volume copy with their own
// plane and in-plane strides.  A block is 8 columns of one view; the grid runs the 32-row
// bands slowest, so the blocks resident together cover every view of the
// batch for one band of rows and share a z-slab of the volume in L2.
//
// Arithmetic.  Per-ray constants come from the geometry's column tables (FP64
// on the host, rounded once to Q.40 fixed point): q_b(m) = qb0 + m*qb1 and
// q_z(m) = n*(h0 + m*h1) + cz.  Stepping from plane to plane adds an integer,
// so every crossing equals its closed form exactly.  Each ray's plane interval
// [m0, m1] is the exact set of planes whose crossing lies inside
// (-1, Nb) x (-1, nz) (an interval: the maps are affine in m); the warp walks
// the union of its rays' intervals -- without per-sample masks where they all
// overlap, and with masks at the two ends, where a ray outside its own
// interval samples the zero row k = -1 with weight 0.  Interpolation and the ray sum
// are FP32; the squared residuals are summed in FP64 across threads and
// blocks in a fixed order.
#include <algorithm>

#include "fbl_internal.cuh"
#include "fbl_reduce.cuh"

namespace fbl {
namespace {

constexpr int K1_ROWS = 32;  // detector rows per warp: one ray per lane

struct ProjArgs {
    DevGeom g;
    const void *vol;
    ZLayout L;
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

// Exact plane interval of one ray ([m0, m1], empty if m0 > m1).
__device__ __forceinline__ void plane_range(const RayConst &rc, int Na, int &m0, int &m1) {
    float mlo = 0.f, mhi = (float)(Na - 1);
    clip_affine(rc.fqb0, rc.fqb1, -1.f, rc.Nb, mlo, mhi);
    clip_affine(fmaf(rc.w, rc.fzc0, rc.cz), rc.w * rc.fzc1, -1.f, rc.Nz, mlo, mhi);
    m0 = 1;
    m1 = 0;
    if (!(mlo <= mhi + 2.f)) return;
    int a = max(0, (int)floorf(mlo) - 1);
    int c = min(Na - 1, (int)ceilf(mhi) + 1);
    while (a <= c && !rc.inside(a)) ++a;
    while (c >= a && !rc.inside(c)) --c;
    if (a > c) return;
    while (a > 0 && rc.inside(a - 1)) --a;
    while (c < Na - 1 && rc.inside(c + 1)) ++c;
    m0 = a;
    m1 = c;
}

// Plane loop over [m_begin, m_end] for a lane's ray.  MASKED: outside its own
// interval [o0, o1] the ray samples the zero row k = -1 with weight 0.
template <bool MASKED, typename TX>
__device__ __forceinline__ float plane_loop(const TX *__restrict__ vol, int m_begin, int m_end,
                                            int ps, int bs, int base, const RayConst &rc, int o0,
                                            int o1) {
    long long qb = rc.qb0 + (long long)m_begin * rc.qb1;
    long long qz = rc.qz0 + (long long)m_begin * rc.qz1;
    int off = base + m_begin * ps;
    float s0 = 0.f, s1 = 0.f;
#pragma unroll 2
    for (int m = m_begin; m <= m_end; ++m) {
        const int b0 = fx_floor(qb);
        const float fb = fx_frac(qb);
        int k0 = fx_floor(qz);
        float fz = fx_frac(qz);
        if (MASKED) {
            const bool in = (m >= o0) & (m <= o1);
            k0 = in ? k0 : -1;
            fz = in ? fz : 0.f;
        }
        const TX *p = vol + (off + b0 * bs + k0);
        const float v00 = ldg_f32(p), v10 = ldg_f32(p + 1);
        const float v01 = ldg_f32(p + bs), v11 = ldg_f32(p + bs + 1);
        const float lo = fmaf(fb, v01 - v00, v00);
        const float hi = fmaf(fb, v11 - v10, v10);
        const float val = fmaf(fz, hi - lo, lo);
        if (m & 1) s1 += val; else s0 += val;
        qb += rc.qb1;
        qz += rc.qz1;
        off += ps;
    }
    return s0 + s1;
}

template <typename TX>
__device__ __forceinline__ void make_ray(const DevGeom &g, const float4 &cA, const FxCol &cF, int Nb,
                                         int iv, RayConst &rc) {
    const int n = 2 * iv - (g.nv - 1);  // w = n * dv / 2
    rc.fqb0 = cA.x;
    rc.fqb1 = cA.y;
    rc.fzc0 = cA.z;
    rc.fzc1 = cA.w;
    rc.w = (float)n * (0.5f * g.dv);
    rc.cz = g.cz;
    rc.Nb = (float)Nb;
    rc.Nz = (float)g.nz;
    rc.qb0 = cF.qb0;
    rc.qb1 = cF.qb1;
    rc.qz0 = (long long)n * cF.h0 + g.cz_fx;
    rc.qz1 = (long long)n * cF.h1;
    rc.hi_b = (long long)Nb << FX_BITS;
    rc.hi_z = (long long)g.nz << FX_BITS;
}

template <typename TX, typename TB, typename TO, int MODE>
__device__ __forceinline__ void epilogue(const ProjArgs &a, const float4 &cB, int s, int iu, int iv,
                                         float w, float sum, float &r2) {
    const DevGeom &g = a.g;
    const float W = cB.x * sqrtf(fmaf(w, w, cB.y));
    const float ax = W * sum;
    if (MODE == PROJ_STORE) {
        ((TO *)a.out)[((size_t)s * g.nv + iv) * g.nu + iu] = from_f32<TO>(ax);
    } else {
        const int bv = a.b_views ? a.b_views[s] : s;
        const float bval = ldg_f32((const TB *)a.b + ((size_t)bv * g.nv + iv) * g.nu + iu);
        const float r = ax - bval;
        if (MODE == PROJ_RESID)
            ((float *)a.out)[((size_t)s * g.nu + iu) * rt_pitch(g.nv) + RT_PAD + iv] = W * r;
        r2 += r * r;
    }
}

// One block's work: COLS detector columns (block column cb) of batch slot s,
// detector rows band*32 .. band*32+31; the block's FP64 sum of squared
// residuals goes to *partial (modes RESID and NORM).  Called by every thread.
template <typename TX, typename TB, typename TO, int MODE, int COLS, bool SPLIT>
__device__ __forceinline__ void k1_tile(const ProjArgs &a, int cb, int s, int band, double *partial) {
    const DevGeom &g = a.g;
    const int lane = threadIdx.x;
    const int iu = cb * COLS + threadIdx.y;  // uniform over the warp
    const int iv = band * K1_ROWS + lane;
    float r2 = 0.f;
    if (iu < g.nu) {
        const int v = a.views[s];
        const size_t col = (size_t)v * g.nu + iu;
        const float4 cA = g.colA[col];
        const float4 cB = g.colB[col];
        const FxCol cF = g.colF[col];
        const bool famY = cB.z != 0.f;
        const int Na = famY ? g.ny : g.nx;  // planes along the dominant axis
        const int Nb = famY ? g.nx : g.ny;  // in-plane extent
        RayConst rc;
        make_ray<TX>(g, cA, cF, Nb, iv, rc);
        int m0 = 1, m1 = 0;
        if (iv < g.nv) plane_range(rc, Na, m0, m1);
        constexpr int BIG = 1 << 30;
        const bool has = m0 <= m1;
        // a ray with no sample is pinned to the zero row k = -1 with weight 0
        if (!has) {
            rc.qz0 = -(1LL << FX_BITS);
            rc.qz1 = 0;
        }
        // warp union of the intervals, and their common part (rays without samples excluded)
        const int u0 = __reduce_min_sync(0xffffffffu, has ? m0 : BIG);
        const int u1 = __reduce_max_sync(0xffffffffu, has ? m1 : -1);
        const int c0 = __reduce_max_sync(0xffffffffu, has ? m0 : -BIG);
        const int c1 = __reduce_min_sync(0xffffffffu, has ? m1 : BIG);
        float acc = 0.f;
        if (u0 <= u1) {
            const TX *vol = (const TX *)a.vol;
            const ZLayout &L = a.L;
            const int ps = L.plane_stride(famY);    // next plane
            const int bs = L.inplane_stride(famY);  // next in-plane voxel
            // element (b, m, k) = vol + [PL + (m+1)*ps + (b+1)*bs + k]
            const int base = L.PL + ps + bs;
            const int o0 = has ? m0 : BIG, o1 = has ? m1 : -1;
            if (SPLIT && c0 <= c1) {
                if (u0 < c0) acc += plane_loop<true, TX>(vol, u0, c0 - 1, ps, bs, base, rc, o0, o1);
                acc += plane_loop<false, TX>(vol, c0, c1, ps, bs, base, rc, o0, o1);
                if (c1 < u1) acc += plane_loop<true, TX>(vol, c1 + 1, u1, ps, bs, base, rc, o0, o1);
            } else {
                acc = plane_loop<true, TX>(vol, u0, u1, ps, bs, base, rc, o0, o1);
            }
        }
        if (iv < g.nv) epilogue<TX, TB, TO, MODE>(a, cB, s, iu, iv, rc.w, acc, r2);
    }
    if (MODE != PROJ_STORE) {
        float vv[1] = {r2};
        double out[1];
        block_sum_f64<32 * COLS, 1>(vv, out);
        if (threadIdx.x == 0 && threadIdx.y == 0) *partial = out[0];
    }
}

template <typename TX, typename TB, typename TO, int MODE, int COLS, bool SPLIT>
__global__ void __launch_bounds__(32 * COLS) k1_project(const ProjArgs a) {
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    k1_tile<TX, TB, TO, MODE, COLS, SPLIT>(a, blockIdx.x, blockIdx.y, blockIdx.z,
                                           MODE != PROJ_STORE ? a.partials + blk : nullptr);
}

// Persistent batched projector: tiles of all volumes (the blocks of
// k1_project, volume by volume) taken from an atomic counter.  MODE NORM
// covers only this trial round's searching volumes.  Registers are capped at
// the single-volume kernel's 48 (40 warps per SM): the few bytes this spills
// outside the plane loop cost less than the occupancy a 64-register
// allocation loses (16-volume workload: 96.4 against 102.9 ms per iteration).
template <typename TX, typename TB, int MODE, int COLS>
__global__ void __launch_bounds__(32 * COLS, 40 / COLS) kb_project(const BatchHdr *hdr, const BatchVol *vols,
                                                                   int *ctr) {
    __shared__ int s_tile;
    __shared__ ProjArgs sa;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    // the trial objective covers this round's searching volumes only
    const int total = MODE == PROJ_NORM ? hdr->rtotal[0] : hdr->total[0];
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(ctr, 1);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= total) break;
        const int vi = MODE == PROJ_NORM ? batch_find_round(*hdr, vols, 0, t) : batch_find(*hdr, vols, 0, t);
        const BatchVol &bv = vols[vi];
        // the volume's arguments, staged in shared memory for the whole block
        stage_words(&sa.g, &bv.g, sizeof(DevGeom), tid, 32 * COLS);
        if (tid == 0) {
            sa.vol = MODE == PROJ_NORM ? bv.x_trial : bv.x_cur;
            sa.L = bv.L;
            sa.views = bv.views;
            sa.b = bv.b;
            sa.b_views = bv.b_views;
            sa.out = bv.rt;
            sa.partials = bv.partials;
        }
        __syncthreads();
        const ProjArgs &a = sa;
        const int local = t - (MODE == PROJ_NORM ? bv.rfirst[0] : bv.first[0]);
        const int ncb = (bv.g.nu + COLS - 1) / COLS;
        const int cb = local % ncb;
        const int rest = local / ncb;
        const int s = rest % bv.N_t;
        const int band = rest / bv.N_t;
        if (bv.g.k1_split)  // each volume keeps its own plane-loop form
            k1_tile<TX, TB, float, MODE, COLS, true>(a, cb, s, band, bv.partials + local);
        else
            k1_tile<TX, TB, float, MODE, COLS, false>(a, cb, s, band, bv.partials + local);
    }
    // the last block to leave resets the counter for the next launch
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(ctr + 1, 1) == (int)gridDim.x - 1) {
            ctr[0] = 0;
            ctr[1] = 0;
            __threadfence();
        }
    }
}

// rt[s][iu][RT_PAD + iv] = W(ray) * y[s][iv][iu], through a 32 x 32 shared tile
// (reads along iu, writes along iv).
template <typename TY>
__global__ void __launch_bounds__(256) k_weight(const DevGeom g, const TY *__restrict__ y,
                                                const int32_t *views, float *__restrict__ rt) {
    __shared__ float tile[32][33];
    const int s = blockIdx.z;
    const int iu0 = blockIdx.x * 32, iv0 = blockIdx.y * 32;
    const int v = views[s];
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int iv = iv0 + ty + 8 * r, iu = iu0 + tx;
        if (iu < g.nu && iv < g.nv) {
            const float4 cB = g.colB[(size_t)v * g.nu + iu];
            const float w = (float)(2 * iv - (g.nv - 1)) * (0.5f * g.dv);
            const float W = cB.x * sqrtf(fmaf(w, w, cB.y));
            tile[ty + 8 * r][tx] = W * to_f32(y[((size_t)s * g.nv + iv) * g.nu + iu]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int iu = iu0 + ty + 8 * r, iv = iv0 + tx;
        if (iu < g.nu && iv < g.nv)
            rt[((size_t)s * g.nu + iu) * rt_pitch(g.nv) + RT_PAD + iv] = tile[tx][ty + 8 * r];
    }
}

template <typename TX, typename TB, typename TO, int MODE>
cudaError_t launch_t(const ProjArgs &a, int n_sel, cudaStream_t st) {
    const int cols = a.g.k1_cols == 4 ? 4 : 8;
    dim3 block(32, cols);
    dim3 grid((a.g.nu + cols - 1) / cols, n_sel, (a.g.nv + K1_ROWS - 1) / K1_ROWS);
    if (cols == 4) {
        if (a.g.k1_split) k1_project<TX, TB, TO, MODE, 4, true><<<grid, block, 0, st>>>(a);
        else k1_project<TX, TB, TO, MODE, 4, false><<<grid, block, 0, st>>>(a);
    } else {
        if (a.g.k1_split) k1_project<TX, TB, TO, MODE, 8, true><<<grid, block, 0, st>>>(a);
        else k1_project<TX, TB, TO, MODE, 8, false><<<grid, block, 0, st>>>(a);
    }
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
    const int cols = g.k1_cols == 4 ? 4 : 8;
    return ((g.nu + cols - 1) / cols) * n_sel * ((g.nv + K1_ROWS - 1) / K1_ROWS);
}

cudaError_t launch_project(int mode, const DevGeom &g, const void *vol, ZLayout L, int x_dtype,
                           const int32_t *views, int n_sel, const void *b, int b_dtype,
                           const int32_t *b_views, void *out, int out_dtype, double *partials,
                           int *n_partials, cudaStream_t st) {
    if (n_sel <= 0) {
        if (n_partials) *n_partials = 0;
        return cudaSuccess;
    }
    ProjArgs a;
    a.g = g;
    a.vol = vol;
    a.L = L;
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

// Blocks of a persistent kernel: as many as can be resident on every SM.
template <class K>
static int persistent_grid(K kernel, int threads) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    return std::max(1, sms) * std::max(1, per_sm);
}

template <typename TX, int MODE, int COLS>
static cudaError_t launch_kb(const BatchHdr *hdr, BatchVol *vols, int *ctr, cudaStream_t st) {
    auto k = kb_project<TX, TX, MODE, COLS>;
    static const int grid = persistent_grid(k, 32 * COLS);
    k<<<grid, dim3(32, COLS), 0, st>>>(hdr, vols, ctr);
    return cudaGetLastError();
}

template <typename TX>
static cudaError_t launch_kb_mode(int mode, int cols, const BatchHdr *hdr, BatchVol *vols, int *ctr,
                                  cudaStream_t st) {
    if (mode == PROJ_NORM)
        return cols == 4 ? launch_kb<TX, PROJ_NORM, 4>(hdr, vols, ctr, st)
                         : launch_kb<TX, PROJ_NORM, 8>(hdr, vols, ctr, st);
    return cols == 4 ? launch_kb<TX, PROJ_RESID, 4>(hdr, vols, ctr, st)
                     : launch_kb<TX, PROJ_RESID, 8>(hdr, vols, ctr, st);
}

cudaError_t launch_batch_project(int mode, const BatchHdr *hdr, BatchVol *vols, int x_dtype,
                                 int b_dtype, int cols, int *ctr, cudaStream_t st) {
    if (b_dtype != x_dtype || (mode != PROJ_RESID && mode != PROJ_NORM)) return cudaErrorInvalidValue;
    switch (x_dtype) {
        case FBL_BF16: return launch_kb_mode<__nv_bfloat16>(mode, cols, hdr, vols, ctr, st);
        case FBL_F16: return launch_kb_mode<__half>(mode, cols, hdr, vols, ctr, st);
        default: return launch_kb_mode<float>(mode, cols, hdr, vols, ctr, st);
    }
}

cudaError_t launch_weight(const DevGeom &g, const void *y, int y_dtype, const int32_t *views,
                          int n_sel, float *rt, cudaStream_t st) {
    if (n_sel <= 0) return cudaSuccess;
    dim3 block(32, 8);
    dim3 grid((g.nu + 31) / 32, (g.nv + 31) / 32, n_sel);
    switch (y_dtype) {
        case FBL_BF16: k_weight<<<grid, block, 0, st>>>(g, (const __nv_bfloat16 *)y, views, rt); break;
        case FBL_F16: k_weight<<<grid, block, 0, st>>>(g, (const __half *)y, views, rt); break;
        default: k_weight<<<grid, block, 0, st>>>(g, (const float *)y, views, rt); break;
    }
    return cudaGetLastError();
}

}  // namespace fbl
