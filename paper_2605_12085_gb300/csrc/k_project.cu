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
// on the host, rounded once to Q.32 fixed point): q_b(m) = qb0 + m*qb1 and
// q_z(m) = n*(h0 + m*h1) + cz.  Stepping from plane to plane adds an integer,
// so every crossing equals its closed form exactly.  The in-plane crossing is
// common to a column's rays: it is formed once per plane for the warp, 32
// planes at a time, into a shared-memory table (plane and row folded into one
// element offset, and the fraction) that every sample reads with one
// broadcast load; a sample then costs one 64-bit add and a funnel shift for
// its vertical crossing, one unsigned minimum (the clamp), four loads and
// three interpolations (the two in-plane ones as one packed FP32x2 FMA).  Each
// ray's plane interval [m0, m1] is the exact set of planes whose crossing lies
// inside (-1, Nb) x (-1, nz) (an interval: the maps are affine in m); the warp
// walks the union of its rays' intervals with no per-sample mask: the
// in-plane crossing is common to the warp, so a ray outside its own interval
// is below or above the volume in z, and its clamped row reads the zero
// elements at the ends of the z rows.  Interpolation and the ray sum are FP32
// (two partial sums, by the parity of the plane index counted from the warp's
// first plane); the squared residuals are summed in FP64 across threads and
// blocks in a fixed order.
#include <algorithm>
#include <climits>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <type_traits>

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

// One ray: FP32 constants for the plane-range estimate, exact fixed-point constants
// for the crossings q_b(m) = qb0 + m*qb1 and q_z(m) = qz0 + m*qz1.
struct RayConst {
    float fqb0, fqb1, fzc0, fzc1, w, cz, Nb, Nz;
    long long qb0, qb1, qz0, qz1;
    long long hi_b, hi_z;  // Nb and nz in fixed point (the lower bound is -1)
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

// The two in-plane interpolations of a sample, lo = a0 + f (b0 - a0) and
// hi = a1 + f (b1 - a1), as one packed FP32x2 subtraction and one packed FMA
// (the same roundings as two fmaf(f, b - a, a)).
__device__ __forceinline__ void lerp2(float f, float a0, float a1, float b0, float b1, float &lo, float &hi) {
    asm("{\n\t.reg .b64 a, b, c, d;\n\t"
        "mov.b64 a, {%2, %3};\n\t"
        "mov.b64 b, {%4, %5};\n\t"
        "sub.rn.f32x2 b, b, a;\n\t"
        "mov.b64 c, {%6, %6};\n\t"
        "fma.rn.f32x2 d, c, b, a;\n\t"
        "mov.b64 {%0, %1}, d;\n\t}"
        : "=f"(lo), "=f"(hi)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1), "f"(f));
}

// Planes per in-plane table chunk: one entry per lane.
constexpr int K1_CHUNK = 32;

// The samples j = 0 .. len-1 of one table chunk for a lane's ray.  tab[j] =
// (element offset of plane mb + j at in-plane row b0, in-plane fraction fb),
// shared by the warp's rays (one detector column); qz is the lane's vertical
// crossing at plane mb in Q.32 (advanced to mb + len).  The warp walks the
// union of its rays' intervals, and the in-plane crossing is common to the
// column, so a sample outside its own ray's interval lies below or above the
// volume in z: its row is clamped to the zero elements each z-row carries at
// either end (qz and the table offsets are shifted by 2 rows, so one unsigned
// minimum sends rows below -2 to the two zeros above nz and rows above nz to
// them too), and it adds exactly +0 -- no mask.  Samples with j even go to s0,
// odd to s1, each in plane order.
// PIPE: the next sample's loads are issued before the current sample is
// interpolated (same operations, same order per partial sum).
template <bool PIPE, typename TX>
__device__ __forceinline__ void chunk_loop(const TX *__restrict__ vol, const int2 *__restrict__ tab, int len,
                                           int bs, int nz, long long &qz, long long qz1, float &s0, float &s1) {
    struct Smp {
        float v00, v10, v01, v11, fb, fz;
    };
    auto fetch = [&](int j, Smp &o) {
        const int2 e = tab[j];
        // qz carries +2: k0 + 2 as unsigned, clamped to nz + 2 (rows below -2
        // wrap to the top: both ends hold two zero elements); e.x carries -2
        const unsigned k2 = min((unsigned)fx32_floor(qz), (unsigned)(nz + 2));
        o.fz = fx32_frac(qz);
        qz += qz1;
        const TX *p = vol + (e.x + (int)k2);
        o.fb = __int_as_float(e.y);
        o.v00 = ldg_f32(p);
        o.v10 = ldg_f32(p + 1);
        o.v01 = ldg_f32(p + bs);
        o.v11 = ldg_f32(p + bs + 1);
    };
    auto value = [](const Smp &o) {
        float lo, hi;
        lerp2(o.fb, o.v00, o.v10, o.v01, o.v11, lo, hi);
        return fmaf(o.fz, hi - lo, lo);
    };
    if (!PIPE) {
        int j = 0;
#pragma unroll 1
        for (; j + 1 < len; j += 2) {
            Smp a, b;
            fetch(j, a);
            fetch(j + 1, b);
            s0 += value(a);
            s1 += value(b);
        }
        if (j < len) {
            Smp a;
            fetch(j, a);
            s0 += value(a);
        }
        return;
    }
    Smp a, b;
    fetch(0, a);
    int j = 0;
#pragma unroll 1
    for (; j + 2 < len; j += 2) {
        fetch(j + 1, b);
        s0 += value(a);
        fetch(j + 2, a);
        s1 += value(b);
    }
    if (j + 1 < len) {
        fetch(j + 1, b);
        s0 += value(a);
        s1 += value(b);
    } else {
        s0 += value(a);
    }
}

// The Q.32 line a ray's samples follow from the warp's first plane u0:
// q_z(u0) and the step rounded once from Q.40, so the sample at plane m sits
// at qz + (m - u0) qz1, within (1 + m - u0) 2^-33 voxel of the Q.40 crossing.
__device__ __forceinline__ void ray_z32(const RayConst &rc, int u0, long long &qz, long long &qz1) {
    qz = fx40_to_32(rc.qz0 + (long long)u0 * rc.qz1);
    qz1 = fx40_to_32(rc.qz1);
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
    // Explicitly rounded operations: the compiler may not contract them into
    // FMAs, so the residual and objective modes (separate instantiations)
    // give the same r and r^2 for the same point, bit for bit -- the line
    // search compares f_N(x) from one with f_N(x_bar) from the other.
    const float W = __fmul_rn(cB.x, sqrtf(__fmaf_rn(w, w, cB.y)));  // the row weight v_a |d| / |d_a|
    const float ax = __fmul_rn(W, sum);
    if (MODE == PROJ_STORE) {
        ((TO *)a.out)[((size_t)s * g.nv + iv) * g.nu + iu] = from_f32<TO>(ax);
    } else {
        const int bv = a.b_views ? a.b_views[s] : s;
        const float bval = ldg_f32((const TB *)a.b + ((size_t)bv * g.nv + iv) * g.nu + iu);
        const float r = __fsub_rn(ax, bval);
        if (MODE == PROJ_RESID)
            ((float *)a.out)[((size_t)s * g.nu + iu) * rt_pitch(g.nv) + RT_PAD + iv] = __fmul_rn(W, r);
        r2 = __fmaf_rn(r, r, r2);
    }
}

// One block's work: COLS detector columns (block column cb) of batch slot s,
// detector rows band*32 .. band*32+31; the block's FP64 sum of squared
// residuals goes to *partial (modes RESID and NORM).  Called by every thread.
//
// The warp walks the union [u0, u1] of its rays' plane intervals in chunks
// of K1_CHUNK planes.  For a chunk, lane l forms the entry of plane mb + l:
// the in-plane crossing q_b is common to the column's rays, so its floor
// (folded with the plane into an element offset) and fraction are computed
// once per plane for the whole warp and read back by every sample with one
// broadcast shared-memory load.  PIPE: the residual and objective modes issue
// each sample's loads one sample ahead (launch configuration k1_split = 1).
template <typename TX, typename TB, typename TO, int MODE, int COLS, bool PIPE>
__device__ __forceinline__ void k1_tile(const ProjArgs &a, int cb, int s, int band, double *partial) {
    __shared__ int2 tab_all[COLS][K1_CHUNK];
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
        // a ray with no sample is pinned below the volume (reads the zero elements)
        if (!has) {
            rc.qz0 = -(2LL << FX_BITS);
            rc.qz1 = 0;
        }
        // warp union of the intervals (rays without samples excluded)
        const int u0 = __reduce_min_sync(0xffffffffu, has ? m0 : BIG);
        const int u1 = __reduce_max_sync(0xffffffffu, has ? m1 : -1);
        float acc = 0.f;
        if (u0 <= u1) {
            const TX *vol = (const TX *)a.vol;
            const ZLayout &L = a.L;
            const int ps = L.plane_stride(famY);    // next plane
            const int bs = L.inplane_stride(famY);  // next in-plane voxel
            // element (b, m, k) = vol + [PL + (m+1)*ps + (b+1)*bs + k]
            const int base = L.PL + ps + bs;
            int2 *tab = tab_all[threadIdx.y];
            // the vertical crossing in Q.32 from the warp's first plane (ray_z32)
            long long qz, qz1;
            ray_z32(rc, u0, qz, qz1);
            qz += 2LL << 32;  // chunk_loop's row index is k0 + 2
            float s0 = 0.f, s1 = 0.f;
            for (int mb = u0; mb <= u1; mb += K1_CHUNK) {
                const int len = min(K1_CHUNK, u1 - mb + 1);
                {
                    const int m = min(mb + lane, u1);
                    const long long qb = rc.qb0 + (long long)m * rc.qb1;
                    tab[lane] = make_int2(base - 2 + m * ps + fx_floor(qb) * bs, __float_as_int(fx_frac(qb)));
                }
                __syncwarp();
                // the store mode always issues loads one sample ahead; the residual
                // and objective modes when the launch configuration asks (PIPE)
                chunk_loop<MODE == PROJ_STORE || PIPE, TX>(vol, tab, len, bs, g.nz, qz, qz1, s0, s1);
                __syncwarp();
            }
            acc = s0 + s1;
        }
        // the column's weight constants and the row offset, reloaded rather than
        // kept live through the plane loop
        if (iv < g.nv)
            epilogue<TX, TB, TO, MODE>(a, g.colB[(size_t)a.views[s] * g.nu + iu], s, iu, iv,
                                       (float)(2 * iv - (g.nv - 1)) * (0.5f * g.dv), acc, r2);
    }
    if (MODE != PROJ_STORE) {
        float vv[1] = {r2};
        double out[1];
        block_sum_f64<32 * COLS, 1>(vv, out);
        if (threadIdx.x == 0 && threadIdx.y == 0) *partial = out[0];
    }
}

// Registers capped at 40 (48 warps per SM): the kernel waits on L1/L2 misses,
// and the extra resident warps hide more of that latency than the capped
// allocation costs (measured 7.09 against 7.68 ms per 40-view launch at 512^3;
// a 32-register cap is slower).
template <typename TX, typename TB, typename TO, int MODE, int COLS, bool PIPE>
__global__ void __launch_bounds__(32 * COLS, 48 / COLS) k1_project(const ProjArgs a) {
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    k1_tile<TX, TB, TO, MODE, COLS, PIPE>(a, blockIdx.x, blockIdx.y, blockIdx.z,
                                           MODE != PROJ_STORE ? a.partials + blk : nullptr);
}

// ---------------------------------------------------------------------------
// TMA-staged projector (launch configuration k1_split = 2).
//
// Same rays, crossings and epilogue as k1_tile, but the volume reaches the
// block through shared memory: the block (8 detector columns x 32 rows of one
// view) walks its planes in chunks of TMA_P, and for every chunk one thread
// issues a single cp.async.bulk.tensor.3d copy of the brick that holds every
// bilinear footprint of the chunk (KZ voxels along z x TMA_KB in-plane rows x
// TMA_P planes) into one of two buffers while the block samples the previous
// chunk.  The brick's origin comes from the band's extreme rays of each
// column, whose crossings are affine in the plane index (exact fixed point), so it
// is exact; its z origin is rounded down to the 16-byte rule of TMA.  Every
// sample still checks its indices against the brick and reads the global
// copy when outside (and so do chunks whose footprint is larger than a brick,
// and blocks whose columns belong to two ray families).  Every wait on a
// brick is bounded: past the limit the kernel records FBL_E_TIMEOUT in *err,
// stops using bricks (global reads, same result) and drains its own copies
// with a second bounded wait before it exits.
constexpr int TMA_COLS = 8;
constexpr int TMA_P = 4;
constexpr int TMA_KB = 24;
constexpr int TMA_SPIN = 1 << 22;  // mbarrier polls before a wait gives up
template <typename TX> struct TmaShape {
    static constexpr int KZ = sizeof(TX) == 4 ? 56 : 64;  // KZ * sizeof(TX): a multiple of 16 bytes
    static constexpr int ALIGN = 16 / (int)sizeof(TX);     // z origin alignment, elements
    static constexpr int BRICK = TMA_P * TMA_KB * KZ;      // elements per brick
};

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
// One bounded wait for the phase with the given parity; false after TMA_SPIN polls.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity) {
    const unsigned a = smem_addr(bar);
    for (int it = 0; it < TMA_SPIN; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

struct TmaMeta {
    int klo, blo, mc, ok;  // brick origin (z, in-plane, plane) and whether it was loaded
};

template <typename TX, typename TB, typename TO, int MODE>
__global__ void __launch_bounds__(32 * TMA_COLS) k1_project_tma(const ProjArgs a,
                                                                const __grid_constant__ CUtensorMap mapX,
                                                                const __grid_constant__ CUtensorMap mapY,
                                                                int *err) {
    constexpr int KZ = TmaShape<TX>::KZ, ALIGN = TmaShape<TX>::ALIGN, BRICK = TmaShape<TX>::BRICK;
    constexpr int P = TMA_P, KB = TMA_KB;
    constexpr unsigned BRICK_BYTES = (unsigned)(BRICK * sizeof(TX));
    extern __shared__ __align__(128) unsigned char tma_dsm[];
    // [2][BRICK], 128-byte aligned (the launch adds 128 bytes of slack)
    TX *bricks = (TX *)(tma_dsm + ((128u - (smem_addr(tma_dsm) & 127u)) & 127u));
    __shared__ __align__(8) unsigned long long full[2];
    __shared__ TmaMeta meta[2];
    __shared__ long long colz[TMA_COLS][4];  // per column: band's lowest / highest row q_z = c0 + m*c1
    __shared__ long long colb[TMA_COLS][2];  // per column: q_b = c0 + m*c1
    __shared__ int colfam[TMA_COLS];         // 0 / 1 family, -1 no column
    __shared__ int s_u0[TMA_COLS], s_u1[TMA_COLS];
    __shared__ int s_mixed, s_famY, s_U0, s_U1, s_broken;
    __shared__ int s_armed[2];

    const DevGeom &g = a.g;
    const int lane = threadIdx.x, warp = threadIdx.y, tid = lane + 32 * warp;
    const int cb = blockIdx.x, s = blockIdx.y, band = blockIdx.z;
    const int iu = cb * TMA_COLS + warp;
    const int iv = band * K1_ROWS + lane;
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    double *partial = MODE != PROJ_STORE ? a.partials + blk : nullptr;

    // family of every column of the block; two families -> plain global path
    if (lane == 0) {
        int fam = -1;
        if (iu < g.nu) fam = g.colB[(size_t)a.views[s] * g.nu + iu].z != 0.f ? 1 : 0;
        colfam[warp] = fam;
    }
    __syncthreads();
    if (tid == 0) {
        int f = -1, mixed = 0;
        for (int q = 0; q < TMA_COLS; ++q) {
            if (colfam[q] < 0) continue;
            if (f < 0) f = colfam[q];
            else if (f != colfam[q]) mixed = 1;
        }
        s_mixed = mixed || f < 0;
        s_famY = f;
    }
    __syncthreads();
    if (s_mixed) {  // the plain loop: the same sums as the brick path
        k1_tile<TX, TB, TO, MODE, TMA_COLS, false>(a, cb, s, band, partial);
        return;
    }
    const bool famY = s_famY == 1;
    const int Na = famY ? g.ny : g.nx, Nb = famY ? g.nx : g.ny;
    const ZLayout &L = a.L;
    const int ps = L.plane_stride(famY), bs = L.inplane_stride(famY);
    const int base = L.PL + ps + bs;
    const TX *vol = (const TX *)a.vol;

    RayConst rc;
    int m0 = 1, m1 = 0;
    bool has = false;
    float4 cB = make_float4(0.f, 0.f, 0.f, 0.f);
    if (iu < g.nu) {
        const size_t col = (size_t)a.views[s] * g.nu + iu;
        const float4 cA = g.colA[col];
        cB = g.colB[col];
        const FxCol cF = g.colF[col];
        make_ray<TX>(g, cA, cF, Nb, iv, rc);
        if (iv < g.nv) plane_range(rc, Na, m0, m1);
        has = m0 <= m1;
        if (lane == 0) {  // the band's extreme valid rows of this column
            const int iv_hi = min(band * K1_ROWS + K1_ROWS - 1, g.nv - 1);
            const long long n_lo = 2LL * (band * K1_ROWS) - (g.nv - 1), n_hi = 2LL * iv_hi - (g.nv - 1);
            colz[warp][0] = n_lo * cF.h0 + g.cz_fx;
            colz[warp][1] = n_lo * cF.h1;
            colz[warp][2] = n_hi * cF.h0 + g.cz_fx;
            colz[warp][3] = n_hi * cF.h1;
            colb[warp][0] = cF.qb0;
            colb[warp][1] = cF.qb1;
        }
    }
    constexpr int BIG = 1 << 30;
    const int u0 = __reduce_min_sync(0xffffffffu, has ? m0 : BIG);
    const int u1 = __reduce_max_sync(0xffffffffu, has ? m1 : -1);
    if (lane == 0) {
        s_u0[warp] = u0;
        s_u1[warp] = u1;
    }
    if (tid == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_broken = 0;
        s_armed[0] = s_armed[1] = -1;
    }
    __syncthreads();
    if (tid == 0) {
        int U0 = BIG, U1 = -1;
        for (int q = 0; q < TMA_COLS; ++q) {
            U0 = min(U0, s_u0[q]);
            U1 = max(U1, s_u1[q]);
        }
        s_U0 = U0;
        s_U1 = U1;
    }
    __syncthreads();
    const int U0 = s_U0, U1 = s_U1;
    const int nch = U1 >= U0 ? (U1 - U0 + P) / P : 0;
    // the lane's vertical crossing on k1_tile's Q.32 line from the warp's first
    // plane; a ray without samples is pinned below the volume, as in k1_tile
    long long qz32_u0 = -(2LL << 32), qz1_32 = 0;
    if (has && u0 <= u1) ray_z32(rc, u0, qz32_u0, qz1_32);

    // produce chunk c into buffer c & 1 (one warp; lanes 0..7 take a column each)
    auto produce = [&](int c) {
        const int q = c & 1;
        const int mc = U0 + c * P, me = min(mc + P - 1, U1);
        long long zlo = LLONG_MAX, zhi = LLONG_MIN, blo = LLONG_MAX, bhi = LLONG_MIN;
        if (lane < TMA_COLS && colfam[lane] >= 0) {
            const long long *z = colz[lane];
            const long long za = z[0] + (long long)mc * z[1], zb = z[0] + (long long)me * z[1];
            const long long zc = z[2] + (long long)mc * z[3], zd = z[2] + (long long)me * z[3];
            zlo = min(min(za, zb), min(zc, zd));
            zhi = max(max(za, zb), max(zc, zd));
            const long long ba = colb[lane][0] + (long long)mc * colb[lane][1];
            const long long bb = colb[lane][0] + (long long)me * colb[lane][1];
            blo = min(ba, bb);
            bhi = max(ba, bb);
        }
        // floors, clamped to the footprint range any inside ray can have
        int klo = zlo == LLONG_MAX ? BIG : max(fx_floor(zlo), -1);
        int khi = zhi == LLONG_MIN ? -BIG : min(fx_floor(zhi), g.nz - 1);
        int b_lo = blo == LLONG_MAX ? BIG : max(fx_floor(blo), -1);
        int b_hi = bhi == LLONG_MIN ? -BIG : min(fx_floor(bhi), Nb - 1);
        klo = __reduce_min_sync(0xffffffffu, klo);
        khi = __reduce_max_sync(0xffffffffu, khi);
        b_lo = __reduce_min_sync(0xffffffffu, b_lo);
        b_hi = __reduce_max_sync(0xffffffffu, b_hi);
        if (lane == 0) {
            const int kal = klo >= BIG ? 0 : (klo & ~(ALIGN - 1));  // 16-byte z origin
            const bool ok = !s_broken && klo <= khi && b_lo <= b_hi && khi + 1 - kal <= KZ - 1 &&
                            b_hi + 1 - b_lo <= KB - 1;
            meta[q] = TmaMeta{kal, b_lo, mc, ok ? 1 : 0};
            if (ok) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive_tx(&full[q], BRICK_BYTES);
                // coordinates of the layout: (L.PL + k, i + 1, j + 1)
                if (famY)
                    tma_load_3d(bricks + q * BRICK, &mapY, L.PL + kal, b_lo + 1, mc + 1, &full[q]);
                else
                    tma_load_3d(bricks + q * BRICK, &mapX, L.PL + kal, mc + 1, b_lo + 1, &full[q]);
                s_armed[q] = (c >> 1) & 1;
            } else {
                mbar_arrive(&full[q]);
            }
        }
    };

    if (nch > 0 && warp == 0) produce(0);
    float s0 = 0.f, s1 = 0.f;
    for (int c = 0; c < nch; ++c) {
        __syncthreads();  // chunk c-1 fully read by every warp; meta[c & 1] visible
        if (c + 1 < nch && warp == ((c + 1) % TMA_COLS)) produce(c + 1);
        const int q = c & 1;
        const TmaMeta mt = meta[q];
        bool ok = mt.ok != 0;
        // every chunk's phase completes (a plain arrive when no copy was issued),
        // so the phases are waited in order; once a wait has given up, no more
        // waits and no brick reads
        if (s_broken) {
            ok = false;
        } else if (!mbar_wait(&full[q], (c >> 1) & 1)) {
            ok = false;
            if (lane == 0) {
                atomicExch(err, (int)FBL_E_TIMEOUT);
                s_broken = 1;
            }
        }
        if (ok && lane == 0 && warp == 0) s_armed[q] = -1;
        const int pa = max(mt.mc, u0), pb = min(mt.mc + P - 1, u1);
        if (iu >= g.nu || pa > pb) continue;
        const TX *br = bricks + q * BRICK;
        const int bstride = famY ? KZ : P * KZ;
        long long qb = rc.qb0 + (long long)pa * rc.qb1;
        long long qz = qz32_u0 + (long long)(pa - u0) * qz1_32;
        for (int m = pa; m <= pb; ++m) {
            const int b0 = fx_floor(qb);
            const float fb = fx_frac(qb);
            // as in k1_tile, a sample outside its ray's interval reads zero elements
            const int k0 = min(max(fx32_floor(qz), -2), g.nz);
            const float fz = fx32_frac(qz);
            float v00, v10, v01, v11;
            const int kk = k0 - mt.klo, bb = b0 - mt.blo, mm = m - mt.mc;
            if (ok && (unsigned)kk <= (unsigned)(KZ - 2) && (unsigned)bb <= (unsigned)(KB - 2)) {
                const int idx = (famY ? (mm * KB + bb) * KZ : (bb * P + mm) * KZ) + kk;
                v00 = to_f32(br[idx]);
                v10 = to_f32(br[idx + 1]);
                v01 = to_f32(br[idx + bstride]);
                v11 = to_f32(br[idx + bstride + 1]);
            } else {
                const TX *p = vol + (base + m * ps + b0 * bs + k0);
                v00 = ldg_f32(p);
                v10 = ldg_f32(p + 1);
                v01 = ldg_f32(p + bs);
                v11 = ldg_f32(p + bs + 1);
            }
            const float lo = fmaf(fb, v01 - v00, v00);
            const float hi = fmaf(fb, v11 - v10, v10);
            const float val = fmaf(fz, hi - lo, lo);
            // the same partition of the sum as k1_tile: by the parity of m - u0
            if ((m - u0) & 1) s1 += val; else s0 += val;
            qb += rc.qb1;
            qz += qz1_32;
        }
    }
    // drain: every copy this block issued has landed before shared memory is released
    __syncthreads();
    if (tid == 0) {
        for (int q = 0; q < 2; ++q)
            if (s_armed[q] >= 0 && !mbar_wait(&full[q], (unsigned)s_armed[q])) atomicExch(err, (int)FBL_E_TIMEOUT);
    }
    float r2 = 0.f;
    if (iu < g.nu && iv < g.nv) epilogue<TX, TB, TO, MODE>(a, cB, s, iu, iv, rc.w, s0 + s1, r2);
    if (MODE != PROJ_STORE) {
        float vv[1] = {r2};
        double out[1];
        block_sum_f64<32 * TMA_COLS, 1>(vv, out);
        if (tid == 0) *partial = out[0];
    }
}

// Persistent batched projector: tiles of all volumes (the blocks of
// k1_project, volume by volume) taken from an atomic counter.  MODE NORM
// covers only this trial round's searching volumes.  Registers are capped at
// the single-volume kernel's 40 (48 warps per SM): the few bytes this spills
// outside the plane loop cost less than the occupancy a 48-register allocation
// loses (16-volume workload 96^3..320^3: 84.7 against 86.6 ms per iteration).
template <typename TX, typename TB, int MODE, int COLS>
__global__ void __launch_bounds__(32 * COLS, 48 / COLS) kb_project(const BatchHdr *hdr, const BatchVol *vols,
                                                                   int *ctr) {
    __shared__ int s_tile;
    __shared__ ProjArgs sa;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    // the trial objective covers only the volumes still searching in this trial
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

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (PFN_cuTensorMapEncodeTiled_v12000)p;
    }();
    return fn;
}

// Tensor map of the library volume layout [ny+2][nx+2][pitch] with a brick box
// (KZ, b1, b2) over (k, i, j).
template <typename TX>
static bool encode_volume_map(CUtensorMap *map, const void *vol, const ZLayout &L, int b1, int b2) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const CUtensorMapDataType dt = sizeof(TX) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : (std::is_same<TX, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                      : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    const cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)(L.nx + 2), (cuuint64_t)(L.ny + 2)};
    const cuuint64_t strides[2] = {(cuuint64_t)L.pitch * sizeof(TX),
                                   (cuuint64_t)L.pitch * (L.nx + 2) * sizeof(TX)};
    const cuuint32_t box[3] = {(cuuint32_t)TmaShape<TX>::KZ, (cuuint32_t)b1, (cuuint32_t)b2};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, dt, 3, const_cast<void *>(vol), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename TX, typename TB, typename TO, int MODE>
cudaError_t launch_tma(const ProjArgs &a, int n_sel, cudaStream_t st) {
    alignas(64) CUtensorMap mapX, mapY;
    // x-plane rays: planes along i, in-plane rows along j; y-plane rays the other way
    if (!encode_volume_map<TX>(&mapX, a.vol, a.L, TMA_P, TMA_KB) ||
        !encode_volume_map<TX>(&mapY, a.vol, a.L, TMA_KB, TMA_P))
        return cudaErrorNotSupported;
    dim3 block(32, TMA_COLS);
    dim3 grid((a.g.nu + TMA_COLS - 1) / TMA_COLS, n_sel, (a.g.nv + K1_ROWS - 1) / K1_ROWS);
    const size_t smem = 2 * (size_t)TmaShape<TX>::BRICK * sizeof(TX) + 128;
    k1_project_tma<TX, TB, TO, MODE><<<grid, block, smem, st>>>(a, mapX, mapY, a.g.err);
    return cudaGetLastError();
}

template <typename TX, typename TB, typename TO, int MODE>
cudaError_t launch_t(const ProjArgs &a, int n_sel, cudaStream_t st) {
    if (a.g.k1_split == 2 && a.g.err) return launch_tma<TX, TB, TO, MODE>(a, n_sel, st);
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
    const int cols = (g.k1_split == 2 && g.err) ? TMA_COLS : (g.k1_cols == 4 ? 4 : 8);
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
