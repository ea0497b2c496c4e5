// K2 -- exact transpose A_N^T of the mini-batch projector (Step 2b's
// grad f_N = (n_theta/N_t) A_N^T (A_N x - b_N), eq. (2.5)) on sm_103a, in
// gather form: every voxel collects the taps that K1 gives it.  No atomics.
//
// A ray of family f touches voxel (i, j, k) only on the plane m of its
// dominant axis that contains the voxel (m = i for x-planes, m = j for
// y-planes), with weight wb * wz: wb from the in-plane crossing q_b(m) of its
// detector column, wz from the vertical crossing q_z(m) of its row.
//
// Work decomposition.  A warp owns 32*VPL voxels of one (i, j) column along z
// (lane l holds the VPL consecutive voxels k0 + VPL*l ...; VPL = 2, 4, 8 or
// 16), or of a 2x2 group of such columns (VPL = 4 or 8), chosen by the
// autotuner: the kernel is issue bound, and the per-column setup below is
// paid once per lane for VPL voxels.  Everything that depends only on (i, j)
// and the view -- the candidate columns within hwu of the voxel column's
// projection, each column's family, plane m, exact in-plane weight wb (from
// the same Q.40 crossing K1 uses) and vertical step -- is uniform over the
// warp.  Along z the kernel forms the column's z-profile, the transpose of
// K1's linear interpolation: the rows of the column cross plane m at q_z =
// q_z(first) + t*step, and a row whose crossing lies in the unit cell
// [k, k + 1) at fraction f gives (1 - f) r to voxel k and f r to voxel k + 1.
// A lane walks the cells kfirst - 1 .. kfirst + VPL - 1 in order, taking each
// row once (at most C = ceil(1 / step) rows per cell, a warp-uniform template
// choice); the offset of the lane's first row is exact from the Q.40
// crossing and the next ones follow by the per-row step, so the weights are
// accurate to about 1e-6.  Columns whose cells all stay inside the zero pads
// skip the clamp (a warp vote).  The residual arrives transposed and
// zero-padded (rt[s][iu][RT_PAD + iv], already multiplied by K1's row weight
// W), so the lanes' row reads are contiguous and need no bounds test.  The
// gradient is written in z-innermost order [j][i][k], coalesced.
#include "fbl_internal.cuh"
#include "fbl_reduce.cuh"

namespace fbl {
namespace {

constexpr int K2_LANES = 32;

// Launch configuration of the backprojector: k2_vpl in {2, 4, 8, 16} is one
// voxel column per warp with that many consecutive voxels per lane; 24 and 28
// are a 2x2 group of voxel columns per warp (k2_tile22) with 4 or 8 voxels per
// lane in each (the same sums, bit for bit).
__host__ __device__ __forceinline__ bool k2_group_of(const DevGeom &g) { return g.k2_vpl == 24 || g.k2_vpl == 28; }
__host__ __device__ __forceinline__ int k2_vpl_of(const DevGeom &g) {
    if (k2_group_of(g)) return g.k2_vpl - 20;
    return (g.k2_vpl == 2 || g.k2_vpl == 8 || g.k2_vpl == 16) ? g.k2_vpl : 4;
}
constexpr int K2_WARPS = 8;   // consecutive i per block

struct BpArgs {
    DevGeom g;
    const float *rt;
    const int32_t *views;
    int n_sel;
    float scale;
    float *gzi;
    double *g2_partials;  // optional: per-block sum of the squared gradient
};

// Packed FP32x2 arithmetic (sm_100 family): the same IEEE operation on each
// half, so results equal two scalar operations bit for bit.
__device__ __forceinline__ void pk_mul(float ax, float ay, float bx, float by, float &dx, float &dy) {
    asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "mul.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(dx), "=f"(dy) : "f"(ax), "f"(ay), "f"(bx), "f"(by));
}
__device__ __forceinline__ void pk_add(float ax, float ay, float bx, float by, float &dx, float &dy) {
    asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "add.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(dx), "=f"(dy) : "f"(ax), "f"(ay), "f"(bx), "f"(by));
}
__device__ __forceinline__ void pk_sub(float ax, float ay, float bx, float by, float &dx, float &dy) {
    asm("{\n\t.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "sub.rn.f32x2 d, a, b;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(dx), "=f"(dy) : "f"(ax), "f"(ay), "f"(bx), "f"(by));
}
__device__ __forceinline__ void pk_fma(float ax, float ay, float bx, float by, float cx, float cy, float &dx,
                                       float &dy) {
    asm("{\n\t.reg .b64 a, b, c, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t"
        "mov.b64 c, {%6, %7};\n\tfma.rn.f32x2 d, a, b, c;\n\tmov.b64 {%0, %1}, d;\n\t}"
        : "=f"(dx), "=f"(dy) : "f"(ax), "f"(ay), "f"(bx), "f"(by), "f"(cx), "f"(cy));
}

// One cell's rows: r[t] the row values already masked (0 where the row is not
// in the cell), et[t] their offsets from the cell's bottom; then the walk
// moves to the next cell.
template <int C, bool CLAMP>
struct CellRows {
    float r[C], et[C];
    __device__ __forceinline__ void load(const float *__restrict__ rcol, int &lo, float &e, float step, int lo_max) {
        // a 32-bit row index, the address formed per cell (cheaper than stepping
        // a 64-bit pointer by the data-dependent row count)
        const float *w = rcol + (CLAMP ? min(max(lo, -RT_PAD), lo_max) : lo);
        bool v[C];
        et[0] = e;
        v[0] = C > 1 ? true : e < 1.f;
        {
            const float r0 = __ldg(w);
            r[0] = v[0] ? r0 : 0.f;
        }
#pragma unroll
        for (int t = 1; t < C; ++t) {
            et[t] = fmaf((float)t, step, e);
            v[t] = et[t] < 1.f;
            r[t] = v[t] ? __ldg(w + t) : 0.f;
        }
        // next cell: e of the first row not taken, minus one
        float en = fmaf((float)C, step, e);
#pragma unroll
        for (int t = C - 1; t >= 0; --t) en = v[t] ? en : fmaf((float)t, step, e);
        e = en - 1.f;
        int n = 0;
#pragma unroll
        for (int t = 0; t < C; ++t) n += v[t] ? 1 : 0;
        lo += n;
    }
};

// The z-profile of one candidate column over the lane's VPL voxels, by unit
// cells: cell c = [k, k + 1) of the z axis holds the rows whose crossing q_z
// lies in it; a row at fraction f = q_z - k gives (1 - f) r to voxel k and
// f r to voxel k + 1 (the transpose of K1's linear interpolation along z).
// The lane walks cells kfirst - 1 .. kfirst + VPL - 1 (VPL + 1 cells) with
// e = q_z(first row not yet taken) - k, in [0, step] (a row on a cell
// boundary may be taken by either cell: f = 1 in the lower cell gives the
// same two weights as f = 0 in the upper one).  C = 1: rows more than one
// voxel apart, at most one per cell, tested.  C >= 2: rows at most one voxel
// apart (step <= 1), so the first row is always in the cell, and at most C
// rows per cell, the others tested.  The cells of voxels q and q + 1 are
// loaded one after the other and their sums formed with packed FP32x2
// operations; add2(q, P_q, P_q+1) receives the two voxels' profile values.
// CLAMP as for the windows: a window outside [-RT_PAD, lo_max] holds only
// zero rows.
template <int C, int VPL, bool CLAMP, class Add2>
__device__ __forceinline__ void column_cells(Add2 add2, const float *__restrict__ rcol, int lo, float e,
                                             float step, int lo_max) {
    float carry;
    {  // cell kfirst - 1: only its f part, to voxel 0
        CellRows<C, CLAMP> a;
        a.load(rcol, lo, e, step, lo_max);
        float s1 = a.et[0] * a.r[0];
#pragma unroll
        for (int t = 1; t < C; ++t) s1 = fmaf(a.et[t], a.r[t], s1);
        carry = s1;
    }
#pragma unroll
    for (int q = 0; q < VPL; q += 2) {  // the cells of voxels q and q + 1, two at a time
        CellRows<C, CLAMP> a, b;
        a.load(rcol, lo, e, step, lo_max);
        b.load(rcol, lo, e, step, lo_max);
        float s0a = a.r[0], s0b = b.r[0], s1a, s1b;
        pk_mul(a.et[0], b.et[0], a.r[0], b.r[0], s1a, s1b);
#pragma unroll
        for (int t = 1; t < C; ++t) {
            pk_add(s0a, s0b, a.r[t], b.r[t], s0a, s0b);
            pk_fma(a.et[t], b.et[t], a.r[t], b.r[t], s1a, s1b, s1a, s1b);
        }
        float da, db, Pa, Pb;
        pk_sub(s0a, s0b, s1a, s1b, da, db);
        pk_add(carry, s1a, da, db, Pa, Pb);
        add2(q, Pa, Pb);
        carry = s1b;
    }
}

// Dispatch on the column's row spacing: one row per cell at most (step > 1),
// else the geometry's largest rows-per-cell bound or one less.
template <int NTAP, int VPL, bool CLAMP, class Add>
__device__ __forceinline__ void column_cells_c(int cc, float step, Add add, const float *__restrict__ rcol, int lo,
                                               float e, int lo_max) {
    constexpr int CM = (NTAP + 1) / 2;
    constexpr int CM1 = CM > 2 ? CM - 1 : 2;
    if (CM < 2 || step > 1.f) column_cells<1, VPL, CLAMP>(add, rcol, lo, e, step, lo_max);
    else if (CM > 2 && cc <= CM1) column_cells<CM1, VPL, CLAMP>(add, rcol, lo, e, step, lo_max);
    else column_cells<(CM < 2 ? 2 : CM), VPL, CLAMP>(add, rcol, lo, e, step, lo_max);
}

// Rows per cell of a column (an upper bound: the geometry's ntap is
// floor(2 x) + 1 and this floor(x) + 1 with the same x).
__device__ __forceinline__ int cells_rows(float inv) { return (int)(inv * 1.0001f + 0.001f) + 1; }

// One candidate column's z-profile over the lane's VPL voxels, added to acc
// with the in-plane weight wb; lo and d0 = q_z(lo) - kfirst in (-1, -1 + step]
// locate the lane's first row.
template <int NTAP, int VPL>
__device__ __forceinline__ void column_profile(float (&acc)[VPL], float wb, const float *__restrict__ rcol,
                                                int lo, float d0, float step, float inv, int lo_max) {
    const int cc = cells_rows(inv);
    const bool inside = lo >= -RT_PAD && lo + (int)((float)VPL * inv) + 2 <= lo_max;
    auto add = [&](int q, float Pa, float Pb) { pk_fma(wb, wb, Pa, Pb, acc[q], acc[q + 1], acc[q], acc[q + 1]); };
    if (__all_sync(0xffffffffu, inside))
        column_cells_c<NTAP, VPL, false>(cc, step, add, rcol, lo, d0 + 1.f, lo_max);
    else
        column_cells_c<NTAP, VPL, true>(cc, step, add, rcol, lo, d0 + 1.f, lo_max);
}

// The first row of one (column, plane) window for the lane's first voxel:
// lo and d0 = q_z(lo) - kfirst in (-1, -1 + step], exact from the Q.40
// crossing (an FP32 estimate and one correction), as in k2_tile.
struct ZWin {
    int lo;
    float d0, step, inv;
};
__device__ __forceinline__ ZWin z_window(const DevGeom &g, const FxCol *cF, int m, int kfirst) {
    constexpr float kInv24 = 1.0f / 16777216.0f;  // 2^-24 (Q.40 >> 16)
    const long long kfirst_fx = (long long)kfirst << FX_BITS;
    const long long Z = __ldg(&cF->h0) + (long long)m * __ldg(&cF->h1);
    const long long zoff = g.cz_fx - (long long)(g.nv - 1) * Z;
    ZWin zw;
    zw.step = (float)(int)(Z >> 15) * kInv24;
    zw.inv = __fdividef(1.f, zw.step);
    const float zoff_f = g.cz - (float)(g.nv - 1) * 0.5f * zw.step;
    int lo = (int)ceilf(((float)kfirst - zoff_f) * zw.inv - zw.inv);
    const long long d_fx = 2LL * lo * Z + zoff - kfirst_fx;
    float d0 = (float)(int)(d_fx >> 16) * kInv24;
    if (d0 <= -1.f) {
        ++lo;
        d0 += zw.step;
    } else if (d0 - zw.step > -1.f) {
        --lo;
        d0 -= zw.step;
    }
    zw.lo = lo;
    zw.d0 = d0;
    return zw;
}

// In-plane weight of voxel row bb from the crossing floor b0, fraction fb.
__device__ __forceinline__ float inplane_weight(int b0, float fb, int bb) {
    return (b0 == bb) ? 1.f - fb : ((b0 + 1 == bb) ? fb : 0.f);
}

// One warp's 2x2 group of voxel columns (i0 + x, j0 + y), x, y in {0, 1}: for
// every view and every candidate detector column, the column's two planes of
// the group (FAMY: planes j0, j0 + 1, in-plane i0, i0 + 1; else the other
// way round) each give one z-profile, computed once and added to the two
// voxel columns of that plane with their in-plane weights.  Every voxel gets
// exactly the terms of k2_tile, in the same column order and the same
// arithmetic, so the sums are bit-identical.
template <int NTAP, int VPL, bool FAMY>
__device__ __forceinline__ void group_column(float (&acc)[2][2][VPL], const DevGeom &g, const FxCol *cF,
                                             const float *__restrict__ rcol, int i0, int j0, int kfirst,
                                             int lo_max) {
    const int mA = FAMY ? j0 : i0, bA = FAMY ? i0 : j0;
    const int Na = FAMY ? g.ny : g.nx;
    // the column constants are read where they are used (an L1 broadcast) rather than kept live
    long long qb = __ldg(&cF->qb0) + (long long)mA * __ldg(&cF->qb1);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        if (p) qb += __ldg(&cF->qb1);
        const int m = mA + p;
        if (m >= Na) break;
        const int b0 = fx_floor(qb);
        const float fb = fx_frac(qb);
        const float w0 = inplane_weight(b0, fb, bA), w1 = inplane_weight(b0, fb, bA + 1);
        if (w0 == 0.f && w1 == 0.f) continue;
        const ZWin zw = z_window(g, cF, m, kfirst);
        float(&a0)[VPL] = acc[FAMY ? 0 : p][FAMY ? p : 0];
        float(&a1)[VPL] = acc[FAMY ? 1 : p][FAMY ? p : 1];
        const int cc = cells_rows(zw.inv);
        // rows per voxel < ntap / 2 on every column of the geometry
        const bool inside = zw.lo >= -RT_PAD && zw.lo + (VPL * NTAP + 1) / 2 + 2 <= lo_max;
        auto add = [&](int q, float Pa, float Pb) {
            pk_fma(w0, w0, Pa, Pb, a0[q], a0[q + 1], a0[q], a0[q + 1]);
            pk_fma(w1, w1, Pa, Pb, a1[q], a1[q + 1], a1[q], a1[q + 1]);
        };
        if (__all_sync(0xffffffffu, inside))
            column_cells_c<NTAP, VPL, false>(cc, zw.step, add, rcol, zw.lo, zw.d0 + 1.f, lo_max);
        else
            column_cells_c<NTAP, VPL, true>(cc, zw.step, add, rcol, zw.lo, zw.d0 + 1.f, lo_max);
    }
}

// One block of 8 warps = 4 x 2 groups: voxel columns i in [8 gx, 8 gx + 8),
// j in [4 gy, 4 gy + 4), z-span bz; the block's sum of squared gradient values
// goes to *g2_partial (if not NULL).  Called by every thread.
template <int NTAP, int VPL>
__device__ __forceinline__ void k2_tile22(const BpArgs &a, int gx, int gy, int bz, double *g2_partial) {
    const DevGeom &g = a.g;
    const int lane = threadIdx.x, w = threadIdx.y;
    const int i0 = 8 * gx + 2 * (w & 3), j0 = 4 * gy + 2 * (w >> 2);
    const int kfirst = bz * K2_LANES * VPL + VPL * lane;
    float acc[2][2][VPL];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y)
#pragma unroll
            for (int q = 0; q < VPL; ++q) acc[x][y][q] = 0.f;
    const int rp = rt_pitch(g.nv);
    const int nsel = (i0 < g.nx && j0 < g.ny) ? a.n_sel : 0;
    const int lo_max = g.nv + RT_PAD - NTAP;
    for (int s = 0; s < nsel; ++s) {
        const int v = a.views[s];
        const float2 cs = g.trig[v];
        // the union of the four voxel columns' candidate windows (k2_tile's),
        // from the extreme projections (ceil and floor are monotone)
        float umin = 3.0e38f, umax = -3.0e38f;
#pragma unroll
        for (int x = 0; x < 2; ++x)
#pragma unroll
            for (int y = 0; y < 2; ++y) {
                const float xc = ((float)(i0 + x) - g.cx) * g.vx;
                const float yc = ((float)(j0 + y) - g.cy) * g.vy;
                const float xi = xc * cs.x + yc * cs.y;
                const float eta = -xc * cs.y + yc * cs.x;
                const float iuc = eta * __fdividef(g.sdd, g.sod - xi) * g.inv_du + g.cu;
                umin = fminf(umin, iuc);
                umax = fmaxf(umax, iuc);
            }
        const int iu_lo = max(0, (int)ceilf(umin - g.hwu));
        const int iu_hi = min(g.nu - 1, (int)floorf(umax + g.hwu));
        for (int iu = iu_lo; iu <= iu_hi; ++iu) {
            const size_t col = (size_t)v * g.nu + iu;
            const FxCol *cF = g.colF + col;
            const float *rcol = a.rt + ((size_t)s * g.nu + iu) * rp + RT_PAD;
            if (g.colB[col].z != 0.f)
                group_column<NTAP, VPL, true>(acc, g, cF, rcol, i0, j0, kfirst, lo_max);
            else
                group_column<NTAP, VPL, false>(acc, g, cF, rcol, i0, j0, kfirst, lo_max);
        }
    }
    float g2 = 0.f;
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
        for (int y = 0; y < 2; ++y) {
            const int i = i0 + x, j = j0 + y;
            if (i < g.nx && j < g.ny) {
                float *out = a.gzi + ((size_t)j * g.nx + i) * g.nz;
#pragma unroll
                for (int q = 0; q < VPL; ++q) {
                    const int k = kfirst + q;
                    if (k < g.nz) {
                        const float val = a.scale * acc[x][y][q];
                        out[k] = val;
                        g2 = fmaf(val, val, g2);
                    }
                }
            }
        }
    if (g2_partial) {
        float vv[1] = {g2};
        double o[1];
        block_sum_f64<K2_LANES * K2_WARPS, 1>(vv, o);
        if (threadIdx.x == 0 && threadIdx.y == 0) *g2_partial = o[0];
    }
}

// One block's work: voxel columns i = bx*8 .. bx*8+7 of row j, z-span bz;
// the block's sum of squared gradient values goes to *g2_partial (if not NULL).
// Called by every thread.
template <int NTAP, int K2_VPL>
__device__ __forceinline__ void k2_tile(const BpArgs &a, int bx, int j, int bz, double *g2_partial) {
    constexpr int K2_KSPAN = K2_LANES * K2_VPL;
    const DevGeom &g = a.g;
    const int lane = threadIdx.x;
    const int i = bx * K2_WARPS + threadIdx.y;  // uniform over the warp
    const int kfirst = bz * K2_KSPAN + K2_VPL * lane;  // this lane: kfirst .. kfirst+VPL-1
    float acc[K2_VPL];
#pragma unroll
    for (int q = 0; q < K2_VPL; ++q) acc[q] = 0.f;
    const float xc = ((float)i - g.cx) * g.vx;
    const float yc = ((float)j - g.cy) * g.vy;
    const int rp = rt_pitch(g.nv);
    const int nsel = i < g.nx ? a.n_sel : 0;  // a warp past the volume edge only joins the block sum
    const int lo_max = g.nv + RT_PAD - NTAP;  // last first-row whose taps stay in the pad
    const long long kfirst_fx = (long long)kfirst << FX_BITS;
    constexpr float kInv24 = 1.0f / 16777216.0f;  // 2^-24 (Q.40 >> 16)
    for (int s = 0; s < nsel; ++s) {
        const int v = a.views[s];
        const float2 cs = g.trig[v];
        const float xi = xc * cs.x + yc * cs.y;
        const float eta = -xc * cs.y + yc * cs.x;
        // the voxel column's projection: an estimate only (the window hwu keeps a
        // slack of 2% + 0.05 columns; the fast division errs by ~1e-4 column)
        const float iuc = eta * __fdividef(g.sdd, g.sod - xi) * g.inv_du + g.cu;
        const int iu_lo = max(0, (int)ceilf(iuc - g.hwu));
        const int iu_hi = min(g.nu - 1, (int)floorf(iuc + g.hwu));
        for (int iu = iu_lo; iu <= iu_hi; ++iu) {
            const size_t col = (size_t)v * g.nu + iu;
            const FxCol cF = g.colF[col];
            const bool famY = g.colB[col].z != 0.f;
            const int m = famY ? j : i;
            const int bb = famY ? i : j;
            const long long qb = cF.qb0 + (long long)m * cF.qb1;
            const int b0 = fx_floor(qb);
            const float fb = fx_frac(qb);
            const float wb = (b0 == bb) ? 1.f - fb : ((b0 + 1 == bb) ? fb : 0.f);
            if (wb == 0.f) continue;
            // row iv crosses plane m at q_z = 2*iv*Z + zoff (Q.40), 0 < Z < 2^40
            const long long Z = cF.h0 + (long long)m * cF.h1;
            const long long zoff = g.cz_fx - (long long)(g.nv - 1) * Z;
            const float step = (float)(int)(Z >> 15) * kInv24;  // dq_z per row = 2Z (32-bit path)
            const float inv = __fdividef(1.f, step);            // rows per voxel (estimate)
            const float zoff_f = g.cz - (float)(g.nv - 1) * 0.5f * step;
            // first row whose crossing lies above kfirst - 1: estimate, then one exact correction
            int lo = (int)ceilf(((float)kfirst - zoff_f) * inv - inv);
            const long long d_fx = 2LL * lo * Z + zoff - kfirst_fx;
            float d0 = (float)(int)(d_fx >> 16) * kInv24;  // q_z(lo) - kfirst (|.| < 2 + step)
            if (d0 <= -1.f) {
                ++lo;
                d0 += step;
            } else if (d0 - step > -1.f) {
                --lo;
                d0 -= step;
            }
            const float *rcol = a.rt + ((size_t)s * g.nu + iu) * rp + RT_PAD;
            column_profile<NTAP, K2_VPL>(acc, wb, rcol, lo, d0, step, inv, lo_max);
        }
    }
    float g2 = 0.f;
    if (i < g.nx) {
        float *out = a.gzi + ((size_t)j * g.nx + i) * g.nz;
#pragma unroll
        for (int q = 0; q < K2_VPL; ++q) {
            const int k = kfirst + q;
            if (k < g.nz) {
                const float val = a.scale * acc[q];
                out[k] = val;
                g2 = fmaf(val, val, g2);
            }
        }
    }
    if (g2_partial) {
        float vv[1] = {g2};
        double o[1];
        block_sum_f64<K2_LANES * K2_WARPS, 1>(vv, o);
        if (threadIdx.x == 0 && threadIdx.y == 0) *g2_partial = o[0];
    }
}

template <int NTAP, int K2_VPL>
// At most 48 registers (5 blocks per SM); with the per-voxel tap loop this
// kernel had before the cell walk, that cap measured 14.47 ms per 40-view
// launch at 512^3 (8 voxels per lane) against 14.68 and 18.9 ms with the
// compiler's own choices (40 registers, and 92-168 with one block per SM).
__global__ void __launch_bounds__(K2_LANES *K2_WARPS, 5) k2_backproject(const BpArgs a) {
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    k2_tile<NTAP, K2_VPL>(a, blockIdx.x, blockIdx.y, blockIdx.z, a.g2_partials ? a.g2_partials + blk : nullptr);
}

// At most 80 registers (3 blocks per SM), no spills: 8.55 against 9.22 ms per
// 40-view launch at 512^3 (8 voxels per lane), and 166.9 against 175.2 ms for
// all 720 views, with 64 registers, 4 blocks per SM and a few spilled values.
template <int NTAP, int VPL>
__global__ void __launch_bounds__(K2_LANES *K2_WARPS, 3) k2_backproject22(const BpArgs a) {
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    k2_tile22<NTAP, VPL>(a, blockIdx.x, blockIdx.y, blockIdx.z, a.g2_partials ? a.g2_partials + blk : nullptr);
}

// Persistent batched backprojector: the blocks of k2_backproject (or of the
// 2x2 group kernel) of every volume, taken from an atomic counter.  Each volume
// keeps its own launch configuration (its geometry's k2_vpl, a warp-uniform
// switch).  Registers are capped at 64 (4 blocks per SM), what the group tiles
// need.
template <int NTAP>
__global__ void __launch_bounds__(K2_LANES *K2_WARPS, 4) kb_backproject(const BatchHdr *hdr,
                                                                        const BatchVol *vols, int *ctr) {
    __shared__ int s_tile;
    __shared__ BpArgs sa;
    const int tid = threadIdx.x + K2_LANES * threadIdx.y;
    const int total = hdr->total[1];
    for (;;) {
        if (tid == 0) s_tile = atomicAdd(ctr, 1);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= total) break;
        const int vi = batch_find(*hdr, vols, 1, t);
        const BatchVol &bv = vols[vi];
        // the volume's arguments, staged in shared memory for the whole block
        stage_words(&sa.g, &bv.g, sizeof(DevGeom), tid, K2_LANES * K2_WARPS);
        if (tid == 0) {
            sa.rt = bv.rt;
            sa.views = bv.views;
            sa.n_sel = bv.N_t;
            sa.scale = bv.scale;
            sa.gzi = bv.grad;
            sa.g2_partials = bv.partials;
        }
        __syncthreads();
        const BpArgs &a = sa;
        const int local = t - bv.first[1];
        const int vpl = k2_vpl_of(bv.g);
        double *gpart = bv.partials + local;
        if (k2_group_of(bv.g)) {
            const int gxn = (bv.g.nx + 7) / 8, gyn = (bv.g.ny + 3) / 4;
            const int gx = local % gxn;
            const int rest = local / gxn;
            if (vpl == 8) k2_tile22<NTAP, 8>(a, gx, rest % gyn, rest / gyn, gpart);
            else k2_tile22<NTAP, 4>(a, gx, rest % gyn, rest / gyn, gpart);
            continue;
        }
        const int gx = (bv.g.nx + K2_WARPS - 1) / K2_WARPS;
        const int bx = local % gx;
        const int rest = local / gx;
        const int j = rest % bv.g.ny;
        const int bz = rest / bv.g.ny;
        double *part = bv.partials + local;
        switch (vpl) {
            case 2: k2_tile<NTAP, 2>(a, bx, j, bz, part); break;
            case 8: k2_tile<NTAP, 8>(a, bx, j, bz, part); break;
            case 16: k2_tile<NTAP, 16>(a, bx, j, bz, part); break;
            default: k2_tile<NTAP, 4>(a, bx, j, bz, part); break;
        }
    }
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(ctr + 1, 1) == (int)gridDim.x - 1) {
            ctr[0] = 0;
            ctr[1] = 0;
            __threadfence();
        }
    }
}

}  // namespace


static dim3 k2_grid(const DevGeom &g) {
    const int vpl = k2_vpl_of(g);
    const unsigned gz = (g.nz + K2_LANES * vpl - 1) / (K2_LANES * vpl);
    if (k2_group_of(g)) return dim3((g.nx + 7) / 8, (g.ny + 3) / 4, gz);
    return dim3((g.nx + K2_WARPS - 1) / K2_WARPS, g.ny, gz);
}

int backproject_num_partials(const DevGeom &g) {
    const dim3 gr = k2_grid(g);
    return (int)(gr.x * gr.y * gr.z);
}

template <int NT>
static void launch_k2(int vpl, dim3 grid, dim3 block, cudaStream_t st, const BpArgs &a) {
    if (k2_group_of(a.g)) {
        if (vpl == 8) k2_backproject22<NT, 8><<<grid, block, 0, st>>>(a);
        else k2_backproject22<NT, 4><<<grid, block, 0, st>>>(a);
        return;
    }
    switch (vpl) {
        case 2: k2_backproject<NT, 2><<<grid, block, 0, st>>>(a); break;
        case 8: k2_backproject<NT, 8><<<grid, block, 0, st>>>(a); break;
        case 16: k2_backproject<NT, 16><<<grid, block, 0, st>>>(a); break;
        default: k2_backproject<NT, 4><<<grid, block, 0, st>>>(a); break;
    }
}

template <class K>
static int k2_persistent_grid(K kernel) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, K2_LANES * K2_WARPS, 0);
    return (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
}

template <int NT>
static cudaError_t launch_kb2(const BatchHdr *hdr, BatchVol *vols, int *ctr, cudaStream_t st) {
    auto k = kb_backproject<NT>;
    static const int grid = k2_persistent_grid(k);
    k<<<grid, dim3(K2_LANES, K2_WARPS), 0, st>>>(hdr, vols, ctr);
    return cudaGetLastError();
}

cudaError_t launch_batch_backproject(const BatchHdr *hdr, BatchVol *vols, int ntap, int *ctr,
                                     cudaStream_t st) {
    switch (ntap) {
        case 1: return launch_kb2<1>(hdr, vols, ctr, st);
        case 2: return launch_kb2<2>(hdr, vols, ctr, st);
        case 3: return launch_kb2<3>(hdr, vols, ctr, st);
        case 4: return launch_kb2<4>(hdr, vols, ctr, st);
        case 5: return launch_kb2<5>(hdr, vols, ctr, st);
        case 6: return launch_kb2<6>(hdr, vols, ctr, st);
        case 7: return launch_kb2<7>(hdr, vols, ctr, st);
        default: return launch_kb2<8>(hdr, vols, ctr, st);
    }
}

cudaError_t launch_backproject(const DevGeom &g, const float *rt, const int32_t *views,
                               int n_sel, float scale, float *gzi, cudaStream_t st,
                               double *g2_partials) {
    BpArgs a;
    a.g2_partials = g2_partials;
    a.g = g;
    a.rt = rt;
    a.views = views;
    a.n_sel = n_sel;
    a.scale = scale;
    a.gzi = gzi;
    dim3 block(K2_LANES, K2_WARPS);
    const int vpl = k2_vpl_of(g);
    const dim3 grid = k2_grid(g);
    switch (g.ntap) {  // rows per voxel and column, fixed per geometry (<= RT_PAD)
        case 1: launch_k2<1>(vpl, grid, block, st, a); break;
        case 2: launch_k2<2>(vpl, grid, block, st, a); break;
        case 3: launch_k2<3>(vpl, grid, block, st, a); break;
        case 4: launch_k2<4>(vpl, grid, block, st, a); break;
        case 5: launch_k2<5>(vpl, grid, block, st, a); break;
        case 6: launch_k2<6>(vpl, grid, block, st, a); break;
        case 7: launch_k2<7>(vpl, grid, block, st, a); break;
        default: launch_k2<8>(vpl, grid, block, st, a); break;
    }
    return cudaGetLastError();
}

}  // namespace fbl
