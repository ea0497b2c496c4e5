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
// k_fdk_filter: a block takes FDK_ROWS consecutive detector rows of one view
// and stages the weighted rows in shared memory; each thread forms 8 filtered
// values of one row (same parity, two columns apart) from a sliding window of
// coefficients in registers, so one shared-memory read feeds 8 FMAs.  It
// writes q transposed, as column pairs:
// entry (s, c, e) = (q(c - 1, e - 2), q(c, e - 2)) for c = 0 .. nu and rows of
// fdk_row_stride(nv) entries, zero outside the detector, so the
// backprojection reads the four taps of a voxel as two aligned float2 loads of
// consecutive entries along z and needs no bounds test at the edges.  The
// block restages its results in shared memory and stores them as float4s.
// k_fdk_bp (one launch per 32 views; each adds into the volume but the very
// first, which writes it): a warp owns one (i, j) voxel
// column and 32 * FDK_KPL voxels along z (lane l: k0 + l + 32 t).  The FP64
// geometry of a (column, view) pair (detector column and weight, the
// vertical map k -> v) is formed by one thread -- lane l of the warp takes
// view s0 + l -- and kept in shared memory for the warp, so FP64 work (slow
// on this part) costs one thread per pair instead of a whole warp; every lane
// then interpolates bilinearly in FP32.  Output in [j][i][k] order.
#include <math.h>

#include "fbl_internal.cuh"

namespace fbl {
namespace {

constexpr int FDK_ROWS = 8;    // detector rows per filter block
constexpr int FDK_FT = 256;    // filter block threads
constexpr int FDK_KPL = 8;     // voxels per lane along z in the backprojection
constexpr int FDK_WARPS = 8;   // voxel columns (consecutive i) per backprojection block
constexpr int FDK_VB = 32;     // views whose pair geometry a block forms at once (one per lane)

// float2 entries per detector column of the filtered projections: row v at
// entry v + 2, two zero entries below row 0 and at least two above row nv - 1,
// even so that every column starts on a 16-byte boundary
__host__ __device__ inline int fdk_row_stride(int nv) { return (nv + 5) & ~1; }

// The filter's row staging: FR_PAD zero columns on each side of a row and a
// row stride of 2 (mod 32) words, so that the 32 lanes of a warp (8 rows x 2
// column groups 16 apart x 2 parities) read 32 different shared-memory banks.
constexpr int FR_PAD = 32;
constexpr int FR_E = 8;  // outputs per thread: columns i0, i0 + 2, .., i0 + 14
__host__ __device__ inline int fr_row_len(int nu) { return ((nu + 2 * FR_PAD + 29) & ~31) + 2; }
__host__ __device__ inline int fr_kh(int nu) { return (nu + FR_PAD + 2 * FR_E - 1) | 1; }  // odd

template <typename TY>
__global__ void __launch_bounds__(FDK_FT) k_fdk_filter(const TY *__restrict__ y, int nu, int nv,
                                                       double sod, double du_m, double dv_m, double cu,
                                                       double cv, float *__restrict__ qt) {
    extern __shared__ float fsm[];
    const int lp = nu + 2 * FR_PAD, rl = fr_row_len(nu), KH = fr_kh(nu);
    float *P = fsm;                      // [FDK_ROWS][rl] weighted rows, zero-padded
    float *Q = fsm + FDK_ROWS * rl;      // [FDK_ROWS][nu] filtered rows
    float *H = Q + FDK_ROWS * nu;        // t h(k t) for odd k in [-KH, KH], at (k + KH) / 2
    const int s = blockIdx.y, r0 = blockIdx.x * FDK_ROWS;
    const double t = du_m;
    // the odd taps in FP32 (k^2 is exact, one rounded division): FP64
    // divisions per block would cost more than the filtering
    const float ct = (float)(-1.0 / (M_PI * M_PI * t));
    for (int j = threadIdx.x; j <= KH; j += FDK_FT) {
        const float k = (float)(2 * j - KH);
        H[j] = ct / (k * k);
    }
    // cosine weight in FP32 (relative error below 1e-6): FP64 arithmetic is
    // slow on this part
    const float sodf = (float)sod, sod2 = (float)(sod * sod), duf = (float)du_m, dvf = (float)dv_m;
    const float cuf = (float)cu, cvf = (float)cv;
    for (int e = threadIdx.x; e < FDK_ROWS * lp; e += FDK_FT) {
        const int r = e / lp, c = e - r * lp, iu = c - FR_PAD, iv = r0 + r;
        float val = 0.f;
        if (iv < nv && iu >= 0 && iu < nu) {
            const float a = ((float)iu - cuf) * duf, b = ((float)iv - cvf) * dvf;
            const float w = sodf * rsqrtf(fmaf(a, a, fmaf(b, b, sod2)));
            val = w * to_f32(y[((size_t)s * nv + iv) * nu + iu]);
        }
        P[r * rl + c] = val;
    }
    __syncthreads();
    // A warp takes the 8 rows and 32 columns [Iw, Iw + 32): lane l the row
    // l / 4 and the 8 outputs i0 + 2e, i0 = Iw + 16 ((l / 2) % 2) + l % 2.
    // Output i sums t h(n - i) P(n) over the odd offsets n - i (the even ones
    // other than 0 vanish); with d = n - i0 the coefficient of output e is
    // t h(d - 2e), so as d steps by 2 the 8 coefficients shift by one place and
    // one new one is read (the same for the whole warp).  d runs over
    // [-Iw - 31, nu - 1 - Iw], which covers n = 0 .. nu - 1 for every lane; the
    // zero padding supplies the rest.
    const float c0 = (float)(1.0 / (4.0 * t));
    const int nseg = (nu + 31) / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = lane >> 2;
    const float *Pr = P + r * rl + FR_PAD;
    for (int seg = warp; seg < nseg; seg += FDK_FT / 32) {
        const int Iw = seg * 32;
        const int i0 = Iw + 16 * ((lane >> 1) & 1) + (lane & 1);
        float acc[FR_E], hw[FR_E];
        const int dmin = -Iw - 31, dmax = nu - 1 - Iw;
#pragma unroll
        for (int e = 0; e < FR_E; ++e) {
            acc[e] = c0 * Pr[i0 + 2 * e];
            hw[e] = H[(dmin - 2 * e + KH) >> 1];
        }
        const float *pp = Pr + i0;
        const float *hh = H + ((dmin + 2 + KH) >> 1);
#pragma unroll 8
        for (int d = dmin; d <= dmax; d += 2, ++hh) {
            const float p = pp[d];
#pragma unroll
            for (int e = 0; e < FR_E; ++e) acc[e] = fmaf(hw[e], p, acc[e]);
#pragma unroll
            for (int e = FR_E - 1; e > 0; --e) hw[e] = hw[e - 1];
            hw[0] = *hh;
        }
#pragma unroll
        for (int e = 0; e < FR_E; ++e)
            if (i0 + 2 * e < nu) Q[r * nu + i0 + 2 * e] = acc[e];
    }
    __syncthreads();
    // column pairs (c - 1, c) of row pairs (r0 + 2p, r0 + 2p + 1) as one float4;
    // rows at or past nv keep the zeros of the cleared buffer
    const int rs = fdk_row_stride(nv);
    float2 *out2 = reinterpret_cast<float2 *>(qt) + (size_t)s * (nu + 1) * rs + r0 + 2;
    for (int e = threadIdx.x; e < (nu + 1) * (FDK_ROWS / 2); e += FDK_FT) {
        const int c = e / (FDK_ROWS / 2), p = e - c * (FDK_ROWS / 2), r = 2 * p;
        if (r0 + r >= nv) continue;
        float4 v;
        v.x = c > 0 ? Q[r * nu + c - 1] : 0.f;
        v.y = c < nu ? Q[r * nu + c] : 0.f;
        v.z = c > 0 ? Q[(r + 1) * nu + c - 1] : 0.f;
        v.w = c < nu ? Q[(r + 1) * nu + c] : 0.f;
        *reinterpret_cast<float4 *>(out2 + (size_t)c * rs + r) = v;
    }
}

struct FdkView {
    double c, s, w;  // cos, sin, dtheta / 2
};

struct FdkPair {
    int off;          // entry of (column iu0 + 1, row 0) in the view's block
    float tu, w, dfv; // horizontal weight, (dtheta/2) / U^2, rows per voxel along z
};
struct FdkBase {
    int ib;    // floor of the detector row of voxel k0 + 32 q
    float fb;  // and its fraction
};

__global__ void __launch_bounds__(32 * FDK_WARPS, 5) k_fdk_bp(const float2 *__restrict__ qt, const FdkView *views,
                                                           int n_sel, int nx, int ny, int nz, int nu, int nv,
                                                           double vx, double vy, double vz, double sod,
                                                           double inv_du_m, double inv_dv_m, double cu, double cv,
                                                           int accumulate, float *__restrict__ gzi) {
    __shared__ FdkPair hp[FDK_WARPS][FDK_VB];
    __shared__ FdkBase hb[FDK_WARPS][FDK_KPL][FDK_VB];
    const int lane = threadIdx.x, wi = threadIdx.y;
    const int i = blockIdx.x * FDK_WARPS + wi, j = blockIdx.y;
    const int k0 = blockIdx.z * 32 * FDK_KPL;
    const bool col = i < nx;  // columns past nx still take part in the barriers
    const double x = (i - 0.5 * (nx - 1)) * vx, yy = (j - 0.5 * (ny - 1)) * vy;
    const double czk = 0.5 * (nz - 1);
    const int rs = fdk_row_stride(nv);
    const size_t vstride = (size_t)(nu + 1) * rs;
    float acc[FDK_KPL];
#pragma unroll
    for (int q = 0; q < FDK_KPL; ++q) acc[q] = 0.f;
    for (int s0 = 0; s0 < n_sel; s0 += FDK_VB) {
        const int nb = min(FDK_VB, n_sel - s0);
        if (lane < nb) {
            const FdkView v = views[s0 + lane];
            const double xi = x * v.c + yy * v.s, eta = -x * v.s + yy * v.c;
            const double invU = sod / (sod - xi);
            const double fu = eta * invU * inv_du_m + cu;
            // a column that projects off the detector reads column 0 with
            // weight 0 and rows that fail the range test below
            FdkPair p{2, 0.f, 0.f, 0.f};
            const bool on = fu > -1.0 && fu < (double)nu;
            const double dfv = vz * invU * inv_dv_m;
            if (on) {
                const double fl = floor(fu);
                p.off = ((int)fl + 1) * rs + 2;
                p.tu = (float)(fu - fl);
                p.w = (float)(v.w * invU * invU);
                p.dfv = (float)dfv;
            }
            // detector row of voxel k: fv0 + k * dfv, as a base per 32 voxels in
            // Q32 fixed point (error <= 2^-33 (1 + 32 q) rows from rounding the
            // start and the step) plus a small FP32 offset per lane: integer
            // steps instead of FP64 ones per base
            const double fv0 = cv - czk * dfv;
            const long long D = __double2ll_rn(dfv * 4294967296.0);
            long long B = __double2ll_rn((fv0 + (double)k0 * dfv) * 4294967296.0);
#pragma unroll
            for (int q = 0; q < FDK_KPL; ++q, B += 32 * D) {
                const int ib = (int)(B >> 32);
                const float fb = (float)(unsigned)(B & 0xffffffffLL) * 2.3283064365386963e-10f;  // 2^-32
                hb[wi][q][lane] = on ? FdkBase{ib, fb} : FdkBase{-(1 << 30), 0.f};
            }
            hp[wi][lane] = p;
        }
        __syncthreads();
        if (col) {
#pragma unroll 2
            for (int t = 0; t < nb; ++t) {
                const FdkPair p = hp[wi][t];
                const float2 *col2 = qt + (size_t)(s0 + t) * vstride + p.off;
                const float lf = (float)lane * p.dfv;  // |.| <= 31 dfv
#pragma unroll
                for (int q = 0; q < FDK_KPL; ++q) {
                    const FdkBase bb = hb[wi][q][t];
                    const float fl = bb.fb + lf;
                    const float fll = floorf(fl);
                    const int iv0 = bb.ib + (int)fll;
                    // taps clamped into the column so the loads need no branch;
                    // a voxel whose rows fall off the detector keeps its sum
                    // (lanes past nz accumulate values that are never stored)
                    const bool ok = iv0 >= -1 && iv0 <= nv - 1;
                    const int ivc = min(max(iv0, -1), nv - 1);
                    const float tv = fl - fll;
                    const float2 A = __ldg(col2 + ivc), B = __ldg(col2 + ivc + 1);  // rows iv0, iv0 + 1
                    const float lo = fmaf(tv, B.x - A.x, A.x), hi = fmaf(tv, B.y - A.y, A.y);
                    const float nxt = fmaf(p.w, fmaf(p.tu, hi - lo, lo), acc[q]);
                    acc[q] = ok ? nxt : acc[q];
                }
            }
        }
        __syncthreads();
    }
    if (!col) return;
    float *out = gzi + ((size_t)j * nx + i) * nz;
#pragma unroll
    for (int q = 0; q < FDK_KPL; ++q) {
        const int k = k0 + lane + 32 * q;
        if (k < nz) out[k] = accumulate ? out[k] + acc[q] : acc[q];
    }
}

}  // namespace

size_t fdk_filtered_elems(int n_sel, int nu, int nv) { return (size_t)n_sel * (nu + 1) * fdk_row_stride(nv) * 2; }

cudaError_t launch_fdk_filter(const void *y, int y_dtype, int n_sel, int nu, int nv, double sod, double sdd,
                              double du, double dv, float *qt, cudaStream_t st) {
    if (n_sel <= 0) return cudaSuccess;
    const double m = sod / sdd;
    const size_t smem = ((size_t)FDK_ROWS * fr_row_len(nu) + (size_t)FDK_ROWS * nu + fr_kh(nu) + 1) * sizeof(float);
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

// One launch per FDK_SUB views (accumulating into the volume): every block of a
// launch reads the same few views, whose filtered rows then stay in L2 for
// the blocks of neighbouring voxel rows (a launch over all views of a chunk
// let blocks drift apart by up to the whole chunk and re-read from DRAM).
constexpr int FDK_SUB = 32;

cudaError_t launch_fdk_bp(const float *qt, const double *view_csw, int n_sel, int nx, int ny, int nz, int nu,
                          int nv, double vx, double vy, double vz, double sod, double sdd, double du, double dv,
                          int accumulate, float *gzi, cudaStream_t st) {
    const double m = sod / sdd;
    dim3 block(32, FDK_WARPS);
    dim3 grid((nx + FDK_WARPS - 1) / FDK_WARPS, ny, (nz + 32 * FDK_KPL - 1) / (32 * FDK_KPL));
    const size_t vstride = (size_t)(nu + 1) * fdk_row_stride(nv);  // float2 entries per view
    for (int s0 = 0; s0 < n_sel; s0 += FDK_SUB) {
        const int ns = n_sel - s0 < FDK_SUB ? n_sel - s0 : FDK_SUB;
        k_fdk_bp<<<grid, block, 0, st>>>((const float2 *)qt + (size_t)s0 * vstride,
                                         (const FdkView *)view_csw + s0, ns, nx, ny, nz, nu, nv, vx, vy, vz, sod,
                                         1.0 / (du * m), 1.0 / (dv * m), 0.5 * (nu - 1), 0.5 * (nv - 1),
                                         (accumulate || s0 > 0) ? 1 : 0, gzi);
    }
    return cudaGetLastError();
}

}  // namespace fbl
