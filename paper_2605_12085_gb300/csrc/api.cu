// C ABI of the FB-LISA hot path: argument checking, geometry tables, the
// mini-batch schedule and sampling (Algorithm 1, Steps 1 and 2a), the
// line-search driver (Steps 2b-2d) and the stateless operator calls.  Every
// numeric step runs in the kernels of k_project.cu, k_backproject.cu and
// k_prox.cu; this file only prepares tables, moves data and makes the (2.3)
// decision on four FP64 scalars.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "fbl_internal.cuh"

using namespace fbl;

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
namespace {

thread_local std::string g_last_error;

fbl_status fail(fbl_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

fbl_status cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(FBL_E_NOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(FBL_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(expr, what)                                   \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool valid_dtype(int dt) { return dt == FBL_F32 || dt == FBL_BF16 || dt == FBL_F16; }

// True when p is device (or managed) memory of the current context.
bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

fbl_status check_device(int want) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (cur != want)
        return fail(FBL_E_INVAL, "object was created on device %d but device %d is current", want,
                    cur);
    return FBL_OK;
}

// Stream-ordered scratch that is released when it goes out of scope.
struct AsyncBuf {
    void *p = nullptr;
    cudaStream_t st = nullptr;
    AsyncBuf() = default;
    AsyncBuf(const AsyncBuf &) = delete;
    AsyncBuf &operator=(const AsyncBuf &) = delete;
    cudaError_t alloc(size_t bytes, cudaStream_t s) {
        st = s;
        return cudaMallocAsync(&p, bytes ? bytes : 16, s);
    }
    ~AsyncBuf() {
        if (p) cudaFreeAsync(p, st);
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
struct fbl_geometry {
    fbl_geometry_desc desc;
    std::vector<double> angles;
    int device = -1;
    DevGeom dg;
    float4 *d_colA = nullptr;
    float4 *d_colB = nullptr;
    FxCol *d_colF = nullptr;
    float2 *d_trig = nullptr;
    int *d_err = nullptr;   // status word of the TMA-staged projector's bounded waits
    int *h_err = nullptr;   // pinned mirror
};

namespace {

ZLayout layout_for(const fbl_geometry *g, int dtype) {
    const fbl_geometry_desc &d = g->desc;
    return make_layout(d.nx, d.ny, d.nz, dtype_size(dtype));
}

// After work on stream st that used the TMA-staged projector: FBL_E_TIMEOUT
// (and the word cleared) if one of its bounded waits gave up.  Synchronises st.
fbl_status check_timeout(const fbl_geometry *g, const DevGeom &dg, cudaStream_t st) {
    if (dg.k1_split != 2 || !g->d_err) return FBL_OK;
    if (cudaMemcpyAsync(g->h_err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FBL_OK;  // the caller's next CUDA call reports the error
    if (*g->h_err == 0) return FBL_OK;
    cudaMemsetAsync(g->d_err, 0, sizeof(int), st);
    return FBL_E_TIMEOUT;
}

double view_angle(const fbl_geometry_desc &d, const std::vector<double> &ang, int v) {
    return ang.empty() ? 2.0 * M_PI * (double)v / (double)d.n_views : ang[v];
}

}  // namespace

extern "C" void fbl_params_default(fbl_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->alpha0 = 1e-3;
    p->beta = 0.5;
    p->mu = 1.0;
    p->C = 1.0;
    p->eps_base = 0.99;
    p->N0 = 8;
    p->n_max = 0;
    p->max_backtracks = 60;
    p->proposal = 0;
    p->seed = 0;
    p->x_dtype = FBL_F32;
    p->b_dtype = FBL_F32;
    p->use_graph = 0;
    p->force_reject = 0;
    p->reg = FBL_REG_L1;
    p->tv_iters = 20;
    p->tv_warm = 1;
    p->x_max = INFINITY;
}

extern "C" fbl_status geometry_create(const fbl_geometry_desc *desc, fbl_geometry **out) {
    if (!desc || !out) return fail(FBL_E_INVAL, "geometry_create: null argument");
    *out = nullptr;
    const fbl_geometry_desc &d = *desc;
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || d.nu < 1 || d.nv < 1 || d.n_views < 1)
        return fail(FBL_E_INVAL, "geometry_create: sizes must be positive");
    if (!(d.vx > 0 && d.vy > 0 && d.vz > 0 && d.du > 0 && d.dv > 0 && d.sod > 0 && d.sdd > d.sod))
        return fail(FBL_E_INVAL, "geometry_create: need positive voxel/pixel sizes and 0 < SOD < SDD");
    const double rxy = 0.5 * std::sqrt((d.nx * d.vx) * (d.nx * d.vx) + (d.ny * d.vy) * (d.ny * d.vy));
    const double slack = std::max(d.vx, d.vy);
    if (!(rxy + slack < d.sod && rxy + slack < d.sdd - d.sod))
        return fail(FBL_E_UNSUPPORTED,
                    "geometry_create: the volume must lie strictly between source and detector");
    for (int es : {2, 4}) {
        const ZLayout L = make_layout(d.nx, d.ny, d.nz, es);
        if (L.elems() >= (int64_t(1) << 31))
            return fail(FBL_E_UNSUPPORTED, "geometry_create: volume too large for 32-bit indexing");
    }
    auto g = new fbl_geometry();
    g->desc = d;
    if (d.angles) {
        g->angles.assign(d.angles, d.angles + d.n_views);
        for (double a : g->angles)
            if (!std::isfinite(a)) {
                delete g;
                return fail(FBL_E_INVAL, "geometry_create: non-finite angle");
            }
    }
    g->desc.angles = nullptr;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "geometry_create: no CUDA device");
    }

    const double cu = 0.5 * (d.nu - 1), cv = 0.5 * (d.nv - 1);
    const double cxyz[3] = {0.5 * (d.nx - 1), 0.5 * (d.ny - 1), 0.5 * (d.nz - 1)};
    const double V[3] = {d.vx, d.vy, d.vz};
    const int Nn[3] = {d.nx, d.ny, d.nz};
    const double wmax = std::max(std::fabs(0.0 - cv), std::fabs(d.nv - 1 - cv)) * d.dv;
    const size_t ncol = (size_t)d.n_views * d.nu;
    std::vector<float4> colA(ncol), colB(ncol);
    std::vector<FxCol> colF(ncol);
    auto fx = [](double v) { return (long long)std::llround(v * FX_ONE); };
    std::vector<float2> trig(d.n_views);
    double hw = 0.0, max_inv = 0.0;
    for (int v = 0; v < d.n_views; ++v) {
        const double th = view_angle(d, g->angles, v);
        const double c = std::cos(th), sn = std::sin(th);
        trig[v] = make_float2((float)c, (float)sn);
        const double s[2] = {d.sod * c, d.sod * sn};
        std::vector<double> m_in_lo(d.nu), m_in_hi(d.nu), qb0v(d.nu), qb1v(d.nu);
        std::vector<int> famv(d.nu);
        for (int iu = 0; iu < d.nu; ++iu) {
            // d = P - s with P = c_det + u e_u, written in the definition's order so
            // that an exact tie |d_x| == |d_y| is decided like the definition says.
            const double u = (iu - cu) * d.du;
            const double off = d.sdd - d.sod;
            const double Px = -off * c - u * sn, Py = -off * sn + u * c;
            const double dxy[2] = {Px - s[0], Py - s[1]};
            const int fam = (std::fabs(dxy[1]) > std::fabs(dxy[0])) ? 1 : 0;
            const int a = fam, b = 1 - fam;
            if (wmax > std::fabs(dxy[a])) {
                delete g;
                return fail(FBL_E_UNSUPPORTED,
                            "geometry_create: view %d column %d has rays dominated by z", v, iu);
            }
            const double da = dxy[a], db = dxy[b];
            const double plane0 = -cxyz[a] * V[a] - s[a];  // A_0 - s_a
            const double qb1 = V[a] * db / (da * V[b]);
            const double qb0 = (s[b] + plane0 * db / da) / V[b] + cxyz[b];
            const double zc1 = V[a] / (da * V[2]);
            const double zc0 = plane0 / (da * V[2]);
            const double wa = V[a] / std::fabs(da);
            const double h2 = dxy[0] * dxy[0] + dxy[1] * dxy[1];
            colA[(size_t)v * d.nu + iu] = make_float4((float)qb0, (float)qb1, (float)zc0, (float)zc1);
            colF[(size_t)v * d.nu + iu] = FxCol{fx(qb0), fx(qb1), fx(0.5 * d.dv * zc0), fx(0.5 * d.dv * zc1)};
            colB[(size_t)v * d.nu + iu] = make_float4((float)wa, (float)h2, (float)fam, 0.f);
            famv[iu] = fam;
            // planes on which this column's crossing is inside the volume: -1 < q_b < Nb
            double mlo = 0, mhi = Nn[a] - 1;
            if (qb1 > 0) {
                mlo = std::max(mlo, (-1.0 - qb0) / qb1);
                mhi = std::min(mhi, ((double)Nn[b] - qb0) / qb1);
            } else if (qb1 < 0) {
                mlo = std::max(mlo, ((double)Nn[b] - qb0) / qb1);
                mhi = std::min(mhi, (-1.0 - qb0) / qb1);
            } else if (!(qb0 > -1.0 && qb0 < Nn[b])) {
                mlo = 1;
                mhi = 0;
            }
            m_in_lo[iu] = mlo;
            m_in_hi[iu] = mhi;
            qb0v[iu] = qb0;
            qb1v[iu] = qb1;
            // detector rows per voxel along z where the column meets the volume:
            // 1/(dv*Zc(m)), Zc affine in m
            if (mlo <= mhi)
                for (double m : {mlo, mhi}) {
                    const double Zc = zc0 + m * zc1;
                    if (Zc > 0) max_inv = std::max(max_inv, 1.0 / (d.dv * Zc));
                }
        }
        // columns per voxel in-plane (the candidate window K2 searches): the
        // inverse step of q_b between neighbouring columns, where both meet the volume
        for (int iu = 0; iu + 1 < d.nu; ++iu) {
            if (famv[iu] != famv[iu + 1]) continue;
            const double lo = std::max(m_in_lo[iu], m_in_lo[iu + 1]);
            const double hi = std::min(m_in_hi[iu], m_in_hi[iu + 1]);
            if (lo > hi) continue;
            for (double m : {lo, hi}) {
                const double dq = std::fabs((qb0v[iu + 1] + m * qb1v[iu + 1]) - (qb0v[iu] + m * qb1v[iu]));
                if (dq > 0) hw = std::max(hw, 1.0 / dq);
            }
        }
    }
    if (hw == 0.0) hw = (double)d.nu;  // a single column: take every column as a candidate
    hw = hw * 1.02 + 0.05;

    DevGeom &dg = g->dg;
    dg.nx = d.nx;
    dg.ny = d.ny;
    dg.nz = d.nz;
    dg.nu = d.nu;
    dg.nv = d.nv;
    dg.n_views = d.n_views;
    dg.cu = (float)cu;
    dg.cv = (float)cv;
    dg.du = (float)d.du;
    dg.dv = (float)d.dv;
    dg.cx = (float)cxyz[0];
    dg.cy = (float)cxyz[1];
    dg.cz = (float)cxyz[2];
    dg.vx = (float)d.vx;
    dg.vy = (float)d.vy;
    dg.vz = (float)d.vz;
    dg.sod = (float)d.sod;
    dg.sdd = (float)d.sdd;
    dg.inv_du = (float)(1.0 / d.du);
    dg.hwu = (float)hw;
    dg.cz_fx = (long long)std::llround(cxyz[2] * FX_ONE);
    dg.k1_cols = 8;
    dg.k1_split = 1;
    dg.k2_vpl = 4;
    // detector rows with a crossing in (k - 1, k + 1) on one column: at most
    // floor(2 max_inv) + 1
    dg.ntap = (int)std::floor(2.0 * max_inv * 1.0001 + 0.002) + 1;
    if (dg.ntap > RT_PAD) {
        geometry_destroy(g);
        return fail(FBL_E_UNSUPPORTED, "geometry_create: detector rows finer than %d per voxel",
                    RT_PAD);
    }

    e = cudaMalloc(&g->d_colA, ncol * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_colB, ncol * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_trig, d.n_views * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_colF, ncol * sizeof(FxCol));
    if (e == cudaSuccess) e = cudaMemcpy(g->d_colF, colF.data(), ncol * sizeof(FxCol), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_colA, colA.data(), ncol * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_colB, colB.data(), ncol * sizeof(float4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_trig, trig.data(), d.n_views * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(g->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&g->h_err, sizeof(int));
    if (e != cudaSuccess) {
        geometry_destroy(g);
        return cuda_fail(e, "geometry_create: device tables");
    }
    dg.colA = g->d_colA;
    dg.colF = g->d_colF;
    dg.colB = g->d_colB;
    dg.trig = g->d_trig;
    dg.err = g->d_err;
    *out = g;
    return FBL_OK;
}

extern "C" void geometry_destroy(fbl_geometry *g) {
    if (!g) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (g->device >= 0 && cur != g->device) cudaSetDevice(g->device);
    cudaFree(g->d_colA);
    cudaFree(g->d_colB);
    cudaFree(g->d_trig);
    cudaFree(g->d_colF);
    cudaFree(g->d_err);
    cudaFreeHost(g->h_err);
    if (g->device >= 0 && cur >= 0 && cur != g->device) cudaSetDevice(cur);
    delete g;
}

// ---------------------------------------------------------------------------
// Host helpers: Step 1 schedule and Step 2a sampling
// ---------------------------------------------------------------------------
namespace {

const uint64_t kGamma = 0x9E3779B97F4A7C15ull;
const uint64_t kEpochKey = 0xD1B54A32D192ED03ull;

// SplitMix64 output function (Steele, Lea & Flood, 2014; "variant 13" mixer).
uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void permutation(uint64_t seed, int32_t epoch, int32_t n, std::vector<int32_t> &perm) {
    const uint64_t state = seed ^ ((uint64_t)(int64_t)epoch * kEpochKey);
    perm.resize(n);
    for (int32_t i = 0; i < n; ++i) perm[i] = i;
    for (int32_t i = 0; i + 1 < n; ++i) {
        const uint64_t z = sm64_mix(state + (uint64_t)(i + 1) * kGamma);
        const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        int32_t j = i + (int32_t)std::floor(u * (double)(n - i));
        if (j > n - 1) j = n - 1;
        std::swap(perm[i], perm[j]);
    }
}

void batches(uint64_t seed, int32_t epoch, int32_t n, int32_t N_t, std::vector<int32_t> &out) {
    std::vector<int32_t> perm;
    permutation(seed, epoch, n, perm);
    const int32_t iters = (n + N_t - 1) / N_t;
    out.assign((size_t)iters * N_t, 0);
    for (int32_t it = 0; it < iters; ++it)
        for (int32_t q = 0; q < N_t; ++q) {
            const int32_t pos = it * N_t + q;
            out[pos] = pos < n ? perm[pos] : perm[pos - n];
        }
}

int32_t next_batch_size(int32_t n_theta, int32_t N0, int32_t n_max, double C, double eps_base,
                        int64_t k_hat, int32_t N_prev) {
    const int64_t K = k_hat + (n_theta + N_prev - 1) / N_prev;
    const double q = std::ceil(C / std::pow(eps_base, (double)K));
    int64_t N = q > 2e9 ? (int64_t)2e9 : (int64_t)q;
    if (N < N0) N = N0;
    if (N > n_max) N = n_max;
    return (int32_t)N;
}

}  // namespace

extern "C" fbl_status fbl_schedule(int32_t n_theta, int32_t N0, int32_t n_max, double C,
                                   double eps_base, int32_t epochs, int32_t *N_out,
                                   int32_t *iters_out) {
    if (n_theta < 1 || N0 < 1 || N0 > n_theta || epochs < 0 || !(C > 0) ||
        !(eps_base > 0 && eps_base < 1) || (epochs > 0 && (!N_out || !iters_out)))
        return fail(FBL_E_INVAL, "fbl_schedule: bad argument");
    if (n_max <= 0) n_max = n_theta;
    if (n_max < N0 || n_max > n_theta) return fail(FBL_E_INVAL, "fbl_schedule: need N0 <= n_max <= n_theta");
    int64_t k_hat = 0;
    int32_t N_prev = N0;
    for (int32_t t = 0; t < epochs; ++t) {
        const int32_t N = next_batch_size(n_theta, N0, n_max, C, eps_base, k_hat, N_prev);
        N_out[t] = N;
        iters_out[t] = (n_theta + N - 1) / N;
        k_hat += iters_out[t];
        N_prev = N;
    }
    return FBL_OK;
}

extern "C" fbl_status fbl_epoch_batches(uint64_t seed, int32_t epoch, int32_t n_theta, int32_t N_t,
                                        int32_t *views_out) {
    if (n_theta < 1 || N_t < 1 || N_t > n_theta || !views_out)
        return fail(FBL_E_INVAL, "fbl_epoch_batches: bad argument");
    std::vector<int32_t> out;
    batches(seed, epoch, n_theta, N_t, out);
    std::memcpy(views_out, out.data(), out.size() * sizeof(int32_t));
    return FBL_OK;
}

// ---------------------------------------------------------------------------
// Stateless operator calls
// ---------------------------------------------------------------------------
namespace {

fbl_status check_views(const fbl_geometry *g, const int32_t *views, int32_t n_sel) {
    if (n_sel < 0) return fail(FBL_E_INVAL, "negative view count");
    if (n_sel > 0 && !views) return fail(FBL_E_INVAL, "null view list");
    if (n_sel > 65535) return fail(FBL_E_INVAL, "at most 65535 views per call");
    for (int32_t q = 0; q < n_sel; ++q)
        if (views[q] < 0 || views[q] >= g->desc.n_views)
            return fail(FBL_E_INVAL, "view index %d out of range [0, %d)", views[q], g->desc.n_views);
    return FBL_OK;
}

// Device copy of a host view list.
fbl_status upload_views(const int32_t *views, int32_t n, AsyncBuf &buf, cudaStream_t st) {
    CK(buf.alloc((size_t)n * sizeof(int32_t), st), "view list");
    if (n) CK(cudaMemcpyAsync(buf.p, views, (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, st),
              "view list copy");
    return FBL_OK;
}

// Device pointer for a caller buffer: itself if on the device, else a staged copy.
fbl_status device_input(const void *p, size_t bytes, AsyncBuf &stage, const void **dev,
                        cudaStream_t st) {
    if (is_device_ptr(p)) {
        *dev = p;
        return FBL_OK;
    }
    CK(stage.alloc(bytes, st), "input staging");
    CK(cudaMemcpyAsync(stage.p, p, bytes, cudaMemcpyHostToDevice, st), "input H2D");
    *dev = stage.p;
    return FBL_OK;
}

// The library layout of a caller volume, stream-ordered.
fbl_status pack_volume(const fbl_geometry *g, const void *xdev, int dtype, AsyncBuf &pv,
                       ZLayout &L, cudaStream_t st) {
    L = layout_for(g, dtype);
    const size_t bytes = (size_t)L.elems() * dtype_size(dtype);
    CK(pv.alloc(bytes, st), "volume layout");
    CK(cudaMemsetAsync(pv.p, 0, bytes, st), "memset");
    CK(launch_pack(xdev, dtype, pv.p, L, st), "pack");
    return FBL_OK;
}

}  // namespace

extern "C" fbl_status project(const fbl_geometry *g, const void *x, int32_t x_dtype,
                              const int32_t *views, int32_t n_sel, void *y, int32_t y_dtype,
                              void *stream) {
    if (!g || !x || (n_sel > 0 && !y)) return fail(FBL_E_INVAL, "project: null argument");
    if (!valid_dtype(x_dtype) || !valid_dtype(y_dtype)) return fail(FBL_E_INVAL, "project: bad dtype");
    fbl_status st = check_views(g, views, n_sel);
    if (st) return st;
    if ((st = check_device(g->device))) return st;
    if (n_sel == 0) return FBL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const fbl_geometry_desc &d = g->desc;
    const size_t nvox = (size_t)d.nx * d.ny * d.nz;
    const size_t ny_out = (size_t)n_sel * d.nv * d.nu;
    AsyncBuf dviews, xs, pv, ys;
    if ((st = upload_views(views, n_sel, dviews, s))) return st;
    const void *xd = nullptr;
    if ((st = device_input(x, nvox * dtype_size(x_dtype), xs, &xd, s))) return st;
    ZLayout L;
    if ((st = pack_volume(g, xd, x_dtype, pv, L, s))) return st;
    const bool y_dev = is_device_ptr(y);
    void *yd = y;
    if (!y_dev) {
        CK(ys.alloc(ny_out * dtype_size(y_dtype), s), "output staging");
        yd = ys.p;
    }
    CK(launch_project(PROJ_STORE, g->dg, pv.p, L, x_dtype, (const int32_t *)dviews.p,
                      n_sel, nullptr, FBL_F32, nullptr, yd, y_dtype, nullptr, nullptr, s),
       "project kernel");
    if (!y_dev) {
        CK(cudaMemcpyAsync(y, yd, ny_out * dtype_size(y_dtype), cudaMemcpyDeviceToHost, s), "output D2H");
        CK(cudaStreamSynchronize(s), "project");
    }
    return FBL_OK;
}

extern "C" fbl_status fdk(const fbl_geometry *g, const void *y, int32_t y_dtype, const int32_t *views,
                          int32_t n_sel, float *x, void *stream) {
    if (!g || !x || (n_sel > 0 && !y) || (n_sel > 0 && !views)) return fail(FBL_E_INVAL, "fdk: null argument");
    if (!valid_dtype(y_dtype)) return fail(FBL_E_INVAL, "fdk: bad dtype");
    fbl_status st = check_views(g, views, n_sel);
    if (st) return st;
    if ((st = check_device(g->device))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const fbl_geometry_desc &d = g->desc;
    const size_t nvox = (size_t)d.nx * d.ny * d.nz;
    const bool x_dev = is_device_ptr(x);
    AsyncBuf xs, gz, qt, vbuf, ys;
    float *xd = x;
    if (!x_dev) {
        CK(xs.alloc(nvox * sizeof(float), s), "output staging");
        xd = (float *)xs.p;
    }
    if (n_sel == 0) {
        CK(cudaMemsetAsync(xd, 0, nvox * sizeof(float), s), "memset");
    } else {
        // dtheta of each selected view: half the circular gaps to its neighbours
        std::vector<std::pair<double, int>> ang(n_sel);
        for (int q = 0; q < n_sel; ++q) {
            double a = std::fmod(view_angle(d, g->angles, views[q]), 2.0 * M_PI);
            if (a < 0) a += 2.0 * M_PI;
            ang[q] = {a, q};
        }
        std::sort(ang.begin(), ang.end());
        std::vector<double> csw(3 * (size_t)n_sel);
        for (int r = 0; r < n_sel; ++r) {
            const int q = ang[r].second;
            double w = 2.0 * M_PI;
            if (n_sel > 1) {
                const double nxt = r + 1 < n_sel ? ang[r + 1].first : ang[0].first + 2.0 * M_PI;
                const double prv = r > 0 ? ang[r - 1].first : ang[n_sel - 1].first - 2.0 * M_PI;
                w = 0.5 * (nxt - prv);
            }
            const double th = view_angle(d, g->angles, views[q]);
            csw[3 * q + 0] = std::cos(th);
            csw[3 * q + 1] = std::sin(th);
            csw[3 * q + 2] = 0.5 * w;
        }
        CK(vbuf.alloc(csw.size() * sizeof(double), s), "view table");
        CK(cudaMemcpyAsync(vbuf.p, csw.data(), csw.size() * sizeof(double), cudaMemcpyHostToDevice, s),
           "view table");
        const size_t per_view_in = (size_t)d.nv * d.nu * dtype_size(y_dtype);
        const void *yd = nullptr;
        if ((st = device_input(y, per_view_in * n_sel, ys, &yd, s))) return st;
        const int chunk = std::min<int>(n_sel, 256);  // bounds the filtered-projection scratch
        CK(qt.alloc(fdk_filtered_elems(chunk, d.nu, d.nv) * sizeof(float), s), "filtered projections");
        CK(gz.alloc(nvox * sizeof(float), s), "volume scratch");
        for (int v0 = 0; v0 < n_sel; v0 += chunk) {
            const int nc = std::min(chunk, n_sel - v0);
            CK(cudaMemsetAsync(qt.p, 0, fdk_filtered_elems(nc, d.nu, d.nv) * sizeof(float), s), "memset");
            CK(launch_fdk_filter((const char *)yd + per_view_in * v0, y_dtype, nc, d.nu, d.nv, d.sod, d.sdd, d.du,
                                 d.dv, (float *)qt.p, s),
               "fdk filter kernel");
            CK(launch_fdk_bp((const float *)qt.p, (const double *)vbuf.p + 3 * (size_t)v0, nc, d.nx, d.ny, d.nz,
                             d.nu, d.nv, d.vx, d.vy, d.vz, d.sod, d.sdd, d.du, d.dv, v0 > 0 ? 1 : 0,
                             (float *)gz.p, s),
               "fdk backprojection kernel");
        }
        CK(launch_zi_to_natural((const float *)gz.p, xd, d.nx, d.ny, d.nz, 0, s), "reorder");
    }
    if (!x_dev) {
        CK(cudaMemcpyAsync(x, xd, nvox * sizeof(float), cudaMemcpyDeviceToHost, s), "x D2H");
        CK(cudaStreamSynchronize(s), "fdk");
    }
    return FBL_OK;
}

extern "C" fbl_status backproject(const fbl_geometry *g, const void *y, int32_t y_dtype,
                                  const int32_t *views, int32_t n_sel, float *x,
                                  int32_t accumulate, void *stream) {
    if (!g || !x || (n_sel > 0 && !y)) return fail(FBL_E_INVAL, "backproject: null argument");
    if (!valid_dtype(y_dtype)) return fail(FBL_E_INVAL, "backproject: bad dtype");
    fbl_status st = check_views(g, views, n_sel);
    if (st) return st;
    if ((st = check_device(g->device))) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const fbl_geometry_desc &d = g->desc;
    const size_t nvox = (size_t)d.nx * d.ny * d.nz;
    const size_t ny_in = (size_t)n_sel * d.nv * d.nu;
    const bool x_dev = is_device_ptr(x);
    AsyncBuf dviews, ys, rt, xs, gz;
    float *xd = x;
    if (!x_dev) {
        CK(xs.alloc(nvox * sizeof(float), s), "output staging");
        xd = (float *)xs.p;
        if (accumulate) CK(cudaMemcpyAsync(xd, x, nvox * sizeof(float), cudaMemcpyHostToDevice, s), "x H2D");
    }
    if (n_sel == 0) {
        if (!accumulate) CK(cudaMemsetAsync(xd, 0, nvox * sizeof(float), s), "memset");
    } else {
        if ((st = upload_views(views, n_sel, dviews, s))) return st;
        const void *yd = nullptr;
        if ((st = device_input(y, ny_in * dtype_size(y_dtype), ys, &yd, s))) return st;
        const size_t rt_elems = (size_t)n_sel * d.nu * rt_pitch(d.nv);
        CK(rt.alloc(rt_elems * sizeof(float), s), "weighted sinogram");
        CK(cudaMemsetAsync(rt.p, 0, rt_elems * sizeof(float), s), "memset");
        CK(launch_weight(g->dg, yd, y_dtype, (const int32_t *)dviews.p, n_sel, (float *)rt.p, s),
           "weight kernel");
        CK(gz.alloc(nvox * sizeof(float), s), "gradient scratch");
        CK(launch_backproject(g->dg, (const float *)rt.p, (const int32_t *)dviews.p, n_sel, 1.0f,
                              (float *)gz.p, s),
           "backproject kernel");
        CK(launch_zi_to_natural((const float *)gz.p, xd, d.nx, d.ny, d.nz, accumulate, s), "reorder");
    }
    if (!x_dev) {
        CK(cudaMemcpyAsync(x, xd, nvox * sizeof(float), cudaMemcpyDeviceToHost, s), "x D2H");
        CK(cudaStreamSynchronize(s), "backproject");
    }
    return FBL_OK;
}

namespace {

// The listed views of b gathered into a batch on the device (b on the host),
// or b itself with a device view map (b on the device).
fbl_status batch_data(const fbl_geometry *g, const void *b, int b_dtype, const int32_t *views_h,
                      const int32_t *views_d, int32_t n_sel, AsyncBuf &stage, const void **bd,
                      const int32_t **bmap, cudaStream_t s) {
    const fbl_geometry_desc &d = g->desc;
    const size_t per_view = (size_t)d.nv * d.nu * dtype_size(b_dtype);
    if (is_device_ptr(b)) {
        *bd = b;
        *bmap = views_d;
        return FBL_OK;
    }
    CK(stage.alloc(per_view * n_sel, s), "data staging");
    for (int32_t q = 0; q < n_sel; ++q)
        CK(cudaMemcpyAsync((char *)stage.p + per_view * q, (const char *)b + per_view * views_h[q],
                           per_view, cudaMemcpyHostToDevice, s),
           "data H2D");
    *bd = stage.p;
    *bmap = nullptr;
    return FBL_OK;
}

}  // namespace

extern "C" fbl_status residual_norm(const fbl_geometry *g, const void *x, int32_t x_dtype,
                                    const int32_t *views, int32_t n_sel, const void *b,
                                    int32_t b_dtype, double *rho_host, void *stream) {
    if (!g || !x || (n_sel > 0 && !b) || !rho_host)
        return fail(FBL_E_INVAL, "residual_norm: null argument");
    if (!valid_dtype(x_dtype) || !valid_dtype(b_dtype)) return fail(FBL_E_INVAL, "residual_norm: bad dtype");
    fbl_status st = check_views(g, views, n_sel);
    if (st) return st;
    if ((st = check_device(g->device))) return st;
    if (n_sel == 0) {
        *rho_host = 0.0;
        return FBL_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const fbl_geometry_desc &d = g->desc;
    const size_t nvox = (size_t)d.nx * d.ny * d.nz;
    AsyncBuf dviews, xs, pv, bs, part, res;
    if ((st = upload_views(views, n_sel, dviews, s))) return st;
    const void *xd = nullptr;
    if ((st = device_input(x, nvox * dtype_size(x_dtype), xs, &xd, s))) return st;
    ZLayout L;
    if ((st = pack_volume(g, xd, x_dtype, pv, L, s))) return st;
    const void *bd = nullptr;
    const int32_t *bmap = nullptr;
    if ((st = batch_data(g, b, b_dtype, views, (const int32_t *)dviews.p, n_sel, bs, &bd, &bmap, s)))
        return st;
    const int np = project_num_partials(g->dg, n_sel);
    CK(part.alloc((size_t)np * sizeof(double), s), "partials");
    CK(res.alloc(sizeof(double), s), "result");
    CK(launch_project(PROJ_NORM, g->dg, pv.p, L, x_dtype, (const int32_t *)dviews.p, n_sel,
                      bd, b_dtype, bmap, nullptr, FBL_F32, (double *)part.p, nullptr, s),
       "objective kernel");
    CK(launch_reduce((const double *)part.p, np, np, 1, (double *)res.p, s), "reduce");
    CK(cudaMemcpyAsync(rho_host, res.p, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
    CK(cudaStreamSynchronize(s), "residual_norm");
    if (!std::isfinite(*rho_host)) return fail(FBL_E_NONFINITE, "residual_norm: non-finite result");
    if ((st = check_timeout(g, g->dg, s))) return fail(st, "residual_norm: a bounded wait of the projector gave up");
    return FBL_OK;
}

extern "C" fbl_status evaluate(const fbl_geometry *g, const void *x, int32_t x_dtype, const void *b,
                               int32_t b_dtype, double mu, const void *x_true, double *out3_host,
                               void *stream) {
    if (!g || !x || !b || !out3_host) return fail(FBL_E_INVAL, "evaluate: null argument");
    if (!valid_dtype(x_dtype) || !valid_dtype(b_dtype)) return fail(FBL_E_INVAL, "evaluate: bad dtype");
    fbl_status st = check_device(g->device);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const fbl_geometry_desc &d = g->desc;
    const size_t nvox = (size_t)d.nx * d.ny * d.nz;
    const size_t xbytes = nvox * dtype_size(x_dtype);
    AsyncBuf xs, xts, pv, dviews, bs, part, res;
    const void *xd = nullptr, *xtd = nullptr;
    if ((st = device_input(x, xbytes, xs, &xd, s))) return st;
    if (x_true && (st = device_input(x_true, xbytes, xts, &xtd, s))) return st;
    ZLayout L;
    if ((st = pack_volume(g, xd, x_dtype, pv, L, s))) return st;
    std::vector<int32_t> all(d.n_views);
    for (int v = 0; v < d.n_views; ++v) all[v] = v;
    if ((st = upload_views(all.data(), d.n_views, dviews, s))) return st;
    const bool b_dev = is_device_ptr(b);
    const int chunk = std::min(d.n_views, 256);
    const int npmax = std::max(project_num_partials(g->dg, chunk), 3 * prox_flat_num_partials((int64_t)nvox));
    const int nchunks = (d.n_views + chunk - 1) / chunk;
    CK(part.alloc((size_t)npmax * sizeof(double), s), "partials");
    CK(res.alloc((size_t)(nchunks + 3) * sizeof(double), s), "results");
    const size_t per_view = (size_t)d.nv * d.nu * dtype_size(b_dtype);
    if (!b_dev) CK(bs.alloc(per_view * chunk, s), "data staging");
    for (int c = 0; c < nchunks; ++c) {
        const int v0 = c * chunk, nsel = std::min(chunk, d.n_views - v0);
        const void *bd = b;
        const int32_t *bmap = (const int32_t *)dviews.p + v0;
        if (!b_dev) {
            CK(cudaMemcpyAsync(bs.p, (const char *)b + per_view * v0, per_view * nsel,
                               cudaMemcpyHostToDevice, s),
               "data H2D");
            bd = bs.p;
            bmap = nullptr;
        }
        int np = 0;
        CK(launch_project(PROJ_NORM, g->dg, pv.p, L, x_dtype, (const int32_t *)dviews.p + v0, nsel, bd,
                          b_dtype, bmap, nullptr, FBL_F32, (double *)part.p, &np, s),
           "objective kernel");
        CK(launch_reduce((const double *)part.p, np, np, 1, (double *)res.p + c, s), "reduce");
    }
    int nn = 0;
    CK(launch_norms(xd, xtd, x_dtype, (int64_t)nvox, (double *)part.p, &nn, s), "norms kernel");
    CK(launch_reduce((const double *)part.p, nn, nn, 3, (double *)res.p + nchunks, s), "reduce");
    std::vector<double> h(nchunks + 3);
    CK(cudaMemcpyAsync(h.data(), res.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
    CK(cudaStreamSynchronize(s), "evaluate");
    if ((st = check_timeout(g, g->dg, s))) return fail(st, "evaluate: a bounded wait of the projector gave up");
    double rho = 0.0;
    for (int c = 0; c < nchunks; ++c) rho += h[c];
    out3_host[1] = 0.5 * rho;
    out3_host[0] = 0.5 * rho + mu * h[nchunks];
    out3_host[2] = x_true ? (h[nchunks + 2] > 0 ? std::sqrt(h[nchunks + 1] / h[nchunks + 2]) : 0.0) : 0.0;
    if (!std::isfinite(out3_host[0])) return fail(FBL_E_NONFINITE, "evaluate: non-finite objective");
    return FBL_OK;
}

extern "C" fbl_status prox_reduce(const void *x, int32_t x_dtype, const float *gr, int64_t n,
                                  double alpha, double mu, void *xbar, double *out3_host,
                                  void *stream) {
    if (!out3_host) return fail(FBL_E_INVAL, "prox_reduce: null argument");
    if (!valid_dtype(x_dtype)) return fail(FBL_E_INVAL, "prox_reduce: bad dtype");
    if (n < 0) return fail(FBL_E_INVAL, "prox_reduce: negative size");
    if (n == 0) {  // empty sums; the buffers (possibly NULL) are not touched
        out3_host[0] = out3_host[1] = out3_host[2] = 0.0;
        return FBL_OK;
    }
    if (!x || !gr || !xbar) return fail(FBL_E_INVAL, "prox_reduce: null argument");
    if (x == xbar) return fail(FBL_E_INVAL, "prox_reduce: x_bar must not alias x");
    if (!(alpha > 0) || !std::isfinite(alpha) || !std::isfinite(mu))
        return fail(FBL_E_INVAL, "prox_reduce: need alpha > 0 and finite mu");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t es = dtype_size(x_dtype);
    AsyncBuf xs, gs, xbs, part, res;
    const void *xd = nullptr;
    const void *gd = nullptr;
    fbl_status st;
    if ((st = device_input(x, (size_t)n * es, xs, &xd, s))) return st;
    if ((st = device_input(gr, (size_t)n * sizeof(float), gs, &gd, s))) return st;
    const bool xb_dev = is_device_ptr(xbar);
    void *xbd = xbar;
    if (!xb_dev) {
        CK(xbs.alloc((size_t)n * es, s), "output staging");
        xbd = xbs.p;
    }
    const int np = prox_flat_num_partials(n);
    CK(part.alloc((size_t)np * 3 * sizeof(double), s), "partials");
    CK(res.alloc(3 * sizeof(double), s), "result");
    CK(launch_prox_flat(xd, (const float *)gd, n, (float)alpha, (float)(alpha * mu), xbd, x_dtype,
                        (double *)part.p, nullptr, s),
       "prox kernel");
    CK(launch_reduce((const double *)part.p, np, np, 3, (double *)res.p, s), "reduce");
    CK(cudaMemcpyAsync(out3_host, res.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
    if (!xb_dev) CK(cudaMemcpyAsync(xbar, xbd, (size_t)n * es, cudaMemcpyDeviceToHost, s), "x_bar D2H");
    CK(cudaStreamSynchronize(s), "prox_reduce");
    return FBL_OK;
}

extern "C" fbl_status prox_tv(const int32_t dims[3], const float *v, double lambda, double x_max, int32_t iters,
                              float *q, int32_t q_in, float *x, void *stream) {
    if (!dims || !v || !x || (q_in && !q)) return fail(FBL_E_INVAL, "prox_tv: null argument");
    const int nx = dims[0], ny = dims[1], nz = dims[2];
    if (!tv_dims_ok(nx, ny, nz)) return fail(FBL_E_INVAL, "prox_tv: need dims > 0 and ny, nz <= 65535");
    if (!(lambda >= 0) || !std::isfinite(lambda) || !(x_max > 0) || iters < 0 || iters > 100000)
        return fail(FBL_E_INVAL, "prox_tv: need lambda >= 0, x_max > 0, 0 <= iters <= 100000");
    if ((const void *)x == (const void *)v) return fail(FBL_E_INVAL, "prox_tv: x must not alias v");
    if (q && ((const void *)q == (const void *)v || q == x)) return fail(FBL_E_INVAL, "prox_tv: q must not alias v or x");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)nx * ny * nz;
    AsyncBuf vs, scratch, xs;
    const void *vd = nullptr;
    fbl_status st;
    if ((st = device_input(v, n * sizeof(float), vs, &vd, s))) return st;
    // two dual pairs: (caller's device q or scratch, r0), (q1, r1); and y
    const bool q_dev = q && is_device_ptr(q);
    CK(scratch.alloc((q_dev ? 10 : 13) * n * sizeof(float), s), "scratch");
    float *base = (float *)scratch.p;
    float *const qp[2] = {q_dev ? q : base + 10 * n, base + 3 * n};
    float *const rp[2] = {base, base + 6 * n};
    float *y = base + 9 * n;
    const float *q_start = nullptr;
    if (q_in) {
        if (!q_dev) CK(cudaMemcpyAsync(qp[0], q, 3 * n * sizeof(float), cudaMemcpyHostToDevice, s), "q H2D");
        q_start = qp[0];
    }
    const bool x_dev = is_device_ptr(x);
    float *xd = x;
    if (!x_dev) {
        CK(xs.alloc(n * sizeof(float), s), "output staging");
        xd = (float *)xs.p;
    }
    int cur = 1;  // the start goes to pair 1 (it reads pair 0's q)
    CK(launch_tv_prox((const float *)vd, nx, ny, nz, (float)lambda, (float)x_max, iters, q_start, qp, rp, y, xd,
                      &cur, s),
       "TV prox kernels");
    if (q) {
        if (q_dev && cur != 0)
            CK(cudaMemcpyAsync(q, qp[cur], 3 * n * sizeof(float), cudaMemcpyDeviceToDevice, s), "q copy");
        if (!q_dev) CK(cudaMemcpyAsync(q, qp[cur], 3 * n * sizeof(float), cudaMemcpyDeviceToHost, s), "q D2H");
    }
    if (!x_dev) CK(cudaMemcpyAsync(x, xd, n * sizeof(float), cudaMemcpyDeviceToHost, s), "x D2H");
    if (!x_dev || (q && !q_dev) || !is_device_ptr(v)) CK(cudaStreamSynchronize(s), "prox_tv");
    return FBL_OK;
}

extern "C" fbl_status tv_norm(const int32_t dims[3], const float *x, double *out_host, void *stream) {
    if (!dims || !x || !out_host) return fail(FBL_E_INVAL, "tv_norm: null argument");
    const int nx = dims[0], ny = dims[1], nz = dims[2];
    if (!tv_dims_ok(nx, ny, nz)) return fail(FBL_E_INVAL, "tv_norm: need dims > 0 and ny, nz <= 65535");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = (size_t)nx * ny * nz;
    AsyncBuf xs, part, res;
    const void *xd = nullptr;
    fbl_status st;
    if ((st = device_input(x, n * sizeof(float), xs, &xd, s))) return st;
    const int np = tv_norm_num_partials(nx, ny, nz);
    CK(part.alloc((size_t)np * sizeof(double), s), "partials");
    CK(res.alloc(sizeof(double), s), "result");
    CK(launch_tv_norm((const float *)xd, nx, ny, nz, (double *)part.p, s), "TV norm kernel");
    CK(launch_reduce((const double *)part.p, np, np, 1, (double *)res.p, s), "reduce");
    CK(cudaMemcpyAsync(out_host, res.p, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
    CK(cudaStreamSynchronize(s), "tv_norm");
    return FBL_OK;
}

// ---------------------------------------------------------------------------
// Solver: Algorithm 1
// ---------------------------------------------------------------------------
struct fbl_solver {
    const fbl_geometry *g = nullptr;
    DevGeom dg;                   // the geometry's tables with this solver's launch configuration
    fbl_params p;
    int device = -1;
    int32_t n_max = 0;
    // schedule / sampling state
    int32_t epoch = 0;            // t of the current epoch (0: none started)
    int32_t N_t = 0, N_prev = 0;
    int32_t iters_epoch = 0, iter_in_epoch = 0;
    int64_t k = 0, k_hat = 0;
    std::vector<int32_t> epoch_views;
    std::vector<int32_t> last_batch;
    // device state
    ZLayout L;                     // z-innermost layout of the iterates
    size_t vol_bytes = 0;
    void *st = nullptr, *tr = nullptr;  // current iterate x and trial point x_bar
    float *grad = nullptr;              // gradient, [j][i][k]
    float *rt = nullptr;                // weighted residual rt[s][iu][RT_PAD + iv]
    size_t rt_cap = 0;
    void *bstage = nullptr;
    size_t bstage_cap = 0;
    void *xstage = nullptr;
    int32_t *d_views = nullptr;
    int32_t *h_views = nullptr;   // pinned
    double *partials = nullptr;
    size_t partials_cap = 0;
    double *d_sc = nullptr;       // [8] device scalars
    double *h_sc = nullptr;       // [8] pinned
    // profiling: launch counts always, CUDA-event times when enabled
    bool prof_on = false;
    double prof_ms[FBL_PROF_CLASSES] = {};
    int64_t prof_launches[FBL_PROF_CLASSES] = {};
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_next = 0;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
    // graph mode: one executable graph per (batch size, data pointer, buffer parity)
    struct GraphEntry {
        int N;
        const void *bd;
        const int32_t *bmap;
        void *st, *tr;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;
    cudaStream_t cap = nullptr, cap2 = nullptr;  // capture streams
    LSState *d_ls = nullptr;                      // line-search state (device)
    LSState *h_ls = nullptr;                      // its host copy (pinned)
    // step proposal: statistics of the previous iteration and the network
    PropState *d_ps = nullptr;
    PropState *h_ps = nullptr;                    // pinned mirror (host-loop mode)
    float *d_mlp = nullptr;                       // network parameters, NULL until set
    float margin = 0.25f;
    // TV prox (reg = FBL_REG_TV): b, y, then (q[3], r[3]) twice, consecutive FP32 volumes
    float *tv_buf = nullptr;
    int tv_cur = 0;                               // the pair holding the previous prox's dual
    bool tv_have_q = false;
};

namespace {

// Step 2c's forward-backward point x_bar = prox_{alpha R}(x - alpha g) into
// s->tr, with the partial sums of (2.3): the l1 prox (with the box), or the
// TV prox by FGP iterations from the previous call's dual.
cudaError_t solver_prox(fbl_solver *s, double alpha, int *npp, cudaStream_t st) {
    const int xdt = s->p.x_dtype;
    if (s->p.reg != FBL_REG_TV)
        return launch_prox_zi(s->st, s->L, s->grad, (float)alpha, (float)(alpha * s->p.mu), (float)s->p.x_max,
                              s->tr, xdt, s->partials, npp, st);
    const size_t n = (size_t)s->L.nx * s->L.ny * s->L.nz;
    float *b = s->tv_buf, *y = b + n;
    float *const q[2] = {y + n, y + 7 * n}, *const r[2] = {y + 4 * n, y + 10 * n};
    const int warm = s->p.tv_warm && s->tv_have_q;
    cudaError_t e = launch_tv_prox_zi(s->st, s->L, s->grad, (float)alpha, (float)(alpha * s->p.mu),
                                      (float)s->p.x_max, s->p.tv_iters, warm, b, q, r, &s->tv_cur, y, s->tr, xdt,
                                      s->partials, npp, st);
    if (e == cudaSuccess) s->tv_have_q = true;
    return e;
}

void solver_free(fbl_solver *s) {
    cudaFree(s->st);
    cudaFree(s->tr);
    cudaFree(s->grad);
    cudaFree(s->tv_buf);
    cudaFree(s->rt);
    cudaFree(s->bstage);
    cudaFree(s->xstage);
    cudaFree(s->d_views);
    cudaFree(s->partials);
    cudaFree(s->d_sc);
    cudaFreeHost(s->h_views);
    cudaFreeHost(s->h_sc);
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    s->ev_pool.clear();
    for (auto &ge : s->graphs) cudaGraphExecDestroy(ge.exec);
    s->graphs.clear();
    if (s->cap) cudaStreamDestroy(s->cap);
    if (s->cap2) cudaStreamDestroy(s->cap2);
    cudaFree(s->d_ls);
    cudaFreeHost(s->h_ls);
    cudaFree(s->d_ps);
    cudaFreeHost(s->h_ps);
    cudaFree(s->d_mlp);
}

cudaEvent_t prof_event(fbl_solver *s) {
    if (s->ev_next == s->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        s->ev_pool.push_back(e);
    }
    return s->ev_pool[s->ev_next++];
}

// Launch a kernel of class cls, counted, and bracketed by events when profiling.
template <class F>
cudaError_t prof_launch(fbl_solver *s, int cls, cudaStream_t st, F &&launch) {
    s->prof_launches[cls] += 1;
    if (!s->prof_on) return launch();
    cudaEvent_t a = prof_event(s), b = prof_event(s);
    if (!a || !b) return launch();
    cudaEventRecord(a, st);
    cudaError_t e = launch();
    cudaEventRecord(b, st);
    s->ev_pending.push_back({cls, {a, b}});
    return e;
}

// After a stream synchronisation: fold the completed event pairs into the totals.
void prof_flush(fbl_solver *s) {
    for (auto &pe : s->ev_pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess)
            s->prof_ms[pe.first] += ms;
    }
    s->ev_pending.clear();
    s->ev_next = 0;
}

void drop_graphs(fbl_solver *s) {
    for (auto &ge : s->graphs) cudaGraphExecDestroy(ge.exec);
    s->graphs.clear();
}

fbl_status ensure_batch_buffers(fbl_solver *s, int32_t N) {
    const fbl_geometry_desc &d = s->g->desc;
    const size_t need = (size_t)N * d.nu * rt_pitch(d.nv);
    if (need > s->rt_cap) {
        drop_graphs(s);  // captured graphs hold the old addresses
        cudaFree(s->rt);
        s->rt = nullptr;
        s->rt_cap = 0;
        CK(cudaMalloc(&s->rt, need * sizeof(float)), "residual buffer");
        CK(cudaMemset(s->rt, 0, need * sizeof(float)), "residual buffer");  // zero row pads
        s->rt_cap = need;
    }
    const size_t np = std::max({(size_t)project_num_partials(s->dg, N),
                                (size_t)3 * prox_zi_num_partials(d.nx, d.ny, d.nz),
                                (size_t)backproject_num_partials(s->dg)});
    if (np > s->partials_cap) {
        drop_graphs(s);
        cudaFree(s->partials);
        s->partials = nullptr;
        s->partials_cap = 0;
        CK(cudaMalloc(&s->partials, np * sizeof(double)), "partials");
        s->partials_cap = np;
    }
    return FBL_OK;
}

// Step 1 (and Step 3 for the epoch just finished) when an epoch ends.
void begin_epoch_if_needed(fbl_solver *s) {
    if (s->epoch > 0 && s->iter_in_epoch < s->iters_epoch) return;
    const fbl_geometry_desc &d = s->g->desc;
    if (s->epoch > 0) s->k_hat = s->k;
    const int32_t prev = s->epoch > 0 ? s->N_t : s->p.N0;
    s->N_t = next_batch_size(d.n_views, s->p.N0, s->n_max, s->p.C, s->p.eps_base, s->k_hat, prev);
    s->N_prev = prev;
    s->epoch += 1;
    s->iters_epoch = (d.n_views + s->N_t - 1) / s->N_t;
    s->iter_in_epoch = 0;
    batches(s->p.seed, s->epoch, d.n_views, s->N_t, s->epoch_views);
}

// Capture one FB-LISA iteration (Steps 2b-2c) as a graph: residual,
// gradient, line-search init, then a WHILE node whose body is one trial
// (prox, reductions, trial objective, decision), then the copy of the
// line-search state to the host.
fbl_status build_graph(fbl_solver *s, fbl_solver::GraphEntry &ge) {
    const fbl_geometry_desc &d = s->g->desc;
    if (!s->cap) CK(cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking), "capture stream");
    if (!s->cap2) CK(cudaStreamCreateWithFlags(&s->cap2, cudaStreamNonBlocking), "capture stream");
    const int xdt = s->p.x_dtype, N = ge.N;
    const float scale = (float)((double)d.n_views / (double)N);
    cudaStream_t cs = s->cap, cb = s->cap2;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "begin capture");
    int np = 0, npp = 0, np2 = 0;
    cudaError_t e = launch_project(PROJ_RESID, s->dg, ge.st, s->L, xdt, s->d_views, N, ge.bd,
                                   s->p.b_dtype, ge.bmap, s->rt, FBL_F32, s->partials, &np, cs);
    if (e == cudaSuccess) e = launch_reduce(s->partials, np, np, 1, s->d_sc + 0, cs);
    if (e == cudaSuccess) e = launch_backproject(s->dg, s->rt, s->d_views, N, scale, s->grad, cs, s->partials);
    const int nbp = backproject_num_partials(s->dg);
    if (e == cudaSuccess) e = launch_reduce(s->partials, nbp, nbp, 1, s->d_sc + 5, cs);
    if (e == cudaSuccess) e = launch_propose(s->d_ls, s->d_ps, s->d_sc, s->p.proposal ? s->d_mlp : nullptr, s->margin, cs);
    if (e == cudaSuccess) e = launch_ls_init(s->d_ls, cs);
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps);
    cudaGraphConditionalHandle cond = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, cg, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &cp);
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cb, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t eb = launch_prox_zi_dev(ge.st, s->L, s->grad, s->d_ls, ge.tr, xdt, s->partials, &npp, cb);
            if (eb == cudaSuccess) eb = launch_reduce(s->partials, npp, npp, 3, s->d_sc + 1, cb);
            if (eb == cudaSuccess)
                eb = launch_project(PROJ_NORM, s->dg, ge.tr, s->L, xdt, s->d_views, N, ge.bd, s->p.b_dtype,
                                    ge.bmap, nullptr, FBL_F32, s->partials, &np2, cb);
            if (eb == cudaSuccess) eb = launch_reduce(s->partials, np2, np2, 1, s->d_sc + 4, cb);
            if (eb == cudaSuccess) eb = launch_ls_decide(s->d_ls, s->d_ps, s->d_sc, cond, cb);
            cudaError_t ee = cudaStreamEndCapture(cb, &body);
            e = eb != cudaSuccess ? eb : ee;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->h_ls, s->d_ls, sizeof(LSState), cudaMemcpyDeviceToHost, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture of the iteration");
    return FBL_OK;
}

// One iteration of Algorithm 1 on the solver's state (s->st).
fbl_status solver_iterate(fbl_solver *s, const void *b, bool b_dev, fbl_step_stats *stats,
                          cudaStream_t st) {
    const fbl_geometry *g = s->g;
    const fbl_geometry_desc &d = g->desc;
    // Remember the schedule position so that a failed iteration leaves it unchanged.
    const int32_t save_epoch = s->epoch, save_N = s->N_t, save_Np = s->N_prev;
    const int32_t save_iters = s->iters_epoch, save_it = s->iter_in_epoch;
    const int64_t save_khat = s->k_hat;
    std::vector<int32_t> save_views;
    const bool new_epoch = !(s->epoch > 0 && s->iter_in_epoch < s->iters_epoch);
    if (new_epoch) save_views = s->epoch_views;
    begin_epoch_if_needed(s);
    auto restore = [&]() {
        s->epoch = save_epoch;
        s->N_t = save_N;
        s->N_prev = save_Np;
        s->iters_epoch = save_iters;
        s->iter_in_epoch = save_it;
        s->k_hat = save_khat;
        if (new_epoch) s->epoch_views = save_views;
    };
    const int32_t N = s->N_t;
    if (s->p.proposal && !s->d_mlp) {
        restore();
        return fail(FBL_E_INVAL, "fblisa_step: proposal enabled but no network set (fblisa_set_proposal)");
    }
    fbl_status rc = ensure_batch_buffers(s, N);
    if (rc) {
        restore();
        return rc;
    }
    const int32_t *views = s->epoch_views.data() + (size_t)s->iter_in_epoch * N;
    std::memcpy(s->h_views, views, N * sizeof(int32_t));
    s->last_batch.assign(views, views + N);
    CK(cudaMemcpyAsync(s->d_views, s->h_views, N * sizeof(int32_t), cudaMemcpyHostToDevice, st),
       "view list");
    const void *bd = b;
    const int32_t *bmap = s->d_views;
    if (!b_dev) {
        const size_t per_view = (size_t)d.nv * d.nu * dtype_size(s->p.b_dtype);
        if (per_view * N > s->bstage_cap) {
            drop_graphs(s);
            cudaFree(s->bstage);
            s->bstage = nullptr;
            s->bstage_cap = 0;
            cudaError_t e = cudaMalloc(&s->bstage, per_view * N);
            if (e != cudaSuccess) {
                restore();
                return cuda_fail(e, "data staging");
            }
            s->bstage_cap = per_view * N;
        }
        for (int32_t q = 0; q < N; ++q)
            CK(cudaMemcpyAsync((char *)s->bstage + per_view * q, (const char *)b + per_view * views[q],
                               per_view, cudaMemcpyHostToDevice, st),
               "data H2D");
        bd = s->bstage;
        bmap = nullptr;
    }
    const int xdt = s->p.x_dtype;
    const double scale = (double)d.n_views / (double)N;
    if (s->p.fixed_step) {
        // forward-backward with the constant step alpha0 and no test of (2.3)
        int np = 0, npp = 0;
        CK(prof_launch(s, 0, st, [&] {
               return launch_project(PROJ_RESID, s->dg, s->st, s->L, xdt, s->d_views, N, bd, s->p.b_dtype,
                                     bmap, s->rt, FBL_F32, s->partials, &np, st);
           }),
           "residual kernel");
        CK(prof_launch(s, 4, st, [&] { return launch_reduce(s->partials, np, np, 1, s->d_sc + 0, st); }),
           "reduce");
        CK(prof_launch(s, 2, st, [&] {
               return launch_backproject(s->dg, s->rt, s->d_views, N, (float)scale, s->grad, st, s->partials);
           }),
           "gradient kernel");
        const int nbp = backproject_num_partials(s->dg);
        CK(prof_launch(s, 4, st, [&] { return launch_reduce(s->partials, nbp, nbp, 1, s->d_sc + 5, st); }),
           "reduce");
        const double alpha = s->p.alpha0;
        CK(prof_launch(s, 3, st, [&] { return solver_prox(s, alpha, &npp, st); }), "prox kernel");
        CK(prof_launch(s, 4, st, [&] { return launch_reduce(s->partials, npp, npp, 3, s->d_sc + 1, st); }),
           "reduce");
        CK(cudaMemcpyAsync(s->h_sc, s->d_sc, 6 * sizeof(double), cudaMemcpyDeviceToHost, st), "D2H");
        CK(cudaStreamSynchronize(st), "fixed step");
        prof_flush(s);
        const double f_x = 0.5 * scale * s->h_sc[0];
        if (!std::isfinite(f_x) || !std::isfinite(s->h_sc[2])) {
            restore();
            return fail(FBL_E_NONFINITE, "fblisa_step: non-finite objective or reduction at k=%lld",
                        (long long)s->k);
        }
        if (check_timeout(g, s->dg, st)) {
            restore();
            return fail(FBL_E_TIMEOUT, "fblisa_step: a bounded wait of the projector gave up");
        }
        if (stats) {
            std::memset(stats, 0, sizeof *stats);
            stats->k = s->k;
            stats->epoch = s->epoch;
            stats->N_t = N;
            stats->alpha = alpha;
            stats->alpha_init = alpha;
            stats->rho0 = s->h_sc[0];
            stats->f_x = f_x;
            stats->f_xbar = std::nan("");
            stats->gTd = s->h_sc[1];
            stats->dnorm2 = s->h_sc[2];
            stats->margin = std::nan("");
            stats->grad_norm2 = s->h_sc[5];
            stats->status = FBL_OK;
        }
        std::swap(s->st, s->tr);
        s->k += 1;
        s->iter_in_epoch += 1;
        return FBL_OK;
    }
    if (s->p.use_graph) {
        // the whole iteration, backtracking included, as one graph launch
        fbl_solver::GraphEntry *ge = nullptr;
        for (auto &c : s->graphs)
            if (c.N == N && c.bd == bd && c.bmap == bmap && c.st == s->st && c.tr == s->tr) ge = &c;
        if (!ge) {
            if (s->graphs.size() >= 8) {
                cudaGraphExecDestroy(s->graphs.front().exec);
                s->graphs.erase(s->graphs.begin());
            }
            fbl_solver::GraphEntry ne{N, bd, bmap, s->st, s->tr, nullptr};
            fbl_status bs = build_graph(s, ne);
            if (bs) {
                restore();
                return bs;
            }
            s->graphs.push_back(ne);
            ge = &s->graphs.back();
        }
        LSState cfg;
        std::memset(&cfg, 0, sizeof cfg);
        cfg.alpha_init = s->p.alpha0;
        cfg.beta = s->p.beta;
        cfg.mu = s->p.mu;
        cfg.x_max = s->p.x_max;
        cfg.scale = scale;
        cfg.max_backtracks = s->p.max_backtracks;
        cfg.force_reject = s->p.force_reject;
        cfg.N_t = N;
        cfg.n_theta = d.n_views;
        *s->h_ls = cfg;
        CK(cudaMemcpyAsync(s->d_ls, s->h_ls, sizeof(LSState), cudaMemcpyHostToDevice, st), "line-search state");
        CK(cudaGraphLaunch(ge->exec, st), "graph launch");
        CK(cudaStreamSynchronize(st), "graph iteration");
        if (check_timeout(g, s->dg, st)) {
            restore();
            return fail(FBL_E_TIMEOUT, "fblisa_step: a bounded wait of the projector gave up");
        }
        const LSState r = *s->h_ls;
        const int trials = r.trials + 1;
        s->prof_launches[0] += 1;
        s->prof_launches[2] += 1;
        s->prof_launches[1] += trials;
        s->prof_launches[3] += trials;
        s->prof_launches[4] += 4 + 3 * trials;
        const bool accepted = r.status == FBL_OK && r.accepted;
        if (stats) {
            stats->k = s->k;
            stats->epoch = s->epoch;
            stats->N_t = N;
            stats->backtracks = r.trials;
            stats->alpha = r.alpha;
            stats->alpha_init = r.alpha_init;
            stats->j_start = r.j_start;
            stats->pred = r.pred;
            stats->grad_norm2 = r.g2;
            for (int q = 0; q < MLP_IN; ++q) stats->features[q] = r.feat[q];
            stats->rho0 = r.rho0;
            stats->f_x = r.f_x;
            stats->f_xbar = r.f_xbar;
            stats->gTd = r.gTd;
            stats->dnorm2 = r.dd;
            stats->margin = r.rhs - r.f_xbar;
            stats->status = accepted ? FBL_OK : r.status;
        }
        if (!accepted) {
            restore();
            if (r.status == FBL_E_NONFINITE)
                return fail(FBL_E_NONFINITE, "fblisa_step: non-finite objective or reduction at k=%lld",
                            (long long)s->k);
            return fail(FBL_E_LINESEARCH, "fblisa_step: no step passed (2.3) within %d backtracks",
                        s->p.max_backtracks);
        }
        std::swap(s->st, s->tr);
        s->k += 1;
        s->iter_in_epoch += 1;
        return FBL_OK;
    }
    // Step 2b: residual, f_N(x), grad f_N(x)
    int np = 0;
    CK(prof_launch(s, 0, st, [&] {
           return launch_project(PROJ_RESID, s->dg, s->st, s->L, xdt, s->d_views, N,
                                 bd, s->p.b_dtype, bmap, s->rt, FBL_F32, s->partials, &np, st);
       }),
       "residual kernel");
    CK(prof_launch(s, 4, st, [&] { return launch_reduce(s->partials, np, np, 1, s->d_sc + 0, st); }),
       "reduce");
    CK(prof_launch(s, 2, st, [&] {
           return launch_backproject(s->dg, s->rt, s->d_views, N, (float)scale, s->grad, st, s->partials);
       }),
       "gradient kernel");
    const int nbp = backproject_num_partials(s->dg);
    CK(prof_launch(s, 4, st, [&] { return launch_reduce(s->partials, nbp, nbp, 1, s->d_sc + 5, st); }),
       "reduce");
    // first trial step: alpha_0 (Step 2d), or the learned proposal on the same grid
    {
        LSState cfg;
        std::memset(&cfg, 0, sizeof cfg);
        cfg.alpha_init = s->p.alpha0;
        cfg.beta = s->p.beta;
        cfg.mu = s->p.mu;
        cfg.x_max = s->p.x_max;
        cfg.scale = scale;
        cfg.max_backtracks = s->p.max_backtracks;
        cfg.N_t = N;
        cfg.n_theta = d.n_views;
        *s->h_ls = cfg;
    }
    CK(cudaMemcpyAsync(s->d_ls, s->h_ls, sizeof(LSState), cudaMemcpyHostToDevice, st), "line-search state");
    CK(prof_launch(s, 4, st, [&] {
           return launch_propose(s->d_ls, s->d_ps, s->d_sc, s->p.proposal ? s->d_mlp : nullptr, s->margin, st);
       }),
       "proposal kernel");
    CK(cudaMemcpyAsync(s->h_ls, s->d_ls, sizeof(LSState), cudaMemcpyDeviceToHost, st), "line-search state");
    CK(cudaStreamSynchronize(st), "proposal");
    const LSState prop = *s->h_ls;
    // Step 2c: backtracking on (2.3)
    double alpha = prop.alpha_init;
    const double alpha_init = alpha;
    const int64_t nvox = (int64_t)d.nx * d.ny * d.nz;
    (void)nvox;
    bool accepted = false;
    int bt = 0;
    double rho0 = 0, rho1 = 0, gTd = 0, dd = 0, f_x = 0, f_xb = 0, rhs = 0;
    for (bt = 0; bt <= s->p.max_backtracks; ++bt) {
        int npp = 0;
        CK(prof_launch(s, 3, st, [&] { return solver_prox(s, alpha, &npp, st); }), "prox kernel");
        CK(prof_launch(s, 4, st, [&] { return launch_reduce(s->partials, npp, npp, 3, s->d_sc + 1, st); }),
           "reduce");
        CK(prof_launch(s, 1, st, [&] {
               return launch_project(PROJ_NORM, s->dg, s->tr, s->L, xdt, s->d_views, N,
                                     bd, s->p.b_dtype, bmap, nullptr, FBL_F32, s->partials, &np, st);
           }),
           "objective kernel");
        CK(prof_launch(s, 4, st, [&] { return launch_reduce(s->partials, np, np, 1, s->d_sc + 4, st); }),
           "reduce");
        CK(cudaMemcpyAsync(s->h_sc, s->d_sc, 5 * sizeof(double), cudaMemcpyDeviceToHost, st), "D2H");
        CK(cudaStreamSynchronize(st), "line search");
        prof_flush(s);
        rho0 = s->h_sc[0];
        gTd = s->h_sc[1];
        dd = s->h_sc[2];
        rho1 = s->h_sc[4];
        f_x = 0.5 * scale * rho0;
        f_xb = 0.5 * scale * rho1;
        rhs = f_x + gTd + dd / (2.0 * alpha);
        if (!std::isfinite(f_x) || !std::isfinite(f_xb) || !std::isfinite(rhs)) {
            restore();
            return fail(FBL_E_NONFINITE, "fblisa_step: non-finite objective or reduction at k=%lld",
                        (long long)s->k);
        }
        if (!s->p.force_reject && f_xb <= rhs) {
            accepted = true;
            break;
        }
        alpha *= s->p.beta;
    }
    if (stats) {
        stats->k = s->k;
        stats->epoch = s->epoch;
        stats->N_t = N;
        stats->backtracks = accepted ? bt : s->p.max_backtracks;
        stats->alpha = accepted ? alpha : alpha / s->p.beta;
        stats->alpha_init = alpha_init;
        stats->j_start = prop.j_start;
        stats->pred = prop.pred;
        stats->grad_norm2 = prop.g2;
        for (int q = 0; q < MLP_IN; ++q) stats->features[q] = prop.feat[q];
        stats->rho0 = rho0;
        stats->f_x = f_x;
        stats->f_xbar = f_xb;
        stats->gTd = gTd;
        stats->dnorm2 = dd;
        stats->margin = rhs - f_xb;
        stats->status = accepted ? FBL_OK : FBL_E_LINESEARCH;
    }
    if (!accepted) {
        restore();
        return fail(FBL_E_LINESEARCH, "fblisa_step: no step passed (2.3) within %d backtracks",
                    s->p.max_backtracks);
    }
    if (check_timeout(g, s->dg, st)) {
        restore();
        return fail(FBL_E_TIMEOUT, "fblisa_step: a bounded wait of the projector gave up");
    }
    // Step 2d: x <- x_bar (swap the state and trial buffers); the next first
    // trial is alpha_0 again, or the proposal's
    std::swap(s->st, s->tr);
    s->h_ps->f_prev = f_x;
    s->h_ps->g2_prev = prop.g2;
    s->h_ps->dj_prev = prop.j_start + bt - s->h_ps->j_prev;
    s->h_ps->have_dj = s->h_ps->have_prev;
    s->h_ps->j_prev = prop.j_start + bt;
    s->h_ps->have_prev = 1;
    s->h_ps->k += 1;
    CK(cudaMemcpyAsync(s->d_ps, s->h_ps, sizeof(PropState), cudaMemcpyHostToDevice, st), "proposal state");
    s->k += 1;
    s->iter_in_epoch += 1;
    return FBL_OK;
}

fbl_status solver_load_x(fbl_solver *s, const void *x, bool x_dev, cudaStream_t st) {
    const fbl_geometry_desc &d = s->g->desc;
    const size_t bytes = (size_t)d.nx * d.ny * d.nz * dtype_size(s->p.x_dtype);
    const void *src = x;
    if (!x_dev) {
        CK(cudaMemcpyAsync(s->xstage, x, bytes, cudaMemcpyHostToDevice, st), "x H2D");
        src = s->xstage;
    }
    CK(prof_launch(s, 5, st, [&] {
           return launch_pack(src, s->p.x_dtype, s->st, s->L, st);
       }),
       "pack");
    return FBL_OK;
}

fbl_status solver_store_x(fbl_solver *s, void *x, bool x_dev, cudaStream_t st) {
    const fbl_geometry_desc &d = s->g->desc;
    const size_t bytes = (size_t)d.nx * d.ny * d.nz * dtype_size(s->p.x_dtype);
    if (x_dev) {
        CK(prof_launch(s, 5, st, [&] {
               return launch_unpack(s->st, s->L, s->p.x_dtype, x, st);
           }),
           "x copy");
    } else {
        CK(prof_launch(s, 5, st, [&] {
               return launch_unpack(s->st, s->L, s->p.x_dtype, s->xstage, st);
           }),
           "x copy");
        CK(cudaMemcpyAsync(x, s->xstage, bytes, cudaMemcpyDeviceToHost, st), "x D2H");
    }
    CK(cudaStreamSynchronize(st), "x store");
    prof_flush(s);
    return FBL_OK;
}

}  // namespace

namespace {

// Time every launch configuration of the projector (trial-objective mode) and
// the backprojector on this geometry, with n_sel views spread over the orbit,
// and keep the fastest in dg.  Buffer contents do not change the work done.
fbl_status autotune_devgeom(const fbl_geometry *g, DevGeom &dg, int x_dtype, int n_sel,
                            cudaStream_t st, fbl_tune_report *rep) {
    const fbl_geometry_desc &d = g->desc;
    if (n_sel < 1) n_sel = 1;
    if (n_sel > d.n_views) n_sel = d.n_views;
    std::vector<int32_t> views(n_sel);
    for (int q = 0; q < n_sel; ++q) views[q] = (int32_t)((int64_t)q * d.n_views / n_sel);
    const ZLayout L = layout_for(g, x_dtype);
    const size_t vbytes = (size_t)L.elems() * dtype_size(x_dtype);
    const size_t nvox = (size_t)d.nx * d.ny * d.nz;
    const size_t bel = (size_t)n_sel * d.nv * d.nu;
    const size_t rtel = (size_t)n_sel * d.nu * rt_pitch(d.nv);
    AsyncBuf vol, b, rt, gz, part, dviews;
    CK(vol.alloc(vbytes, st), "autotune");
    CK(cudaMemsetAsync(vol.p, 0x3c, vbytes, st), "autotune");
    CK(b.alloc(bel * sizeof(float), st), "autotune");
    CK(cudaMemsetAsync(b.p, 0, bel * sizeof(float), st), "autotune");
    CK(rt.alloc(rtel * sizeof(float), st), "autotune");
    CK(cudaMemsetAsync(rt.p, 0x3c, rtel * sizeof(float), st), "autotune");
    CK(gz.alloc(nvox * sizeof(float), st), "autotune");
    CK(dviews.alloc((size_t)n_sel * sizeof(int32_t), st), "autotune");
    CK(cudaMemcpyAsync(dviews.p, views.data(), (size_t)n_sel * sizeof(int32_t), cudaMemcpyHostToDevice, st),
       "autotune");
    size_t np = 0;
    for (int cols : {4, 8}) {
        DevGeom t = dg;
        t.k1_cols = cols;
        np = std::max(np, (size_t)project_num_partials(t, n_sel));
    }
    CK(part.alloc(np * sizeof(double), st), "autotune");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "autotune");
    CK(cudaEventCreate(&e1), "autotune");
    auto time_it = [&](auto &&launch, float &ms) -> cudaError_t {
        cudaError_t e = launch();  // warm-up
        if (e != cudaSuccess) return e;
        cudaEventRecord(e0, st);
        for (int r = 0; r < 2; ++r) launch();
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return e;
        cudaEventElapsedTime(&ms, e0, e1);
        ms *= 0.5f;
        return cudaGetLastError();
    };
    float best = 1e30f;
    int qi = 0;
    const int k1_cfg[5][2] = {{8, 1}, {8, 0}, {4, 1}, {4, 0}, {8, 2}};  // (columns, plane-loop form)
    for (const auto &cfg : k1_cfg) {
        {
            const int cols = cfg[0], split = cfg[1];
            DevGeom t = dg;
            t.k1_cols = cols;
            t.k1_split = split;
            float ms = 0.f;
            cudaError_t e = time_it(
                [&] {
                    return launch_project(PROJ_NORM, t, vol.p, L, x_dtype, (const int32_t *)dviews.p, n_sel,
                                          b.p, FBL_F32, nullptr, nullptr, FBL_F32, (double *)part.p, nullptr,
                                          st);
                },
                ms);
            if (e == cudaErrorNotSupported && split == 2) {  // no tensor-map support: not a candidate
                cudaGetLastError();
                ++qi;
                continue;
            }
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(e, "autotune projector");
            }
            if (rep && qi < 5) rep->k1_ms[qi] = ms;
            ++qi;
            if (ms < best) {
                best = ms;
                dg.k1_cols = cols;
                dg.k1_split = split;
            }
        }
    }
    best = 1e30f;
    qi = 0;
    for (int vpl : {4, 2, 8, 16, 24, 28}) {
        DevGeom t = dg;
        t.k2_vpl = vpl;
        float ms = 0.f;
        cudaError_t e = time_it(
            [&] {
                return launch_backproject(t, (const float *)rt.p, (const int32_t *)dviews.p, n_sel, 1.0f,
                                          (float *)gz.p, st);
            },
            ms);
        if (e != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return cuda_fail(e, "autotune backprojector");
        }
        if (rep && qi < 6) rep->k2_ms[qi] = ms;
        ++qi;
        if (ms < best) {
            best = ms;
            dg.k2_vpl = vpl;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rep) {
        rep->k1_cols = dg.k1_cols;
        rep->k1_split = dg.k1_split;
        rep->k2_vpl = dg.k2_vpl;
    }
    return FBL_OK;
}

}  // namespace

extern "C" fbl_status geometry_autotune(fbl_geometry *g, int32_t x_dtype, int32_t n_sel, void *stream,
                                        fbl_tune_report *report) {
    if (!g) return fail(FBL_E_INVAL, "geometry_autotune: null geometry");
    if (!valid_dtype(x_dtype)) return fail(FBL_E_INVAL, "geometry_autotune: bad dtype");
    fbl_status st = check_device(g->device);
    if (st) return st;
    if (report) std::memset(report, 0, sizeof *report);
    return autotune_devgeom(g, g->dg, x_dtype, n_sel, (cudaStream_t)stream, report);
}

extern "C" fbl_status mlp_forward(const float *params, const float *X, int32_t n, float *y, void *stream) {
    if (!params || (n > 0 && (!X || !y)) || n < 0) return fail(FBL_E_INVAL, "mlp_forward: bad argument");
    if (!is_device_ptr(params) || (n > 0 && (!is_device_ptr(X) || !is_device_ptr(y))))
        return fail(FBL_E_INVAL, "mlp_forward: arrays must be device memory");
    CK(launch_mlp_forward(params, X, n, y, (cudaStream_t)stream), "mlp forward");
    return FBL_OK;
}

extern "C" fbl_status mlp_gradient(const float *params, const float *X, const float *t, int32_t n,
                                   float *grad, double *loss_host, void *stream) {
    if (!params || !X || !t || !grad || !loss_host || n < 1) return fail(FBL_E_INVAL, "mlp_gradient: bad argument");
    if (!is_device_ptr(params) || !is_device_ptr(X) || !is_device_ptr(t) || !is_device_ptr(grad))
        return fail(FBL_E_INVAL, "mlp_gradient: arrays must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    AsyncBuf loss;
    CK(loss.alloc(sizeof(double), s), "mlp loss");
    CK(launch_mlp_train(const_cast<float *>(params), nullptr, nullptr, X, t, n, n, 1, 0.f, 0, grad,
                        (double *)loss.p, nullptr, s),
       "mlp gradient");
    CK(cudaMemcpyAsync(loss_host, loss.p, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
    CK(cudaStreamSynchronize(s), "mlp_gradient");
    return FBL_OK;
}

extern "C" fbl_status mlp_train(float *params, float *adam_m, float *adam_v, int32_t *adam_step,
                                const float *X, const float *t, int32_t n, int32_t batch,
                                int32_t epochs, float lr, double *last_loss_host, void *stream) {
    if (!params || !adam_m || !adam_v || !adam_step || !X || !t || n < 1 || batch < 1 || epochs < 0 ||
        !(lr > 0))
        return fail(FBL_E_INVAL, "mlp_train: bad argument");
    for (const void *p : {(const void *)params, (const void *)adam_m, (const void *)adam_v,
                          (const void *)adam_step, (const void *)X, (const void *)t})
        if (!is_device_ptr(p)) return fail(FBL_E_INVAL, "mlp_train: arrays must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    AsyncBuf loss;
    CK(loss.alloc(sizeof(double), s), "mlp loss");
    CK(cudaMemsetAsync(loss.p, 0, sizeof(double), s), "memset");
    CK(launch_mlp_train(params, adam_m, adam_v, X, t, n, batch, epochs, lr, 1, nullptr,
                        (double *)loss.p, adam_step, s),
       "mlp train");
    double l = 0.0;
    CK(cudaMemcpyAsync(&l, loss.p, sizeof(double), cudaMemcpyDeviceToHost, s), "D2H");
    CK(cudaStreamSynchronize(s), "mlp_train");
    if (last_loss_host) *last_loss_host = l;
    return FBL_OK;
}

extern "C" fbl_status geometry_set_launch(fbl_geometry *g, int32_t k1_cols, int32_t k1_split,
                                          int32_t k2_vpl) {
    if (!g) return fail(FBL_E_INVAL, "geometry_set_launch: null geometry");
    if ((k1_cols != 4 && k1_cols != 8) || (k1_split < 0 || k1_split > 2) ||
        (k2_vpl != 2 && k2_vpl != 4 && k2_vpl != 8 && k2_vpl != 16 && k2_vpl != 24 && k2_vpl != 28))
        return fail(FBL_E_INVAL,
                    "geometry_set_launch: need k1_cols in {4,8}, k1_split in {0,1,2}, "
                    "k2_vpl in {2,4,8,16,24,28}");
    g->dg.k1_cols = k1_cols;
    g->dg.k1_split = k1_split;
    g->dg.k2_vpl = k2_vpl;
    return FBL_OK;
}

extern "C" fbl_status fblisa_create(const fbl_geometry *g, const fbl_params *p, fbl_solver **out) {
    if (!g || !p || !out) return fail(FBL_E_INVAL, "fblisa_create: null argument");
    *out = nullptr;
    fbl_status st = check_device(g->device);
    if (st) return st;
    const fbl_geometry_desc &d = g->desc;
    if (!valid_dtype(p->x_dtype) || !valid_dtype(p->b_dtype)) return fail(FBL_E_INVAL, "fblisa_create: bad dtype");
    if (!(p->alpha0 > 0) || !(p->beta > 0 && p->beta < 1) || !(p->mu >= 0) || !(p->C > 0) ||
        !(p->eps_base > 0 && p->eps_base < 1) || p->max_backtracks < 0)
        return fail(FBL_E_INVAL, "fblisa_create: need alpha0 > 0, 0 < beta < 1, mu >= 0, C > 0, 0 < eps_base < 1");
    const int32_t n_max = p->n_max > 0 ? p->n_max : d.n_views;
    if (p->N0 < 1 || p->N0 > n_max || n_max > d.n_views)
        return fail(FBL_E_INVAL, "fblisa_create: need 1 <= N0 <= n_max <= n_views");
    if (p->proposal != 0 && p->proposal != 1) return fail(FBL_E_INVAL, "fblisa_create: proposal must be 0 or 1");
    if (p->fixed_step != 0 && p->fixed_step != 1) return fail(FBL_E_INVAL, "fblisa_create: fixed_step must be 0 or 1");
    if (p->reg != FBL_REG_L1 && p->reg != FBL_REG_TV) return fail(FBL_E_INVAL, "fblisa_create: reg must be 0 or 1");
    if (!(p->x_max > 0.0)) return fail(FBL_E_INVAL, "fblisa_create: need x_max > 0 (+inf: no upper bound)");
    if (p->reg == FBL_REG_TV) {
        if (p->tv_iters < 0 || p->tv_iters > 100000 || (p->tv_warm != 0 && p->tv_warm != 1))
            return fail(FBL_E_INVAL, "fblisa_create: need 0 <= tv_iters <= 100000 and tv_warm 0 or 1");
        if (p->use_graph)
            return fail(FBL_E_UNSUPPORTED, "fblisa_create: the TV prox runs in host-loop mode (use_graph 0)");
        if (!tv_dims_ok(d.nz, d.nx, d.ny)) return fail(FBL_E_UNSUPPORTED, "fblisa_create: volume too large for TV");
    }
    auto s = new fbl_solver();
    s->g = g;
    s->dg = g->dg;
    s->p = *p;
    s->device = g->device;
    s->n_max = n_max;
    s->L = layout_for(g, p->x_dtype);
    const int es = dtype_size(p->x_dtype);
    s->vol_bytes = (size_t)s->L.elems() * es;
    const size_t nvox = (size_t)d.nx * d.ny * d.nz;
    cudaError_t e = cudaSuccess;
    void **vols[2] = {&s->st, &s->tr};
    for (int q = 0; q < 2 && e == cudaSuccess; ++q) {
        e = cudaMalloc(vols[q], s->vol_bytes);
        if (e == cudaSuccess) e = cudaMemset(*vols[q], 0, s->vol_bytes);  // zero border, once
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->grad, nvox * sizeof(float));
    if (e == cudaSuccess && p->reg == FBL_REG_TV) {
        // b, y and two dual pairs (q, r) of the TV prox: 14 volumes of FP32
        e = cudaMalloc(&s->tv_buf, 14 * nvox * sizeof(float));
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->xstage, nvox * es);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_views, (size_t)d.n_views * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_sc, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_views, (size_t)d.n_views * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_sc, 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_ls, sizeof(LSState));
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_ls, sizeof(LSState));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_ps, sizeof(PropState));
    if (e == cudaSuccess) e = cudaMemset(s->d_ps, 0, sizeof(PropState));
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_ps, sizeof(PropState));
    if (e == cudaSuccess) std::memset(s->h_ps, 0, sizeof(PropState));
    if (e != cudaSuccess) {
        solver_free(s);
        delete s;
        return cuda_fail(e, "fblisa_create");
    }
    if (p->autotune) {
        const int32_t Nt = std::min(n_max, std::max(p->N0, 1));
        fbl_status ts = autotune_devgeom(g, s->dg, p->x_dtype, Nt, nullptr, nullptr);
        if (ts) {
            std::string keep = g_last_error;
            solver_free(s);
            delete s;
            g_last_error = keep;
            return ts;
        }
    }
    *out = s;
    return FBL_OK;
}

extern "C" void fblisa_destroy(fbl_solver *s) {
    if (!s) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != s->device) cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    solver_free(s);
    if (cur >= 0 && cur != s->device) cudaSetDevice(cur);
    delete s;
}

extern "C" fbl_status fblisa_step(fbl_solver *s, void *x, const void *b, fbl_step_stats *stats,
                                  void *stream) {
    if (!s || !x || !b) return fail(FBL_E_INVAL, "fblisa_step: null argument");
    fbl_status st = check_device(s->device);
    if (st) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    const bool x_dev = is_device_ptr(x), b_dev = is_device_ptr(b);
    if ((st = solver_load_x(s, x, x_dev, cs))) return st;
    if ((st = solver_iterate(s, b, b_dev, stats, cs))) return st;
    return solver_store_x(s, x, x_dev, cs);
}

extern "C" fbl_status fblisa_run(fbl_solver *s, void *x, const void *b, int32_t epochs,
                                 fbl_step_stats *trace, int64_t trace_cap, int64_t *n_steps,
                                 void *stream) {
    if (!s || !x || !b) return fail(FBL_E_INVAL, "fblisa_run: null argument");
    if (epochs < 0 || trace_cap < 0) return fail(FBL_E_INVAL, "fblisa_run: negative count");
    fbl_status st = check_device(s->device);
    if (st) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    const bool x_dev = is_device_ptr(x), b_dev = is_device_ptr(b);
    if (n_steps) *n_steps = 0;
    if ((st = solver_load_x(s, x, x_dev, cs))) return st;
    const int32_t target = s->epoch + epochs - ((s->epoch > 0 && s->iter_in_epoch < s->iters_epoch) ? 1 : 0);
    int64_t done = 0;
    fbl_status rc = FBL_OK;
    while (true) {
        const bool epoch_open = s->epoch > 0 && s->iter_in_epoch < s->iters_epoch;
        if (!epoch_open && s->epoch >= target) break;
        fbl_step_stats rec;
        rc = solver_iterate(s, b, b_dev, &rec, cs);
        if (trace && done < trace_cap) trace[done] = rec;
        if (rc) break;
        ++done;
    }
    if (n_steps) *n_steps = done;
    std::string keep = g_last_error;
    fbl_status st2 = solver_store_x(s, x, x_dev, cs);
    if (rc) {
        g_last_error = keep;
        return rc;
    }
    return st2;
}

extern "C" fbl_status fblisa_set_proposal(fbl_solver *s, const float *params, float margin,
                                          int32_t enable) {
    if (!s || (enable && !params)) return fail(FBL_E_INVAL, "fblisa_set_proposal: null argument");
    if (!std::isfinite(margin)) return fail(FBL_E_INVAL, "fblisa_set_proposal: bad margin");
    fbl_status st = check_device(s->device);
    if (st) return st;
    if (params) {
        if (!s->d_mlp) CK(cudaMalloc(&s->d_mlp, MLP_PARAMS * sizeof(float)), "proposal network");
        CK(cudaMemcpy(s->d_mlp, params, MLP_PARAMS * sizeof(float), cudaMemcpyDefault), "proposal network");
        drop_graphs(s);  // graphs captured without the network
    }
    if (margin != s->margin) drop_graphs(s);  // captured graphs hold the margin as an argument
    s->margin = margin;
    if (s->p.proposal != (enable ? 1 : 0)) drop_graphs(s);
    s->p.proposal = enable ? 1 : 0;
    return FBL_OK;
}

extern "C" fbl_status fblisa_profile(fbl_solver *s, int32_t enable, fbl_profile *out) {
    if (!s) return fail(FBL_E_INVAL, "fblisa_profile: null solver");
    if (out) {
        for (int c = 0; c < FBL_PROF_CLASSES; ++c) {
            out->ms[c] = s->prof_ms[c];
            out->launches[c] = s->prof_launches[c];
            s->prof_ms[c] = 0.0;
            s->prof_launches[c] = 0;
        }
    }
    s->prof_on = enable != 0;
    return FBL_OK;
}

extern "C" fbl_status fblisa_last_batch(const fbl_solver *s, int32_t *views, int32_t cap, int32_t *n) {
    if (!s || !n) return fail(FBL_E_INVAL, "fblisa_last_batch: null argument");
    *n = (int32_t)s->last_batch.size();
    if (views) {
        if (cap < *n) return fail(FBL_E_INVAL, "fblisa_last_batch: buffer too small");
        std::memcpy(views, s->last_batch.data(), s->last_batch.size() * sizeof(int32_t));
    }
    return FBL_OK;
}

extern "C" const char *fbl_last_error(void) { return g_last_error.c_str(); }

void fbl::set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

// ---------------------------------------------------------------------------
// Batched iteration over several volumes: every volume runs its own
// Algorithm 1 (geometry, schedule, sampling, line search), and each phase of
// one iteration of all of them is one persistent launch (fbl_internal.cuh).

struct fbl_batch {
    int device = -1;
    int n_vol = 0;
    std::vector<fbl_solver *> sv;   // per-volume state and buffers
    std::vector<int> order;         // volumes in tile order (largest first)
    int x_dtype = FBL_F32, b_dtype = FBL_F32;
    int cols = 8, split = 1, vpl = 4, ntap = 1;
    // descriptor blob: BatchHdr, BatchVol[n_vol] (tile order), view lists
    size_t blob_bytes = 0, vols_off = 0, views_off = 0;
    std::vector<size_t> view_slot;  // offset (in int32) of each volume's view list
    void *d_blob = nullptr, *h_blob = nullptr;
    LSState *d_ls = nullptr, *h_ls = nullptr;  // [n_vol], volume order
    int *d_ctr = nullptr;                      // 2 ints per persistent launch site
    float *d_mlp = nullptr;
    bool have_mlp = false;
    float margin = 0.25f;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr, cap2 = nullptr;
    int64_t k = 0;
    int64_t launches = 0;                      // kernels launched by the batch so far
};

namespace {

constexpr int BATCH_SITES = 4;  // persistent launch sites: K1 residual, K2, K3, K1 objective

void batch_free(fbl_batch *bt) {
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    if (bt->cap) cudaStreamDestroy(bt->cap);
    if (bt->cap2) cudaStreamDestroy(bt->cap2);
    cudaFree(bt->d_blob);
    cudaFreeHost(bt->h_blob);
    cudaFree(bt->d_ls);
    cudaFreeHost(bt->h_ls);
    cudaFree(bt->d_ctr);
    cudaFree(bt->d_mlp);
    for (fbl_solver *s : bt->sv) {
        if (!s) continue;
        solver_free(s);
        delete s;
    }
    bt->sv.clear();
}

BatchHdr *blob_hdr(fbl_batch *bt, bool dev) {
    return (BatchHdr *)((char *)(dev ? bt->d_blob : bt->h_blob));
}
BatchVol *blob_vols(fbl_batch *bt, bool dev) {
    return (BatchVol *)((char *)(dev ? bt->d_blob : bt->h_blob) + bt->vols_off);
}
int32_t *blob_views(fbl_batch *bt, bool dev) {
    return (int32_t *)((char *)(dev ? bt->d_blob : bt->h_blob) + bt->views_off);
}

// The whole batched iteration (Steps 2b-2c of every volume) as one graph.
fbl_status batch_build_graph(fbl_batch *bt) {
    if (!bt->cap) CK(cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking), "capture stream");
    if (!bt->cap2) CK(cudaStreamCreateWithFlags(&bt->cap2, cudaStreamNonBlocking), "capture stream");
    const BatchHdr *hdr = blob_hdr(bt, true);
    BatchVol *vols = blob_vols(bt, true);
    const int n = bt->n_vol;
    cudaStream_t cs = bt->cap, cb = bt->cap2;
    // relaxed: the persistent launchers query occupancy on first use
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed), "begin capture");
    cudaError_t e = launch_batch_project(PROJ_RESID, hdr, vols, bt->x_dtype, bt->b_dtype, bt->cols,
                                         bt->d_ctr + 0, cs);
    if (e == cudaSuccess) e = launch_batch_reduce(hdr, vols, n, 0, 1, 0, 0, cs);
    if (e == cudaSuccess) e = launch_batch_backproject(hdr, vols, bt->ntap, bt->d_ctr + 2, cs);
    if (e == cudaSuccess) e = launch_batch_reduce(hdr, vols, n, 1, 1, 5, 0, cs);
    if (e == cudaSuccess) e = launch_batch_propose(vols, n, bt->have_mlp ? bt->d_mlp : nullptr, bt->margin, cs);
    if (e == cudaSuccess) e = launch_batch_ls_init(blob_hdr(bt, true), vols, n, cs);
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps);
    cudaGraphConditionalHandle cond = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, cg, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &cp);
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(cb, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            cudaError_t eb = launch_batch_prox(hdr, vols, bt->x_dtype, bt->d_ctr + 4, cb);
            if (eb == cudaSuccess) eb = launch_batch_reduce(hdr, vols, n, 2, 3, 1, 1, cb);
            if (eb == cudaSuccess)
                eb = launch_batch_project(PROJ_NORM, hdr, vols, bt->x_dtype, bt->b_dtype, bt->cols,
                                          bt->d_ctr + 6, cb);
            if (eb == cudaSuccess) eb = launch_batch_reduce(hdr, vols, n, 0, 1, 4, 1, cb);
            if (eb == cudaSuccess) eb = launch_batch_decide(blob_hdr(bt, true), vols, n, cond, cb);
            cudaError_t ee = cudaStreamEndCapture(cb, &body);
            e = eb != cudaSuccess ? eb : ee;
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bt->h_ls, bt->d_ls, (size_t)n * sizeof(LSState), cudaMemcpyDeviceToHost, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = ee;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bt->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        bt->exec = nullptr;
        return cuda_fail(e, "graph capture of the batched iteration");
    }
    return FBL_OK;
}

// One iteration of every volume.  stats: [n_vol] (volume order), may be NULL.
// Returns FBL_OK when every volume accepted a step; otherwise the status of
// the first volume that did not (its x and schedule position are unchanged;
// the other volumes have advanced).
fbl_status batch_iterate(fbl_batch *bt, const void *const *b, const char *b_dev, fbl_step_stats *stats,
                         cudaStream_t st) {
    const int n = bt->n_vol;
    struct Saved {
        int32_t epoch, N_t, N_prev, iters, it;
        int64_t khat;
        bool new_epoch;
        std::vector<int32_t> views;
    };
    std::vector<Saved> saved(n);
    auto restore = [&](int v) {
        fbl_solver *s = bt->sv[v];
        const Saved &sv = saved[v];
        s->epoch = sv.epoch;
        s->N_t = sv.N_t;
        s->N_prev = sv.N_prev;
        s->iters_epoch = sv.iters;
        s->iter_in_epoch = sv.it;
        s->k_hat = sv.khat;
        if (sv.new_epoch) s->epoch_views = sv.views;
    };
    BatchHdr *hh = blob_hdr(bt, false);
    BatchVol *hv = blob_vols(bt, false);
    int32_t *hviews = blob_views(bt, false);
    const int32_t *dviews = blob_views(bt, true);
    hh->n_vol = n;
    int first[3] = {0, 0, 0};
    for (int q = 0; q < n; ++q) {
        const int v = bt->order[q];
        fbl_solver *s = bt->sv[v];
        const fbl_geometry_desc &d = s->g->desc;
        Saved &sv = saved[v];
        sv.epoch = s->epoch;
        sv.N_t = s->N_t;
        sv.N_prev = s->N_prev;
        sv.iters = s->iters_epoch;
        sv.it = s->iter_in_epoch;
        sv.khat = s->k_hat;
        sv.new_epoch = !(s->epoch > 0 && s->iter_in_epoch < s->iters_epoch);
        if (sv.new_epoch) sv.views = s->epoch_views;
        begin_epoch_if_needed(s);
        const int32_t N = s->N_t;
        fbl_status rc = ensure_batch_buffers(s, N);
        if (rc) {
            for (int r = 0; r <= q; ++r) restore(bt->order[r]);
            return rc;
        }
        const int32_t *views = s->epoch_views.data() + (size_t)s->iter_in_epoch * N;
        std::memcpy(hviews + bt->view_slot[v], views, N * sizeof(int32_t));
        s->last_batch.assign(views, views + N);
        const void *bd = b[v];
        const int32_t *bmap = dviews + bt->view_slot[v];
        if (!b_dev[v]) {  // stage the batch's views of host data
            const size_t per_view = (size_t)d.nv * d.nu * dtype_size(s->p.b_dtype);
            if (per_view * N > s->bstage_cap) {
                cudaFree(s->bstage);
                s->bstage = nullptr;
                s->bstage_cap = 0;
                cudaError_t e = cudaMalloc(&s->bstage, per_view * N);
                if (e != cudaSuccess) {
                    for (int r = 0; r <= q; ++r) restore(bt->order[r]);
                    return cuda_fail(e, "data staging");
                }
                s->bstage_cap = per_view * N;
            }
            for (int32_t w = 0; w < N; ++w)
                CK(cudaMemcpyAsync((char *)s->bstage + per_view * w, (const char *)b[v] + per_view * views[w],
                                   per_view, cudaMemcpyHostToDevice, st),
                   "data H2D");
            bd = s->bstage;
            bmap = nullptr;
        }
        BatchVol &bv = hv[q];
        std::memset(&bv, 0, sizeof bv);
        bv.g = s->dg;
        bv.L = s->L;
        bv.x_cur = s->st;
        bv.x_trial = s->tr;
        bv.b = bd;
        bv.b_views = bmap;
        bv.views = dviews + bt->view_slot[v];
        bv.rt = s->rt;
        bv.grad = s->grad;
        bv.partials = s->partials;
        bv.sc = s->d_sc;
        bv.ls = bt->d_ls + v;
        bv.ps = s->d_ps;
        bv.scale = (float)((double)d.n_views / (double)N);
        bv.N_t = N;
        bv.proposal = s->p.proposal;
        bv.tiles[0] = project_num_partials(s->dg, N);
        bv.tiles[1] = backproject_num_partials(s->dg);
        bv.tiles[2] = prox_zi_num_partials(d.nx, d.ny, d.nz);
        for (int ph = 0; ph < 3; ++ph) {
            bv.first[ph] = first[ph];
            first[ph] += bv.tiles[ph];
        }
        LSState &cfg = bt->h_ls[v];
        std::memset(&cfg, 0, sizeof cfg);
        cfg.alpha_init = s->p.alpha0;
        cfg.beta = s->p.beta;
        cfg.mu = s->p.mu;
        cfg.x_max = s->p.x_max;
        cfg.scale = (double)d.n_views / (double)N;
        cfg.max_backtracks = s->p.max_backtracks;
        cfg.force_reject = s->p.force_reject;
        cfg.N_t = N;
        cfg.n_theta = d.n_views;
    }
    for (int ph = 0; ph < 3; ++ph) hh->total[ph] = first[ph];
    auto fail_all = [&](fbl_status r) {
        for (int v = 0; v < n; ++v) restore(v);
        return r;
    };
    cudaError_t e = cudaMemcpyAsync(bt->d_blob, bt->h_blob, bt->blob_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(bt->d_ls, bt->h_ls, (size_t)n * sizeof(LSState), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail_all(cuda_fail(e, "batch descriptors"));
    if (!bt->exec) {
        fbl_status rc = batch_build_graph(bt);
        if (rc) return fail_all(rc);
    }
    e = cudaGraphLaunch(bt->exec, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_all(cuda_fail(e, "batched iteration"));
    int max_trials = 0;
    fbl_status first_bad = FBL_OK;
    int bad_v = -1;
    for (int v = 0; v < n; ++v) {
        fbl_solver *s = bt->sv[v];
        const LSState r = bt->h_ls[v];
        max_trials = std::max(max_trials, r.trials + 1);
        const bool accepted = r.status == FBL_OK && r.accepted;
        if (stats) {
            fbl_step_stats &o = stats[v];
            std::memset(&o, 0, sizeof o);
            o.k = s->k;
            o.epoch = s->epoch;
            o.N_t = s->N_t;
            o.backtracks = r.trials;
            o.alpha = r.alpha;
            o.alpha_init = r.alpha_init;
            o.j_start = r.j_start;
            o.pred = r.pred;
            o.grad_norm2 = r.g2;
            for (int q = 0; q < MLP_IN; ++q) o.features[q] = r.feat[q];
            o.rho0 = r.rho0;
            o.f_x = r.f_x;
            o.f_xbar = r.f_xbar;
            o.gTd = r.gTd;
            o.dnorm2 = r.dd;
            o.margin = r.rhs - r.f_xbar;
            o.status = accepted ? FBL_OK : (r.status ? r.status : FBL_E_LINESEARCH);
        }
        if (accepted) {
            std::swap(s->st, s->tr);  // mirrors the swap the decision kernel made
            s->k += 1;
            s->iter_in_epoch += 1;
        } else {
            restore(v);
            if (first_bad == FBL_OK) {
                first_bad = r.status == FBL_E_NONFINITE ? FBL_E_NONFINITE : FBL_E_LINESEARCH;
                bad_v = v;
            }
        }
    }
    bt->k += 1;
    bt->launches += 6 + 5 * (int64_t)max_trials;
    if (first_bad != FBL_OK) {
        if (first_bad == FBL_E_NONFINITE)
            return fail(FBL_E_NONFINITE, "fblisa_batch_step: volume %d: non-finite objective or reduction", bad_v);
        return fail(FBL_E_LINESEARCH, "fblisa_batch_step: volume %d: no step passed (2.3) within the cap", bad_v);
    }
    return FBL_OK;
}

}  // namespace

extern "C" fbl_status fblisa_batch_create(const fbl_geometry *const *geoms, const fbl_params *params,
                                          int32_t n_vol, fbl_batch **out) {
    if (!geoms || !params || !out) return fail(FBL_E_INVAL, "fblisa_batch_create: null argument");
    *out = nullptr;
    if (n_vol < 1 || n_vol > 1024) return fail(FBL_E_INVAL, "fblisa_batch_create: need 1 <= n_vol <= 1024");
    for (int v = 0; v < n_vol; ++v)
        if (!geoms[v]) return fail(FBL_E_INVAL, "fblisa_batch_create: null geometry %d", v);
    const int dev = geoms[0]->device;
    for (int v = 0; v < n_vol; ++v) {
        if (geoms[v]->device != dev) return fail(FBL_E_INVAL, "fblisa_batch_create: geometries on different devices");
        if (params[v].x_dtype != params[0].x_dtype || params[v].b_dtype != params[0].b_dtype)
            return fail(FBL_E_INVAL, "fblisa_batch_create: every volume needs the same x_dtype and b_dtype");
        if (params[v].fixed_step)
            return fail(FBL_E_UNSUPPORTED, "fblisa_batch_create: the batch runs the line search (fixed_step 0)");
        if (params[v].reg != FBL_REG_L1)
            return fail(FBL_E_UNSUPPORTED, "fblisa_batch_create: the batch runs the l1 prox (reg 0)");
    }
    if (params[0].b_dtype != params[0].x_dtype)
        return fail(FBL_E_UNSUPPORTED, "fblisa_batch_create: b_dtype must equal x_dtype");
    fbl_status st = check_device(dev);
    if (st) return st;
    auto bt = new fbl_batch();
    bt->device = dev;
    bt->n_vol = n_vol;
    bt->x_dtype = params[0].x_dtype;
    bt->b_dtype = params[0].b_dtype;
    // launch configuration shared by the batch: the largest volume's
    int big = 0;
    for (int v = 1; v < n_vol; ++v) {
        const fbl_geometry_desc &a = geoms[v]->desc, &c = geoms[big]->desc;
        if ((int64_t)a.nx * a.ny * a.nz > (int64_t)c.nx * c.ny * c.nz) big = v;
    }
    bt->cols = geoms[big]->dg.k1_cols == 4 ? 4 : 8;
    bt->split = geoms[big]->dg.k1_split ? 1 : 0;
    bt->vpl = geoms[big]->dg.k2_vpl;
    bt->ntap = 1;
    for (int v = 0; v < n_vol; ++v) bt->ntap = std::max(bt->ntap, geoms[v]->dg.ntap);
    bt->sv.assign(n_vol, nullptr);
    for (int v = 0; v < n_vol; ++v) {
        fbl_params p = params[v];
        p.autotune = 0;
        p.use_graph = 0;
        fbl_solver *s = nullptr;
        st = fblisa_create(geoms[v], &p, &s);
        if (st) {
            std::string keep = g_last_error;
            batch_free(bt);
            delete bt;
            g_last_error = "fblisa_batch_create: volume " + std::to_string(v) + ": " + keep;
            return st;
        }
        s->dg.k1_cols = bt->cols;  // the block width is common; split and vpl stay per volume
        bt->sv[v] = s;
    }
    bt->order.resize(n_vol);
    for (int v = 0; v < n_vol; ++v) bt->order[v] = v;
    std::stable_sort(bt->order.begin(), bt->order.end(), [&](int a, int c) {
        const fbl_geometry_desc &da = geoms[a]->desc, &dc = geoms[c]->desc;
        return (int64_t)da.nx * da.ny * da.nz > (int64_t)dc.nx * dc.ny * dc.nz;
    });
    bt->vols_off = (sizeof(BatchHdr) + 255) / 256 * 256;
    bt->views_off = bt->vols_off + ((size_t)n_vol * sizeof(BatchVol) + 255) / 256 * 256;
    bt->view_slot.resize(n_vol);
    size_t nviews = 0;
    for (int v = 0; v < n_vol; ++v) {
        bt->view_slot[v] = nviews;
        nviews += (size_t)geoms[v]->desc.n_views;
    }
    bt->blob_bytes = bt->views_off + nviews * sizeof(int32_t);
    cudaError_t e = cudaMalloc(&bt->d_blob, bt->blob_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&bt->h_blob, bt->blob_bytes);
    if (e == cudaSuccess) std::memset(bt->h_blob, 0, bt->blob_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_ls, (size_t)n_vol * sizeof(LSState));
    if (e == cudaSuccess) e = cudaMallocHost(&bt->h_ls, (size_t)n_vol * sizeof(LSState));
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_ctr, 2 * BATCH_SITES * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(bt->d_ctr, 0, 2 * BATCH_SITES * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_mlp, MLP_PARAMS * sizeof(float));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        batch_free(bt);
        delete bt;
        return cuda_fail(e, "fblisa_batch_create");
    }
    *out = bt;
    return FBL_OK;
}

extern "C" void fblisa_batch_destroy(fbl_batch *bt) {
    if (!bt) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != bt->device) cudaSetDevice(bt->device);
    cudaDeviceSynchronize();
    batch_free(bt);
    if (cur >= 0 && cur != bt->device) cudaSetDevice(cur);
    delete bt;
}

extern "C" fbl_status fblisa_batch_set_proposal(fbl_batch *bt, const float *params, float margin,
                                                int32_t enable) {
    if (!bt || (enable && !params && !bt->have_mlp))
        return fail(FBL_E_INVAL, "fblisa_batch_set_proposal: null argument");
    if (!std::isfinite(margin)) return fail(FBL_E_INVAL, "fblisa_batch_set_proposal: bad margin");
    fbl_status st = check_device(bt->device);
    if (st) return st;
    if (params) {
        CK(cudaMemcpy(bt->d_mlp, params, MLP_PARAMS * sizeof(float), cudaMemcpyDefault), "proposal network");
        if (!bt->have_mlp && bt->exec) {  // the graph was captured without the network
            cudaGraphExecDestroy(bt->exec);
            bt->exec = nullptr;
        }
        bt->have_mlp = true;
    }
    if (margin != bt->margin && bt->exec) {  // the graph holds the margin as an argument
        cudaGraphExecDestroy(bt->exec);
        bt->exec = nullptr;
    }
    bt->margin = margin;
    for (fbl_solver *s : bt->sv) s->p.proposal = enable ? 1 : 0;
    return FBL_OK;
}

namespace {

fbl_status batch_load(fbl_batch *bt, void *const *x, const void *const *b, std::vector<char> &x_dev,
                      std::vector<char> &b_dev, cudaStream_t cs) {
    x_dev.assign(bt->n_vol, 0);
    b_dev.assign(bt->n_vol, 0);
    for (int v = 0; v < bt->n_vol; ++v) {
        if (!x[v] || !b[v]) return fail(FBL_E_INVAL, "fblisa_batch: null x or b of volume %d", v);
        x_dev[v] = is_device_ptr(x[v]);
        b_dev[v] = is_device_ptr(b[v]);
    }
    for (int v = 0; v < bt->n_vol; ++v) {
        fbl_status st = solver_load_x(bt->sv[v], x[v], x_dev[v], cs);
        if (st) return st;
    }
    return FBL_OK;
}

fbl_status batch_store(fbl_batch *bt, void *const *x, const std::vector<char> &x_dev, cudaStream_t cs) {
    for (int v = 0; v < bt->n_vol; ++v) {
        fbl_status st = solver_store_x(bt->sv[v], x[v], x_dev[v], cs);
        if (st) return st;
    }
    return FBL_OK;
}

}  // namespace

extern "C" fbl_status fblisa_batch_step(fbl_batch *bt, void *const *x, const void *const *b,
                                        fbl_step_stats *stats, void *stream) {
    if (!bt || !x || !b) return fail(FBL_E_INVAL, "fblisa_batch_step: null argument");
    fbl_status st = check_device(bt->device);
    if (st) return st;
    for (fbl_solver *s : bt->sv)
        if (s->p.proposal && !bt->have_mlp)
            return fail(FBL_E_INVAL, "fblisa_batch_step: proposal enabled but no network set");
    cudaStream_t cs = (cudaStream_t)stream;
    std::vector<char> x_dev, b_dev;
    if ((st = batch_load(bt, x, b, x_dev, b_dev, cs))) return st;
    fbl_status rc = batch_iterate(bt, b, b_dev.data(), stats, cs);
    std::string keep = g_last_error;
    st = batch_store(bt, x, x_dev, cs);
    if (rc) {
        g_last_error = keep;
        return rc;
    }
    return st;
}

extern "C" fbl_status fblisa_batch_run(fbl_batch *bt, void *const *x, const void *const *b,
                                       int32_t iterations, fbl_step_stats *trace, int64_t trace_cap,
                                       int64_t *n_steps, void *stream) {
    if (!bt || !x || !b) return fail(FBL_E_INVAL, "fblisa_batch_run: null argument");
    if (iterations < 0 || trace_cap < 0) return fail(FBL_E_INVAL, "fblisa_batch_run: negative count");
    fbl_status st = check_device(bt->device);
    if (st) return st;
    for (fbl_solver *s : bt->sv)
        if (s->p.proposal && !bt->have_mlp)
            return fail(FBL_E_INVAL, "fblisa_batch_run: proposal enabled but no network set");
    cudaStream_t cs = (cudaStream_t)stream;
    if (n_steps) *n_steps = 0;
    std::vector<char> x_dev, b_dev;
    if ((st = batch_load(bt, x, b, x_dev, b_dev, cs))) return st;
    std::vector<fbl_step_stats> rec(bt->n_vol);
    fbl_status rc = FBL_OK;
    int64_t done = 0;
    for (int32_t it = 0; it < iterations; ++it) {
        rc = batch_iterate(bt, b, b_dev.data(), rec.data(), cs);
        if (trace && done < trace_cap)
            std::memcpy(trace + (size_t)done * bt->n_vol, rec.data(), bt->n_vol * sizeof(fbl_step_stats));
        if (rc) break;
        ++done;
    }
    if (n_steps) *n_steps = done;
    std::string keep = g_last_error;
    st = batch_store(bt, x, x_dev, cs);
    if (rc) {
        g_last_error = keep;
        return rc;
    }
    return st;
}

extern "C" fbl_status fblisa_batch_info(const fbl_batch *bt, int32_t *launch_cfg, int64_t *launches) {
    if (!bt) return fail(FBL_E_INVAL, "fblisa_batch_info: null batch");
    if (launch_cfg) {
        launch_cfg[0] = bt->cols;
        launch_cfg[1] = bt->split;
        launch_cfg[2] = bt->vpl;
        launch_cfg[3] = bt->ntap;
    }
    if (launches) *launches = bt->launches;
    return FBL_OK;
}

extern "C" fbl_status fblisa_batch_last_batch(const fbl_batch *bt, int32_t v, int32_t *views, int32_t cap,
                                              int32_t *n) {
    if (!bt || v < 0 || v >= bt->n_vol) return fail(FBL_E_INVAL, "fblisa_batch_last_batch: bad volume");
    return fblisa_last_batch(bt->sv[v], views, cap, n);
}
