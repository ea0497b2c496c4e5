// prox_reduce_static: the prox + line-search reductions of prox_reduce for
// callers that cannot allocate device memory.  The per-block partial sums and
// the three results live in a fixed, file-scope device array instead of
// memory obtained from cudaMalloc/cudaMallocAsync; nothing is allocated on any
// call.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on it.  The launch is the one prox_reduce makes (same grid,
// same fixed-order reduction), so both calls return identical sums.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "fbl_internal.cuh"

namespace {

// The grid-stride prox kernel runs on prox_flat_num_partials(n) blocks, never
// more than PROX_STATIC_MAX_BLOCKS; sizes are capped at n <= 2^27 elements
// (a 512^3 volume).
constexpr int PROX_STATIC_MAX_BLOCKS = 152 * 16;
constexpr long long PROX_STATIC_MAX_N = 1LL << 27;

// [0, 3*MAX_BLOCKS): partial sums (three components, stride = blocks used);
// [3*MAX_BLOCKS, 3*MAX_BLOCKS + 3): the reduced results.  57 KiB per device.
static __device__ __align__(256) double g_prox_scratch[3 * PROX_STATIC_MAX_BLOCKS + 4];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

fbl_status fail(fbl_status st, const char *msg) {
    fbl::set_last_error(msg);
    return st;
}

fbl_status fail_cuda(cudaError_t e, const char *what) {
    char buf[256];
    snprintf(buf, sizeof buf, "prox_reduce_static: %s: %s", what, cudaGetErrorString(e));
    fbl::set_last_error(buf);
    return FBL_E_CUDA;
}

// True when p is device (or managed) memory of device dev.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

// Device address of g_prox_scratch on device dev, the current device (looked
// up once per device and cached; not valid after a cudaDeviceReset).
fbl_status scratch_for_device(int dev, double **out) {
    cudaError_t e;
    if (dev < 0 || dev >= kMaxDevices) return fail(FBL_E_UNSUPPORTED, "prox_reduce_static: device index too large");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_prox_scratch);
        if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress");
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return FBL_OK;
}

}  // namespace

extern "C" fbl_status prox_reduce_static(const void *x, int32_t x_dtype, const float *g, int64_t n,
                                         double alpha, double mu, void *xbar, double *out3_host,
                                         void *stream) {
    if (!out3_host) return fail(FBL_E_INVAL, "prox_reduce_static: null argument");
    if (x_dtype != FBL_F32 && x_dtype != FBL_BF16 && x_dtype != FBL_F16)
        return fail(FBL_E_INVAL, "prox_reduce_static: bad dtype");
    if (n < 0) return fail(FBL_E_INVAL, "prox_reduce_static: negative size");
    if (n == 0) {  // empty sums; the buffers (possibly NULL) are not touched
        out3_host[0] = out3_host[1] = out3_host[2] = 0.0;
        return FBL_OK;
    }
    if (!x || !g || !xbar) return fail(FBL_E_INVAL, "prox_reduce_static: null argument");
    if (n > PROX_STATIC_MAX_N) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "prox_reduce_static: n = %lld exceeds the fixed scratch capacity of %lld elements",
                 (long long)n, PROX_STATIC_MAX_N);
        return fail(FBL_E_INVAL, buf);
    }
    if (x == xbar) return fail(FBL_E_INVAL, "prox_reduce_static: x_bar must not alias x");
    if (!(alpha > 0) || !std::isfinite(alpha) || !std::isfinite(mu))
        return fail(FBL_E_INVAL, "prox_reduce_static: need alpha > 0 and finite mu");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
    if (!on_device(x, dev) || !on_device(g, dev) || !on_device(xbar, dev))
        return fail(FBL_E_INVAL,
                    "prox_reduce_static: x, g and x_bar must be memory of the current device "
                    "(no staging is allocated)");
    double *scratch = nullptr;
    fbl_status st = scratch_for_device(dev, &scratch);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = fbl::prox_flat_num_partials(n);
    if (nb < 1 || nb > PROX_STATIC_MAX_BLOCKS)
        return fail(FBL_E_INVAL, "prox_reduce_static: grid larger than the fixed scratch");
    double *results = scratch + 3 * PROX_STATIC_MAX_BLOCKS;
    e = fbl::launch_prox_flat_grid(x, g, n, (float)alpha, (float)(alpha * mu), xbar, x_dtype, nb, scratch, s);
    if (e != cudaSuccess) return fail_cuda(e, "prox kernel");
    e = fbl::launch_reduce(scratch, nb, nb, 3, results, s);
    if (e != cudaSuccess) return fail_cuda(e, "reduce kernel");
    e = cudaMemcpyAsync(out3_host, results, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return fail_cuda(e, "result copy");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e, "synchronize");
    return FBL_OK;
}
