// spg_objective_noalloc: the objective F(x) = data + l1 + TV of one volume
// computed without any device allocation, for callers that cannot call
// cudaMalloc (see include/spg.h). Its scratch (per-plane partial sums and the
// last-CTA counter) lives in a file-scope device array that every GPU loading
// this library keeps until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "spg.h"
#include "spg_trace.h"

namespace {

constexpr int kMaxPlanes = SPG_NOALLOC_MAX_PLANES;
constexpr int kThreads = 256;

// [0, 4*kMaxPlanes): per-plane partials (data, l1, tv, spare);
// [4*kMaxPlanes]: the arrival counter of the last-CTA reduction.
static __device__ __align__(256) double g_noalloc_scratch[4 * kMaxPlanes + 32];

struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// One CTA per z-plane; the last CTA sums the plane partials in plane order.
__global__ void objective_noalloc_kernel(int nx, int ny, int nz, float lambda_l1, float lambda_tv, float mu,
                                         const float *__restrict__ x, const float *__restrict__ b,
                                         const float *__restrict__ w, const float *__restrict__ om1,
                                         const float *__restrict__ omtv, double *out, double *scratch)
{
    __shared__ double red[32 * 3];
    __shared__ int last;
    const int z = blockIdx.x;
    const long long plane = (long long)nx * ny;
    KSum kd, kl, kt;
    for (int t = threadIdx.x; t < nx * ny; t += blockDim.x) {
        const int xx = t % nx, y = t / nx;
        const long long i = (long long)z * plane + t;
        const float xv = x[i];
        const float gx = xx >= 1 ? xv - x[i - 1] : 0.f;
        const float gy = y >= 1 ? xv - x[i - nx] : 0.f;
        const float gz = z >= 1 ? xv - x[i - plane] : 0.f;
        const float q = gx * gx + gy * gy + gz * gz;
        const float h = q <= mu * mu ? q * (0.5f / mu) : sqrtf(q) - 0.5f * mu;
        const float r = xv - b[i];
        kd.add(0.5f * w[i] * r * r);
        kl.add(om1[i] * fabsf(xv));
        kt.add(omtv[i] * h);
    }
    double v[3] = {kd.value(), kl.value(), kt.value()};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 3; q++) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    if (lane == 0)
        for (int q = 0; q < 3; q++) red[warp * 3 + q] = v[q];
    __syncthreads();
    unsigned int *counter = reinterpret_cast<unsigned int *>(scratch + 4 * kMaxPlanes);
    if (threadIdx.x == 0) {
        double a[3] = {0, 0, 0};
        for (int k = 0; k < (int)(blockDim.x / 32); k++)
            for (int q = 0; q < 3; q++) a[q] += red[k * 3 + q];
        for (int q = 0; q < 3; q++) scratch[(long long)z * 4 + q] = a[q];
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1 ? 1 : 0;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double d = 0, l = 0, tv = 0;
    for (int q = 0; q < nz; q++) {
        d += __ldcg(scratch + (long long)q * 4 + 0);
        l += __ldcg(scratch + (long long)q * 4 + 1);
        tv += __ldcg(scratch + (long long)q * 4 + 2);
    }
    out[0] = d;
    out[1] = (double)lambda_l1 * l;
    out[2] = (double)lambda_tv * tv;
    out[3] = out[0] + out[1] + out[2];
    *counter = 0u;
}

// The scratch array's device address belongs to one CUDA context: the primary
// context of a device, or a context the caller created with the driver API
// and made current. It is looked up once per context and cached under the
// context's ID, which the driver never reuses within a process, so a context
// created after another was destroyed (or after cudaDeviceReset) gets a fresh
// lookup.
typedef int (*PfnCtxGetCurrent)(void **ctx);
typedef int (*PfnCtxGetId)(void *ctx, unsigned long long *id);

struct DriverFns {
    PfnCtxGetCurrent get_current = nullptr;
    PfnCtxGetId get_id = nullptr;
};

const DriverFns &driver_fns()
{
    static DriverFns f = [] {
        DriverFns d;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            d.get_current = reinterpret_cast<PfnCtxGetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            d.get_id = reinterpret_cast<PfnCtxGetId>(p);
        return d;
    }();
    return f;
}

constexpr int kMaxContexts = 64;
std::mutex g_mu;
struct CacheEntry {
    unsigned long long ctx_id;
    double *ptr;
};
CacheEntry g_cache[kMaxContexts];
int g_cache_n = 0;

// Device address of the scratch array in the calling thread's current context
// (the current device's primary context unless the caller made another one
// current). `msg` names the step that failed.
cudaError_t scratch_for_current_context(double **ptr, const char **msg)
{
    const DriverFns &f = driver_fns();
    if (!f.get_current || !f.get_id) {
        *msg = "driver entry points cuCtxGetCurrent/cuCtxGetId unavailable";
        return cudaErrorNotSupported;
    }
    void *ctx = nullptr;
    if (f.get_current(&ctx) != 0) {
        *msg = "cuCtxGetCurrent failed";
        return cudaErrorDeviceUninitialized;
    }
    if (!ctx) {
        // no context yet on this thread: bind the current device's primary one
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaSetDevice(dev);
        if (e != cudaSuccess) {
            *msg = "no usable CUDA device";
            return e;
        }
        if (f.get_current(&ctx) != 0 || !ctx) {
            *msg = "no current CUDA context";
            return cudaErrorDeviceUninitialized;
        }
    }
    unsigned long long id = 0;
    if (f.get_id(ctx, &id) != 0) {
        *msg = "cuCtxGetId failed";
        return cudaErrorDeviceUninitialized;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (int i = 0; i < g_cache_n; i++)
        if (g_cache[i].ctx_id == id) {
            *ptr = g_cache[i].ptr;
            return cudaSuccess;
        }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        *msg = "cudaGetSymbolAddress of the scratch array failed";
        return e;
    }
    // a full table drops its oldest entry (contexts that old are rarely alive)
    if (g_cache_n == kMaxContexts) {
        for (int i = 1; i < kMaxContexts; i++) g_cache[i - 1] = g_cache[i];
        g_cache_n--;
    }
    g_cache[g_cache_n++] = CacheEntry{id, static_cast<double *>(p)};
    *ptr = static_cast<double *>(p);
    return cudaSuccess;
}

thread_local char g_noalloc_msg[256] = "no error";

spg_status noalloc_fail(spg_status st, const char *what, cudaError_t e)
{
    if (e != cudaSuccess)
        snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "spg_objective_noalloc: %s (%s)", what, cudaGetErrorString(e));
    else
        snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "spg_objective_noalloc: %s", what);
    return st;
}

}  // namespace

extern "C" const char *spg_noalloc_last_error(void) { return g_noalloc_msg; }

extern "C" spg_status spg_objective_noalloc(int nx, int ny, int nz, float lambda_l1, float lambda_tv, float mu,
                                            const float *x, const float *b, const float *w, const float *om1,
                                            const float *omtv, double *out, void *stream)
{
    SPG_TRACE();
    if (nx <= 0 || ny <= 0 || nz <= 0 || !x || !b || !w || !om1 || !omtv || !out || !(mu > 0.f))
        return noalloc_fail(SPG_EINVAL, "bad arguments", cudaSuccess);
    if (nz > kMaxPlanes)
        return noalloc_fail(SPG_EINVAL, "nz exceeds SPG_NOALLOC_MAX_PLANES (4096)", cudaSuccess);
    if ((long long)nx * ny > (1LL << 30)) return noalloc_fail(SPG_EINVAL, "plane too large", cudaSuccess);
    double *scratch = nullptr;
    const char *what = "scratch set-up failed";
    cudaError_t e = scratch_for_current_context(&scratch, &what);
    if (e != cudaSuccess) return noalloc_fail(SPG_ECUDA, what, e);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the arrival counter must start at zero on every call
    e = cudaMemsetAsync(scratch + 4 * kMaxPlanes, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return noalloc_fail(SPG_ECUDA, "clearing the scratch counter failed", e);
    // cudaLaunchKernel reports this launch's own error (no stale error of
    // earlier, unrelated work is picked up from the runtime's last-error slot)
    void *args[] = {&nx, &ny, &nz, &lambda_l1, &lambda_tv, &mu, &x, &b, &w, &om1, &omtv, &out, &scratch};
    e = cudaLaunchKernel(reinterpret_cast<const void *>(objective_noalloc_kernel), dim3(nz), dim3(kThreads), args,
                         0, s);
    if (e != cudaSuccess) return noalloc_fail(SPG_ECUDA, "kernel launch failed", e);
    snprintf(g_noalloc_msg, sizeof(g_noalloc_msg), "no error");
    return SPG_OK;
}
