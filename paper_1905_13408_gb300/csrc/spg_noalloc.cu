// spg_objective_noalloc: the objective F(x) = data + l1 + TV of one volume
// computed without any device allocation, for callers that cannot call
// cudaMalloc (see include/spg.h). Its scratch (per-plane partial sums and the
// last-CTA counter) lives in a file-scope device array that every GPU loading
// this library keeps until the process exits.
#include <cuda_runtime.h>

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

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (set up once per
// device, with that device current).
cudaError_t scratch_for_current_device(double **ptr, int *dev_out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *ptr = g_scratch_ptr[dev];
    *dev_out = dev;
    return cudaSuccess;
}

thread_local const char *g_noalloc_err = "no error";

}  // namespace

extern "C" const char *spg_noalloc_last_error(void) { return g_noalloc_err; }

extern "C" spg_status spg_objective_noalloc(int nx, int ny, int nz, float lambda_l1, float lambda_tv, float mu,
                                            const float *x, const float *b, const float *w, const float *om1,
                                            const float *omtv, double *out, void *stream)
{
    SPG_TRACE();
    if (nx <= 0 || ny <= 0 || nz <= 0 || !x || !b || !w || !om1 || !omtv || !out || !(mu > 0.f)) {
        g_noalloc_err = "spg_objective_noalloc: bad arguments";
        return SPG_EINVAL;
    }
    if (nz > kMaxPlanes) {
        g_noalloc_err = "spg_objective_noalloc: nz exceeds SPG_NOALLOC_MAX_PLANES (4096)";
        return SPG_EINVAL;
    }
    if ((long long)nx * ny > (1LL << 30)) {
        g_noalloc_err = "spg_objective_noalloc: plane too large";
        return SPG_EINVAL;
    }
    double *scratch = nullptr;
    int dev = 0;
    cudaError_t e = scratch_for_current_device(&scratch, &dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g_noalloc_err = "spg_objective_noalloc: scratch set-up failed (no usable CUDA device?)";
        return SPG_ECUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the arrival counter must start at zero on every call
    e = cudaMemsetAsync(scratch + 4 * kMaxPlanes, 0, sizeof(unsigned int), s);
    if (e == cudaSuccess) {
        objective_noalloc_kernel<<<nz, kThreads, 0, s>>>(nx, ny, nz, lambda_l1, lambda_tv, mu, x, b, w, om1, omtv,
                                                         out, scratch);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        g_noalloc_err = "spg_objective_noalloc: launch failed";
        return SPG_ECUDA;
    }
    return SPG_OK;
}
