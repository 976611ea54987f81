// Fourier shell correlation of two maps (Sec. 2.3, Eq. 30) on the GPU:
// cuFFT real-to-complex transforms of both maps, then one pass that bins
// every coefficient of the half spectrum into its shell and accumulates
// Re(F G*), |F|^2 and |G|^2 in double precision. Coefficients with
// 0 < h < n/2 stand for themselves and their conjugates (weight 2).
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <string>
#include <vector>

#include "spg.h"
#include "spg_trace.h"
#include "spg_cufft.h"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = 1216;  // 8 per SM on 152 SMs

thread_local std::string g_fsc_err = "no error";

// Nearest integer to sqrt(r2) for an integer r2 (no tie: (s + 1/2)^2 is never an integer).
__device__ __forceinline__ int shell_of(long long r2)
{
    long long s = (long long)sqrt((double)r2);
    while (s * s > r2) s--;
    while ((s + 1) * (s + 1) <= r2) s++;
    return (int)(r2 > s * s + s ? s + 1 : s);
}

__device__ __forceinline__ int freq(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }

// Per-block shell sums in shared memory, written to partials[block][shell][3].
__global__ void fsc_shell_kernel(const cufftComplex *__restrict__ F, const cufftComplex *__restrict__ G, int n,
                                 int nshell, double *partials)
{
    extern __shared__ double acc[];  // [nshell][3]
    for (int i = threadIdx.x; i < nshell * 3; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    const int nh = n / 2 + 1;
    const long long total = (long long)n * n * nh;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int h = (int)(q % nh);
        const int k = (int)((q / nh) % n);
        const int l = (int)(q / ((long long)nh * n));
        const long long fk = freq(k, n), fl = freq(l, n);
        const int s = shell_of((long long)h * h + fk * fk + fl * fl);
        if (s >= nshell) continue;
        const double wgt = (h == 0 || (n % 2 == 0 && h == n / 2)) ? 1.0 : 2.0;
        const cufftComplex a = F[q], b = G[q];
        const double re = (double)a.x * b.x + (double)a.y * b.y;
        const double fa = (double)a.x * a.x + (double)a.y * a.y;
        const double gb = (double)b.x * b.x + (double)b.y * b.y;
        atomicAdd(&acc[s * 3 + 0], wgt * re);
        atomicAdd(&acc[s * 3 + 1], wgt * fa);
        atomicAdd(&acc[s * 3 + 2], wgt * gb);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nshell * 3; i += blockDim.x) partials[(long long)blockIdx.x * nshell * 3 + i] = acc[i];
}

// Sum the block partials of every shell in block order; out[shell][3].
__global__ void fsc_reduce_kernel(const double *partials, int nblocks, int nshell, double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nshell * 3) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; b++) s += partials[(long long)b * nshell * 3 + i];
    out[i] = s;
}

// Coefficient counts per shell (full spectrum), independent of the data.
__global__ void fsc_count_kernel(int n, int nshell, unsigned long long *counts)
{
    const int nh = n / 2 + 1;
    const long long total = (long long)n * n * nh;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int h = (int)(q % nh);
        const int k = (int)((q / nh) % n);
        const int l = (int)(q / ((long long)nh * n));
        const long long fk = freq(k, n), fl = freq(l, n);
        const int s = shell_of((long long)h * h + fk * fk + fl * fl);
        if (s >= nshell) continue;
        const unsigned long long wgt = (h == 0 || (n % 2 == 0 && h == n / 2)) ? 1ull : 2ull;
        atomicAdd(&counts[s], wgt);
    }
}

struct Buf {
    void *p = nullptr;
    ~Buf()
    {
        if (p) cudaFree(p);
    }
};

struct Plan {
    cufftHandle h = 0;
    bool made = false;
    ~Plan()
    {
        if (made) spg::cufft_api().destroy(h);
    }
};

spg_status fsc_fail(spg_status s, const std::string &m)
{
    g_fsc_err = m;
    return s;
}

}  // namespace

extern "C" const char *spg_fsc_last_error(void) { return g_fsc_err.c_str(); }

extern "C" spg_status spg_fsc(int n, const float *a, const float *b, int max_shells, double *fsc, double *counts,
                              void *stream)
{
    SPG_TRACE();
    if (n < 2 || !a || !b || !fsc || max_shells < n / 2 + 1)
        return fsc_fail(SPG_EINVAL, "spg_fsc: bad arguments (n >= 2, max_shells >= n/2 + 1)");
    if ((long long)n * n * n > (1LL << 31)) return fsc_fail(SPG_EINVAL, "spg_fsc: volume too large");
    const int nshell = n / 2 + 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t vox = (size_t)n * n * n;
    const size_t ncplx = (size_t)n * n * (n / 2 + 1);
    Buf ra, rb, fa, fb, part, sums, cnt;
    cudaError_t e;
#define FSC_CK(call)                                                                                \
    do {                                                                                            \
        e = (call);                                                                                 \
        if (e != cudaSuccess) {                                                                     \
            cudaGetLastError();                                                                     \
            return fsc_fail(e == cudaErrorMemoryAllocation ? SPG_ENOMEM : SPG_ECUDA,                \
                            std::string("spg_fsc: ") + cudaGetErrorString(e));                      \
        }                                                                                           \
    } while (0)
    FSC_CK(cudaMalloc(&ra.p, vox * sizeof(float)));
    FSC_CK(cudaMalloc(&rb.p, vox * sizeof(float)));
    FSC_CK(cudaMalloc(&fa.p, ncplx * sizeof(cufftComplex)));
    FSC_CK(cudaMalloc(&fb.p, ncplx * sizeof(cufftComplex)));
    FSC_CK(cudaMalloc(&part.p, (size_t)kBlocks * nshell * 3 * sizeof(double)));
    FSC_CK(cudaMalloc(&sums.p, (size_t)nshell * 3 * sizeof(double)));
    FSC_CK(cudaMalloc(&cnt.p, (size_t)nshell * sizeof(unsigned long long)));
    FSC_CK(cudaMemcpyAsync(ra.p, a, vox * sizeof(float), cudaMemcpyDefault, s));
    FSC_CK(cudaMemcpyAsync(rb.p, b, vox * sizeof(float), cudaMemcpyDefault, s));
    const size_t smem = (size_t)nshell * 3 * sizeof(double);
    if (smem > 48 * 1024) return fsc_fail(SPG_EINVAL, "spg_fsc: too many shells (n <= 2046)");
    const spg::CufftApi &cf = spg::cufft_api();
    if (!cf.ok) return fsc_fail(SPG_ECUDA, "spg_fsc: cuFFT library could not be loaded");
    Plan plan;
    if (cf.plan3d(&plan.h, n, n, n, CUFFT_R2C) != CUFFT_SUCCESS) return fsc_fail(SPG_ECUDA, "spg_fsc: cufft plan");
    plan.made = true;
    const bool ok =
        cf.set_stream(plan.h, s) == CUFFT_SUCCESS &&
        cf.exec_r2c(plan.h, static_cast<cufftReal *>(ra.p), static_cast<cufftComplex *>(fa.p)) == CUFFT_SUCCESS &&
        cf.exec_r2c(plan.h, static_cast<cufftReal *>(rb.p), static_cast<cufftComplex *>(fb.p)) == CUFFT_SUCCESS;
    if (!ok) return fsc_fail(SPG_ECUDA, "spg_fsc: cufft execution");
    fsc_shell_kernel<<<kBlocks, kThreads, smem, s>>>(static_cast<cufftComplex *>(fa.p),
                                                      static_cast<cufftComplex *>(fb.p), n, nshell,
                                                      static_cast<double *>(part.p));
    fsc_reduce_kernel<<<(nshell * 3 + 255) / 256, 256, 0, s>>>(static_cast<double *>(part.p), kBlocks, nshell,
                                                                static_cast<double *>(sums.p));
    FSC_CK(cudaMemsetAsync(cnt.p, 0, (size_t)nshell * sizeof(unsigned long long), s));
    fsc_count_kernel<<<kBlocks, kThreads, 0, s>>>(n, nshell, static_cast<unsigned long long *>(cnt.p));
    FSC_CK(cudaGetLastError());
    std::vector<double> hs((size_t)nshell * 3);
    std::vector<unsigned long long> hc(nshell);
    FSC_CK(cudaMemcpyAsync(hs.data(), sums.p, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    FSC_CK(cudaMemcpyAsync(hc.data(), cnt.p, hc.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    FSC_CK(cudaStreamSynchronize(s));
#undef FSC_CK
    for (int k = 0; k < nshell; k++) {
        const double d = std::sqrt(hs[k * 3 + 1] * hs[k * 3 + 2]);
        fsc[k] = d > 0 ? hs[k * 3 + 0] / d : NAN;
        if (counts) counts[k] = (double)hc[k];
    }
    return SPG_OK;
}
