// Kernel-regression back-projection (Sec. 2.2, Eq. 24-28) on the GPU.
//
// Image i's coefficient X at 2-D frequency index (kx, ky) lands at the 3-D
// position p = R_i (kx, ky, 0) (Eq. 24). Every grid point n of the kernel's
// support around p receives
//     num(n) += P K CTF X,    N(n) += P K CTF^2        (Eq. 26-28)
// with P the posterior weight of the image-pose pair (1 for known poses)
// with K = exp(-|p - n|^2 / h) on the 27 points round(p) + {-1,0,1}^3 (the
// Gaussian kernel of Sec. 2.2) or the trilinear weights on the 8 corners of
// p's cell (the interpolation kernel the paper attributes to Relion). One
// thread per image coefficient scatters with double-precision atomics into
// full-spectrum accumulators; a second pass writes the half spectrum of the
// Eq. 31 data term: N' = V N and y = (-1)^(kx+ky+kz) num / sqrt(N), the sign
// moving the transform's origin from the box centre (image convention) to
// voxel 0 (the solver's convention; n even).
#include <cuda_runtime.h>

#include <string>

#include "spg.h"

namespace {

thread_local std::string g_grid_err = "no error";

__device__ __forceinline__ int fidx(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }
__device__ __forceinline__ int wrap(int i, int n) { return ((i % n) + n) % n; }

__global__ void scatter_kernel(int n, int m, const float *__restrict__ rot, const float2 *__restrict__ X,
                               const float *__restrict__ ctf, const float *__restrict__ pw, int kernel, float h,
                               double *num_re, double *num_im, double *N)
{
    const long long per_image = (long long)n * n;
    const long long total = per_image * m;
    const float rmax2 = (n * 0.5f - 2.0f) * (n * 0.5f - 2.0f);
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int img = (int)(q / per_image);
        const int rem = (int)(q % per_image);
        const int ky = fidx(rem / n, n), kx = fidx(rem % n, n);
        if ((float)(kx * kx + ky * ky) > rmax2) continue;
        const float *R = rot + (long long)img * 9;  // row-major 3x3; columns 0 and 1 span the image plane
        // positions in double so the nearest-point decisions match a double-precision reference
        const double px = __dadd_rn(__dmul_rn(R[0], kx), __dmul_rn(R[1], ky));
        const double py = __dadd_rn(__dmul_rn(R[3], kx), __dmul_rn(R[4], ky));
        const double pz = __dadd_rn(__dmul_rn(R[6], kx), __dmul_rn(R[7], ky));
        const float2 x = X[q];
        const float c = ctf[q];
        const double pc = pw ? (double)pw[img] * c : (double)c;
        const double cx = pc * x.x, cy = pc * x.y, cc = pc * c;
        if (kernel == 0) {
            const int bx = __double2int_rn(px), by = __double2int_rn(py), bz = __double2int_rn(pz);
            for (int dz = -1; dz <= 1; dz++)
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        const double ex = px - (bx + dx), ey = py - (by + dy), ez = pz - (bz + dz);
                        const double K = exp(-(ex * ex + ey * ey + ez * ez) / h);
                        const long long g =
                            ((long long)wrap(bz + dz, n) * n + wrap(by + dy, n)) * n + wrap(bx + dx, n);
                        atomicAdd(num_re + g, K * cx);
                        atomicAdd(num_im + g, K * cy);
                        atomicAdd(N + g, K * cc);
                    }
        } else {
            const int bx = (int)floor(px), by = (int)floor(py), bz = (int)floor(pz);
            for (int dz = 0; dz <= 1; dz++)
                for (int dy = 0; dy <= 1; dy++)
                    for (int dx = 0; dx <= 1; dx++) {
                        const double K = (1.0 - fabs(px - (bx + dx))) * (1.0 - fabs(py - (by + dy))) *
                                         (1.0 - fabs(pz - (bz + dz)));
                        const long long g =
                            ((long long)wrap(bz + dz, n) * n + wrap(by + dy, n)) * n + wrap(bx + dx, n);
                        atomicAdd(num_re + g, K * cx);
                        atomicAdd(num_im + g, K * cy);
                        atomicAdd(N + g, K * cc);
                    }
        }
    }
}

__global__ void finalize_kernel(int n, const double *num_re, const double *num_im, const double *N, float2 *y_half,
                                float *N_half)
{
    const int nh = n / 2 + 1;
    const long long total = (long long)n * n * nh;
    const double V = (double)n * n * n;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(q % nh);
        const int ky = (int)((q / nh) % n);
        const int kz = (int)(q / ((long long)nh * n));
        const long long g = ((long long)kz * n + ky) * n + kx;
        const double w = N[g];
        const double sgn = ((kx + ky + kz) & 1) ? -1.0 : 1.0;
        float2 y = make_float2(0.f, 0.f);
        if (w > 0) {
            const double s = sgn / sqrt(w);
            y = make_float2((float)(num_re[g] * s), (float)(num_im[g] * s));
        }
        y_half[q] = y;
        N_half[q] = (float)(V * w);
    }
}

struct Buf {
    void *p = nullptr;
    ~Buf()
    {
        if (p) cudaFree(p);
    }
};

spg_status grid_fail(spg_status s, const std::string &m)
{
    g_grid_err = m;
    return s;
}

}  // namespace

extern "C" const char *spg_backproject_last_error(void) { return g_grid_err.c_str(); }

extern "C" spg_status spg_backproject(int n, int m, const float *rot, const void *X, const float *ctf,
                                      const float *pw, int kernel, float h, void *y_half, float *N_half, void *stream)
{
    if (n < 4 || n % 2 || m < 1 || !rot || !X || !ctf || !y_half || !N_half || (kernel != 0 && kernel != 1) ||
        !(h > 0.f))
        return grid_fail(SPG_EINVAL, "spg_backproject: bad arguments (even n >= 4, m >= 1, kernel 0 or 1, h > 0)");
    if ((long long)n * n * n > (1LL << 31)) return grid_fail(SPG_EINVAL, "spg_backproject: volume too large");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t vox = (size_t)n * n * n;
    const size_t img = (size_t)m * n * n;
    Buf re, im, nn, dR, dX, dC, dP;
    cudaError_t e;
#define GRID_CK(call)                                                                              \
    do {                                                                                           \
        e = (call);                                                                                \
        if (e != cudaSuccess) {                                                                    \
            cudaGetLastError();                                                                    \
            return grid_fail(e == cudaErrorMemoryAllocation ? SPG_ENOMEM : SPG_ECUDA,              \
                             std::string("spg_backproject: ") + cudaGetErrorString(e));            \
        }                                                                                          \
    } while (0)
    GRID_CK(cudaMalloc(&re.p, vox * sizeof(double)));
    GRID_CK(cudaMalloc(&im.p, vox * sizeof(double)));
    GRID_CK(cudaMalloc(&nn.p, vox * sizeof(double)));
    GRID_CK(cudaMalloc(&dR.p, (size_t)m * 9 * sizeof(float)));
    GRID_CK(cudaMalloc(&dX.p, img * sizeof(float2)));
    GRID_CK(cudaMalloc(&dC.p, img * sizeof(float)));
    GRID_CK(cudaMemsetAsync(re.p, 0, vox * sizeof(double), s));
    GRID_CK(cudaMemsetAsync(im.p, 0, vox * sizeof(double), s));
    GRID_CK(cudaMemsetAsync(nn.p, 0, vox * sizeof(double), s));
    GRID_CK(cudaMemcpyAsync(dR.p, rot, (size_t)m * 9 * sizeof(float), cudaMemcpyDefault, s));
    GRID_CK(cudaMemcpyAsync(dX.p, X, img * sizeof(float2), cudaMemcpyDefault, s));
    GRID_CK(cudaMemcpyAsync(dC.p, ctf, img * sizeof(float), cudaMemcpyDefault, s));
    if (pw) {
        GRID_CK(cudaMalloc(&dP.p, (size_t)m * sizeof(float)));
        GRID_CK(cudaMemcpyAsync(dP.p, pw, (size_t)m * sizeof(float), cudaMemcpyDefault, s));
    }
    scatter_kernel<<<4864, 256, 0, s>>>(n, m, static_cast<float *>(dR.p), static_cast<float2 *>(dX.p),
                                        static_cast<float *>(dC.p), static_cast<float *>(dP.p), kernel, h,
                                        static_cast<double *>(re.p),
                                        static_cast<double *>(im.p), static_cast<double *>(nn.p));
    GRID_CK(cudaGetLastError());
    const size_t half = (size_t)n * n * (n / 2 + 1);
    Buf yo, no;
    GRID_CK(cudaMalloc(&yo.p, half * sizeof(float2)));
    GRID_CK(cudaMalloc(&no.p, half * sizeof(float)));
    finalize_kernel<<<4864, 256, 0, s>>>(n, static_cast<double *>(re.p), static_cast<double *>(im.p),
                                         static_cast<double *>(nn.p), static_cast<float2 *>(yo.p),
                                         static_cast<float *>(no.p));
    GRID_CK(cudaGetLastError());
    GRID_CK(cudaMemcpyAsync(y_half, yo.p, half * sizeof(float2), cudaMemcpyDefault, s));
    GRID_CK(cudaMemcpyAsync(N_half, no.p, half * sizeof(float), cudaMemcpyDefault, s));
    GRID_CK(cudaStreamSynchronize(s));
#undef GRID_CK
    return SPG_OK;
}
