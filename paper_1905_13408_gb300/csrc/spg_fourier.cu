// Kernels of the Fourier-domain data term (Sec. 2.5, Eq. 31):
//   1/2 |y - D A x|^2, A the unitary DFT, D = diag sqrt(N),
// whose gradient A^H (N A x - D y) is formed each iteration at the
// extrapolated point y_k by per-plane real-to-complex transforms (cuFFT), one
// pass along z that transforms, scales by N, subtracts the data spectrum and
// transforms back (spg_zfft.cu, power-of-two nz), and per-plane
// complex-to-real transforms; for other nz by 3-D transforms around a
// separate spectrum pass (spec_scale_kernel). The fused step consumes it. Subtracting before the inverse transform
// keeps FP32 rounding relative to the residual rather than to A^H N A y_k,
// which for the strongly uneven N of gridded data (many orders of magnitude
// between low and high frequencies) is the difference between errors of 1e-7
// and 1e-5 after a hundred iterations.
// Spectra use the real-to-complex half layout [nz][ny][nx/2+1]; this file
// holds the data preparation, value and scale kernels.
#include "spg_internal.h"

namespace spg {
namespace {

// y_k = x_k + beta d_k, with x_k = X[cur], d_k = X[2 + cur] (increment storage).
__global__ void form_y_kernel(const DevState *st, const VolDesc *vols, const float *beta, float *x0, float *x1,
                              float *d0, float *d1, float *y, long long n)
{
    const int cur = st->cur;
    const float b = beta[vols[0].kmom];
    const float *x = cur == 0 ? x0 : x1;
    const float *d = cur == 0 ? d0 : d1;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = fmaf(b, d[i], x[i]);
}

// F <- N F scale - C: the unnormalised spectrum of the residual (scale = 1/V,
// C = sqrt(N) y / sqrt(V)), the separate spectrum pass between 3-D transforms.
__global__ void spec_scale_kernel(float2 *F, const float *N, const float2 *C, long long n, float scale)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float m = N[i] * scale;
        const float2 c = C[i];
        float2 f = F[i];
        f.x = fmaf(f.x, m, -c.x);
        f.y = fmaf(f.y, m, -c.y);
        F[i] = f;
    }
}

__global__ void spec_prep_kernel(float2 *F, const float2 *Y, const float *N, long long n, float scale)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float m = sqrtf(N[i]) * scale;
        const float2 y = Y[i];
        F[i] = make_float2(y.x * m, y.y * m);
    }
}

// The implicit-gradient term gamma |x - a|^2 (Eq. 22, Eq. 31) in the
// spectrum pass: its gradient 2 gamma (y - a) = A^H (2 gamma A y - 2 gamma A a),
// so the step uses N + 2 gamma and C + 2 gamma FA / V (FA the unnormalised
// transform of the anchor a).
__global__ void spec_anchor_kernel(const float *N, const float2 *C, const float2 *FA, long long n, float two_gamma,
                                   float inv_v, float *Nst, float2 *Cst)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        Nst[i] = N[i] + two_gamma;
        const float2 c = C[i], f = FA[i];
        Cst[i] = make_float2(fmaf(two_gamma * inv_v, f.x, c.x), fmaf(two_gamma * inv_v, f.y, c.y));
    }
}

// sum over the volume's voxels of (x - a)^2 (pitched layout, padding skipped).
__global__ void sq_diff_kernel(const float *x, const float *a, int nx, int pitch, long long n, double *partials)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if ((int)(i % pitch) >= nx) continue;
        const double d = (double)x[i] - (double)a[i];
        acc += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); w++) s += red[w];
        partials[blockIdx.x] = s;
    }
}

__global__ void spec_max_kernel(const float *N, long long n, unsigned int *out)
{
    float m = 0.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, N[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    // non-negative floats order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// Half-spectrum sum of 1/2 |Y - sqrt(N) F scale|^2, coefficients 0 < h < nx/2
// counted twice. A block walks whole rows (no index division per element).
// The data term's residual cancels Y against sqrt(N) F scale, so m =
// sqrt(N) scale is carried as a pair of floats (m_hi + m_lo, about 44
// significant bits) and the product m F is split exactly by fused
// multiply-adds (Dekker's two-product); the residual
// r = (Y - m_hi F) - (m_lo F + the product's rounding) is then accurate to
// float rounding of r itself, as a double evaluation would be, without the
// double-precision pipe (narrow on this GPU). sqrt(N): s0 = N rsqrt(N) in
// float and one Newton correction (N - s0^2) / (2 s0), its numerator formed
// by one fused multiply-add. Per thread the squares are summed compensated
// (Kahan) in float; blocks reduce in double.
__global__ void spec_value_kernel(const float2 *F, const float2 *Y, const float *N, int nz, int ny, int nx,
                                  float scale, double *partials)
{
    __shared__ double red[32];
    const int nxh = nx / 2 + 1;
    const long long rows = (long long)nz * ny;
    float sum = 0.f, comp = 0.f;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        const long long o = r * nxh;
        for (int h = threadIdx.x; h < nxh; h += blockDim.x) {
            const float nf = N[o + h];
            float mh = 0.f, ml = 0.f;
            if (nf > 0.f) {
                const float rs = rsqrtf(nf);
                const float s0 = nf * rs;
                const float sl = 0.5f * fmaf(-s0, s0, nf) * rs;  // sqrt(N) ~ s0 + sl
                mh = s0 * scale;
                ml = fmaf(s0, scale, -mh) + sl * scale;
            }
            const float2 f = F[o + h], y = Y[o + h];
            const float px = mh * f.x, py = mh * f.y;
            const float rx = (y.x - px) - (fmaf(mh, f.x, -px) + ml * f.x);
            const float ry = (y.y - py) - (fmaf(mh, f.y, -py) + ml * f.y);
            const float wgt = (h == 0 || (nx % 2 == 0 && h == nx / 2)) ? 0.5f : 1.0f;
            const float v = wgt * fmaf(rx, rx, ry * ry) - comp;
            const float t = sum + v;
            comp = (t - sum) - v;
            sum = t;
        }
    }
    double acc = (double)sum - (double)comp;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); w++) s += red[w];
        partials[blockIdx.x] = s;
    }
}

// Sec. 2.5 scales from the spectrum, full-spectrum sums through the half
// layout (coefficients 0 < h < nx/2 counted twice): partials[block] =
// {sum |C|^2, sum N, max N, min N} with C = sqrt(N) y / sqrt(V), so that
// sum |C|^2 = |D y|^2 / V = |A^H D y|^2 / V (A unitary) = RMS(A^H D y)^2.
__global__ void spec_scales_kernel(const float2 *C, const float *N, int nz, int ny, int nx, double *partials)
{
    __shared__ double red[4][32];
    const int nxh = nx / 2 + 1;
    const long long n = (long long)nz * ny * nxh;
    double s1 = 0.0, s2 = 0.0, mx = 0.0, mn = 1e300;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int h = (int)(i % nxh);
        const double wgt = (h == 0 || (nx % 2 == 0 && h == nx / 2)) ? 1.0 : 2.0;
        const double cx = C[i].x, cy = C[i].y, nv = N[i];
        s1 += wgt * (cx * cx + cy * cy);
        s2 += wgt * nv;
        mx = fmax(mx, nv);
        mn = fmin(mn, nv);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
        mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s1;
        red[1][threadIdx.x >> 5] = s2;
        red[2][threadIdx.x >> 5] = mx;
        red[3][threadIdx.x >> 5] = mn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0, d = 1e300;
        for (int w = 0; w < (int)(blockDim.x / 32); w++) {
            a += red[0][w];
            b += red[1][w];
            c = fmax(c, red[2][w]);
            d = fmin(d, red[3][w]);
        }
        double *p = partials + (long long)blockIdx.x * 4;
        p[0] = a;
        p[1] = b;
        p[2] = c;
        p[3] = d;
    }
}

__global__ void sum_scales_kernel(const double *partials, int nblocks, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double a = 0.0, b = 0.0, c = 0.0, d = 1e300;
        for (int i = 0; i < nblocks; i++) {
            a += partials[i * 4 + 0];
            b += partials[i * 4 + 1];
            c = fmax(c, partials[i * 4 + 2]);
            d = fmin(d, partials[i * 4 + 3]);
        }
        out[0] = a;
        out[1] = b;
        out[2] = c;
        out[3] = d;
    }
}

// One warp, fixed order: lane l sums partials l, l + 32, ... (its loads in
// flight together), then a fixed tree over the lanes.
__global__ void sum_partials_kernel(const double *partials, int n, double *out)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 32) s += partials[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
}

int grid_for(long long n)
{
    long long g = (n + 255) / 256;
    return (int)(g < 4864 ? (g > 0 ? g : 1) : 4864);
}

}  // namespace

cudaError_t launch_form_y(const DevState *st, const VolDesc *vols, const float *beta, float *const *xbuf, float *y,
                          long long n, cudaStream_t s)
{
    form_y_kernel<<<grid_for(n), 256, 0, s>>>(st, vols, beta, xbuf[0], xbuf[1], xbuf[2], xbuf[3], y, n);
    return cudaGetLastError();
}

cudaError_t launch_spec_scale(float2 *F, const float *N, const float2 *C, long long n, float scale, cudaStream_t s)
{
    spec_scale_kernel<<<grid_for(n), 256, 0, s>>>(F, N, C, n, scale);
    return cudaGetLastError();
}

cudaError_t launch_spec_prep(float2 *F, const float2 *Y, const float *N, long long n, float scale, cudaStream_t s)
{
    spec_prep_kernel<<<grid_for(n), 256, 0, s>>>(F, Y, N, n, scale);
    return cudaGetLastError();
}

cudaError_t launch_spec_max(const float *N, long long n, float *out, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    spec_max_kernel<<<grid_for(n), 256, 0, s>>>(N, n, reinterpret_cast<unsigned int *>(out));
    return cudaGetLastError();
}

cudaError_t launch_spec_data_value(const float2 *F, const float2 *Y, const float *N, int nz, int ny, int nx,
                                   float scale, double *partials, double *out, cudaStream_t s)
{
    const int g = 1024;
    spec_value_kernel<<<g, 256, 0, s>>>(F, Y, N, nz, ny, nx, scale, partials);
    sum_partials_kernel<<<1, 32, 0, s>>>(partials, g, out);
    return cudaGetLastError();
}

cudaError_t launch_spec_scales(const float2 *C, const float *N, int nz, int ny, int nx, double *partials,
                               double *out, cudaStream_t s)
{
    const int g = 1024;
    spec_scales_kernel<<<g, 256, 0, s>>>(C, N, nz, ny, nx, partials);
    sum_scales_kernel<<<1, 32, 0, s>>>(partials, g, out);
    return cudaGetLastError();
}

cudaError_t launch_spec_anchor(const float *N, const float2 *C, const float2 *FA, long long n, float two_gamma,
                               float inv_v, float *Nst, float2 *Cst, cudaStream_t s)
{
    spec_anchor_kernel<<<grid_for(n), 256, 0, s>>>(N, C, FA, n, two_gamma, inv_v, Nst, Cst);
    return cudaGetLastError();
}

cudaError_t launch_sq_diff(const float *x, const float *a, int nx, int pitch, long long n, double *partials,
                           double *out, cudaStream_t s)
{
    const int g = 1024;
    sq_diff_kernel<<<g, 256, 0, s>>>(x, a, nx, pitch, n, partials);
    sum_partials_kernel<<<1, 32, 0, s>>>(partials, g, out);
    return cudaGetLastError();
}

}  // namespace spg
