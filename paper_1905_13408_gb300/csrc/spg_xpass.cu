// Row pass of the Fourier-domain data term (Sec. 2.5, Eq. 31) for
// power-of-two nx = 128 .. 1024: the real-to-complex transform along x of
// every row of y_k, written with kx as the slow in-plane index, and the
// complex-to-real transform back. The spectrum between the two is held as
// [nz][nx/2+1][ny] (kx-major), so the transform along y is a batch of
// contiguous lines, the library's fastest case, and the pass along z treats
// the nx/2+1 by ny positions of a plane as it treats any other order (its N
// and C are held in the same order). Unnormalised transforms, as those of
// the library.
//
// A real row x[0..n) is read as the complex sequence u[m] = x[2m] + i x[2m+1]
// of length n/2 and transformed (U); the half spectrum X[0..n/2] follows from
//   E = (U[k] + conj U[n/2-k]) / 2,  O = -i (U[k] - conj U[n/2-k]) / 2,
//   X[k] = E + w^k O,  X[n/2-k] = conj(E - w^k O),  w = e^(-2 pi i / n),
//   X[0] = Re U[0] + Im U[0],  X[n/2] = Re U[0] - Im U[0].
// Back, from a row's half spectrum G[0..n/2], of which only the real parts of
// G[0] and G[n/2] count (they are real for the spectrum of a real row),
//   Z[k] = (G[k] + conj G[n/2-k]) + i (G[k] - conj G[n/2-k]) conj(w^k),
// whose inverse transform z gives x[2m] = Re z[m], x[2m+1] = Im z[m].
//
// A CTA takes R consecutive rows of one plane; each row's length-n/2
// transform is the register-resident Stockham form of spg_zfft.cu (n/16
// threads per row, each holding 8 values), with exchanges through shared
// memory laid out row by row, which keeps a warp (the threads of one row)
// free of bank conflicts. The untwisted rows pass through the same shared
// memory, where the kx-major writes (and reads) are gathered into runs of R
// consecutive rows.
#include <cmath>
#include <vector>

#include "spg_fft.cuh"
#include "spg_internal.h"

namespace spg {
namespace {

using namespace fft;

template <int LOG2N>
struct Rows {
    static constexpr int N = 1 << LOG2N, H = N / 2, NXH = H + 1;
    static constexpr int T = H / 8;             // threads per row transform
    static constexpr int THREADS = 512;
    static constexpr int R = THREADS / T;       // rows per CTA
    // a row's slots in shared memory: n/2 + 1 (the exchanges of the row
    // transform are swizzled in place, see swz), which is 1 modulo 16, so that
    // one column read across 16 rows (the kx-major runs) falls on 16
    // different bank pairs
    static constexpr int LP = H + 1;
    static constexpr int L = H;                 // length of a row transform
    // per-stage twiddle tables of the row transform (see stage_table_size)
    static constexpr int NS8 = (LOG2N - 1) / 3, REM = (LOG2N - 1) % 3;
    static constexpr int STAGES = 7 * ((NS8 >= 2 ? 8 : 0) + (NS8 >= 3 ? 64 : 0));
    static constexpr int LAST = REM == 1 ? L / 2 : (REM == 2 ? 3 * (L / 4) : 0);
    static constexpr int TW = N + STAGES + LAST;  // w_n^m (m < n), then the stage tables
    static constexpr size_t SMEM = (size_t)(R * LP + TW) * sizeof(float2);  // rows + twiddles
    static_assert(LOG2N >= 7 && LOG2N <= 10, "rows of 128 .. 1024");
    static_assert(LP >= NXH, "a row's slots hold its half spectrum");
};

// Slot of position z of a row during the transform's exchanges: bits 0-3 of z
// XORed with bits 3-6 (a bijection within each aligned run of 128, so the row
// needs no padding). The writes of a stage (8 consecutive positions of a
// thread, Ns apart) and the reads (t + i L/8, consecutive over t) then each
// take the minimum of two wavefronts per warp for L = 128 .. 512.
__device__ __forceinline__ int swz(int z) { return z ^ ((z >> 3) & 15); }

// In-register Stockham transform of length L = 2^LOG2L (L >= 64) and sign S;
// row r's thread t holds positions t + i L/8 before and after. The threads of
// a row are consecutive, so each stage reads its twiddles from a table laid
// out in thread order (stw, from xpass_twiddles): radix-8 stage s (span
// Ns = 8^s, s >= 1) at [q - 1][k], k = t mod Ns, holding w_L^(q k L/(8 Ns));
// a last radix-2 stage at [m][t] (w_L^j, j = t + m L/8); a last radix-4
// stage at [p - 1][j] (w_L^(p j)). Every thread of the block takes part.
template <int LOG2L, int LP, int S>
__device__ __forceinline__ void row_fft(float2 (&v)[8], const float2 *stw, float2 *buf, int t, int r)
{
    constexpr int L = 1 << LOG2L, T = L / 8, NS8 = LOG2L / 3, REM = LOG2L % 3;
    static_assert(L >= 64, "at least two radix-8 stages");
    float2 *row = buf + r * LP;
    int off = 0;
#pragma unroll
    for (int s = 0; s < NS8; s++) {
        const int Ns = 1 << (3 * s);
        const int k = t & (Ns - 1);
        if (s > 0) {
#pragma unroll
            for (int q = 1; q < 8; q++) v[q] = cmul(v[q], twiddle<S>(stw, off + (q - 1) * Ns + k));
            off += 7 * Ns;
        }
        dft8<S>(v);
        if (s < NS8 - 1 || REM != 0) {
            const int base = (t - k) * 8 + k;
            __syncthreads();  // the previous exchange's (or the caller's) reads are done
#pragma unroll
            for (int q = 0; q < 8; q++) row[swz(base + q * Ns)] = v[q];
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 8; i++) v[i] = row[swz(t + i * T)];
        }
    }
    if (REM == 1) {  // radix 2, span L/2: butterfly t + m L/8 on slots m, m + 4
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const float2 a = v[m], b = cmul(v[m + 4], twiddle<S>(stw, off + m * T + t));
            v[m] = cadd(a, b);
            v[m + 4] = csub(a, b);
        }
    } else if (REM == 2) {  // radix 4, span L/4: butterfly t + m L/8 on slots m, m + 2, m + 4, m + 6
#pragma unroll
        for (int m = 0; m < 2; m++) {
            const int jp = t + m * T;
            float2 a0 = v[m], a1 = cmul(v[m + 2], twiddle<S>(stw, off + jp));
            float2 a2 = cmul(v[m + 4], twiddle<S>(stw, off + L / 4 + jp));
            float2 a3 = cmul(v[m + 6], twiddle<S>(stw, off + L / 2 + jp));
            dft4<S>(a0, a1, a2, a3);
            v[m] = a0;
            v[m + 2] = a1;
            v[m + 4] = a2;
            v[m + 6] = a3;
        }
    }
}

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 scale2(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }  // -i a

template <int LOG2N>
__global__ void __launch_bounds__(Rows<LOG2N>::THREADS, 4)
    xpass_r2c_kernel(const float *__restrict__ Y, int pitch, int ny, float2 *__restrict__ F,
                     const float2 *__restrict__ tw)
{
    using P = Rows<LOG2N>;
    extern __shared__ __align__(16) float2 xsm[];
    float2 *const buf = xsm;
    float2 *const tws = xsm + P::R * P::LP;
    for (int i = threadIdx.x; i < P::TW; i += P::THREADS) tws[i] = tw[i];
    __syncthreads();
    const int z = blockIdx.y, y0 = blockIdx.x * P::R;
    const int t = threadIdx.x % P::T, r = threadIdx.x / P::T, y = y0 + r;
    const bool in = y < ny;
    const float2 *row = reinterpret_cast<const float2 *>(Y + ((long long)z * ny + (in ? y : 0)) * pitch);
    float2 v[8];
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = in ? __ldg(row + t + i * P::T) : make_float2(0.f, 0.f);
    row_fft<LOG2N - 1, P::LP, -1>(v, tws + P::N, buf, t, r);
    float2 *u = buf + r * P::LP;
    if constexpr (P::T <= 32) {
        // U[n/2 - k] of k = t + i T is held by thread T - t of the row at slot
        // 7 - i (thread 0: its own slot 8 - i), within the row's lanes
        const int lane = threadIdx.x & 31;
        const int partner = (lane & ~(P::T - 1)) | ((P::T - t) & (P::T - 1));
        __syncthreads();  // the transform's last exchange is read
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const float2 got = make_float2(__shfl_sync(0xffffffffu, v[7 - i].x, partner),
                                           __shfl_sync(0xffffffffu, v[7 - i].y, partner));
            const float2 uk = v[i];
            const int k = t + i * P::T;
            if (k == 0) {
                u[0] = make_float2(uk.x + uk.y, 0.f);
                u[P::H] = make_float2(uk.x - uk.y, 0.f);
            } else {
                const float2 um = conjf2(t == 0 ? v[(8 - i) & 7] : got);
                const float2 e = scale2(cadd(uk, um), 0.5f);
                const float2 o = scale2(mul_mi(csub(uk, um)), 0.5f);
                u[k] = cadd(e, cmul(tws[k], o));
            }
        }
    } else {
        __syncthreads();  // the transform's last exchange is read
#pragma unroll
        for (int i = 0; i < 8; i++) u[t + i * P::T] = v[i];
        __syncthreads();
        for (int k = t; k <= P::H / 2; k += P::T) {
            const float2 uk = u[k];
            if (k == 0) {
                u[0] = make_float2(uk.x + uk.y, 0.f);
                u[P::H] = make_float2(uk.x - uk.y, 0.f);
            } else {
                const float2 um = conjf2(u[P::H - k]);
                const float2 e = scale2(cadd(uk, um), 0.5f);
                const float2 o = scale2(mul_mi(csub(uk, um)), 0.5f);
                const float2 wo = cmul(tws[k], o);
                u[k] = cadd(e, wo);
                if (k != P::H - k) u[P::H - k] = conjf2(csub(e, wo));
            }
        }
    }
    __syncthreads();
    // kx-major: F[z][kx][y], runs of R consecutive rows
    float2 *const Fz = F + (long long)z * P::NXH * ny;
    for (int idx = threadIdx.x; idx < P::R * P::NXH; idx += P::THREADS) {
        const int rr = idx % P::R, kx = idx / P::R, yy = y0 + rr;
        if (yy < ny) Fz[(long long)kx * ny + yy] = buf[rr * P::LP + kx];
    }
}

template <int LOG2N>
__global__ void __launch_bounds__(Rows<LOG2N>::THREADS, 4)
    xpass_c2r_kernel(const float2 *__restrict__ F, int ny, float *__restrict__ Y, int pitch,
                     const float2 *__restrict__ tw)
{
    using P = Rows<LOG2N>;
    extern __shared__ __align__(16) float2 xsm[];
    float2 *const buf = xsm;
    float2 *const tws = xsm + P::R * P::LP;
    for (int i = threadIdx.x; i < P::TW; i += P::THREADS) tws[i] = tw[i];
    const int z = blockIdx.y, y0 = blockIdx.x * P::R;
    const float2 *const Fz = F + (long long)z * P::NXH * ny;
    // kx-major runs of R rows; all of a thread's loads issued before its stores
    constexpr int NG = (P::R * P::NXH + P::THREADS - 1) / P::THREADS;
    float2 g[NG];
#pragma unroll
    for (int j = 0; j < NG; j++) {
        const int idx = threadIdx.x + j * P::THREADS;
        const int rr = idx % P::R, kx = idx / P::R, yy = y0 + rr;
        g[j] = (idx < P::R * P::NXH && yy < ny) ? Fz[(long long)kx * ny + yy] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < NG; j++) {
        const int idx = threadIdx.x + j * P::THREADS;
        if (idx < P::R * P::NXH) buf[(idx % P::R) * P::LP + idx / P::R] = g[j];
    }
    __syncthreads();
    const int t = threadIdx.x % P::T, r = threadIdx.x / P::T, y = y0 + r;
    const float2 *u = buf + r * P::LP;
    float2 v[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int k = t + i * P::T;  // 0 .. n/2 - 1
        const float2 gk = k == 0 ? make_float2(u[0].x, 0.f) : u[k];
        const float2 gm = k == 0 ? make_float2(u[P::H].x, 0.f) : u[P::H - k];
        const float2 gmc = conjf2(gm);
        const float2 e = cadd(gk, gmc);
        const float2 o = cmul(csub(gk, gmc), conjf2(tws[k]));
        v[i] = make_float2(e.x - o.y, e.y + o.x);  // e + i o
    }
    row_fft<LOG2N - 1, P::LP, 1>(v, tws + P::N, buf, t, r);  // its first barrier follows every read of the rows
    if (y < ny) {
        float2 *row = reinterpret_cast<float2 *>(Y + ((long long)z * ny + y) * pitch);
#pragma unroll
        for (int i = 0; i < 8; i++) row[t + i * P::T] = v[i];
    }
}

// out[z][c][r] = in[z][r][c] for planes of rows x cols elements.
template <class T>
__global__ void plane_transpose_kernel(const T *__restrict__ in, T *__restrict__ out, int rows, int cols)
{
    __shared__ T tile[32][33];
    const long long plane = (long long)rows * cols;
    const T *src = in + blockIdx.z * plane;
    T *dst = out + blockIdx.z * plane;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = r0 + j, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[j][threadIdx.x] = src[(long long)r * cols + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int c = c0 + j, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[(long long)c * rows + r] = tile[threadIdx.x][j];
    }
}

template <int LOG2N>
cudaError_t xpass(bool forward, const float *Yin, float *Yout, int pitch, int ny, int nz, const float2 *Fin,
                  float2 *Fout, const float2 *tw, cudaStream_t s)
{
    using P = Rows<LOG2N>;
    const dim3 grid((ny + P::R - 1) / P::R, nz);
    if (forward)
        xpass_r2c_kernel<LOG2N><<<grid, P::THREADS, P::SMEM, s>>>(Yin, pitch, ny, Fout, tw);
    else
        xpass_c2r_kernel<LOG2N><<<grid, P::THREADS, P::SMEM, s>>>(Fin, ny, Yout, pitch, tw);
    return cudaGetLastError();
}

cudaError_t xpass_dispatch(int nx, bool forward, const float *Yin, float *Yout, int pitch, int ny, int nz,
                           const float2 *Fin, float2 *Fout, const float2 *tw, cudaStream_t s)
{
    switch (nx) {
    case 128: return xpass<7>(forward, Yin, Yout, pitch, ny, nz, Fin, Fout, tw, s);
    case 256: return xpass<8>(forward, Yin, Yout, pitch, ny, nz, Fin, Fout, tw, s);
    case 512: return xpass<9>(forward, Yin, Yout, pitch, ny, nz, Fin, Fout, tw, s);
    case 1024: return xpass<10>(forward, Yin, Yout, pitch, ny, nz, Fin, Fout, tw, s);
    default: return cudaErrorInvalidValue;
    }
}

template <class T>
cudaError_t transpose_planes(const T *in, T *out, int rows, int cols, int nz, cudaStream_t s)
{
    if (nz > 65535) return cudaErrorInvalidValue;
    const dim3 grid((cols + 31) / 32, (rows + 31) / 32, nz), block(32, 8);
    plane_transpose_kernel<T><<<grid, block, 0, s>>>(in, out, rows, cols);
    return cudaGetLastError();
}

}  // namespace

bool xpass_supported(int nx, int nz) { return (nx == 128 || nx == 256 || nx == 512 || nx == 1024) && nz <= 65535; }

void xpass_twiddles(int nx, std::vector<float2> *table)
{
    // w_n^m for m < n (the untwist), then the row transform's stage tables
    // (length L = n/2) in the order row_fft reads them, each entry w_L^e
    // evaluated directly in double precision
    const double pi = 3.14159265358979323846;
    auto w = [&](long long e, long long len) {
        const double a = -2.0 * pi * (double)(e % len) / (double)len;
        return make_float2((float)std::cos(a), (float)std::sin(a));
    };
    table->clear();
    for (int m = 0; m < nx; m++) table->push_back(w(m, nx));
    const int L = nx / 2;
    int log2l = 0;
    while ((1 << log2l) < L) log2l++;
    const int ns8 = log2l / 3, rem = log2l % 3;
    for (int s = 1; s < ns8; s++) {
        const int Ns = 1 << (3 * s), step = L / (8 * Ns);
        for (int q = 1; q < 8; q++)
            for (int k = 0; k < Ns; k++) table->push_back(w((long long)q * k * step, L));
    }
    if (rem == 1)
        for (int j = 0; j < L / 2; j++) table->push_back(w(j, L));
    else if (rem == 2)
        for (int p = 1; p <= 3; p++)
            for (int j = 0; j < L / 4; j++) table->push_back(w((long long)p * j, L));
}

cudaError_t launch_xpass_r2c(int nx, const float *Y, int pitch, int ny, int nz, float2 *F, const float2 *tw,
                             cudaStream_t s)
{
    return xpass_dispatch(nx, true, Y, nullptr, pitch, ny, nz, nullptr, F, tw, s);
}

cudaError_t launch_xpass_c2r(int nx, const float2 *F, int ny, int nz, float *Y, int pitch, const float2 *tw,
                             cudaStream_t s)
{
    return xpass_dispatch(nx, false, nullptr, Y, pitch, ny, nz, F, nullptr, tw, s);
}

cudaError_t launch_kx_major(const float *in, float *out, int ny, int nxh, int nz, cudaStream_t s)
{
    return transpose_planes<float>(in, out, ny, nxh, nz, s);
}

cudaError_t launch_kx_major(const float2 *in, float2 *out, int ny, int nxh, int nz, cudaStream_t s)
{
    return transpose_planes<float2>(in, out, ny, nxh, nz, s);
}

}  // namespace spg
