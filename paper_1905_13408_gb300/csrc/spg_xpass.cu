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
// memory laid out row by row (Slots: padded per exchange, conflict-free), on
// which only the row's own threads synchronise. The untwisted rows pass
// through the same shared memory, where the kx-major writes (and reads) are
// gathered into runs of R consecutive rows.
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
    // a row's slots in shared memory: those of its transform's exchanges
    // (Slots) and n/2 + 1, rounded to 1 modulo 16, so that one column read
    // across 16 rows (the kx-major runs) falls on 16 different bank pairs
    static constexpr int LP = ((H >= 128 ? H + H / 8 : H) + 15) / 16 * 16 + 1;
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

// Slots of a row's positions z in the exchange after radix-8 stage s. A
// warp-wide access of 8-byte values is served per half-warp, so a pattern is
// conflict-free when the 16 threads of each half-warp reach 16 different
// bank pairs. Rows of 128 and more pad each exchange for its own pattern:
// after stage 0 (writes 8 t + q, reads t + i L/8) one slot per 16,
// z + z/16; after stage 1 (writes 64 (t/8) + t mod 8 + 8 q) 8 slots per 64,
// z + 8 (z/64); after stage 2 (writes and reads contiguous in t) none. Both
// the writes and the reads of every exchange are then conflict-free and
// reach their slots from one per-thread base at constant offsets
// (at(s, base + q Ns) - at(s, base) = at(s, q Ns), and at(s, t + i L/8) -
// at(s, t) = at(s, i L/8)). Rows of 64: bits 0-3 of z XORed with bits 3-6.
// Input rows of the forward row pass: a real volume y, or (y null) the
// extrapolated point y_k = x_k + beta_k d_k of an increment-storage solve,
// formed while the rows are read: x_k in xs[cur], d_k in ds[cur], with cur
// and beta_k = beta[kmom] read from the device state and descriptor when the
// launch runs.
struct RowSrc {
    const float *y;
    const float *xs[2], *ds[2];
    const DevState *st;
    const VolDesc *vols;
    const float *beta;
};

template <int L>
struct Slots {
    static constexpr bool PAD = L >= 128;
    static constexpr int SPAN = PAD ? L + L / 8 : L;  // slots a row takes
    __device__ static __forceinline__ int at(int s, int z)
    {
        if constexpr (!PAD) return z ^ ((z >> 3) & 15);
        return s == 0 ? z + (z >> 4) : (s == 1 ? z + 8 * (z >> 6) : z);
    }
};

// Barrier over the T threads of one row r (its exchanges touch only its own
// slots): the warp where rows fit in one, else a named barrier per row.
template <int T>
__device__ __forceinline__ void row_sync(int r)
{
    if constexpr (T <= 32)
        __syncwarp();
    else
        asm volatile("bar.sync %0, %1;" ::"r"(1 + r), "n"(T) : "memory");
}

// In-register Stockham transform of length L = 2^LOG2L (L >= 64) and sign S;
// row r's thread t holds positions t + i L/8 before and after. Only the row's
// threads synchronise (row_sync; rows of 64 threads take named barriers
// 1 .. 8): the caller orders the row's slots against other threads' use of
// them. The threads of
// a row are consecutive, so each stage reads its twiddles from a table laid
// out in thread order (stw, from xpass_twiddles): radix-8 stage s (span
// Ns = 8^s, s >= 1) at [q - 1][k], k = t mod Ns, holding w_L^(q k L/(8 Ns));
// a last radix-2 stage at [m][t] (w_L^j, j = t + m L/8); a last radix-4
// stage at [p - 1][j] (w_L^(p j)).
template <int LOG2L, int LP, int S>
__device__ __forceinline__ void row_fft(float2 (&v)[8], const float2 *stw, float2 *buf, int t, int r)
{
    constexpr int L = 1 << LOG2L, T = L / 8, NS8 = LOG2L / 3, REM = LOG2L % 3;
    static_assert(L >= 64, "at least two radix-8 stages");
    static_assert(LP >= Slots<L>::SPAN, "a row's stride holds its exchange slots");
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
            using Sl = Slots<L>;
            const int base = (t - k) * 8 + k;
            row_sync<T>(r);  // the row's previous exchange (or the caller's reads of the row) is done
            if constexpr (Sl::PAD) {
                float2 *w = row + Sl::at(s, base);
#pragma unroll
                for (int q = 0; q < 8; q++) w[Sl::at(s, q * Ns)] = v[q];
                row_sync<T>(r);
                const float2 *rd = row + Sl::at(s, t);
#pragma unroll
                for (int i = 0; i < 8; i++) v[i] = rd[Sl::at(s, i * T)];
            } else {
#pragma unroll
                for (int q = 0; q < 8; q++) row[Sl::at(s, base + q * Ns)] = v[q];
                row_sync<T>(r);
#pragma unroll
                for (int i = 0; i < 8; i++) v[i] = row[Sl::at(s, t + i * T)];
            }
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

// R rows y0 .. y0 + R - 1 of plane z: real-to-complex transform along x,
// written kx-major (runs of R consecutive rows). tws: the row pass's table in
// shared memory; buf: R LP slots.
// With EXT the rows are those of y = x + beta d, formed from Y (x) and D (d)
// by one fused multiply-add per value, as the fused step forms y.
template <int LOG2N, bool EXT>
__device__ __forceinline__ void r2c_rows(const float *__restrict__ Y, const float *__restrict__ D, float beta,
                                         int pitch, int ny, float2 *__restrict__ F, const float2 *tws, float2 *buf,
                                         int z, int y0)
{
    using P = Rows<LOG2N>;
    const int t = threadIdx.x % P::T, r = threadIdx.x / P::T, y = y0 + r;
    const bool in = y < ny;
    const long long ro = ((long long)z * ny + (in ? y : 0)) * pitch;
    const float2 *row = reinterpret_cast<const float2 *>(Y + ro);
    float2 v[8];
    if constexpr (EXT) {
        const float2 *drow = reinterpret_cast<const float2 *>(D + ro);
#pragma unroll
        for (int i = 0; i < 8; i++) {
            if (in) {
                const float2 xv = __ldg(row + t + i * P::T), dv = __ldg(drow + t + i * P::T);
                v[i] = make_float2(fmaf(beta, dv.x, xv.x), fmaf(beta, dv.y, xv.y));
            } else {
                v[i] = make_float2(0.f, 0.f);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < 8; i++) v[i] = in ? __ldg(row + t + i * P::T) : make_float2(0.f, 0.f);
    }
    row_fft<LOG2N - 1, P::LP, -1>(v, tws + P::N, buf, t, r);
    float2 *u = buf + r * P::LP;
    if constexpr (P::T <= 32) {
        // thread t untwists the pairs (k, n/2 - k), k = t + i T, i < 4: U[n/2 - k]
        // is slot 7 - i of thread T - t of the row (for thread 0 its own slot
        // 8 - i, and k = 0 gives X[0] and X[n/2]); thread 0 also takes
        // k = n/4, which pairs with itself
        const int lane = threadIdx.x & 31;
        const int partner = (lane & ~(P::T - 1)) | ((P::T - t) & (P::T - 1));
        row_sync<P::T>(r);  // the transform's last exchange is read
#pragma unroll
        for (int i = 0; i < 4; i++) {
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
                const float2 wo = cmul(tws[k], o);
                u[k] = cadd(e, wo);
                u[P::H - k] = conjf2(csub(e, wo));
            }
        }
        if (t == 0) {
            const float2 uk = v[4], um = conjf2(uk);
            const float2 e = scale2(cadd(uk, um), 0.5f);
            const float2 o = scale2(mul_mi(csub(uk, um)), 0.5f);
            u[P::H / 2] = cadd(e, cmul(tws[P::H / 2], o));
        }
    } else {
        row_sync<P::T>(r);  // the transform's last exchange is read
#pragma unroll
        for (int i = 0; i < 8; i++) u[t + i * P::T] = v[i];
        row_sync<P::T>(r);
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
    // kx-major: F[z][kx][y], runs of R consecutive rows; thread (rr, kx0)
    // takes kx = kx0 + j KS of row rr
    constexpr int KS = P::THREADS / P::R, NJ = (P::NXH + KS - 1) / KS;
    const int rr = threadIdx.x % P::R, kx0 = threadIdx.x / P::R;
    if (y0 + rr < ny) {
        float2 *const dst = F + ((long long)z * P::NXH + kx0) * ny + y0 + rr;
        const float2 *const src = buf + rr * P::LP + kx0;
#pragma unroll
        for (int j = 0; j < NJ; j++)
            if (kx0 + j * KS < P::NXH) dst[(long long)j * KS * ny] = src[j * KS];
    }
}

// R rows y0 .. y0 + R - 1 of plane z from the kx-major half spectrum:
// complex-to-real transform along x into Y (the gather streams through L2).
template <int LOG2N>
__device__ __forceinline__ void c2r_rows(const float2 *__restrict__ F, int ny, float *__restrict__ Y, int pitch,
                                         const float2 *tws, float2 *buf, int z, int y0)
{
    using P = Rows<LOG2N>;
    const float2 *const Fz = F + (long long)z * P::NXH * ny;
    // kx-major runs of R rows, thread (rr, kx0) taking kx = kx0 + j KS of row
    // rr; all of a thread's loads issued before its stores
    constexpr int KS = P::THREADS / P::R, NG = (P::NXH + KS - 1) / KS;
    {
        const int rr = threadIdx.x % P::R, kx0 = threadIdx.x / P::R;
        const bool in = y0 + rr < ny;
        const float2 *const src = Fz + (long long)kx0 * ny + y0 + rr;
        float2 g[NG];
#pragma unroll
        for (int j = 0; j < NG; j++)
            g[j] = (in && kx0 + j * KS < P::NXH) ? __ldcg(src + (long long)j * KS * ny) : make_float2(0.f, 0.f);
        float2 *const dst = buf + rr * P::LP + kx0;
#pragma unroll
        for (int j = 0; j < NG; j++)
            if (kx0 + j * KS < P::NXH) dst[j * KS] = g[j];
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

// Both row passes take the planes from the last to the first (CTAs start
// in about blockIdx order): their neighbours in an iteration walk the planes
// upwards (the fused step's z march; the library's batched transforms along
// y, line index z (nx/2+1) + kx), so the planes a pass reads first are the
// ones its producer wrote last, still in L2, and the planes it writes last
// are the ones its consumer reads first.
__device__ __forceinline__ int plane_descending() { return (int)(gridDim.y - 1 - blockIdx.y); }

template <int LOG2N, bool EXT>
__global__ void __launch_bounds__(Rows<LOG2N>::THREADS, 4)
    xpass_r2c_kernel(const RowSrc src, int pitch, int ny, float2 *__restrict__ F, const float2 *__restrict__ tw)
{
    using P = Rows<LOG2N>;
    extern __shared__ __align__(16) float2 xsm[];
    float2 *const buf = xsm;
    float2 *const tws = xsm + P::R * P::LP;
    for (int i = threadIdx.x; i < P::TW; i += P::THREADS) tws[i] = tw[i];
    const float *Y = src.y, *D = nullptr;
    float beta = 0.f;
    if constexpr (EXT) {
        // the solver's current pair and extrapolation weight, as the device
        // state holds them when this launch runs
        const int cur = src.st->cur;
        Y = cur == 0 ? src.xs[0] : src.xs[1];
        D = cur == 0 ? src.ds[0] : src.ds[1];
        beta = src.beta[src.vols[0].kmom];
    }
    __syncthreads();
    r2c_rows<LOG2N, EXT>(Y, D, beta, pitch, ny, F, tws, buf, plane_descending(), blockIdx.x * P::R);
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
    for (int i = threadIdx.x; i < P::TW; i += P::THREADS) tws[i] = tw[i];  // c2r_rows syncs before reading
    c2r_rows<LOG2N>(F, ny, Y, pitch, tws, buf, plane_descending(), blockIdx.x * P::R);
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
cudaError_t xpass(bool forward, const RowSrc &src, float *Yout, int pitch, int ny, int nz, const float2 *Fin,
                  float2 *Fout, const float2 *tw, cudaStream_t s)
{
    using P = Rows<LOG2N>;
    const dim3 grid((ny + P::R - 1) / P::R, nz);
    if constexpr (P::SMEM > 48 * 1024) {
        // above the default dynamic shared-memory limit: opt in once per device
        static bool opted[64] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!opted[dev]) {
            e = cudaFuncSetAttribute(xpass_r2c_kernel<LOG2N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)P::SMEM);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(xpass_r2c_kernel<LOG2N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)P::SMEM);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(xpass_c2r_kernel<LOG2N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)P::SMEM);
            if (e != cudaSuccess) return e;
            opted[dev] = true;
        }
    }
    if (forward && src.y)
        xpass_r2c_kernel<LOG2N, false><<<grid, P::THREADS, P::SMEM, s>>>(src, pitch, ny, Fout, tw);
    else if (forward)
        xpass_r2c_kernel<LOG2N, true><<<grid, P::THREADS, P::SMEM, s>>>(src, pitch, ny, Fout, tw);
    else
        xpass_c2r_kernel<LOG2N><<<grid, P::THREADS, P::SMEM, s>>>(Fin, ny, Yout, pitch, tw);
    return cudaGetLastError();
}

cudaError_t xpass_dispatch(int nx, bool forward, const RowSrc &src, float *Yout, int pitch, int ny, int nz,
                           const float2 *Fin, float2 *Fout, const float2 *tw, cudaStream_t s)
{
    switch (nx) {
    case 128: return xpass<7>(forward, src, Yout, pitch, ny, nz, Fin, Fout, tw, s);
    case 256: return xpass<8>(forward, src, Yout, pitch, ny, nz, Fin, Fout, tw, s);
    case 512: return xpass<9>(forward, src, Yout, pitch, ny, nz, Fin, Fout, tw, s);
    case 1024: return xpass<10>(forward, src, Yout, pitch, ny, nz, Fin, Fout, tw, s);
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

// Per-stage tables of a length-L row transform in the order row_fft reads
// them, each entry w_L^e evaluated directly in double precision.
void append_stage_tables(int L, std::vector<float2> *table)
{
    const double pi = 3.14159265358979323846;
    auto w = [&](long long e) {
        const double a = -2.0 * pi * (double)(e % L) / (double)L;
        return make_float2((float)std::cos(a), (float)std::sin(a));
    };
    int log2l = 0;
    while ((1 << log2l) < L) log2l++;
    const int ns8 = log2l / 3, rem = log2l % 3;
    for (int s = 1; s < ns8; s++) {
        const int Ns = 1 << (3 * s), step = L / (8 * Ns);
        for (int q = 1; q < 8; q++)
            for (int k = 0; k < Ns; k++) table->push_back(w((long long)q * k * step));
    }
    if (rem == 1)
        for (int j = 0; j < L / 2; j++) table->push_back(w(j));
    else if (rem == 2)
        for (int p = 1; p <= 3; p++)
            for (int j = 0; j < L / 4; j++) table->push_back(w((long long)p * j));
}

}  // namespace

bool xpass_supported(int nx, int nz) { return (nx == 128 || nx == 256 || nx == 512 || nx == 1024) && nz <= 65535; }

void xpass_twiddles(int nx, std::vector<float2> *table)
{
    // w_n^m for m < n (the untwist), then the row transform's stage tables
    // (length L = n/2)
    const double pi = 3.14159265358979323846;
    table->clear();
    for (int m = 0; m < nx; m++) {
        const double a = -2.0 * pi * (double)m / (double)nx;
        table->push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
    }
    append_stage_tables(nx / 2, table);
}

cudaError_t launch_xpass_r2c(int nx, const float *Y, int pitch, int ny, int nz, float2 *F, const float2 *tw,
                             cudaStream_t s)
{
    if (!Y) return cudaErrorInvalidValue;
    RowSrc src{};
    src.y = Y;
    return xpass_dispatch(nx, true, src, nullptr, pitch, ny, nz, nullptr, F, tw, s);
}

cudaError_t launch_xpass_r2c_extrap(int nx, const DevState *st, const VolDesc *vols, const float *beta,
                                    float *const *xbuf, int pitch, int ny, int nz, float2 *F, const float2 *tw,
                                    cudaStream_t s)
{
    RowSrc src{};
    src.xs[0] = xbuf[0];
    src.xs[1] = xbuf[1];
    src.ds[0] = xbuf[2];
    src.ds[1] = xbuf[3];
    src.st = st;
    src.vols = vols;
    src.beta = beta;
    if (!src.xs[0] || !src.xs[1] || !src.ds[0] || !src.ds[1] || !st || !vols || !beta) return cudaErrorInvalidValue;
    return xpass_dispatch(nx, true, src, nullptr, pitch, ny, nz, nullptr, F, tw, s);
}

cudaError_t launch_xpass_c2r(int nx, const float2 *F, int ny, int nz, float *Y, int pitch, const float2 *tw,
                             cudaStream_t s)
{
    return xpass_dispatch(nx, false, RowSrc{}, Y, pitch, ny, nz, F, nullptr, tw, s);
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
