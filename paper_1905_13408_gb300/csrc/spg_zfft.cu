// Transform along z of a half spectrum, and the Fourier-domain data term's
// spectrum pass fused between a forward and an inverse z transform (Sec. 2.5,
// Eq. 31), for power-of-two nz from 8 to 4096. The half spectrum
// [nz][ny][nx/2+1] is viewed as [nz][M] with M = ny (nx/2+1) columns, each a
// line along z; a CTA takes C consecutive columns (16 where 1024 threads
// allow it), so every z row of its tile is one contiguous run of C complex
// values in HBM.
//
// Each line goes through a Stockham auto-sort FFT (the formulation of
// Govindaraju et al., SC 2008): for a stage of radix R over sub-transforms of
// span Ns, butterfly j takes the R inputs j + r n/R, multiplies input r by
// w^(r k n/(Ns R)) (k = j mod Ns, w = e^(-2 pi i/n)), transforms them with an
// R-point DFT and writes output q to (j - k) R + k + q Ns; after the last
// stage the line is in natural order. Stages are radix 8 and one final radix
// 2 or 4. The twiddle table w^m (m < n) is computed on the host in double
// precision.
//
// Fused mode: F <- A_z^-1 ( (A_z F) N s - C ) per column, which together with
// the per-plane 2-D transforms on either side gives the residual spectrum of
// the data gradient without a separate pass over the spectrum.
#include <cmath>

#include "spg_internal.h"

namespace spg {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// a * (s i), s = +1 or -1
template <int S>
__device__ __forceinline__ float2 mul_si(float2 a)
{
    return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Twiddle w^m of the transform's sign (S = -1 forward, +1 inverse).
template <int S>
__device__ __forceinline__ float2 twiddle(const float2 *T, int m)
{
    const float2 t = T[m];
    return S < 0 ? t : make_float2(t.x, -t.y);
}

// 4-point DFT of sign S in place.
template <int S>
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3)
{
    const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_si<S>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// 8-point DFT of sign S in place: two 4-point DFTs of the even and odd
// inputs, combined with the eighth roots of unity.
template <int S>
__device__ __forceinline__ void dft8(float2 *v)
{
    float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<S>(e0, e1, e2, e3);
    dft4<S>(o0, o1, o2, o3);
    const float h = 0.70710678118654752f;
    const float2 w1 = make_float2(h, S * h), w3 = make_float2(-h, S * h);
    o1 = cmul(o1, w1);
    o2 = mul_si<S>(o2);
    o3 = cmul(o3, w3);
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

// Power-of-two lengths 8 .. 4096: a register-resident form of the same
// Stockham transform. Thread t of a column holds the 8 values at positions
// t + i N/8 (slot i) before and after every stage: a radix-8 stage is one
// butterfly per thread on exactly those inputs, its outputs go through a
// shared-memory exchange back to that arrangement, and the last stage (radix
// 8 with span N/8, or a radix-2/4 stage with span N/R, whose butterflies
// j' = t + m N/8 also read and write slots only) needs no exchange. The
// forward transform therefore ends where the inverse one starts, and the
// fused mode scales in registers. Columns sit in shared memory as
// [z + z/8][C] (one padding row per 8), which keeps every exchange free of
// bank conflicts.
template <int LOG2N>
struct Pow2 {
    static constexpr int N = 1 << LOG2N, T = N / 8, NS8 = LOG2N / 3, REM = LOG2N % 3;
    // 16 columns (128 contiguous bytes per z row) where 1024 threads allow it:
    // narrower runs of a row leave HBM bandwidth unused on this strided pass
    static constexpr int C = (8192 >> LOG2N) < 1 ? 1 : ((8192 >> LOG2N) > 16 ? 16 : (8192 >> LOG2N));
    static constexpr int THREADS = C * T;
    static constexpr int BUF = C * (N + N / 8);  // float2 per exchange buffer
    static constexpr size_t SMEM = (size_t)(N + 2 * BUF) * sizeof(float2);
};

__device__ __forceinline__ int padded(int z) { return z + (z >> 3); }

template <int LOG2N, int S>
__device__ __forceinline__ void transform8(float2 (&v)[8], const float2 *tws, float2 *bufs, int t, int c,
                                           int &parity)
{
    using P = Pow2<LOG2N>;
#pragma unroll
    for (int s = 0; s < P::NS8; s++) {
        const int Ns = 1 << (3 * s);
        const int k = t & (Ns - 1);
        const int step = P::N / (8 * Ns);
        if (s > 0) {
#pragma unroll
            for (int r = 1; r < 8; r++) v[r] = cmul(v[r], twiddle<S>(tws, r * k * step));
        }
        dft8<S>(v);
        if (s < P::NS8 - 1 || P::REM != 0) {
            float2 *b = bufs + (parity ? P::BUF : 0);
            parity ^= 1;
            const int base = (t - k) * 8 + k;
#pragma unroll
            for (int q = 0; q < 8; q++) b[padded(base + q * Ns) * P::C + c] = v[q];
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 8; i++) v[i] = b[padded(t + i * P::T) * P::C + c];
        }
    }
    if (P::REM == 1) {  // radix 2, span N/2: butterfly t + m N/8 on slots m, m + 4
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const float2 a = v[m], b = cmul(v[m + 4], twiddle<S>(tws, t + m * P::T));
            v[m] = cadd(a, b);
            v[m + 4] = csub(a, b);
        }
    } else if (P::REM == 2) {  // radix 4, span N/4: butterfly t + m N/8 on slots m, m + 2, m + 4, m + 6
#pragma unroll
        for (int m = 0; m < 2; m++) {
            const int jp = t + m * P::T;
            float2 a0 = v[m], a1 = cmul(v[m + 2], twiddle<S>(tws, jp));
            float2 a2 = cmul(v[m + 4], twiddle<S>(tws, 2 * jp)), a3 = cmul(v[m + 6], twiddle<S>(tws, 3 * jp));
            dft4<S>(a0, a1, a2, a3);
            v[m] = a0;
            v[m + 2] = a1;
            v[m + 4] = a2;
            v[m + 6] = a3;
        }
    }
}

template <int LOG2N, bool FUSED>
__global__ void __launch_bounds__(Pow2<LOG2N>::THREADS, 1) zfft_pow2_kernel(float2 *F, const float *Nw, const float2 *Cd,
                                                                          float scale, long long M, const float2 *tw)
{
    using P = Pow2<LOG2N>;
    extern __shared__ float2 zsm[];
    float2 *tws = zsm, *bufs = zsm + P::N;
    const int c = threadIdx.x % P::C, t = threadIdx.x / P::C;
    const long long col = (long long)blockIdx.x * P::C + c;
    const bool valid = col < M;
    for (int i = threadIdx.x; i < P::N; i += P::THREADS) tws[i] = tw[i];
    float2 v[8];
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = valid ? F[(long long)(t + i * P::T) * M + col] : make_float2(0.f, 0.f);
    __syncthreads();
    int parity = 0;
    transform8<LOG2N, -1>(v, tws, bufs, t, c, parity);
    if (FUSED) {
        if (valid) {
#pragma unroll
            for (int i = 0; i < 8; i++) {
                const long long g = (long long)(t + i * P::T) * M + col;
                const float m = Nw[g] * scale;
                const float2 cd = Cd[g];
                v[i] = make_float2(fmaf(v[i].x, m, -cd.x), fmaf(v[i].y, m, -cd.y));
            }
        }
        transform8<LOG2N, 1>(v, tws, bufs, t, c, parity);
    }
    if (valid) {
#pragma unroll
        for (int i = 0; i < 8; i++) F[(long long)(t + i * P::T) * M + col] = v[i];
    }
}

template <int LOG2N, bool FUSED>
cudaError_t launch_pow2(float2 *F, const float *Nw, const float2 *Cd, float scale, const ZPlan &p, const float2 *tw,
                        cudaStream_t s)
{
    using P = Pow2<LOG2N>;
    const long long grid = (p.M + P::C - 1) / P::C;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
    zfft_pow2_kernel<LOG2N, FUSED><<<(unsigned)grid, P::THREADS, P::SMEM, s>>>(F, Nw, Cd, scale, p.M, tw);
    return cudaGetLastError();
}

template <bool FUSED>
cudaError_t launch_pow2_any(float2 *F, const float *Nw, const float2 *Cd, float scale, const ZPlan &p,
                            const float2 *tw, cudaStream_t s)
{
    switch (p.log2n) {
    case 3: return launch_pow2<3, FUSED>(F, Nw, Cd, scale, p, tw, s);
    case 4: return launch_pow2<4, FUSED>(F, Nw, Cd, scale, p, tw, s);
    case 5: return launch_pow2<5, FUSED>(F, Nw, Cd, scale, p, tw, s);
    case 6: return launch_pow2<6, FUSED>(F, Nw, Cd, scale, p, tw, s);
    case 7: return launch_pow2<7, FUSED>(F, Nw, Cd, scale, p, tw, s);
    case 8: return launch_pow2<8, FUSED>(F, Nw, Cd, scale, p, tw, s);
    case 9: return launch_pow2<9, FUSED>(F, Nw, Cd, scale, p, tw, s);
    case 10: return launch_pow2<10, FUSED>(F, Nw, Cd, scale, p, tw, s);
    case 11: return launch_pow2<11, FUSED>(F, Nw, Cd, scale, p, tw, s);
    case 12: return launch_pow2<12, FUSED>(F, Nw, Cd, scale, p, tw, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int LOG2N>
cudaError_t set_pow2_limits()
{
    using P = Pow2<LOG2N>;
    cudaError_t e = cudaFuncSetAttribute((const void *)zfft_pow2_kernel<LOG2N, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute((const void *)zfft_pow2_kernel<LOG2N, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P::SMEM);
    return e;
}

template <bool FUSED>
cudaError_t launch_any(float2 *F, const float *N, const float2 *Cd, float scale, const ZPlan &p, const float2 *tw,
                       cudaStream_t s)
{
    return launch_pow2_any<FUSED>(F, N, Cd, scale, p, tw, s);
}

// The opt-in shared-memory limit of every instance, set when a plan is made
// (before any launch, so never inside a graph capture).
cudaError_t set_smem_limits()
{
    const cudaError_t es[] = {set_pow2_limits<3>(), set_pow2_limits<4>(),  set_pow2_limits<5>(),
                              set_pow2_limits<6>(), set_pow2_limits<7>(),  set_pow2_limits<8>(),
                              set_pow2_limits<9>(), set_pow2_limits<10>(), set_pow2_limits<11>(),
                              set_pow2_limits<12>()};
    for (cudaError_t e : es)
        if (e != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace

bool zfft_plan(int nz, long long M, ZPlan *p, std::vector<float2> *table)
{
    if (nz < 8 || nz > kZMaxN || (nz & (nz - 1)) != 0 || M < 1) return false;
    static const cudaError_t limits = set_smem_limits();
    if (limits != cudaSuccess) return false;
    ZPlan q{};
    q.n = nz;
    q.M = M;
    while ((1 << q.log2n) < nz) q.log2n++;
    table->resize(nz);
    const double pi = 3.14159265358979323846;
    for (int j = 0; j < nz; j++) {
        const double a = -2.0 * pi * (double)j / (double)nz;
        (*table)[j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    *p = q;
    return true;
}

cudaError_t launch_zfft(float2 *F, const ZPlan &p, const float2 *tw, cudaStream_t s)
{
    return launch_any<false>(F, nullptr, nullptr, 0.f, p, tw, s);
}

cudaError_t launch_zfft_residual(float2 *F, const float *N, const float2 *Cd, float scale, const ZPlan &p,
                                 const float2 *tw, cudaStream_t s)
{
    return launch_any<true>(F, N, Cd, scale, p, tw, s);
}

}  // namespace spg
