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

#include "spg_fft.cuh"
#include "spg_internal.h"

namespace spg {
namespace {

using namespace fft;

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

// Fused mode for lengths 128 .. 512 as a persistent pipeline fed by TMA: a
// CTA walks its tiles (16 columns each); while it transforms one tile in
// registers, with that tile's shared-memory buffer as the exchange buffer
// (unpadded: with 16 columns a half-warp covers one row, free of bank
// conflicts), the next tile's spectrum arrives by 2-D tensor copies into the
// other buffer, and the next tile's N and C into their buffer once the
// current tile has been scaled; each is waited for only where it is needed
// (an mbarrier per buffer, bounded waits). The one CTA that fits on an SM
// thus overlaps its copies with its arithmetic.
__device__ __forceinline__ uint32_t zs_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void zbar_init(uint64_t *b)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(zs_u32(b)) : "memory");
}

__device__ __forceinline__ void zbar_expect(uint64_t *b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(zs_u32(b)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool zbar_try(uint64_t *b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(zs_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait (2 s of %globaltimer): false on expiry.
__device__ __forceinline__ bool zbar_wait(uint64_t *b, uint32_t parity)
{
    if (zbar_try(b, parity)) return true;
    long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        for (int i = 0; i < 32; i++)
            if (zbar_try(b, parity)) return true;
        long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 2000000000LL) return false;
    }
}

__device__ __forceinline__ void ztma_2d(void *dst, const CUtensorMap *m, int x, int y, uint64_t *b)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(zs_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(zs_u32(b))
        : "memory");
}

// transform8 with one unpadded 16-column exchange buffer (a second barrier
// after each exchange's reads, since the same buffer serves every exchange)
template <int LOG2N, int S>
__device__ __forceinline__ void transform16(float2 (&v)[8], const float2 *__restrict__ tw, float2 *buf, int t,
                                            int c)
{
    using P = Pow2<LOG2N>;
    static_assert(P::C == 16, "16-column tiles");
#pragma unroll
    for (int s = 0; s < P::NS8; s++) {
        const int Ns = 1 << (3 * s);
        const int k = t & (Ns - 1);
        const int step = P::N / (8 * Ns);
        if (s > 0) {
#pragma unroll
            for (int r = 1; r < 8; r++) v[r] = cmul(v[r], twiddle<S>(tw, r * k * step));
        }
        dft8<S>(v);
        if (s < P::NS8 - 1 || P::REM != 0) {
            const int base = (t - k) * 8 + k;
#pragma unroll
            for (int q = 0; q < 8; q++) buf[(base + q * Ns) * 16 + c] = v[q];
            __syncthreads();
#pragma unroll
            for (int i = 0; i < 8; i++) v[i] = buf[(t + i * P::T) * 16 + c];
            __syncthreads();
        }
    }
    if (P::REM == 1) {
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const float2 a = v[m], b = cmul(v[m + 4], twiddle<S>(tw, t + m * P::T));
            v[m] = cadd(a, b);
            v[m + 4] = csub(a, b);
        }
    } else if (P::REM == 2) {
#pragma unroll
        for (int m = 0; m < 2; m++) {
            const int jp = t + m * P::T;
            float2 a0 = v[m], a1 = cmul(v[m + 2], twiddle<S>(tw, jp));
            float2 a2 = cmul(v[m + 4], twiddle<S>(tw, 2 * jp)), a3 = cmul(v[m + 6], twiddle<S>(tw, 3 * jp));
            dft4<S>(a0, a1, a2, a3);
            v[m] = a0;
            v[m + 2] = a1;
            v[m + 4] = a2;
            v[m + 6] = a3;
        }
    }
}

template <int LOG2N>
struct Tma {
    using P = Pow2<LOG2N>;
    static constexpr int ROWS = P::N < 256 ? P::N : 256;  // rows per tensor box
    static constexpr int BOXES = P::N / ROWS;
    static constexpr int TILE = P::N * 16;                 // complex values per tile
    static constexpr size_t SMEM = (size_t)TILE * (2 * sizeof(float2) + sizeof(float) + sizeof(float2)) + 4 * 8;
};

template <int LOG2N>
__global__ void __launch_bounds__(Pow2<LOG2N>::THREADS, 1)
    zfft_tma_kernel(float2 *F, float scale, long long M, const float2 *__restrict__ tw,
                    const __grid_constant__ ZMaps maps, int *err)
{
    using P = Pow2<LOG2N>;
    using Q = Tma<LOG2N>;
    extern __shared__ __align__(128) unsigned char zsm_tma[];
    float2 *buf0 = reinterpret_cast<float2 *>(zsm_tma);
    float2 *buf1 = buf0 + Q::TILE;
    float *ns = reinterpret_cast<float *>(buf1 + Q::TILE);
    float2 *cs = reinterpret_cast<float2 *>(ns + Q::TILE);
    uint64_t *bars = reinterpret_cast<uint64_t *>(cs + Q::TILE);  // spectrum of buffer 0, of buffer 1, N and C
    const int c = threadIdx.x % 16, t = threadIdx.x / 16;
    const long long ntiles = (M + 15) / 16;
    if (threadIdx.x == 0) {
        zbar_init(&bars[0]);
        zbar_init(&bars[1]);
        zbar_init(&bars[2]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto fetch_f = [&](long long tile, float2 *dst, uint64_t *b) {
        zbar_expect(b, Q::TILE * 8);
#pragma unroll
        for (int r = 0; r < Q::BOXES; r++) ztma_2d(dst + r * Q::ROWS * 16, &maps.f, (int)(tile * 32), r * Q::ROWS, b);
    };
    auto fetch_nc = [&](long long tile) {
        zbar_expect(&bars[2], Q::TILE * 12);
#pragma unroll
        for (int r = 0; r < Q::BOXES; r++) {
            ztma_2d(ns + r * Q::ROWS * 16, &maps.n, (int)(tile * 16), r * Q::ROWS, &bars[2]);
            ztma_2d(cs + r * Q::ROWS * 16, &maps.c, (int)(tile * 32), r * Q::ROWS, &bars[2]);
        }
    };
    long long tile = blockIdx.x;
    unsigned armed = 0;  // bit j: a phase of barrier j is armed and not yet waited for
    if (tile < ntiles) {
        if (threadIdx.x == 0) {
            fetch_f(tile, buf0, &bars[0]);
            fetch_nc(tile);
        }
        armed = 5u;
    }
    uint32_t ph0 = 0, ph1 = 0, phnc = 0;
    // on a timeout every thread leaves together, after thread 0 has waited
    // (again bounded) for the copies still in flight
    auto bail = [&]() {
        if (threadIdx.x == 0) {
            atomicCAS(err, 0, (int)SPG_ETIMEOUT);
            if (armed & 1u) zbar_wait(&bars[0], ph0);
            if (armed & 2u) zbar_wait(&bars[1], ph1);
            if (armed & 4u) zbar_wait(&bars[2], phnc);
        }
    };
    for (int b = 0; tile < ntiles; tile += gridDim.x, b ^= 1) {
        float2 *buf = b ? buf1 : buf0;
        const bool ok = zbar_wait(&bars[b], b ? ph1 : ph0);
        if (__syncthreads_or(!ok)) {
            bail();
            return;
        }
        if (b) ph1 ^= 1u; else ph0 ^= 1u;
        armed &= ~(1u << b);
        float2 v[8];
#pragma unroll
        for (int i = 0; i < 8; i++) v[i] = buf[(t + i * P::T) * 16 + c];
        __syncthreads();  // the tile's buffer now serves the exchanges
        const long long next = tile + gridDim.x;
        if (next < ntiles) {
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                fetch_f(next, b ? buf0 : buf1, &bars[b ^ 1]);
            }
            armed |= 1u << (b ^ 1);
        }
        transform16<LOG2N, -1>(v, tw, buf, t, c);
        const bool ok_nc = zbar_wait(&bars[2], phnc);
        if (__syncthreads_or(!ok_nc)) {
            bail();
            return;
        }
        phnc ^= 1u;
        armed &= ~4u;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int z = t + i * P::T;
            const float m = ns[z * 16 + c] * scale;
            const float2 cd = cs[z * 16 + c];
            v[i] = make_float2(fmaf(v[i].x, m, -cd.x), fmaf(v[i].y, m, -cd.y));
        }
        __syncthreads();  // N and C of this tile consumed
        if (next < ntiles) {
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                fetch_nc(next);
            }
            armed |= 4u;
        }
        transform16<LOG2N, 1>(v, tw, buf, t, c);
        const long long col = tile * 16 + c;
        if (col < M) {
            float2 *g = F + (long long)t * M + col;
#pragma unroll
            for (int i = 0; i < 8; i++, g += (long long)P::T * M) *g = v[i];
        }
    }
}

template <int LOG2N>
cudaError_t launch_tma(float2 *F, float scale, const ZPlan &p, const float2 *tw, const ZMaps &maps, int *err,
                       cudaStream_t s)
{
    using P = Pow2<LOG2N>;
    static int blocks = -1;
    if (blocks < 0) {
        int dev = 0, nsm = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, zfft_tma_kernel<LOG2N>, P::THREADS, Tma<LOG2N>::SMEM);
        blocks = nsm * (per_sm > 0 ? per_sm : 1);
    }
    const long long ntiles = (p.M + 15) / 16;
    const int grid = (int)(ntiles < blocks ? ntiles : blocks);
    zfft_tma_kernel<LOG2N><<<grid, P::THREADS, Tma<LOG2N>::SMEM, s>>>(F, scale, p.M, tw, maps, err);
    return cudaGetLastError();
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
    const void *tma[] = {(const void *)zfft_tma_kernel<7>, (const void *)zfft_tma_kernel<8>,
                         (const void *)zfft_tma_kernel<9>};
    const size_t tma_smem[] = {Tma<7>::SMEM, Tma<8>::SMEM, Tma<9>::SMEM};
    for (int i = 0; i < 3; i++) {
        const cudaError_t e = cudaFuncSetAttribute(tma[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tma_smem[i]);
        if (e != cudaSuccess) return e;
    }
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

bool zfft_tma_ok(const ZPlan &p) { return p.log2n >= 7 && p.log2n <= 9 && p.M % 4 == 0; }

cudaError_t launch_zfft_residual_tma(float2 *F, float scale, const ZPlan &p, const float2 *tw, const ZMaps &maps,
                                     int *err, cudaStream_t s)
{
    switch (p.log2n) {
    case 7: return launch_tma<7>(F, scale, p, tw, maps, err, s);
    case 8: return launch_tma<8>(F, scale, p, tw, maps, err, s);
    case 9: return launch_tma<9>(F, scale, p, tw, maps, err, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace spg
