// Fused smoothing-proximal-gradient iteration for sm_103a (one launch per
// iteration for every volume of a context).
//
// Per voxel v the launch computes, from x_k, d_k = x_k - x_{k-1}, b, w, om1,
// omtv (Sec. 2.1 Eq. 12, 16, 17, 20, 21; Sec. 2.2 Eq. 28 data term):
//   (Dy)_a = [v_a >= 1] ((x_k[v] - x_k[v-e_a]) + beta (d[v] - d[v-e_a]))       Eq. 12 on y
//   p_a    = omtv_v (Dy)_a / max(mu, |Dy_v|)                                   Eq. 16, weighted
//   div    = sum_a p_a[v] - p_a[v+e_a]                                          Eq. 17
//   g      = w ((x_k - b) + beta d) + lambda_tv div                             grad f(y)
//   delta  = beta d - tau g,  z = x_k + delta                                   Eq. 20
//   x_{k+1} = 0 if |z| < t else x_k + (delta - t sign z),  t = tau lambda_l1 om1   Eq. 21
// and, when the step is recorded, the three sums of F(x_k) (data, l1, TV).
//
// y = x_k + beta d is never rounded on its own: differences and the data
// residual are formed from x_k and d separately, and the update is added to
// x_k once, so each iteration commits a single float32 rounding per voxel.
// Two storage forms of the extrapolation pair (template flag XD):
//  - XD = false: x_k and x_{k-1} are stored (three rotating buffers) and
//    d = x_k - x_{k-1} is formed in registers;
//  - XD = true: x_k and the increment d_k are stored (two ping-pong pairs);
//    the kernel writes x_{k+1} = x_k + inc and d_{k+1} = inc, where inc is
//    the float32 increment before it is added to x_k. The momentum term then
//    never sees the rounding of x, which keeps a float32 solve within ~1e-6
//    of exact arithmetic at the cost of one more 4-byte write per voxel.
//
// Data movement: a CTA owns an x-y tile (TX = 32*VX by TY voxels) and marches
// over z. Each z-step's inputs arrive by TMA (cp.async.bulk.tensor) into one
// of S shared-memory stages, tracked by an mbarrier: x_k and x_{k-1} (or d_k) with a
// one-voxel x-y halo (the box starts 4 elements left of the tile so the
// innermost coordinate stays 16-byte aligned), omtv with a +1 halo, and b, w,
// om1 of the plane being written. Plane z's p is computed while plane z-1 is
// written, so each voxel's inputs are read from HBM once per iteration; the
// halo rows come from L2 because neighbouring tiles march the same planes at
// the same time. Warp r of TY computes row r; one extra warp computes the +y
// halo row and the +x halo column. p_y crosses warps through a 3-deep shared
// ring, p_x through a lane shuffle; p_z and the z-1 values stay in registers.
#pragma once

#include <cuda_bf16.h>

#include "spg_internal.h"

namespace spg {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: false when `limit_ns` passed without the phase completing.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 32; i++)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Index checks of the checked build (compiled with -DSPG_CHECK, in place of
// a memory checker): SPG_GUARD(st, cond, code) is `true` in the production
// build; in the checked build a false `cond` records SPG_ECHECK and `code` in
// the device state and the guarded access is skipped.
#ifdef SPG_CHECK
__device__ __noinline__ void check_failed(DevState *st, unsigned code)
{
    atomicCAS(&st->err, 0, (int)SPG_ECHECK);
    atomicCAS(&st->err_info, 0u, code);
}
#define SPG_GUARD(st, cond, code) ((cond) ? true : (::spg::check_failed((st), (code)), false))
#else
#define SPG_GUARD(st, cond, code) true
#endif

// Compensated float32 accumulator (Kahan): per-thread objective sums.
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

// Packed float32 pairs (sm_100 and later issue one instruction for two
// lanes' worth of add, multiply or fused multiply-add). Each lane rounds to
// nearest exactly as the scalar operation does, so the results are bitwise
// those of the scalar code; only the issue slots are halved.
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b rounded once: the product b * (-1) is exact
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// Two compensated (Kahan) float32 accumulators advanced together.
struct KSum2 {
    float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    __device__ __forceinline__ void add(float2 v)
    {
        const float2 y = sub2(v, c);
        const float2 t = add2(s, y);
        c = sub2(sub2(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value_x() const { return (double)s.x - (double)c.x; }
    __device__ __forceinline__ double value_y() const { return (double)s.y - (double)c.y; }
};

// Phase A of one z-step at a thread's VX voxels of plane z: the weighted
// clipped gradient p = omtv (Dy) / max(mu, |Dy|) (Eq. 12, 16) and, with REC,
// the weighted smoothed norm omtv h_mu(D x_k) (Eq. 14) summed into *tsum.
// xl, ld: x_k and d at the voxel left of the first one; xu, du: the row
// above; xz, dz: the plane below. Pairs of voxels go through the packed
// operations; the differences along x (operands one register apart) stay
// scalar.
template <int VX, bool REC>
__device__ __forceinline__ void phase_a(const float (&xc)[VX], const float (&dc)[VX], const float (&xu)[VX],
                                        const float (&du)[VX], const float (&xz)[VX], const float (&dz)[VX],
                                        const float (&om)[VX], float xl, float ld, float beta, float inv_mu,
                                        float half_inv_mu, float half_mu, float mu2, float (&pc)[3][VX],
                                        float *tsum)
{
    if constexpr (VX % 2 == 0) {
        float ex[VX], exd[VX];
#pragma unroll
        for (int i = 0; i < VX; i++) {
            ex[i] = xc[i] - (i ? xc[i - 1] : xl);
            exd[i] = dc[i] - (i ? dc[i - 1] : ld);
        }
        const float2 B = dup2(beta);
        float2 ts = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < VX / 2; q++) {
            const int i = 2 * q;
            const float2 X = make_float2(xc[i], xc[i + 1]), D = make_float2(dc[i], dc[i + 1]);
            const float2 EX = make_float2(ex[i], ex[i + 1]);
            const float2 EY = sub2(X, make_float2(xu[i], xu[i + 1]));
            const float2 EZ = sub2(X, make_float2(xz[i], xz[i + 1]));
            const float2 AX = fma2(B, make_float2(exd[i], exd[i + 1]), EX);
            const float2 AY = fma2(B, sub2(D, make_float2(du[i], du[i + 1])), EY);
            const float2 AZ = fma2(B, sub2(D, make_float2(dz[i], dz[i + 1])), EZ);
            const float2 S2 = fma2(AX, AX, fma2(AY, AY, mul2(AZ, AZ)));
            const float2 SC = mul2(make_float2(om[i], om[i + 1]),
                                   make_float2(fminf(inv_mu, rsqrtf(S2.x)), fminf(inv_mu, rsqrtf(S2.y))));
            const float2 P0 = mul2(AX, SC), P1 = mul2(AY, SC), P2 = mul2(AZ, SC);
            pc[0][i] = P0.x; pc[0][i + 1] = P0.y;
            pc[1][i] = P1.x; pc[1][i + 1] = P1.y;
            pc[2][i] = P2.x; pc[2][i + 1] = P2.y;
            if constexpr (REC) {
                const float2 Q = fma2(EX, EX, fma2(EY, EY, mul2(EZ, EZ)));
                const float2 HQ = mul2(Q, dup2(half_inv_mu));
                const float2 HL = fma2(Q, make_float2(rsqrtf(Q.x), rsqrtf(Q.y)), dup2(-half_mu));
                const float2 H = make_float2(Q.x <= mu2 ? HQ.x : HL.x, Q.y <= mu2 ? HQ.y : HL.y);
                ts = fma2(make_float2(om[i], om[i + 1]), H, ts);
            }
        }
        if constexpr (REC) *tsum = ts.x + ts.y;
    } else {
        float t = 0.f;
#pragma unroll
        for (int i = 0; i < VX; i++) {
            const float lx = i ? xc[i - 1] : xl;
            const float l_d = i ? dc[i - 1] : ld;
            const float ex = xc[i] - lx, ey = xc[i] - xu[i], ez = xc[i] - xz[i];
            const float ax = fmaf(beta, dc[i] - l_d, ex);
            const float ay = fmaf(beta, dc[i] - du[i], ey);
            const float az = fmaf(beta, dc[i] - dz[i], ez);
            const float s2 = fmaf(ax, ax, fmaf(ay, ay, az * az));
            const float sc = om[i] * fminf(inv_mu, rsqrtf(s2));
            pc[0][i] = ax * sc;
            pc[1][i] = ay * sc;
            pc[2][i] = az * sc;
            if constexpr (REC) {
                const float q = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                const float h = q <= mu2 ? q * half_inv_mu : fmaf(q, rsqrtf(q), -half_mu);
                t = fmaf(om[i], h, t);
            }
        }
        if constexpr (REC) *tsum = t;
    }
}

// Phase B at a thread's VX voxels of plane z-1: divergence (Eq. 17), data
// gradient, gradient step and weighted soft-threshold (Eq. 20-21). Writes the
// new iterate `out` and the increment `inc`; with REC adds the data and l1
// terms of F(x_k) into dl (x: data, y: l1), with DOT the restart product
// (y - x+).(x+ - x) into *rsum. pxr: p_x of the voxel right of the last one.
template <int VX, bool REC, bool DOT, bool FOURIER>
__device__ __forceinline__ void phase_b(const float (&pp)[3][VX], float pxn, const float (&pyd)[VX],
                                        const float (&pz)[VX], const float (&xz)[VX], const float (&dz)[VX],
                                        const float (&bb)[VX], const float (&ww)[VX], const float (&oo)[VX],
                                        float beta, float tau, float lam_tv, float tl1, float (&out)[VX],
                                        float (&inc)[VX], float2 *dl, float *rsum)
{
    if constexpr (VX % 2 == 0) {
        float dxx[VX];
#pragma unroll
        for (int i = 0; i < VX; i++) dxx[i] = pp[0][i] - (i < VX - 1 ? pp[0][i + 1] : pxn);
        const float2 B = dup2(beta), NT = dup2(-tau), LT = dup2(lam_tv), TL = dup2(tl1);
        float2 d2 = make_float2(0.f, 0.f), l2 = make_float2(0.f, 0.f);
        float r = 0.f;
#pragma unroll
        for (int q = 0; q < VX / 2; q++) {
            const int i = 2 * q;
            const float2 XZ = make_float2(xz[i], xz[i + 1]), DZ = make_float2(dz[i], dz[i + 1]);
            const float2 DIV = add2(add2(make_float2(dxx[i], dxx[i + 1]),
                                         sub2(make_float2(pp[1][i], pp[1][i + 1]), make_float2(pyd[i], pyd[i + 1]))),
                                    sub2(make_float2(pp[2][i], pp[2][i + 1]), make_float2(pz[i], pz[i + 1])));
            const float2 BB = make_float2(bb[i], bb[i + 1]);
            const float2 RES = sub2(XZ, BB);
            const float2 GD = FOURIER ? BB : mul2(make_float2(ww[i], ww[i + 1]), fma2(B, DZ, RES));
            const float2 G = fma2(LT, DIV, GD);
            const float2 DL = fma2(B, DZ, mul2(NT, G));
            const float2 ZZ = add2(XZ, DL);
            const float2 T = mul2(TL, make_float2(oo[i], oo[i + 1]));
            const float2 CS = make_float2(copysignf(T.x, ZZ.x), copysignf(T.y, ZZ.y));
            const float2 IN0 = sub2(DL, CS);
            const float2 IN = make_float2(fabsf(ZZ.x) < T.x ? -XZ.x : IN0.x, fabsf(ZZ.y) < T.y ? -XZ.y : IN0.y);
            const float2 OUT = add2(XZ, IN);
            out[i] = OUT.x; out[i + 1] = OUT.y;
            inc[i] = IN.x; inc[i + 1] = IN.y;
            if constexpr (DOT) {
                r = fmaf(fmaf(beta, DZ.x, -IN.x), IN.x, r);
                r = fmaf(fmaf(beta, DZ.y, -IN.y), IN.y, r);
            }
            if constexpr (REC) {
                if constexpr (!FOURIER) d2 = fma2(mul2(make_float2(ww[i], ww[i + 1]), RES), RES, d2);
                l2 = fma2(make_float2(oo[i], oo[i + 1]), make_float2(fabsf(XZ.x), fabsf(XZ.y)), l2);
            }
        }
        if constexpr (REC) *dl = make_float2(d2.x + d2.y, l2.x + l2.y);
        if constexpr (DOT) *rsum = r;
    } else {
        float dsum = 0.f, lsum = 0.f, r = 0.f;
#pragma unroll
        for (int i = 0; i < VX; i++) {
            const float pxr = (i < VX - 1) ? pp[0][i + 1] : pxn;
            const float div = (pp[0][i] - pxr) + (pp[1][i] - pyd[i]) + (pp[2][i] - pz[i]);
            const float res = xz[i] - bb[i];
            const float gdat = FOURIER ? bb[i] : ww[i] * fmaf(beta, dz[i], res);
            const float g = fmaf(lam_tv, div, gdat);
            const float delta = fmaf(beta, dz[i], -tau * g);
            const float zz = xz[i] + delta;
            const float t = tl1 * oo[i];
            inc[i] = fabsf(zz) < t ? -xz[i] : delta - copysignf(t, zz);
            out[i] = xz[i] + inc[i];
            if constexpr (DOT) r = fmaf(fmaf(beta, dz[i], -inc[i]), inc[i], r);
            if constexpr (REC) {
                if constexpr (!FOURIER) dsum = fmaf(ww[i] * res, res, dsum);
                lsum = fmaf(oo[i], fabsf(xz[i]), lsum);
            }
        }
        if constexpr (REC) *dl = make_float2(dsum, lsum);
        if constexpr (DOT) *rsum = r;
    }
}

template <int VX>
__device__ __forceinline__ void ld_vec(const float *p, float (&v)[VX])
{
    if constexpr (VX == 4) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else if constexpr (VX == 2) {
        float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x; v[1] = t.y;
    } else {
        v[0] = p[0];
    }
}

template <int VX>
__device__ __forceinline__ void st_vec(float *p, const float (&v)[VX])
{
    if constexpr (VX == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else if constexpr (VX == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
        p[0] = v[0];
    }
}

__device__ __forceinline__ float bf16_bits_to_f32(uint32_t h) { return __uint_as_float(h << 16); }

// Load VX data values stored as float32 or bfloat16 (raw bits widened exactly).
template <int VX, bool BF16>
__device__ __forceinline__ void ld_data(const unsigned char *tile, int idx, float (&v)[VX])
{
    if constexpr (!BF16) {
        ld_vec<VX>(reinterpret_cast<const float *>(tile) + idx, v);
    } else {
        const uint16_t *t = reinterpret_cast<const uint16_t *>(tile) + idx;
        // the low half moves up by 16 bits, the high half is masked in place
        if constexpr (VX == 4) {
            uint2 u = *reinterpret_cast<const uint2 *>(t);
            v[0] = __uint_as_float(u.x << 16); v[1] = __uint_as_float(u.x & 0xffff0000u);
            v[2] = __uint_as_float(u.y << 16); v[3] = __uint_as_float(u.y & 0xffff0000u);
        } else if constexpr (VX == 2) {
            uint32_t u = *reinterpret_cast<const uint32_t *>(t);
            v[0] = __uint_as_float(u << 16); v[1] = __uint_as_float(u & 0xffff0000u);
        } else {
            v[0] = bf16_bits_to_f32(t[0]);
        }
    }
}

template <int VX, int TY, int S, bool BF16>
struct Cfg {
    static constexpr int TX = 32 * VX;
    static constexpr int XW = TX + 8, XH = TY + 2;   // x tiles: origin (x0-4, y0-1)
    static constexpr int OW = TX + 4, OH = TY + 1;   // omtv tile: origin (x0, y0)
    static constexpr int ES = BF16 ? 2 : 4;
    static constexpr int XT_BYTES = XW * XH * 4;
    static constexpr int OM_BYTES = OW * OH * 4;
    static constexpr int BW_BYTES = TX * TY * ES;
    static constexpr int O1_BYTES = TX * TY * 4;
    static constexpr int al(int n) { return (n + 127) / 128 * 128; }
    static constexpr int OFF_XK = 0;
    static constexpr int OFF_XM = OFF_XK + al(XT_BYTES);
    static constexpr int OFF_OM = OFF_XM + al(XT_BYTES);
    static constexpr int OFF_B = OFF_OM + al(OM_BYTES);
    static constexpr int OFF_W = OFF_B + al(BW_BYTES);
    static constexpr int OFF_O1 = OFF_W + al(BW_BYTES);
    static constexpr int STAGE = OFF_O1 + al(O1_BYTES);
    static constexpr int OFF_PY = S * STAGE;                  // 3 x (TY+1) x TX floats
    static constexpr int OFF_HX = OFF_PY + al(3 * (TY + 1) * TX * 4);  // 3 x 32 floats
    static constexpr int OFF_RED = OFF_HX + 3 * 32 * 4;       // 32 x 4 doubles
    static constexpr int OFF_BAR = OFF_RED + 32 * 4 * 8;      // S mbarriers
    static constexpr int OFF_ST = OFF_BAR + al(S * 8);        // state snapshot
    static constexpr int TOTAL = OFF_ST + 128 + 128;          // + alignment slack
    static constexpr int THREADS = 32 * (TY + 1);
    static_assert(TY + 1 <= 32, "reduction scratch sized for at most 32 warps");
    static_assert(TY <= 32, "halo column handled by one lane per row");
};

// Producer (one thread): stage contents for step j of work item W, i.e.
// plane z = z0-1+j of x_k (buffer ia) and of x_{k-1} or d_k (buffer ib), both
// with halo, and of omtv, and plane z-1 of b, w and om1. Steps 0 and 1 skip
// what they do not consume.
template <class C, int S, bool LOADW>
__device__ __forceinline__ void issue_stage(unsigned char *sm, uint64_t *bars, const TmapSet *tm,
                                            const WorkItem &W, int ia, int ib, unsigned gstep, int j)
{
    const int s = (int)((gstep + (unsigned)j) % S);
    unsigned char *base = sm + s * C::STAGE;
    const int z = W.z0 - 1 + j;
    const bool need_om = j >= 1, need_bwo = j >= 2;
    const uint32_t bytes = 2 * C::XT_BYTES + (need_om ? C::OM_BYTES : 0) +
                           (need_bwo ? (LOADW ? 2 : 1) * C::BW_BYTES + C::O1_BYTES : 0);
    mbar_arrive_expect_tx(&bars[s], bytes);
    tma_load_3d(base + C::OFF_XK, &tm->x[ia], W.x0 - 4, W.y0 - 1, z, &bars[s]);
    tma_load_3d(base + C::OFF_XM, &tm->x[ib], W.x0 - 4, W.y0 - 1, z, &bars[s]);
    if (need_om) tma_load_3d(base + C::OFF_OM, &tm->omtv, W.x0, W.y0, z, &bars[s]);
    if (need_bwo) {
        tma_load_3d(base + C::OFF_B, &tm->b, W.x0, W.y0, z - 1, &bars[s]);
        if (LOADW) tma_load_3d(base + C::OFF_W, &tm->w, W.x0, W.y0, z - 1, &bars[s]);
        tma_load_3d(base + C::OFF_O1, &tm->om1, W.x0, W.y0, z - 1, &bars[s]);
    }
}

struct StateSnap {
    int cur, k_round, rec, last;
    long long k_total;
    float pad0, pad1;
};

// Shared-memory carve-up of one CTA.
struct Smem {
    unsigned char *sm;
    uint64_t *bars;
    float *py_ring;
    float *hx_ring;
    double *red;
    StateSnap *snap;
};

// Pipeline bookkeeping of one CTA (owned by thread 0 where noted).
struct Pipe {
    unsigned gstep;         // steps consumed so far
    unsigned issued_upto;   // steps issued so far (thread 0)
    unsigned drain_from;    // first step that may be pending after an abort
};

// One work item: plane-by-plane march over [z0, z1) of one x-y tile.
// REC adds the three sums of F(x_k) (data, l1, TV) for the item.
// Returns true when a barrier wait gave up (the CTA then stops).
template <int VX, int TY, int S, bool BF16, bool XD, bool REC, bool DOT, bool FOURIER>
__device__ __forceinline__ bool run_item(const StepParams &P, const Smem &sh, Pipe &pp_, const WorkItem &W, int it,
                                         int ia, int ib, float *xout_base, float *dout_base)
{
    using C = Cfg<VX, TY, S, BF16>;
    constexpr int TX = C::TX, XW = C::XW, OW = C::OW;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool main_warp = warp < TY;
    const int r = warp;  // tile row of this warp (r == TY: the +y halo row)
    const VolDesc V = P.vols[W.vol];
    const TmapSet *tm = P.tmaps + W.vol;
    const int nsteps = (W.z1 - W.z0) + 2;
    const float beta = SPG_GUARD(P.st, V.kmom >= 0 && V.kmom < P.beta_len, 2u) ? P.beta[V.kmom] : 0.f;
    const float beta_next = (FOURIER && V.kmom + 1 < P.beta_len) ? P.beta[V.kmom + 1] : 0.f;
    // (per volume: restarts reset a volume's extrapolation index)
    const float tau = V.tau, lam_tv = V.lambda_tv, tl1 = V.tau * V.lambda_l1;
    const float inv_mu = 1.0f / V.mu, half_inv_mu = 0.5f / V.mu, half_mu = 0.5f * V.mu;
    const float mu2 = V.mu * V.mu;
    const unsigned g0 = pp_.gstep;

    // the TMA producer is lane 0 of the halo warp, which has no write phase
    const bool producer = (warp == TY) && (lane == 0);
    if (producer) {
        const int pro = nsteps < S ? nsteps : S;
        for (int j = 0; j < pro; j++) issue_stage<C, S, !FOURIER>(sh.sm, sh.bars, tm, W, ia, ib, g0, j);
        pp_.issued_upto = g0 + pro;
    }

    // registers carried across z-steps
    float xz[VX], dz[VX];         // x_k and d on plane z-1, own columns
    float pp[3][VX];              // p on plane z-1, own columns
    float cxz = 0.f, cdz = 0.f;   // +x halo column values on plane z-1
#pragma unroll
    for (int i = 0; i < VX; i++) {
        xz[i] = 0.f;
        dz[i] = 0.f;
        pp[0][i] = pp[1][i] = pp[2][i] = 0.f;
    }
    KSum2 kdl;            // objective sums: data (x) and l1 (y)
    KSum kt, kr;          // TV sum and (DOT) the restart test <y - x+, x+ - x>

    const int gy = W.y0 + r;
    const int gx0 = W.x0 + VX * lane;
    const bool col_lane = (warp == TY) && (lane < TY);
    const bool gy_in = gy < V.ny;

    // Outside the volume the TMA boxes read zeros, so omtv, b, w and om1 are 0
    // there and p and every objective term vanish without per-voxel masks.
    // The zero differences on the first column, row and plane (Eq. 12) are
    // made by substituting the voxel itself for its missing neighbour.
    bool aborted = false;
    // output offset of plane z-1 = W.z0 - 2 + j, advanced by one plane per step
    const long long plane_elems = (long long)V.ny * V.pitch;
    long long o = V.off + ((long long)(W.z0 - 2) * V.ny + gy) * V.pitch + gx0;
    int slot = 0, slot_prev = 2;  // j % 3 and (j - 1) % 3 (p_y and p_x halo rings)
#pragma unroll 2
    for (int j = 0; j < nsteps; j++) {
        const int s = (int)((g0 + j) % S);
        const uint32_t parity = (uint32_t)(((g0 + j) / S) & 1);
        const unsigned char *base = sh.sm + s * C::STAGE;
        const float *XK = reinterpret_cast<const float *>(base + C::OFF_XK);
        const float *XM = reinterpret_cast<const float *>(base + C::OFF_XM);
        const float *OM = reinterpret_cast<const float *>(base + C::OFF_OM);
        const int z = W.z0 - 1 + j;

        const bool ok = mbar_wait(&sh.bars[s], parity, P.timeout_ns);

        // ---- A: p on plane z at this thread's columns ----
        const int tr = r + 1;
        float xc[VX] = {}, mc[VX] = {}, xu[VX] = {}, mu_[VX] = {}, dc[VX];
        if (SPG_GUARD(P.st, tr >= 1 && tr * XW + 4 + VX * (lane + 1) <= XW * C::XH, 3u)) {
            ld_vec<VX>(XK + tr * XW + 4 + VX * lane, xc);
            ld_vec<VX>(XM + tr * XW + 4 + VX * lane, mc);
            ld_vec<VX>(XK + (tr - 1) * XW + 4 + VX * lane, xu);
            ld_vec<VX>(XM + (tr - 1) * XW + 4 + VX * lane, mu_);
        }
        float xl = __shfl_up_sync(FULL, xc[VX - 1], 1);
        float ml = __shfl_up_sync(FULL, mc[VX - 1], 1);
        if (lane == 0) {
            xl = W.x0 == 0 ? xc[0] : XK[tr * XW + 3];
            ml = W.x0 == 0 ? mc[0] : XM[tr * XW + 3];
        }
        if (gy == 0) {
#pragma unroll
            for (int i = 0; i < VX; i++) {
                xu[i] = xc[i];
                mu_[i] = mc[i];
            }
        }
#pragma unroll
        for (int i = 0; i < VX; i++) dc[i] = XD ? mc[i] : xc[i] - mc[i];
        float pc[3][VX];
        if (j >= 1) {
            float om[VX] = {};
            if (SPG_GUARD(P.st, r * OW + VX * (lane + 1) <= OW * C::OH, 5u)) ld_vec<VX>(OM + r * OW + VX * lane, om);
            if (z == 0) {
#pragma unroll
                for (int i = 0; i < VX; i++) {
                    xz[i] = xc[i];
                    dz[i] = dc[i];
                }
            }
            float tsum = 0.f;
            float dup_[VX];
#pragma unroll
            for (int i = 0; i < VX; i++) dup_[i] = XD ? mu_[i] : xu[i] - mu_[i];
            phase_a<VX, REC>(xc, dc, xu, dup_, xz, dz, om, xl, XD ? ml : xl - ml, beta, inv_mu, half_inv_mu,
                             half_mu, mu2, pc, &tsum);
            if constexpr (REC) {
                if (main_warp && z < W.z1) kt.add(tsum);
            }
            // +x halo column (only p_x is consumed), one lane per tile row
            if (col_lane && SPG_GUARD(P.st, (lane + 1) * XW + TX + 4 < XW * C::XH && lane * OW + TX < OW * C::OH, 4u)) {
                const int cr = lane + 1, cc = TX + 4;
                const float cx = XK[cr * XW + cc], cm = XM[cr * XW + cc];
                const float cxl = XK[cr * XW + cc - 1], cml = XM[cr * XW + cc - 1];
                const float cxu = XK[(cr - 1) * XW + cc], cmu = XM[(cr - 1) * XW + cc];
                const float cd = XD ? cm : cx - cm;
                const int hx = W.x0 + TX, hy = W.y0 + lane;
                const float ax = (cx - cxl) + beta * (cd - (XD ? cml : cxl - cml));
                const float ay = hy >= 1 ? (cx - cxu) + beta * (cd - (XD ? cmu : cxu - cmu)) : 0.f;
                const float az = z >= 1 ? (cx - cxz) + beta * (cd - cdz) : 0.f;
                const float s2 = ax * ax + ay * ay + az * az;
                const bool in = hx < V.nx && hy < V.ny && z < V.nz;
                const float sc = in ? OM[lane * OW + TX] * fminf(inv_mu, rsqrtf(s2)) : 0.f;
                sh.hx_ring[slot * 32 + lane] = ax * sc;
            }
            if (SPG_GUARD(P.st, r <= TY && slot == j % 3 && (slot * (TY + 1) + r) * TX + VX * (lane + 1) <= 3 * (TY + 1) * TX, 6u))
                st_vec<VX>(sh.py_ring + (slot * (TY + 1) + r) * TX + VX * lane, pc[1]);
        } else {
#pragma unroll
            for (int i = 0; i < VX; i++) pc[0][i] = pc[1][i] = pc[2][i] = 0.f;
        }
        if (col_lane) {
            const int cr = lane + 1, cc = TX + 4;
            const float cx = XK[cr * XW + cc], cm = XM[cr * XW + cc];
            cxz = cx;
            cdz = XD ? cm : cx - cm;
        }

        if (__syncthreads_or(ok ? 0 : 1)) {
            aborted = true;
            pp_.drain_from = g0 + j;
            break;
        }
        // refill the stage consumed in step j-1
        if (producer && j >= 1 && j - 1 + S < nsteps) {
            issue_stage<C, S, !FOURIER>(sh.sm, sh.bars, tm, W, ia, ib, g0, j - 1 + S);
            pp_.issued_upto = g0 + j + S;
        }

        // ---- B: write plane z-1 ----
        if (main_warp && j >= 2) {
            const int zo = z - 1;
            float bb[VX] = {}, ww[VX] = {}, oo[VX] = {}, pyd[VX] = {};
            if (SPG_GUARD(P.st, r < TY && r * TX + VX * (lane + 1) <= TX * TY, 7u)) {
                ld_data<VX, BF16>(base + C::OFF_B, r * TX + VX * lane, bb);
                if constexpr (!FOURIER) ld_data<VX, BF16>(base + C::OFF_W, r * TX + VX * lane, ww);
                ld_vec<VX>(reinterpret_cast<const float *>(base + C::OFF_O1) + r * TX + VX * lane, oo);
                ld_vec<VX>(sh.py_ring + ((slot_prev * (TY + 1)) + r + 1) * TX + VX * lane, pyd);
            }
            float pxn = __shfl_down_sync(FULL, pp[0][0], 1);
            if (lane == 31) pxn = sh.hx_ring[slot_prev * 32 + r];
            float out[VX], inc[VX];
            float2 dl = make_float2(0.f, 0.f);
            float rsum = 0.f;
            phase_b<VX, REC, DOT, FOURIER>(pp, pxn, pyd, pc[2], xz, dz, bb, ww, oo, beta, tau, lam_tv, tl1, out, inc,
                                           &dl, &rsum);
            if constexpr (REC) kdl.add(dl);
            if constexpr (DOT) kr.add(rsum);
            if (gy_in && gx0 < V.pitch &&
                SPG_GUARD(P.st, zo >= 0 && zo < V.nz && gx0 + VX <= V.pitch &&
                          o == V.off + ((long long)zo * V.ny + gy) * V.pitch + gx0, 8u)) {
                st_vec<VX>(xout_base + o, out);
                if constexpr (XD) st_vec<VX>(dout_base + o, inc);
                if constexpr (FOURIER) {
                    // the next step's extrapolated point, input of its forward transform
                    if (P.ybuf) {
                        float yv[VX];
#pragma unroll
                        for (int i = 0; i < VX; i++) yv[i] = fmaf(beta_next, inc[i], out[i]);
                        st_vec<VX>(P.ybuf + o, yv);
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < VX; i++) {
            xz[i] = xc[i];
            dz[i] = dc[i];
            pp[0][i] = pc[0][i];
            pp[1][i] = pc[1][i];
            pp[2][i] = pc[2][i];
        }
        o += plane_elems;
        slot_prev = slot;
        slot = slot == 2 ? 0 : slot + 1;
    }

    if (!aborted && (REC || DOT)) {
        // block reduction of the item's sums, fixed order
        double v[4] = {0.5 * kdl.value_x(), kdl.value_y(), kt.value(), kr.value()};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int q = 0; q < 4; q++) v[q] += __shfl_down_sync(FULL, v[q], o);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < 4; q++) sh.red[warp * 4 + q] = v[q];
        __syncthreads();
        if (tid == 0) {
            double a[4] = {0, 0, 0, 0};
            for (int w = 0; w < TY + 1; w++)
                for (int q = 0; q < 4; q++) a[q] += sh.red[w * 4 + q];
            for (int q = 0; q < 4; q++) P.partials[(long long)it * 4 + q] = a[q];
        }
    }
    __syncthreads();  // every stage consumed before the next item's prologue
    if (!aborted) pp_.gstep = g0 + nsteps;
    return aborted;
}

template <int VX, int TY, int S, bool BF16, bool XD, int MINB>
__global__ void __launch_bounds__(32 * (TY + 1), MINB)
    spg_step_kernel(const StepParams P)
{
    using C = Cfg<VX, TY, S, BF16>;
    extern __shared__ unsigned char smem_raw[];
    Smem sh;
    // 128-byte aligned start, kept as an offset into the shared array so the
    // compiler addresses every tile as shared memory
    sh.sm = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    sh.bars = reinterpret_cast<uint64_t *>(sh.sm + C::OFF_BAR);
    sh.py_ring = reinterpret_cast<float *>(sh.sm + C::OFF_PY);
    sh.hx_ring = reinterpret_cast<float *>(sh.sm + C::OFF_HX);
    sh.red = reinterpret_cast<double *>(sh.sm + C::OFF_RED);
    sh.snap = reinterpret_cast<StateSnap *>(sh.sm + C::OFF_ST);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        volatile DevState *st = P.st;
        StateSnap s;
        s.cur = st->cur;
        s.k_round = st->k_round;
        s.k_total = st->k_total;
        s.rec = (P.hist_every > 0 && (s.k_total % P.hist_every) == 0) ? 1 : 0;
        s.last = 0;
        *sh.snap = s;
        for (int i = 0; i < S; i++) mbar_init(&sh.bars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // buffers: XD keeps x in 0/1 and d in 2/3; otherwise x_{k-1}, x_k, x_{k+1} rotate over 0..2
    const int cur = sh.snap->cur;
    const int nxt = XD ? (cur ^ 1) : (cur + 1) % 3;
    const int ia = cur, ib = XD ? 2 + cur : (cur + 2) % 3;
    const bool rec = sh.snap->rec != 0;
    // select without indexing the parameter array (keeps the parameters out of local memory)
    auto pick = [&](int i) { return i == 0 ? P.xbuf[0] : (i == 1 ? P.xbuf[1] : (i == 2 ? P.xbuf[2] : P.xbuf[3])); };
    float *const xout_base = pick(nxt);
    float *const dout_base = XD ? pick(2 + nxt) : nullptr;
    if (tid == 0) {
        const int p0 = P.sched[blockIdx.x];
        const TmapSet *tm = P.tmaps + P.items[P.sched[gridDim.x + 1 + (p0 < P.nitems ? p0 : 0)]].vol;
        prefetch_tmap(&tm->x[ia]);
        prefetch_tmap(&tm->x[ib]);
        prefetch_tmap(&tm->omtv);
        prefetch_tmap(&tm->b);
        prefetch_tmap(&tm->w);
        prefetch_tmap(&tm->om1);
    }

    Pipe pipe{0, 0, 0};
    bool aborted = false;
    const int p1 = P.sched[blockIdx.x + 1];
    for (int p = P.sched[blockIdx.x]; p < p1 && !aborted; p++) {
        const int it = P.sched[gridDim.x + 1 + p];
        if (!SPG_GUARD(P.st, p1 <= P.nitems && it >= 0 && it < P.nitems, 1u)) break;
        const WorkItem W = P.items[it];
        bool done = false;
        if constexpr (!BF16 && XD) {
            // Fourier-domain data term (float32 storage, increment storage only)
            if (P.fourier) {
                aborted = rec ? run_item<VX, TY, S, BF16, XD, true, false, true>(P, sh, pipe, W, it, ia, ib,
                                                                                 xout_base, dout_base)
                              : run_item<VX, TY, S, BF16, XD, false, false, true>(P, sh, pipe, W, it, ia, ib,
                                                                                  xout_base, dout_base);
                done = true;
            }
        }
        if (!done) {
            if (P.restart)
                aborted = rec ? run_item<VX, TY, S, BF16, XD, true, true, false>(P, sh, pipe, W, it, ia, ib,
                                                                                 xout_base, dout_base)
                              : run_item<VX, TY, S, BF16, XD, false, true, false>(P, sh, pipe, W, it, ia, ib,
                                                                                  xout_base, dout_base);
            else
                aborted = rec ? run_item<VX, TY, S, BF16, XD, true, false, false>(P, sh, pipe, W, it, ia, ib,
                                                                                  xout_base, dout_base)
                              : run_item<VX, TY, S, BF16, XD, false, false, false>(P, sh, pipe, W, it, ia, ib,
                                                                                   xout_base, dout_base);
        }
    }

    if (aborted && warp == TY && lane == 0) {
        // record the timeout, then wait (bounded) for copies still in flight
        atomicCAS(&P.st->err, 0, (int)SPG_ETIMEOUT);
        for (unsigned q = pipe.drain_from; q < pipe.issued_upto; q++) {
            const int s = (int)(q % S);
            (void)mbar_wait(&sh.bars[s], (uint32_t)((q / S) & 1), P.timeout_ns);
        }
    }

    // ---- last CTA: per-volume objective, then advance the device state ----
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&P.st->ticket, 1u);
        sh.snap->last = (t == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!sh.snap->last) return;
    __threadfence();
    {
        // per volume: objective history (recorded steps), restart test, and
        // the extrapolation index of the next step
        const int hslot = P.st->hist_count % P.hist_cap;
        const bool sums = rec || P.restart != 0;
        VolDesc *vols_rw = const_cast<VolDesc *>(P.vols);
        for (int v = warp; v < P.nvol; v += TY + 1) {
            const VolDesc V = P.vols[v];
            double a[4] = {0, 0, 0, 0};
            if (sums) {
                for (int q = V.item_begin + lane; q < V.item_end; q += 32)
                    for (int c = 0; c < 4; c++) a[c] += __ldcg(P.partials + (long long)q * 4 + c);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int c = 0; c < 4; c++) a[c] += __shfl_down_sync(FULL, a[c], o);
            }
            if (lane == 0) {
                if (rec) {
                    double *h = P.hist + ((long long)hslot * P.nvol + v) * 5;
                    const double l1 = (double)V.lambda_l1 * a[1], tv = (double)V.lambda_tv * a[2];
                    const double tot = a[0] + l1 + tv;
                    h[0] = (double)sh.snap->k_total;
                    h[1] = a[0];
                    h[2] = l1;
                    h[3] = tv;
                    h[4] = tot;
                    if (!isfinite(tot)) atomicCAS(&P.st->err, 0, (int)SPG_ENONFINITE);
                }
                vols_rw[v].beta_last = P.beta[V.kmom];
                vols_rw[v].kmom = (P.restart != 0 && a[3] > 0.0) ? 0 : V.kmom + 1;
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        DevState *st = P.st;
        if (rec) st->hist_count = st->hist_count + 1;
        st->cur = nxt;
        st->k_round = sh.snap->k_round + 1;
        st->k_total = sh.snap->k_total + 1;
        st->ticket = 0;
        __threadfence();
    }
}

template <int VX, int TY, int S, bool BF16, bool XD, int MINB>
struct Launcher {
    using C = Cfg<VX, TY, S, BF16>;
    static cudaError_t configure(int *ctas_per_sm)
    {
        auto k = spg_step_kernel<VX, TY, S, BF16, XD, MINB>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::TOTAL);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k, C::THREADS, C::TOTAL);
    }
    static cudaError_t launch(int grid, const StepParams &p, cudaStream_t s)
    {
        spg_step_kernel<VX, TY, S, BF16, XD, MINB><<<grid, C::THREADS, C::TOTAL, s>>>(p);
        return cudaGetLastError();
    }
};

// Every compiled variant: (vx, ty, stages, minimum resident CTAs per SM).
#define SPG_VARIANTS(X) \
    X(4, 8, 3, 2)       \
    X(4, 7, 3, 2)       \
    X(4, 7, 4, 2)       \
    X(4, 15, 2, 1)      \
    X(4, 4, 4, 3)       \
    X(2, 8, 4, 2)       \
    X(2, 7, 4, 2)       \
    X(2, 4, 4, 3)

}  // namespace

// Dispatch over the compiled variants for one data dtype (BF16_).
#define SPG_DEFINE_DISPATCH(BF16_, SUFFIX)                                                          \
    size_t step_smem_bytes_##SUFFIX(const StepVariant &v)                                           \
    {                                                                                               \
        SPG_VARIANTS(SPG_SM_CASE)                                                                   \
        return 0;                                                                                   \
    }                                                                                               \
    cudaError_t step_configure_##SUFFIX(const StepVariant &v, int *occ)                             \
    {                                                                                               \
        SPG_VARIANTS(SPG_CF_CASE)                                                                   \
        return cudaErrorInvalidValue;                                                               \
    }                                                                                               \
    cudaError_t step_launch_##SUFFIX(const StepVariant &v, int grid, const StepParams &p, cudaStream_t s) \
    {                                                                                               \
        SPG_VARIANTS(SPG_LN_CASE)                                                                   \
        return cudaErrorInvalidValue;                                                               \
    }
#define SPG_SM_CASE(VX_, TY_, S_, MB_) \
    if (v.vx == VX_ && v.ty == TY_ && v.stages == S_) return Cfg<VX_, TY_, S_, SPG_BF16_FLAG>::TOTAL;
#define SPG_CF_CASE(VX_, TY_, S_, MB_)                                                             \
    if (v.vx == VX_ && v.ty == TY_ && v.stages == S_)                                              \
        return v.xd ? Launcher<VX_, TY_, S_, SPG_BF16_FLAG, true, MB_>::configure(occ)              \
                    : Launcher<VX_, TY_, S_, SPG_BF16_FLAG, false, MB_>::configure(occ);
#define SPG_LN_CASE(VX_, TY_, S_, MB_)                                                             \
    if (v.vx == VX_ && v.ty == TY_ && v.stages == S_)                                              \
        return v.xd ? Launcher<VX_, TY_, S_, SPG_BF16_FLAG, true, MB_>::launch(grid, p, s)          \
                    : Launcher<VX_, TY_, S_, SPG_BF16_FLAG, false, MB_>::launch(grid, p, s);

}  // namespace spg
