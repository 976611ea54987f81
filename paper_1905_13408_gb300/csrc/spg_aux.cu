// Auxiliary kernels of the GB300 SPG solver: input validation and dtype
// conversion, the re-weighting pass (Eq. 11), the objective (Eq. 14 / 31),
// the strong-convexity certificate, the passes of the adjoint of one step,
// and the plain step used under alternative readings of the paper.
//
// None of them is on the fused hot path, so they use plain global loads.
// All but the two adjoint passes run AUX_SEG CTAs per z-plane (one per row
// segment), every reduction keeps one partial per segment, and the last CTA
// to finish sums the partials of each volume in segment order, so the
// results are deterministic; the adjoint passes march over z (a CTA per
// tile of rows and run of planes) and keep one scalar partial per CTA,
// which the host sums in a fixed order. No kernel here waits on another CTA.
#include <cuda_bf16.h>

#include <algorithm>

#include "spg_internal.h"

namespace spg {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int AUX_THREADS = 256;

// Each z-plane is split into AUX_SEG row segments, one CTA each; partial sums
// are kept per segment (index plane * AUX_SEG + segment).
__device__ __forceinline__ void seg_rows(int ny, int seg, int &r0, int &r1)
{
    r0 = (int)((long long)ny * seg / AUX_SEG);
    r1 = (int)((long long)ny * (seg + 1) / AUX_SEG);
}

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

__device__ __forceinline__ float ld_data(const void *p, bool bf16, long long i)
{
    if (bf16) return __uint_as_float(((uint32_t) reinterpret_cast<const uint16_t *>(p)[i]) << 16);
    return reinterpret_cast<const float *>(p)[i];
}

// Block-wide sum of up to 4 doubles in a fixed order; result valid in thread 0.
template <int N>
__device__ void block_sum(double (&v)[N], double *scratch /* 32*N */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < N; q++) v[q] += __shfl_down_sync(FULL, v[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < N; q++) scratch[warp * N + q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x / 32;
        for (int q = 0; q < N; q++) {
            double a = 0;
            for (int k = 0; k < nw; k++) a += scratch[k * N + q];
            v[q] = a;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ double block_max(double v, double *scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(FULL, v, o));
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x / 32;
        for (int k = 0; k < nw; k++) v = fmax(v, scratch[k]);
    }
    __syncthreads();
    return v;
}

// Last-CTA election on a counter; returns true in every thread of the last CTA.
__device__ bool last_block(unsigned int *ticket, int *flag_smem)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        *flag_smem = (t == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    const bool last = *flag_smem != 0;
    if (last) __threadfence();
    return last;
}

// ---------------- validation ----------------
// One CTA per z-plane of volume `vol`: max w, min w, count(w <= 0 or w not
// finite), count(b not finite).
__global__ void validate_kernel(AuxParams a, int vol, const void *b, const void *w, bool bf16, double *maxw_out)
{
    __shared__ double scratch[32 * 4];
    __shared__ int flag;
    const VolDesc V = a.vols[vol];
    const int z = blockIdx.x / AUX_SEG;
    int r0, r1;
    seg_rows(V.ny, blockIdx.x % AUX_SEG, r0, r1);
    // per-thread work in float32 and integers (max and min are exact in any precision)
    float fmx = 0.f, fmn = INFINITY;
    int bad_w = 0, bad_b = 0;
    for (int t = threadIdx.x; t < (r1 - r0) * V.nx; t += blockDim.x) {
        const int x = t % V.nx, y = r0 + t / V.nx;
        const long long i = V.off + ((long long)z * V.ny + y) * V.pitch + x;
        const float wv = ld_data(w, bf16, i), bv = ld_data(b, bf16, i);
        const bool wfin = isfinite(wv);
        bad_w += (!(wv > 0.f) || !wfin) ? 1 : 0;
        bad_b += isfinite(bv) ? 0 : 1;
        if (wfin) {
            fmx = fmaxf(fmx, wv);
            fmn = fminf(fmn, wv);
        }
    }
    double mx = block_max((double)fmx, scratch);
    const double nmn = block_max(-(double)fmn, scratch);
    double c[2] = {(double)bad_w, (double)bad_b};
    block_sum<2>(c, scratch);
    if (threadIdx.x == 0) {
        double *pp = a.plane_part + (long long)blockIdx.x * 4;
        pp[0] = mx;
        pp[1] = -nmn;
        pp[2] = c[0];
        pp[3] = c[1];
    }
    if (!last_block(&a.st->ticket_aux, &flag)) return;
    {
        double m = 0, n = INFINITY, c2[2] = {0, 0};
        for (int q = threadIdx.x; q < V.nz * AUX_SEG; q += blockDim.x) {
            const double *pp = a.plane_part + (long long)q * 4;
            m = fmax(m, __ldcg(pp + 0));
            n = fmin(n, __ldcg(pp + 1));
            c2[0] += __ldcg(pp + 2);
            c2[1] += __ldcg(pp + 3);
        }
        m = block_max(m, scratch);
        n = -block_max(-n, scratch);
        block_sum<2>(c2, scratch);
        const double bw = c2[0], bb = c2[1];
        if (threadIdx.x != 0) return;
        double *o = a.vol_out + (long long)vol * 8;
        o[0] = m;
        o[1] = n;
        o[2] = bw;
        o[3] = bb;
        maxw_out[vol] = m;
        a.st->ticket_aux = 0;
        __threadfence();
    }
}

// ---------------- implicit-gradient anchor (Eq. 22 / Eq. 31) ----------------
__device__ __forceinline__ void st_data(void *p, bool bf16, long long i, float v)
{
    if (bf16) {
        __nv_bfloat16 h = __float2bfloat16_rn(v);
        reinterpret_cast<uint16_t *>(p)[i] = *reinterpret_cast<uint16_t *>(&h);
    } else {
        reinterpret_cast<float *>(p)[i] = v;
    }
}

// w' = w + 2 gamma, b' = (w b + 2 gamma a) / w'; then max w' per volume.
__global__ void anchor_kernel(AuxParams a, int vol, void *b, void *w, bool bf16, const float *anchor, float gamma,
                              double *maxw_out)
{
    __shared__ double scratch[32 * 4];
    __shared__ int flag;
    const VolDesc V = a.vols[vol];
    const int z = blockIdx.x / AUX_SEG;
    int r0, r1;
    seg_rows(V.ny, blockIdx.x % AUX_SEG, r0, r1);
    double mx = 0.0;
    for (int t = threadIdx.x; t < (r1 - r0) * V.nx; t += blockDim.x) {
        const int x = t % V.nx, y = r0 + t / V.nx;
        const long long i = V.off + ((long long)z * V.ny + y) * V.pitch + x;
        const float wv = ld_data(w, bf16, i), bv = ld_data(b, bf16, i);
        const float w2 = wv + 2.0f * gamma;
        const float b2 = (wv * bv + 2.0f * gamma * anchor[i]) / w2;
        st_data(w, bf16, i, w2);
        st_data(b, bf16, i, b2);
        mx = fmax(mx, (double)ld_data(w, bf16, i));
    }
    mx = block_max(mx, scratch);
    if (threadIdx.x == 0) a.plane_part[(long long)blockIdx.x * 4] = mx;
    if (!last_block(&a.st->ticket_aux, &flag)) return;
    double m = 0;
    for (int q = threadIdx.x; q < V.nz * AUX_SEG; q += blockDim.x) m = fmax(m, __ldcg(a.plane_part + (long long)q * 4));
    m = block_max(m, scratch);
    if (threadIdx.x == 0) {
        maxw_out[vol] = m;
        a.st->ticket_aux = 0;
        __threadfence();
    }
}

// Sec. 2.5 scales: sum (w b)^2, sum w, max w, min w of one volume.
__global__ void scales_kernel(AuxParams a, int vol, const void *b, const void *w, bool bf16)
{
    __shared__ double scratch[32 * 4];
    __shared__ int flag;
    const VolDesc V = a.vols[vol];
    const int z = blockIdx.x / AUX_SEG;
    int r0, r1;
    seg_rows(V.ny, blockIdx.x % AUX_SEG, r0, r1);
    KSum s2, sw;
    double mx = 0.0, mn = INFINITY;
    for (int t = threadIdx.x; t < (r1 - r0) * V.nx; t += blockDim.x) {
        const int x = t % V.nx, y = r0 + t / V.nx;
        const long long i = V.off + ((long long)z * V.ny + y) * V.pitch + x;
        const float wv = ld_data(w, bf16, i), bv = ld_data(b, bf16, i);
        const float n = wv * bv;
        s2.add(n * n);
        sw.add(wv);
        mx = fmax(mx, (double)wv);
        mn = fmin(mn, (double)wv);
    }
    mx = block_max(mx, scratch);
    const double nmn = block_max(-mn, scratch);
    double v[2] = {s2.value(), sw.value()};
    block_sum<2>(v, scratch);
    if (threadIdx.x == 0) {
        double *pp = a.plane_part + (long long)blockIdx.x * 4;
        pp[0] = v[0];
        pp[1] = v[1];
        pp[2] = mx;
        pp[3] = -nmn;
    }
    if (!last_block(&a.st->ticket_aux, &flag)) return;
    double c2[2] = {0, 0}, m = 0, n = INFINITY;
    for (int q = threadIdx.x; q < V.nz * AUX_SEG; q += blockDim.x) {
        const double *pp = a.plane_part + (long long)q * 4;
        c2[0] += __ldcg(pp + 0);
        c2[1] += __ldcg(pp + 1);
        m = fmax(m, __ldcg(pp + 2));
        n = fmin(n, __ldcg(pp + 3));
    }
    block_sum<2>(c2, scratch);
    m = block_max(m, scratch);
    n = -block_max(-n, scratch);
    if (threadIdx.x == 0) {
        const double q2 = c2[0], qw = c2[1];
        const double cnt = (double)V.nx * V.ny * V.nz;
        double *o = a.vol_out + (long long)vol * 8;
        o[0] = sqrt(q2 / cnt);
        o[1] = qw / cnt;
        o[2] = m;
        o[3] = n;
        a.st->ticket_aux = 0;
        __threadfence();
    }
}

__global__ void to_bf16_kernel(const float *src, uint16_t *dst, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        __nv_bfloat16 h = __float2bfloat16_rn(src[i]);
        dst[i] = *reinterpret_cast<uint16_t *>(&h);
    }
}

__global__ void to_f32_kernel(const uint16_t *src, float *dst, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = __uint_as_float(((uint32_t)src[i]) << 16);
}

// ---------------- stencil helpers (plain global loads) ----------------

// Value of u = x_k + beta (x_k - x_{k-1}) is never formed; differences are
// taken of x_k and of d = x_k - x_{k-1} separately (one rounding each).
struct Field {
    const float *xk, *xkm1;   // xkm1 may be null (then d = 0, unless dk is given)
    float beta;
    const float *dk = nullptr;  // stored increment x_k - x_{k-1}, if any
    __device__ __forceinline__ float x(long long i) const { return xk[i]; }
    __device__ __forceinline__ float d(long long i) const
    {
        return dk ? dk[i] : (xkm1 ? xk[i] - xkm1[i] : 0.f);
    }
};

// D u at (x, y, z) under the SPG_READ_* flags of the volume (forward
// differences and/or a periodic boundary); kept out of line so the adopted
// reading's code below stays small.
__device__ __noinline__ void grad_at_readings(const VolDesc &V, const Field &F, int x, int y, int z, float g[3])
{
    const long long i = V.off + ((long long)z * V.ny + y) * V.pitch + x;
    const float xc = F.x(i), dc = F.d(i);
    const bool fwd = (V.readings & SPG_READ_FORWARD) != 0, per = (V.readings & SPG_READ_PERIODIC) != 0;
    const int co[3] = {x, y, z}, ext[3] = {V.nx, V.ny, V.nz};
    const long long stp[3] = {1, V.pitch, (long long)V.pitch * V.ny};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int c = co[a], n = ext[a];
        long long j;
        if (!fwd) {
            if (c >= 1) j = i - stp[a];
            else if (per && n > 1) j = i + (long long)(n - 1) * stp[a];
            else { g[a] = 0.f; continue; }
            g[a] = (xc - F.x(j)) + F.beta * (dc - F.d(j));
        } else {
            if (c + 1 <= n - 1) j = i + stp[a];
            else if (per && n > 1) j = i - (long long)(n - 1) * stp[a];
            else { g[a] = 0.f; continue; }
            g[a] = (F.x(j) - xc) + F.beta * (F.d(j) - dc);
        }
    }
}

// D u at (x, y, z) in volume V. Adopted reading: backward differences that
// vanish on the first plane of each axis (Eq. 12).
__device__ __forceinline__ void grad_at(const VolDesc &V, const Field &F, int x, int y, int z, float g[3])
{
    if (V.readings != 0) {
        grad_at_readings(V, F, x, y, z, g);
        return;
    }
    const long long i = V.off + ((long long)z * V.ny + y) * V.pitch + x;
    const float xc = F.x(i), dc = F.d(i);
    g[0] = x >= 1 ? (xc - F.x(i - 1)) + F.beta * (dc - F.d(i - 1)) : 0.f;
    g[1] = y >= 1 ? (xc - F.x(i - V.pitch)) + F.beta * (dc - F.d(i - V.pitch)) : 0.f;
    const long long ps = (long long)V.pitch * V.ny;
    g[2] = z >= 1 ? (xc - F.x(i - ps)) + F.beta * (dc - F.d(i - ps)) : 0.f;
}

// p = omtv * D u / max(mu, |D u|) at (x, y, z) (without omtv under
// SPG_READ_POST_DIV); zero outside the volume.
__device__ __forceinline__ void p_at(const VolDesc &V, const Field &F, const float *omtv, int x, int y, int z,
                                     float p[3])
{
    if (x < 0 || y < 0 || z < 0 || x >= V.nx || y >= V.ny || z >= V.nz) {
        p[0] = p[1] = p[2] = 0.f;
        return;
    }
    float g[3];
    grad_at(V, F, x, y, z, g);
    const long long i = V.off + ((long long)z * V.ny + y) * V.pitch + x;
    const float s2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    const float om = (V.readings & SPG_READ_POST_DIV) ? 1.0f : omtv[i];
    const float sc = om * fminf(1.0f / V.mu, rsqrtf(s2));
    p[0] = g[0] * sc;
    p[1] = g[1] * sc;
    p[2] = g[2] * sc;
}

// (D^T p)(x, y, z) with p evaluated on the fly (Eq. 17 for the adopted
// reading; the adjoint of the selected D otherwise, times omtv under
// SPG_READ_POST_DIV).
__device__ __forceinline__ float div_at(const VolDesc &V, const Field &F, const float *omtv, int x, int y, int z)
{
    float pc[3], px[3], pyv[3], pz[3];
    p_at(V, F, omtv, x, y, z, pc);
    if (V.readings == 0) {
        p_at(V, F, omtv, x + 1, y, z, px);
        p_at(V, F, omtv, x, y + 1, z, pyv);
        p_at(V, F, omtv, x, y, z + 1, pz);
        return (pc[0] - px[0]) + (pc[1] - pyv[1]) + (pc[2] - pz[2]);
    }
    const bool fwd = (V.readings & SPG_READ_FORWARD) != 0, per = (V.readings & SPG_READ_PERIODIC) != 0;
    // neighbour along each axis: successor (backward D) or predecessor (forward D),
    // wrapped under the periodic boundary, else possibly outside (p = 0 there)
    auto nb = [&](int c, int n) {
        const int d = fwd ? c - 1 : c + 1;
        return per ? (d + n) % n : d;
    };
    p_at(V, F, omtv, nb(x, V.nx), y, z, px);
    p_at(V, F, omtv, x, nb(y, V.ny), z, pyv);
    p_at(V, F, omtv, x, y, nb(z, V.nz), pz);
    float r = fwd ? (px[0] - pc[0]) + (pyv[1] - pc[1]) + (pz[2] - pc[2])
                  : (pc[0] - px[0]) + (pc[1] - pyv[1]) + (pc[2] - pz[2]);
    if (V.readings & SPG_READ_POST_DIV) r *= omtv[V.off + ((long long)z * V.ny + y) * V.pitch + x];
    return r;
}

// ---------------- row-vector walks for the adopted reading ----------------
// The re-weighting and the objective read every voxel once plus three
// neighbours; with one voxel per thread they wait on memory latency. The
// adopted reading's kernels instead walk a row segment in 128-voxel chunks:
// each warp takes a chunk of a row, each lane 4 consecutive voxels (16-byte
// loads: rows start 32-byte aligned, the pitch being a multiple of 8 and
// volume offsets of 64 elements). The x-neighbour of a lane's first voxel
// comes from the lane before it (the first lane of a chunk loads it).
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

__device__ __forceinline__ float4 ld4_data(const void *p, bool bf16, long long i)
{
    if (!bf16) return ld4(reinterpret_cast<const float *>(p) + i);
    const uint2 u = *reinterpret_cast<const uint2 *>(reinterpret_cast<const uint16_t *>(p) + i);
    return make_float4(__uint_as_float((u.x & 0xffffu) << 16), __uint_as_float(u.x & 0xffff0000u),
                       __uint_as_float((u.y & 0xffffu) << 16), __uint_as_float(u.y & 0xffff0000u));
}

__device__ __forceinline__ void unpack4(const float4 v, float (&o)[4])
{
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
}

// x and D x (Eq. 12, zero on first planes) at voxels x0 .. x0+3 of row (y, z);
// inactive lanes (x0 >= nx) get zeros but still take part in the shuffle.
__device__ __forceinline__ void grad4_at(const VolDesc &V, const float *xs, int x0, int y, int z, int lane,
                                         bool act, float (&xc)[4], float (&gx)[4], float (&gy)[4], float (&gz)[4])
{
    const long long row = V.off + ((long long)z * V.ny + y) * V.pitch;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 c = act ? ld4(xs + row + x0) : zero;
    float xl = __shfl_up_sync(FULL, c.w, 1);
    if (lane == 0) xl = (act && x0 >= 1) ? xs[row + x0 - 1] : c.x;
    if (x0 == 0) xl = c.x;
    const float4 u = (act && y >= 1) ? ld4(xs + row - V.pitch + x0) : c;
    const float4 w = (act && z >= 1) ? ld4(xs + row - (long long)V.pitch * V.ny + x0) : c;
    float uu[4], ww[4];
    unpack4(c, xc);
    unpack4(u, uu);
    unpack4(w, ww);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        gx[q] = xc[q] - (q ? xc[q - 1] : xl);
        gy[q] = xc[q] - uu[q];
        gz[q] = xc[q] - ww[q];
    }
}

__global__ void reweight4_kernel(AuxParams a, const float *xcur, float *om1, float *omtv, const double *maxw,
                                 double *rstats, VolDesc *vols_rw);
__global__ void objective4_kernel(AuxParams a, const float *xcur, const void *b, const void *w, bool bf16,
                                  const float *om1, const float *omtv);

// Last CTA of a re-weighting launch: per-volume max omtv, nnz, sums, and
// tau = 1/L (FP64), then the round restarts.
__device__ void reweight_finish(const AuxParams &a, const double *maxw, double *rstats, VolDesc *vols_rw,
                                double *scratch)
{
    for (int v = 0; v < a.nvol; v++) {
        const VolDesc W = a.vols[v];
        double m = 0, c3[3] = {0, 0, 0};
        for (int q = (W.plane_begin + W.halo_lo) * AUX_SEG + threadIdx.x; q < (W.plane_begin + W.nz - W.halo_hi) * AUX_SEG; q += blockDim.x) {
            const double *pp = a.plane_part + (long long)q * 4;
            m = fmax(m, __ldcg(pp + 0));
            c3[0] += __ldcg(pp + 1);
            c3[1] += __ldcg(pp + 2);
            c3[2] += __ldcg(pp + 3);
        }
        m = block_max(m, scratch);
        block_sum<3>(c3, scratch);
        const double n = c3[0], s1 = c3[1], s2 = c3[2];
        if (threadIdx.x == 0) {
            const double L = maxw[v] + 12.0 * (double)W.lambda_tv * m / (double)W.mu;
            const double tau = 1.0 / L;
            double *o = rstats + (long long)v * 6;
            o[0] = m;
            o[1] = n;
            o[2] = s1;
            o[3] = s2;
            o[4] = L;
            o[5] = tau;
            vols_rw[v].tau = (float)tau;
            vols_rw[v].kmom = 0;  // extrapolation restarts with the round
            vols_rw[v].beta_last = 0.f;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.st->k_round = 0;
        a.st->ticket_aux = 0;
        __threadfence();
    }
}

// Last CTA of an objective launch: per-volume (data, l1, tv, total).
__device__ void objective_finish(const AuxParams &a, double *scratch)
{
    for (int v = 0; v < a.nvol; v++) {
        const VolDesc W = a.vols[v];
        double c3[3] = {0, 0, 0};
        for (int q = (W.plane_begin + W.halo_lo) * AUX_SEG + threadIdx.x; q < (W.plane_begin + W.nz - W.halo_hi) * AUX_SEG; q += blockDim.x) {
            const double *pp = a.plane_part + (long long)q * 4;
            c3[0] += __ldcg(pp + 0);
            c3[1] += __ldcg(pp + 1);
            c3[2] += __ldcg(pp + 2);
        }
        block_sum<3>(c3, scratch);
        if (threadIdx.x != 0) continue;
        const double d = c3[0], l = c3[1], t = c3[2];
        double *o = a.vol_out + (long long)v * 8;
        o[0] = d;
        o[1] = (double)W.lambda_l1 * l;
        o[2] = (double)W.lambda_tv * t;
        o[3] = o[0] + o[1] + o[2];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.st->ticket_aux = 0;
        __threadfence();
    }
}

// ---------------- re-weighting (Eq. 11, eps scaling of Sec. 2.5) ----------------
__global__ void reweight_kernel(AuxParams a, const float *xcur, float *om1, float *omtv, const double *maxw,
                                double *rstats, VolDesc *vols_rw)
{
    __shared__ double scratch[32 * 4];
    __shared__ int flag;
    const int plane = blockIdx.x / AUX_SEG;
    const int vol = a.plane_vol[plane];
    const VolDesc V = a.vols[vol];
    const int z = plane - V.plane_begin;
    int r0, r1;
    seg_rows(V.ny, blockIdx.x % AUX_SEG, r0, r1);
    const Field F{xcur, nullptr, 0.f};
    float fmx = 0.f;
    KSum c1, c2;
    float nnz = 0.f;
    for (int t = threadIdx.x; t < (r1 - r0) * V.nx; t += blockDim.x) {
        const int x = t % V.nx, y = r0 + t / V.nx;
        const long long i = V.off + ((long long)z * V.ny + y) * V.pitch + x;
        float g[3];
        grad_at(V, F, x, y, z, g);
        const float gn = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        const float xv = xcur[i];
        const float o1 = V.eps / (fabsf(xv) + V.eps);
        const float ot = V.eps_tv / (gn + V.eps_tv);
        om1[i] = o1;
        omtv[i] = ot;
        fmx = fmaxf(fmx, ot);
        nnz += xv != 0.f ? 1.f : 0.f;
        c1.add(o1);
        c2.add(ot);
    }
    const double mx = block_max((double)fmx, scratch);
    double s[3] = {(double)nnz, c1.value(), c2.value()};
    block_sum<3>(s, scratch);
    if (threadIdx.x == 0) {
        double *pp = a.plane_part + (long long)blockIdx.x * 4;
        pp[0] = mx;
        pp[1] = s[0];
        pp[2] = s[1];
        pp[3] = s[2];
    }
    if (!last_block(&a.st->ticket_aux, &flag)) return;
    reweight_finish(a, maxw, rstats, vols_rw, scratch);
}

// ---------------- objective F(x) at the current iterate ----------------
__global__ void objective_kernel(AuxParams a, const float *xcur, const void *b, const void *w, bool bf16,
                                 const float *om1, const float *omtv)
{
    __shared__ double scratch[32 * 4];
    __shared__ int flag;
    const int plane = blockIdx.x / AUX_SEG;
    const int vol = a.plane_vol[plane];
    const VolDesc V = a.vols[vol];
    const int z = plane - V.plane_begin;
    int r0, r1;
    seg_rows(V.ny, blockIdx.x % AUX_SEG, r0, r1);
    const Field F{xcur, nullptr, 0.f};
    KSum kd, kl, kt;
    const float mu = V.mu;
    for (int t = threadIdx.x; t < (r1 - r0) * V.nx; t += blockDim.x) {
        const int x = t % V.nx, y = r0 + t / V.nx;
        const long long i = V.off + ((long long)z * V.ny + y) * V.pitch + x;
        float g[3];
        grad_at(V, F, x, y, z, g);
        const float q = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        const float h = q <= mu * mu ? q * (0.5f / mu) : q * rsqrtf(q) - 0.5f * mu;
        const float xv = xcur[i];
        if (w) {  // no real-space data term when the Fourier-domain term is in use
            const float r = xv - ld_data(b, bf16, i);
            kd.add(0.5f * ld_data(w, bf16, i) * r * r);
        }
        kl.add(om1[i] * fabsf(xv));
        kt.add(omtv[i] * h);
    }
    double s[3] = {kd.value(), kl.value(), kt.value()};
    block_sum<3>(s, scratch);
    if (threadIdx.x == 0) {
        double *pp = a.plane_part + (long long)blockIdx.x * 4;
        pp[0] = s[0];
        pp[1] = s[1];
        pp[2] = s[2];
        pp[3] = 0;
    }
    if (!last_block(&a.st->ticket_aux, &flag)) return;
    objective_finish(a, scratch);
}

// Re-weighting of the adopted reading, row-vector walk (same results as
// reweight_kernel; padding columns of the pitch get zero weights).
__global__ void reweight4_kernel(AuxParams a, const float *xcur, float *om1, float *omtv, const double *maxw,
                                 double *rstats, VolDesc *vols_rw)
{
    __shared__ double scratch[32 * 4];
    __shared__ int flag;
    const int plane = blockIdx.x / AUX_SEG;
    const int vol = a.plane_vol[plane];
    const VolDesc V = a.vols[vol];
    const int z = plane - V.plane_begin;
    int r0, r1;
    seg_rows(V.ny, blockIdx.x % AUX_SEG, r0, r1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nchunk = (V.nx + 127) / 128;
    float fmx = 0.f, nnz = 0.f;
    KSum c1, c2;
    for (int rc = warp; rc < (r1 - r0) * nchunk; rc += nwarps) {
        const int y = r0 + rc / nchunk, x0 = (rc % nchunk) * 128 + 4 * lane;
        const bool act = x0 < V.nx;
        float xc[4], gx[4], gy[4], gz[4], o1[4], ot[4];
        grad4_at(V, xcur, x0, y, z, lane, act, xc, gx, gy, gz);
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const bool valid = act && x0 + q < V.nx;
            const float gn = sqrtf(gx[q] * gx[q] + gy[q] * gy[q] + gz[q] * gz[q]);
            o1[q] = valid ? V.eps / (fabsf(xc[q]) + V.eps) : 0.f;
            ot[q] = valid ? V.eps_tv / (gn + V.eps_tv) : 0.f;
            fmx = fmaxf(fmx, ot[q]);
            nnz += (valid && xc[q] != 0.f) ? 1.f : 0.f;
            s1 += o1[q];
            s2 += ot[q];
        }
        if (act) {
            const long long i = V.off + ((long long)z * V.ny + y) * V.pitch + x0;
            *reinterpret_cast<float4 *>(om1 + i) = make_float4(o1[0], o1[1], o1[2], o1[3]);
            *reinterpret_cast<float4 *>(omtv + i) = make_float4(ot[0], ot[1], ot[2], ot[3]);
        }
        c1.add(s1);
        c2.add(s2);
    }
    const double mx = block_max((double)fmx, scratch);
    double sm[3] = {(double)nnz, c1.value(), c2.value()};
    block_sum<3>(sm, scratch);
    if (threadIdx.x == 0) {
        double *pp = a.plane_part + (long long)blockIdx.x * 4;
        pp[0] = mx;
        pp[1] = sm[0];
        pp[2] = sm[1];
        pp[3] = sm[2];
    }
    if (!last_block(&a.st->ticket_aux, &flag)) return;
    reweight_finish(a, maxw, rstats, vols_rw, scratch);
}

// Objective of the adopted reading, row-vector walk (same sums as
// objective_kernel; padding columns contribute nothing).
__global__ void objective4_kernel(AuxParams a, const float *xcur, const void *b, const void *w, bool bf16,
                                  const float *om1, const float *omtv)
{
    __shared__ double scratch[32 * 4];
    __shared__ int flag;
    const int plane = blockIdx.x / AUX_SEG;
    const int vol = a.plane_vol[plane];
    const VolDesc V = a.vols[vol];
    const int z = plane - V.plane_begin;
    int r0, r1;
    seg_rows(V.ny, blockIdx.x % AUX_SEG, r0, r1);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int nchunk = (V.nx + 127) / 128;
    const float mu = V.mu;
    KSum kd, kl, kt;
    for (int rc = warp; rc < (r1 - r0) * nchunk; rc += nwarps) {
        const int y = r0 + rc / nchunk, x0 = (rc % nchunk) * 128 + 4 * lane;
        const bool act = x0 < V.nx;
        const long long i = V.off + ((long long)z * V.ny + y) * V.pitch + x0;
        float xc[4], gx[4], gy[4], gz[4], o1[4], ot[4], bv[4], wv[4];
        grad4_at(V, xcur, x0, y, z, lane, act, xc, gx, gy, gz);
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        unpack4(act ? ld4(om1 + i) : zero, o1);
        unpack4(act ? ld4(omtv + i) : zero, ot);
        unpack4((act && w) ? ld4_data(b, bf16, i) : zero, bv);
        unpack4((act && w) ? ld4_data(w, bf16, i) : zero, wv);
        float sd = 0.f, sl = 0.f, st = 0.f;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            if (!(act && x0 + q < V.nx)) continue;
            const float qq = gx[q] * gx[q] + gy[q] * gy[q] + gz[q] * gz[q];
            const float h = qq <= mu * mu ? qq * (0.5f / mu) : qq * rsqrtf(qq) - 0.5f * mu;
            const float r = xc[q] - bv[q];
            sd += 0.5f * wv[q] * r * r;
            sl += o1[q] * fabsf(xc[q]);
            st += ot[q] * h;
        }
        kd.add(sd);
        kl.add(sl);
        kt.add(st);
    }
    double sm[3] = {kd.value(), kl.value(), kt.value()};
    block_sum<3>(sm, scratch);
    if (threadIdx.x == 0) {
        double *pp = a.plane_part + (long long)blockIdx.x * 4;
        pp[0] = sm[0];
        pp[1] = sm[1];
        pp[2] = sm[2];
        pp[3] = 0;
    }
    if (!last_block(&a.st->ticket_aux, &flag)) return;
    objective_finish(a, scratch);
}

// ---------------- one iteration under alternative readings ----------------
// The fused step's arithmetic for volumes with SPG_READ_* flags, written
// plainly: one CTA per row segment of a z-plane; D^T(p) re-evaluates p at the
// voxel and its three neighbours; the objective at x_k is summed when the
// step records history. The last CTA writes the history entries, advances
// each volume's extrapolation index and the device state, as the fused
// kernel does, so the two paths are interchangeable between launches.
__global__ void generic_step_kernel(GenericParams g)
{
    __shared__ double scratch[32 * 4];
    __shared__ int flag, s_cur, s_rec, s_kr;
    __shared__ long long s_kt;
    if (threadIdx.x == 0) {
        volatile DevState *st = g.st;
        s_cur = st->cur;
        s_kr = st->k_round;
        s_kt = st->k_total;
        s_rec = (g.hist_every > 0 && (s_kt % g.hist_every) == 0) ? 1 : 0;
    }
    __syncthreads();
    const int cur = s_cur;
    const bool rec = s_rec != 0;
    const int nxt = g.xd ? (cur ^ 1) : (cur + 1) % 3;
    auto pick = [&](int i) { return i == 0 ? g.xbuf[0] : (i == 1 ? g.xbuf[1] : (i == 2 ? g.xbuf[2] : g.xbuf[3])); };
    const float *xk = pick(cur);
    const float *aux = pick(g.xd ? 2 + cur : (cur + 2) % 3);
    float *xout = pick(nxt);
    float *dout = g.xd ? pick(2 + nxt) : nullptr;

    const int plane = blockIdx.x / AUX_SEG;
    const int vol = g.plane_vol[plane];
    const VolDesc V = g.vols[vol];
    const int z = plane - V.plane_begin;
    int r0, r1;
    seg_rows(V.ny, blockIdx.x % AUX_SEG, r0, r1);
    const float beta = g.beta[V.kmom];
    const Field F{xk, g.xd ? nullptr : aux, beta, g.xd ? aux : nullptr};
    const Field X0{xk, nullptr, 0.f};
    const float tau = V.tau, tl1 = V.tau * V.lambda_l1, mu = V.mu;
    KSum kd, kl, kt;
    for (int t = threadIdx.x; t < (r1 - r0) * V.nx; t += blockDim.x) {
        const int x = t % V.nx, y = r0 + t / V.nx;
        const long long i = V.off + ((long long)z * V.ny + y) * V.pitch + x;
        const float xc = xk[i], dc = F.d(i), wv = g.w[i], o1 = g.om1[i];
        const float res = xc - g.b[i];
        const float gtot = fmaf(V.lambda_tv, div_at(V, F, g.omtv, x, y, z), wv * fmaf(beta, dc, res));
        const float delta = fmaf(beta, dc, -tau * gtot);
        const float zz = xc + delta;
        const float th = tl1 * o1;
        const float inc = fabsf(zz) < th ? -xc : delta - copysignf(th, zz);
        xout[i] = xc + inc;
        if (dout) dout[i] = inc;
        if (rec) {
            float gq[3];
            grad_at(V, X0, x, y, z, gq);
            const float q = gq[0] * gq[0] + gq[1] * gq[1] + gq[2] * gq[2];
            const float h = q <= mu * mu ? q * (0.5f / mu) : q * rsqrtf(q) - 0.5f * mu;
            kd.add(0.5f * wv * res * res);
            kl.add(o1 * fabsf(xc));
            kt.add(g.omtv[i] * h);
        }
    }
    if (rec) {
        double sm[3] = {kd.value(), kl.value(), kt.value()};
        block_sum<3>(sm, scratch);
        if (threadIdx.x == 0) {
            double *pp = g.plane_part + (long long)blockIdx.x * 4;
            pp[0] = sm[0];
            pp[1] = sm[1];
            pp[2] = sm[2];
        }
    }
    if (!last_block(&g.st->ticket, &flag)) return;
    const int hslot = g.st->hist_count % g.hist_cap;
    for (int v = 0; v < g.nvol; v++) {
        const VolDesc W = g.vols[v];
        if (rec) {
            double c3[3] = {0, 0, 0};
            for (int q = (W.plane_begin + W.halo_lo) * AUX_SEG + threadIdx.x; q < (W.plane_begin + W.nz - W.halo_hi) * AUX_SEG;
                 q += blockDim.x) {
                const double *pp = g.plane_part + (long long)q * 4;
                c3[0] += __ldcg(pp + 0);
                c3[1] += __ldcg(pp + 1);
                c3[2] += __ldcg(pp + 2);
            }
            block_sum<3>(c3, scratch);
            if (threadIdx.x == 0) {
                double *h = g.hist + ((long long)hslot * g.nvol + v) * 5;
                const double l1 = (double)W.lambda_l1 * c3[1], tv = (double)W.lambda_tv * c3[2];
                const double tot = c3[0] + l1 + tv;
                h[0] = (double)s_kt;
                h[1] = c3[0];
                h[2] = l1;
                h[3] = tv;
                h[4] = tot;
                if (!isfinite(tot)) atomicCAS(&g.st->err, 0, (int)SPG_ENONFINITE);
            }
        }
        if (threadIdx.x == 0) {
            g.vols[v].beta_last = g.beta[W.kmom];
            g.vols[v].kmom = W.kmom + 1;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        DevState *st = g.st;
        if (rec) st->hist_count = st->hist_count + 1;
        st->cur = nxt;
        st->k_round = s_kr + 1;
        st->k_total = s_kt + 1;
        st->ticket = 0;
        __threadfence();
    }
}

// ---------------- adjoint of one step ----------------
// Two passes, each a march over z (a CTA owns TY rows of a 128-voxel chunk
// of x over ZC planes, warp r row y0 + r, one more warp the row below the
// tile), 4 voxels per lane with 16-byte loads and x-neighbours by shuffle:
//   1. mask: p = omtv grad h_mu(D y) (Eq. 12, 16), tvg = D^T p (Eq. 17),
//      the step's z, the soft-threshold mask m = gnext [pass] (Eq. 21), the
//      l1 / TV scalar partials, gb += tau w m, gw += -tau (y - b) m;
//   2. apply: hq = omtv H_mu(D y) D m, H_mu = I/mu inside the smoothing ball
//      and (I - e e^T)/|D y| outside (the Hessian of Eq. 14);
//      ybar = m - tau (w m + lambda_tv D^T hq); gcur += (1+beta) ybar,
//      gprev += -beta ybar (gprev is written, not accumulated, when it has
//      no earlier contribution).
// Each step of the march evaluates p (hq) on the next plane once per voxel
// and keeps it in registers, where it is the forward z-neighbour now and the
// voxel's own value one step later; the y-component of the row below comes
// from the warp that owns that row through a 3-plane shared ring; the
// x-neighbour from the next lane (a chunk's last lane evaluates it). Only m
// is stored between the passes.
struct Lane4 {
    int x0, y, z, lane;
    bool act;
    long long i;  // element index of voxel x0 of the row
};

__device__ __forceinline__ float4 ldz4(const float *p, bool ok)
{
    return ok ? *reinterpret_cast<const float4 *>(p) : make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ void st4(float *p, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// f at x0-1 .. x0+2 (the backward x-neighbours of the lane's voxels), x0-1
// from the previous lane or, for a chunk's first lane, loaded; f(x0-1) := f(x0)
// at the volume's first column (zero difference).
__device__ __forceinline__ void left4(const float *f, const Lane4 &L, const float (&c)[4], float (&l)[4])
{
    float xl = __shfl_up_sync(FULL, c[3], 1);
    if (L.lane == 0) xl = (L.act && L.x0 >= 1) ? f[L.i - 1] : c[0];
    if (L.x0 == 0) xl = c[0];
    l[0] = xl;
    l[1] = c[0];
    l[2] = c[1];
    l[3] = c[2];
}

// f at x0+1 .. x0+4 (the forward x-neighbours), zero beyond the volume.
__device__ __forceinline__ void right4(const VolDesc &V, const float *f, const Lane4 &L, const float (&c)[4],
                                       float (&r)[4])
{
    float xr = __shfl_down_sync(FULL, c[0], 1);
    if (L.lane == 31) xr = (L.act && L.x0 + 4 < V.nx) ? f[L.i + 4] : 0.f;
    r[0] = c[1];
    r[1] = c[2];
    r[2] = c[3];
    r[3] = xr;
#pragma unroll
    for (int q = 0; q < 4; q++)
        if (L.x0 + q + 1 >= V.nx) r[q] = 0.f;
}

namespace adj {
constexpr int TY = 7;                  // output rows per CTA
constexpr int THREADS = 32 * (TY + 1); // warp TY: the row below the tile
constexpr int ZC = 8;                  // planes per CTA
}  // namespace adj

// f at the lane's voxels of the row whose voxel x0 is element i (zeros where
// `ok` is false) and at x0-1: from the lane before, loaded by a chunk's first
// lane, and the voxel's own value at the volume's first column (zero backward
// difference along x). Every lane of the warp calls it.
__device__ __forceinline__ void row4(const float *f, const Lane4 &L, long long i, bool ok, float (&c)[4], float &l)
{
    unpack4(ldz4(f + i, ok), c);
    l = __shfl_up_sync(FULL, c[3], 1);
    if (L.lane == 0) l = (ok && L.x0 >= 1) ? f[i - 1] : c[0];
    if (L.x0 == 0) l = c[0];
}

// f on the row whose voxel x0 is element i when `have`, else a copy of c
// (a missing backward neighbour: the voxel stands in for it).
__device__ __forceinline__ void row4_or(const float *f, long long i, bool have, bool ok, const float (&c)[4],
                                        float (&r)[4])
{
    if (have) {
        unpack4(ldz4(f + i, ok), r);
    } else {
#pragma unroll
        for (int q = 0; q < 4; q++) r[q] = c[q];
    }
}

// (D y)_a at the lane's 4 voxels (Eq. 12 on y = x_k + beta (x_k - x_{k-1})),
// differences of x_k and of d = x_k - x_{k-1} taken separately: xc, mc on
// the voxels' row (xl, ml at x0-1), xu, mu_ on the row below in y, xw, mw on
// the plane below.
__device__ __forceinline__ void dy4(const float (&xc)[4], const float (&mc)[4], float xl, float ml,
                                    const float (&xu)[4], const float (&mu_)[4], const float (&xw)[4],
                                    const float (&mw)[4], float beta, float (&g)[3][4])
{
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const float dc = xc[q] - mc[q];
        const float lx = q ? xc[q - 1] : xl, lm = q ? mc[q - 1] : ml;
        g[0][q] = (xc[q] - lx) + beta * (dc - (lx - lm));
        g[1][q] = (xc[q] - xu[q]) + beta * (dc - (xu[q] - mu_[q]));
        g[2][q] = (xc[q] - xw[q]) + beta * (dc - (xw[q] - mw[q]));
    }
}

// The same at one voxel: (xa, ma) there, (xl, ml) at x-1, (xu, mu_) at y-1,
// (xw, mw) at z-1.
__device__ __forceinline__ void dy1(float xa, float ma, float xl, float ml, float xu, float mu_, float xw, float mw,
                                    float beta, float (&g)[3])
{
    const float dc = xa - ma;
    g[0] = (xa - xl) + beta * (dc - (xl - ml));
    g[1] = (xa - xu) + beta * (dc - (xu - mu_));
    g[2] = (xa - xw) + beta * (dc - (xw - mw));
}

// omtv / max(mu, |g|): the factor by which omtv grad h_mu(g) (Eq. 16) scales g.
__device__ __forceinline__ float p_scale(float g0, float g1, float g2, float ot, float mu)
{
    const float s2 = g0 * g0 + g1 * g1 + g2 * g2;
    return ot * fminf(1.0f / mu, rsqrtf(s2));
}

// omtv H_mu(g) q at one voxel, H_mu the Hessian of the smoothed norm (Eq. 14):
// I/mu inside the ball |g| <= mu, (I - e e^T)/|g| with e = g/|g| outside.
__device__ __forceinline__ void hq1(float g0, float g1, float g2, float q0, float q1, float q2, float ot, float mu,
                                    float (&h)[3])
{
    const float s = sqrtf(g0 * g0 + g1 * g1 + g2 * g2);
    if (s <= mu) {
        const float c = ot / mu;
        h[0] = q0 * c;
        h[1] = q1 * c;
        h[2] = q2 * c;
    } else {
        const float inv = 1.0f / s;
        const float e0 = g0 * inv, e1 = g1 * inv, e2 = g2 * inv;
        const float eq = e0 * q0 + e1 * q1 + e2 * q2;
        const float c = ot * inv;
        h[0] = (q0 - e0 * eq) * c;
        h[1] = (q1 - e1 * eq) * c;
        h[2] = (q2 - e2 * eq) * c;
    }
}

// Where a thread of the two passes works: chunk of x, tile of rows, planes.
struct AdjPlace {
    Lane4 L;
    int r, z0, z1;
    bool row_in;   // the warp's row is inside the volume
    long long PS;  // plane stride
};

__device__ __forceinline__ AdjPlace adj_place(const VolDesc &V)
{
    AdjPlace P;
    const int nchunk = (V.nx + 127) / 128, ntile = (V.ny + adj::TY - 1) / adj::TY;
    int b = blockIdx.x;
    const int cx = b % nchunk;
    b /= nchunk;
    const int by = b % ntile, bz = b / ntile;
    P.r = threadIdx.x >> 5;
    P.L.lane = threadIdx.x & 31;
    P.L.x0 = cx * 128 + 4 * P.L.lane;
    P.L.y = by * adj::TY + P.r;
    P.row_in = P.L.y < V.ny;
    P.L.act = P.row_in && P.L.x0 < V.nx;
    P.z0 = bz * adj::ZC;
    P.z1 = min(V.nz, P.z0 + adj::ZC);
    P.PS = (long long)V.pitch * V.ny;
    return P;
}

// element index of voxel x0 of row (y, z); only formed for rows in the volume
__device__ __forceinline__ long long adj_row(const VolDesc &V, int x0, int y, int z)
{
    return V.off + ((long long)z * V.ny + y) * V.pitch + x0;
}

__global__ void __launch_bounds__(adj::THREADS) adjoint_mask_kernel(AdjParams a)
{
    __shared__ __align__(16) float ring[3][adj::TY + 1][128];  // p_y of the tile's rows and the row below it
    __shared__ double scratch[32 * 4];
    const VolDesc V = a.vols[0];
    AdjPlace P = adj_place(V);
    Lane4 &L = P.L;
    const float beta = a.beta, mu = V.mu;
    KSum k1, k2;
    // x_k, x_{k-1} on the warp's row of the current plane, and p there
    float xc[4], mc[4], xl, ml, pc[3][4];
    {
        const int z = P.z0;
        L.z = z;
        L.i = P.row_in ? adj_row(V, L.x0, L.y, z) : 0;
        float xu[4], mu_[4], xw[4], mw[4], ot[4], g[3][4];
        row4(a.xk, L, L.i, L.act, xc, xl);
        row4(a.xkm1, L, L.i, L.act, mc, ml);
        row4_or(a.xk, L.i - V.pitch, L.y >= 1, L.act, xc, xu);
        row4_or(a.xkm1, L.i - V.pitch, L.y >= 1, L.act, mc, mu_);
        row4_or(a.xk, L.i - P.PS, z >= 1, L.act, xc, xw);
        row4_or(a.xkm1, L.i - P.PS, z >= 1, L.act, mc, mw);
        unpack4(ldz4(a.omtv + L.i, L.act), ot);
        dy4(xc, mc, xl, ml, xu, mu_, xw, mw, beta, g);
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const bool valid = L.act && L.x0 + q < V.nx;
            const float sc = p_scale(g[0][q], g[1][q], g[2][q], ot[q], mu);
#pragma unroll
            for (int c = 0; c < 3; c++) pc[c][q] = valid ? g[c][q] * sc : 0.f;
        }
        *reinterpret_cast<float4 *>(&ring[z % 3][P.r][4 * L.lane]) = make_float4(pc[1][0], pc[1][1], pc[1][2], pc[1][3]);
    }
    for (int z = P.z0; z < P.z1; z++) {
        // p on the next plane (zero beyond the volume)
        const bool zn = z + 1 < V.nz;
        const bool okn = L.act && zn;
        const long long in_ = L.i + P.PS;
        float xn[4], mn[4], xnl, mnl, pn[3][4];
        {
            float xu[4], mu_[4], ot[4], g[3][4];
            row4(a.xk, L, in_, okn, xn, xnl);
            row4(a.xkm1, L, in_, okn, mn, mnl);
            row4_or(a.xk, in_ - V.pitch, L.y >= 1, okn, xn, xu);
            row4_or(a.xkm1, in_ - V.pitch, L.y >= 1, okn, mn, mu_);
            unpack4(ldz4(a.omtv + in_, okn), ot);
            dy4(xn, mn, xnl, mnl, xu, mu_, xc, mc, beta, g);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const bool valid = okn && L.x0 + q < V.nx;
                const float sc = p_scale(g[0][q], g[1][q], g[2][q], ot[q], mu);
#pragma unroll
                for (int c = 0; c < 3; c++) pn[c][q] = valid ? g[c][q] * sc : 0.f;
            }
            *reinterpret_cast<float4 *>(&ring[(z + 1) % 3][P.r][4 * L.lane]) =
                make_float4(pn[1][0], pn[1][1], pn[1][2], pn[1][3]);
        }
        __syncthreads();  // p_y of plane z of every row of the tile is in the ring
        // p_x at x+1: the next lane's first voxel; a chunk's last lane evaluates it
        float pxn = __shfl_down_sync(FULL, pc[0][0], 1);
        if (L.lane == 31) {
            pxn = 0.f;
            if (L.act && L.x0 + 4 < V.nx) {
                const long long j = L.i + 4;
                const float xa = a.xk[j], ma = a.xkm1[j];
                const float xau = L.y >= 1 ? a.xk[j - V.pitch] : xa, mau = L.y >= 1 ? a.xkm1[j - V.pitch] : ma;
                const float xaw = z >= 1 ? a.xk[j - P.PS] : xa, maw = z >= 1 ? a.xkm1[j - P.PS] : ma;
                float ga[3];
                dy1(xa, ma, xc[3], mc[3], xau, mau, xaw, maw, beta, ga);
                pxn = ga[0] * p_scale(ga[0], ga[1], ga[2], a.omtv[j], mu);
            }
        }
        if (P.r < adj::TY && P.row_in) {
            float px[4] = {pc[0][1], pc[0][2], pc[0][3], pxn};
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (L.x0 + q + 1 >= V.nx) px[q] = 0.f;
            const float4 pyv = *reinterpret_cast<const float4 *>(&ring[z % 3][P.r + 1][4 * L.lane]);
            const float py[4] = {pyv.x, pyv.y, pyv.z, pyv.w};  // zero when row y + 1 is outside
            float bv[4], wv[4], o1[4], gn[4], gb[4], gw[4], m[4];
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            unpack4(L.act ? ld4_data(a.b, a.bf16, L.i) : zero, bv);
            unpack4(L.act ? ld4_data(a.w, a.bf16, L.i) : zero, wv);
            unpack4(ldz4(a.om1 + L.i, L.act), o1);
            unpack4(ldz4(a.gnext + L.i, L.act), gn);
            unpack4(ldz4(a.gb + L.i, L.act), gb);
            unpack4(ldz4(a.gw + L.i, L.act), gw);
            float s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const bool valid = L.act && L.x0 + q < V.nx;
                const float d = xc[q] - mc[q];
                const float tvg = (pc[0][q] - px[q]) + (pc[1][q] - py[q]) + (pc[2][q] - pn[2][q]);
                const float g = wv[q] * ((xc[q] - bv[q]) + beta * d) + V.lambda_tv * tvg;
                const float delta = beta * d - V.tau * g;
                const float zz = xc[q] + delta;
                const float th = V.tau * V.lambda_l1 * o1[q];
                const bool pass = fabsf(zz) > th || th <= 0.f;
                m[q] = (valid && pass) ? gn[q] : 0.f;
                const float sg = zz > 0.f ? 1.f : (zz < 0.f ? -1.f : 0.f);
                s1 += -V.tau * o1[q] * sg * m[q];
                s2 += -V.tau * tvg * m[q];
                gb[q] += V.tau * wv[q] * m[q];
                gw[q] += -V.tau * ((xc[q] - bv[q]) + beta * d) * m[q];
            }
            if (L.act) {
                st4(a.m + L.i, m);
                st4(a.gb + L.i, gb);
                st4(a.gw + L.i, gw);
            }
            k1.add(s1);
            k2.add(s2);
        }
        // the next plane becomes the current one
#pragma unroll
        for (int q = 0; q < 4; q++) {
            xc[q] = xn[q];
            mc[q] = mn[q];
#pragma unroll
            for (int c = 0; c < 3; c++) pc[c][q] = pn[c][q];
        }
        xl = xnl;
        ml = mnl;
        L.i = in_;
    }
    double sm[2] = {k1.value(), k2.value()};
    block_sum<2>(sm, scratch);
    if (threadIdx.x == 0) {
        a.plane_part[(long long)blockIdx.x * 4 + 0] = sm[0];
        a.plane_part[(long long)blockIdx.x * 4 + 1] = sm[1];
    }
}

// hq at the lane's 4 voxels from D y and D m there (zero where !ok or beyond nx)
__device__ __forceinline__ void hq4(const float (&g)[3][4], const float (&qc)[4], float ql, const float (&qu)[4],
                                    const float (&qw)[4], const float (&ot)[4], float mu, bool ok, int x0, int nx,
                                    float (&h)[3][4])
{
#pragma unroll
    for (int q = 0; q < 4; q++) {
        float t[3];
        hq1(g[0][q], g[1][q], g[2][q], qc[q] - (q ? qc[q - 1] : ql), qc[q] - qu[q], qc[q] - qw[q], ot[q], mu, t);
        const bool valid = ok && x0 + q < nx;
#pragma unroll
        for (int c = 0; c < 3; c++) h[c][q] = valid ? t[c] : 0.f;
    }
}

__global__ void __launch_bounds__(adj::THREADS) adjoint_apply_kernel(AdjParams a)
{
    __shared__ __align__(16) float ring[3][adj::TY + 1][128];  // hq_y of the tile's rows and the row below it
    const VolDesc V = a.vols[0];
    AdjPlace P = adj_place(V);
    Lane4 &L = P.L;
    const float beta = a.beta, mu = V.mu;
    // x_k, x_{k-1} and m on the warp's row of the current plane, and hq there
    float xc[4], mc[4], qc[4], xl, ml, ql, hc[3][4];
    {
        const int z = P.z0;
        L.z = z;
        L.i = P.row_in ? adj_row(V, L.x0, L.y, z) : 0;
        float xu[4], mu_[4], qu[4], xw[4], mw[4], qw[4], ot[4], g[3][4];
        row4(a.xk, L, L.i, L.act, xc, xl);
        row4(a.xkm1, L, L.i, L.act, mc, ml);
        row4(a.m, L, L.i, L.act, qc, ql);
        row4_or(a.xk, L.i - V.pitch, L.y >= 1, L.act, xc, xu);
        row4_or(a.xkm1, L.i - V.pitch, L.y >= 1, L.act, mc, mu_);
        row4_or(a.m, L.i - V.pitch, L.y >= 1, L.act, qc, qu);
        row4_or(a.xk, L.i - P.PS, z >= 1, L.act, xc, xw);
        row4_or(a.xkm1, L.i - P.PS, z >= 1, L.act, mc, mw);
        row4_or(a.m, L.i - P.PS, z >= 1, L.act, qc, qw);
        unpack4(ldz4(a.omtv + L.i, L.act), ot);
        dy4(xc, mc, xl, ml, xu, mu_, xw, mw, beta, g);
        hq4(g, qc, ql, qu, qw, ot, mu, L.act, L.x0, V.nx, hc);
        *reinterpret_cast<float4 *>(&ring[z % 3][P.r][4 * L.lane]) = make_float4(hc[1][0], hc[1][1], hc[1][2], hc[1][3]);
    }
    for (int z = P.z0; z < P.z1; z++) {
        const bool zn = z + 1 < V.nz;
        const bool okn = L.act && zn;
        const long long in_ = L.i + P.PS;
        float xn[4], mn[4], qn[4], xnl, mnl, qnl, hn[3][4];
        {
            float xu[4], mu_[4], qu[4], ot[4], g[3][4];
            row4(a.xk, L, in_, okn, xn, xnl);
            row4(a.xkm1, L, in_, okn, mn, mnl);
            row4(a.m, L, in_, okn, qn, qnl);
            row4_or(a.xk, in_ - V.pitch, L.y >= 1, okn, xn, xu);
            row4_or(a.xkm1, in_ - V.pitch, L.y >= 1, okn, mn, mu_);
            row4_or(a.m, in_ - V.pitch, L.y >= 1, okn, qn, qu);
            unpack4(ldz4(a.omtv + in_, okn), ot);
            dy4(xn, mn, xnl, mnl, xu, mu_, xc, mc, beta, g);
            hq4(g, qn, qnl, qu, qc, ot, mu, okn, L.x0, V.nx, hn);
            *reinterpret_cast<float4 *>(&ring[(z + 1) % 3][P.r][4 * L.lane]) =
                make_float4(hn[1][0], hn[1][1], hn[1][2], hn[1][3]);
        }
        __syncthreads();  // hq_y of plane z of every row of the tile is in the ring
        // hq_x at x+1: the next lane's first voxel; a chunk's last lane evaluates it
        float hxn = __shfl_down_sync(FULL, hc[0][0], 1);
        if (L.lane == 31) {
            hxn = 0.f;
            if (L.act && L.x0 + 4 < V.nx) {
                const long long j = L.i + 4;
                const float xa = a.xk[j], ma = a.xkm1[j], qa = a.m[j];
                const bool u = L.y >= 1, w = z >= 1;
                const float xau = u ? a.xk[j - V.pitch] : xa, mau = u ? a.xkm1[j - V.pitch] : ma;
                const float qau = u ? a.m[j - V.pitch] : qa;
                const float xaw = w ? a.xk[j - P.PS] : xa, maw = w ? a.xkm1[j - P.PS] : ma;
                const float qaw = w ? a.m[j - P.PS] : qa;
                float ga[3], h[3];
                dy1(xa, ma, xc[3], mc[3], xau, mau, xaw, maw, beta, ga);
                hq1(ga[0], ga[1], ga[2], qa - qc[3], qa - qau, qa - qaw, a.omtv[j], mu, h);
                hxn = h[0];
            }
        }
        if (P.r < adj::TY && P.row_in) {
            float hx[4] = {hc[0][1], hc[0][2], hc[0][3], hxn};
#pragma unroll
            for (int q = 0; q < 4; q++)
                if (L.x0 + q + 1 >= V.nx) hx[q] = 0.f;
            const float4 hyv = *reinterpret_cast<const float4 *>(&ring[z % 3][P.r + 1][4 * L.lane]);
            const float hy[4] = {hyv.x, hyv.y, hyv.z, hyv.w};
            float wv[4], gc[4], gp[4] = {0.f, 0.f, 0.f, 0.f};
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            unpack4(L.act ? ld4_data(a.w, a.bf16, L.i) : zero, wv);
            unpack4(ldz4(a.gcur + L.i, L.act), gc);
            const bool alias = a.gprev == a.gcur;  // k = 0: x_{-1} = x_0
            if (!alias && !a.prev_fresh) unpack4(ldz4(a.gprev + L.i, L.act), gp);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const bool valid = L.act && L.x0 + q < V.nx;
                const float dtv = (hc[0][q] - hx[q]) + (hc[1][q] - hy[q]) + (hc[2][q] - hn[2][q]);
                const float ybar = valid ? qc[q] - V.tau * (wv[q] * qc[q] + V.lambda_tv * dtv) : 0.f;
                gc[q] += (1.f + beta) * ybar;
                if (alias) gc[q] += -beta * ybar;
                else if (a.prev_fresh) gp[q] = -beta * ybar;
                else gp[q] += -beta * ybar;
            }
            if (L.act) {
                st4(a.gcur + L.i, gc);
                if (!alias) st4(a.gprev + L.i, gp);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            xc[q] = xn[q];
            mc[q] = mn[q];
            qc[q] = qn[q];
#pragma unroll
            for (int c = 0; c < 3; c++) hc[c][q] = hn[c][q];
        }
        xl = xnl;
        ml = mnl;
        ql = qnl;
        L.i = in_;
    }
}

// closes the row walks of the certificate passes below
#define ADJ_WALK_END }

// ---------------- certificate, two row-vector passes ----------------
// Q = P(x+) - P(y) with P = omtv grad h_mu(D .), stored as 3 fields; then
// r = (y - x+)(1/tau - w) + lambda_tv D^T Q and the sum of r^2 (D^T is
// linear: D^T P(x+) - D^T P(y) = D^T Q), each P evaluated once per voxel.
// xbuf = {x_{k+1}, x_k, x_{k-1} or null, d_k or null}.
#define CERT_WALK_BEGIN                                                                  \
    const int plane_ = blockIdx.x / AUX_SEG;                                             \
    const VolDesc V = a.vols[a.plane_vol[plane_]];                                       \
    const int zz_ = plane_ - V.plane_begin;                                              \
    int r0, r1;                                                                          \
    seg_rows(V.ny, blockIdx.x % AUX_SEG, r0, r1);                                        \
    const int lane_ = threadIdx.x & 31, warp_ = threadIdx.x >> 5, nw_ = blockDim.x >> 5; \
    const int nchunk_ = (V.nx + 127) / 128;                                              \
    const long long PS = (long long)V.pitch * V.ny;                                      \
    for (int rc = warp_; rc < (r1 - r0) * nchunk_; rc += nw_) {                          \
        Lane4 L;                                                                         \
        L.y = r0 + rc / nchunk_;                                                         \
        L.z = zz_;                                                                       \
        L.x0 = (rc % nchunk_) * 128 + 4 * lane_;                                         \
        L.lane = lane_;                                                                  \
        L.act = L.x0 < V.nx;                                                             \
        L.i = V.off + ((long long)L.z * V.ny + L.y) * V.pitch + L.x0;

// D y at the lane's voxels, y = x + beta d with d = aux (increment storage)
// or x - aux; differences of x and of d are taken separately (Eq. 12).
__device__ __forceinline__ void grad4_y(const VolDesc &V, const float *x, const float *aux, bool xd, float beta,
                                        const Lane4 &L, long long PS, float (&g)[3][4])
{
    float xc[4], ac[4], xl[4], al[4], xu[4], au[4], xw[4], aw[4];
    unpack4(ldz4(x + L.i, L.act), xc);
    unpack4(ldz4(aux + L.i, L.act), ac);
    left4(x, L, xc, xl);
    left4(aux, L, ac, al);
    if (L.y >= 1) {
        unpack4(ldz4(x + L.i - V.pitch, L.act), xu);
        unpack4(ldz4(aux + L.i - V.pitch, L.act), au);
    } else {
#pragma unroll
        for (int q = 0; q < 4; q++) xu[q] = xc[q], au[q] = ac[q];
    }
    if (L.z >= 1) {
        unpack4(ldz4(x + L.i - PS, L.act), xw);
        unpack4(ldz4(aux + L.i - PS, L.act), aw);
    } else {
#pragma unroll
        for (int q = 0; q < 4; q++) xw[q] = xc[q], aw[q] = ac[q];
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const float dc = xd ? ac[q] : xc[q] - ac[q];
        const float dl = xd ? al[q] : xl[q] - al[q];
        const float du = xd ? au[q] : xu[q] - au[q];
        const float dw = xd ? aw[q] : xw[q] - aw[q];
        g[0][q] = (xc[q] - xl[q]) + beta * (dc - dl);
        g[1][q] = (xc[q] - xu[q]) + beta * (dc - du);
        g[2][q] = (xc[q] - xw[q]) + beta * (dc - dw);
    }
}

__global__ void certificate_q_kernel(AuxParams a, const float *xplus, const float *xk, const float *aux, int xd,
                                     const float *omtv, float *Q, long long S)
{
    CERT_WALK_BEGIN
    float gp[3][4], gy[3][4], ot[4], q3[3][4];
    grad4_y(V, xplus, xplus, false, 0.f, L, PS, gp);
    grad4_y(V, xk, aux, xd != 0, V.beta_last, L, PS, gy);
    unpack4(ldz4(omtv + L.i, L.act), ot);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const bool valid = L.act && L.x0 + q < V.nx;
        const float sp = ot[q] * fminf(1.0f / V.mu, rsqrtf(gp[0][q] * gp[0][q] + gp[1][q] * gp[1][q] + gp[2][q] * gp[2][q]));
        const float sy = ot[q] * fminf(1.0f / V.mu, rsqrtf(gy[0][q] * gy[0][q] + gy[1][q] * gy[1][q] + gy[2][q] * gy[2][q]));
#pragma unroll
        for (int c = 0; c < 3; c++) q3[c][q] = valid ? gp[c][q] * sp - gy[c][q] * sy : 0.f;
    }
    if (L.act) {
#pragma unroll
        for (int c = 0; c < 3; c++) st4(Q + c * S + L.i, q3[c]);
    }
    ADJ_WALK_END
}

__global__ void certificate_r_kernel(AuxParams a, const float *xplus, const float *xk, const float *aux, int xd,
                                     const void *w, bool bf16, const float *Q, long long S)
{
    __shared__ double scratch[32 * 4];
    __shared__ int flag;
    KSum ks;
    CERT_WALK_BEGIN
    float q0[4], q1[4], q2[4], qx[4], qy[4], qz[4], xp[4], xc[4], ac[4], wv[4];
    unpack4(ldz4(Q + L.i, L.act), q0);
    unpack4(ldz4(Q + S + L.i, L.act), q1);
    unpack4(ldz4(Q + 2 * S + L.i, L.act), q2);
    right4(V, Q, L, q0, qx);
    unpack4(ldz4(Q + S + L.i + V.pitch, L.act && L.y + 1 < V.ny), qy);
    unpack4(ldz4(Q + 2 * S + L.i + PS, L.act && L.z + 1 < V.nz), qz);
    unpack4(ldz4(xplus + L.i, L.act), xp);
    unpack4(ldz4(xk + L.i, L.act), xc);
    unpack4(ldz4(aux + L.i, L.act), ac);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    unpack4(L.act ? ld4_data(w, bf16, L.i) : zero, wv);
    const float beta = V.beta_last;  // extrapolation weight of the step that produced x+
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        if (!(L.act && L.x0 + q < V.nx)) continue;
        const float d = xd ? ac[q] : xc[q] - ac[q];
        const float dy = (xc[q] - xp[q]) + beta * d;
        const float dv = (q0[q] - qx[q]) + (q1[q] - qy[q]) + (q2[q] - qz[q]);
        const float r = dy * (1.0f / V.tau - wv[q]) + V.lambda_tv * dv;
        acc += r * r;
    }
    ks.add(acc);
    ADJ_WALK_END
    double sm[1] = {ks.value()};
    block_sum<1>(sm, scratch);
    if (threadIdx.x == 0) a.plane_part[(long long)blockIdx.x * 4] = sm[0];
    if (!last_block(&a.st->ticket_aux, &flag)) return;
    for (int v = 0; v < a.nvol; v++) {
        const VolDesc W = a.vols[v];
        double accv[1] = {0};
        for (int q = (W.plane_begin + W.halo_lo) * AUX_SEG + threadIdx.x; q < (W.plane_begin + W.nz - W.halo_hi) * AUX_SEG; q += blockDim.x)
            accv[0] += __ldcg(a.plane_part + (long long)q * 4);
        block_sum<1>(accv, scratch);
        if (threadIdx.x == 0) a.vol_out[(long long)v * 8 + 4] = accv[0];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.st->ticket_aux = 0;
        __threadfence();
    }
}

}  // namespace

cudaError_t launch_validate(const AuxParams &a, int vol, int nz, const void *b, const void *w, bool bf16,
                            double *maxw_out, cudaStream_t s)
{
    validate_kernel<<<nz * AUX_SEG, AUX_THREADS, 0, s>>>(a, vol, b, w, bf16, maxw_out);
    return cudaGetLastError();
}

cudaError_t launch_anchor(const AuxParams &a, int vol, int nz, void *b, void *w, bool bf16, const float *anchor,
                          float gamma, double *maxw_out, cudaStream_t s)
{
    anchor_kernel<<<nz * AUX_SEG, AUX_THREADS, 0, s>>>(a, vol, b, w, bf16, anchor, gamma, maxw_out);
    return cudaGetLastError();
}

cudaError_t launch_scales(const AuxParams &a, int vol, int nz, const void *b, const void *w, bool bf16,
                          cudaStream_t s)
{
    scales_kernel<<<nz * AUX_SEG, AUX_THREADS, 0, s>>>(a, vol, b, w, bf16);
    return cudaGetLastError();
}

// In-place reversal of every axis of one pitched volume: element (z, y, x)
// trades places with (nz-1-z, ny-1-y, nx-1-x). Element i of the unpadded
// order pairs with element nvox-1-i, so the first half of the order visits
// every pair once (the middle element of an odd volume stays); padding is
// not touched.
template <typename T>
__global__ void __launch_bounds__(256) reverse_axes_kernel(T *v, int nx, int ny, int pitch, long long nvox)
{
    const long long half = nvox / 2;
    const long long nxy = (long long)nx * ny;
    auto at = [&](long long i) {
        const long long z = i / nxy;
        const long long r = i - z * nxy;
        const long long y = r / nx;
        return (z * ny + y) * pitch + (r - y * nx);
    };
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < half;
         i += (long long)gridDim.x * blockDim.x) {
        const long long a = at(i), b = at(nvox - 1 - i);
        const T t = v[a];
        v[a] = v[b];
        v[b] = t;
    }
}

cudaError_t launch_reverse_axes(void *v, size_t es, int nx, int ny, int nz, int pitch, cudaStream_t s)
{
    const long long nvox = (long long)nx * ny * nz;
    const long long half = nvox / 2;
    if (half == 0) return cudaSuccess;
    const int grid = (int)std::min<long long>((half + 255) / 256, 4096);
    if (es == 4)
        reverse_axes_kernel<uint32_t><<<grid, 256, 0, s>>>(static_cast<uint32_t *>(v), nx, ny, pitch, nvox);
    else if (es == 2)
        reverse_axes_kernel<uint16_t><<<grid, 256, 0, s>>>(static_cast<uint16_t *>(v), nx, ny, pitch, nvox);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_convert_to_bf16(const float *src, uint16_t *dst, long long n, cudaStream_t s)
{
    to_bf16_kernel<<<1024, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_convert_to_f32(const uint16_t *src, float *dst, long long n, cudaStream_t s)
{
    to_f32_kernel<<<1024, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_reweight(const AuxParams &a, const float *const *xbuf, float *om1, float *omtv,
                            const double *maxw, double *rstats, VolDesc *vols_rw, cudaStream_t s)
{
    if (a.readings == 0)
        reweight4_kernel<<<a.nplanes * AUX_SEG, AUX_THREADS, 0, s>>>(a, xbuf[0], om1, omtv, maxw, rstats, vols_rw);
    else
        reweight_kernel<<<a.nplanes * AUX_SEG, AUX_THREADS, 0, s>>>(a, xbuf[0], om1, omtv, maxw, rstats, vols_rw);
    return cudaGetLastError();
}

cudaError_t launch_objective(const AuxParams &a, const float *const *xbuf, const void *b, const void *w,
                             bool bf16, const float *om1, const float *omtv, cudaStream_t s)
{
    if (a.readings == 0)
        objective4_kernel<<<a.nplanes * AUX_SEG, AUX_THREADS, 0, s>>>(a, xbuf[0], b, w, bf16, om1, omtv);
    else
        objective_kernel<<<a.nplanes * AUX_SEG, AUX_THREADS, 0, s>>>(a, xbuf[0], b, w, bf16, om1, omtv);
    return cudaGetLastError();
}

cudaError_t launch_certificate4(const AuxParams &a, const float *const *xbuf, const void *w, bool bf16,
                                const float *omtv, float *Q, long long stride, cudaStream_t s)
{
    const bool xd = xbuf[3] != nullptr;
    const float *aux = xd ? xbuf[3] : xbuf[2];
    certificate_q_kernel<<<a.nplanes * AUX_SEG, AUX_THREADS, 0, s>>>(a, xbuf[0], xbuf[1], aux, xd ? 1 : 0, omtv, Q,
                                                                     stride);
    certificate_r_kernel<<<a.nplanes * AUX_SEG, AUX_THREADS, 0, s>>>(a, xbuf[0], xbuf[1], aux, xd ? 1 : 0, w, bf16, Q,
                                                                     stride);
    return cudaGetLastError();
}

cudaError_t launch_generic_step(const GenericParams &g, cudaStream_t s)
{
    generic_step_kernel<<<g.nplanes * AUX_SEG, AUX_THREADS, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_mask(const AdjParams &a, cudaStream_t s)
{
    adjoint_mask_kernel<<<a.nblocks, adj::THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_apply(const AdjParams &a, cudaStream_t s)
{
    adjoint_apply_kernel<<<a.nblocks, adj::THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

int adjoint_blocks(int nx, int ny, int nz)
{
    return ((nx + 127) / 128) * ((ny + adj::TY - 1) / adj::TY) * ((nz + adj::ZC - 1) / adj::ZC);
}

}  // namespace spg
