// Building blocks of the own power-of-two FFTs (the z pass in spg_zfft.cu and
// the row pass in spg_xpass.cu): complex arithmetic, the 4- and 8-point DFTs
// of either sign, twiddle lookup in a table of w^m, w = e^(-2 pi i / n),
// computed on the host in double precision, and the shared-memory padding of
// the exchanges (one slot per 8).
#pragma once

#include <cuda_runtime.h>

namespace spg {
namespace fft {

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

__device__ __forceinline__ int padded(int z) { return z + (z >> 3); }

}  // namespace fft
}  // namespace spg
