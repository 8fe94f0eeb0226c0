// fv_pair.cuh -- arithmetic on pairs of volumes held by one lane (two
// adjacent rows of a plane), for the FP32 fused 3D kernels: every step on
// the pair is one f32x2 instruction (fma/add/mul .f32x2 of sm_100 and
// later), which halves the issue cost of the flux, face and update
// arithmetic.  Ideal-gas Euler in three dimensions, five unknowns
// (rho, rho u, rho v, rho w, E); the textbook formulas of fv_physics.cuh.
#pragma once

#include <cuda_runtime.h>

namespace fv {
namespace pair {

constexpr int kN = 5;


// Packed (f32x2) or per-component arithmetic on volume pairs; both round
// every operation to nearest once, so they give identical bits.
template <bool Packed> struct Arith;
template <> struct Arith<true> {
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
};
template <> struct Arith<false> {
    static __device__ __forceinline__ float2 add(float2 a, float2 b)
    {
        return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
    }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b)
    {
        return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
    }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c)
    {
        return make_float2(__fmaf_rn(a.x, b.x, c.x), __fmaf_rn(a.y, b.y, c.y));
    }
};

__device__ __forceinline__ float2 bcast(float s) { return make_float2(s, s); }

// shuffle of a packed pair as one 64-bit value (the halves land in a
// register pair, ready for the f32x2 instructions)
__device__ __forceinline__ float2 shfl2(float2 v, int src)
{
    unsigned long long u = (unsigned long long)__float_as_uint(v.x) | ((unsigned long long)__float_as_uint(v.y) << 32);
    u = __shfl_sync(0xffffffffu, u, src);
    return make_float2(__uint_as_float((unsigned)u), __uint_as_float((unsigned)(u >> 32)));
}
__device__ __forceinline__ float2 abs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 max2(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }

// a - b, exactly rounded once (b * -1 is exact)
template <bool Pk>
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    return Arith<Pk>::fma(b, bcast(-1.0f), a);
}

// Primitive quantities of a volume pair (textbook ideal-gas Euler, as in
// fv_physics.cuh): velocities, pressure, sound speed and E + p.
struct Prim2 {
    float2 u[3];
    float2 p, c, ep;
};

template <bool Pk>
__device__ __forceinline__ Prim2 prim2(const float2 (&q)[kN], float2 g, float2 gm1)
{
    using A = Arith<Pk>;
    Prim2 s;
    const float2 rinv = make_float2(1.0f / q[0].x, 1.0f / q[0].y);
    s.u[0] = A::mul(q[1], rinv);
    s.u[1] = A::mul(q[2], rinv);
    s.u[2] = A::mul(q[3], rinv);
    const float2 kin = A::fma(q[3], s.u[2], A::fma(q[2], s.u[1], A::mul(q[1], s.u[0])));
    s.p = A::mul(gm1, A::fma(bcast(-0.5f), kin, q[4]));
    const float2 cs = A::mul(A::mul(g, s.p), rinv);
    s.c = make_float2(sqrtf(cs.x), sqrtf(cs.y));
    s.ep = A::add(q[4], s.p);
    return s;
}

// Physical flux along axis n; F[0] (= q[1+n]) is filled too.
template <int n, bool Pk>
__device__ __forceinline__ void flux2(const float2 (&q)[kN], const Prim2 &s, float2 (&F)[kN])
{
    using A = Arith<Pk>;
    const float2 un = s.u[n];
    F[0] = q[1 + n];
#pragma unroll
    for (int a = 0; a < 3; ++a) F[1 + a] = a == n ? A::fma(q[1 + a], un, s.p) : A::mul(q[1 + a], un);
    F[4] = A::mul(s.ep, un);
}

template <bool Pk>
__device__ __forceinline__ float2 lam2(float2 un, float2 c)
{
    return Arith<Pk>::add(abs2(un), c);
}

// Doubled Rusanov face flux (Eq. 2) of two faces at once:
// 2 Fhat = (F_L + F_R) - max(lam_L, lam_R) (Q_R - Q_L).
template <bool Pk>
__device__ __forceinline__ void face2(const float2 (&qL)[kN], const float2 (&qR)[kN], const float2 (&FL)[kN],
                                      const float2 (&FR)[kN], float2 lL, float2 lR, float2 (&Fh)[kN])
{
    using A = Arith<Pk>;
    const float2 nl = make_float2(-fmaxf(lL.x, lR.x), -fmaxf(lL.y, lR.y));
#pragma unroll
    for (int k = 0; k < kN; ++k) Fh[k] = A::fma(nl, sub2<Pk>(qR[k], qL[k]), A::add(FL[k], FR[k]));
}

}  // namespace pair
}  // namespace fv
