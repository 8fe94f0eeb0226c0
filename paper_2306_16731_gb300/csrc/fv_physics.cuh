// fv_physics.cuh -- device microkernels of the finite-volume patch update
// (arXiv:2306.16731, Sec. 2.2 Def. 1: flux, eigenvalue, face flux, update)
// and the storage <-> compute conversions of the state layout (Sec. 4,
// array of structures: the N = d+2 unknowns of a volume are contiguous).
//
// The Euler functions are the textbook ideal-gas system (the paper studies
// the compressible Euler equations, Sec. 5, without printing formulas):
//   u_k = (rho u_k) / rho,  p = (gamma-1) (E - 1/2 sum_k (rho u_k) u_k),
//   c = sqrt(gamma p / rho),  lambda_n = |u_n| + c,
//   F_n = (rho u_n, rho u_1 u_n + delta_1n p, .., rho u_d u_n + delta_dn p, (E+p) u_n).
// The Rusanov face flux (Eq. 2) is formed doubled,
//   2 Fhat = (F_L + F_R) - max(lambda_L, lambda_R) (Q_R - Q_L),
// and the update applies dt/(2h) to the flux difference, which equals
// dt/h applied to Fhat (halving is exact).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fv {

// ------------------------------------------------------------- storage types

template <typename S> struct StorageTraits;
template <> struct StorageTraits<double> { using Compute = double; };
template <> struct StorageTraits<float> { using Compute = float; };
template <> struct StorageTraits<__nv_bfloat16> { using Compute = float; };

__device__ __forceinline__ double to_compute(double v) { return v; }
__device__ __forceinline__ float to_compute(float v) { return v; }
__device__ __forceinline__ float to_compute(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename S> __device__ __forceinline__ S from_compute(double v);
template <> __device__ __forceinline__ double from_compute<double>(double v) { return v; }
template <typename S> __device__ __forceinline__ S from_compute(float v);
template <> __device__ __forceinline__ float from_compute<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_compute<__nv_bfloat16>(float v)
{
    return __float2bfloat16_rn(v);
}

// Load the N unknowns of one volume (element pointer) into compute type.
template <int N, typename S, typename C>
__device__ __forceinline__ void load_volume(const S *__restrict__ p, C (&q)[N])
{
#pragma unroll
    for (int k = 0; k < N; ++k) q[k] = to_compute(p[k]);
}

// 2D float volumes are one 16-byte vector.
template <>
__device__ __forceinline__ void load_volume<4, float, float>(const float *__restrict__ p, float (&q)[4])
{
    float4 v = *reinterpret_cast<const float4 *>(p);
    q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
}

// 2D double volumes are two 16-byte vectors.
template <>
__device__ __forceinline__ void load_volume<4, double, double>(const double *__restrict__ p, double (&q)[4])
{
    double2 a = reinterpret_cast<const double2 *>(p)[0];
    double2 b = reinterpret_cast<const double2 *>(p)[1];
    q[0] = a.x; q[1] = a.y; q[2] = b.x; q[3] = b.y;
}

// 2D bfloat16 volumes are one 8-byte vector.
template <>
__device__ __forceinline__ void load_volume<4, __nv_bfloat16, float>(const __nv_bfloat16 *__restrict__ p,
                                                                     float (&q)[4])
{
    uint2 v = *reinterpret_cast<const uint2 *>(p);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162 *>(&v.x);
    __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162 *>(&v.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    q[0] = fa.x; q[1] = fa.y; q[2] = fb.x; q[3] = fb.y;
}

template <int N, typename S, typename C>
__device__ __forceinline__ void store_volume(S *__restrict__ p, const C (&q)[N])
{
#pragma unroll
    for (int k = 0; k < N; ++k) p[k] = from_compute<S>(q[k]);
}

template <>
__device__ __forceinline__ void store_volume<4, float, float>(float *__restrict__ p, const float (&q)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(q[0], q[1], q[2], q[3]);
}

template <>
__device__ __forceinline__ void store_volume<4, double, double>(double *__restrict__ p, const double (&q)[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(q[0], q[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(q[2], q[3]);
}

template <>
__device__ __forceinline__ void store_volume<4, __nv_bfloat16, float>(__nv_bfloat16 *__restrict__ p,
                                                                      const float (&q)[4])
{
    __nv_bfloat162 a = __floats2bfloat162_rn(q[0], q[1]);
    __nv_bfloat162 b = __floats2bfloat162_rn(q[2], q[3]);
    uint2 v;
    v.x = *reinterpret_cast<uint32_t *>(&a);
    v.y = *reinterpret_cast<uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(p) = v;
}

// ------------------------------------------------------------ math helpers

__device__ __forceinline__ double fv_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float fv_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double fv_abs(double x) { return fabs(x); }
__device__ __forceinline__ float fv_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double fv_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float fv_max(float a, float b) { return fmaxf(a, b); }

// ------------------------------------------------------------- Euler physics

// Physical constants of the ideal gas in compute type.
template <typename C> struct Gas {
    C gamma;      // adiabatic index
    C gm1;        // gamma - 1
};

// Primitive quantities of one volume: velocity, pressure, sound speed.
template <int D, typename C>
struct Prim {
    C u[D];
    C p;
    C c;
};

template <int D, typename C>
__device__ __forceinline__ Prim<D, C> primitives(const C (&q)[D + 2], Gas<C> g)
{
    Prim<D, C> s;
    C rinv = C(1) / q[0];
    C kin = C(0);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        s.u[a] = q[1 + a] * rinv;
        kin += q[1 + a] * s.u[a];
    }
    s.p = g.gm1 * (q[D + 1] - C(0.5) * kin);
    s.c = fv_sqrt(g.gamma * s.p * rinv);
    return s;
}

// Largest eigenvalue along axis n: |u_n| + c.
template <int D, typename C>
__device__ __forceinline__ C eigenvalue(const Prim<D, C> &s, int n)
{
    return fv_abs(s.u[n]) + s.c;
}

// Largest eigenvalue over all directions: max_n |u_n| + c.
template <int D, typename C>
__device__ __forceinline__ C max_eigenvalue(const Prim<D, C> &s)
{
    C m = fv_abs(s.u[0]);
#pragma unroll
    for (int a = 1; a < D; ++a) m = fv_max(m, fv_abs(s.u[a]));
    return m + s.c;
}

// Physical flux along axis n.
template <int D, typename C>
__device__ __forceinline__ void flux(const C (&q)[D + 2], const Prim<D, C> &s, int n, C (&F)[D + 2])
{
    C un = s.u[n];
    F[0] = q[1 + n];
#pragma unroll
    for (int a = 0; a < D; ++a) F[1 + a] = q[1 + a] * un + (a == n ? s.p : C(0));
    F[D + 1] = (q[D + 1] + s.p) * un;
}

// Doubled Rusanov face flux (Eq. 2): 2 Fhat = (F_L + F_R) - max(lam_L, lam_R) (Q_R - Q_L).
template <int N, typename C>
__device__ __forceinline__ void rusanov2(const C (&qL)[N], const C (&qR)[N], const C (&FL)[N],
                                         const C (&FR)[N], C lamL, C lamR, C (&Fh)[N])
{
    C lam = fv_max(lamL, lamR);
#pragma unroll
    for (int k = 0; k < N; ++k) Fh[k] = (FL[k] + FR[k]) - lam * (qR[k] - qL[k]);
}

// ------------------------------------------- 2D FP32: one rounding per step
//
// The FP32 2D microkernels spell every operation out (round-to-nearest
// add/sub/mul/fma, the approximate reciprocal and square root of the
// fast-math FP32 build) in a fixed order: which multiplies and adds become
// one fma is then fixed by the source, not left to the compiler, so every
// 2D FP32 kernel rounds a volume's arithmetic at the same places.

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <>
__device__ __forceinline__ Prim<2, float> primitives<2, float>(const float (&q)[4], Gas<float> g)
{
    Prim<2, float> s;
    const float r = rcp_approx(q[0]);
    s.u[0] = __fmul_rn(q[1], r);
    s.u[1] = __fmul_rn(q[2], r);
    const float kin = __fmaf_rn(q[2], s.u[1], __fmul_rn(q[1], s.u[0]));
    s.p = __fmul_rn(g.gm1, __fmaf_rn(-0.5f, kin, q[3]));
    s.c = sqrt_approx(__fmul_rn(__fmul_rn(g.gamma, s.p), r));
    return s;
}

template <>
__device__ __forceinline__ float eigenvalue<2, float>(const Prim<2, float> &s, int n)
{
    return __fadd_rn(fabsf(s.u[n]), s.c);
}

template <>
__device__ __forceinline__ float max_eigenvalue<2, float>(const Prim<2, float> &s)
{
    return __fadd_rn(fmaxf(fabsf(s.u[0]), fabsf(s.u[1])), s.c);
}

template <>
__device__ __forceinline__ void flux<2, float>(const float (&q)[4], const Prim<2, float> &s, int n, float (&F)[4])
{
    const float un = s.u[n];
    F[0] = q[1 + n];
    F[1] = n == 0 ? __fmaf_rn(q[1], un, s.p) : __fmul_rn(q[1], un);
    F[2] = n == 1 ? __fmaf_rn(q[2], un, s.p) : __fmul_rn(q[2], un);
    F[3] = __fmul_rn(__fadd_rn(q[3], s.p), un);
}

template <>
__device__ __forceinline__ void rusanov2<4, float>(const float (&qL)[4], const float (&qR)[4], const float (&FL)[4],
                                                   const float (&FR)[4], float lamL, float lamR, float (&Fh)[4])
{
    const float nl = -fmaxf(lamL, lamR);
#pragma unroll
    for (int k = 0; k < 4; ++k) Fh[k] = __fmaf_rn(nl, __fsub_rn(qR[k], qL[k]), __fadd_rn(FL[k], FR[k]));
}

// 3D FP32, the same way: five unknowns (rho, rho u, rho v, rho w, E).
template <>
__device__ __forceinline__ Prim<3, float> primitives<3, float>(const float (&q)[5], Gas<float> g)
{
    Prim<3, float> s;
    const float r = rcp_approx(q[0]);
    s.u[0] = __fmul_rn(q[1], r);
    s.u[1] = __fmul_rn(q[2], r);
    s.u[2] = __fmul_rn(q[3], r);
    const float kin = __fmaf_rn(q[3], s.u[2], __fmaf_rn(q[2], s.u[1], __fmul_rn(q[1], s.u[0])));
    s.p = __fmul_rn(g.gm1, __fmaf_rn(-0.5f, kin, q[4]));
    s.c = sqrt_approx(__fmul_rn(__fmul_rn(g.gamma, s.p), r));
    return s;
}

template <>
__device__ __forceinline__ float eigenvalue<3, float>(const Prim<3, float> &s, int n)
{
    return __fadd_rn(fabsf(s.u[n]), s.c);
}

template <>
__device__ __forceinline__ float max_eigenvalue<3, float>(const Prim<3, float> &s)
{
    return __fadd_rn(fmaxf(fmaxf(fabsf(s.u[0]), fabsf(s.u[1])), fabsf(s.u[2])), s.c);
}

template <>
__device__ __forceinline__ void flux<3, float>(const float (&q)[5], const Prim<3, float> &s, int n, float (&F)[5])
{
    const float un = s.u[n];
    F[0] = q[1 + n];
#pragma unroll
    for (int a = 0; a < 3; ++a) F[1 + a] = a == n ? __fmaf_rn(q[1 + a], un, s.p) : __fmul_rn(q[1 + a], un);
    F[4] = __fmul_rn(__fadd_rn(q[4], s.p), un);
}

template <>
__device__ __forceinline__ void rusanov2<5, float>(const float (&qL)[5], const float (&qR)[5], const float (&FL)[5],
                                                   const float (&FR)[5], float lamL, float lamR, float (&Fh)[5])
{
    const float nl = -fmaxf(lamL, lamR);
#pragma unroll
    for (int k = 0; k < 5; ++k) Fh[k] = __fmaf_rn(nl, __fsub_rn(qR[k], qL[k]), __fadd_rn(FL[k], FR[k]));
}

// Update of one unknown from the doubled face fluxes: Q_new = Q - (dt/2h)
// (d + (2F_up - 2F_low)), d the difference of the other directions (x, or
// x then y), the last direction's difference formed first.
template <typename C>
__device__ __forceinline__ C update_dq(C q, C sc, C dfx, C fy_up, C fy_low)
{
    return q - sc * (dfx + (fy_up - fy_low));
}
template <>
__device__ __forceinline__ float update_dq<float>(float q, float sc, float dfx, float fy_up, float fy_low)
{
    return __fmaf_rn(-sc, __fadd_rn(dfx, __fsub_rn(fy_up, fy_low)), q);
}

// Non-physical state test used by the error flag: rho <= 0, p <= 0 or a
// non-finite eigenvalue (NaN compares false).
template <typename C>
__device__ __forceinline__ bool non_physical(C rho, C p, C lam)
{
    return !(rho > C(0)) || !(p > C(0)) || !(lam < C(INFINITY));
}

// --------------------------------------------------------- layout helpers

// Cells of a halo-inclusive patch.
__host__ __device__ __forceinline__ int64_t patch_cells(int dim, int p)
{
    int64_t e = p + 2;
    return dim == 2 ? e * e : e * e * e;
}

// Wrapped coordinate for periodic halos: -1 -> p-1, p -> 0.
__device__ __forceinline__ int wrap(int i, int p)
{
    return i < 0 ? i + p : (i >= p ? i - p : i);
}

// Error flag bits: a non-physical state; a bounded device wait that ran out.
enum : unsigned { FV_FLAG_NONPHYSICAL = 1u, FV_FLAG_TIMEOUT = 2u };

// Atomic maximum of a non-negative double via its bit pattern (ordered as
// a signed 64-bit integer for non-negative values).
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v)
{
    atomicMax(reinterpret_cast<long long *>(addr), __double_as_longlong(v));
}

}  // namespace fv
