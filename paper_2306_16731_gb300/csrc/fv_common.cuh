// fv_common.cuh -- small device utilities shared by the kernel translation
// units: patch lookup, per-precision dispatch, block reductions.
#pragma once

#include "fv_internal.h"
#include "fv_physics.cuh"

namespace fv {

enum { PREC_F64 = 0, PREC_F32 = 1, PREC_BF16 = 2 };

// Index i with off[i] <= x < off[i+1] (off has T+1 ascending entries).
__device__ __forceinline__ int find_patch(const int64_t *__restrict__ off, int T, int64_t x)
{
    int lo = 0, hi = T - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fv_max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide maximum of non-negative values; result valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_max_nonneg(T v, T *smem /* >= 32 entries */)
{
    v = warp_max(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) smem[w] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    if (w == 0) {
        T x = l < nw ? smem[l] : T(0);
        x = warp_max(x);
        if (l == 0) smem[0] = x;
    }
    __syncthreads();
    T r = smem[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_sum(double v, double *smem /* >= 32 entries */)
{
    v = warp_sum(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) smem[w] = v;
    __syncthreads();
    int nw = (blockDim.x + 31) >> 5;
    if (w == 0) {
        double x = l < nw ? smem[l] : 0.0;
        x = warp_sum(x);
        if (l == 0) smem[0] = x;
    }
    __syncthreads();
    double r = smem[0];
    __syncthreads();
    return r;
}

// double -> float, rounded to nearest even, on the integer units: GB300's
// FP64 unit, which also converts, is slow enough that a few conversions
// per work item queue behind one another.  Normal float results only;
// zero, subnormal, overflowing and non-finite inputs take the conversion
// instruction.
__device__ __forceinline__ float d2f_rn(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32);
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;      // float exponent field
    if (e < 1 || e > 254) return float(v);
    const unsigned long long m = b & 0xfffffffffffffull;            // 52 fraction bits
    const unsigned long long rest = m & ((1ull << 29) - 1);          // the 29 bits rounded away
    unsigned r = (unsigned)(m >> 29);
    r += (rest > (1ull << 28) || (rest == (1ull << 28) && (r & 1u))) ? 1u : 0u;
    // a carry out of the fraction moves into the exponent (and to infinity
    // above the largest float), as rounding to nearest requires
    return __uint_as_float((hi & 0x80000000u) | (((unsigned)e << 23) + r));
}

// CFL time step (dt = cfl h / (d lambda)), same association as the oracle.
__device__ __forceinline__ double cfl_dt(double cfl, double h, int dim, double lam)
{
    return (cfl * h) / (double(dim) * lam);
}

}  // namespace fv

// Dispatch a templated launcher body (the variadic argument) on (dim,
// storage type S); D is the dimension.
#define FV_DISPATCH(dim, prec, ...)                                           \
    do {                                                                       \
        if ((dim) == 2) {                                                      \
            constexpr int D = 2;                                               \
            if ((prec) == fv::PREC_F64) { using S = double; __VA_ARGS__; }            \
            else if ((prec) == fv::PREC_F32) { using S = float; __VA_ARGS__; }        \
            else { using S = __nv_bfloat16; __VA_ARGS__; }                            \
        } else {                                                               \
            constexpr int D = 3;                                               \
            if ((prec) == fv::PREC_F64) { using S = double; __VA_ARGS__; }            \
            else if ((prec) == fv::PREC_F32) { using S = float; __VA_ARGS__; }        \
            else { using S = __nv_bfloat16; __VA_ARGS__; }                            \
        }                                                                      \
    } while (0)
