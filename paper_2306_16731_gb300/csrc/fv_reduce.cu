// fv_reduce.cu -- per-patch reductions over the interior volumes of a state:
// the maximum eigenvalue that feeds the CFL condition (arXiv:2306.16731,
// Sec. 2.2 and Sec. 4 "Reduction"), the CFL time step, and double-precision
// conservation totals.  One warp group per patch; warp-shuffle maxima.
#include "fv_common.cuh"

namespace fv {

namespace {

constexpr int kThreads = 128;

template <int D>
__device__ __forceinline__ int64_t interior_local(int64_t j, int p)
{
    const int64_t e = p + 2;
    int64_t x = j % p, r = j / p;
    if (D == 2) return (r + 1) * e + (x + 1);
    int64_t y = r % p, z = r / p;
    return ((z + 1) * e + (y + 1)) * e + (x + 1);
}

template <int D, typename S, typename C>
__global__ void __launch_bounds__(kThreads) k_max_eigenvalue(BatchView b, const S *__restrict__ q,
                                                             double *__restrict__ lambda_out)
{
    constexpr int N = D + 2;
    __shared__ C red[32];
    const Gas<C> g{C(b.gamma), C(b.gamma - 1.0)};
    const int i = blockIdx.x;
    const int p = __ldg(b.psize + i);
    const int64_t nint = D == 2 ? (int64_t)p * p : (int64_t)p * p * p;
    const S *base = q + __ldg(b.elem_off + i);
    C m = C(0);
    bool bad = false;
    for (int64_t j = threadIdx.x; j < nint; j += blockDim.x) {
        C qv[N];
        load_volume<N>(base + interior_local<D>(j, p) * N, qv);
        Prim<D, C> s = primitives<D>(qv, g);
        C l = max_eigenvalue<D>(s);
        bad = bad || non_physical(qv[0], s.p, l);
        m = fv_max(m, l);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(b.flags, FV_FLAG_NONPHYSICAL);
    m = block_max_nonneg(m, red);
    if (threadIdx.x == 0) lambda_out[i] = double(m);
}

__global__ void k_cfl(int T, int dim, const double *__restrict__ lam, const double *__restrict__ dx,
                      double cfl, double *__restrict__ dt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < T) dt[i] = cfl_dt(cfl, dx[i], dim, lam[i]);
}

template <int D, typename S>
__global__ void __launch_bounds__(kThreads) k_totals(BatchView b, const S *__restrict__ q,
                                                     double *__restrict__ totals)
{
    constexpr int N = D + 2;
    __shared__ double red[32];
    const int i = blockIdx.x;
    const int p = __ldg(b.psize + i);
    const int64_t nint = D == 2 ? (int64_t)p * p : (int64_t)p * p * p;
    const S *base = q + __ldg(b.elem_off + i);
    double acc[N];
#pragma unroll
    for (int k = 0; k < N; ++k) acc[k] = 0.0;
    for (int64_t j = threadIdx.x; j < nint; j += blockDim.x) {
        const S *v = base + interior_local<D>(j, p) * N;
#pragma unroll
        for (int k = 0; k < N; ++k) acc[k] += double(to_compute(v[k]));
    }
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double t = block_sum(acc[k], red);
        if (threadIdx.x == 0) totals[(int64_t)i * N + k] = t;
    }
}

}  // namespace

cudaError_t launch_max_eigenvalue(const BatchView &b, int precision, const void *q,
                                  double *lambda_out, cudaStream_t st)
{
    if (b.num_patches == 0) return cudaSuccess;
    FV_DISPATCH(b.dim, precision, {
        using C = typename StorageTraits<S>::Compute;
        k_max_eigenvalue<D, S, C><<<b.num_patches, kThreads, 0, st>>>(b, static_cast<const S *>(q),
                                                                      lambda_out);
    });
    return cudaGetLastError();
}

cudaError_t launch_cfl_time_step(const BatchView &b, const double *lambda, const double *dx,
                                 double cfl, double *dt_out, cudaStream_t st)
{
    if (b.num_patches == 0) return cudaSuccess;
    int grid = (b.num_patches + 255) / 256;
    k_cfl<<<grid, 256, 0, st>>>(b.num_patches, b.dim, lambda, dx, cfl, dt_out);
    return cudaGetLastError();
}

cudaError_t launch_conserved_totals(const BatchView &b, int precision, const void *q,
                                    double *totals_out, cudaStream_t st)
{
    if (b.num_patches == 0) return cudaSuccess;
    FV_DISPATCH(b.dim, precision, {
        k_totals<D, S><<<b.num_patches, kThreads, 0, st>>>(b, static_cast<const S *>(q), totals_out);
    });
    return cudaGetLastError();
}

}  // namespace fv
