// fv_pde.cu -- the generic first-order hyperbolic PDE of Eq. 1 (arXiv:2306.16731,
// Sec. 2: dQ/dt + div F(Q) + sum_n B_n(Q) dQ/dx_n = S(Q)) on the patch-wise
// realisation: one thread block per patch, the halo-inclusive patch staged
// in shared memory.  The PDE enters through a device functor with the
// microkernels of Sec. 2.2 Def. 1 -- flux, eigenvalue -- plus the
// non-conservative product and the source:
//   struct Phys {
//     static constexpr int N;    // unknowns per volume
//     static constexpr int NV;   // the first NV are evolved, the rest are parameters
//     flux(q, n, F); lambda(q, n); ncp(qL, qR, n, D) = B_n(Qbar)(qR - qL);
//     source(q, S); bad(q, lambda);
//   };
// Discretisation (readings R13-R15): at each face the Rusanov flux of Eq. 2
// on the evolved unknowns and the product D = B_n((Q_L+Q_R)/2)(Q_R - Q_L),
// half of it to each side; per interior volume
//   acc = sum_n ((Fhat_r - Fhat_l) + 1/2 (D_r + D_l)),
//   Q_new = Q - (dt/h) acc + dt S(Q)   (evolved unknowns; parameters copied).
// The functor here is the 2D shallow water system over a bathymetry with a
// Coriolis force, Q = (h, hu, hv, b).
#include "fv_common.cuh"

namespace fv {

namespace {

constexpr int kThreads = 256;
constexpr size_t kMaxSmem = 227 * 1024;

// Shallow water: F_x = (hu, hu u + g h^2/2, hv u, 0), F_y = (hv, hu v,
// hv v + g h^2/2, 0); B_x dQ/dx = (0, g h db/dx, 0, 0), B_y likewise in the
// hv row; S = (0, f hv, -f hu, 0); lambda_n = |u_n| + sqrt(g h).
template <typename C> struct ShallowWater {
    static constexpr int N = 4;
    static constexpr int NV = 3;
    C g, f;

    __device__ __forceinline__ void flux(const C (&q)[N], int n, C (&F)[N]) const
    {
        const C h = q[0], un = q[1 + n] / h, pg = C(0.5) * g * h * h;
        F[0] = q[1 + n];
        F[1] = q[1] * un + (n == 0 ? pg : C(0));
        F[2] = q[2] * un + (n == 1 ? pg : C(0));
        F[3] = C(0);
    }
    __device__ __forceinline__ C lambda(const C (&q)[N], int n) const
    {
        return fv_abs(q[1 + n] / q[0]) + fv_sqrt(g * q[0]);
    }
    __device__ __forceinline__ void ncp(const C (&qL)[N], const C (&qR)[N], int n, C (&D)[N]) const
    {
        const C gh = g * (C(0.5) * (qL[0] + qR[0])) * (qR[3] - qL[3]);
        D[0] = C(0);
        D[1] = n == 0 ? gh : C(0);
        D[2] = n == 1 ? gh : C(0);
        D[3] = C(0);
    }
    __device__ __forceinline__ void source(const C (&q)[N], C (&S)[N]) const
    {
        S[0] = C(0);
        S[1] = f * q[2];
        S[2] = -f * q[1];
        S[3] = C(0);
    }
    __device__ __forceinline__ bool bad(const C (&q)[N], C lam) const
    {
        return !(q[0] > C(0)) || !(lam < C(INFINITY));
    }
};

// Rusanov flux (Eq. 2, doubled) on the evolved unknowns of one face.
template <class P, typename C>
__device__ __forceinline__ void face2(const P &ph, const C (&qL)[P::N], const C (&qR)[P::N], int n,
                                      C (&Fh)[P::N])
{
    C FL[P::N], FR[P::N];
    ph.flux(qL, n, FL);
    ph.flux(qR, n, FR);
    const C lam = fv_max(ph.lambda(qL, n), ph.lambda(qR, n));
#pragma unroll
    for (int k = 0; k < P::N; ++k) Fh[k] = k < P::NV ? (FL[k] + FR[k]) - lam * (qR[k] - qL[k]) : C(0);
}

// dt / h in the compute type: in FP32 from the rounded operands (every
// thread forms it, and GB300's FP64 unit would queue 8 warps' FP64
// divisions per patch); in FP64 exactly.
template <typename C> __device__ __forceinline__ C step_ratio(double tau, double h);
template <> __device__ __forceinline__ float step_ratio<float>(double tau, double h)
{
    return __fdividef(float(tau), float(h));
}
template <> __device__ __forceinline__ double step_ratio<double>(double tau, double h) { return tau / h; }

template <class P, typename S, typename C>
__global__ void __launch_bounds__(kThreads) k_tile_pde(BatchView b, P ph, const S *__restrict__ q,
                                                       S *__restrict__ qout, const double *__restrict__ dx,
                                                       const double *__restrict__ dt, double *__restrict__ lambda_out,
                                                       double *__restrict__ dt_next_out, double cfl)
{
    constexpr int N = P::N;
    extern __shared__ __align__(16) unsigned char smem_pde[];
    C *Qs = reinterpret_cast<C *>(smem_pde);        // [cells][N]
    __shared__ C red[32];
    const bool periodic = b.halo_mode == 1;

    for (int i = blockIdx.x; i < b.num_patches; i += gridDim.x) {
        const int p = __ldg(b.psize + i), e = p + 2, cells = e * e, nint = p * p;
        const S *src = q + __ldg(b.elem_off + i);
        for (int idx = threadIdx.x; idx < cells; idx += blockDim.x) {
            int x = idx % e - 1, y = idx / e - 1;
            int64_t s = idx;
            if (periodic) s = (int64_t)(wrap(y, p) + 1) * e + (wrap(x, p) + 1);
#pragma unroll
            for (int k = 0; k < N; ++k) Qs[idx * N + k] = to_compute(src[s * N + k]);
        }
        __syncthreads();

        const double h = __ldg(dx + i), tau = __ldg(dt + i);
        const C scale = step_ratio<C>(tau, h), ct = C(tau);
        S *dst = qout + __ldg(b.elem_off + i);
        C lmax = C(0);
        bool bad = false;
        for (int j = threadIdx.x; j < nint; j += blockDim.x) {
            const int x = j % p, y = j / p, c = (y + 1) * e + (x + 1);
            C qc[N], acc[N];
#pragma unroll
            for (int k = 0; k < N; ++k) { qc[k] = Qs[c * N + k]; acc[k] = C(0); }
#pragma unroll
            for (int n = 0; n < 2; ++n) {
                const int st = n == 0 ? 1 : e;
                C ql[N], qr[N], Fl[N], Fr[N], Dl[N], Dr[N];
#pragma unroll
                for (int k = 0; k < N; ++k) { ql[k] = Qs[(c - st) * N + k]; qr[k] = Qs[(c + st) * N + k]; }
                face2<P, C>(ph, ql, qc, n, Fl);
                face2<P, C>(ph, qc, qr, n, Fr);
                ph.ncp(ql, qc, n, Dl);
                ph.ncp(qc, qr, n, Dr);
                // doubled face fluxes: (2Fr - 2Fl)/2 + (Dr + Dl)/2
#pragma unroll
                for (int k = 0; k < N; ++k) acc[k] += C(0.5) * ((Fr[k] - Fl[k]) + (Dr[k] + Dl[k]));
            }
            C Sv[N], qn[N];
            ph.source(qc, Sv);
#pragma unroll
            for (int k = 0; k < N; ++k) qn[k] = k < P::NV ? (qc[k] - scale * acc[k]) + ct * Sv[k] : qc[k];
#pragma unroll
            for (int k = 0; k < N; ++k) dst[(int64_t)c * N + k] = from_compute<S>(qn[k]);
            const C l = fv_max(ph.lambda(qn, 0), ph.lambda(qn, 1));
            bad = bad || ph.bad(qn, l);
            lmax = fv_max(lmax, l);
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(b.flags, FV_FLAG_NONPHYSICAL);
        if (lambda_out || dt_next_out) {
            lmax = block_max_nonneg(lmax, red);
            if (threadIdx.x == 0) {
                const double l = double(lmax);
                if (lambda_out) lambda_out[i] = l;
                if (dt_next_out) dt_next_out[i] = cfl_dt(cfl, h, 2, l);
            }
        }
        __syncthreads();
    }
}

template <class P, typename S, typename C>
__global__ void __launch_bounds__(kThreads) k_pde_max_eigenvalue(BatchView b, P ph, const S *__restrict__ q,
                                                                 double *__restrict__ lambda_out)
{
    constexpr int N = P::N;
    __shared__ C red[32];
    for (int i = blockIdx.x; i < b.num_patches; i += gridDim.x) {
        const int p = __ldg(b.psize + i), e = p + 2;
        const S *src = q + __ldg(b.elem_off + i);
        C lmax = C(0);
        bool bad = false;
        for (int j = threadIdx.x; j < p * p; j += blockDim.x) {
            const int c = (j / p + 1) * e + (j % p + 1);
            C v[N];
#pragma unroll
            for (int k = 0; k < N; ++k) v[k] = to_compute(src[(int64_t)c * N + k]);
            const C l = fv_max(ph.lambda(v, 0), ph.lambda(v, 1));
            bad = bad || ph.bad(v, l);
            lmax = fv_max(lmax, l);
        }
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(b.flags, FV_FLAG_NONPHYSICAL);
        lmax = block_max_nonneg(lmax, red);
        if (threadIdx.x == 0) lambda_out[i] = double(lmax);
        __syncthreads();
    }
}

size_t pde_smem(const BatchView &b, int precision)
{
    return (size_t)(b.max_p + 2) * (b.max_p + 2) * 4 * (precision == PREC_F64 ? 8 : 4);
}

template <typename S>
cudaError_t launch_swe(const BatchView &b, int precision, const StepArgs *a, double *lambda_only, const void *q,
                       cudaStream_t st)
{
    using C = typename StorageTraits<S>::Compute;
    ShallowWater<C> ph{C(b.pde_param[0]), C(b.pde_param[1])};
    const int grid = b.num_patches;
    if (a) {
        const size_t smem = pde_smem(b, precision);
        auto kern = k_tile_pde<ShallowWater<C>, S, C>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<grid, kThreads, smem, st>>>(b, ph, static_cast<const S *>(a->q_in), static_cast<S *>(a->q_out),
                                           a->dx, a->dt, a->lambda_out, a->dt_next_out, a->cfl);
    } else {
        k_pde_max_eigenvalue<ShallowWater<C>, S, C><<<grid, kThreads, 0, st>>>(b, ph, static_cast<const S *>(q),
                                                                              lambda_only);
    }
    return cudaGetLastError();
}

}  // namespace

bool pde_tile_supported(const BatchView &b, int precision)
{
    return b.pde == PDE_SHALLOW_WATER && b.dim == 2 && precision != PREC_BF16 && pde_smem(b, precision) <= kMaxSmem;
}

cudaError_t launch_pde_update(const BatchView &b, int precision, const StepArgs &a, cudaStream_t st)
{
    if (b.num_patches == 0) return cudaSuccess;
    if (precision == PREC_F64) return launch_swe<double>(b, precision, &a, nullptr, nullptr, st);
    return launch_swe<float>(b, precision, &a, nullptr, nullptr, st);
}

cudaError_t launch_pde_max_eigenvalue(const BatchView &b, int precision, const void *q, double *lambda_out,
                                      cudaStream_t st)
{
    if (b.num_patches == 0) return cudaSuccess;
    if (precision == PREC_F64) return launch_swe<double>(b, precision, nullptr, lambda_out, q, st);
    return launch_swe<float>(b, precision, nullptr, lambda_out, q, st);
}

}  // namespace fv
