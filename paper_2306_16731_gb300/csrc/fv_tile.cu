// fv_tile.cu -- the "patch-wise" realisation (arXiv:2306.16731, Sec. 3 Def.
// of the patch-wise realisation, Sec. 4 Alg. 2 and its idioms): one thread
// block per patch; the halo-inclusive patch is staged in shared memory, and
// block barriers separate the logical steps of Algorithm 1 (directional
// fluxes and eigenvalues, face fluxes, update, eigenvalue reduction).
// Instead of masking one thread per union-range index, every step loops its
// own range over the block's threads.
#include "fv_common.cuh"

namespace fv {

namespace {

// dt / (2h) in the compute type: in FP32 from the rounded operands (every
// thread forms it, and an FP64 division per warp queues on GB300's slow
// FP64 unit); in FP64 exactly.
template <typename C> __device__ __forceinline__ C tile_half_ratio(double dt, double h);
template <> __device__ __forceinline__ float tile_half_ratio<float>(double dt, double h)
{
    return __fdividef(float(dt), 2.0f * float(h));
}
template <> __device__ __forceinline__ double tile_half_ratio<double>(double dt, double h) { return dt / (2.0 * h); }


constexpr int kThreads = 256;
constexpr int kMaxPerThread = 8;              // interior volumes per thread
constexpr size_t kMaxSmem = 227 * 1024;

template <int D>
__device__ __forceinline__ int64_t interior_local(int j, int p)
{
    const int e = p + 2;
    int x = j % p, r = j / p;
    if (D == 2) return (int64_t)(r + 1) * e + (x + 1);
    int y = r % p, z = r / p;
    return ((int64_t)(z + 1) * e + (y + 1)) * e + (x + 1);
}

template <int D, typename S, typename C>
__global__ void __launch_bounds__(kThreads) k_tile(BatchView b, const S *__restrict__ q,
                                                   S *__restrict__ qout,
                                                   const double *__restrict__ dx,
                                                   const double *__restrict__ dt,
                                                   double *__restrict__ lambda_out,
                                                   double *__restrict__ dt_next_out, double cfl,
                                                   int cells_max)
{
    constexpr int N = D + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *Qs = reinterpret_cast<C *>(smem_raw);   // [cells][N] staged state
    C *Fs = Qs + (size_t)cells_max * N;         // [cells][N] F_n of the current direction
    C *Ls = Fs + (size_t)cells_max * N;         // [cells]    lambda_n of the current direction
    __shared__ C red[32];
    __shared__ C s_sc;                               // dt / (2h) of the patch
    const Gas<C> g{C(b.gamma), C(b.gamma - 1.0)};
    const bool periodic = b.halo_mode == 1;

    for (int i = blockIdx.x; i < b.num_patches; i += gridDim.x) {
        const int p = __ldg(b.psize + i);
        const int e = p + 2;
        const int cells = D == 2 ? e * e : e * e * e;
        const int nint = D == 2 ? p * p : p * p * p;
        const S *src = q + __ldg(b.elem_off + i);

        // Stage the patch (periodic halos wrap to the interior).
        for (int idx = threadIdx.x; idx < cells; idx += blockDim.x) {
            int x = idx % e - 1, r = idx / e;
            int y = (D == 2 ? r : r % e) - 1;
            int z = D == 2 ? 0 : r / e - 1;
            int64_t s = idx;
            if (periodic) {
                int xs = wrap(x, p), ys = wrap(y, p), zs = D == 2 ? 0 : wrap(z, p);
                s = D == 2 ? (int64_t)(ys + 1) * e + (xs + 1)
                           : ((int64_t)(zs + 1) * e + (ys + 1)) * e + (xs + 1);
            }
            C v[N];
            load_volume<N>(src + s * N, v);
#pragma unroll
            for (int k = 0; k < N; ++k) Qs[idx * N + k] = v[k];
        }
        // the step ratio from FP64 once per patch, not once per warp
        if (threadIdx.x == 0) s_sc = tile_half_ratio<C>(__ldg(dt + i), __ldg(dx + i));
        __syncthreads();

        C acc[kMaxPerThread][N];
#pragma unroll
        for (int m = 0; m < kMaxPerThread; ++m)
#pragma unroll
            for (int k = 0; k < N; ++k) acc[m][k] = C(0);

#pragma unroll
        for (int n = 0; n < D; ++n) {
            // Directional flux and eigenvalue over the face-halo range of n.
            for (int idx = threadIdx.x; idx < cells; idx += blockDim.x) {
                int x = idx % e - 1, r = idx / e;
                int y = (D == 2 ? r : r % e) - 1;
                int z = D == 2 ? 0 : r / e - 1;
                int c3[3] = {x, y, z};
                bool ok = true;
#pragma unroll
                for (int a = 0; a < D; ++a) {
                    int lo = a == n ? -1 : 0, hi = a == n ? p : p - 1;
                    ok = ok && c3[a] >= lo && c3[a] <= hi;
                }
                if (!ok) continue;
                C v[N], F[N];
#pragma unroll
                for (int k = 0; k < N; ++k) v[k] = Qs[idx * N + k];
                Prim<D, C> s = primitives<D>(v, g);
                flux<D>(v, s, n, F);
#pragma unroll
                for (int k = 0; k < N; ++k) Fs[idx * N + k] = F[k];
                Ls[idx] = eigenvalue<D>(s, n);
            }
            __syncthreads();
            // Face fluxes left and right of every interior volume.
            const int stride = n == 0 ? 1 : (n == 1 ? e : e * e);
#pragma unroll
            for (int m = 0; m < kMaxPerThread; ++m) {
                int j = threadIdx.x + m * blockDim.x;
                if (j >= nint) break;
                int c = (int)interior_local<D>(j, p);
                int cl = c - stride, cr = c + stride;
                C qc[N], ql[N], qr[N], fc[N], fl[N], fr[N], hl[N], hr[N];
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    qc[k] = Qs[c * N + k]; ql[k] = Qs[cl * N + k]; qr[k] = Qs[cr * N + k];
                    fc[k] = Fs[c * N + k]; fl[k] = Fs[cl * N + k]; fr[k] = Fs[cr * N + k];
                }
                rusanov2<N>(ql, qc, fl, fc, Ls[cl], Ls[c], hl);
                rusanov2<N>(qc, qr, fc, fr, Ls[c], Ls[cr], hr);
#pragma unroll
                for (int k = 0; k < N; ++k) acc[m][k] += hr[k] - hl[k];
            }
            __syncthreads();
        }

        // Update, store, eigenvalue of the new state.
        const double h = __ldg(dx + i);
        const C sc = s_sc;
        S *dst = qout + __ldg(b.elem_off + i);
        C lmax = C(0);
        bool bad = false;
#pragma unroll
        for (int m = 0; m < kMaxPerThread; ++m) {
            int j = threadIdx.x + m * blockDim.x;
            if (j >= nint) break;
            int c = (int)interior_local<D>(j, p);
            C v[N];
#pragma unroll
            for (int k = 0; k < N; ++k) v[k] = Qs[c * N + k] - sc * acc[m][k];
            store_volume<N>(dst + (int64_t)c * N, v);
            Prim<D, C> s = primitives<D>(v, g);
            C l = max_eigenvalue<D>(s);
            bad = bad || non_physical(v[0], s.p, l);
            lmax = fv_max(lmax, l);
        }
        if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(b.flags, FV_FLAG_NONPHYSICAL);
        if (lambda_out || dt_next_out) {
            lmax = block_max_nonneg(lmax, red);
            if (threadIdx.x == 0) {
                double l = double(lmax);
                if (lambda_out) lambda_out[i] = l;
                if (dt_next_out) dt_next_out[i] = cfl_dt(cfl, h, D, l);
            }
        }
        __syncthreads();
    }
}

size_t tile_smem(const BatchView &b, int precision)
{
    size_t cs = precision == PREC_F64 ? 8 : 4;
    size_t cells = (size_t)patch_cells(b.dim, b.max_p);
    size_t N = b.dim + 2;
    return cells * (2 * N + 1) * cs;
}

}  // namespace

bool tile_supported(const BatchView &b, int precision)
{
    int64_t nint = b.dim == 2 ? (int64_t)b.max_p * b.max_p : (int64_t)b.max_p * b.max_p * b.max_p;
    return nint <= (int64_t)kThreads * kMaxPerThread && tile_smem(b, precision) <= kMaxSmem;
}

cudaError_t launch_tile_update(const BatchView &b, int precision, const StepArgs &a,
                               cudaStream_t st)
{
    if (b.num_patches == 0) return cudaSuccess;
    const size_t smem = tile_smem(b, precision);
    const int cells_max = (int)patch_cells(b.dim, b.max_p);
    int grid = b.num_patches;
    cudaError_t err = cudaSuccess;
    FV_DISPATCH(b.dim, precision, {
        using C = typename StorageTraits<S>::Compute;
        auto kern = k_tile<D, S, C>;
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err == cudaSuccess) {
            kern<<<grid, kThreads, smem, st>>>(b, static_cast<const S *>(a.q_in),
                                               static_cast<S *>(a.q_out), a.dx, a.dt,
                                               a.lambda_out, a.dt_next_out, a.cfl, cells_max);
            err = cudaGetLastError();
        }
    });
    return err;
}

}  // namespace fv
