// fv_cascade.cu -- the plain "batched" realisation (arXiv:2306.16731, Sec. 3
// Def. of the batched realisation, Sec. 4 "Kernels"): the steps of
// Algorithm 1 run one after the other, each as one launch over all volumes
// of all patches, with every intermediate in device memory:
//   K1 directional flux F_n and eigenvalue lambda_n of each volume in the
//      face-halo extended range (along n over [-1, p], elsewhere [0, p-1]);
//   K2 Rusanov flux (Eq. 2) at every face, stored at the face's upper volume;
//   K3 update Q_new = Q - dt/(2h) sum_n (2Fhat(c+1/2) - 2Fhat(c-1/2));
//   K4 max eigenvalue of every interior volume of the new state;
//   K5 per-patch maximum and CFL time step.
// Launch order on one stream gives the global synchronisation between
// steps that the paper realises with event waits.
#include "fv_common.cuh"

namespace fv {

namespace {

constexpr int kThreads = 256;

// Decoded halo-inclusive coordinates of a cell of the batch.
struct CellPos {
    int patch;
    int p;
    int x, y, z;          // each in [-1, p]
    int64_t local;        // cell index inside the patch
};

template <int D>
__device__ __forceinline__ CellPos decode(const BatchView &b, int64_t cell)
{
    CellPos c;
    c.patch = find_patch(b.cell_off, b.num_patches, cell);
    c.p = __ldg(b.psize + c.patch);
    c.local = cell - __ldg(b.cell_off + c.patch);
    int e = c.p + 2;
    int64_t r = c.local;
    c.x = int(r % e) - 1;
    r /= e;
    if (D == 2) {
        c.y = int(r) - 1;
        c.z = 0;
    } else {
        c.y = int(r % e) - 1;
        c.z = int(r / e) - 1;
    }
    return c;
}

template <int D>
__device__ __forceinline__ int coord(const CellPos &c, int a)
{
    return a == 0 ? c.x : (a == 1 ? c.y : c.z);
}

// Element pointer of the volume at (x, y, z) of a patch, wrapping the halo
// for periodic patches.
template <int D, typename S>
__device__ __forceinline__ const S *volume_ptr(const BatchView &b, const S *q, int patch, int p,
                                               int x, int y, int z)
{
    if (b.halo_mode == 1) {
        x = wrap(x, p);
        y = wrap(y, p);
        if (D == 3) z = wrap(z, p);
    }
    int64_t e = p + 2;
    int64_t local = D == 2 ? (int64_t)(y + 1) * e + (x + 1)
                           : ((int64_t)(z + 1) * e + (y + 1)) * e + (x + 1);
    return q + __ldg(b.elem_off + patch) + local * (D + 2);
}

// K1: directional fluxes and eigenvalues of every volume in a face-halo range.
template <int D, typename S, typename C>
__global__ void __launch_bounds__(kThreads) k_flux(BatchView b, const S *__restrict__ q,
                                                   C *__restrict__ fbuf, C *__restrict__ lam)
{
    constexpr int N = D + 2;
    const Gas<C> g{C(b.gamma), C(b.gamma - 1.0)};
    const int64_t total = b.total_cells;
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < total;
         cell += (int64_t)gridDim.x * blockDim.x) {
        CellPos c = decode<D>(b, cell);
        bool need[D];
        bool any = false;
#pragma unroll
        for (int n = 0; n < D; ++n) {
            bool ok = true;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                int v = coord<D>(c, a);
                int lo = a == n ? -1 : 0, hi = a == n ? c.p : c.p - 1;
                ok = ok && v >= lo && v <= hi;
            }
            need[n] = ok;
            any = any || ok;
        }
        if (!any) continue;
        C qv[N];
        load_volume<N>(volume_ptr<D>(b, q, c.patch, c.p, c.x, c.y, c.z), qv);
        Prim<D, C> s = primitives<D>(qv, g);
#pragma unroll
        for (int n = 0; n < D; ++n) {
            if (!need[n]) continue;
            C F[N];
            flux<D>(qv, s, n, F);
            C *dst = fbuf + ((int64_t)n * total + cell) * N;
#pragma unroll
            for (int k = 0; k < N; ++k) dst[k] = F[k];
            lam[(int64_t)n * total + cell] = eigenvalue<D>(s, n);
        }
    }
}

// K2: Rusanov flux at the lower face (along n) of every volume whose
// coordinate along n is in [0, p] and elsewhere in [0, p-1].
template <int D, typename S, typename C>
__global__ void __launch_bounds__(kThreads) k_face(BatchView b, const S *__restrict__ q,
                                                   const C *__restrict__ fbuf,
                                                   const C *__restrict__ lam,
                                                   C *__restrict__ face)
{
    constexpr int N = D + 2;
    const int64_t total = b.total_cells;
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < total;
         cell += (int64_t)gridDim.x * blockDim.x) {
        CellPos c = decode<D>(b, cell);
        const int64_t e = c.p + 2;
#pragma unroll
        for (int n = 0; n < D; ++n) {
            bool ok = true;
#pragma unroll
            for (int a = 0; a < D; ++a) {
                int v = coord<D>(c, a);
                int hi = a == n ? c.p : c.p - 1;
                ok = ok && v >= 0 && v <= hi;
            }
            if (!ok) continue;
            const int64_t stride = n == 0 ? 1 : (n == 1 ? e : e * e);
            const int64_t cl = cell - stride;
            int xl = c.x - (n == 0), yl = c.y - (n == 1), zl = c.z - (n == 2);
            C qL[N], qR[N], FL[N], FR[N], Fh[N];
            load_volume<N>(volume_ptr<D>(b, q, c.patch, c.p, xl, yl, zl), qL);
            load_volume<N>(volume_ptr<D>(b, q, c.patch, c.p, c.x, c.y, c.z), qR);
            const C *fl = fbuf + ((int64_t)n * total + cl) * N;
            const C *fr = fbuf + ((int64_t)n * total + cell) * N;
#pragma unroll
            for (int k = 0; k < N; ++k) { FL[k] = fl[k]; FR[k] = fr[k]; }
            rusanov2<N>(qL, qR, FL, FR, lam[(int64_t)n * total + cl], lam[(int64_t)n * total + cell], Fh);
            C *dst = face + ((int64_t)n * total + cell) * N;
#pragma unroll
            for (int k = 0; k < N; ++k) dst[k] = Fh[k];
        }
    }
}

// K3: volume update of every interior volume.
template <int D, typename S, typename C>
__global__ void __launch_bounds__(kThreads) k_update(BatchView b, const S *__restrict__ q,
                                                     S *__restrict__ qout,
                                                     const C *__restrict__ face,
                                                     const double *__restrict__ dx,
                                                     const double *__restrict__ dt)
{
    constexpr int N = D + 2;
    const int64_t total = b.total_cells;
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < total;
         cell += (int64_t)gridDim.x * blockDim.x) {
        CellPos c = decode<D>(b, cell);
        bool interior = c.x >= 0 && c.x < c.p && c.y >= 0 && c.y < c.p &&
                        (D == 2 || (c.z >= 0 && c.z < c.p));
        if (!interior) continue;
        const int64_t e = c.p + 2;
        C acc[N];
#pragma unroll
        for (int k = 0; k < N; ++k) acc[k] = C(0);
#pragma unroll
        for (int n = 0; n < D; ++n) {
            const int64_t stride = n == 0 ? 1 : (n == 1 ? e : e * e);
            const C *fl = face + ((int64_t)n * total + cell) * N;
            const C *fr = face + ((int64_t)n * total + cell + stride) * N;
#pragma unroll
            for (int k = 0; k < N; ++k) acc[k] += fr[k] - fl[k];
        }
        const double h = __ldg(dx + c.patch), tau = __ldg(dt + c.patch);
        const C s = C(tau / (2.0 * h));
        C qv[N];
        const int64_t eo = __ldg(b.elem_off + c.patch) + c.local * N;
        load_volume<N>(q + eo, qv);
#pragma unroll
        for (int k = 0; k < N; ++k) qv[k] = qv[k] - s * acc[k];
        store_volume<N>(qout + eo, qv);
    }
}

// K4: max eigenvalue of every interior volume of the new state.
template <int D, typename S, typename C>
__global__ void __launch_bounds__(kThreads) k_lambda(BatchView b, const S *__restrict__ q,
                                                     C *__restrict__ lam_new)
{
    constexpr int N = D + 2;
    const Gas<C> g{C(b.gamma), C(b.gamma - 1.0)};
    bool bad = false;
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < b.total_cells;
         cell += (int64_t)gridDim.x * blockDim.x) {
        CellPos c = decode<D>(b, cell);
        bool interior = c.x >= 0 && c.x < c.p && c.y >= 0 && c.y < c.p &&
                        (D == 2 || (c.z >= 0 && c.z < c.p));
        if (!interior) continue;
        C qv[N];
        load_volume<N>(q + __ldg(b.elem_off + c.patch) + c.local * N, qv);
        Prim<D, C> s = primitives<D>(qv, g);
        C l = max_eigenvalue<D>(s);
        bad = bad || non_physical(qv[0], s.p, l);
        lam_new[cell] = l;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(b.flags, FV_FLAG_NONPHYSICAL);
}

// K5: per-patch maximum and CFL time step (one block per patch).
template <int D, typename C>
__global__ void __launch_bounds__(kThreads) k_reduce(BatchView b, const C *__restrict__ lam_new,
                                                     const double *__restrict__ dx, double cfl,
                                                     double *__restrict__ lambda_out,
                                                     double *__restrict__ dt_next_out)
{
    __shared__ C red[32];
    const int i = blockIdx.x;
    const int p = __ldg(b.psize + i);
    const int64_t e = p + 2;
    const int64_t base = __ldg(b.cell_off + i);
    const int64_t nint = D == 2 ? (int64_t)p * p : (int64_t)p * p * p;
    C m = C(0);
    for (int64_t j = threadIdx.x; j < nint; j += blockDim.x) {
        int64_t x = j % p, r = j / p;
        int64_t y = D == 2 ? r : r % p;
        int64_t z = D == 2 ? 0 : r / p;
        int64_t local = D == 2 ? (y + 1) * e + (x + 1) : ((z + 1) * e + (y + 1)) * e + (x + 1);
        m = fv_max(m, lam_new[base + local]);
    }
    m = block_max_nonneg(m, red);
    if (threadIdx.x == 0) {
        double l = double(m);
        if (lambda_out) lambda_out[i] = l;
        if (dt_next_out) dt_next_out[i] = cfl_dt(cfl, __ldg(dx + i), D, l);
    }
}

int grid_for(int64_t work)
{
    int64_t blocks = (work + kThreads - 1) / kThreads;
    int64_t cap = (int64_t)num_sms() * 16;
    if (blocks > cap) blocks = cap;
    return int(blocks < 1 ? 1 : blocks);
}

}  // namespace

size_t cascade_scratch_bytes(const BatchView &b, int precision)
{
    size_t cs = precision == PREC_F64 ? 8 : 4;
    size_t N = b.dim + 2, M = (size_t)b.total_cells;
    size_t bytes = 0;
    bytes += (size_t)b.dim * M * N * cs;   // flux
    bytes += 256;
    bytes += (size_t)b.dim * M * cs;       // lam
    bytes += 256;
    bytes += (size_t)b.dim * M * N * cs;   // face
    bytes += 256;
    bytes += M * cs;                       // lam_new
    return bytes + 256;
}

void cascade_scratch_carve(void *base, const BatchView &b, int precision, CascadeScratch *s)
{
    size_t cs = precision == PREC_F64 ? 8 : 4;
    size_t N = b.dim + 2, M = (size_t)b.total_cells;
    auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
    char *p = static_cast<char *>(base);
    s->flux = p;
    p += align((size_t)b.dim * M * N * cs);
    s->lam = p;
    p += align((size_t)b.dim * M * cs);
    s->face = p;
    p += align((size_t)b.dim * M * N * cs);
    s->lam_new = p;
}

cudaError_t launch_cascade_update(const BatchView &b, int precision, const StepArgs &a,
                                  const CascadeScratch &s, cudaStream_t st)
{
    const int grid = grid_for(b.total_cells);
    FV_DISPATCH(b.dim, precision, {
        using C = typename StorageTraits<S>::Compute;
        const S *q = static_cast<const S *>(a.q_in);
        S *qo = static_cast<S *>(a.q_out);
        C *fl = static_cast<C *>(s.flux);
        C *lm = static_cast<C *>(s.lam);
        C *fc = static_cast<C *>(s.face);
        C *ln = static_cast<C *>(s.lam_new);
        k_flux<D, S, C><<<grid, kThreads, 0, st>>>(b, q, fl, lm);
        k_face<D, S, C><<<grid, kThreads, 0, st>>>(b, q, fl, lm, fc);
        k_update<D, S, C><<<grid, kThreads, 0, st>>>(b, q, qo, fc, a.dx, a.dt);
        if (a.lambda_out || a.dt_next_out) {
            k_lambda<D, S, C><<<grid, kThreads, 0, st>>>(b, qo, ln);
            k_reduce<D, C><<<b.num_patches, kThreads, 0, st>>>(b, ln, a.dx, a.cfl, a.lambda_out,
                                                               a.dt_next_out);
        }
    });
    return cudaGetLastError();
}

}  // namespace fv
