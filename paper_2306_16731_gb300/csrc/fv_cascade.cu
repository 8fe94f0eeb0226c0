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

// dt / (2h) in the compute type: in FP32 from the rounded operands (every
// thread forms it, and an FP64 division per warp queues on GB300's slow
// FP64 unit); in FP64 exactly.
template <typename C> __device__ __forceinline__ C cascade_half_ratio(double dt, double h);
template <> __device__ __forceinline__ float cascade_half_ratio<float>(double dt, double h)
{
    return __fdividef(float(dt), 2.0f * float(h));
}
template <> __device__ __forceinline__ double cascade_half_ratio<double>(double dt, double h) { return dt / (2.0 * h); }


constexpr int kThreads = 256;

// Layout of the per-face and per-volume vector temporaries (F_n and the face
// fluxes), the ablation of the paper's App. C: element (n, cell, k) of a
// batch with `total` cells (padded to a multiple of 32 in the scratch).
//   AoS   [n][cell][k]   the N unknowns of a volume contiguous
//   SoA   [n][k][cell]   one array per unknown
//   AoSoA [n][cell/32][k][cell%32]   blocks of 32 volumes, unknown-major
template <int L> struct Layout;
template <> struct Layout<CASCADE_AOS> {
    static __device__ __forceinline__ int64_t at(int n, int64_t cell, int k, int64_t total, int N)
    {
        return ((int64_t)n * total + cell) * N + k;
    }
};
template <> struct Layout<CASCADE_SOA> {
    static __device__ __forceinline__ int64_t at(int n, int64_t cell, int k, int64_t total, int N)
    {
        return ((int64_t)n * N + k) * total + cell;
    }
};
template <> struct Layout<CASCADE_AOSOA> {
    static __device__ __forceinline__ int64_t at(int n, int64_t cell, int k, int64_t total, int N)
    {
        return (((int64_t)n * (total >> 5) + (cell >> 5)) * N + k) * 32 + (cell & 31);
    }
};

// Cell range and direction of one launch: the whole batch and every axis for
// the batched realisation, one patch (and one axis for K1/K2) for the
// task-graph realisation.
struct Range {
    int64_t c0, c1;       // cells [c0, c1)
    int dir;              // axis, or -1 for all
};

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
template <int D, typename S, typename C, int L>
__global__ void __launch_bounds__(kThreads) k_flux(BatchView b, const S *__restrict__ q,
                                                   C *__restrict__ fbuf, C *__restrict__ lam, int64_t pad,
                                                   Range r)
{
    constexpr int N = D + 2;
    const Gas<C> g{C(b.gamma), C(b.gamma - 1.0)};
    for (int64_t cell = r.c0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < r.c1;
         cell += (int64_t)gridDim.x * blockDim.x) {
        CellPos c = decode<D>(b, cell);
        bool need[D];
        bool any = false;
#pragma unroll
        for (int n = 0; n < D; ++n) {
            bool ok = r.dir < 0 || r.dir == n;
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
#pragma unroll
            for (int k = 0; k < N; ++k) fbuf[Layout<L>::at(n, cell, k, pad, N)] = F[k];
            lam[(int64_t)n * pad + cell] = eigenvalue<D>(s, n);
        }
    }
}

// K2: Rusanov flux at the lower face (along n) of every volume whose
// coordinate along n is in [0, p] and elsewhere in [0, p-1].
template <int D, typename S, typename C, int L>
__global__ void __launch_bounds__(kThreads) k_face(BatchView b, const S *__restrict__ q,
                                                   const C *__restrict__ fbuf,
                                                   const C *__restrict__ lam,
                                                   C *__restrict__ face, int64_t pad, Range r)
{
    constexpr int N = D + 2;
    for (int64_t cell = r.c0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < r.c1;
         cell += (int64_t)gridDim.x * blockDim.x) {
        CellPos c = decode<D>(b, cell);
        const int64_t e = c.p + 2;
#pragma unroll
        for (int n = 0; n < D; ++n) {
            bool ok = r.dir < 0 || r.dir == n;
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
#pragma unroll
            for (int k = 0; k < N; ++k) {
                FL[k] = fbuf[Layout<L>::at(n, cl, k, pad, N)];
                FR[k] = fbuf[Layout<L>::at(n, cell, k, pad, N)];
            }
            rusanov2<N>(qL, qR, FL, FR, lam[(int64_t)n * pad + cl], lam[(int64_t)n * pad + cell], Fh);
#pragma unroll
            for (int k = 0; k < N; ++k) face[Layout<L>::at(n, cell, k, pad, N)] = Fh[k];
        }
    }
}

// K3: volume update of every interior volume.
template <int D, typename S, typename C, int L>
__global__ void __launch_bounds__(kThreads) k_update(BatchView b, const S *__restrict__ q,
                                                     S *__restrict__ qout,
                                                     const C *__restrict__ face,
                                                     const double *__restrict__ dx,
                                                     const double *__restrict__ dt, int64_t pad, Range r)
{
    constexpr int N = D + 2;
    for (int64_t cell = r.c0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < r.c1;
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
#pragma unroll
            for (int k = 0; k < N; ++k)
                acc[k] += face[Layout<L>::at(n, cell + stride, k, pad, N)] - face[Layout<L>::at(n, cell, k, pad, N)];
        }
        const double h = __ldg(dx + c.patch), tau = __ldg(dt + c.patch);
        const C s = cascade_half_ratio<C>(tau, h);
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
                                                     C *__restrict__ lam_new, Range r)
{
    constexpr int N = D + 2;
    const Gas<C> g{C(b.gamma), C(b.gamma - 1.0)};
    bool bad = false;
    for (int64_t cell = r.c0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < r.c1;
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
                                                     double *__restrict__ dt_next_out, int first_patch)
{
    __shared__ C red[32];
    const int i = first_patch + blockIdx.x;
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

// cells of the scratch arrays: the batch's cells rounded up to whole blocks
// of 32 (the AoSoA layout's block)
int64_t cascade_pad(const BatchView &b) { return (b.total_cells + 31) & ~int64_t(31); }

size_t cascade_scratch_bytes(const BatchView &b, int precision)
{
    size_t cs = precision == PREC_F64 ? 8 : 4;
    size_t N = b.dim + 2, M = (size_t)cascade_pad(b);
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
    size_t N = b.dim + 2, M = (size_t)cascade_pad(b);
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

template <int L>
cudaError_t launch_cascade_layout(const BatchView &b, int precision, const StepArgs &a, const CascadeScratch &s,
                                  cudaStream_t st)
{
    const int grid = grid_for(b.total_cells);
    const int64_t pad = cascade_pad(b);
    const Range all{0, b.total_cells, -1};
    FV_DISPATCH(b.dim, precision, {
        using C = typename StorageTraits<S>::Compute;
        const S *q = static_cast<const S *>(a.q_in);
        S *qo = static_cast<S *>(a.q_out);
        C *fl = static_cast<C *>(s.flux);
        C *lm = static_cast<C *>(s.lam);
        C *fc = static_cast<C *>(s.face);
        C *ln = static_cast<C *>(s.lam_new);
        k_flux<D, S, C, L><<<grid, kThreads, 0, st>>>(b, q, fl, lm, pad, all);
        k_face<D, S, C, L><<<grid, kThreads, 0, st>>>(b, q, fl, lm, fc, pad, all);
        k_update<D, S, C, L><<<grid, kThreads, 0, st>>>(b, q, qo, fc, a.dx, a.dt, pad, all);
        if (a.lambda_out || a.dt_next_out) {
            k_lambda<D, S, C><<<grid, kThreads, 0, st>>>(b, qo, ln, all);
            k_reduce<D, C><<<b.num_patches, kThreads, 0, st>>>(b, ln, a.dx, a.cfl, a.lambda_out,
                                                               a.dt_next_out, 0);
        }
    });
    return cudaGetLastError();
}

// One kernel node of the task graph.
cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t *node, const cudaGraphNode_t *deps, size_t ndeps, void *func,
                       int grid, void **args)
{
    cudaKernelNodeParams np{};
    np.func = func;
    np.gridDim = dim3((unsigned)grid);
    np.blockDim = dim3(kThreads);
    np.sharedMemBytes = 0;
    np.kernelParams = args;
    np.extra = nullptr;
    return cudaGraphAddKernelNode(node, g, deps, ndeps, &np);
}

// The paper's task-graph realisation (Sec. 3): per patch, one node per
// algorithmic step and axis, linked by their data dependencies only:
//   K1(n) -> K2(n) for every axis n (the axes run concurrently),
//   all K2(n) -> K3 -> K4 -> K5 (one block).
// Patches share no edge, so the graph exposes all patch-level parallelism;
// each node runs the batched realisation's kernel restricted to the
// patch's cells (and axis), so results are bitwise those of the batched form.
template <int L>
cudaError_t build_taskgraph_layout(const BatchView &bv, const int64_t *cell_off, int precision, const StepArgs &a,
                                   const CascadeScratch &sc, cudaGraph_t g)
{
    BatchView b = bv;
    int64_t pad = cascade_pad(b);
    const double *dx = a.dx, *dt = a.dt;
    double *lam_out = a.lambda_out, *dt_next = a.dt_next_out;
    double cfl = a.cfl;
    cudaError_t e = cudaSuccess;
    FV_DISPATCH(b.dim, precision, {
        using C = typename StorageTraits<S>::Compute;
        const S *q = static_cast<const S *>(a.q_in);
        S *qo = static_cast<S *>(a.q_out);
        C *fl = static_cast<C *>(sc.flux);
        C *lm = static_cast<C *>(sc.lam);
        C *fc = static_cast<C *>(sc.face);
        C *ln = static_cast<C *>(sc.lam_new);
        for (int i = 0; i < b.num_patches && e == cudaSuccess; ++i) {
            Range r{cell_off[i], cell_off[i + 1], -1};
            const int grid = (int)((r.c1 - r.c0 + kThreads - 1) / kThreads);
            cudaGraphNode_t faces[3];
            for (int n = 0; n < D && e == cudaSuccess; ++n) {
                Range rn{r.c0, r.c1, n};
                cudaGraphNode_t fnode;
                void *fargs[] = {&b, &q, &fl, &lm, &pad, &rn};
                e = add_kernel(g, &fnode, nullptr, 0, (void *)k_flux<D, S, C, L>, grid, fargs);
                if (e != cudaSuccess) break;
                void *cargs[] = {&b, &q, &fl, &lm, &fc, &pad, &rn};
                e = add_kernel(g, &faces[n], &fnode, 1, (void *)k_face<D, S, C, L>, grid, cargs);
            }
            if (e != cudaSuccess) break;
            cudaGraphNode_t un;
            void *uargs[] = {&b, &q, &qo, &fc, &dx, &dt, &pad, &r};
            e = add_kernel(g, &un, faces, D, (void *)k_update<D, S, C, L>, grid, uargs);
            if (e != cudaSuccess || !(lam_out || dt_next)) continue;
            cudaGraphNode_t ln_node, rd;
            void *largs[] = {&b, &qo, &ln, &r};
            e = add_kernel(g, &ln_node, &un, 1, (void *)k_lambda<D, S, C>, grid, largs);
            if (e != cudaSuccess) break;
            int first = i;
            void *rargs[] = {&b, &ln, &dx, &cfl, &lam_out, &dt_next, &first};
            e = add_kernel(g, &rd, &ln_node, 1, (void *)k_reduce<D, C>, 1, rargs);
        }
    });
    return e;
}

cudaError_t build_cascade_taskgraph(const BatchView &b, const int64_t *cell_off_host, int precision,
                                    const StepArgs &a, const CascadeScratch &s, int layout, cudaGraph_t g)
{
    switch (layout) {
    case CASCADE_SOA: return build_taskgraph_layout<CASCADE_SOA>(b, cell_off_host, precision, a, s, g);
    case CASCADE_AOSOA: return build_taskgraph_layout<CASCADE_AOSOA>(b, cell_off_host, precision, a, s, g);
    default: return build_taskgraph_layout<CASCADE_AOS>(b, cell_off_host, precision, a, s, g);
    }
}

cudaError_t launch_cascade_update(const BatchView &b, int precision, const StepArgs &a,
                                  const CascadeScratch &s, cudaStream_t st, int layout)
{
    switch (layout) {
    case CASCADE_SOA: return launch_cascade_layout<CASCADE_SOA>(b, precision, a, s, st);
    case CASCADE_AOSOA: return launch_cascade_layout<CASCADE_AOSOA>(b, precision, a, s, st);
    default: return launch_cascade_layout<CASCADE_AOS>(b, precision, a, s, st);
    }
}

}  // namespace fv
