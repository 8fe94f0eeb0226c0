// fv_sweep.cu -- the fused form: one launch per time step in which every warp
// owns whole patches and sweeps them row by row, keeping all fluxes and
// eigenvalues on chip (arXiv:2306.16731: Algorithm 1's steps for one patch,
// Sec. 2.2 Eq. 2 face fluxes, Sec. 4 per-patch eigenvalue reduction).
//
// 2D mapping.  A warp takes one work item: up to 32/p patches of edge p
// (lanes sub*p .. sub*p+p-1 hold the p columns x of patch slot sub).  Each
// lane walks its column from the lower halo row y = -1 to the upper halo
// row y = p:
//   * the state of row y+1 .. y+PF is loaded ahead into registers (coalesced
//     rows: consecutive lanes read consecutive volumes);
//   * per volume: primitives, F_x, F_y, lambda_x, lambda_y (once each);
//   * y faces: the previous row's F_y, lambda_y and Q stay in registers, so
//     the face below row y is formed without any exchange;
//   * x faces: the right neighbour's Q, F_x, lambda_x arrive by one warp
//     shuffle; the left face is the left lane's right face (one shuffle);
//   * the two faces on the patch's x boundary of every row (which need the
//     x-halo volumes) are computed before the sweep by all 32 lanes packed
//     together and kept in shared memory;
//   * row y-1 is finished once the face above it (computed at row y) is
//     known: Q_new = Q - dt/(2h) ((2Fx_r - 2Fx_l) + (2Fy_r - 2Fy_l)),
//     the oracle's order; its max eigenvalue joins the lane's running max.
// The per-patch maximum is reduced through shared memory, and the CFL time
// step of the next step is written by one lane per patch.
//
// Scheduling.  Work items (equal-size patch groups, largest first) are
// either mapped one per warp (grid covers all items) or taken from a device
// counter by persistent warps; the last warp to finish resets the counter,
// so a launch needs no separate reset and stays graph-capturable.
// No block-wide barrier is used: warps are independent.
#include "fv_common.cuh"

namespace fv {

namespace {

constexpr int kMaxWarpsPerBlock = 16;
constexpr int kPF = 2;   // rows loaded ahead of the row being computed

struct SweepParams {
    BatchView b;
    const void *q_in;
    void *q_out;
    const double *dx;
    const double *dt;
    double *lambda_out;
    double *dt_next_out;
    double cfl;
    const WorkItem *items;
    const int32_t *order;
    int num_items;
    unsigned *counter;      // [0] = next item, [1] = finished warps
    int persistent;
};

template <typename C>
__host__ __device__ constexpr int warp_smem_bytes2d()
{
    return (64 * 4 + 32) * (int)sizeof(C);
}

template <int N, typename C>
__device__ __forceinline__ void shfl_down_vec(const C (&v)[N], C (&o)[N])
{
#pragma unroll
    for (int k = 0; k < N; ++k) o[k] = __shfl_down_sync(0xffffffffu, v[k], 1);
}

// x-direction physics of one volume: F_x and lambda_x.
template <typename C>
__device__ __forceinline__ void xphys(const C (&q)[4], Gas<C> g, C (&F)[4], C &lam)
{
    Prim<2, C> s = primitives<2>(q, g);
    flux<2>(q, s, 0, F);
    lam = eigenvalue<2>(s, 0);
}

// y-direction physics of one volume: F_y and lambda_y.
template <typename C>
__device__ __forceinline__ void yphys(const C (&q)[4], Gas<C> g, C (&F)[4], C &lam)
{
    Prim<2, C> s = primitives<2>(q, g);
    flux<2>(q, s, 1, F);
    lam = eigenvalue<2>(s, 1);
}

template <typename S, typename C>
__device__ __forceinline__ void sweep2d_item(const SweepParams sp, const WorkItem it, int lane,
                                             C *__restrict__ bface, C *__restrict__ red,
                                             bool &bad)
{
    constexpr int N = 4;
    const Gas<C> g{C(sp.b.gamma), C(sp.b.gamma - 1.0)};
    const S *__restrict__ q = static_cast<const S *>(sp.q_in);
    S *__restrict__ qo = static_cast<S *>(sp.q_out);
    const int P = it.p, cnt = it.count;
    const int E = P + 2;
    const bool periodic = sp.b.halo_mode == 1;

    // ---- boundary x faces of every row, packed over the warp
    const int nf = 2 * P * cnt;
    for (int f = lane; f < nf; f += 32) {
        const int fs = f / (2 * P);
        const int r = f - fs * 2 * P;
        const int yy = r >> 1, side = r & 1;
        const int ip = __ldg(sp.order + it.first_patch + fs);
        const S *ps = q + __ldg(sp.b.elem_off + ip);
        int xl = side ? P - 1 : -1, xr = side ? P : 0;
        if (periodic) { xl = wrap(xl, P); xr = wrap(xr, P); }
        C qL[N], qR[N], FL[N], FR[N], Fh[N], lL, lR;
        load_volume<N>(ps + ((int64_t)(yy + 1) * E + (xl + 1)) * N, qL);
        load_volume<N>(ps + ((int64_t)(yy + 1) * E + (xr + 1)) * N, qR);
        xphys(qL, g, FL, lL);
        xphys(qR, g, FR, lR);
        rusanov2<N>(qL, qR, FL, FR, lL, lR, Fh);
        C *dstf = bface + ((fs * P + yy) * 2 + side) * N;
#pragma unroll
        for (int k = 0; k < N; ++k) dstf[k] = Fh[k];
    }
    __syncwarp();

    // ---- lane -> (patch slot, column)
    const int sub = lane / P;
    const int x = lane - sub * P;
    const bool active = sub < cnt;
    const int slot = active ? sub : 0;
    const int i = __ldg(sp.order + it.first_patch + slot);
    const int64_t base = __ldg(sp.b.elem_off + i);
    const S *src = q + base + (int64_t)(x + 1) * N;
    S *dst = qo + base + (int64_t)(x + 1) * N;
    const int64_t RS = (int64_t)E * N;               // row stride in elements
    const double h = __ldg(sp.dx + i);
    const C sc = C(__ldg(sp.dt + i) / (2.0 * h));
    const C *bf = bface + (slot * P) * 2 * N;

    C q0[N], q1[N], q2[N];
    load_volume<N>(src + (int64_t)((periodic ? wrap(-1, P) : (-1)) + 1) * RS, q0);
    load_volume<N>(src + (int64_t)((periodic ? wrap(0, P) : (0)) + 1) * RS, q1);
    load_volume<N>(src + (int64_t)((periodic ? wrap(1, P) : (1)) + 1) * RS, q2);          // row 1 <= P always exists (P >= 1)

    // lower halo row: F_y and lambda_y only
    C qp[N], Fyp[N], lyp;
    yphys(q0, g, Fyp, lyp);
#pragma unroll
    for (int k = 0; k < N; ++k) { qp[k] = q0[k]; q0[k] = q1[k]; q1[k] = q2[k]; }
    if (2 <= P) load_volume<N>(src + (int64_t)((periodic ? wrap(2, P) : (2)) + 1) * RS, q2);

    C dxp[N], Fylp[N];
    C lmax = C(0);
    for (int y = 0; y < P; ++y) {
        // physics of row y
        Prim<2, C> s = primitives<2>(q0, g);
        C Fx[N], Fy[N];
        flux<2>(q0, s, 0, Fx);
        flux<2>(q0, s, 1, Fy);
        const C lx = eigenvalue<2>(s, 0), ly = eigenvalue<2>(s, 1);

        // y face below row y
        C Fyl[N];
        rusanov2<N>(qp, q0, Fyp, Fy, lyp, ly, Fyl);

        // finish row y-1 now that its upper face is known
        if (y > 0) {
            C qn[N];
#pragma unroll
            for (int k = 0; k < N; ++k) qn[k] = qp[k] - sc * (dxp[k] + (Fyl[k] - Fylp[k]));
            if (active) store_volume<N>(dst + (int64_t)y * RS, qn);      // row y-1 lives at y
            Prim<2, C> t = primitives<2>(qn, g);
            const C l = max_eigenvalue<2>(t);
            bad = bad || non_physical(qn[0], t.p, l);
            lmax = fv_max(lmax, l);
        }

        // x faces of row y
        C qr[N], Fr_[N], Fr[N], Fl[N];
        shfl_down_vec<N>(q0, qr);
        shfl_down_vec<N>(Fx, Fr_);
        const C lr = __shfl_down_sync(0xffffffffu, lx, 1);
        rusanov2<N>(q0, qr, Fx, Fr_, lx, lr, Fr);
        if (x == P - 1) {
#pragma unroll
            for (int k = 0; k < N; ++k) Fr[k] = bf[(y * 2 + 1) * N + k];
        }
#pragma unroll
        for (int k = 0; k < N; ++k) Fl[k] = __shfl_up_sync(0xffffffffu, Fr[k], 1);
        if (x == 0) {
#pragma unroll
            for (int k = 0; k < N; ++k) Fl[k] = bf[(y * 2) * N + k];
        }

        // carry row y to the next iteration
#pragma unroll
        for (int k = 0; k < N; ++k) {
            dxp[k] = Fr[k] - Fl[k];
            Fylp[k] = Fyl[k];
            qp[k] = q0[k];
            Fyp[k] = Fy[k];
            q0[k] = q1[k];
            q1[k] = q2[k];
        }
        lyp = ly;
        if (y + 3 <= P) load_volume<N>(src + (int64_t)((periodic ? wrap(y + 3, P) : (y + 3)) + 1) * RS, q2);
    }

    // upper halo row: its y face closes row P-1
    {
        C Fy[N], ly, Fyu[N];
        yphys(q0, g, Fy, ly);
        rusanov2<N>(qp, q0, Fyp, Fy, lyp, ly, Fyu);
        C qn[N];
#pragma unroll
        for (int k = 0; k < N; ++k) qn[k] = qp[k] - sc * (dxp[k] + (Fyu[k] - Fylp[k]));
        if (active) store_volume<N>(dst + (int64_t)P * RS, qn);
        Prim<2, C> t = primitives<2>(qn, g);
        const C l = max_eigenvalue<2>(t);
        bad = bad || non_physical(qn[0], t.p, l);
        lmax = fv_max(lmax, l);
    }

    // per-patch maximum eigenvalue and next time step
    red[lane] = lmax;
    __syncwarp();
    if (active && x == 0 && (sp.lambda_out || sp.dt_next_out)) {
        C m = red[lane];
        for (int j = 1; j < P; ++j) m = fv_max(m, red[lane + j]);
        const double l = double(m);
        if (sp.lambda_out) sp.lambda_out[i] = l;
        if (sp.dt_next_out) sp.dt_next_out[i] = cfl_dt(sp.cfl, h, 2, l);
    }
    __syncwarp();
}

template <typename S>
__global__ void __launch_bounds__(kMaxWarpsPerBlock * 32, 1) k_sweep2d(SweepParams sp)
{
    using C = typename StorageTraits<S>::Compute;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C *bface = reinterpret_cast<C *>(smem_raw + warp * warp_smem_bytes2d<C>());
    C *red = bface + 64 * 4;
    bool bad = false;
    const int wpb = blockDim.x >> 5;
    if (!sp.persistent) {
        const int item = blockIdx.x * wpb + warp;
        if (item < sp.num_items) sweep2d_item<S, C>(sp, sp.items[item], lane, bface, red, bad);
    } else {
        for (;;) {
            int item = 0;
            if (lane == 0) item = (int)atomicAdd(sp.counter, 1u);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item >= sp.num_items) break;
            sweep2d_item<S, C>(sp, sp.items[item], lane, bface, red, bad);
        }
        // the last warp to finish resets the counters for the next launch
        if (lane == 0) {
            __threadfence();
            const unsigned total = gridDim.x * (unsigned)wpb;
            if (atomicAdd(sp.counter + 1, 1u) == total - 1) {
                sp.counter[0] = 0;
                sp.counter[1] = 0;
                __threadfence();
            }
        }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(sp.b.flags, FV_FLAG_NONPHYSICAL);
}

}  // namespace

bool fused_supported(const BatchView &b, int precision, int *kernel)
{
    (void)precision;
    *kernel = FUSED_NONE;
    if (b.num_patches <= 0) return false;
    if (b.dim == 2 && b.max_p <= 32) {
        *kernel = FUSED_SWEEP2D;
        return true;
    }
    return false;
}

int fused_items_for(int dim, int p, int *patches_per_item)
{
    *patches_per_item = (dim == 2 && p <= 32) ? 32 / p : 1;
    return *patches_per_item;
}

cudaError_t launch_fused_update(const BatchView &b, int precision, const StepArgs &a,
                                const FusedPlan &plan, cudaStream_t st)
{
    if (plan.kernel != FUSED_SWEEP2D) return cudaErrorNotSupported;
    SweepParams sp;
    sp.b = b;
    sp.q_in = a.q_in;
    sp.q_out = a.q_out;
    sp.dx = a.dx;
    sp.dt = a.dt;
    sp.lambda_out = a.lambda_out;
    sp.dt_next_out = a.dt_next_out;
    sp.cfl = a.cfl;
    sp.items = plan.items;
    sp.order = plan.order;
    sp.num_items = plan.num_items;
    sp.counter = plan.work_counter;
    int wpb = plan.shape.warps_per_block;
    if (wpb < 1) wpb = 1;
    if (wpb > kMaxWarpsPerBlock) wpb = kMaxWarpsPerBlock;
    sp.persistent = plan.shape.blocks_per_sm > 0;
    int grid = sp.persistent ? plan.shape.blocks_per_sm * num_sms() : (plan.num_items + wpb - 1) / wpb;
    if (grid < 1) grid = 1;
    if (precision == PREC_F64) {
        k_sweep2d<double><<<grid, wpb * 32, wpb * warp_smem_bytes2d<double>(), st>>>(sp);
    } else if (precision == PREC_F32) {
        k_sweep2d<float><<<grid, wpb * 32, wpb * warp_smem_bytes2d<float>(), st>>>(sp);
    } else {
        k_sweep2d<__nv_bfloat16><<<grid, wpb * 32, wpb * warp_smem_bytes2d<float>(), st>>>(sp);
    }
    return cudaGetLastError();
}

}  // namespace fv
