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
#include <algorithm>

#include "fv_common.cuh"

namespace fv {

namespace {

constexpr int kMaxWarpsPerBlock = 16;
constexpr int kMaxBlockSmem = 227 * 1024;      // opt-in dynamic shared memory per block

struct SweepParams {
    BatchView b;
    const void *q_in;
    void *q_out;
    const double *dx;
    const double *dt;
    double *lambda_out;
    double *dt_next_out;
    double cfl;
    float gamma_f, gm1_f;   // gas constants in float (the double ones are in b)
    int64_t uniform_elems;  // elements per patch if all patches share one edge, else 0
    const WorkItem *items;
    const int32_t *order;
    int item_begin;         // first item of this launch's size class
    int num_items;          // items of this launch's size class
    unsigned *counter;      // [0] = next item, [1] = finished warps (per class)
    int persistent;
};

// Ring depth (rows in flight per warp) of the compile-time-edge sweep.
#ifndef FV_RING_DEPTH
#define FV_RING_DEPTH 8
#endif
#ifndef FV_SWEEP_MINB
#define FV_SWEEP_MINB 1
#endif
#ifndef FV_SWEEP_MAXT
#define FV_SWEEP_MAXT (kMaxWarpsPerBlock * 32)
#endif
template <typename S> struct RingDepth { static constexpr int value = FV_RING_DEPTH; };
template <> struct RingDepth<double> { static constexpr int value = 4; };

// Per-warp shared memory: 64 boundary faces and 64 x-halo volumes of N=4
// values, 32 eigenvalue slots, and a ring of R rows of 32 volumes in
// storage type.
template <typename S, int R = RingDepth<S>::value>
__host__ __device__ constexpr int warp_smem_bytes2d()
{
    using C = typename StorageTraits<S>::Compute;
    return (2 * 64 * 4 + 32) * (int)sizeof(C) + R * 32 * 4 * (int)sizeof(S);
}

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// Asynchronous global -> shared copies (cp.async; completion tracked per
// thread with commit/wait groups, so no spin-wait is involved).
__device__ __forceinline__ void cp_async_16(unsigned s, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_8(unsigned s, const void *g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(n) : "memory");
}

// One 2D volume (4 unknowns) from global to shared memory.
template <typename S> __device__ __forceinline__ void copy_volume4_async(unsigned s, const S *g);
template <> __device__ __forceinline__ void copy_volume4_async<float>(unsigned s, const float *g)
{
    cp_async_16(s, g);
}
template <> __device__ __forceinline__ void copy_volume4_async<double>(unsigned s, const double *g)
{
    cp_async_16(s, g);
    cp_async_16(s + 16, g + 2);
}
template <> __device__ __forceinline__ void copy_volume4_async<__nv_bfloat16>(unsigned s, const __nv_bfloat16 *g)
{
    cp_async_8(s, g);
}

// Element offset of patch i (arithmetic for uniform batches).
__device__ __forceinline__ int64_t patch_base2(const SweepParams &sp, int i)
{
    return sp.uniform_elems ? (int64_t)i * sp.uniform_elems : __ldg(sp.b.elem_off + i);
}

template <typename C> __device__ __forceinline__ Gas<C> gas_of(const SweepParams &sp);
template <> __device__ __forceinline__ Gas<float> gas_of<float>(const SweepParams &sp)
{
    return Gas<float>{sp.gamma_f, sp.gm1_f};
}
template <> __device__ __forceinline__ Gas<double> gas_of<double>(const SweepParams &sp)
{
    return Gas<double>{sp.b.gamma, sp.b.gamma - 1.0};
}

// dt / (2h) in compute type (float arithmetic for float compute).
template <typename C> __device__ __forceinline__ C half_step_ratio(double dt, double h);
template <> __device__ __forceinline__ float half_step_ratio<float>(double dt, double h)
{
    return __fdividef(d2f_rn(dt), 2.0f * d2f_rn(h));
}
template <> __device__ __forceinline__ double half_step_ratio<double>(double dt, double h)
{
    return dt / (2.0 * h);
}

// Per-patch maximum eigenvalue and next time step; one lane per patch
// writes.  Edges that are powers of two give P-aligned lane segments, which
// reduce by xor shuffles (log2 P steps); other edges through shared memory.
template <typename C>
__device__ __forceinline__ void patch_lambda2(const SweepParams &sp, C lmax, int lane, int x, int P, bool active,
                                              int i, double h, C *red)
{
    if ((P & (P - 1)) == 0) {
        C m = lmax;
        for (int o = P >> 1; o > 0; o >>= 1) m = fv_max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (active && x == 0 && (sp.lambda_out || sp.dt_next_out)) {
            const double l = double(m);
            if (sp.lambda_out) sp.lambda_out[i] = l;
            if (sp.dt_next_out) sp.dt_next_out[i] = cfl_dt(sp.cfl, h, 2, l);
        }
        return;
    }
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

// Cheap running check of the new states: the minimum of density and
// pressure must stay positive and the sum of eigenvalues finite (NaN and
// infinity propagate through the sum).
template <typename C> struct Health {
    C min_rp = C(INFINITY);
    C sum_l = C(0);
    __device__ __forceinline__ void add(C rho, C p, C l)
    {
        min_rp = min_rp < rho ? min_rp : rho;
        min_rp = min_rp < p ? min_rp : p;
        sum_l += l;
    }
    __device__ __forceinline__ bool bad() const { return !(min_rp > C(0)) || !(sum_l < C(INFINITY)); }
};

// Store a new interior volume; with fixed halos the lanes on the patch's x
// boundary also write the neighbouring halo volume (Q_in's value, kept from
// the boundary pass), so every 32-byte sector of the row is written whole
// and no partial-sector read-modify-write reaches DRAM.
template <int N, typename S, typename C>
__device__ __forceinline__ void store_row_volume(S *dst_row, const C (&qn)[N], bool active, bool fixed,
                                                 int x, int P, const C *hv)
{
    if (!active) return;
    store_volume<N>(dst_row, qn);
    if (fixed && x == 0) {
        C h[N];
        load_volume<N>(hv, h);
        store_volume<N>(dst_row - N, h);
    }
    if (fixed && x == P - 1) {
        C h[N];
        load_volume<N>(hv + N, h);
        store_volume<N>(dst_row + N, h);
    }
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
                                             C *__restrict__ bface, C *__restrict__ hvol,
                                             C *__restrict__ red, Health<C> &hl)
{
    constexpr int N = 4;
    const Gas<C> g = gas_of<C>(sp);
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
        const int ip = sp.uniform_elems ? it.first_patch + fs : __ldg(sp.order + it.first_patch + fs);
        const S *ps = q + (sp.uniform_elems ? (int64_t)ip * sp.uniform_elems : __ldg(sp.b.elem_off + ip));
        int xl = side ? P - 1 : -1, xr = side ? P : 0;
        if (periodic) { xl = wrap(xl, P); xr = wrap(xr, P); }
        C qL[N], qR[N], FL[N], FR[N], Fh[N], lL, lR;
        load_volume<N>(ps + ((int64_t)(yy + 1) * E + (xl + 1)) * N, qL);
        load_volume<N>(ps + ((int64_t)(yy + 1) * E + (xr + 1)) * N, qR);
        xphys(qL, g, FL, lL);
        xphys(qR, g, FR, lR);
        rusanov2<N>(qL, qR, FL, FR, lL, lR, Fh);
        store_volume<N>(bface + ((fs * P + yy) * 2 + side) * N, Fh);
        store_volume<N>(hvol + ((fs * P + yy) * 2 + side) * N, side ? qR : qL);
    }
    __syncwarp();

    // ---- lane -> (patch slot, column)
    const int sub = lane / P;
    const int x = lane - sub * P;
    const bool active = sub < cnt;
    const int slot = active ? sub : 0;
    // uniform batches: the sorted order is the identity and offsets are
    // arithmetic, so no dependent loads precede the first data loads
    const int i = sp.uniform_elems ? it.first_patch + slot : __ldg(sp.order + it.first_patch + slot);
    const int64_t base = sp.uniform_elems ? (int64_t)i * sp.uniform_elems : __ldg(sp.b.elem_off + i);
    const S *src = q + base + (int64_t)(x + 1) * N;
    S *dst = qo + base + (int64_t)(x + 1) * N;
    const int64_t RS = (int64_t)E * N;               // row stride in elements
    const double h = __ldg(sp.dx + i);
    const C sc = half_step_ratio<C>(__ldg(sp.dt + i), h);
    const C *bf = bface + (slot * P) * 2 * N;
    const C *hv_row = hvol + (slot * P) * 2 * N;

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
            for (int k = 0; k < N; ++k) qn[k] = update_dq(qp[k], sc, dxp[k], Fyl[k], Fylp[k]);
            store_row_volume<N>(dst + (int64_t)y * RS, qn, active, !periodic, x, P, hv_row + (y - 1) * 2 * N);   // row y-1 lives at y
            Prim<2, C> t = primitives<2>(qn, g);
            const C l = max_eigenvalue<2>(t);
            hl.add(qn[0], t.p, l);
            lmax = fv_max(lmax, l);
        }

        // x faces of row y
        C qr[N], Fr_[N], Fr[N], Fl[N];
        shfl_down_vec<N>(q0, qr);
        shfl_down_vec<N>(Fx, Fr_);
        const C lr = __shfl_down_sync(0xffffffffu, lx, 1);
        rusanov2<N>(q0, qr, Fx, Fr_, lx, lr, Fr);
        if (x == P - 1) load_volume<N>(bf + (y * 2 + 1) * N, Fr);
#pragma unroll
        for (int k = 0; k < N; ++k) Fl[k] = __shfl_up_sync(0xffffffffu, Fr[k], 1);
        if (x == 0) load_volume<N>(bf + (y * 2) * N, Fl);

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
        for (int k = 0; k < N; ++k) qn[k] = update_dq(qp[k], sc, dxp[k], Fyu[k], Fylp[k]);
        store_row_volume<N>(dst + (int64_t)P * RS, qn, active, !periodic, x, P, hv_row + (P - 1) * 2 * N);
        Prim<2, C> t = primitives<2>(qn, g);
        const C l = max_eigenvalue<2>(t);
        hl.add(qn[0], t.p, l);
        lmax = fv_max(lmax, l);
    }

    // per-patch maximum eigenvalue and next time step
    patch_lambda2(sp, lmax, lane, x, P, active, i, h, red);
}


// Row-sweep carries of one lane: the previous row's state, y flux and
// eigenvalue, its x-face difference and the y face below it.
template <typename C> struct Row2 {
    C qp[4], Fyp[4], lyp, dxp[4], Fylp[4];
};

// Lower halo row: only F_y and lambda_y are needed.
template <typename C>
__device__ __forceinline__ void row2_lower_halo(Row2<C> &st, const C (&q0)[4], Gas<C> g)
{
    yphys(q0, g, st.Fyp, st.lyp);
#pragma unroll
    for (int k = 0; k < 4; ++k) st.qp[k] = q0[k];
}

// Interior row y of the own column: physics, the y face below (which closes
// row y-1: update, store, eigenvalue), the x faces (right face from the
// right lane's volume, left face from the left lane, boundary faces from the
// boundary pass), then row y becomes the carry.
template <typename S, typename C>
__device__ __forceinline__ void row2_interior(Row2<C> &st, const C (&q0)[4], Gas<C> g, int y, int P, int x,
                                              C sc, bool active, bool fixed, S *dst, const C *bf,
                                              const C *hv_row, Health<C> &hl, C &lmax)
{
    constexpr int N = 4;
    const int64_t RS = (int64_t)(P + 2) * N;
    Prim<2, C> s = primitives<2>(q0, g);
    C Fx[N], Fy[N];
    flux<2>(q0, s, 0, Fx);
    flux<2>(q0, s, 1, Fy);
    const C lx = eigenvalue<2>(s, 0), ly = eigenvalue<2>(s, 1);

    C Fyl[N];
    rusanov2<N>(st.qp, q0, st.Fyp, Fy, st.lyp, ly, Fyl);
    if (y > 0) {
        C qn[N];
#pragma unroll
        for (int k = 0; k < N; ++k) qn[k] = update_dq(st.qp[k], sc, st.dxp[k], Fyl[k], st.Fylp[k]);
        store_row_volume<N>(dst + y * RS, qn, active, fixed, x, P, hv_row + (y - 1) * 2 * N);
        Prim<2, C> t = primitives<2>(qn, g);
        const C l = max_eigenvalue<2>(t);
        hl.add(qn[0], t.p, l);
        lmax = fv_max(lmax, l);
    }

    C qr[N], Fr_[N], Fr[N], Fl[N];
    shfl_down_vec<N>(q0, qr);
    shfl_down_vec<N>(Fx, Fr_);
    const C lr = __shfl_down_sync(0xffffffffu, lx, 1);
    rusanov2<N>(q0, qr, Fx, Fr_, lx, lr, Fr);
    if (x == P - 1) load_volume<N>(bf + (y * 2 + 1) * N, Fr);
#pragma unroll
    for (int k = 0; k < N; ++k) Fl[k] = __shfl_up_sync(0xffffffffu, Fr[k], 1);
    if (x == 0) load_volume<N>(bf + (y * 2) * N, Fl);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        st.dxp[k] = Fr[k] - Fl[k];
        st.Fylp[k] = Fyl[k];
        st.qp[k] = q0[k];
        st.Fyp[k] = Fy[k];
    }
    st.lyp = ly;
}

// Upper halo row: its y face closes row P-1.
template <typename S, typename C>
__device__ __forceinline__ void row2_upper_halo(Row2<C> &st, const C (&q0)[4], Gas<C> g, int P, int x, C sc,
                                                bool active, bool fixed, S *dst, const C *hv_row,
                                                Health<C> &hl, C &lmax)
{
    constexpr int N = 4;
    const int64_t RS = (int64_t)(P + 2) * N;
    C Fy[N], ly, Fyu[N];
    yphys(q0, g, Fy, ly);
    rusanov2<N>(st.qp, q0, st.Fyp, Fy, st.lyp, ly, Fyu);
    C qn[N];
#pragma unroll
    for (int k = 0; k < N; ++k) qn[k] = update_dq(st.qp[k], sc, st.dxp[k], Fyu[k], st.Fylp[k]);
    store_row_volume<N>(dst + P * RS, qn, active, fixed, x, P, hv_row + (P - 1) * 2 * N);
    Prim<2, C> t = primitives<2>(qn, g);
    const C l = max_eigenvalue<2>(t);
    hl.add(qn[0], t.p, l);
    lmax = fv_max(lmax, l);
}

// Boundary x faces (and halo volumes) of one packed face slot from the two
// volumes adjacent to it.
template <typename C>
__device__ __forceinline__ void boundary_face2(const C (&qL)[4], const C (&qR)[4], Gas<C> g, int side,
                                               C *bface_slot, C *hvol_slot)
{
    constexpr int N = 4;
    C FL[N], FR[N], Fh[N], lL, lR;
    xphys(qL, g, FL, lL);
    xphys(qR, g, FR, lR);
    rusanov2<N>(qL, qR, FL, FR, lL, lR, Fh);
    store_volume<N>(bface_slot, Fh);
    store_volume<N>(hvol_slot, side ? qR : qL);
}


// Compile-time edge P (32/P patches per warp): rows stream through a
// per-warp shared-memory ring of R rows filled by cp.async, R-1 rows ahead
// of the row being computed, so many loads are in flight without holding
// registers.  Same arithmetic and order as sweep2d_item, whatever R.
template <typename S, typename C, int P, int R = RingDepth<S>::value>
__device__ __forceinline__ void sweep2d_tpl(const SweepParams sp, const WorkItem it, int lane,
                                            C *__restrict__ bface, C *__restrict__ hvol,
                                            C *__restrict__ red, unsigned char *__restrict__ ring,
                                            Health<C> &hl)
{
    constexpr int N = 4, E = P + 2;
    constexpr int VB = 4 * (int)sizeof(S);
    constexpr int RS = E * N;
    const Gas<C> g = gas_of<C>(sp);
    const S *__restrict__ q = static_cast<const S *>(sp.q_in);
    S *__restrict__ qo = static_cast<S *>(sp.q_out);
    const int cnt = it.count;
    const bool periodic = sp.b.halo_mode == 1;

    const int sub = lane / P;
    const int x = lane - sub * P;
    const bool active = sub < cnt;
    const int slot = active ? sub : 0;
    // uniform batches: the sorted order is the identity and offsets are
    // arithmetic, so no dependent loads precede the first data loads
    const int i = sp.uniform_elems ? it.first_patch + slot : __ldg(sp.order + it.first_patch + slot);
    const int64_t base = sp.uniform_elems ? (int64_t)i * sp.uniform_elems : __ldg(sp.b.elem_off + i);
    const S *src = q + base + (x + 1) * N;
    S *dst = qo + base + (x + 1) * N;
    const unsigned rbase = smem_u32(ring) + lane * VB;
    const unsigned char *rlane = ring + lane * VB;

    // the two halo rows: own halo memory, the wrapped interior (periodic) or
    // the neighbour's edge row across y (neighbour table registered)
    const S *row_lo = src + (periodic ? P : 0) * RS, *row_hi = src + (periodic ? 1 : P + 1) * RS;
    if (sp.b.nbr) {
        const int nlo = __ldg(sp.b.nbr + (int64_t)i * 4 + 2), nhi = __ldg(sp.b.nbr + (int64_t)i * 4 + 3);
        if (nlo >= 0) row_lo = q + patch_base2(sp, nlo) + (x + 1) * N + P * RS;     // its row P-1
        if (nhi >= 0) row_hi = q + patch_base2(sp, nhi) + (x + 1) * N + 1 * RS;     // its row 0
    }
    auto row_src = [&](int y) { return y < 0 ? row_lo : (y >= P ? row_hi : src + (y + 1) * RS); };

    // rows -1 .. R-3 in flight before anything else
#pragma unroll
    for (int r = 0; r < R - 1; ++r) {
        const int y = r - 1;
        if (y <= P) copy_volume4_async<S>(rbase + ((y + 1) % R) * 32 * VB, row_src(y));
        cp_async_commit();
    }

    // boundary x faces of every row, packed over the warp
    const int nf = 2 * P * cnt;
    for (int f = lane; f < nf; f += 32) {
        const int fs = f / (2 * P);
        const int r = f - fs * 2 * P;
        const int yy = r >> 1, side = r & 1;
        const int ip = sp.uniform_elems ? it.first_patch + fs : __ldg(sp.order + it.first_patch + fs);
        const S *ps = q + patch_base2(sp, ip);
        int xl = side ? P - 1 : -1, xr = side ? P : 0;
        if (periodic) { xl = wrap(xl, P); xr = wrap(xr, P); }
        const S *pl = ps + ((yy + 1) * E + (xl + 1)) * N, *pr = ps + ((yy + 1) * E + (xr + 1)) * N;
        if (sp.b.nbr) {                        // the halo volume comes from the neighbour across x
            const int n = __ldg(sp.b.nbr + (int64_t)ip * 4 + side);
            if (n >= 0) {
                const S *pn = q + patch_base2(sp, n) + (yy + 1) * E * N;
                if (side) pr = pn + 1 * N;               // neighbour's column 0
                else pl = pn + P * N;                    // neighbour's column P-1
            }
        }
        C qL[N], qR[N], FL[N], FR[N], Fh[N], lL, lR;
        load_volume<N>(pl, qL);
        load_volume<N>(pr, qR);
        xphys(qL, g, FL, lL);
        xphys(qR, g, FR, lR);
        rusanov2<N>(qL, qR, FL, FR, lL, lR, Fh);
        store_volume<N>(bface + ((fs * P + yy) * 2 + side) * N, Fh);
        store_volume<N>(hvol + ((fs * P + yy) * 2 + side) * N, side ? qR : qL);
    }
    __syncwarp();

    const double h = __ldg(sp.dx + i);
    const C sc = half_step_ratio<C>(__ldg(sp.dt + i), h);
    const C *bf = bface + (slot * P) * 2 * N;
    const C *hv_row = hvol + (slot * P) * 2 * N;

    // issue row y+R-1, then wait until row y (ring slot (y+1) % R) has landed
    auto advance = [&](int y, C (&qv)[N]) {
        const int yn = y + R - 1;
        if (yn <= P) copy_volume4_async<S>(rbase + ((yn + 1) % R) * 32 * VB, row_src(yn));
        cp_async_commit();
        cp_async_wait<R - 1>();
        load_volume<N>(reinterpret_cast<const S *>(rlane + ((y + 1) % R) * 32 * VB), qv);
    };

    Row2<C> st;
    C lmax = C(0);
    {
        C q0[N];
        advance(-1, q0);
        row2_lower_halo(st, q0, g);
    }
#pragma unroll 2
    for (int y = 0; y < P; ++y) {
        C q0[N];
        advance(y, q0);
        row2_interior<S>(st, q0, g, y, P, x, sc, active, !periodic, dst, bf, hv_row, hl, lmax);
    }
    {
        C q0[N];
        advance(P, q0);
        row2_upper_halo<S>(st, q0, g, P, x, sc, active, !periodic, dst, hv_row, hl, lmax);
    }
    cp_async_wait<0>();

    patch_lambda2(sp, lmax, lane, x, P, active, i, h, red);
}

// P > 0 selects the compile-time-edge sweep for one patch-size class, P == 0
// the runtime-edge one; P < 0 takes the items of every class in one launch
// when all edges are 4, 8, 16 or 32 (each item dispatched on its edge; items
// sorted largest patches first, so persistent warps end on the small ones).
// Items [item_begin, item_begin + num_items) of the sorted work list belong
// to the launch.

// Register cap: the launch over every size class inlines four sweeps and
// would take 104 registers in FP32; held to 72 (28 warps per SM, a few bytes
// spilled) it measured 11% faster than unheld on a 50,000-patch uneven
// batch, and 1.8% faster than held to 64.  The other instances take what
// 512-thread blocks allow.
template <typename S, int P>
constexpr int sweep2d_max_regs()
{
    return (P < 0 && sizeof(S) < 8) ? 72 : 65536 / FV_SWEEP_MAXT;
}

template <typename S, int P, int R = RingDepth<S>::value>
__global__ void __maxnreg__((sweep2d_max_regs<S, P>())) k_sweep2d(SweepParams sp)
{
    using C = typename StorageTraits<S>::Compute;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem_raw + warp * warp_smem_bytes2d<S, R>();
    C *bface = reinterpret_cast<C *>(wbase);
    C *hvol = bface + 64 * 4;
    C *red = hvol + 64 * 4;
    unsigned char *ring = wbase + (2 * 64 * 4 + 32) * sizeof(C);
    Health<C> hl;
    const int wpb = blockDim.x >> 5;
    auto run = [&](int item) {
        WorkItem it;
        if (sp.uniform_elems) {            // items of a uniform batch: K = 32/p patches each
            const int p = sp.b.uniform_p, K = 32 / p;
            it.first_patch = item * K;
            it.count = (int16_t)min(K, sp.b.num_patches - item * K);
            it.p = (int16_t)p;
        } else {
            it = sp.items[item];
        }
        if (P > 0) {
            sweep2d_tpl<S, C, (P > 0 ? P : 4), R>(sp, it, lane, bface, hvol, red, ring, hl);
        } else if (P < 0) {                 // every size class in one launch
            switch (it.p) {
            case 4: sweep2d_tpl<S, C, 4>(sp, it, lane, bface, hvol, red, ring, hl); break;
            case 8: sweep2d_tpl<S, C, 8>(sp, it, lane, bface, hvol, red, ring, hl); break;
            case 16: sweep2d_tpl<S, C, 16>(sp, it, lane, bface, hvol, red, ring, hl); break;
            default: sweep2d_tpl<S, C, 32>(sp, it, lane, bface, hvol, red, ring, hl); break;   // 32
            }
        } else {
            sweep2d_item<S, C>(sp, it, lane, bface, hvol, red, hl);
        }
    };
    if (!sp.persistent) {
        const int item = blockIdx.x * wpb + warp;
        if (item < sp.num_items) run(sp.item_begin + item);
    } else {
        for (;;) {
            int item = 0;
            if (lane == 0) item = (int)atomicAdd(sp.counter, 1u);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item >= sp.num_items) break;
            run(sp.item_begin + item);
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
    if (__any_sync(0xffffffffu, hl.bad()) && lane == 0) atomicOr(sp.b.flags, FV_FLAG_NONPHYSICAL);
}


// ---------------------------------------------------------------------------
// Streaming variant for uniform batches: persistent warps take items
// round-robin (item = warp + j * warps), and the row ring runs across item
// boundaries, so the next item's rows -- and the volumes its boundary pass
// needs, staged by cp.async one item ahead -- are in flight while the
// current item finishes.  Same arithmetic as sweep2d_tpl.
constexpr int kRingS = 6;

template <typename S>
__host__ __device__ constexpr int warp_smem_bytes2d_stream()
{
    using C = typename StorageTraits<S>::Compute;
    return (2 * 64 * 4 + 32) * (int)sizeof(C) + (kRingS + 4) * 32 * 4 * (int)sizeof(S);
}

// cp.async the two volumes of each of this lane's (at most two) boundary
// face slots of item k into the staging area.
template <typename S, int P>
__device__ __forceinline__ void stage_boundary2(const SweepParams &sp, int k, int lane, unsigned stage_s)
{
    constexpr int N = 4, E = P + 2, K = 32 / P, VB = 4 * (int)sizeof(S);
    const S *q = static_cast<const S *>(sp.q_in);
    const bool periodic = sp.b.halo_mode == 1;
    const int cnt = min(K, sp.b.num_patches - k * K);
    const int nf = 2 * P * cnt;
#pragma unroll
    for (int fi = 0; fi < 2; ++fi) {
        const int f = lane + 32 * fi;
        if (f < nf) {
            const int fs = f / (2 * P), r = f - fs * 2 * P;
            const int yy = r >> 1, side = r & 1;
            int xl = side ? P - 1 : -1, xr = side ? P : 0;
            if (periodic) { xl = wrap(xl, P); xr = wrap(xr, P); }
            const S *ps = q + (int64_t)(k * K + fs) * sp.uniform_elems + (yy + 1) * E * N;
            copy_volume4_async<S>(stage_s + ((fi * 2 + 0) * 32 + lane) * VB, ps + (xl + 1) * N);
            copy_volume4_async<S>(stage_s + ((fi * 2 + 1) * 32 + lane) * VB, ps + (xr + 1) * N);
        }
    }
}

// Boundary pass of item k from the staged volumes (each lane reads only what
// it staged itself).
template <typename S, typename C, int P>
__device__ __forceinline__ void boundary_from_stage2(const SweepParams &sp, int k, int lane,
                                                     const unsigned char *stage, C *bface, C *hvol, Gas<C> g)
{
    constexpr int N = 4, K = 32 / P, VB = 4 * (int)sizeof(S);
    const int cnt = min(K, sp.b.num_patches - k * K);
    const int nf = 2 * P * cnt;
#pragma unroll
    for (int fi = 0; fi < 2; ++fi) {
        const int f = lane + 32 * fi;
        if (f < nf) {
            const int fs = f / (2 * P), r = f - fs * 2 * P;
            const int yy = r >> 1, side = r & 1;
            C qL[N], qR[N];
            load_volume<N>(reinterpret_cast<const S *>(stage + ((fi * 2 + 0) * 32 + lane) * VB), qL);
            load_volume<N>(reinterpret_cast<const S *>(stage + ((fi * 2 + 1) * 32 + lane) * VB), qR);
            boundary_face2(qL, qR, g, side, bface + ((fs * P + yy) * 2 + side) * N,
                           hvol + ((fs * P + yy) * 2 + side) * N);
        }
    }
}

template <typename S, typename C, int P>
__device__ __forceinline__ void sweep2d_stream(const SweepParams sp, int gw, int W, int lane,
                                               C *__restrict__ bface, C *__restrict__ hvol,
                                               C *__restrict__ red, unsigned char *__restrict__ ring,
                                               unsigned char *__restrict__ stage, Health<C> &hl)
{
    constexpr int N = 4, E = P + 2, K = 32 / P, R = kRingS, RPI = P + 2;
    constexpr int VB = 4 * (int)sizeof(S);
    constexpr int RS = E * N;
    const int nitems = sp.num_items;
    if (gw >= nitems) return;
    const int n_my = (nitems - gw + W - 1) / W;
    const int total_rows = n_my * RPI;
    const Gas<C> g = gas_of<C>(sp);
    const S *__restrict__ q = static_cast<const S *>(sp.q_in);
    S *__restrict__ qo = static_cast<S *>(sp.q_out);
    const bool periodic = sp.b.halo_mode == 1;
    const int T = sp.b.num_patches;
    const int sub = lane / P, x = lane - sub * P;
    const unsigned rbase = smem_u32(ring) + lane * VB, sbase = smem_u32(stage);
    const unsigned char *rlane = ring + lane * VB;

    // stream position t -> (item j of this warp, row y); issue its row
    auto issue = [&](int t) {
        if (t < total_rows) {
            const int j = t / RPI, y = t - j * RPI - 1;
            const int k = gw + j * W;
            const int cnt = min(K, T - k * K);
            const int slot = sub < cnt ? sub : 0;
            const int yy = periodic ? wrap(y, P) : y;
            const S *src = q + (int64_t)(k * K + slot) * sp.uniform_elems + (x + 1) * N + (yy + 1) * RS;
            copy_volume4_async<S>(rbase + (t % R) * 32 * VB, src);
        }
    };
    auto advance = [&](int t, C (&qv)[N]) {
        issue(t + R - 1);
        cp_async_commit();
        cp_async_wait<R - 1>();
        load_volume<N>(reinterpret_cast<const S *>(rlane + (t % R) * 32 * VB), qv);
    };

    stage_boundary2<S, P>(sp, gw, lane, sbase);               // joins the first row's group
#pragma unroll
    for (int t = 0; t < R - 1; ++t) {
        issue(t);
        cp_async_commit();
    }
    cp_async_wait<R - 2>();                                    // the first group has landed

    for (int j = 0; j < n_my; ++j) {
        const int k = gw + j * W;
        const int cnt = min(K, T - k * K);
        const bool active = sub < cnt;
        const int slot = active ? sub : 0;
        const int i = k * K + slot;
        boundary_from_stage2<S, C, P>(sp, k, lane, stage, bface, hvol, g);
        __syncwarp();
        // staged volumes consumed: stage the next item's (they join the
        // group of the next row issue and land one item ahead)
        if (j + 1 < n_my) stage_boundary2<S, P>(sp, k + W, lane, sbase);

        const int64_t base = (int64_t)i * sp.uniform_elems;
        S *dst = qo + base + (x + 1) * N;
        const double h = __ldg(sp.dx + i);
        const C sc = half_step_ratio<C>(__ldg(sp.dt + i), h);
        const C *bf = bface + (slot * P) * 2 * N;
        const C *hv_row = hvol + (slot * P) * 2 * N;
        const int t0 = j * RPI;

        Row2<C> st;
        C lmax = C(0);
        {
            C q0[N];
            advance(t0, q0);
            row2_lower_halo(st, q0, g);
        }
#pragma unroll 2
        for (int y = 0; y < P; ++y) {
            C q0[N];
            advance(t0 + 1 + y, q0);
            row2_interior<S>(st, q0, g, y, P, x, sc, active, !periodic, dst, bf, hv_row, hl, lmax);
        }
        {
            C q0[N];
            advance(t0 + P + 1, q0);
            row2_upper_halo<S>(st, q0, g, P, x, sc, active, !periodic, dst, hv_row, hl, lmax);
        }
        patch_lambda2(sp, lmax, lane, x, P, active, i, h, red);
    }
    cp_async_wait<0>();
}

template <typename S, int P>
__global__ void __launch_bounds__(FV_SWEEP_MAXT, FV_SWEEP_MINB) k_sweep2d_stream(SweepParams sp)
{
    using C = typename StorageTraits<S>::Compute;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem_raw + warp * warp_smem_bytes2d_stream<S>();
    C *bface = reinterpret_cast<C *>(wbase);
    C *hvol = bface + 64 * 4;
    C *red = hvol + 64 * 4;
    unsigned char *ring = wbase + (2 * 64 * 4 + 32) * sizeof(C);
    unsigned char *stage = ring + kRingS * 32 * 4 * sizeof(S);
    Health<C> hl;
    const int wpb = blockDim.x >> 5;
    sweep2d_stream<S, C, P>(sp, blockIdx.x * wpb + warp, gridDim.x * wpb, lane, bface, hvol, red, ring, stage, hl);
    if (__any_sync(0xffffffffu, hl.bad()) && lane == 0) atomicOr(sp.b.flags, FV_FLAG_NONPHYSICAL);
}

template <typename S, int P>
cudaError_t launch_stream(const SweepParams &sp, int wpb, cudaStream_t st)
{
    static bool attr_set = false;
    // warps per block limited by the shared memory a block may use (FP64
    // rings of 16 warps would exceed it; results do not depend on the shape)
    constexpr int kMaxWarpsSmem = kMaxBlockSmem / warp_smem_bytes2d_stream<S>();
    wpb = std::min(wpb, kMaxWarpsSmem);
    const int bytes = wpb * warp_smem_bytes2d_stream<S>();
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep2d_stream<S, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             std::min(kMaxWarpsPerBlock, kMaxWarpsSmem) * warp_smem_bytes2d_stream<S>());
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int per_sm = 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep2d_stream<S, P>, wpb * 32, bytes);
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    int grid = std::min((sp.num_items + wpb - 1) / wpb, per_sm * num_sms());
    if (grid < 1) grid = 1;
    k_sweep2d_stream<S, P><<<grid, wpb * 32, bytes, st>>>(sp);
    return cudaGetLastError();
}

// Grid: one warp per item, or (persistent) blocks_per_sm blocks per SM,
// where blocks_per_sm < 0 means as many as can be resident at once.
template <typename S, int P, int R = RingDepth<S>::value>
cudaError_t launch_class(const SweepParams &sp, int wpb, int bps, cudaStream_t st)
{
    static bool attr_set = false;
    constexpr int kMaxWarpsSmem = kMaxBlockSmem / warp_smem_bytes2d<S, R>();
    wpb = std::min(wpb, kMaxWarpsSmem);
    const int bytes = wpb * warp_smem_bytes2d<S, R>();
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep2d<S, P, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             std::min(kMaxWarpsPerBlock, kMaxWarpsSmem) * warp_smem_bytes2d<S, R>());
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int grid = (sp.num_items + wpb - 1) / wpb;
    if (sp.persistent) {
        int per_sm = bps;
        if (per_sm < 0) {
            per_sm = 1;
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep2d<S, P, R>, wpb * 32, bytes);
            if (e != cudaSuccess || per_sm < 1) per_sm = 1;
        }
        grid = std::min(grid, per_sm * num_sms());
    }
    if (grid < 1) grid = 1;
    k_sweep2d<S, P, R><<<grid, wpb * 32, bytes, st>>>(sp);
    return cudaGetLastError();
}

// compile-time edge p with a row ring of `ring` rows (4 or 6; otherwise the
// default depth)
template <typename S, int P>
cudaError_t launch_class_ring(int ring, const SweepParams &sp, int wpb, int bps, cudaStream_t st)
{
    if (sizeof(S) < 8) {                    // FP32 / BF16 storage: ring depths are tuned
        if (ring == 4) return launch_class<S, P, 4>(sp, wpb, bps, st);
        if (ring == 6) return launch_class<S, P, 6>(sp, wpb, bps, st);
    }
    return launch_class<S, P>(sp, wpb, bps, st);
}

template <typename S>
cudaError_t launch_class_p(int p, int ring, const SweepParams &sp, int wpb, int bps, cudaStream_t st)
{
    if (bps == -2 && sp.uniform_elems && !sp.b.nbr) {   // streaming persistent warps (uniform batches)
        switch (p) {
        case 8: return launch_stream<S, 8>(sp, wpb, st);
        case 16: return launch_stream<S, 16>(sp, wpb, st);
        case 32: return launch_stream<S, 32>(sp, wpb, st);
        default: break;
        }
        bps = -1;
    }
    switch (p) {
    case 4: return launch_class_ring<S, 4>(ring, sp, wpb, bps, st);
    case 8: return launch_class_ring<S, 8>(ring, sp, wpb, bps, st);
    case 16: return launch_class_ring<S, 16>(ring, sp, wpb, bps, st);
    case 32: return launch_class_ring<S, 32>(ring, sp, wpb, bps, st);
    default: return launch_class<S, 0>(sp, wpb, bps, st);
    }
}

}  // namespace

bool fused_reads_neighbours(const FusedPlan &plan)
{
    if (plan.kernel != FUSED_SWEEP2D) return false;
    for (int c = 0; c < plan.num_classes; ++c) {
        const int p = plan.class_p[c];
        if (p != 4 && p != 8 && p != 16 && p != 32) return false;   // runtime-edge sweep reads own halos
    }
    return true;
}

bool sweep_ring_applies(const BatchView &b, int precision)
{
    const int p = b.uniform_p;
    return b.dim == 2 && precision != PREC_F64 && (p == 4 || p == 8 || p == 16 || p == 32);
}

bool fused_supported(const BatchView &b, int precision, int *kernel)
{
    *kernel = FUSED_NONE;
    if (b.num_patches <= 0) return false;
    if (b.dim == 2 && b.max_p <= 32) {
        *kernel = FUSED_SWEEP2D;
        return true;
    }
    if (b.dim == 3 && fused3d_supported(b, precision)) {
        *kernel = FUSED_SWEEP3D;
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
    if (plan.kernel == FUSED_SWEEP3D) return launch_fused3d_update(b, precision, a, plan, st);
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
    sp.gamma_f = float(b.gamma);
    sp.gm1_f = float(b.gamma - 1.0);
    sp.uniform_elems = b.uniform_p > 0 ? patch_cells(2, b.uniform_p) * 4 : 0;
    sp.items = plan.items;
    sp.order = plan.order;
    int wpb = plan.shape.warps_per_block;
    if (wpb < 1) wpb = 1;
    if (wpb > kMaxWarpsPerBlock) wpb = kMaxWarpsPerBlock;
    sp.persistent = plan.shape.blocks_per_sm != 0;      // -1 and -2 are persistent too
    bool compiled_edges = true;
    for (int c = 0; c < plan.num_classes; ++c) {
        const int p = plan.class_p[c];
        compiled_edges = compiled_edges && (p == 4 || p == 8 || p == 16 || p == 32);
    }
    if (plan.num_classes > 1 && compiled_edges) {
        // uneven batch of compiled edges: one launch over all items
        sp.item_begin = plan.class_begin[0];
        sp.num_items = plan.class_end[plan.num_classes - 1] - plan.class_begin[0];
        sp.counter = plan.work_counter;
        const int bps = plan.shape.blocks_per_sm == -2 ? -1 : plan.shape.blocks_per_sm;
        if (precision == PREC_F64) return launch_class<double, -1>(sp, wpb, bps, st);
        if (precision == PREC_F32) return launch_class<float, -1>(sp, wpb, bps, st);
        return launch_class<__nv_bfloat16, -1>(sp, wpb, bps, st);
    }
    for (int c = 0; c < plan.num_classes; ++c) {
        sp.item_begin = plan.class_begin[c];
        sp.num_items = plan.class_end[c] - plan.class_begin[c];
        sp.counter = plan.work_counter + 2 * c;
        const int p = plan.class_p[c], bps = plan.shape.blocks_per_sm;
        cudaError_t e;
        const int ring = plan.shape.ring;
        if (precision == PREC_F64) e = launch_class_p<double>(p, ring, sp, wpb, bps, st);
        else if (precision == PREC_F32) e = launch_class_p<float>(p, ring, sp, wpb, bps, st);
        else e = launch_class_p<__nv_bfloat16>(p, ring, sp, wpb, bps, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fv
