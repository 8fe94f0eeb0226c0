// fv_sweep3d.cu -- fused 3D form: one thread block per patch, one thread per
// (x, y) column, sweeping the patch plane by plane along z (arXiv:2306.16731:
// the steps of Algorithm 1 for one patch, Rusanov faces of Eq. 2 in x, y and
// z, per-patch eigenvalue reduction of Sec. 4).
//
//   * Halo-inclusive z-planes ((p+2)^2 volumes) stream through a shared-
//     memory ring of R planes filled with cp.async in 16/8/4-byte chunks,
//     R-1 planes ahead.  Periodic patches copy plane p-1 as plane -1 and
//     plane 0 as plane p, and read x/y halo volumes at wrapped positions.
//   * Per plane each thread evaluates its volume once (primitives, F_x,
//     F_y, F_z and the three eigenvalues) and publishes F_x, lambda_x,
//     F_y, lambda_y in shared memory; the first 4p threads also evaluate
//     the plane's x/y halo volumes.  After a barrier each thread forms its
//     left and right x and y faces from shared data.
//   * z faces: the previous plane's Q, F_z and lambda_z stay in registers;
//     plane z-1 is finished when plane z's lower face is known:
//     Q_new = Q - dt/(2h) (((2Fx_r - 2Fx_l) + (2Fy_r - 2Fy_l)) + (2Fz_r - 2Fz_l)),
//     the oracle's order.
//   * Threads on the x boundary also write the x-halo volume of their row
//     (fixed: Q_in's halo value; periodic: the wrapped new value), so rows
//     are written whole.
#include <algorithm>

#include "fv_bulk.cuh"
#include "fv_common.cuh"

namespace fv {

namespace {

constexpr int kRing3 = 4;     // planes in the ring

constexpr int kMaxThreads3 = 256;    // p <= 16: one thread per (x, y) column

// Register budget: three 256-thread blocks per SM in float (80 registers),
// two in double.
template <typename C> struct MinBlocks3 { static constexpr int value = 3; };
template <> struct MinBlocks3<double> { static constexpr int value = 2; };

struct Sweep3Params {
    BatchView b;
    const void *q_in;
    void *q_out;
    const double *dx;
    const double *dt;
    double *lambda_out;
    double *dt_next_out;
    double cfl;
    float gamma_f, gm1_f;
    const int32_t *order;     // patch indices sorted by size class
    int first;                // first sorted position of this launch's class
    int count;                // patches of this class
    int p;                    // their edge length
};

template <typename C> __device__ __forceinline__ Gas<C> gas3(const Sweep3Params &sp);
template <> __device__ __forceinline__ Gas<float> gas3<float>(const Sweep3Params &sp)
{
    return Gas<float>{sp.gamma_f, sp.gm1_f};
}
template <> __device__ __forceinline__ Gas<double> gas3<double>(const Sweep3Params &sp)
{
    return Gas<double>{sp.b.gamma, sp.b.gamma - 1.0};
}

template <typename C> __device__ __forceinline__ C half_ratio3(double dt, double h);
template <> __device__ __forceinline__ float half_ratio3<float>(double dt, double h)
{
    return __fdividef(float(dt), 2.0f * float(h));
}
template <> __device__ __forceinline__ double half_ratio3<double>(double dt, double h)
{
    return dt / (2.0 * h);
}

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

template <int B>
__device__ __forceinline__ void cp_async_chunk(unsigned s, const void *g)
{
    if (B == 16) asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g) : "memory");
    else if (B == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(g) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int n>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(n) : "memory");
}

// Copy one contiguous plane of `bytes` into shared memory, chunked over the
// block's threads.
__device__ __forceinline__ void copy_plane(unsigned sdst, const unsigned char *gsrc, int bytes, int chunk)
{
    const int n = bytes / chunk;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        if (chunk == 16) cp_async_chunk<16>(sdst + c * 16, gsrc + c * 16);
        else if (chunk == 8) cp_async_chunk<8>(sdst + c * 8, gsrc + c * 8);
        else cp_async_chunk<4>(sdst + c * 4, gsrc + c * 4);
    }
}

template <int n, typename C>
__device__ __forceinline__ void physics_dir(const C (&q)[5], Gas<C> g, C (&F)[5], C &lam)
{
    Prim<3, C> s = primitives<3>(q, g);
    flux<3>(q, s, n, F);
    lam = eigenvalue<3>(s, n);
}

// Finish the owner's volume of plane zz (stored at memory plane zz+1):
// Q_new = Q - dt/(2h) ((x/y difference) + (upper - lower z face)), store,
// fold its eigenvalue into the running maximum and health.
template <typename S, typename C>
__device__ __forceinline__ void finish3(int zz, const C (&upper)[5], const C (&qp)[5], const C (&dxy)[5],
                                        const C (&lower)[5], C sc, Gas<C> g, int x, int y, int P, int E,
                                        int EE, bool periodic, const S *__restrict__ qin,
                                        S *__restrict__ qout, C &lmax, C &min_rp, C &sum_l)
{
    constexpr int N = 5;
    C qn[N];
#pragma unroll
    for (int k = 0; k < N; ++k) qn[k] = update_dq(qp[k], sc, dxy[k], upper[k], lower[k]);
    const int64_t prow = (int64_t)(zz + 1) * EE + (y + 1) * E;
    store_volume<N>(qout + (prow + x + 1) * N, qn);
    Prim<3, C> st = primitives<3>(qn, g);
    const C l = max_eigenvalue<3>(st);
    min_rp = min_rp < qn[0] ? min_rp : qn[0];
    min_rp = min_rp < st.p ? min_rp : st.p;
    sum_l += l;
    lmax = fv_max(lmax, l);
    // periodic patches: the volume at x = 0 is the halo volume at x = P and
    // vice versa; writing it keeps rows whole (fixed halos are copied from
    // the staged plane by fixed_halo3 instead)
    if (periodic && x == 0) store_volume<N>(qout + (prow + P + 1) * N, qn);
    if (periodic && x == P - 1) store_volume<N>(qout + prow * N, qn);
}

// Fixed halos: copy the x-halo volumes of row y of plane z from the staged
// plane to Q_out while the plane is current, so that with the interior
// written one plane later every 32-byte sector of the row is written whole.
template <typename S>
__device__ __forceinline__ void fixed_halo3(const S *pl, S *__restrict__ qout, int z, int x, int y, int P, int E,
                                            int EE)
{
    constexpr int N = 5;
    const int64_t prow = (int64_t)(z + 1) * EE + (y + 1) * E;
    if (x == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) qout[prow * N + k] = pl[((y + 1) * E) * N + k];
    }
    if (x == P - 1) {
#pragma unroll
        for (int k = 0; k < N; ++k) qout[(prow + P + 1) * N + k] = pl[((y + 1) * E + P + 1) * N + k];
    }
}

template <typename S, typename C>
__global__ void __launch_bounds__(kMaxThreads3, MinBlocks3<C>::value) k_sweep3d(Sweep3Params sp, int plane_bytes, int chunk)
{
    constexpr int N = 5;
    extern __shared__ __align__(16) unsigned char smem3[];
    const int P = sp.p, E = P + 2, EE = E * E;
    // layout: ring[kRing3][EE*N] (S) | Fx[N][EE] | Lx[EE] | Fy[N][EE] | Ly[EE] | red[32]
    unsigned char *ring = smem3;
    const int ring_plane = (plane_bytes + 15) & ~15;
    C *sFx = reinterpret_cast<C *>(ring + kRing3 * ring_plane);
    C *sLx = sFx + N * EE;
    C *sFy = sLx + EE;
    C *sLy = sFy + N * EE;
    C *red = sLy + EE;

    const int patch = sp.b.uniform_p > 0 ? sp.first + (int)blockIdx.x : __ldg(sp.order + sp.first + blockIdx.x);
    const int64_t base = sp.b.uniform_p > 0 ? (int64_t)patch * patch_cells(3, sp.b.uniform_p) * 5
                                            : __ldg(sp.b.elem_off + patch);
    const S *__restrict__ qin = static_cast<const S *>(sp.q_in) + base;
    S *__restrict__ qout = static_cast<S *>(sp.q_out) + base;
    const unsigned char *gpatch = reinterpret_cast<const unsigned char *>(qin);
    const bool periodic = sp.b.halo_mode == 1;
    const Gas<C> g = gas3<C>(sp);

    const int t = threadIdx.x;
    const bool owner = t < P * P;
    const int x = owner ? t % P : 0, y = owner ? t / P : 0;
    const int cell = (y + 1) * E + (x + 1);                  // in-plane index
    const double h = __ldg(sp.dx + patch);
    const C sc = half_ratio3<C>(__ldg(sp.dt + patch), h);

    // ring cells of a plane: thread t < 4P evaluates one halo volume
    int hx = 0, hy = 0, hdir = 0, hsrc = 0, hcell = 0;
    const bool ring_thread = t < 4 * P;
    if (ring_thread) {
        const int side = t / P, r = t - side * P;
        if (side == 0) { hx = -1; hy = r; hdir = 0; }
        else if (side == 1) { hx = P; hy = r; hdir = 0; }
        else if (side == 2) { hx = r; hy = -1; hdir = 1; }
        else { hx = r; hy = P; hdir = 1; }
        hcell = (hy + 1) * E + (hx + 1);
        const int sx = periodic ? wrap(hx, P) : hx, sy = periodic ? wrap(hy, P) : hy;
        hsrc = (sy + 1) * E + (sx + 1);
    }
    auto src_plane = [&](int z) { return periodic ? wrap(z, P) : z; };
    auto wrapped = [&](int xx, int yy) {
        if (periodic) { xx = wrap(xx, P); yy = wrap(yy, P); }
        return (yy + 1) * E + (xx + 1);
    };
    auto plane_ptr = [&](int z) {               // ring slot of plane z in [-1, P]
        return reinterpret_cast<const S *>(ring + ((z + 1) % kRing3) * ring_plane);
    };

    // prologue: planes -1 .. kRing3-3
    const unsigned ring_s = smem_addr(ring);
#pragma unroll
    for (int r = 0; r < kRing3 - 1; ++r) {
        const int z = r - 1;
        if (z <= P)
            copy_plane(ring_s + ((z + 1) % kRing3) * ring_plane,
                       gpatch + (int64_t)(src_plane(z) + 1) * plane_bytes, plane_bytes, chunk);
        cp_commit();
    }

    // carried from plane z-1: its state, physical F_z and lambda_z, its x/y
    // face difference and its lower z face
    C qp[N], Fzp[N], lzp = C(0), dxy[N], Fzlow[N];
#pragma unroll
    for (int k = 0; k < N; ++k) { qp[k] = C(1); Fzp[k] = C(0); dxy[k] = C(0); Fzlow[k] = C(0); }
    C lmax = C(0), min_rp = C(INFINITY), sum_l = C(0);

    for (int z = -1; z <= P; ++z) {
        cp_wait<kRing3 - 2>();
        __syncthreads();                                     // plane z visible; plane z-1 reads done
        {
            const int zn = z + kRing3 - 1;
            if (zn <= P)
                copy_plane(ring_s + ((zn + 1) % kRing3) * ring_plane,
                           gpatch + (int64_t)(src_plane(zn) + 1) * plane_bytes, plane_bytes, chunk);
            cp_commit();
        }
        const S *pl = plane_ptr(z);
        C q[N];
        if (owner) {
            load_volume<N>(pl + wrapped(x, y) * N, q);
        } else {
#pragma unroll
            for (int k = 0; k < N; ++k) q[k] = C(1);
            q[N - 1] = C(4);
        }
        if (z == -1) {                                       // lower halo plane
            physics_dir<2>(q, g, Fzp, lzp);
#pragma unroll
            for (int k = 0; k < N; ++k) qp[k] = q[k];
            continue;
        }
        if (z == P) {                                        // upper halo plane closes plane P-1
            C Fz[N], lz, Fh[N];
            physics_dir<2>(q, g, Fz, lz);
            rusanov2<N>(qp, q, Fzp, Fz, lzp, lz, Fh);
            if (owner)
                finish3<S, C>(P - 1, Fh, qp, dxy, Fzlow, sc, g, x, y, P, E, EE, periodic, qin, qout, lmax,
                              min_rp, sum_l);
            continue;
        }

        if (owner && !periodic) fixed_halo3<S>(pl, qout, z, x, y, P, E, EE);

        // interior plane z: full physics of the own volume, published
        Prim<3, C> s = primitives<3>(q, g);
        C Fx[N], Fy[N], Fz[N];
        flux<3>(q, s, 0, Fx);
        flux<3>(q, s, 1, Fy);
        flux<3>(q, s, 2, Fz);
        const C lx = eigenvalue<3>(s, 0), ly = eigenvalue<3>(s, 1), lz = eigenvalue<3>(s, 2);
        if (owner) {
#pragma unroll
            for (int k = 0; k < N; ++k) { sFx[k * EE + cell] = Fx[k]; sFy[k * EE + cell] = Fy[k]; }
            sLx[cell] = lx;
            sLy[cell] = ly;
        }
        if (ring_thread) {
            C hq[N], hF[N], hl;
            load_volume<N>(pl + hsrc * N, hq);
            if (hdir == 0) physics_dir<0>(hq, g, hF, hl);
            else physics_dir<1>(hq, g, hF, hl);
            C *dF = hdir == 0 ? sFx : sFy;
            C *dL = hdir == 0 ? sLx : sLy;
#pragma unroll
            for (int k = 0; k < N; ++k) dF[k * EE + hcell] = hF[k];
            dL[hcell] = hl;
        }

        // z face below plane z closes plane z-1; then plane z becomes the carry
        {
            C Fzl[N];
            rusanov2<N>(qp, q, Fzp, Fz, lzp, lz, Fzl);
            if (z > 0 && owner)
                finish3<S, C>(z - 1, Fzl, qp, dxy, Fzlow, sc, g, x, y, P, E, EE, periodic, qin, qout, lmax,
                              min_rp, sum_l);
#pragma unroll
            for (int k = 0; k < N; ++k) {
                Fzlow[k] = Fzl[k];
                Fzp[k] = Fz[k];
                qp[k] = q[k];
            }
            lzp = lz;
        }
        __syncthreads();                                     // F and lambda of the plane published

        // x and y faces of the own volume, from the published fluxes
        C d[N];
#pragma unroll
        for (int k = 0; k < N; ++k) d[k] = C(0);
        if (owner) {
#pragma unroll
            for (int n = 0; n < 2; ++n) {
                const C *sF = n == 0 ? sFx : sFy;
                const C *sL = n == 0 ? sLx : sLy;
                const int dxn = n == 0 ? 1 : 0, dyn = n == 0 ? 0 : 1;
                const int cl = (y - dyn + 1) * E + (x - dxn + 1), cr = (y + dyn + 1) * E + (x + dxn + 1);
                C qL[N], qR[N], FL[N], FR[N], Fc[N], hl[N], hr[N];
                load_volume<N>(pl + wrapped(x - dxn, y - dyn) * N, qL);
                load_volume<N>(pl + wrapped(x + dxn, y + dyn) * N, qR);
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    FL[k] = sF[k * EE + cl];
                    FR[k] = sF[k * EE + cr];
                    Fc[k] = sF[k * EE + cell];
                }
                const C lc = sL[cell];
                rusanov2<N>(qL, qp, FL, Fc, sL[cl], lc, hl);
                rusanov2<N>(qp, qR, Fc, FR, lc, sL[cr], hr);
#pragma unroll
                for (int k = 0; k < N; ++k) d[k] += hr[k] - hl[k];
            }
        }
#pragma unroll
        for (int k = 0; k < N; ++k) dxy[k] = d[k];
    }
    cp_wait<0>();

    // per-patch maximum eigenvalue, next time step, health flag
    const bool bad = owner && (!(min_rp > C(0)) || !(sum_l < C(INFINITY)));
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(sp.b.flags, FV_FLAG_NONPHYSICAL);
    if (sp.lambda_out || sp.dt_next_out) {
        lmax = block_max_nonneg(lmax, red);
        if (threadIdx.x == 0) {
            const double l = double(lmax);
            if (sp.lambda_out) sp.lambda_out[patch] = l;
            if (sp.dt_next_out) sp.dt_next_out[patch] = cfl_dt(sp.cfl, h, 3, l);
        }
    }
}

size_t smem3_bytes(int P, int precision)
{
    const size_t E = P + 2, EE = E * E, N = 5;
    const size_t s = precision == PREC_F64 ? 8 : (precision == PREC_F32 ? 4 : 2);
    const size_t c = precision == PREC_F64 ? 8 : 4;
    const size_t plane = (EE * N * s + 15) & ~size_t(15);
    return kRing3 * plane + (2 * N + 2) * EE * c + 32 * c;
}

// Largest power of two <= 16 dividing `bytes`.
int pow2_align(size_t bytes)
{
    int a = 16;
    while (a > 1 && bytes % a != 0) a >>= 1;
    return a;
}

template <typename S>
cudaError_t launch3(const Sweep3Params &sp, int chunk, cudaStream_t st, int precision)
{
    using C = typename StorageTraits<S>::Compute;
    const int P = sp.p;
    const int plane_bytes = (P + 2) * (P + 2) * 5 * (int)sizeof(S);
    const size_t smem = smem3_bytes(P, precision);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep3d<S, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int threads = std::max(32, ((P * P + 31) / 32) * 32);
    k_sweep3d<S, C><<<sp.count, threads, smem, st>>>(sp, plane_bytes, std::min(chunk, pow2_align(plane_bytes)));
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Edge lengths that are multiples of 8: one warp per 8 x 8 column block of a
// patch (the patch's (p/8)^2 warps share only the plane ring), two volumes
// per lane: lane = (x, yb) with x = lane % 8, yb = lane / 8, owning rows 2yb
// (cell A) and 2yb + 1 (cell B) of column x of the block.
//   * x faces: the right neighbour's Q, F_x, lambda_x by shuffle (lane + 1),
//     the left face as the left lane's right face (lane - 1);
//   * y faces: the face between the lane's two rows in registers; the face
//     above row 2yb + 1 with cell A of lane + 8; the face below row 2yb is
//     the upper face of lane - 8's cell B, by one shuffle back;
//   * the 32 faces between the block and its ring (patch halo or the
//     neighbouring block's volumes) are computed first, one per lane, into
//     shared memory, so no lane does extra face work inside the sweep;
//   * z faces by the register recurrence, as in the general kernel.
//   * Planes arrive in a ring of kRingB shared-memory slots, two planes
//     ahead.  With BULK (device-resident state whose patches start on
//     16-byte boundaries) thread 0 fetches each plane by one bulk
//     asynchronous copy whose completion is counted on the slot's mbarrier,
//     and every thread waits on that barrier, bounded in time: a wait that
//     runs out ends the block at the next plane step, after thread 0 has
//     waited (again bounded) for its copies in flight, and sets
//     FV_FLAG_TIMEOUT.  Otherwise every thread copies its share of the
//     plane in 16/8/4-byte cp.async chunks.
constexpr int kRingB = 3;
constexpr int kB8BarBytes = 32;      // the ring's mbarriers, at the start of shared memory

// Bytes of one ring slot: a halo-inclusive plane, plus (bulk copies) up to
// 15 bytes of 16-byte alignment padding on each side, rounded to 16 bytes.
inline __host__ __device__ int b8_slot_bytes(int plane_bytes, bool bulk)
{
    return bulk ? (plane_bytes + 30 + 15) & ~15 : (plane_bytes + 15) & ~15;
}

template <int N, typename C>
__device__ __forceinline__ void shfl_vec(C (&o)[N], const C (&v)[N], int delta, bool down)
{
#pragma unroll
    for (int k = 0; k < N; ++k)
        o[k] = down ? __shfl_down_sync(0xffffffffu, v[k], delta) : __shfl_up_sync(0xffffffffu, v[k], delta);
}

// Flux and eigenvalue along x (ydir false) or y (ydir true) without a
// branch: the normal velocity and the pressure slot are selected.
template <typename C>
__device__ __forceinline__ void physics_sel(const C (&q)[5], Gas<C> g, bool ydir, C (&F)[5], C &lam)
{
    Prim<3, C> s = primitives<3>(q, g);
    const C un = ydir ? s.u[1] : s.u[0];
    F[0] = ydir ? q[2] : q[1];
    F[1] = q[1] * un + (ydir ? C(0) : s.p);
    F[2] = q[2] * un + (ydir ? s.p : C(0));
    F[3] = q[3] * un;
    F[4] = (q[4] + s.p) * un;
    lam = fv_abs(un) + s.c;
}

// z planes per iteration of the 8x8-block kernel's plane loop
#ifndef FV_B8_UNROLL
#define FV_B8_UNROLL 2
#endif
constexpr int kB8Unroll = FV_B8_UNROLL;

// Doubled Rusanov face between a ring volume r and the interior volume i
// next to it: r is the lower-index side when ring_low, else the upper one.
template <typename C>
__device__ __forceinline__ void ring_face(const C (&qr)[5], const C (&qi)[5], const C (&Fr)[5], const C (&Fi)[5],
                                          C lr, C li, bool ring_low, C (&Fh)[5])
{
    const C nl = ring_low ? -fv_max(lr, li) : fv_max(lr, li);
#pragma unroll
    for (int k = 0; k < 5; ++k) Fh[k] = (Fr[k] + Fi[k]) + nl * (qi[k] - qr[k]);
}
template <>
__device__ __forceinline__ void ring_face<float>(const float (&qr)[5], const float (&qi)[5], const float (&Fr)[5],
                                                 const float (&Fi)[5], float lr, float li, bool ring_low,
                                                 float (&Fh)[5])
{
    const float nl = ring_low ? -fmaxf(lr, li) : fmaxf(lr, li);
#pragma unroll
    for (int k = 0; k < 5; ++k) Fh[k] = __fmaf_rn(nl, __fsub_rn(qi[k], qr[k]), __fadd_rn(Fr[k], Fi[k]));
}

// PC > 0: the edge length compiled in (all index arithmetic folds); 0: sp.p.
// Register budget: the 16-edge instance (128 threads) is held to five
// resident blocks per SM (96 registers, no spills: 20 warps; 121 registers
// and 16 warps otherwise); other edges take up to 512 threads.
template <typename S, typename C, int PC, bool BULK>
__global__ void __launch_bounds__(PC == 16 ? 128 : 512, PC == 16 ? 5 : 1)
    k_sweep3d_b8(Sweep3Params sp, int plane_bytes, int chunk)
{
    constexpr int N = 5;
    extern __shared__ __align__(16) unsigned char smemb[];
    const int P = PC > 0 ? PC : sp.p, E = P + 2, EE = E * E, nb = P / 8;
    const int ring_plane = b8_slot_bytes(plane_bytes, BULK);
    unsigned char *ring = smemb + kB8BarBytes;
    const unsigned bar0 = bulk::saddr(smemb);
    C *bfall = reinterpret_cast<C *>(ring + kRingB * ring_plane);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C *bf = bfall + warp * 32 * N;                   // this warp's 32 boundary faces
    C *red = bfall + (blockDim.x >> 5) * 32 * N;     // 32 slots

    const int patch = sp.b.uniform_p > 0 ? sp.first + (int)blockIdx.x : __ldg(sp.order + sp.first + blockIdx.x);
    const int64_t base = sp.b.uniform_p > 0 ? (int64_t)patch * patch_cells(3, sp.b.uniform_p) * 5
                                            : __ldg(sp.b.elem_off + patch);
    const S *__restrict__ qin = static_cast<const S *>(sp.q_in) + base;
    S *__restrict__ qout = static_cast<S *>(sp.q_out) + base;
    const unsigned char *gpatch = reinterpret_cast<const unsigned char *>(qin);
    const bool periodic = sp.b.halo_mode == 1;
    const Gas<C> g = gas3<C>(sp);
    const double h = __ldg(sp.dx + patch);
    const C sc = half_ratio3<C>(__ldg(sp.dt + patch), h);

    const int x0 = (warp % nb) * 8, y0 = (warp / nb) * 8;
    const int x = lane & 7, yb = lane >> 3;
    const int gx = x0 + x, gyA = y0 + 2 * yb, gyB = gyA + 1;
    const int cellA = (gyA + 1) * E + (gx + 1), cellB = (gyB + 1) * E + (gx + 1);

    // this lane's ring volume and the interior volume next to it
    const int side = lane >> 3, r = lane & 7;
    int rx, ry, ix, iy;
    if (side == 0) { rx = x0 - 1; ry = y0 + r; ix = x0; iy = ry; }
    else if (side == 1) { rx = x0 + 8; ry = y0 + r; ix = x0 + 7; iy = ry; }
    else if (side == 2) { rx = x0 + r; ry = y0 - 1; ix = rx; iy = y0; }
    else { rx = x0 + r; ry = y0 + 8; ix = rx; iy = y0 + 7; }
    if (periodic) { rx = wrap(rx, P); ry = wrap(ry, P); }
    const int rcell = (ry + 1) * E + (rx + 1), icell = (iy + 1) * E + (ix + 1);

    const unsigned ring_s = smem_addr(ring);
    auto src_plane = [&](int z) { return periodic ? wrap(z, P) : z; };
    // bulk copies: plane z (memory plane src_plane(z) + 1) is fill (z+1)/kRingB
    // of slot (z+1) % kRingB; the copied range is the plane widened to
    // 16-byte boundaries (inside the patch, whose bytes are a multiple of
    // 16), the plane starting at offset (start mod 16) of the slot
    auto plane_src = [&](int z) { return gpatch + (int64_t)(src_plane(z) + 1) * plane_bytes; };
    auto issue_bulk = [&](int z, unsigned extra) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(plane_src(z));
        const uintptr_t lo = a & ~uintptr_t(15), hi = (a + (uintptr_t)plane_bytes + 15) & ~uintptr_t(15);
        const int slot = (z + 1) % kRingB;
        bulk::mbar_expect_tx(bar0 + 8u * slot, (unsigned)(hi - lo) + extra);
        bulk::bulk_g2s(ring_s + slot * ring_plane, reinterpret_cast<const void *>(lo), (unsigned)(hi - lo),
                       bar0 + 8u * slot);
    };
    auto bar_of = [&](int z) { return bar0 + 8u * (unsigned)((z + 1) % kRingB); };
    auto parity_of = [&](int z) { return (unsigned)((z + 1) / kRingB) & 1u; };
    bool timed_out = false;
    int observed = -1, issued = -1;                  // thread 0: next plane not yet seen complete, last issued
    // after a wait ran out: thread 0 lets the copies in flight land, then
    // flags the batch; the caller returns
    auto drain = [&]() {
        if (threadIdx.x == 0) {
            for (int t = observed; t <= issued; ++t) bulk::mbar_wait_bounded(bar_of(t), parity_of(t));
            atomicOr(sp.b.flags, FV_FLAG_TIMEOUT);
        }
    };
    if (BULK) {
        if (threadIdx.x == 0) {
            for (int i = 0; i < kRingB; ++i) bulk::mbar_init(bar0 + 8u * i, 1);
            bulk::mbar_init_fence();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int z = -1; z <= kRingB - 3 && z <= P; ++z) {
                issue_bulk(z, z == -1 && sp.b.test_wait_expiry ? 16u : 0u);
                issued = z;
            }
        }
    } else {
#pragma unroll
        for (int rr = 0; rr < kRingB - 1; ++rr) {
            const int z = rr - 1;
            if (z <= P)
                copy_plane(ring_s + ((z + 1) % kRingB) * ring_plane, plane_src(z), plane_bytes, chunk);
            cp_commit();
        }
    }

    C qpA[N], FzpA[N], lzpA = C(0), dA[N], FlowA[N];
    C qpB[N], FzpB[N], lzpB = C(0), dB[N], FlowB[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        qpA[k] = qpB[k] = C(0);
        FzpA[k] = FzpB[k] = C(0);
        dA[k] = dB[k] = C(0);
        FlowA[k] = FlowB[k] = C(0);
    }
    C lmax = C(0), min_rp = C(INFINITY), sum_l = C(0);

    // planes two at a time: the carried values alternate between two
    // register sets instead of being moved
#pragma unroll (kB8Unroll)
    for (int z = -1; z <= P; ++z) {
        const int zn = z + kRingB - 1;
        if (BULK) {
            // every thread is done with plane z-1, whose slot plane zn takes
            if (__syncthreads_or(timed_out)) {
                drain();
                return;
            }
            if (threadIdx.x == 0 && zn <= P) {
                issue_bulk(zn, 0u);
                issued = zn;
            }
            if (!bulk::mbar_wait_bounded(bar_of(z), parity_of(z))) timed_out = true;
            else if (threadIdx.x == 0) observed = z + 1;
        } else {
            cp_wait<kRingB - 2>();
            __syncthreads();
            if (zn <= P) copy_plane(ring_s + ((zn + 1) % kRingB) * ring_plane, plane_src(zn), plane_bytes, chunk);
            cp_commit();
        }
        const S *pl = reinterpret_cast<const S *>(
            ring + ((z + 1) % kRingB) * ring_plane +
            (BULK ? (int)(reinterpret_cast<uintptr_t>(plane_src(z)) & 15) : 0));

        if (z == -1 || z == P) {
            C qA[N], qB[N], FzA[N], FzB[N], lzA, lzB;
            load_volume<N>(pl + cellA * N, qA);
            load_volume<N>(pl + cellB * N, qB);
            physics_dir<2>(qA, g, FzA, lzA);
            physics_dir<2>(qB, g, FzB, lzB);
            if (z == P) {
                C FhA[N], FhB[N];
                rusanov2<N>(qpA, qA, FzpA, FzA, lzpA, lzA, FhA);
                rusanov2<N>(qpB, qB, FzpB, FzB, lzpB, lzB, FhB);
                finish3<S, C>(P - 1, FhA, qpA, dA, FlowA, sc, g, gx, gyA, P, E, EE, periodic, qin, qout, lmax,
                              min_rp, sum_l);
                finish3<S, C>(P - 1, FhB, qpB, dB, FlowB, sc, g, gx, gyB, P, E, EE, periodic, qin, qout, lmax,
                              min_rp, sum_l);
            } else {
#pragma unroll
                for (int k = 0; k < N; ++k) { qpA[k] = qA[k]; qpB[k] = qB[k]; FzpA[k] = FzA[k]; FzpB[k] = FzB[k]; }
                lzpA = lzA;
                lzpB = lzB;
            }
            continue;
        }

        if (!periodic) {
            fixed_halo3<S>(pl, qout, z, gx, gyA, P, E, EE);
            fixed_halo3<S>(pl, qout, z, gx, gyB, P, E, EE);
        }

        // boundary faces of the block, one per lane (x faces for sides 0, 1,
        // y faces for sides 2, 3; the ring volume is the lower one for sides
        // 0 and 2)
        {
            C qr[N], qi[N], Fr[N], Fi[N], lr, li, Fh[N];
            load_volume<N>(pl + rcell * N, qr);
            load_volume<N>(pl + icell * N, qi);
            const bool ydir = side >= 2, ring_low = (side & 1) == 0;
            physics_sel(qr, g, ydir, Fr, lr);
            physics_sel(qi, g, ydir, Fi, li);
            // Eq. 2 with the lower volume first: for a ring volume above the
            // interior one, swapping the sides only flips the sign of the
            // dissipation term (exactly), so no operand needs selecting
            ring_face(qr, qi, Fr, Fi, lr, li, ring_low, Fh);
#pragma unroll
            for (int k = 0; k < N; ++k) bf[lane * N + k] = Fh[k];
        }

        // own volumes: physics, z faces, finish plane z-1
        C qA[N], qB[N];
        load_volume<N>(pl + cellA * N, qA);
        load_volume<N>(pl + cellB * N, qB);
        Prim<3, C> sA = primitives<3>(qA, g), sB = primitives<3>(qB, g);
        {
            C FzA[N], FzB[N], FlA[N], FlB[N];
            flux<3>(qA, sA, 2, FzA);
            flux<3>(qB, sB, 2, FzB);
            const C lzA = eigenvalue<3>(sA, 2), lzB = eigenvalue<3>(sB, 2);
            rusanov2<N>(qpA, qA, FzpA, FzA, lzpA, lzA, FlA);
            rusanov2<N>(qpB, qB, FzpB, FzB, lzpB, lzB, FlB);
            if (z > 0) {
                finish3<S, C>(z - 1, FlA, qpA, dA, FlowA, sc, g, gx, gyA, P, E, EE, periodic, qin, qout, lmax,
                              min_rp, sum_l);
                finish3<S, C>(z - 1, FlB, qpB, dB, FlowB, sc, g, gx, gyB, P, E, EE, periodic, qin, qout, lmax,
                              min_rp, sum_l);
            }
#pragma unroll
            for (int k = 0; k < N; ++k) {
                FlowA[k] = FlA[k]; FlowB[k] = FlB[k];
                FzpA[k] = FzA[k]; FzpB[k] = FzB[k];
                qpA[k] = qA[k]; qpB[k] = qB[k];
            }
            lzpA = lzA;
            lzpB = lzB;
        }
        __syncwarp();                                        // boundary faces visible

        // x faces
        {
            C FxA[N], FxB[N], nq[N], nF[N], FrA[N], FrB[N], FlA[N], FlB[N];
            flux<3>(qA, sA, 0, FxA);
            flux<3>(qB, sB, 0, FxB);
            const C lxA = eigenvalue<3>(sA, 0), lxB = eigenvalue<3>(sB, 0);
            shfl_vec<N>(nq, qA, 1, true);
            shfl_vec<N>(nF, FxA, 1, true);
            C nl = __shfl_down_sync(0xffffffffu, lxA, 1);
            rusanov2<N>(qA, nq, FxA, nF, lxA, nl, FrA);
            shfl_vec<N>(nq, qB, 1, true);
            shfl_vec<N>(nF, FxB, 1, true);
            nl = __shfl_down_sync(0xffffffffu, lxB, 1);
            rusanov2<N>(qB, nq, FxB, nF, lxB, nl, FrB);
            // every lane reads one edge entry per row (side 1 for column 7,
            // side 0 otherwise), so the edge columns cost one set of loads
            C eA[N], eB[N];
            const int ex = (x == 7 ? 8 : 0) + 2 * yb;
#pragma unroll
            for (int k = 0; k < N; ++k) { eA[k] = bf[ex * N + k]; eB[k] = bf[(ex + 1) * N + k]; }
            if (x == 7) {
#pragma unroll
                for (int k = 0; k < N; ++k) { FrA[k] = eA[k]; FrB[k] = eB[k]; }
            }
            shfl_vec<N>(FlA, FrA, 1, false);
            shfl_vec<N>(FlB, FrB, 1, false);
            if (x == 0) {
#pragma unroll
                for (int k = 0; k < N; ++k) { FlA[k] = eA[k]; FlB[k] = eB[k]; }
            }
#pragma unroll
            for (int k = 0; k < N; ++k) { dA[k] = FrA[k] - FlA[k]; dB[k] = FrB[k] - FlB[k]; }
        }
        // y faces: rows 2yb | 2yb+1 inside the lane; row 2yb+1 | 2yb+2 with
        // the A row of lane + 8 (the block's top edge face for yb = 3); the
        // face below row 2yb is the upper face of row 2yb-1, B of lane - 8
        // (the block's bottom edge face for yb = 0)
        {
            C FyA[N], FyB[N], nq[N], nF[N], FuA[N], FuB[N], FdA[N];
            flux<3>(qA, sA, 1, FyA);
            flux<3>(qB, sB, 1, FyB);
            const C lyA = eigenvalue<3>(sA, 1), lyB = eigenvalue<3>(sB, 1);
            const bool top = yb == 3, bottom = yb == 0;
            rusanov2<N>(qA, qB, FyA, FyB, lyA, lyB, FuA);
            shfl_vec<N>(nq, qA, 8, true);
            shfl_vec<N>(nF, FyA, 8, true);
            const C nl = __shfl_down_sync(0xffffffffu, lyA, 8);
            rusanov2<N>(qB, nq, FyB, nF, lyB, nl, FuB);
            C ey[N];                                          // side 3 for the top row, side 2 otherwise
#pragma unroll
            for (int k = 0; k < N; ++k) ey[k] = bf[((top ? 24 : 16) + x) * N + k];
            if (top) {
#pragma unroll
                for (int k = 0; k < N; ++k) FuB[k] = ey[k];
            }
            shfl_vec<N>(FdA, FuB, 8, false);
            if (bottom) {
#pragma unroll
                for (int k = 0; k < N; ++k) FdA[k] = ey[k];
            }
#pragma unroll
            for (int k = 0; k < N; ++k) { dA[k] += FuA[k] - FdA[k]; dB[k] += FuB[k] - FuA[k]; }
        }
        __syncwarp();                                        // boundary faces consumed
    }
    if (BULK) {
        if (__syncthreads_or(timed_out)) {
            drain();
            return;
        }
    } else {
        cp_wait<0>();
    }

    const bool bad = !(min_rp > C(0)) || !(sum_l < C(INFINITY));
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(sp.b.flags, FV_FLAG_NONPHYSICAL);
    if (sp.lambda_out || sp.dt_next_out) {
        lmax = block_max_nonneg(lmax, red);
        if (threadIdx.x == 0) {
            const double l = double(lmax);
            if (sp.lambda_out) sp.lambda_out[patch] = l;
            if (sp.dt_next_out) sp.dt_next_out[patch] = cfl_dt(sp.cfl, h, 3, l);
        }
    }
}

size_t smem3b_bytes(int P, int precision, bool bulk)
{
    const size_t E = P + 2, EE = E * E, N = 5;
    const size_t s = precision == PREC_F64 ? 8 : (precision == PREC_F32 ? 4 : 2);
    const size_t c = precision == PREC_F64 ? 8 : 4;
    const size_t slot = (size_t)b8_slot_bytes((int)(EE * N * s), bulk);
    const size_t warps = (size_t)(P / 8) * (P / 8);
    return kB8BarBytes + kRingB * slot + warps * 32 * N * c + 32 * c;
}

template <typename S, bool BULK>
cudaError_t launch3b_t(const Sweep3Params &sp, int chunk, cudaStream_t st, int precision)
{
    using C = typename StorageTraits<S>::Compute;
    const int P = sp.p;
    const int plane_bytes = (P + 2) * (P + 2) * 5 * (int)sizeof(S);
    const size_t smem = smem3b_bytes(P, precision, BULK);
    // the workloads' edges 8 and 16 compiled in, other multiples of 8 at run time
    auto kern = P == 16 ? k_sweep3d_b8<S, C, 16, BULK>
                        : (P == 8 ? k_sweep3d_b8<S, C, 8, BULK> : k_sweep3d_b8<S, C, 0, BULK>);
    static bool attr[3] = {false, false, false};
    const int ai = P == 16 ? 0 : (P == 8 ? 1 : 2);
    if (!attr[ai]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr[ai] = true;
    }
    const int threads = 32 * (P / 8) * (P / 8);
    kern<<<sp.count, threads, smem, st>>>(sp, plane_bytes, std::min(chunk, pow2_align(plane_bytes)));
    return cudaGetLastError();
}

template <typename S>
cudaError_t launch3b(const Sweep3Params &sp, int chunk, cudaStream_t st, int precision, bool bulk)
{
    return bulk ? launch3b_t<S, true>(sp, chunk, st, precision) : launch3b_t<S, false>(sp, chunk, st, precision);
}


}  // namespace

bool fused3d_supported(const BatchView &b, int precision)
{
    if (b.dim != 3 || b.num_patches <= 0) return false;
    // cp.async copies 4, 8 or 16 bytes: every patch and plane must start on
    // a 4-byte boundary (bfloat16 patches of odd edge length do not)
    if (b.align_bytes < 4) return false;
    const bool general = b.max_p * b.max_p <= kMaxThreads3 && smem3_bytes(b.max_p, precision) <= 227 * 1024;
    const bool blocks8 = precision != PREC_F64 && b.uniform_p > 0 && b.uniform_p % 8 == 0 && b.uniform_p <= 32;
    return general || blocks8;
}

const char *fused3d_kernel_name(const BatchView &b, int precision)
{
    if (b.dim != 3) return "none";
    if (b.uniform_p == 8 && b.halo_mode == 1 && precision != PREC_F64) return "sweep3d_p8";
    if (b.uniform_p > 0 && b.uniform_p % 8 == 0 && b.uniform_p <= 32 && precision != PREC_F64) return "sweep3d_b8";
    return "sweep3d";
}

cudaError_t launch_fused3d_update(const BatchView &b, int precision, const StepArgs &a, const FusedPlan &plan,
                                  cudaStream_t st)
{
    Sweep3Params sp;
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
    sp.order = plan.order;
    // every patch base is a multiple of the smallest power-of-two alignment
    // of all patch sizes in bytes (the buffer itself is 16-byte aligned)
    if (fused3d_p8_applies(b, precision, a.q_in, a.q_out)) {
        // uniform batch: one size class (or the item range of a sub-plan)
        for (int c = 0; c < plan.num_classes; ++c) {
            cudaError_t e = launch_fused3d_p8(b, precision, a, plan.class_begin[c],
                                              plan.class_end[c] - plan.class_begin[c], plan.shape, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const size_t es = precision == PREC_F64 ? 8 : (precision == PREC_F32 ? 4 : 2);
    int chunk = 16;
    for (int c = 0; c < plan.num_classes; ++c) {
        const size_t E = plan.class_p[c] + 2;
        chunk = std::min(chunk, pow2_align(E * E * E * 5 * es));
    }
    for (int c = 0; c < plan.num_classes; ++c) {
        sp.first = plan.class_begin[c];
        sp.count = plan.class_end[c] - plan.class_begin[c];
        sp.p = plan.class_p[c];
        cudaError_t e;
        // the block kernel needs 124 registers in float; double stays on the
        // general kernel (it would spill)
        const bool blocks8 = precision != PREC_F64 && sp.p % 8 == 0 && sp.p <= 32 &&
                             smem3b_bytes(sp.p, precision, true) <= 227 * 1024;
        if (blocks8) {
            // bulk plane copies: uniform batch (patch bases are multiples of
            // the patch bytes), 16-byte aligned patches, device-resident input
            const size_t E = sp.p + 2;
            const bool bulk = b.uniform_p > 0 && (E * E * E * 5 * es) % 16 == 0 &&
                              reinterpret_cast<uintptr_t>(a.q_in) % 16 == 0 && is_device_memory(a.q_in);
            if (precision == PREC_F32) e = launch3b<float>(sp, chunk, st, precision, bulk);
            else e = launch3b<__nv_bfloat16>(sp, chunk, st, precision, bulk);
        } else if (precision == PREC_F64) e = launch3<double>(sp, chunk, st, precision);
        else if (precision == PREC_F32) e = launch3<float>(sp, chunk, st, precision);
        else e = launch3<__nv_bfloat16>(sp, chunk, st, precision);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fv
