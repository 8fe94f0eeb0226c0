// fv_pde.cu -- the generic first-order hyperbolic PDE of Eq. 1 (arXiv:2306.16731,
// Sec. 2: dQ/dt + div F(Q) + sum_n B_n(Q) dQ/dx_n = S(Q)) in two realisations:
// the patch-wise one (one thread block per patch, the halo-inclusive patch
// staged in shared memory) and a fused row sweep (warps own patches, lanes
// own columns; below).  The PDE enters through a device functor with the
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
#include <algorithm>

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

// ---------------------------------------------------------------------------
// Fused row sweep of the generic PDE (the Euler sweep's design, fv_sweep.cu,
// with the non-conservative product and the source of Eq. 1): a warp takes
// 32/P patches of edge P (lane = column x), rows stream through a per-warp
// shared-memory ring (cp.async, R-1 rows ahead), y faces by the register
// recurrence, x faces with the right lane's volume by shuffle, the faces on
// the patch's x boundary from a packed pass before the sweep.  At every face
// the doubled Rusanov flux 2Fhat of the evolved unknowns and the product
// D = B_n((Q_L+Q_R)/2)(Q_R - Q_L); per volume, as the patch-wise kernel:
//   acc = 1/2 ((2Fhat_r - 2Fhat_l) + (D_r + D_l))_x + 1/2 (...)_y,
//   Q_new = Q - (dt/h) acc + dt S(Q)  (evolved unknowns; parameters copied).

struct PdeSweepParams {
    BatchView b;
    const void *q_in;
    void *q_out;
    const double *dx, *dt;
    double *lambda_out, *dt_next_out;
    double cfl;
    const WorkItem *items;
    const int32_t *order;
    int item_begin, num_items;
    unsigned *counter;          // [0] next item, [1] finished warps
    int persistent;
    int64_t uniform_elems;      // elements per patch of a uniform batch, else 0
};

template <typename S> struct PdeRing { static constexpr int value = 8; };
template <> struct PdeRing<double> { static constexpr int value = 4; };

// Per-warp shared memory: 64 boundary faces (2Fhat and D) and 64 x-halo
// volumes of N values in compute type, then the ring of R rows of 32 volumes.
template <int N, typename S, typename C>
__host__ __device__ constexpr int pde_warp_smem()
{
    return 3 * 64 * N * (int)sizeof(C) + PdeRing<S>::value * 32 * N * (int)sizeof(S);
}

__device__ __forceinline__ void pde_cp16(unsigned s, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(g) : "memory");
}
__device__ __forceinline__ void pde_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int n> __device__ __forceinline__ void pde_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(n) : "memory"); }

// one stored volume of N unknowns (16-byte multiples) into shared memory
template <int N, typename S>
__device__ __forceinline__ void pde_copy_volume(unsigned s, const S *g)
{
#pragma unroll
    for (int c = 0; c < N * (int)sizeof(S) / 16; ++c) pde_cp16(s + 16 * c, reinterpret_cast<const char *>(g) + 16 * c);
}

// The physics of one volume along axis n: flux and eigenvalue.
template <class Ph, typename C>
__device__ __forceinline__ void pde_phys(const Ph &ph, const C (&q)[Ph::N], int n, C (&F)[Ph::N], C &lam)
{
    ph.flux(q, n, F);
    lam = ph.lambda(q, n);
}

// Doubled Rusanov flux on the evolved unknowns from both sides' fluxes and
// eigenvalues (Eq. 2), and the non-conservative product of the face.
template <class Ph, typename C>
__device__ __forceinline__ void pde_face(const Ph &ph, const C (&qL)[Ph::N], const C (&qR)[Ph::N],
                                         const C (&FL)[Ph::N], const C (&FR)[Ph::N], C lL, C lR, int n,
                                         C (&Fh)[Ph::N], C (&D)[Ph::N])
{
    const C lam = fv_max(lL, lR);
#pragma unroll
    for (int k = 0; k < Ph::N; ++k) Fh[k] = k < Ph::NV ? (FL[k] + FR[k]) - lam * (qR[k] - qL[k]) : C(0);
    ph.ncp(qL, qR, n, D);
}

template <class Ph, typename S, typename C, int P>
__device__ __forceinline__ void pde_sweep_item(const PdeSweepParams &sp, const Ph &ph, const WorkItem it, int lane,
                                               C *__restrict__ bface, C *__restrict__ bD, C *__restrict__ hvol,
                                               unsigned char *__restrict__ ring, bool &bad)
{
    constexpr int N = Ph::N, E = P + 2, RS = E * N, R = PdeRing<S>::value, VB = N * (int)sizeof(S);
    const S *__restrict__ q = static_cast<const S *>(sp.q_in);
    S *__restrict__ qo = static_cast<S *>(sp.q_out);
    const bool periodic = sp.b.halo_mode == 1;
    const int cnt = it.count;
    const int sub = lane / P, x = lane - sub * P;
    const bool active = sub < cnt;
    const int slot = active ? sub : 0;
    auto patch_of = [&](int s_) { return sp.uniform_elems ? it.first_patch + s_ : __ldg(sp.order + it.first_patch + s_); };
    auto base_of = [&](int i_) { return sp.uniform_elems ? (int64_t)i_ * sp.uniform_elems : __ldg(sp.b.elem_off + i_); };
    const int i = patch_of(slot);
    const S *src = q + base_of(i) + (x + 1) * N;
    S *dst = qo + base_of(i) + (x + 1) * N;
    const S *row_lo = src + (periodic ? P : 0) * RS, *row_hi = src + (periodic ? 1 : P + 1) * RS;
    auto row_src = [&](int y) { return y < 0 ? row_lo : (y >= P ? row_hi : src + (y + 1) * RS); };
    const unsigned rbase = (unsigned)__cvta_generic_to_shared(ring) + lane * VB;
    const unsigned char *rlane = ring + lane * VB;

#pragma unroll
    for (int r = 0; r < R - 1; ++r) {
        const int y = r - 1;
        if (y <= P) pde_copy_volume<N>(rbase + ((y + 1) % R) * 32 * VB, row_src(y));
        pde_commit();
    }

    // boundary x faces of every row, packed over the warp: 2Fhat, D and the
    // x-halo volume (Q_in's value, written back with the row)
    for (int f = lane; f < 2 * P * cnt; f += 32) {
        const int fs = f / (2 * P), r = f - fs * 2 * P, yy = r >> 1, side = r & 1;
        const S *ps = q + base_of(patch_of(fs));
        int xl = side ? P - 1 : -1, xr = side ? P : 0;
        if (periodic) { xl = wrap(xl, P); xr = wrap(xr, P); }
        C qL[N], qR[N], FL[N], FR[N], Fh[N], D[N], lL, lR;
        load_volume<N>(ps + ((yy + 1) * E + (xl + 1)) * N, qL);
        load_volume<N>(ps + ((yy + 1) * E + (xr + 1)) * N, qR);
        pde_phys(ph, qL, 0, FL, lL);
        pde_phys(ph, qR, 0, FR, lR);
        pde_face(ph, qL, qR, FL, FR, lL, lR, 0, Fh, D);
        const int e = ((fs * P + yy) * 2 + side) * N;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            bface[e + k] = Fh[k];
            bD[e + k] = D[k];
            hvol[e + k] = side ? qR[k] : qL[k];
        }
    }
    __syncwarp();

    const double h = __ldg(sp.dx + i), tau = __ldg(sp.dt + i);
    const C scale = step_ratio<C>(tau, h), ct = C(tau), half = C(0.5);
    const C *bf = bface + (slot * P) * 2 * N, *bd = bD + (slot * P) * 2 * N, *hv = hvol + (slot * P) * 2 * N;

    auto advance = [&](int y, C (&qv)[N]) {
        const int yn = y + R - 1;
        if (yn <= P) pde_copy_volume<N>(rbase + ((yn + 1) % R) * 32 * VB, row_src(yn));
        pde_commit();
        pde_wait<R - 1>();
        load_volume<N>(reinterpret_cast<const S *>(rlane + ((y + 1) % R) * 32 * VB), qv);
    };

    // carries of the row below: state, F_y and lambda_y, its lower y face
    // (2Fhat and D) and its x contribution
    C qp[N], Fyp[N], lyp, Fylp[N], Dylp[N], cxp[N];
    C lmax = C(0);
    // row yf is finished once its upper y face (Fu, Du) is known
    auto finish = [&](int yf, const C (&Fu)[N], const C (&Du)[N]) {
        C Sv[N], qn[N];
        ph.source(qp, Sv);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const C acc = half * cxp[k] + half * ((Fu[k] - Fylp[k]) + (Du[k] + Dylp[k]));
            qn[k] = k < Ph::NV ? (qp[k] - scale * acc) + ct * Sv[k] : qp[k];
        }
        if (active) {
            S *d = dst + (yf + 1) * RS;
            store_volume<N>(d, qn);
            // whole rows: the x-halo volumes keep Q_in's values
            if (!periodic && x == 0) {
                C hq[N];
                load_volume<N>(hv + (yf * 2) * N, hq);
                store_volume<N>(d - N, hq);
            }
            if (!periodic && x == P - 1) {
                C hq[N];
                load_volume<N>(hv + (yf * 2 + 1) * N, hq);
                store_volume<N>(d + N, hq);
            }
        }
        const C l = fv_max(ph.lambda(qn, 0), ph.lambda(qn, 1));
        bad = bad || ph.bad(qn, l);
        lmax = fv_max(lmax, l);
    };

    {   // lower halo row: F_y and lambda_y only
        C q0[N];
        advance(-1, q0);
        pde_phys(ph, q0, 1, Fyp, lyp);
#pragma unroll
        for (int k = 0; k < N; ++k) qp[k] = q0[k];
    }
#pragma unroll 2
    for (int y = 0; y < P; ++y) {
        C q0[N], Fx[N], Fy[N], lx, ly;
        advance(y, q0);
        pde_phys(ph, q0, 0, Fx, lx);
        pde_phys(ph, q0, 1, Fy, ly);
        C Fyl[N], Dyl[N];
        pde_face(ph, qp, q0, Fyp, Fy, lyp, ly, 1, Fyl, Dyl);
        if (y > 0) finish(y - 1, Fyl, Dyl);

        // x faces: right face with the right lane's volume, left face from the left lane
        C qr[N], Fr_[N], Frx[N], Drx[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            qr[k] = __shfl_down_sync(0xffffffffu, q0[k], 1);
            Fr_[k] = __shfl_down_sync(0xffffffffu, Fx[k], 1);
        }
        const C lr = __shfl_down_sync(0xffffffffu, lx, 1);
        pde_face(ph, q0, qr, Fx, Fr_, lx, lr, 0, Frx, Drx);
        if (x == P - 1) {
            load_volume<N>(bf + (y * 2 + 1) * N, Frx);
            load_volume<N>(bd + (y * 2 + 1) * N, Drx);
        }
        C Flx[N], Dlx[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            Flx[k] = __shfl_up_sync(0xffffffffu, Frx[k], 1);
            Dlx[k] = __shfl_up_sync(0xffffffffu, Drx[k], 1);
        }
        if (x == 0) {
            load_volume<N>(bf + (y * 2) * N, Flx);
            load_volume<N>(bd + (y * 2) * N, Dlx);
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {
            cxp[k] = (Frx[k] - Flx[k]) + (Drx[k] + Dlx[k]);
            qp[k] = q0[k];
            Fyp[k] = Fy[k];
            Fylp[k] = Fyl[k];
            Dylp[k] = Dyl[k];
        }
        lyp = ly;
    }
    {   // upper halo row: its y face closes row P-1
        C q0[N], Fy[N], ly, Fyu[N], Dyu[N];
        advance(P, q0);
        pde_phys(ph, q0, 1, Fy, ly);
        pde_face(ph, qp, q0, Fyp, Fy, lyp, ly, 1, Fyu, Dyu);
        finish(P - 1, Fyu, Dyu);
    }
    pde_wait<0>();

    // per-patch maximum eigenvalue (xor shuffles over the patch's P lanes)
    // and next time step; one lane per patch writes
    C m = lmax;
#pragma unroll
    for (int o = P >> 1; o > 0; o >>= 1) m = fv_max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (active && x == 0 && (sp.lambda_out || sp.dt_next_out)) {
        const double l = double(m);
        if (sp.lambda_out) sp.lambda_out[i] = l;
        if (sp.dt_next_out) sp.dt_next_out[i] = cfl_dt(sp.cfl, h, 2, l);
    }
}

// P > 0: one compile-time edge per launch (items [item_begin, item_begin +
// num_items) of the size-sorted work list).  Items one per warp, or taken by
// persistent warps from a device counter; the last warp resets it.
template <class Ph, typename S, int P>
__global__ void __launch_bounds__(512, 1) k_sweep_pde(PdeSweepParams sp, Ph ph)
{
    using C = typename StorageTraits<S>::Compute;
    constexpr int N = Ph::N;
    extern __shared__ __align__(16) unsigned char smem_sw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *wbase = smem_sw + warp * pde_warp_smem<N, S, C>();
    C *bface = reinterpret_cast<C *>(wbase);
    C *bD = bface + 64 * N;
    C *hvol = bD + 64 * N;
    unsigned char *ring = wbase + 3 * 64 * N * sizeof(C);
    bool bad = false;
    const int wpb = blockDim.x >> 5;
    auto run = [&](int item) {
        WorkItem it;
        if (sp.uniform_elems) {
            it.first_patch = item * (32 / P);
            it.count = (int16_t)min(32 / P, sp.b.num_patches - item * (32 / P));
            it.p = (int16_t)P;
        } else {
            it = sp.items[item];
        }
        pde_sweep_item<Ph, S, C, P>(sp, ph, it, lane, bface, bD, hvol, ring, bad);
        __syncwarp();           // the next item's boundary pass overwrites the faces
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

template <class Ph, typename S, int P>
cudaError_t launch_sweep_pde(const PdeSweepParams &sp, const Ph &ph, int wpb, int bps, cudaStream_t st)
{
    using C = typename StorageTraits<S>::Compute;
    constexpr int bytes_w = pde_warp_smem<Ph::N, S, C>();
    static bool attr_set = false;
    wpb = std::min(wpb, std::min(16, (int)(kMaxSmem / bytes_w)));
    const int bytes = wpb * bytes_w;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep_pde<Ph, S, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             std::min(16, (int)(kMaxSmem / bytes_w)) * bytes_w);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int grid = (sp.num_items + wpb - 1) / wpb;
    if (sp.persistent) {
        int per_sm = bps;
        if (per_sm < 0) {
            per_sm = 1;
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_pde<Ph, S, P>, wpb * 32, bytes);
            if (e != cudaSuccess || per_sm < 1) per_sm = 1;
        }
        grid = std::min(grid, per_sm * num_sms());
    }
    if (grid < 1) grid = 1;
    k_sweep_pde<Ph, S, P><<<grid, wpb * 32, bytes, st>>>(sp, ph);
    return cudaGetLastError();
}

template <class Ph, typename S>
cudaError_t launch_sweep_pde_p(int p, const PdeSweepParams &sp, const Ph &ph, int wpb, int bps, cudaStream_t st)
{
    switch (p) {
    case 4: return launch_sweep_pde<Ph, S, 4>(sp, ph, wpb, bps, st);
    case 8: return launch_sweep_pde<Ph, S, 8>(sp, ph, wpb, bps, st);
    case 16: return launch_sweep_pde<Ph, S, 16>(sp, ph, wpb, bps, st);
    default: return launch_sweep_pde<Ph, S, 32>(sp, ph, wpb, bps, st);
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

bool pde_fused_supported(const BatchView &b, int precision, const int32_t *sizes_host)
{
    if (b.pde != PDE_SHALLOW_WATER || b.dim != 2 || precision == PREC_BF16 || b.num_patches <= 0) return false;
    for (int i = 0; i < b.num_patches; ++i) {
        const int p = sizes_host[i];
        if (p != 4 && p != 8 && p != 16 && p != 32) return false;
    }
    return true;
}

cudaError_t launch_pde_fused_update(const BatchView &b, int precision, const StepArgs &a, const FusedPlan &plan,
                                    cudaStream_t st)
{
    if (b.num_patches == 0) return cudaSuccess;
    PdeSweepParams sp;
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
    sp.uniform_elems = b.uniform_p > 0 ? patch_cells(2, b.uniform_p) * 4 : 0;
    const int wpb = std::max(1, std::min(16, plan.shape.warps_per_block));
    sp.persistent = plan.shape.blocks_per_sm != 0;
    const int bps = plan.shape.blocks_per_sm == -2 ? -1 : plan.shape.blocks_per_sm;
    for (int c = 0; c < plan.num_classes; ++c) {
        sp.item_begin = plan.class_begin[c];
        sp.num_items = plan.class_end[c] - plan.class_begin[c];
        sp.counter = plan.work_counter + 2 * c;
        const int p = plan.class_p[c];
        cudaError_t e;
        if (precision == PREC_F64) {
            ShallowWater<double> ph{b.pde_param[0], b.pde_param[1]};
            e = launch_sweep_pde_p<ShallowWater<double>, double>(p, sp, ph, wpb, bps, st);
        } else {
            ShallowWater<float> ph{float(b.pde_param[0]), float(b.pde_param[1])};
            e = launch_sweep_pde_p<ShallowWater<float>, float>(p, sp, ph, wpb, bps, st);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fv
