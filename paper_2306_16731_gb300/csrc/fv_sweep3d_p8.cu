// fv_sweep3d_p8.cu -- fused 3D form for periodic patches of 8 x 8 x 8
// volumes, one warp per patch (arXiv:2306.16731: the steps of Algorithm 1
// for one patch, the Rusanov faces of Eq. 2 along x, y and z, the per-patch
// eigenvalue reduction of Sec. 4; periodic halos of Sec. 2.2).
//
//   * Lane (x, j), x = lane % 8, j = lane / 8, owns the columns (x, 2j) and
//     (x, 2j+1) of every z-plane.  The two volumes form one packed pair and
//     each arithmetic step on them is one f32x2 instruction (fma/add/mul
//     .f32x2 of sm_100 and later), which halves the issue cost of the
//     flux, face and update arithmetic.
//   * Periodic halos wrap inside the patch, so every x and y face joins two
//     volumes of the same warp: the x neighbour is lane (x+1) mod 8 of the
//     same row group; the face between rows 2j and 2j+1 stays inside the
//     lane; the face above row 2j+1 meets row 2j+2 (mod 8), the first
//     volume of lane + 8 (mod 32).  Each face is computed once and handed
//     to the volume on its other side by one shuffle.
//   * z faces by the register recurrence of the other fused kernels, over
//     planes 7, 0, 1, ..., 7, 0 (the first and last close the wrap).
//   * The interior rows of each plane arrive by one bulk asynchronous copy
//     (cp.async.bulk, completion counted on an mbarrier) into a per-warp
//     ring of shared-memory slots, kSlots-1 planes ahead, continuing across
//     the warp's patches.  Halo volumes of the stored input are read only as
//     the 16-byte padding of the copied range.  Every wait on a slot is
//     bounded in time; a wait that runs out sets FV_FLAG_TIMEOUT, drains the
//     copies in flight (again bounded) and ends the warp's work.
//   * Rows are written whole: the x-halo volumes get the wrapped new values.
//     A finished plane's 8 rows are one contiguous byte range; they are
//     assembled in a shared-memory staging buffer and leave by one
//     bulk store (cp.async.bulk shared -> global) plus a few 2-byte stores
//     for the unaligned ends, instead of scalar stores at the 20-byte volume
//     stride that touch ten sectors per warp instruction.
#include <algorithm>

#include "fv_bulk.cuh"
#include "fv_common.cuh"
#include "fv_pair.cuh"

namespace fv {

namespace {

using namespace pair;
using namespace bulk;

constexpr int kP = 8, kE = kP + 2;
constexpr int kSlots = 5;                  // plane slots per warp
constexpr int kMaxWarps = 4;               // warps per block
// resident blocks per SM the register budget is sized for: 4 (16 warps,
// <= 128 registers) measured faster than 5 (20 warps at 96 registers with
// spills)
#ifndef FV_P8_MIN_BLOCKS
#define FV_P8_MIN_BLOCKS 4
#endif
constexpr int kStepsPerPatch = kP + 2;     // planes 7, 0..7, 0

// 1: pair arithmetic as f32x2 instructions; 0: two scalar instructions per
// pair (identical bits; kept for the packed-versus-scalar comparison)
#ifndef FV_P8_PACKED
#define FV_P8_PACKED 1
#endif
constexpr bool kPacked = FV_P8_PACKED != 0;

struct P8Params {
    const unsigned char *q_in;    // state bytes, 16-byte aligned
    unsigned char *q_out;
    const double *dx;
    const double *dt;
    double *lambda_out;
    double *dt_next_out;
    double cfl;
    float gamma, gm1;
    unsigned *flags;
    int first;                    // first patch of the launch
    int count;                    // patches
    unsigned extra_tx;            // test hook: bytes the first plane wait expects beyond its copy
};

// ------------------------------------------------------------------ kernel

// Byte geometry of one stored patch of storage type S.
template <typename S> struct Geo {
    static constexpr int vol = kN * (int)sizeof(S);          // one volume
    static constexpr int row = kE * vol;                      // one halo-inclusive row
    static constexpr int plane = kE * row;
    static constexpr int64_t patch = (int64_t)kE * plane;
    // shared-memory slot of one plane's 8 interior rows: up to 15 bytes of
    // alignment padding on each side, rounded to 16 bytes
    static constexpr int slot = (8 * row + 30 + 15) & ~15;
    // start of interior row 0 of plane zz (stored plane zz + 1), patch-relative
    static __device__ __forceinline__ int rows_begin(int zz) { return (zz + 1) * plane + row; }
};

template <typename S>
__device__ __forceinline__ void store_pair(S *__restrict__ a, S *__restrict__ b, const float2 (&q)[kN])
{
#pragma unroll
    for (int k = 0; k < kN; ++k) {
        a[k] = from_compute<S>(q[k].x);
        b[k] = from_compute<S>(q[k].y);
    }
}

template <typename S, bool Pk>
__global__ void __launch_bounds__(kMaxWarps * 32, FV_P8_MIN_BLOCKS) k_sweep3d_p8(P8Params sp)
{
    using A = Arith<Pk>;
    using G = Geo<S>;
    extern __shared__ __align__(16) unsigned char smem8[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = blockDim.x >> 5;
    const unsigned bar0 = saddr(smem8) + 8u * (unsigned)(warp * kSlots);
    // per warp: kSlots input plane slots, then two output staging buffers
    unsigned char *slots = smem8 + ((W * kSlots * 8 + 15) & ~15) + (size_t)warp * (kSlots + 2) * G::slot;
    const unsigned slot0 = saddr(slots);

    const int gw = blockIdx.x * W + warp, nwarps = gridDim.x * W;
    const int mine = gw < sp.count ? (sp.count - 1 - gw) / nwarps + 1 : 0;
    if (mine == 0) return;

    if (lane == 0) {
        for (int i = 0; i < kSlots; ++i) mbar_init(bar0 + 8u * i, 1);
        mbar_init_fence();
    }
    __syncwarp();

    // Step s (0..9) of a patch reads plane (s + 7) mod 8 into slot s mod 5;
    // with ten steps per patch and five slots, slot and mbarrier parity
    // ((s / 5) mod 2) are the same for every patch, so after unrolling the
    // steps they are constants.  The load of step s + 4 is issued at step s
    // (for s + 4 >= 10: step s - 6 of the warp's next patch).
    auto issue = [&](int64_t patch, int zz, int slot, unsigned extra) {
        if (lane != 0) return;
        const int rb = G::rows_begin(zz);
        const int lo = rb & ~15, hi = (rb + 8 * G::row + 15) & ~15;
        // the slot's previous plane was loaded into registers and used by
        // every lane before the __syncwarp that precedes this call
        mbar_expect_tx(bar0 + 8u * slot, (unsigned)(hi - lo) + extra);
        bulk_g2s(slot0 + (unsigned)(slot * G::slot), sp.q_in + patch * G::patch + lo, (unsigned)(hi - lo),
                 bar0 + 8u * slot);
    };
    const int64_t patch0 = sp.first + gw;
#pragma unroll
    for (int s = 0; s < kSlots - 1; ++s) issue(patch0, (s + kP - 1) & (kP - 1), s, s == 0 ? sp.extra_tx : 0u);

    const int x = lane & 7, j = lane >> 3;
    const int src_r = (lane & 24) | ((x + 1) & 7), src_l = (lane & 24) | ((x + 7) & 7);
    const int src_u = (lane + 8) & 31, src_d = (lane + 24) & 31;
    const float2 g2 = bcast(sp.gamma), gm12 = bcast(sp.gm1);
    // the wrapped x-halo column this lane's volumes are copied to as well
    // (column 8 -> column 0, column 1 -> column 9), or none
    const int halo_col = x == kP - 1 ? 0 : (x == 0 ? kP + 1 : -1);

    // Output staging: the plane finished in step t is assembled in buffer
    // t & 1 and leaves at the start of step t + 1 (after the one warp
    // barrier of that step), so assembling never waits for a store.
    unsigned char *const stg0 = slots + kSlots * G::slot;
    // Publish the plane assembled in the previous step: called by every lane
    // after the step's barrier; lane 0 has issued the bulk store of the
    // 16-byte aligned middle, the lanes write the ragged ends.
    auto store_ends = [&](int64_t opatch, int zf, int buf) {
        const unsigned char *stg = stg0 + buf * G::slot;
        const int sa = G::rows_begin(zf) & 15;
        unsigned char *gbase = sp.q_out + opatch * G::patch + (G::rows_begin(zf) - sa);   // 16-aligned
        constexpr int kRows = 8 * G::row;
        const int mlo = (sa + 15) & ~15, end = sa + kRows, mhi = end & ~15;
        const int o = lane < 16 ? sa + 2 * lane : mhi + 2 * (lane - 16);
        if (lane < 16 ? o < mlo : o < end)
            *reinterpret_cast<unsigned short *>(gbase + o) = *reinterpret_cast<const unsigned short *>(stg + o);
    };
    auto store_middle = [&](int64_t opatch, int zf, int buf) {     // lane 0
        const int sa = G::rows_begin(zf) & 15;
        unsigned char *gbase = sp.q_out + opatch * G::patch + (G::rows_begin(zf) - sa);
        constexpr int kRows = 8 * G::row;
        const int mlo = (sa + 15) & ~15, mhi = (sa + kRows) & ~15;
        bulk_s2g(gbase + mlo, saddr(stg0 + buf * G::slot) + (unsigned)mlo, (unsigned)(mhi - mlo));
        bulk_commit();
    };

    // carried from the previous plane: state, F_z, lambda_z, its x/y face
    // difference and its lower z face
    float2 qp[kN], Fzp[kN], lzp = bcast(0.0f), d[kN], Flo[kN];
#pragma unroll
    for (int k = 0; k < kN; ++k) qp[k] = Fzp[k] = d[k] = Flo[k] = bcast(0.0f);
    float2 sum_l = bcast(0.0f);
    float min_rp = INFINITY;
    int waited = 0;                                     // steps whose slot was waited for

    for (int pi = 0; pi < mine; ++pi) {
        const int64_t patch = patch0 + (int64_t)pi * nwarps;
        const bool has_next = pi + 1 < mine;
        const double h = __ldg(sp.dx + patch);
        const float2 nsc = bcast(-__fdividef(float(__ldg(sp.dt + patch)), 2.0f * float(h)));
        float2 lmax = bcast(0.0f);
#pragma unroll
        for (int s = 0; s < kStepsPerPatch; ++s) {
            // the previous step's output plane, if it made one: plane s - 3 of
            // this patch, or plane 7 of the warp's previous patch
            const bool prev_out = s >= 3 || (s == 0 && pi > 0);
            const int64_t opatch = s == 0 ? patch - nwarps : patch;
            const int ozf = s == 0 ? kP - 1 : s - 3;
            const int obuf = (s + 1) & 1;
            if (prev_out) fence_proxy_async_smem();     // this lane's staging writes -> async proxy
            __syncwarp();                               // slot of step s-1 consumed, staging complete
            if (lane == 0) {
                const int sn = s + kSlots - 1;
                if (sn < kStepsPerPatch) issue(patch, (sn + kP - 1) & (kP - 1), sn % kSlots, 0u);
                else if (has_next) issue(patch + nwarps, (sn - kStepsPerPatch + kP - 1) & (kP - 1), sn % kSlots, 0u);
                if (prev_out) store_middle(opatch, ozf, obuf);
                bulk_wait_read_1();                     // the store before it has read its buffer
            }
            if (prev_out) store_ends(opatch, ozf, obuf);
            // the vote also orders every lane's staging writes below after
            // lane 0's wait above
            if (!__all_sync(0xffffffffu, mbar_wait_bounded(bar0 + 8u * (s % kSlots), (s / kSlots) & 1))) {
                waited = pi * kStepsPerPatch + s;
                goto timeout;
            }

            const int zz = (s + kP - 1) & (kP - 1);
            const unsigned char *sl = slots + (s % kSlots) * G::slot + (G::rows_begin(zz) & 15);
            const S *vA = reinterpret_cast<const S *>(sl + (2 * j) * G::row + (x + 1) * G::vol);
            const S *vB = reinterpret_cast<const S *>(sl + (2 * j + 1) * G::row + (x + 1) * G::vol);
            float2 q[kN];
#pragma unroll
            for (int k = 0; k < kN; ++k) q[k] = make_float2(to_compute(vA[k]), to_compute(vB[k]));

            const Prim2 st = prim2<Pk>(q, g2, gm12);
            float2 Fz[kN];
            flux2<2, Pk>(q, st, Fz);
            const float2 lz = lam2<Pk>(st.u[2], st.c);
            if (s == 0) {                               // plane 7 below plane 0
#pragma unroll
                for (int k = 0; k < kN; ++k) { qp[k] = q[k]; Fzp[k] = Fz[k]; }
                lzp = lz;
                continue;
            }

            // z face below this plane closes the previous plane
            float2 Fzl[kN];
            face2<Pk>(qp, q, Fzp, Fz, lzp, lz, Fzl);
            if (s >= 2) {
                const int zf = s - 2;                   // plane being finished
                float2 qn[kN];
#pragma unroll
                for (int k = 0; k < kN; ++k) qn[k] = A::fma(nsc, A::add(d[k], sub2<Pk>(Fzl[k], Flo[k])), qp[k]);
                // rows 0..7 of the plane (x-halo volumes included) are one
                // contiguous byte range, assembled in staging buffer s & 1
                // laid out like an input slot (range start at offset
                // start mod 16); the lanes of columns 8 and 1 also fill the
                // wrapped x-halo columns 0 and 9
                unsigned char *stg = stg0 + (s & 1) * G::slot + (G::rows_begin(zf) & 15);
                S *ra = reinterpret_cast<S *>(stg + (2 * j) * G::row);
                S *rb = reinterpret_cast<S *>(stg + (2 * j + 1) * G::row);
                store_pair<S>(ra + (x + 1) * kN, rb + (x + 1) * kN, qn);
                if (halo_col >= 0) store_pair<S>(ra + halo_col * kN, rb + halo_col * kN, qn);
                const Prim2 sn = prim2<Pk>(qn, g2, gm12);
                const float2 l = A::add(max2(max2(abs2(sn.u[0]), abs2(sn.u[1])), abs2(sn.u[2])), sn.c);
                lmax = max2(lmax, l);
                sum_l = A::add(sum_l, l);
                min_rp = fminf(min_rp, fminf(fminf(qn[0].x, qn[0].y), fminf(sn.p.x, sn.p.y)));
            }
            if (s == kStepsPerPatch - 1) {              // plane 0 above plane 7: patch done
                const float m = warp_max(fmaxf(lmax.x, lmax.y));
                if (lane == 0) {
                    const double lm = double(m);
                    if (sp.lambda_out) sp.lambda_out[patch] = lm;
                    if (sp.dt_next_out) sp.dt_next_out[patch] = cfl_dt(sp.cfl, h, 3, lm);
                }
                continue;
            }
#pragma unroll
            for (int k = 0; k < kN; ++k) { Flo[k] = Fzl[k]; Fzp[k] = Fz[k]; qp[k] = q[k]; }
            lzp = lz;

            // x faces: right face with lane (x+1) mod 8, left face from lane (x-1) mod 8
            {
                float2 Fx[kN], nq[kN], nF[kN], Fr[kN];
                flux2<0, Pk>(q, st, Fx);
                const float2 lx = lam2<Pk>(st.u[0], st.c);
#pragma unroll
                for (int k = 0; k < kN; ++k) nq[k] = shfl2(q[k], src_r);
                nF[0] = nq[1];
#pragma unroll
                for (int k = 1; k < kN; ++k) nF[k] = shfl2(Fx[k], src_r);
                const float2 nl = shfl2(lx, src_r);
                face2<Pk>(q, nq, Fx, nF, lx, nl, Fr);
#pragma unroll
                for (int k = 0; k < kN; ++k) d[k] = sub2<Pk>(Fr[k], shfl2(Fr[k], src_l));
            }
            // y faces: (row 2j | 2j+1) in the lane, (row 2j+1 | 2j+2) with
            // lane + 8; the face below row 2j is the face above row 2j-1 of
            // lane - 8
            {
                float2 Fy[kN], qR[kN], FR[kN], Fh[kN];
                flux2<1, Pk>(q, st, Fy);
                const float2 ly = lam2<Pk>(st.u[1], st.c);
#pragma unroll
                for (int k = 0; k < kN; ++k) qR[k] = make_float2(q[k].y, __shfl_sync(0xffffffffu, q[k].x, src_u));
                FR[0] = qR[2];
#pragma unroll
                for (int k = 1; k < kN; ++k) FR[k] = make_float2(Fy[k].y, __shfl_sync(0xffffffffu, Fy[k].x, src_u));
                const float2 lR = make_float2(ly.y, __shfl_sync(0xffffffffu, ly.x, src_u));
                face2<Pk>(q, qR, Fy, FR, ly, lR, Fh);
#pragma unroll
                for (int k = 0; k < kN; ++k) {
                    const float2 below = make_float2(__shfl_sync(0xffffffffu, Fh[k].y, src_d), Fh[k].x);
                    d[k] = A::add(d[k], sub2<Pk>(Fh[k], below));
                }
            }
        }
    }
    // the last plane of the warp's last patch
    fence_proxy_async_smem();
    __syncwarp();
    if (lane == 0) store_middle(patch0 + (int64_t)(mine - 1) * nwarps, kP - 1, 1);
    store_ends(patch0 + (int64_t)(mine - 1) * nwarps, kP - 1, 1);
    if (lane == 0) bulk_wait_all();                    // output stores complete, staging free
    {
        const bool bad = !(min_rp > 0.0f) || !(sum_l.x + sum_l.y < INFINITY);
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(sp.flags, FV_FLAG_NONPHYSICAL);
    }
    return;

timeout:
    // the wait for step `waited` ran out: let the output stores finish,
    // drain the loads issued beyond it (bounded), flag the batch, stop
    if (lane == 0) bulk_wait_all();
    {
        const int total = mine * kStepsPerPatch;
        const int issued = total < waited + kSlots ? total : waited + kSlots;
        for (int t = waited; t < issued; ++t)
            mbar_wait_bounded(bar0 + 8u * (unsigned)(t % kSlots), (unsigned)(t / kSlots) & 1u);
    }
    if (lane == 0) atomicOr(sp.flags, FV_FLAG_TIMEOUT);
}

size_t slot_bytes_for(int precision)
{
    return precision == PREC_F32 ? (size_t)Geo<float>::slot : (size_t)Geo<__nv_bfloat16>::slot;
}

size_t smem_bytes_for(int warps, int precision)
{
    return (((size_t)warps * kSlots * 8 + 15) & ~size_t(15)) +
           (size_t)warps * (kSlots + 2) * slot_bytes_for(precision);
}

template <typename S>
cudaError_t launch_p8(const P8Params &sp0, int precision, const FusedShape &shape, cudaStream_t st)
{
    P8Params sp = sp0;
    const int W = std::max(1, std::min(kMaxWarps, shape.warps_per_block > 0 ? shape.warps_per_block : 4));
    const size_t smem = smem_bytes_for(W, precision);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_sweep3d_p8<S, kPacked>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int per_item = (sp.count + W - 1) / W;     // blocks for one patch per warp
    int grid = per_item;
    if (shape.blocks_per_sm > 0) {
        grid = std::min(per_item, shape.blocks_per_sm * num_sms());
    } else if (shape.blocks_per_sm < 0) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sweep3d_p8<S, kPacked>, 32 * W, smem);
        if (e != cudaSuccess) return e;
        grid = std::min(per_item, std::max(1, nb) * num_sms());
    }
    k_sweep3d_p8<S, kPacked><<<grid, 32 * W, smem, st>>>(sp);
    return cudaGetLastError();
}

}  // namespace

bool fused3d_p8_applies(const BatchView &b, int precision, const void *q_in, const void *q_out)
{
    if (b.dim != 3 || b.uniform_p != kP || b.halo_mode != 1 || precision == PREC_F64) return false;
    // bulk copies need 16-byte aligned sources: buffers and patch bases
    const size_t patch_bytes = (size_t)kE * kE * kE * kN * (precision == PREC_F32 ? 4 : 2);
    if (patch_bytes % 16 != 0 || reinterpret_cast<uintptr_t>(q_in) % 16 != 0 ||
        reinterpret_cast<uintptr_t>(q_out) % 16 != 0)
        return false;
    // the bulk copies and stores address device memory only; mapped host
    // buffers (the direct host-state update) take the block kernel's loads
    return is_device_memory(q_in) && is_device_memory(q_out);
}

bool is_device_memory(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return false;
    }
    return true;
}

cudaError_t launch_fused3d_p8(const BatchView &b, int precision, const StepArgs &a, int first, int count,
                              const FusedShape &shape, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    P8Params sp;
    sp.q_in = static_cast<const unsigned char *>(a.q_in);
    sp.q_out = static_cast<unsigned char *>(a.q_out);
    sp.dx = a.dx;
    sp.dt = a.dt;
    sp.lambda_out = a.lambda_out;
    sp.dt_next_out = a.dt_next_out;
    sp.cfl = a.cfl;
    sp.gamma = float(b.gamma);
    sp.gm1 = float(b.gamma - 1.0);
    sp.flags = b.flags;
    sp.first = first;
    sp.count = count;
    sp.extra_tx = b.test_wait_expiry ? 16u : 0u;
    if (precision == PREC_F32) return launch_p8<float>(sp, precision, shape, st);
    return launch_p8<__nv_bfloat16>(sp, precision, shape, st);
}

}  // namespace fv
