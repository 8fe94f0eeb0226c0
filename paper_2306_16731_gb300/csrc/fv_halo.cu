// fv_halo.cu -- face-halo fill from neighbouring patches of the batch: the
// step that precedes the kernel call in the paper's framework, which equips
// every patch with a halo layer of width one before the update
// (arXiv:2306.16731, Sec. 2.2).  Each face with a neighbour receives the
// neighbour's interior volumes that touch the face (across -x the
// neighbour's column p-1, across +x its column 0, likewise in y and z);
// corner and edge halo volumes are not written (the update never reads
// them).  One thread per halo face volume; rows along x are contiguous, so
// the y and z faces copy coalesced runs.
#include "fv_common.cuh"

namespace fv {

namespace {

constexpr int kThreads = 256;

template <int D, typename S>
__global__ void __launch_bounds__(kThreads) k_halo_exchange(BatchView b, const int32_t *__restrict__ nbr, S *q)
{
    constexpr int N = D + 2;
    const int i = blockIdx.x;                       // one block per patch
    const int P = __ldg(b.psize + i), E = P + 2;
    const int per_face = D == 2 ? P : P * P;
    const int64_t base = __ldg(b.elem_off + i);
    for (int w = threadIdx.x; w < 2 * D * per_face; w += blockDim.x) {
        const int face = w / per_face, t = w - face * per_face;
        const int j = __ldg(nbr + (int64_t)i * 2 * D + face);
        if (j < 0) continue;
        const int axis = face >> 1, upper = face & 1;
        const int ta = t % P, tb = D == 2 ? 0 : t / P;    // tangential coordinates
        int dc[3], sc[3];
        int tt = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) {
            if (a == axis) {
                dc[a] = upper ? P : -1;
                sc[a] = upper ? 0 : P - 1;
            } else {
                dc[a] = tt == 0 ? ta : tb;
                sc[a] = dc[a];
                ++tt;
            }
        }
        const int64_t dcell = D == 2 ? (int64_t)(dc[1] + 1) * E + (dc[0] + 1)
                                     : ((int64_t)(dc[2] + 1) * E + (dc[1] + 1)) * E + (dc[0] + 1);
        const int64_t scell = D == 2 ? (int64_t)(sc[1] + 1) * E + (sc[0] + 1)
                                     : ((int64_t)(sc[2] + 1) * E + (sc[1] + 1)) * E + (sc[0] + 1);
        const S *src = q + __ldg(b.elem_off + j) + scell * N;
        S *dst = q + base + dcell * N;
#pragma unroll
        for (int k = 0; k < N; ++k) dst[k] = src[k];
    }
}

}  // namespace

cudaError_t launch_halo_exchange(const BatchView &b, int precision, const int32_t *nbr, void *q, cudaStream_t st)
{
    if (b.num_patches == 0) return cudaSuccess;
    FV_DISPATCH(b.dim, precision, {
        k_halo_exchange<D, S><<<b.num_patches, kThreads, 0, st>>>(b, nbr, static_cast<S *>(q));
    });
    return cudaGetLastError();
}

}  // namespace fv
