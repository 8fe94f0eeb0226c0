// fv_scatter.cu -- patches kept as separate host allocations (the paper's
// framework holds each patch on the heap and its run time is dominated by
// moving them to the accelerator and back, Sec. 4 "Data transfer", Sec. 5
// Fig. 4).  On Grace-Blackwell page-locked host memory is addressable from
// the GPU, so the gather of the scattered patches into the batch's device
// layout and the scatter of the updated interiors back are kernels that read
// and write host memory over the coherent link: one block per patch, no
// per-patch copy call.
#include "fv_common.cuh"

namespace fv {

namespace {

constexpr int kThreads = 256;

// Largest of 16, 8, 4, 2, 1 dividing both addresses and the byte count.
__device__ __forceinline__ int common_align(uintptr_t a, uintptr_t b, size_t n)
{
    const uintptr_t m = a | b | (uintptr_t)n;
    return (m & 15) == 0 ? 16 : ((m & 7) == 0 ? 8 : ((m & 3) == 0 ? 4 : ((m & 1) == 0 ? 2 : 1)));
}

__device__ __forceinline__ void copy_bytes(unsigned char *d, const unsigned char *s, size_t n)
{
    const int a = common_align(reinterpret_cast<uintptr_t>(d), reinterpret_cast<uintptr_t>(s), n);
    if (a == 16) {
        for (size_t i = threadIdx.x; i < n / 16; i += blockDim.x)
            reinterpret_cast<uint4 *>(d)[i] = reinterpret_cast<const uint4 *>(s)[i];
    } else if (a == 8) {
        for (size_t i = threadIdx.x; i < n / 8; i += blockDim.x)
            reinterpret_cast<uint2 *>(d)[i] = reinterpret_cast<const uint2 *>(s)[i];
    } else if (a == 4) {
        for (size_t i = threadIdx.x; i < n / 4; i += blockDim.x)
            reinterpret_cast<unsigned *>(d)[i] = reinterpret_cast<const unsigned *>(s)[i];
    } else if (a == 2) {
        for (size_t i = threadIdx.x; i < n / 2; i += blockDim.x)
            reinterpret_cast<unsigned short *>(d)[i] = reinterpret_cast<const unsigned short *>(s)[i];
    } else {
        for (size_t i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
    }
}

// Patch i (halo-inclusive, N (p+2)^d values) from src[i] to its place in the
// batch buffer dst.
__global__ void __launch_bounds__(kThreads) k_gather(BatchView b, const unsigned char *const *__restrict__ src,
                                                     unsigned char *__restrict__ dst, int es)
{
    for (int i = blockIdx.x; i < b.num_patches; i += gridDim.x) {
        const int64_t e0 = __ldg(b.elem_off + i), e1 = __ldg(b.elem_off + i + 1);
        copy_bytes(dst + e0 * es, src[i], (size_t)(e1 - e0) * es);
    }
}

// The interior volumes of patch i from the batch buffer src to dst[i], one
// interior row of p volumes at a time; halo volumes of dst[i] are not written.
__global__ void __launch_bounds__(kThreads) k_scatter_interior(BatchView b, const unsigned char *__restrict__ src,
                                                               unsigned char *const *__restrict__ dst, int es)
{
    const int N = b.dim + 2;
    for (int i = blockIdx.x; i < b.num_patches; i += gridDim.x) {
        const int p = __ldg(b.psize + i);
        const int64_t e = p + 2;
        const int rows = b.dim == 2 ? p : p * p;
        const size_t row_bytes = (size_t)p * N * es;
        const unsigned char *s0 = src + __ldg(b.elem_off + i) * es;
        unsigned char *d0 = dst[i];
        // one warp per row
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int r = warp; r < rows; r += nw) {
            const int y = r % p, z = b.dim == 2 ? 0 : r / p;
            const int64_t cell = b.dim == 2 ? (int64_t)(y + 1) * e + 1 : ((int64_t)(z + 1) * e + (y + 1)) * e + 1;
            const unsigned char *s = s0 + cell * N * es;
            unsigned char *d = d0 + cell * N * es;
            const int a = common_align(reinterpret_cast<uintptr_t>(d), reinterpret_cast<uintptr_t>(s), row_bytes);
            if (a >= 4) {
                for (size_t k = lane; k < row_bytes / 4; k += 32)
                    reinterpret_cast<unsigned *>(d)[k] = reinterpret_cast<const unsigned *>(s)[k];
            } else {
                for (size_t k = lane; k < row_bytes / 2; k += 32)
                    reinterpret_cast<unsigned short *>(d)[k] = reinterpret_cast<const unsigned short *>(s)[k];
            }
        }
    }
}

}  // namespace

cudaError_t launch_gather_patches(const BatchView &b, const void *const *src, void *dst, int es, cudaStream_t st)
{
    if (b.num_patches == 0) return cudaSuccess;
    const int grid = b.num_patches < 65535 ? b.num_patches : 65535;
    k_gather<<<grid, kThreads, 0, st>>>(b, reinterpret_cast<const unsigned char *const *>(src),
                                        static_cast<unsigned char *>(dst), es);
    return cudaGetLastError();
}

cudaError_t launch_scatter_interiors(const BatchView &b, const void *src, void *const *dst, int es, cudaStream_t st)
{
    if (b.num_patches == 0) return cudaSuccess;
    const int grid = b.num_patches < 65535 ? b.num_patches : 65535;
    k_scatter_interior<<<grid, kThreads, 0, st>>>(b, static_cast<const unsigned char *>(src),
                                                  reinterpret_cast<unsigned char *const *>(dst), es);
    return cudaGetLastError();
}

}  // namespace fv
