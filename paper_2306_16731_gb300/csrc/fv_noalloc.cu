// fv_noalloc.cu -- fv_patch_batch_update_noalloc: one loop-cascade update of
// a batch of equal-size patches that allocates no device memory.
//
// Who needs it: code that cannot call cudaMalloc at the point where it
// wants to advance its patches -- for instance a host callback or a
// library hook that runs while a CUDA graph is being captured (allocation
// is not allowed then), a process whose device memory is entirely owned by
// a pooling allocator it must not bypass, or a plugin that is handed only
// its input and output buffers.  Such a caller cannot create an fv_batch
// (creation reserves device memory for the metadata and the cascade's
// intermediates).
//
// How: the metadata and the cascade's intermediates live in one file-scope
// device array of kNoAllocScratchBytes (64 MiB).  Every GPU that loads this
// library holds that array until the process exits.  Host code cannot use
// the array's name as a device address (in host code it names a host-side
// stand-in), so the first call on each device, with that device current,
// asks the runtime for the array's device address (cudaGetSymbolAddress)
// and caches it; that first call should therefore come before any stream
// capture.  A call with num_patches == 0 (argument checks passed) does that
// lookup and nothing else, so it primes a device cheaply.  Every call
// shares the one array: calls whose work overlaps on the GPU (different
// streams, or different host threads on one device) race and corrupt each
// other's intermediates; serialise them.
#include <algorithm>
#include <mutex>

#include "../../include/fv_batch.h"
#include "fv_common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_symbol_mu;
void *g_symbol_addr[kMaxDevices] = {nullptr};

// Fill the batch metadata of T equal patches of edge p inside the scratch
// array, and clear the error flags (called before each update).
__global__ void k_noalloc_metadata(int dim, int T, int p, int64_t *elem_off, int64_t *cell_off,
                                   int64_t *int_off, int32_t *psize, unsigned *flags)
{
    const int64_t cells = fv::patch_cells(dim, p);
    const int64_t nint = dim == 2 ? (int64_t)p * p : (int64_t)p * p * p;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= T; i += gridDim.x * blockDim.x) {
        elem_off[i] = (int64_t)i * cells * (dim + 2);
        cell_off[i] = (int64_t)i * cells;
        int_off[i] = (int64_t)i * nint;
        if (i < T) psize[i] = p;
        if (i == 0) flags[0] = 0u;
    }
}

int noalloc_fail(int code, const char *msg)
{
    fv::set_last_error(msg);
    return code;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

extern "C" int fv_patch_batch_update_noalloc(int dim, int num_patches, int patch_size, int precision,
                                             int halo_mode, double gamma, const void *Q_in, void *Q_out,
                                             const double *dx, const double *dt, double *lambda_out,
                                             double *dt_next_out, double cfl, void *cuda_stream)
{
    fv::set_last_error("");
    if (dim != 2 && dim != 3) return noalloc_fail(FV_EINVAL, "dim must be 2 or 3");
    if (num_patches < 0) return noalloc_fail(FV_EINVAL, "num_patches must be >= 0");
    if (precision < FV_F64 || precision > FV_BF16_F32) return noalloc_fail(FV_EINVAL, "unknown precision");
    if (halo_mode != FV_HALO_FIXED && halo_mode != FV_HALO_PERIODIC) return noalloc_fail(FV_EINVAL, "unknown halo mode");
    if (!(gamma > 1.0) || !(gamma < 1e300)) return noalloc_fail(FV_EINVAL, "gamma must be finite and > 1");
    if (patch_size < 1 || patch_size > (dim == 2 ? 1024 : 128))
        return noalloc_fail(FV_EINVAL, "patch edge length out of range");
    // the scratch array's device address on the current device: looked up
    // by the first call there (a call with num_patches == 0 does only this)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(FV_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(FV_EUNSUPPORTED, "device index beyond 63");
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_symbol_mu);
        if (!g_symbol_addr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                cudaGetLastError();
                return noalloc_fail(FV_ECUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                               : "no device address for the scratch array");
            }
            g_symbol_addr[dev] = ptr;
        }
        base = static_cast<unsigned char *>(g_symbol_addr[dev]);
    }
    if (num_patches == 0) return FV_OK;
    if (!Q_in || !Q_out || !dx || !dt) return noalloc_fail(FV_EINVAL, "NULL state, dx or dt pointer");
    if ((reinterpret_cast<uintptr_t>(Q_in) | reinterpret_cast<uintptr_t>(Q_out)) & 15u)
        return noalloc_fail(FV_EINVAL, "state buffers must be 16-byte aligned");
    if (dt_next_out && !(cfl > 0.0 && cfl < 1e300)) return noalloc_fail(FV_EINVAL, "cfl must be finite and > 0");

    const int N = dim + 2;
    const size_t es = precision == FV_F64 ? 8 : (precision == FV_F32 ? 4 : 2);
    const int64_t cells = fv::patch_cells(dim, patch_size);
    const size_t state_bytes = (size_t)num_patches * (size_t)cells * N * es;

    // Layout inside the array: offsets, sizes, flags, then the cascade's
    // intermediates.
    const size_t n1 = (size_t)num_patches + 1;
    const size_t off_elem = 0, off_cell = off_elem + 8 * n1, off_int = off_cell + 8 * n1;
    const size_t off_ps = off_int + 8 * n1;
    const size_t off_flags = align256(off_ps + 4 * (size_t)num_patches);
    const size_t off_cascade = align256(off_flags + 16);

    fv::BatchView v{};
    v.dim = dim;
    v.num_patches = num_patches;
    v.halo_mode = halo_mode;
    v.gamma = gamma;
    v.total_cells = (int64_t)num_patches * cells;
    v.total_interior = (int64_t)num_patches * (dim == 2 ? (int64_t)patch_size * patch_size
                                                        : (int64_t)patch_size * patch_size * patch_size);
    v.max_p = patch_size;
    v.uniform_p = patch_size;
    v.align_bytes = 1;
    const size_t need = off_cascade + fv::cascade_scratch_bytes(v, precision);
    if (need > kNoAllocScratchBytes)
        return noalloc_fail(FV_EINVAL, "batch needs more than the 64 MiB of built-in scratch; "
                                       "use fv_batch_create / fv_patch_batch_update");
    {
        uintptr_t a = reinterpret_cast<uintptr_t>(Q_in), b = reinterpret_cast<uintptr_t>(Q_out);
        if (a < b + state_bytes && b < a + state_bytes)
            return noalloc_fail(FV_EINVAL, "Q_in and Q_out overlap (in-place update is not allowed)");
    }

    v.elem_off = reinterpret_cast<const int64_t *>(base + off_elem);
    v.cell_off = reinterpret_cast<const int64_t *>(base + off_cell);
    v.int_off = reinterpret_cast<const int64_t *>(base + off_int);
    v.psize = reinterpret_cast<const int32_t *>(base + off_ps);
    v.flags = reinterpret_cast<unsigned *>(base + off_flags);

    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int threads = 256;
    const int grid = (int)std::min<int64_t>((num_patches + threads) / threads, 4096);
    k_noalloc_metadata<<<grid, threads, 0, st>>>(dim, num_patches, patch_size,
                                                 reinterpret_cast<int64_t *>(base + off_elem),
                                                 reinterpret_cast<int64_t *>(base + off_cell),
                                                 reinterpret_cast<int64_t *>(base + off_int),
                                                 reinterpret_cast<int32_t *>(base + off_ps),
                                                 reinterpret_cast<unsigned *>(base + off_flags));
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(FV_ECUDA, cudaGetErrorString(e));

    fv::CascadeScratch cs{};
    fv::cascade_scratch_carve(base + off_cascade, v, precision, &cs);
    fv::StepArgs a{Q_in, Q_out, dx, dt, lambda_out, dt_next_out, cfl};
    e = fv::launch_cascade_update(v, precision, a, cs, st, fv::CASCADE_AOS);
    if (e != cudaSuccess) return noalloc_fail(FV_ECUDA, cudaGetErrorString(e));
    return FV_OK;
}
