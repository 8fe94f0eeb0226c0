// fv_batch.cu -- the C ABI declared in include/fv_batch.h: batch object,
// argument validation, metadata upload, form selection, dispatch to the
// kernel launchers, device-side CFL chaining over many steps with CUDA-graph
// capture, the launch-shape autotuner and error reporting.
//
// The batch follows the paper's "managed memory" idiom (arXiv:2306.16731,
// Sec. 4 "Data transfer"): device memory is reserved once at creation and
// recycled by every later call; no call after creation allocates.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <atomic>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/fv_batch.h"
#include "fv_internal.h"
#include "fv_physics.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    // clear the runtime's last-error state, so that a failed call does not
    // surface again at the caller's next, unrelated CUDA call
    cudaGetLastError();
    return fail(FV_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr int kMaxEdge2D = 1024;
constexpr int kMaxEdge3D = 128;

struct GraphKey {
    const void *qa, *qb, *dx;
    const double *dta, *dtb, *lam;
    int steps;
    double cfl;
    int form;
    bool operator<(const GraphKey &o) const
    {
        return std::tie(qa, qb, dx, dta, dtb, lam, steps, cfl, form) <
               std::tie(o.qa, o.qb, o.dx, o.dta, o.dtb, o.lam, o.steps, o.cfl, o.form);
    }
};

}  // namespace

struct fv_batch {
    int device = 0;
    int dim = 2, T = 0, precision = 0, halo_mode = 0;
    double gamma = 1.4;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    int form = FV_FORM_FUSED;
    int cascade_layout = FV_LAYOUT_AOS;

    std::vector<int32_t> psize;
    std::vector<int64_t> elem_off, cell_off, int_off;
    int64_t state_elems = 0;

    void *meta = nullptr;              // device metadata block
    fv::BatchView view{};

    void *scratch = nullptr;           // cascade intermediates
    size_t scratch_bytes = 0;
    fv::CascadeScratch cs{};

    int fused_kernel = fv::FUSED_NONE;
    fv::FusedPlan plan{};
    std::vector<fv::WorkItem> items_h;

    std::map<GraphKey, cudaGraphExec_t> graphs;

    int32_t *nbr = nullptr;            // device neighbour table (fv_batch_set_neighbours)

    // host-state updates (fv_patch_batch_update_host): device staging and
    // the copy streams, created by the first such call
    void *hs_in = nullptr, *hs_out = nullptr;
    double *hs_arrays = nullptr;       // dx, dt, lambda, dt_next (T each)
    cudaStream_t hs_copy_in = nullptr, hs_copy_out = nullptr;
    std::vector<cudaEvent_t> hs_events;

    // scattered host patches (fv_batch_set_host_patches): device table of
    // device-visible addresses [in T | out T] and the host addresses
    void **sp_table = nullptr;
    std::vector<void *> sp_in, sp_out;
};

namespace fv {

void set_last_error(const char *msg) { g_last_error = msg ? msg : ""; }

int num_sms()
{
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cache[dev] = n;
    return n;
}

}  // namespace fv

namespace {

size_t elem_bytes(int precision) { return precision == FV_F64 ? 8 : (precision == FV_F32 ? 4 : 2); }

// RAII: make the batch's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
        if (!ok) cudaGetLastError();      // reported by the caller as FV_ECUDA
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Device allocations of the batch object go through here, so that a test
// can make the k-th one fail (fv_test_fail_device_alloc) and check that every
// call returns FV_ENOMEM cleanly.
std::atomic<int> g_fail_alloc_countdown{0};

cudaError_t dev_alloc(void **p, size_t bytes)
{
    int k = g_fail_alloc_countdown.load();
    while (k > 0) {
        if (g_fail_alloc_countdown.compare_exchange_weak(k, k - 1)) {
            if (k == 1) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

// Handles returned by fv_batch_create and not yet destroyed.
std::mutex g_live_mu;
std::set<const void *> g_live;

bool overlaps(const void *a, const void *b, size_t bytes)
{
    uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + bytes && y < x + bytes;
}

int ensure_scratch(fv_batch *b)
{
    if (b->scratch || b->T == 0) return FV_OK;
    size_t bytes = fv::cascade_scratch_bytes(b->view, b->precision);
    void *p = nullptr;
    cudaError_t e = dev_alloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FV_ENOMEM, "cascade scratch of %zu bytes: %s", bytes, cudaGetErrorString(e));
    }
    b->scratch = p;
    b->scratch_bytes = bytes;
    fv::cascade_scratch_carve(p, b->view, b->precision, &b->cs);
    return FV_OK;
}

void drop_graphs(fv_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

// Build the fused sweep work list: patches grouped by edge length (largest
// first), groups cut into items of fv::fused_items_for() patches.
void build_work_list(fv_batch *b, std::vector<int32_t> &order, std::vector<fv::WorkItem> &items)
{
    order.resize(b->T);
    for (int i = 0; i < b->T; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int c) { return b->psize[a] > b->psize[c]; });
    items.clear();
    int i = 0;
    while (i < b->T) {
        int p = b->psize[order[i]];
        int per = 1;
        fv::fused_items_for(b->dim, p, &per);
        int j = i;
        while (j < b->T && b->psize[order[j]] == p) ++j;
        for (int s = i; s < j; s += per) {
            fv::WorkItem w;
            w.first_patch = s;
            w.count = (int16_t)std::min(per, j - s);
            w.p = (int16_t)p;
            items.push_back(w);
        }
        i = j;
    }
}

}  // namespace

extern "C" {

const char *fv_last_error(void) { return g_last_error.c_str(); }

static int create_batch(fv_batch_t **out, int pde, int dim, int num_patches, const int32_t *patch_size,
                        int halo, int unknowns, int precision, int halo_mode, double p0, double p1,
                        void *cuda_stream)
{
    g_last_error.clear();
    if (!out) return fail(FV_EINVAL, "out is NULL");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(FV_EINVAL, "dim must be 2 or 3 (got %d)", dim);
    if (num_patches < 0) return fail(FV_EINVAL, "num_patches must be >= 0 (got %d)", num_patches);
    if (num_patches > 0 && !patch_size) return fail(FV_EINVAL, "patch_size is NULL");
    if (halo != 1) return fail(FV_EINVAL, "halo width must be 1 (got %d)", halo);
    if (precision < FV_F64 || precision > FV_BF16_F32) return fail(FV_EINVAL, "unknown precision %d", precision);
    if (halo_mode != FV_HALO_FIXED && halo_mode != FV_HALO_PERIODIC)
        return fail(FV_EINVAL, "unknown halo mode %d", halo_mode);
    const double gamma = pde == FV_PDE_EULER ? p0 : 1.4;
    if (pde == FV_PDE_EULER) {
        if (unknowns != dim + 2) return fail(FV_EINVAL, "Euler in %dD has %d unknowns (got %d)", dim, dim + 2, unknowns);
        if (!(gamma > 1.0) || !(gamma < 1e300)) return fail(FV_EINVAL, "gamma must be finite and > 1");
    } else if (pde == FV_PDE_SHALLOW_WATER) {
        if (dim != 2) return fail(FV_EINVAL, "the shallow water equations are two-dimensional (got dim %d)", dim);
        if (unknowns != 4) return fail(FV_EINVAL, "shallow water has 4 unknowns (h, hu, hv, b)");
        if (precision == FV_BF16_F32) return fail(FV_EUNSUPPORTED, "shallow water: FP64 or FP32 storage only");
        if (!(p0 > 0.0) || !(p0 < 1e300)) return fail(FV_EINVAL, "gravity g must be finite and > 0");
        if (!(p1 > -1e300 && p1 < 1e300)) return fail(FV_EINVAL, "Coriolis parameter f must be finite");
    } else {
        return fail(FV_EINVAL, "unknown PDE %d", pde);
    }
    const int max_edge = dim == 2 ? kMaxEdge2D : kMaxEdge3D;
    for (int i = 0; i < num_patches; ++i)
        if (patch_size[i] < 1 || patch_size[i] > max_edge)
            return fail(FV_EINVAL, "patch %d: edge length %d outside [1, %d]", i, patch_size[i], max_edge);

    fv_batch *b = new (std::nothrow) fv_batch;
    if (!b) return fail(FV_ENOMEM, "host allocation");
    cudaGetDevice(&b->device);
    b->dim = dim;
    b->T = num_patches;
    b->precision = precision;
    b->halo_mode = halo_mode;
    b->gamma = gamma;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->psize.assign(patch_size, patch_size + num_patches);
    b->elem_off.resize(num_patches + 1);
    b->cell_off.resize(num_patches + 1);
    b->int_off.resize(num_patches + 1);
    b->elem_off[0] = b->cell_off[0] = b->int_off[0] = 0;
    int max_p = 0, uni = num_patches > 0 ? patch_size[0] : 0;
    for (int i = 0; i < num_patches; ++i) {
        int64_t p = patch_size[i];
        int64_t cells = fv::patch_cells(dim, (int)p);
        int64_t nint = dim == 2 ? p * p : p * p * p;
        b->cell_off[i + 1] = b->cell_off[i] + cells;
        b->elem_off[i + 1] = b->elem_off[i] + cells * (dim + 2);
        b->int_off[i + 1] = b->int_off[i] + nint;
        max_p = std::max<int>(max_p, (int)p);
        if (patch_size[i] != uni) uni = 0;
    }
    b->state_elems = b->elem_off[num_patches];
    int align = 16;
    {
        const size_t es = elem_bytes(precision);
        auto pow2 = [](size_t v) { int a = 16; while (a > 1 && v % a != 0) a >>= 1; return a; };
        for (int i = 0; i < num_patches; ++i) {
            const size_t e = (size_t)patch_size[i] + 2;
            align = std::min(align, pow2((size_t)fv::patch_cells(dim, patch_size[i]) * (dim + 2) * es));
            if (dim == 3) align = std::min(align, pow2(e * e * (dim + 2) * es));
        }
    }

    // Fused work list (host side first, uploaded with the metadata).
    std::vector<int32_t> order;
    int fk = fv::FUSED_NONE;
    fv::BatchView probe{};
    probe.dim = dim;
    probe.num_patches = num_patches;
    probe.max_p = max_p;
    probe.uniform_p = uni;
    probe.halo_mode = halo_mode;
    probe.align_bytes = align;
    probe.pde = pde == FV_PDE_SHALLOW_WATER ? fv::PDE_SHALLOW_WATER : fv::PDE_EULER;
    if (pde == FV_PDE_EULER && num_patches > 0 && fv::fused_supported(probe, precision, &fk))
        build_work_list(b, order, b->items_h);
    else if (pde != FV_PDE_EULER && fv::pde_fused_supported(probe, precision, patch_size)) {
        fk = fv::FUSED_SWEEP_PDE;
        build_work_list(b, order, b->items_h);
    }
    b->fused_kernel = fk;

    // One device block: offsets, sizes, flags, work list, order, counter.
    const size_t n1 = (size_t)num_patches + 1;
    size_t off_elem = 0, off_cell = off_elem + 8 * n1, off_int = off_cell + 8 * n1;
    size_t off_ps = off_int + 8 * n1;
    size_t off_flags = (off_ps + 4 * (size_t)num_patches + 15) & ~(size_t)15;
    size_t off_items = off_flags + 16;
    size_t off_order = off_items + sizeof(fv::WorkItem) * b->items_h.size();
    size_t off_ctr = (off_order + 4 * order.size() + 15) & ~(size_t)15;
    size_t total = off_ctr + 8 * fv::kMaxSizeClasses;
    std::vector<unsigned char> host(total, 0);
    memcpy(host.data() + off_elem, b->elem_off.data(), 8 * n1);
    memcpy(host.data() + off_cell, b->cell_off.data(), 8 * n1);
    memcpy(host.data() + off_int, b->int_off.data(), 8 * n1);
    if (num_patches) memcpy(host.data() + off_ps, b->psize.data(), 4 * (size_t)num_patches);
    if (!b->items_h.empty()) memcpy(host.data() + off_items, b->items_h.data(), sizeof(fv::WorkItem) * b->items_h.size());
    if (!order.empty()) memcpy(host.data() + off_order, order.data(), 4 * order.size());

    cudaError_t e = dev_alloc(&b->meta, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(FV_ENOMEM, "metadata (%zu bytes): %s", total, cudaGetErrorString(e));
    }
    e = cudaMemcpy(b->meta, host.data(), total, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "batch set-up");
        cudaFree(b->meta);
        delete b;
        return rc;
    }
    unsigned char *m = static_cast<unsigned char *>(b->meta);
    fv::BatchView &v = b->view;
    v.dim = dim;
    v.num_patches = num_patches;
    v.halo_mode = halo_mode;
    v.gamma = gamma;
    v.elem_off = reinterpret_cast<const int64_t *>(m + off_elem);
    v.cell_off = reinterpret_cast<const int64_t *>(m + off_cell);
    v.int_off = reinterpret_cast<const int64_t *>(m + off_int);
    v.psize = reinterpret_cast<const int32_t *>(m + off_ps);
    v.flags = reinterpret_cast<unsigned *>(m + off_flags);
    v.total_cells = b->cell_off[num_patches];
    v.total_interior = b->int_off[num_patches];
    v.max_p = max_p;
    v.uniform_p = uni;
    v.align_bytes = align;
    v.pde = pde == FV_PDE_SHALLOW_WATER ? fv::PDE_SHALLOW_WATER : fv::PDE_EULER;
    v.pde_param[0] = p0;
    v.pde_param[1] = p1;
    b->plan.items = reinterpret_cast<const fv::WorkItem *>(m + off_items);
    b->plan.order = reinterpret_cast<const int32_t *>(m + off_order);
    b->plan.num_items = (int)b->items_h.size();
    b->plan.work_counter = reinterpret_cast<unsigned *>(m + off_ctr);
    b->plan.kernel = fk;
    b->plan.num_classes = 0;
    for (size_t k = 0; k < b->items_h.size(); ++k) {
        int p = b->items_h[k].p;
        int &nc = b->plan.num_classes;
        if (nc == 0 || b->plan.class_p[nc - 1] != p) {
            b->plan.class_p[nc] = p;
            b->plan.class_begin[nc] = (int)k;
            ++nc;
        }
        b->plan.class_end[nc - 1] = (int)k + 1;
    }
    b->plan.shape.warps_per_block = 4;
    b->plan.shape.blocks_per_sm = 0;
    b->plan.shape.ring = 0;

    // Default form: fused sweep if the library has a kernel for the shapes, else the
    // patch-wise tile kernel, else the loop cascade.  Other PDEs than Euler
    // run on the generic fused sweep (edges 4, 8, 16, 32) or the generic
    // patch-wise kernel.
    if (pde != FV_PDE_EULER) {
        if (fk == fv::FUSED_SWEEP_PDE) {
            b->form = FV_FORM_FUSED;
        } else if (num_patches > 0 && !fv::pde_tile_supported(v, precision)) {
            cudaStreamDestroy(b->capture_stream);
            cudaFree(b->meta);
            delete b;
            return fail(FV_EUNSUPPORTED, "generic PDE kernel: patch too large for shared memory");
        } else {
            b->form = FV_FORM_TILE;
        }
    } else if (fk != fv::FUSED_NONE) b->form = FV_FORM_FUSED;
    else if (num_patches == 0 || fv::tile_supported(v, precision)) b->form = FV_FORM_TILE;
    else {
        b->form = FV_FORM_CASCADE;
        int rc = ensure_scratch(b);
        if (rc) {
            cudaStreamDestroy(b->capture_stream);
            cudaFree(b->meta);
            delete b;
            return rc;
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        g_live.insert(b);
    }
    *out = b;
    return FV_OK;
}

int fv_batch_create(fv_batch_t **out, int dim, int num_patches, const int32_t *patch_size,
                    int halo, int unknowns, int precision, int halo_mode, double gamma,
                    void *cuda_stream)
{
    return create_batch(out, FV_PDE_EULER, dim, num_patches, patch_size, halo, unknowns, precision, halo_mode,
                        gamma, 0.0, cuda_stream);
}

int fv_test_fail_device_alloc(int k)
{
    g_fail_alloc_countdown.store(k > 0 ? k : 0);
    return FV_OK;
}

int fv_batch_create_pde(fv_batch_t **out, int pde, int dim, int num_patches, const int32_t *patch_size,
                        int precision, int halo_mode, const double *params, int num_params, void *cuda_stream)
{
    g_last_error.clear();
    if (out) *out = nullptr;
    if (pde == FV_PDE_EULER) {
        if (!params || num_params != 1) return fail(FV_EINVAL, "Euler takes one parameter (gamma)");
        return create_batch(out, pde, dim, num_patches, patch_size, 1, dim + 2, precision, halo_mode, params[0],
                            0.0, cuda_stream);
    }
    if (pde == FV_PDE_SHALLOW_WATER) {
        if (!params || num_params != 2) return fail(FV_EINVAL, "shallow water takes two parameters (g, f)");
        return create_batch(out, pde, dim, num_patches, patch_size, 1, 4, precision, halo_mode, params[0],
                            params[1], cuda_stream);
    }
    return fail(FV_EINVAL, "unknown PDE %d", pde);
}

int fv_batch_set_form(fv_batch_t *b, int form)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    if (b->view.pde != fv::PDE_EULER && form != FV_FORM_TILE && form != FV_FORM_FUSED)
        return fail(FV_EUNSUPPORTED, "this PDE runs on the generic fused sweep or patch-wise kernel only");
    if (b->view.pde != fv::PDE_EULER && form == FV_FORM_TILE && b->T > 0 && !fv::pde_tile_supported(b->view, b->precision))
        return fail(FV_EUNSUPPORTED, "generic PDE kernel: patch too large for shared memory");
    if (form == FV_FORM_CASCADE || form == FV_FORM_TASKGRAPH) {
        int rc = ensure_scratch(b);
        if (rc) return rc;
    } else if (form == FV_FORM_TILE) {
        if (b->view.pde == fv::PDE_EULER && b->T > 0 && !fv::tile_supported(b->view, b->precision))
            return fail(FV_EUNSUPPORTED, "patch-wise tile kernel: patch too large for shared memory");
    } else if (form == FV_FORM_FUSED) {
        if (b->T > 0 && b->fused_kernel == fv::FUSED_NONE)
            return fail(FV_EUNSUPPORTED, "no fused kernel for these patch shapes/precision");
    } else {
        return fail(FV_EINVAL, "unknown form %d", form);
    }
    if (b->form != form) drop_graphs(b);
    b->form = form;
    return FV_OK;
}

int fv_batch_set_neighbours(fv_batch_t *b, const int32_t *neighbours)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    if (!neighbours) {
        if (b->nbr) cudaFree(b->nbr);
        b->nbr = nullptr;
        b->view.nbr = nullptr;
        drop_graphs(b);
        return FV_OK;
    }
    const int faces = 2 * b->dim;
    for (int i = 0; i < b->T; ++i)
        for (int f = 0; f < faces; ++f) {
            const int j = neighbours[(size_t)i * faces + f];
            if (j < -1 || j >= b->T)
                return fail(FV_EINVAL, "patch %d face %d: neighbour %d out of range", i, f, j);
            if (j >= 0 && b->psize[j] != b->psize[i])
                return fail(FV_EINVAL, "patch %d face %d: neighbour %d has edge %d, not %d", i, f, j, b->psize[j],
                            b->psize[i]);
        }
    const size_t bytes = (size_t)b->T * faces * sizeof(int32_t);
    if (!b->nbr && bytes) {
        void *p = nullptr;
        cudaError_t e = dev_alloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(FV_ENOMEM, "neighbour table: %s", cudaGetErrorString(e));
        }
        b->nbr = static_cast<int32_t *>(p);
    }
    if (bytes) {
        cudaError_t e = cudaMemcpy(b->nbr, neighbours, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "neighbour table upload");
    }
    b->view.nbr = b->nbr;
    drop_graphs(b);
    return FV_OK;
}

int fv_halo_exchange(fv_batch_t *b, void *Q)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    if (b->T == 0) return FV_OK;
    if (!b->view.nbr) return fail(FV_EINVAL, "no neighbour table registered (fv_batch_set_neighbours)");
    if (!Q) return fail(FV_EINVAL, "state pointer is NULL");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    cudaError_t e = fv::launch_halo_exchange(b->view, b->precision, b->view.nbr, Q, b->stream);
    return e == cudaSuccess ? FV_OK : cuda_fail(e, "halo exchange launch");
}

int fv_batch_set_launch_shape(fv_batch_t *b, int warps_per_block, int blocks_per_sm)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    if (warps_per_block < 1 || warps_per_block > 16) return fail(FV_EINVAL, "warps_per_block must be in [1, 16]");
    if (blocks_per_sm < -2 || blocks_per_sm > 32) return fail(FV_EINVAL, "blocks_per_sm must be in [-2, 32]");
    b->plan.shape = fv::FusedShape{warps_per_block, blocks_per_sm, b->plan.shape.ring};
    drop_graphs(b);
    return FV_OK;
}

int fv_batch_set_sweep_ring(fv_batch_t *b, int rows)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    if (rows != 0 && rows != 4 && rows != 6 && rows != 8) return fail(FV_EINVAL, "ring depth must be 0, 4, 6 or 8");
    if (rows == 8) rows = 0;                 // the default depth
    if (rows != 0 && !(b->fused_kernel == fv::FUSED_SWEEP2D && fv::sweep_ring_applies(b->view, b->precision)))
        return fail(FV_EUNSUPPORTED, "the ring depth is chosen for uniform 2D FP32/BF16 batches of edge 4, 8, 16 "
                                     "or 32 only");
    if (b->plan.shape.ring != rows) drop_graphs(b);
    b->plan.shape.ring = rows;
    return FV_OK;
}

int fv_batch_set_cascade_layout(fv_batch_t *b, int layout)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    if (layout != FV_LAYOUT_AOS && layout != FV_LAYOUT_SOA && layout != FV_LAYOUT_AOSOA)
        return fail(FV_EINVAL, "unknown cascade layout %d", layout);
    if (b->cascade_layout != layout) drop_graphs(b);
    b->cascade_layout = layout;
    return FV_OK;
}

int fv_batch_test_wait_expiry(fv_batch_t *b, int enable)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    b->view.test_wait_expiry = enable ? 1 : 0;
    drop_graphs(b);
    return FV_OK;
}

int fv_batch_set_stream(fv_batch_t *b, void *cuda_stream)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    return FV_OK;
}

// Task-graph form: build and instantiate the per-patch graph of this buffer
// set on first use (cached with the batch's graphs), then launch it.
static int launch_taskgraph(fv_batch_t *b, cudaStream_t st, const fv::StepArgs &a)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return cuda_fail(e, "capture query");
    if (cs != cudaStreamCaptureStatusNone)
        return fail(FV_EUNSUPPORTED, "the task-graph form is itself a graph and cannot be stream-captured");
    GraphKey key{a.q_in, a.q_out, a.dx, a.dt, a.dt_next_out, a.lambda_out, -1, a.cfl, FV_FORM_TASKGRAPH};
    auto it = b->graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    if (it != b->graphs.end()) {
        exec = it->second;
    } else {
        cudaGraph_t graph = nullptr;
        e = cudaGraphCreate(&graph, 0);
        if (e != cudaSuccess) return cuda_fail(e, "graph create");
        e = fv::build_cascade_taskgraph(b->view, b->cell_off.data(), b->precision, a, b->cs, b->cascade_layout, graph);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "task graph build");
        b->graphs[key] = exec;
    }
    e = cudaGraphLaunch(exec, st);
    return e == cudaSuccess ? FV_OK : cuda_fail(e, "task graph launch");
}

static int launch_update(fv_batch_t *b, cudaStream_t st, const void *Q_in, void *Q_out,
                         const double *dx, const double *dt, double *lambda_out,
                         double *dt_next_out, double cfl)
{
    if (b->T == 0) return FV_OK;
    fv::StepArgs a{Q_in, Q_out, dx, dt, lambda_out, dt_next_out, cfl};
    cudaError_t e;
    switch (b->form) {
    case FV_FORM_CASCADE:
        e = fv::launch_cascade_update(b->view, b->precision, a, b->cs, st, b->cascade_layout);
        break;
    case FV_FORM_TASKGRAPH: return launch_taskgraph(b, st, a);
    case FV_FORM_TILE:
        e = b->view.pde == fv::PDE_EULER ? fv::launch_tile_update(b->view, b->precision, a, st)
                                         : fv::launch_pde_update(b->view, b->precision, a, st);
        break;
    default:
        e = b->plan.kernel == fv::FUSED_SWEEP_PDE ? fv::launch_pde_fused_update(b->view, b->precision, a, b->plan, st)
                                                  : fv::launch_fused_update(b->view, b->precision, a, b->plan, st);
        break;
    }
    if (e != cudaSuccess) return cuda_fail(e, "update launch");
    return FV_OK;
}

static int check_update_args(fv_batch_t *b, const void *Q_in, const void *Q_out, const double *dx,
                             const double *dt, const double *dt_next_out, double cfl)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    if (b->T == 0) return FV_OK;
    if (!Q_in || !Q_out) return fail(FV_EINVAL, "state pointer is NULL");
    if (!dx || !dt) return fail(FV_EINVAL, "dx/dt pointer is NULL");
    if (!aligned16(Q_in) || !aligned16(Q_out)) return fail(FV_EINVAL, "state buffers must be 16-byte aligned");
    size_t bytes = (size_t)b->state_elems * elem_bytes(b->precision);
    if (overlaps(Q_in, Q_out, bytes)) return fail(FV_EINVAL, "Q_in and Q_out overlap (in-place update is not allowed)");
    if (dt_next_out && !(cfl > 0.0 && cfl < 1e300)) return fail(FV_EINVAL, "cfl must be finite and > 0");
    return FV_OK;
}

int fv_patch_batch_update(fv_batch_t *b, const void *Q_in, void *Q_out, const double *dx,
                          const double *dt, double *lambda_out, double *dt_next_out, double cfl)
{
    int rc = check_update_args(b, Q_in, Q_out, dx, dt, dt_next_out, cfl);
    if (rc) return rc;
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    return launch_update(b, b->stream, Q_in, Q_out, dx, dt, lambda_out, dt_next_out, cfl);
}

int fv_max_eigenvalue(fv_batch_t *b, const void *Q, double *lambda_out)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    if (b->T == 0) return FV_OK;
    if (!Q || !lambda_out) return fail(FV_EINVAL, "NULL pointer");
    if (!aligned16(Q)) return fail(FV_EINVAL, "state buffer must be 16-byte aligned");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    cudaError_t e = b->view.pde == fv::PDE_EULER
                        ? fv::launch_max_eigenvalue(b->view, b->precision, Q, lambda_out, b->stream)
                        : fv::launch_pde_max_eigenvalue(b->view, b->precision, Q, lambda_out, b->stream);
    return e == cudaSuccess ? FV_OK : cuda_fail(e, "max eigenvalue launch");
}

int fv_cfl_time_step(fv_batch_t *b, const double *lambda, const double *dx, double cfl, double *dt_out)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    if (b->T == 0) return FV_OK;
    if (!lambda || !dx || !dt_out) return fail(FV_EINVAL, "NULL pointer");
    if (!(cfl > 0.0 && cfl < 1e300)) return fail(FV_EINVAL, "cfl must be finite and > 0");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    cudaError_t e = fv::launch_cfl_time_step(b->view, lambda, dx, cfl, dt_out, b->stream);
    return e == cudaSuccess ? FV_OK : cuda_fail(e, "cfl launch");
}

int fv_conserved_totals(fv_batch_t *b, const void *Q, double *totals_out)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    if (b->T == 0) return FV_OK;
    if (!Q || !totals_out) return fail(FV_EINVAL, "NULL pointer");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    cudaError_t e = fv::launch_conserved_totals(b->view, b->precision, Q, totals_out, b->stream);
    return e == cudaSuccess ? FV_OK : cuda_fail(e, "totals launch");
}

static int enqueue_steps(fv_batch_t *b, cudaStream_t st, void *Q_a, void *Q_b, const double *dx,
                         double *dt_a, double *dt_b, double *lambda_out, int steps, double cfl)
{
    for (int s = 0; s < steps; ++s) {
        const void *qi = (s & 1) ? Q_b : Q_a;
        void *qo = (s & 1) ? Q_a : Q_b;
        const double *dti = (s & 1) ? dt_b : dt_a;
        double *dto = (s & 1) ? dt_a : dt_b;
        double *lam = (s == steps - 1) ? lambda_out : nullptr;
        if (b->view.nbr && !(b->form == FV_FORM_FUSED && fv::fused_reads_neighbours(b->plan))) {
            cudaError_t e = fv::launch_halo_exchange(b->view, b->precision, b->view.nbr, const_cast<void *>(qi), st);
            if (e != cudaSuccess) return cuda_fail(e, "halo exchange launch");
        }
        int rc = launch_update(b, st, qi, qo, dx, dti, lam, dto, cfl);
        if (rc) return rc;
    }
    return FV_OK;
}

int fv_batch_run(fv_batch_t *b, void *Q_a, void *Q_b, const double *dx, double *dt_a,
                 double *dt_b, double *lambda_out, int steps, double cfl, int use_graph)
{
    int rc = check_update_args(b, Q_a, Q_b, dx, dt_a, dt_b, cfl);
    if (rc) return rc;
    if (steps < 0) return fail(FV_EINVAL, "steps must be >= 0");
    if (b->T > 0 && !dt_b) return fail(FV_EINVAL, "dt_b is NULL");
    if (steps == 0 || b->T == 0) return FV_OK;
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    // the task-graph form launches one graph per step already
    if (!use_graph || b->form == FV_FORM_TASKGRAPH)
        return enqueue_steps(b, b->stream, Q_a, Q_b, dx, dt_a, dt_b, lambda_out, steps, cfl);

    GraphKey key{Q_a, Q_b, dx, dt_a, dt_b, lambda_out, steps, cfl, b->form};
    auto it = b->graphs.find(key);
    cudaGraphExec_t exec = nullptr;
    if (it != b->graphs.end()) {
        exec = it->second;
    } else {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "begin capture");
        rc = enqueue_steps(b, b->capture_stream, Q_a, Q_b, dx, dt_a, dt_b, lambda_out, steps, cfl);
        e = cudaStreamEndCapture(b->capture_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "end capture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
        b->graphs[key] = exec;
    }
    cudaError_t e = cudaGraphLaunch(exec, b->stream);
    return e == cudaSuccess ? FV_OK : cuda_fail(e, "graph launch");
}

int fv_batch_status(fv_batch_t *b)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    unsigned flags = 0;
    e = cudaMemcpy(&flags, b->view.flags, sizeof flags, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read status flags");
    if (flags) {
        unsigned zero = 0;
        e = cudaMemcpy(b->view.flags, &zero, sizeof zero, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "clear status flags");
        if (flags & fv::FV_FLAG_TIMEOUT)
            return fail(FV_ETIMEOUT, "a bounded device wait for a copy ran out; the update's results are invalid");
        return fail(FV_ENONPHYSICAL, "non-physical state (rho <= 0, p <= 0 or non-finite eigenvalue) met on the device");
    }
    return FV_OK;
}

int fv_batch_destroy(fv_batch_t *b)
{
    if (!b) return FV_OK;
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        if (!g_live.erase(b)) return fail(FV_EINVAL, "not a live batch (destroyed twice?)");
    }
    DeviceGuard dg(b->device);
    cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    if (b->scratch) cudaFree(b->scratch);
    if (b->nbr) cudaFree(b->nbr);
    if (b->hs_in) cudaFree(b->hs_in);
    if (b->hs_out) cudaFree(b->hs_out);
    if (b->hs_arrays) cudaFree(b->hs_arrays);
    if (b->sp_table) cudaFree(b->sp_table);
    if (b->hs_copy_in) cudaStreamDestroy(b->hs_copy_in);
    if (b->hs_copy_out) cudaStreamDestroy(b->hs_copy_out);
    for (cudaEvent_t e : b->hs_events) cudaEventDestroy(e);
    if (b->meta) cudaFree(b->meta);
    delete b;
    return FV_OK;
}

size_t fv_batch_state_elems(const fv_batch_t *b) { return b ? (size_t)b->state_elems : 0; }

size_t fv_batch_scratch_bytes(const fv_batch_t *b) { return b ? b->scratch_bytes : 0; }

int fv_batch_launches_per_update(const fv_batch_t *b)
{
    if (!b || b->T == 0) return 0;
    switch (b->form) {
    case FV_FORM_CASCADE: return 5;
    case FV_FORM_TILE: return 1;
    case FV_FORM_TASKGRAPH: return b->T * (2 * b->dim + 3);   // kernel nodes of the one graph launch
    default: {  // 2D edges 4, 8, 16, 32: one launch over every size class; else one per class
        bool compiled = b->fused_kernel == fv::FUSED_SWEEP2D;
        for (int c = 0; c < b->plan.num_classes; ++c) {
            const int p = b->plan.class_p[c];
            compiled = compiled && (p == 4 || p == 8 || p == 16 || p == 32);
        }
        return compiled ? 1 : b->plan.num_classes;
    }
    }
}

int fv_batch_describe(const fv_batch_t *b, char *buf, size_t len)
{
    if (!b || !buf || len == 0) return fail(FV_EINVAL, "NULL argument");
    const char *form = b->form == FV_FORM_CASCADE ? "cascade"
                       : (b->form == FV_FORM_TILE ? "tile" : (b->form == FV_FORM_TASKGRAPH ? "taskgraph" : "fused"));
    const char *lay = b->cascade_layout == FV_LAYOUT_SOA ? "soa" : (b->cascade_layout == FV_LAYOUT_AOSOA ? "aosoa" : "aos");
    const char *prec = b->precision == FV_F64 ? "f64" : (b->precision == FV_F32 ? "f32" : "bf16/f32");
    const char *fk = b->fused_kernel == fv::FUSED_SWEEP_PDE ? "sweep_pde"
                     : b->fused_kernel == fv::FUSED_SWEEP2D ? "sweep2d"
                     : (b->fused_kernel == fv::FUSED_SWEEP3D ? fv::fused3d_kernel_name(b->view, b->precision)
                                                             : "none");
    snprintf(buf, len, "form=%s precision=%s dim=%d patches=%d max_p=%d uniform_p=%d fused_kernel=%s "
             "items=%d warps_per_block=%d blocks_per_sm=%d ring=%d scratch_bytes=%zu cascade_layout=%s pde=%s",
             form, prec, b->dim, b->T, b->view.max_p, b->view.uniform_p, fk, b->plan.num_items,
             b->plan.shape.warps_per_block, b->plan.shape.blocks_per_sm,
             b->plan.shape.ring ? b->plan.shape.ring : 8, b->scratch_bytes, lay,
             b->view.pde == fv::PDE_EULER ? "euler" : "shallow_water");
    return FV_OK;
}

}  // extern "C"


namespace {

constexpr int kMaxHostChunks = 64;

int host_staging(fv_batch *b)
{
    if (b->hs_in) return FV_OK;
    const size_t bytes = (size_t)b->state_elems * elem_bytes(b->precision);
    void *in = nullptr, *out = nullptr, *arr = nullptr;
    cudaStream_t ci = nullptr, co = nullptr;
    std::vector<cudaEvent_t> evs;
    cudaError_t e = dev_alloc(&in, bytes);
    if (e == cudaSuccess) e = dev_alloc(&out, bytes);
    if (e == cudaSuccess) e = dev_alloc(&arr, 4 * (size_t)b->T * sizeof(double));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ci, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&co, cudaStreamNonBlocking);
    for (int i = 0; e == cudaSuccess && i < 3 * kMaxHostChunks + 2; ++i) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) evs.push_back(ev);
    }
    if (e != cudaSuccess) {
        // nothing partial stays behind: the next call starts over
        cudaGetLastError();
        for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
        if (ci) cudaStreamDestroy(ci);
        if (co) cudaStreamDestroy(co);
        cudaFree(in);
        cudaFree(out);
        cudaFree(arr);
        return fail(FV_ENOMEM, "host-update staging: %s", cudaGetErrorString(e));
    }
    b->hs_in = in;
    b->hs_out = out;
    b->hs_arrays = static_cast<double *>(arr);
    b->hs_copy_in = ci;
    b->hs_copy_out = co;
    b->hs_events = evs;
    return FV_OK;
}

struct HostPipeline {
    const void *q_in;
    void *q_out;
    const double *dx, *dt;
    double *lambda, *dt_next;
    double cfl;
    int chunks;
    bool split;
};

bool page_locked(const void *p)
{
    if (!p) return true;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost;
}

bool all_page_locked(const HostPipeline &hp)
{
    return page_locked(hp.q_in) && page_locked(hp.q_out) && page_locked(hp.dx) && page_locked(hp.dt) &&
           page_locked(hp.lambda) && page_locked(hp.dt_next);
}

// Patches [p_lo, p_hi) and work items [item_lo, item_hi) of chunk c of C
// (split: ranges of the uniform fused batch's work list; otherwise chunk 0
// is the whole batch).
struct ChunkRange {
    int item_lo, item_hi, p_lo, p_hi;
    size_t byte_off, bytes;
};

ChunkRange chunk_range(const fv_batch *b, bool split, int c, int C)
{
    const bool rows2d = b->plan.kernel == fv::FUSED_SWEEP2D || b->plan.kernel == fv::FUSED_SWEEP_PDE;
    const int per_item = split ? (rows2d ? 32 / b->view.uniform_p : 1) : b->T;
    ChunkRange r;
    r.item_lo = split ? (int)((int64_t)b->plan.num_items * c / C) : 0;
    r.item_hi = split ? (int)((int64_t)b->plan.num_items * (c + 1) / C) : 0;
    r.p_lo = split ? std::min(b->T, r.item_lo * per_item) : 0;
    r.p_hi = split ? std::min(b->T, r.item_hi * per_item) : b->T;
    const size_t es = elem_bytes(b->precision);
    r.byte_off = (size_t)b->elem_off[r.p_lo] * es;
    r.bytes = (size_t)(b->elem_off[r.p_hi] - b->elem_off[r.p_lo]) * es;
    return r;
}

// The update of one chunk's patches on stream st (the whole batch when not
// split).
int launch_chunk(fv_batch *b, cudaStream_t st, bool split, const ChunkRange &r, const fv::StepArgs &a)
{
    if (!split) return launch_update(b, st, a.q_in, a.q_out, a.dx, a.dt, a.lambda_out, a.dt_next_out, a.cfl);
    fv::FusedPlan sub = b->plan;
    sub.num_classes = 1;
    sub.class_begin[0] = r.item_lo;
    sub.class_end[0] = r.item_hi;
    const cudaError_t e = b->plan.kernel == fv::FUSED_SWEEP_PDE
                              ? fv::launch_pde_fused_update(b->view, b->precision, a, sub, st)
                              : fv::launch_fused_update(b->view, b->precision, a, sub, st);
    return e == cudaSuccess ? FV_OK : cuda_fail(e, "host update launch");
}

// Enqueue one host-state update on stream `org`: dx and dt of every patch in
// once, then per chunk its state in (copy-in stream), its update (org) and
// its state out (copy-out stream), so the copies of neighbouring chunks
// overlap the updates and each other; the per-patch outputs leave once
// after the last update; the copy streams join `org` at the end.
int enqueue_host_pipeline(fv_batch *b, cudaStream_t org, const HostPipeline &hp)
{
    double *d_dx = b->hs_arrays, *d_dt = d_dx + b->T, *d_lam = d_dt + b->T, *d_dtn = d_lam + b->T;
    unsigned char *qi = static_cast<unsigned char *>(b->hs_in), *qo = static_cast<unsigned char *>(b->hs_out);
    const unsigned char *hi = static_cast<const unsigned char *>(hp.q_in);
    unsigned char *ho = static_cast<unsigned char *>(hp.q_out);
    const int C = hp.chunks;
    const size_t arr = (size_t)b->T * sizeof(double);
    cudaEvent_t start = b->hs_events[2 * kMaxHostChunks], joined = b->hs_events[2 * kMaxHostChunks + 1];
    cudaError_t e = cudaEventRecord(start, org);      // order after earlier work on the stream
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->hs_copy_in, start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->hs_copy_out, start, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_dx, hp.dx, arr, cudaMemcpyHostToDevice, b->hs_copy_in);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_dt, hp.dt, arr, cudaMemcpyHostToDevice, b->hs_copy_in);
    for (int c = 0; c < C && e == cudaSuccess; ++c) {
        const ChunkRange r = chunk_range(b, hp.split, c, C);
        const size_t o = r.byte_off, n = r.bytes;
        cudaEvent_t ev_in = b->hs_events[2 * c], ev_done = b->hs_events[2 * c + 1];
        e = cudaMemcpyAsync(qi + o, hi + o, n, cudaMemcpyHostToDevice, b->hs_copy_in);
        if (e == cudaSuccess) e = cudaEventRecord(ev_in, b->hs_copy_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(org, ev_in, 0);
        if (e != cudaSuccess) break;
        // fixed halos: the staged output starts as the input, so the halo
        // volumes the update leaves untouched go back as Q_in's
        if (b->halo_mode == FV_HALO_FIXED) e = cudaMemcpyAsync(qo + o, qi + o, n, cudaMemcpyDeviceToDevice, org);
        if (e != cudaSuccess) break;
        fv::StepArgs args{qi, qo, d_dx, d_dt, hp.lambda ? d_lam : nullptr, hp.dt_next ? d_dtn : nullptr, hp.cfl};
        const int rc = launch_chunk(b, org, hp.split, r, args);
        if (rc) return rc;
        e = cudaEventRecord(ev_done, org);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->hs_copy_out, ev_done, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ho + o, qo + o, n, cudaMemcpyDeviceToHost, b->hs_copy_out);
    }
    if (e == cudaSuccess && hp.lambda) e = cudaMemcpyAsync(hp.lambda, d_lam, arr, cudaMemcpyDeviceToHost, b->hs_copy_out);
    if (e == cudaSuccess && hp.dt_next)
        e = cudaMemcpyAsync(hp.dt_next, d_dtn, arr, cudaMemcpyDeviceToHost, b->hs_copy_out);
    if (e == cudaSuccess) e = cudaEventRecord(joined, b->hs_copy_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(org, joined, 0);
    return e == cudaSuccess ? FV_OK : cuda_fail(e, "host update enqueue");
}

}  // namespace

extern "C" int fv_patch_batch_update_host(fv_batch_t *b, const void *Q_in_host, void *Q_out_host,
                                          const double *dx_host, const double *dt_host, double *lambda_host,
                                          double *dt_next_host, double cfl, int chunks)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    if (b->T == 0) return FV_OK;
    if (!Q_in_host || !Q_out_host || !dx_host || !dt_host) return fail(FV_EINVAL, "NULL host pointer");
    if (dt_next_host && !(cfl > 0.0 && cfl < 1e300)) return fail(FV_EINVAL, "cfl must be finite and > 0");
    if (chunks < 0 || chunks > kMaxHostChunks) return fail(FV_EINVAL, "chunks must be in [0, %d]", kMaxHostChunks);
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    if (chunks == 0) {
        // direct: the kernels read and write the page-locked host buffers
        // through their device mappings (coherent host memory), no staging
        void *dqi = nullptr, *dqo = nullptr, *ddx = nullptr, *ddt = nullptr, *dl = nullptr, *dn = nullptr;
        cudaError_t e = cudaHostGetDevicePointer(&dqi, const_cast<void *>(Q_in_host), 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&dqo, Q_out_host, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&ddx, const_cast<double *>(dx_host), 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&ddt, const_cast<double *>(dt_host), 0);
        if (e == cudaSuccess && lambda_host) e = cudaHostGetDevicePointer(&dl, lambda_host, 0);
        if (e == cudaSuccess && dt_next_host) e = cudaHostGetDevicePointer(&dn, dt_next_host, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(FV_EINVAL, "direct host update needs page-locked, mapped host buffers: %s",
                        cudaGetErrorString(e));
        }
        int rc = check_update_args(b, dqi, dqo, static_cast<double *>(ddx), static_cast<double *>(ddt),
                                   static_cast<double *>(dn), cfl);
        if (rc) return rc;
        rc = launch_update(b, b->stream, dqi, dqo, static_cast<double *>(ddx), static_cast<double *>(ddt),
                           static_cast<double *>(dl), static_cast<double *>(dn), cfl);
        if (rc) return rc;
        e = cudaStreamSynchronize(b->stream);
        return e == cudaSuccess ? FV_OK : cuda_fail(e, "direct host update");
    }
    int rc = host_staging(b);
    if (rc) return rc;
    // Chunks are ranges of work items of a uniform fused batch (so each
    // chunk's update is one launch over its own patches); any other batch
    // runs as a single chunk.
    const bool split = b->form == FV_FORM_FUSED && b->view.uniform_p > 0 && b->plan.num_classes == 1 &&
                       !b->view.nbr && chunks > 1;
    const int C = split ? std::min(chunks, b->plan.num_items) : 1;
    HostPipeline hp{Q_in_host, Q_out_host, dx_host, dt_host, lambda_host, dt_next_host, cfl, C, split};

    // The pipeline is captured once per set of host buffers as a CUDA graph
    // (one launch per call instead of several runtime calls per chunk); the
    // buffers must still be page-locked when a cached graph is replayed.
    const GraphKey key{Q_in_host, Q_out_host, dx_host, dt_host, dt_next_host, lambda_host, -1000 - C, cfl, b->form};
    auto it = b->graphs.find(key);
    if (it != b->graphs.end() && !all_page_locked(hp)) {
        cudaGraphExecDestroy(it->second);
        b->graphs.erase(it);
        it = b->graphs.end();
    }
    cudaGraphExec_t exec = it != b->graphs.end() ? it->second : nullptr;
    if (!exec && all_page_locked(hp)) {
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            rc = enqueue_host_pipeline(b, b->capture_stream, hp);
            e = cudaStreamEndCapture(b->capture_stream, &graph);
            if (rc == FV_OK && e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (rc != FV_OK || e != cudaSuccess) exec = nullptr;
        }
        if (exec) {
            b->graphs[key] = exec;
        } else {
            // not capturable (e.g. the task-graph form): run it eagerly
            cudaGetLastError();
            g_last_error.clear();
        }
    }
    if (exec) {
        cudaError_t e = cudaGraphLaunch(exec, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        return e == cudaSuccess ? FV_OK : cuda_fail(e, "host update");
    }
    rc = enqueue_host_pipeline(b, b->stream, hp);
    if (rc) return rc;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? FV_OK : cuda_fail(e, "host update");
}

// ------------------------------------------- host-resident time stepping

extern "C" int fv_patch_batch_run_host(fv_batch_t *b, void *Q_a_host, void *Q_b_host, const double *dx_host,
                                       double *dt_a_host, double *dt_b_host, double *lambda_host, int steps,
                                       double cfl, int chunks)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    if (steps < 0) return fail(FV_EINVAL, "steps must be >= 0");
    if (chunks < 1 || chunks > kMaxHostChunks) return fail(FV_EINVAL, "chunks must be in [1, %d]", kMaxHostChunks);
    if (!(cfl > 0.0 && cfl < 1e300)) return fail(FV_EINVAL, "cfl must be finite and > 0");
    if (b->T == 0 || steps == 0) return FV_OK;
    if (!Q_a_host || !Q_b_host || !dx_host || !dt_a_host || !dt_b_host) return fail(FV_EINVAL, "NULL host pointer");
    const size_t bytes = (size_t)b->state_elems * elem_bytes(b->precision);
    const size_t arr = (size_t)b->T * sizeof(double);
    if (overlaps(Q_a_host, Q_b_host, bytes)) return fail(FV_EINVAL, "Q_a and Q_b overlap");
    if (overlaps(dt_a_host, dt_b_host, arr)) return fail(FV_EINVAL, "dt_a and dt_b overlap");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    int rc = host_staging(b);
    if (rc) return rc;

    const bool split = b->form == FV_FORM_FUSED && b->view.uniform_p > 0 && b->plan.num_classes == 1 &&
                       !b->view.nbr && chunks > 1;
    const int C = split ? std::min(chunks, b->plan.num_items) : 1;
    double *d_dx = b->hs_arrays, *d_dt = d_dx + b->T, *d_lam = d_dt + b->T, *d_dtn = d_lam + b->T;
    unsigned char *qi = static_cast<unsigned char *>(b->hs_in), *qo = static_cast<unsigned char *>(b->hs_out);
    unsigned char *hq[2] = {static_cast<unsigned char *>(Q_a_host), static_cast<unsigned char *>(Q_b_host)};
    double *hdt[2] = {dt_a_host, dt_b_host};
    cudaStream_t org = b->stream, cin = b->hs_copy_in, cout = b->hs_copy_out;
    cudaEvent_t start = b->hs_events[2 * kMaxHostChunks], joined = b->hs_events[2 * kMaxHostChunks + 1];
    std::vector<ChunkRange> ranges;
    for (int c = 0; c < C; ++c) ranges.push_back(chunk_range(b, split, c, C));

    // Per chunk a chain through the steps: copy in (state and time steps of
    // its patches), update, copy out, then the next step's copy in of the
    // same chunk once its copy out has landed.  The chains of different
    // chunks are independent, so copies in both directions and the updates
    // of different chunks (and steps) overlap.  The device staging buffers
    // are reused safely along each chain: a chunk's copy in waits for its
    // previous copy out, which follows the update that read its input.
    cudaError_t e = cudaEventRecord(start, org);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cin, start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cout, start, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_dx, dx_host, arr, cudaMemcpyHostToDevice, cin);
    for (int st = 0; st < steps && e == cudaSuccess; ++st) {
        const int src = st & 1, dst = 1 - src;
        const bool last = st == steps - 1;
        for (int c = 0; c < C && e == cudaSuccess; ++c) {
            const ChunkRange &r = ranges[c];
            const size_t po = (size_t)r.p_lo * sizeof(double), pn = (size_t)(r.p_hi - r.p_lo) * sizeof(double);
            cudaEvent_t ev_in = b->hs_events[2 * c], ev_done = b->hs_events[2 * c + 1];
            cudaEvent_t ev_out = b->hs_events[2 * kMaxHostChunks + 2 + c];
            if (st > 0) e = cudaStreamWaitEvent(cin, ev_out, 0);
            if (e == cudaSuccess) e = cudaMemcpyAsync(qi + r.byte_off, hq[src] + r.byte_off, r.bytes,
                                                      cudaMemcpyHostToDevice, cin);
            if (e == cudaSuccess && pn)
                e = cudaMemcpyAsync(reinterpret_cast<unsigned char *>(d_dt) + po,
                                    reinterpret_cast<const unsigned char *>(hdt[src]) + po, pn,
                                    cudaMemcpyHostToDevice, cin);
            if (e == cudaSuccess) e = cudaEventRecord(ev_in, cin);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(org, ev_in, 0);
            // fixed halos: the staged output starts as the first input, so the
            // halo volumes no update writes go back as Q_a's; later updates
            // rewrite only interiors and copied x-halo volumes, so once is enough
            if (e == cudaSuccess && st == 0 && b->halo_mode == FV_HALO_FIXED)
                e = cudaMemcpyAsync(qo + r.byte_off, qi + r.byte_off, r.bytes, cudaMemcpyDeviceToDevice, org);
            // a neighbour table: halos filled from the neighbours before each
            // update, as fv_batch_run does (the batch then runs as one chunk)
            if (e == cudaSuccess && b->view.nbr && !(b->form == FV_FORM_FUSED && fv::fused_reads_neighbours(b->plan)))
                e = fv::launch_halo_exchange(b->view, b->precision, b->view.nbr, qi, org);
            if (e != cudaSuccess) break;
            const fv::StepArgs args{qi, qo, d_dx, d_dt, last && lambda_host ? d_lam : nullptr, d_dtn, cfl};
            rc = launch_chunk(b, org, split, r, args);
            if (rc) break;
            e = cudaEventRecord(ev_done, org);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cout, ev_done, 0);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hq[dst] + r.byte_off, qo + r.byte_off, r.bytes,
                                                      cudaMemcpyDeviceToHost, cout);
            if (e == cudaSuccess && pn)
                e = cudaMemcpyAsync(reinterpret_cast<unsigned char *>(hdt[dst]) + po,
                                    reinterpret_cast<const unsigned char *>(d_dtn) + po, pn,
                                    cudaMemcpyDeviceToHost, cout);
            if (e == cudaSuccess && last && lambda_host && pn)
                e = cudaMemcpyAsync(reinterpret_cast<unsigned char *>(lambda_host) + po,
                                    reinterpret_cast<const unsigned char *>(d_lam) + po, pn,
                                    cudaMemcpyDeviceToHost, cout);
            if (e == cudaSuccess) e = cudaEventRecord(ev_out, cout);
        }
        if (rc) break;
    }
    if (e == cudaSuccess && rc == FV_OK) e = cudaEventRecord(joined, cout);
    if (e == cudaSuccess && rc == FV_OK) e = cudaStreamWaitEvent(org, joined, 0);
    // whatever was enqueued finishes before the call returns (the host
    // buffers stay the caller's once it has)
    const cudaError_t s1 = cudaStreamSynchronize(cin), s2 = cudaStreamSynchronize(cout),
                      s3 = cudaStreamSynchronize(org);
    if (rc) return rc;
    if (e == cudaSuccess) e = s1 != cudaSuccess ? s1 : (s2 != cudaSuccess ? s2 : s3);
    return e == cudaSuccess ? FV_OK : cuda_fail(e, "host time stepping");
}

// --------------------------------------------------------------- autotuner

namespace {

// Read a buffer larger than L2 (clean lines replace whatever the last
// launch left there); the sink store never happens for a zeroed buffer.
__global__ void k_l2_sweep(const uint4 *__restrict__ buf, size_t n, unsigned *sink)
{
    unsigned acc = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const uint4 v = buf[i];
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == 0x9e3779b9u) *sink = acc;
}

std::mutex g_tune_mu;
std::map<std::string, fv::FusedShape> g_tune_cache;
bool g_tune_loaded = false;

std::string tune_key(const fv_batch *b)
{
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, b->device);
    char k[256];
    snprintf(k, sizeof k, "%s|sm%d%d|d%d|prec%d|halo%d|T%d|maxp%d|unip%d|items%d", prop.name, prop.major,
             prop.minor, b->dim, b->precision, b->halo_mode, b->T, b->view.max_p, b->view.uniform_p,
             b->plan.num_items);
    std::string s(k);
    for (auto &c : s)
        if (c == ' ') c = '_';
    return s;
}

void load_tune_file()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("FVBATCH_TUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    // one line per batch signature: key, warps per block, blocks per SM and
    // the ring depth (0 = default; absent in files written before it existed)
    char line[640], key[512];
    while (fgets(line, sizeof line, f)) {
        int w = 0, bps = 0, ring = 0;
        const int n = sscanf(line, "%511s %d %d %d", key, &w, &bps, &ring);
        if (n >= 3) g_tune_cache[key] = fv::FusedShape{w, bps, n == 4 ? ring : 0};
    }
    fclose(f);
}

void save_tune_file()
{
    const char *path = getenv("FVBATCH_TUNE_CACHE");
    if (!path || !*path) return;
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    for (auto &kv : g_tune_cache)
        fprintf(f, "%s %d %d %d\n", kv.first.c_str(), kv.second.warps_per_block, kv.second.blocks_per_sm,
                kv.second.ring);
    fclose(f);
    rename(tmp.c_str(), path);
}

}  // namespace

extern "C" int fv_batch_tune(fv_batch_t *b, const void *Q_in, void *Q_out, const double *dx,
                             const double *dt)
{
    int rc = check_update_args(b, Q_in, Q_out, dx, dt, nullptr, 0.0);
    if (rc) return rc;
    if (b->T == 0 || b->fused_kernel == fv::FUSED_NONE) return FV_OK;
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    std::string key = tune_key(b);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_tune_file();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->plan.shape = it->second;
            drop_graphs(b);
            return FV_OK;
        }
    }
    const size_t bytes = (size_t)b->state_elems * elem_bytes(b->precision);
    std::vector<unsigned char> ref(bytes), got(bytes);
    const int warps[] = {1, 2, 4, 8, 16};
    const int bps[] = {0, -1, -2, 1, 2, 4};
    fv::FusedShape best{0, 0, 0};
    float best_ms = 1e30f;
    bool have_ref = false;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // cold-cache timing: before each timed launch the L2 is refilled with
    // clean lines of a scratch buffer twice its size, so every candidate
    // reads its input from HBM (as for states larger than L2)
    int l2_bytes = 0;
    cudaDeviceGetAttribute(&l2_bytes, cudaDevAttrL2CacheSize, b->device);
    const size_t flush_n = (size_t)std::max(l2_bytes, 1 << 20) * 2 / sizeof(uint4);
    uint4 *flush = nullptr;
    if (dev_alloc(reinterpret_cast<void **>(&flush), flush_n * sizeof(uint4) + 16) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(FV_ENOMEM, "autotune: no room for the %zu-byte cache-clearing buffer", flush_n * sizeof(uint4));
    }
    unsigned *sink = reinterpret_cast<unsigned *>(flush + flush_n);
    cudaMemsetAsync(flush, 0, flush_n * sizeof(uint4) + 16, b->stream);
    const int sweep_grid = 4 * fv::num_sms();
    fv::FusedShape saved = b->plan.shape;
    int form = b->form;
    b->form = FV_FORM_FUSED;
    // eigenvalue and time-step outputs as in a time-stepping loop
    double *outs = nullptr;
    std::vector<fv::FusedShape> cands;
    if (dev_alloc(reinterpret_cast<void **>(&outs), 2 * (size_t)b->T * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        rc = fail(FV_ENOMEM, "autotune: eigenvalue/time-step scratch");
        goto done;
    }
    {
        // ring depths of the 2D sweep (rows in flight per warp): the default
        // and, where the batch can choose, 4 and 6 -- instantiated kernels,
        // timed and checked bitwise like the launch shapes
        std::vector<int> rings{0};
        if (b->fused_kernel == fv::FUSED_SWEEP2D && fv::sweep_ring_applies(b->view, b->precision))
            rings.insert(rings.end(), {4, 6});
        for (int r : rings)
            for (int w : warps)
                for (int k : bps) {
                    if (k > 0 && w * k > 64) continue;
                    if (w == 1 && k > 0) continue;
                    if (r != 0 && k == -2) continue;     // the streaming schedule has its own ring
                    cands.push_back(fv::FusedShape{w, k, r});
                }
    }
    {
        // every candidate once: results must be bitwise identical
        for (const fv::FusedShape &c : cands) {
            b->plan.shape = c;
            cudaError_t e = cudaMemsetAsync(Q_out, 0, bytes, b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
            if (e != cudaSuccess) { rc = cuda_fail(e, "tune reset"); goto done; }
            rc = launch_update(b, b->stream, Q_in, Q_out, dx, dt, nullptr, nullptr, 0.0);
            if (rc) goto done;
            e = cudaMemcpyAsync(got.data(), Q_out, bytes, cudaMemcpyDeviceToHost, b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
            if (e != cudaSuccess) { rc = cuda_fail(e, "tune readback"); goto done; }
            if (!have_ref) {
                ref = got;
                have_ref = true;
            } else if (memcmp(ref.data(), got.data(), bytes) != 0) {
                rc = fail(FV_ECUDA, "autotune: launch shape (%d warps, %d blocks/SM, ring %d) changed the result",
                          c.warps_per_block, c.blocks_per_sm, c.ring);
                goto done;
            }
        }
        // timing: rounds over all candidates (so slow drifts of the clock or
        // of neighbours on the machine hit every candidate alike), each launch
        // after an L2 refill; the lowest median wins
        constexpr int kRounds = 5, kPerRound = 4;
        std::vector<std::vector<float>> samples(cands.size());
        for (int round = 0; round < kRounds; ++round)
            for (size_t ci = 0; ci < cands.size(); ++ci) {
                b->plan.shape = cands[ci];
                if (round == 0)
                    for (int r = 0; r < 2; ++r) launch_update(b, b->stream, Q_in, Q_out, dx, dt, nullptr, nullptr, 0.0);
                for (int r = 0; r < kPerRound; ++r) {
                    k_l2_sweep<<<sweep_grid, 256, 0, b->stream>>>(flush, flush_n, sink);
                    cudaEventRecord(e0, b->stream);
                    launch_update(b, b->stream, Q_in, Q_out, dx, dt, outs, outs + b->T, 0.4);
                    cudaEventRecord(e1, b->stream);
                    cudaError_t e = cudaEventSynchronize(e1);
                    if (e != cudaSuccess) { rc = cuda_fail(e, "tune timing"); goto done; }
                    float one = 0;
                    cudaEventElapsedTime(&one, e0, e1);
                    samples[ci].push_back(one);
                }
            }
        for (size_t ci = 0; ci < cands.size(); ++ci) {
            std::vector<float> &v = samples[ci];
            std::sort(v.begin(), v.end());
            const float med = v[v.size() / 2];
            if (med < best_ms) {
                best_ms = med;
                best = cands[ci];
            }
        }
    }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(flush);
    if (outs) cudaFree(outs);
    b->form = form;
    if (rc) {
        b->plan.shape = saved;
        return rc;
    }
    b->plan.shape = best;
    drop_graphs(b);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
        save_tune_file();
    }
    return FV_OK;
}

// ------------------------------------------------ scattered host patches

extern "C" int fv_batch_set_host_patches(fv_batch_t *b, const void *const *patch_in, void *const *patch_out)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    if (!patch_in && !patch_out) {
        b->sp_in.clear();
        b->sp_out.clear();
        return FV_OK;
    }
    if (!patch_in || !patch_out) return fail(FV_EINVAL, "both patch tables are needed (or both NULL)");
    std::vector<void *> dev(2 * (size_t)b->T);
    for (int side = 0; side < 2; ++side)
        for (int i = 0; i < b->T; ++i) {
            const void *ptr = side == 0 ? patch_in[i] : patch_out[i];
            if (!ptr) return fail(FV_EINVAL, "patch %d: NULL %s pointer", i, side ? "output" : "input");
            cudaPointerAttributes at;
            cudaError_t e = cudaPointerGetAttributes(&at, ptr);
            if (e != cudaSuccess || at.type != cudaMemoryTypeHost || !at.devicePointer) {
                cudaGetLastError();
                return fail(FV_EINVAL, "patch %d: %s is not page-locked host memory (cudaHostAlloc/cudaHostRegister)",
                            i, side ? "output" : "input");
            }
            dev[side * (size_t)b->T + i] = at.devicePointer;
        }
    for (int i = 0; i < b->T; ++i)
        if (patch_in[i] == patch_out[i]) return fail(FV_EINVAL, "patch %d: input and output alias", i);
    if (!b->sp_table && b->T > 0) {
        cudaError_t e = dev_alloc(reinterpret_cast<void **>(&b->sp_table), 2 * (size_t)b->T * sizeof(void *));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(FV_ENOMEM, "patch address table");
        }
    }
    if (b->T > 0) {
        cudaError_t e = cudaMemcpy(b->sp_table, dev.data(), dev.size() * sizeof(void *), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "patch address table upload");
    }
    b->sp_in.resize(b->T);
    b->sp_out.resize(b->T);
    for (int i = 0; i < b->T; ++i) {
        b->sp_in[i] = const_cast<void *>(patch_in[i]);
        b->sp_out[i] = patch_out[i];
    }
    return FV_OK;
}

extern "C" int fv_patch_batch_update_scattered(fv_batch_t *b, const double *dx_host, const double *dt_host,
                                               double *lambda_host, double *dt_next_host, double cfl, int flags)
{
    if (!b) return fail(FV_EINVAL, "batch is NULL");
    if (b->T == 0) return FV_OK;
    if ((int)b->sp_in.size() != b->T) return fail(FV_EINVAL, "no host patches registered (fv_batch_set_host_patches)");
    if (!dx_host || !dt_host) return fail(FV_EINVAL, "NULL host pointer");
    if (dt_next_host && !(cfl > 0.0 && cfl < 1e300)) return fail(FV_EINVAL, "cfl must be finite and > 0");
    if (flags & ~(FV_SCATTER_SWAP | FV_SCATTER_COPIES)) return fail(FV_EINVAL, "unknown flags 0x%x", flags);
    DeviceGuard dg(b->device);
    if (!dg.ok) return fail(FV_ECUDA, "cannot make device %d current", b->device);
    int rc = host_staging(b);
    if (rc) return rc;
    const bool swap = flags & FV_SCATTER_SWAP, copies = flags & FV_SCATTER_COPIES;
    const size_t es = elem_bytes(b->precision);
    const int T = b->T;
    double *ddx = b->hs_arrays, *ddt = ddx + T, *dl = ddt + T, *dn = dl + T;
    cudaStream_t st = b->stream;
    cudaError_t e = cudaMemcpyAsync(ddx, dx_host, (size_t)T * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ddt, dt_host, (size_t)T * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "dx/dt upload");
    unsigned char *qi = static_cast<unsigned char *>(b->hs_in), *qo = static_cast<unsigned char *>(b->hs_out);
    const std::vector<void *> &src = swap ? b->sp_out : b->sp_in;
    const std::vector<void *> &dst = swap ? b->sp_in : b->sp_out;
    void **src_tab = b->sp_table + (swap ? T : 0), **dst_tab = b->sp_table + (swap ? 0 : T);
    if (copies) {
        // the paper's explicit transfers: one copy per patch
        for (int i = 0; i < T && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(qi + b->elem_off[i] * es, src[i], (size_t)(b->elem_off[i + 1] - b->elem_off[i]) * es,
                                cudaMemcpyHostToDevice, st);
    } else {
        e = fv::launch_gather_patches(b->view, src_tab, qi, (int)es, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "patch gather");
    rc = launch_update(b, st, qi, qo, ddx, ddt, lambda_host ? dl : nullptr, dt_next_host ? dn : nullptr, cfl);
    if (rc) return rc;
    if (copies) {
        // interior rows back: one pitched copy per 2D patch, per z-plane in 3D
        const int N = b->dim + 2;
        for (int i = 0; i < T && e == cudaSuccess; ++i) {
            const int p = b->psize[i];
            const size_t e1 = (size_t)p + 2, pitch = e1 * N * es, width = (size_t)p * N * es;
            const int planes = b->dim == 2 ? 1 : p;
            for (int z = 0; z < planes && e == cudaSuccess; ++z) {
                const size_t first = (b->dim == 2 ? e1 + 1 : ((size_t)(z + 1) * e1 + 1) * e1 + 1) * N * es;
                e = cudaMemcpy2DAsync(static_cast<unsigned char *>(dst[i]) + first, pitch,
                                      qo + b->elem_off[i] * es + first, pitch, width, (size_t)p,
                                      cudaMemcpyDeviceToHost, st);
            }
        }
    } else {
        e = fv::launch_scatter_interiors(b->view, qo, dst_tab, (int)es, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "patch scatter");
    if (lambda_host) e = cudaMemcpyAsync(lambda_host, dl, (size_t)T * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && dt_next_host)
        e = cudaMemcpyAsync(dt_next_host, dn, (size_t)T * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? FV_OK : cuda_fail(e, "scattered update");
}
