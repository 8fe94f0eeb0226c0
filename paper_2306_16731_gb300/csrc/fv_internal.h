// fv_internal.h -- launcher interface between the C ABI (fv_batch.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace fv {

// Device-resident description of a batch, passed by value to kernels.
struct BatchView {
    int dim;                   // 2 or 3
    int num_patches;           // T
    int halo_mode;             // FV_HALO_FIXED / FV_HALO_PERIODIC
    double gamma;
    const int64_t *elem_off;   // [T+1] element offset of each patch
    const int64_t *cell_off;   // [T+1] halo-inclusive cell offset of each patch
    const int64_t *int_off;    // [T+1] interior-volume offset of each patch
    const int32_t *psize;      // [T] edge length p_i
    unsigned *flags;           // device error flags (FV_FLAG_*)
    int64_t total_cells;       // sum (p_i + 2)^d
    int64_t total_interior;    // sum p_i^d
    int max_p;
    int uniform_p;             // p if all patches share it, else 0
    int align_bytes;           // largest power of two <= 16 dividing every patch's (and 3D plane's) bytes
    const int32_t *nbr;        // [T][2 dim] neighbour across -x,+x,-y,+y[,-z,+z] or -1; null = none registered
    int test_wait_expiry;      // test hook: bounded copy waits are made to run out (FV_ETIMEOUT)
    int pde;                   // PDE_EULER or PDE_SHALLOW_WATER
    double pde_param[2];       // shallow water: gravity g, Coriolis parameter f
};

enum PdeKind { PDE_EULER = 0, PDE_SHALLOW_WATER = 1 };

// Arguments of one update.
struct StepArgs {
    const void *q_in;
    void *q_out;
    const double *dx;
    const double *dt;
    double *lambda_out;        // may be null
    double *dt_next_out;       // may be null
    double cfl;
};

// Scratch of the loop-cascade form (all in compute type, halo-inclusive
// cell indexing, array of structures).
struct CascadeScratch {
    void *flux;                // [dim][total_cells][N]  F_n of each volume
    void *lam;                 // [dim][total_cells]     lambda_n of each volume
    void *face;                // [dim][total_cells][N]  2 Fhat at the lower face of each volume
    void *lam_new;             // [total_cells]          max eigenvalue of the new state
};

size_t cascade_scratch_bytes(const BatchView &b, int precision);
void cascade_scratch_carve(void *base, const BatchView &b, int precision, CascadeScratch *s);

// Launch-shape choice of the fused form (the autotuner's search space).
struct FusedShape {
    int warps_per_block;       // 1..16
    int blocks_per_sm;         // grid = blocks_per_sm * SMs (persistent); 0 = one block per work item
    int ring;                  // rows in flight per warp of the 2D sweep (FP32/BF16, one compiled edge):
                               // 4 or 6; 0 = the default depth (8)
};

// true if the ring depth of the fused 2D sweep can be chosen for this batch
bool sweep_ring_applies(const BatchView &b, int precision);

// Work list of the fused sweep kernels: one item per group of equal-size
// patches handled by one warp, largest patches first.
struct WorkItem {
    int32_t first_patch;       // index into the sorted patch order
    int16_t count;             // patches in this item
    int16_t p;                 // edge length of these patches
};

constexpr int kMaxSizeClasses = 129;   // distinct edge lengths a plan can hold

struct FusedPlan {
    const WorkItem *items;     // device
    const int32_t *order;      // device [T] patch indices sorted by size class
    int num_items;
    unsigned *work_counter;    // device: 2 counters per size class for dynamic scheduling
    FusedShape shape;
    int kernel;                // which fused kernel family
    int num_classes;           // size classes, largest edge first (one launch each)
    int class_p[kMaxSizeClasses];
    int class_begin[kMaxSizeClasses];
    int class_end[kMaxSizeClasses];
};

enum FusedKernel { FUSED_NONE = 0, FUSED_SWEEP2D = 1, FUSED_SWEEP3D = 2, FUSED_SWEEP_PDE = 3 };

// Layout of the loop cascade's vector temporaries (F_n, face fluxes).
enum CascadeLayout { CASCADE_AOS = 0, CASCADE_SOA = 1, CASCADE_AOSOA = 2 };

// All launchers return cudaSuccess or the launch error; they never sync.
cudaError_t launch_cascade_update(const BatchView &b, int precision, const StepArgs &a,
                                  const CascadeScratch &s, cudaStream_t st, int layout);
// Add the task-graph realisation of one update (per-patch nodes of the
// cascade's kernels) to graph g; cell_off_host has T+1 entries.
cudaError_t build_cascade_taskgraph(const BatchView &b, const int64_t *cell_off_host, int precision,
                                    const StepArgs &a, const CascadeScratch &s, int layout, cudaGraph_t g);
cudaError_t launch_tile_update(const BatchView &b, int precision, const StepArgs &a,
                               cudaStream_t st);
bool tile_supported(const BatchView &b, int precision);
cudaError_t launch_fused_update(const BatchView &b, int precision, const StepArgs &a,
                                const FusedPlan &plan, cudaStream_t st);
bool fused_supported(const BatchView &b, int precision, int *kernel);
bool fused3d_supported(const BatchView &b, int precision);
cudaError_t launch_fused3d_update(const BatchView &b, int precision, const StepArgs &a,
                                  const FusedPlan &plan, cudaStream_t st);
// name of the fused 3D kernel an update of this batch runs
const char *fused3d_kernel_name(const BatchView &b, int precision);
// periodic 8^3 patches, one warp per patch (fv_sweep3d_p8.cu)
bool fused3d_p8_applies(const BatchView &b, int precision, const void *q_in, const void *q_out);
cudaError_t launch_fused3d_p8(const BatchView &b, int precision, const StepArgs &a, int first, int count,
                              const FusedShape &shape, cudaStream_t st);
int fused_items_for(int dim, int p, int *patches_per_item);

// Patches held as separate host allocations (fv_scatter.cu): gather into the
// batch layout, scatter the updated interiors back; src/dst are device
// tables of device-visible host addresses.
cudaError_t launch_gather_patches(const BatchView &b, const void *const *src, void *dst, int es, cudaStream_t st);
cudaError_t launch_scatter_interiors(const BatchView &b, const void *src, void *const *dst, int es, cudaStream_t st);

// Generic PDE of Eq. 1 on the patch-wise realisation (fv_pde.cu).
bool pde_tile_supported(const BatchView &b, int precision);
cudaError_t launch_pde_update(const BatchView &b, int precision, const StepArgs &a, cudaStream_t st);
cudaError_t launch_pde_max_eigenvalue(const BatchView &b, int precision, const void *q, double *lambda_out,
                                      cudaStream_t st);
// Fused row sweep of a generic-PDE batch (fv_pde.cu): 2D, edges 4, 8, 16 or
// 32 only (sizes_host: the T edge lengths), FP32 or FP64 storage.
bool pde_fused_supported(const BatchView &b, int precision, const int32_t *sizes_host);
cudaError_t launch_pde_fused_update(const BatchView &b, int precision, const StepArgs &a, const FusedPlan &plan,
                                    cudaStream_t st);

cudaError_t launch_halo_exchange(const BatchView &b, int precision, const int32_t *nbr, void *q,
                                 cudaStream_t st);
// true if the fused kernel chosen for this plan reads neighbours' volumes
// itself (so an update needs no separate exchange)
bool fused_reads_neighbours(const FusedPlan &plan);
cudaError_t launch_max_eigenvalue(const BatchView &b, int precision, const void *q,
                                  double *lambda_out, cudaStream_t st);
cudaError_t launch_cfl_time_step(const BatchView &b, const double *lambda, const double *dx,
                                 double cfl, double *dt_out, cudaStream_t st);
cudaError_t launch_conserved_totals(const BatchView &b, int precision, const void *q,
                                    double *totals_out, cudaStream_t st);

int num_sms();

// true if p is device memory (not mapped or managed host memory): the bulk
// asynchronous copies of the 3D kernels address device memory only
bool is_device_memory(const void *p);

// Record the thread-local message returned by fv_last_error().
void set_last_error(const char *msg);

}  // namespace fv
