/*
 * fv_batch.h -- C ABI of the GB300 (sm_103a) batched finite-volume patch
 * update: one explicit Euler time step of T Cartesian patches with a
 * one-volume halo, Rusanov face fluxes on the compressible Euler equations,
 * and the per-patch maximum eigenvalue that feeds the CFL condition.
 *
 * Method: arXiv:2306.16731, "SYCL compute kernels for ExaHyPE".
 *   - Sec. 2.2: volume update from face fluxes, Rusanov flux (Eq. 2), halo
 *     layer of width one, per-patch maximum eigenvalue of the new solution
 *     for the CFL condition (local time stepping).
 *   - Sec. 2.3: the kernel takes N (p+2)^d T values (with halo) and yields
 *     the N p^d T interior values of the next time step; Algorithm 1 lists
 *     its steps.
 *   - Sec. 3: patch-wise, batched and task-graph realisations (the
 *     "cascade" form below is the batched one, the "tile" form the
 *     patch-wise one).
 *   - Sec. 4: array-of-structures data layout, per-patch reductions.
 *   - Sec. 5: Euler equations, N = d + 2 unknowns.
 * Readings of passages the paper leaves garbled: the update is
 * Q_new = Q - dt/h * sum_n (Fhat_n(c+1/2) - Fhat_n(c-1/2)); the Rusanov
 * dissipation is 1/2 max(lambda_L, lambda_R) (Q_R - Q_L); the CFL time step
 * is dt = cfl * h / (d * lambda_max).
 *
 * Data layout (all state buffers): array of structures with halo,
 *   Q[patch][z][y][x][k],  x fastest, the N = d+2 unknowns of a volume
 *   contiguous (rho, rho u_1 .. rho u_d, E); patch i starts at element
 *   sum_{j<i} N (p_j + 2)^d.  Element type: double (FV_F64), float
 *   (FV_F32) or bfloat16 (FV_BF16_F32).  fv_batch_state_elems() gives the
 *   element count.  Buffers must be 16-byte aligned.
 *
 * Ownership: the caller owns every state, dx, dt, lambda and dt buffer and
 * the CUDA stream; they are DEVICE pointers unless stated otherwise.  A
 * batch owns only its metadata (patch offsets and sizes on the device, the
 * kernel choice) and the scratch of the loop-cascade form.  Batches are not
 * thread-safe: use one batch per host thread.
 *
 * Errors: every entry point returns FV_OK (0) or a negative FV_E* code and
 * never aborts; fv_last_error() returns a thread-local message for the last
 * failure.  Argument errors are reported synchronously.  Non-physical
 * states met on the device (density or pressure not positive, eigenvalue
 * not finite) set a device flag; fv_batch_status() synchronises the stream,
 * reports FV_ENONPHYSICAL and clears the flag.  Update, eigenvalue, time
 * step and totals calls are asynchronous on the batch's stream, allocate
 * nothing and may be captured in a CUDA graph.
 */
#ifndef FV_BATCH_H
#define FV_BATCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fv_batch fv_batch_t;

/* Status codes. */
enum {
    FV_OK = 0,
    FV_EINVAL = -1,         /* bad argument (size, pointer, alias, mode) */
    FV_ENOMEM = -2,         /* host or device allocation failed */
    FV_ECUDA = -3,          /* a CUDA runtime call failed */
    FV_EUNSUPPORTED = -4,   /* valid request that no kernel of the library covers */
    FV_ENONPHYSICAL = -5,   /* device met rho <= 0, p <= 0 or a non-finite eigenvalue */
    FV_ETIMEOUT = -6        /* a kernel's bounded wait for its own copy ran out (1 s); that
                               update's results are invalid, the context stays usable */
};

/* Storage / compute precision of the state. */
enum {
    FV_F64 = 0,             /* double storage, double arithmetic */
    FV_F32 = 1,             /* float storage, float arithmetic */
    FV_BF16_F32 = 2         /* bfloat16 storage, float arithmetic */
};
/* In every precision the per-patch eigenvalue maximum, the CFL time step
 * and the conservation totals are double. */

/* Halo treatment (the halo layer of width one, Sec. 2.2). */
enum {
    FV_HALO_FIXED = 0,      /* halo volumes are read from Q_in as given; each halo volume of Q_out is
                               either left as it is or set to Q_in's value (the fused 2D kernels write
                               the x-halo volumes of interior rows so that rows are written whole) */
    FV_HALO_PERIODIC = 1    /* halo volumes are the wrapped interior of the same patch; halo memory of Q_in is
                               never read; halo volumes of Q_out are left untouched or set to the wrapped
                               new values (fused kernels write rows whole, x-halo volumes included) */
};

/* PDE of the batch (Eq. 1: dQ/dt + div F(Q) + sum_n B_n(Q) dQ/dx_n = S(Q)). */
enum {
    FV_PDE_EULER = 0,          /* compressible Euler (Sec. 5), N = dim + 2; parameter: gamma */
    FV_PDE_SHALLOW_WATER = 1   /* 2D shallow water over a bathymetry with Coriolis force, Q = (h, hu, hv, b),
                                  N = 4, b a parameter; parameters: gravity g, Coriolis f; non-conservative
                                  product g h grad b and source (0, f hv, -f hu, 0) */
};

/* Kernel realisation (Sec. 3). */
enum {
    FV_FORM_FUSED = 0,      /* default: every step fused (warp-level sweep kernels); one persistent launch for a 2D
                               batch whose edges are all 4, 8, 16 or 32, else one launch per patch-size class */
    FV_FORM_CASCADE = 1,    /* one launch per algorithmic step over all volumes, intermediates in device memory (batched realisation) */
    FV_FORM_TILE = 2,       /* one thread block per patch staged in shared memory (patch-wise realisation) */
    FV_FORM_TASKGRAPH = 3   /* task-graph realisation (Sec. 3): one CUDA graph per update whose nodes are the
                               cascade's kernels restricted to one patch (and one axis for fluxes and faces),
                               linked only by data dependencies; axes and patches run concurrently; bitwise
                               equal to FV_FORM_CASCADE; the graph is built and instantiated on the first
                               update with a buffer set (cost grows with T) and cannot be stream-captured */
};

/*
 * Create a batch of num_patches patches of dimension dim (2 or 3) with
 * edge lengths patch_size[i] >= 1 (HOST array of num_patches entries; copied).
 * halo must be 1 and unknowns must be dim + 2 (Euler).  precision is an
 * FV_F64/FV_F32/FV_BF16_F32 value, halo_mode an FV_HALO_* value, gamma > 1
 * the adiabatic index.  cuda_stream is a cudaStream_t (0 = legacy default
 * stream) on which every later call of this batch runs.  The device current
 * at creation is the batch's device.  On success *out receives the batch;
 * on failure *out is NULL.
 */
int fv_batch_create(fv_batch_t **out, int dim, int num_patches,
                    const int32_t *patch_size, int halo, int unknowns,
                    int precision, int halo_mode, double gamma,
                    void *cuda_stream);

/*
 * Create a batch for one of the FV_PDE_* systems (Eq. 1; the paper studies
 * Euler only, Sec. 5).  params holds num_params values: Euler {gamma} (this
 * is fv_batch_create); shallow water {g > 0, f}, dim must be 2, precision
 * FV_F64 or FV_F32.  Other PDEs than Euler run on generic kernels that take
 * the PDE as a device functor: a fused row sweep (FV_FORM_FUSED, the default
 * when every edge is 4, 8, 16 or 32) or a patch-wise kernel (FV_FORM_TILE,
 * the default otherwise); set_form accepts these two.  Both form at each
 * face the Rusanov flux of Eq. 2 on the evolved unknowns and the
 * non-conservative product B_n((Q_L+Q_R)/2)(Q_R - Q_L), half to each side;
 * Q_new = Q - dt/h sum_n [(Fhat_r - Fhat_l) + (D_r + D_l)/2] + dt S(Q);
 * parameter unknowns (b) are copied.  Layout, halos, dx/dt/lambda/dt_next,
 * status, graphs and host updates work as for Euler.  FV_EINVAL for bad
 * arguments, FV_EUNSUPPORTED for an unsupported precision or patch size.
 */
int fv_batch_create_pde(fv_batch_t **out, int pde, int dim, int num_patches, const int32_t *patch_size,
                        int precision, int halo_mode, const double *params, int num_params, void *cuda_stream);

/* Select the kernel realisation (FV_FORM_*).  FV_EUNSUPPORTED if this
 * build has no kernel of that form for the batch's shapes; the previous
 * form stays selected.  May allocate the cascade's scratch (FV_ENOMEM). */
int fv_batch_set_form(fv_batch_t *b, int form);

/* Layout of the cascade's and the task graph's vector temporaries (the
 * fluxes F_n and face fluxes; the paper's App. C): FV_LAYOUT_AOS (default,
 * [axis][cell][unknown]), FV_LAYOUT_SOA ([axis][unknown][cell]) or
 * FV_LAYOUT_AOSOA ([axis][cell/32][unknown][cell%32]).  Results are bitwise
 * independent of the layout.  FV_EINVAL for another value. */
enum { FV_LAYOUT_AOS = 0, FV_LAYOUT_SOA = 1, FV_LAYOUT_AOSOA = 2 };
int fv_batch_set_cascade_layout(fv_batch_t *b, int layout);

/* Launch shape of the fused form: warps_per_block in [1, 16]; blocks_per_sm
 * 0 = one warp per work item (grid covers the work list), > 0 = that many
 * persistent blocks per SM taking items from a device counter, -1 =
 * persistent with as many blocks per SM as can be resident, -2 = resident
 * persistent warps taking items round-robin with the row stream running
 * across items (2D batches of one edge length 8, 16 or 32; otherwise as -1).
 * Results do not depend on the shape (every shape computes the same
 * arithmetic). */
int fv_batch_set_launch_shape(fv_batch_t *b, int warps_per_block, int blocks_per_sm);

/* Staging depth of the fused 2D sweep (Sec. 2.3 leaves the staging of the
 * patch data to the realisation): the number of patch rows each warp keeps
 * in flight in its shared-memory ring, for uniform 2D batches of edge 4, 8,
 * 16 or 32 in FP32 or BF16 storage.  rows = 4 or 6, or 0 / 8 for the
 * default depth of 8; the streaming launch shape (blocks_per_sm = -2) keeps
 * its own ring.  Every depth computes the same bits; fv_batch_tune searches
 * the depths together with the launch shapes and records its choice in the
 * tuning cache.  FV_EINVAL for another value, FV_EUNSUPPORTED for a batch
 * without the choice (depth unchanged). */
int fv_batch_set_sweep_ring(fv_batch_t *b, int rows);

/*
 * Register which patch lies across each face (the halo layer of width one
 * that the paper's framework fills from neighbouring patches before the
 * kernel call, Sec. 2.2).  neighbours is a HOST array of num_patches * 2 *
 * dim entries in the order -x, +x, -y, +y[, -z, +z]: the index of the patch
 * across that face (it must have the same edge length), or -1 for a face
 * whose halo is taken from the patch itself (the halo mode).  NULL clears
 * the table.  Copied to the device (allocates once; FV_ENOMEM).  With a
 * table registered, fv_halo_exchange fills face halos from neighbours, the
 * fused 2D kernels for edge lengths 4, 8, 16 and 32 read the neighbours'
 * edge volumes directly in fv_patch_batch_update (no exchange needed), and
 * fv_batch_run runs an exchange before each update for every other kernel.
 */
int fv_batch_set_neighbours(fv_batch_t *b, const int32_t *neighbours);

/* Fill every face-halo volume that has a neighbour with the neighbour's
 * interior volume touching that face (across -x its column p-1, across +x
 * its column 0, likewise in y and z), in place on the device state Q;
 * corner and edge halo volumes are not written.  Asynchronous on the
 * batch's stream.  FV_EINVAL without a registered table. */
int fv_halo_exchange(fv_batch_t *b, void *Q);

/*
 * Patches kept as separate host allocations, as in the paper's framework
 * (each patch a heap object; moving them dominates its run time, Sec. 4
 * "Data transfer", Sec. 5 Fig. 4).  patch_in[i] and patch_out[i] (HOST
 * arrays of num_patches pointers) each address one halo-inclusive patch in
 * the batch layout of a single patch (N (p_i+2)^d values of the storage
 * type), in page-locked host memory (cudaHostAlloc or cudaHostRegister;
 * anything else gives FV_EINVAL).  The caller keeps every buffer alive and
 * at least that large while registered.  Pointers are validated and
 * translated once and their device table is uploaded (allocates once,
 * FV_ENOMEM); both NULL clears the registration.
 */
int fv_batch_set_host_patches(fv_batch_t *b, const void *const *patch_in, void *const *patch_out);

/*
 * One update of the registered host patches: gather them into the batch's
 * device staging (the buffers of fv_patch_batch_update_host), update,
 * write each patch's interior volumes back (halo volumes of the output
 * patches are not written), with dx/dt/lambda/dt_next as HOST arrays as in
 * fv_patch_batch_update_host.  flags: FV_SCATTER_SWAP reads the output
 * patches and writes the input patches (ping-pong); FV_SCATTER_COPIES moves
 * the patches with one cudaMemcpyAsync per patch in and pitched copies of the
 * interior rows out instead of the gather and scatter kernels (which read and
 * write the page-locked memory over the coherent CPU-GPU link, one block per
 * patch).  Synchronous.
 */
enum { FV_SCATTER_SWAP = 1, FV_SCATTER_COPIES = 2 };
int fv_patch_batch_update_scattered(fv_batch_t *b, const double *dx_host, const double *dt_host,
                                    double *lambda_host, double *dt_next_host, double cfl, int flags);

/* Rebind the batch to another stream (e.g. a capture stream). */
int fv_batch_set_stream(fv_batch_t *b, void *cuda_stream);

/* Test hook for the timeout path; the paper has no counterpart.  With
 * enable != 0, updates that run the periodic 8^3 kernel make each warp's
 * first plane wait expect 16 bytes more than its copy delivers, so the
 * bounded wait runs out after 1 s: the warp drains its copies, writes
 * nothing more and the next fv_batch_status reports FV_ETIMEOUT.  Nothing
 * faults; the context stays usable.  enable = 0 restores normal updates.
 * Other kernels ignore it. */
int fv_batch_test_wait_expiry(fv_batch_t *b, int enable);

/*
 * One explicit time step (Sec. 2.2, Eq. 2, Algorithm 1):
 *   Q_out = Q_in - dt_i/dx_i * sum_n (Fhat_n(c+1/2) - Fhat_n(c-1/2))
 * on the interior of every patch i.  Q_in and Q_out are device state
 * buffers of the batch's layout and precision; Q_out != Q_in and they must
 * not overlap (the update reads old neighbour values).  Q_out's interior
 * receives the new state; its halo follows the halo mode (FV_HALO_*).
 * dx and dt are device arrays of num_patches doubles (mesh width and time
 * step per patch, > 0).  If lambda_out (device,
 * num_patches doubles) is not NULL it receives the maximum over interior
 * volumes and directions of |u_n| + c of Q_out; if dt_next_out is not NULL
 * it receives cfl * dx_i / (dim * lambda_i) (requires cfl > 0).
 */
int fv_patch_batch_update(fv_batch_t *b, const void *Q_in, void *Q_out,
                          const double *dx, const double *dt,
                          double *lambda_out, double *dt_next_out, double cfl);

/*
 * One update of a batch whose state lives in HOST memory (the data
 * movement that dominates the paper's end-to-end runtimes, Sec. 5 and
 * Sec. 4 "Data transfer").  Q_in_host / Q_out_host are host state buffers
 * (page-locked for full speed), dx_host / dt_host host arrays of
 * num_patches doubles, lambda_host / dt_next_host optional host outputs.
 * With chunks = 0 ("direct") the update kernels read Q_in_host and write
 * Q_out_host through their device mappings (page-locked host memory is
 * coherently addressable from the GPU on Grace-Blackwell); no staging is
 * made, and unmapped buffers give FV_EINVAL.  With chunks in 1..64, a
 * uniform batch using the fused form is cut into that many ranges of
 * patches whose host-to-device copies, updates and device-to-host copies
 * run on three streams, so copies in both directions overlap each other and
 * the updates; any other batch runs as one chunk.  The first such call
 * creates the device staging (two state buffers and four arrays of
 * num_patches doubles) and two copy streams, kept until fv_batch_destroy
 * (FV_ENOMEM).  When all host buffers are page-locked, the copies and
 * updates of a call are captured once as a CUDA graph, cached per set of
 * host buffers (and chunks, cfl, form) and replayed by later calls with the
 * same buffers; a cached graph is dropped when a buffer is no longer
 * page-locked, and by the calls that drop the update graphs (form, launch
 * shape, tuning, neighbour table).
 * Synchronous: returns when Q_out_host and the outputs are complete.  With
 * chunks >= 1 and fixed halos the halo volumes of Q_out_host are those of
 * Q_in_host (so steps chain); with periodic halos they are unspecified;
 * with chunks = 0 they are as after fv_patch_batch_update.
 */
int fv_patch_batch_update_host(fv_batch_t *b, const void *Q_in_host, void *Q_out_host,
                               const double *dx_host, const double *dt_host,
                               double *lambda_host, double *dt_next_host, double cfl,
                               int chunks);

/*
 * `steps` CFL-chained updates of a batch whose state lives in HOST memory,
 * every step's state copied to the device and back (the host-resident
 * patches of Sec. 4 "Data transfer" and Sec. 5, over a time-stepping loop).
 * Q_a_host / Q_b_host: host state buffers (page-locked for full speed);
 * step s reads Q_a (s even) or Q_b (s odd) and writes the other, so the
 * final state is in Q_b if steps is odd, else in Q_a.  dx_host: num_patches
 * doubles, copied once.  dt_a_host holds the first step's time steps; step
 * s reads dt_a (s even) or dt_b (s odd) and writes the CFL time steps of
 * its new state, dt = cfl dx / (d lambda), into the other (both num_patches
 * doubles, host).  lambda_host (may be NULL): the eigenvalues of the final
 * state.  chunks in 1..64 as in fv_patch_batch_update_host: for a uniform
 * batch in the fused form the patches are cut into that many ranges, and
 * each range runs as a chain through the steps -- its state and time steps
 * in, its update, its state and next time steps out, then its next step's
 * copy in -- while the chains of the other ranges proceed independently, so
 * one step's copies out overlap the next step's copies in; any other batch
 * runs as one range.  With a neighbour table (fv_batch_set_neighbours) each
 * step first fills the face halos from the neighbours where the kernel does
 * not read them itself, as fv_batch_run does.  Results are bitwise those of
 * fv_batch_run on device copies of the buffers (and, without a neighbour
 * table, of `steps` calls of fv_patch_batch_update_host with the buffers
 * alternated).  steps = 0 or an
 * empty batch: no-op.  FV_EINVAL for NULL pointers, steps < 0, chunks
 * outside 1..64, a non-positive cfl, or overlapping Q_a/Q_b or dt_a/dt_b;
 * the device staging is that of fv_patch_batch_update_host (FV_ENOMEM).
 * Synchronous: returns when the final state and outputs are on the host.
 * With fixed halos and no neighbour table every state written keeps the
 * first state's halo volumes; otherwise the halo volumes written are
 * unspecified (the updates never read them: they are exchanged or wrapped).
 */
int fv_patch_batch_run_host(fv_batch_t *b, void *Q_a_host, void *Q_b_host, const double *dx_host,
                            double *dt_a_host, double *dt_b_host, double *lambda_host, int steps,
                            double cfl, int chunks);

/* Per-patch maximum eigenvalue of Q (Sec. 2.2, Sec. 4 "Reduction"):
 * lambda_out[i] = max over interior volumes and directions n of |u_n| + c
 * (device arrays). */
int fv_max_eigenvalue(fv_batch_t *b, const void *Q, double *lambda_out);

/* CFL time step per patch: dt_out[i] = cfl * dx[i] / (dim * lambda[i])
 * (device arrays of num_patches doubles; cfl > 0). */
int fv_cfl_time_step(fv_batch_t *b, const double *lambda, const double *dx,
                     double cfl, double *dt_out);

/* Conservation diagnostics: totals_out[i*N + k] = sum over the interior
 * volumes of patch i of unknown k, accumulated in double (device array of
 * num_patches * N doubles). */
int fv_conserved_totals(fv_batch_t *b, const void *Q, double *totals_out);

/*
 * steps explicit steps with device-side CFL chaining, ping-ponging between
 * two state buffers: step s reads Q_a (s even) or Q_b (s odd) and writes
 * the other; dt_a holds the first step's time steps and dt_a/dt_b
 * alternate as time-step buffers likewise.  lambda_out (may be NULL)
 * receives the eigenvalues of the final state.  With use_graph != 0 the
 * steps are captured once into a CUDA graph (cached per buffer set and
 * step count) and replayed; the result is identical to eager launches.
 * The final state is in Q_b if steps is odd, else in Q_a.
 */
int fv_batch_run(fv_batch_t *b, void *Q_a, void *Q_b, const double *dx,
                 double *dt_a, double *dt_b, double *lambda_out, int steps,
                 double cfl, int use_graph);

/*
 * Autotune the fused form: time every candidate launch shape of this
 * batch's kernel on the given buffers.  Q_out is scratch: it is zeroed
 * before each candidate, so afterwards its contents, halo volumes included,
 * are unspecified (pass a buffer other than the next step's input).  The
 * tuner checks that every candidate's output is bitwise identical to the first
 * one's, and keep the fastest.  Each timed launch follows a read of a
 * scratch buffer twice the size of L2 (allocated for the call, FV_ENOMEM if
 * it cannot be), so candidates are timed with their input in HBM.  Results are cached per device and batch
 * shape in memory and, if the environment variable FVBATCH_TUNE_CACHE names
 * a file, in that file.  Synchronises the stream.
 */
int fv_batch_tune(fv_batch_t *b, const void *Q_in, void *Q_out,
                  const double *dx, const double *dt);

/* Synchronise the batch's stream and report FV_ETIMEOUT if any kernel
 * since the last status check gave up a bounded wait, else FV_ENONPHYSICAL
 * if one met a non-physical state (and clear both). */
int fv_batch_status(fv_batch_t *b);

/* Free the batch (NULL-safe).  Synchronises its stream first.  A handle
 * that is not live (already destroyed, or never created) gives FV_EINVAL
 * and is not touched. */
int fv_batch_destroy(fv_batch_t *b);

/* Test hook for the out-of-memory paths; the paper has no counterpart.
 * k > 0 makes the k-th following device allocation of the library fail
 * (every call then returns FV_ENOMEM and leaves its batch usable); k <= 0
 * disarms it.  Process-wide. */
int fv_test_fail_device_alloc(int k);

/* Thread-local description of the last failure ("" if none). */
const char *fv_last_error(void);

/* Elements (not bytes) of one halo-inclusive state buffer of the batch. */
size_t fv_batch_state_elems(const fv_batch_t *b);

/* Device scratch bytes the batch holds (loop-cascade intermediates). */
size_t fv_batch_scratch_bytes(const fv_batch_t *b);

/* Write a one-line description of the selected kernels and launch shapes
 * into buf (NUL-terminated, truncated to len). */
int fv_batch_describe(const fv_batch_t *b, char *buf, size_t len);

/* Number of kernel launches one fv_patch_batch_update call makes with the
 * current form and arguments (lambda/dt outputs present): for the fused form
 * 1 when the batch is 2D with edges 4, 8, 16 and 32 only, else one per
 * patch-size class. */
int fv_batch_launches_per_update(const fv_batch_t *b);

/*
 * One update, like fv_patch_batch_update with the loop-cascade form, that
 * allocates no device memory; the paper has no counterpart (it is a service
 * for callers that cannot allocate).  For callers that cannot call
 * cudaMalloc where they step their patches: host callbacks or hooks that
 * run during CUDA-graph capture, processes whose device memory belongs to a
 * pooling allocator, plugins handed only their buffers.
 *
 * All num_patches patches have the edge length patch_size.  Arguments
 * otherwise mean what they mean in fv_batch_create and
 * fv_patch_batch_update; Q_in, Q_out, dx, dt, lambda_out and dt_next_out are
 * device pointers the caller owns, and the call runs asynchronously on
 * cuda_stream (a cudaStream_t, 0 = legacy default stream) on the current
 * device.  The metadata and the cascade's intermediates live in a built-in
 * 64 MiB device array that every GPU loading this library holds until the
 * process exits; a batch that needs more (about 1,300 two-dimensional
 * 16 x 16 patches in FP64, 2,700 in FP32) is rejected with FV_EINVAL and
 * nothing is launched.  The first call on a device looks up the array's
 * device address (make it before any stream capture); a call with
 * num_patches = 0 on that device does this lookup and nothing else, so it
 * serves as a cheap first call (no buffers needed).  All calls share the
 * array: calls whose work overlaps on the GPU race, so serialise them.
 * Non-physical states are not reported by this entry point (see the
 * returned eigenvalues instead).  Returns FV_OK or an FV_E* code.
 */
int fv_patch_batch_update_noalloc(int dim, int num_patches, int patch_size,
                                  int precision, int halo_mode, double gamma,
                                  const void *Q_in, void *Q_out,
                                  const double *dx, const double *dt,
                                  double *lambda_out, double *dt_next_out,
                                  double cfl, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FV_BATCH_H */
