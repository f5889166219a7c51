/*
 * sph.h -- C-ABI of the B300 SPH cell-pair offload library (libsph.so).
 *
 * The library implements the GPU-offload cycle of Sec. 2.3: cell-pair tasks
 * are gathered into bundles; for each bundle, "pack" gathers the particle
 * fields a loop reads (its view, Table 1) into a compact buffer, applying
 * the periodic shift to positions; the interaction kernel of the loop runs
 * on the buffer; "unpack" reduces the per-slot results back into the
 * particle store.  The particle store can use any of the memory layouts of
 * Sec. 3.1 (AoS, random-order AoS, split AoS by kernel view and by type,
 * SoA).  The loops are density, gradient and force, in that order
 * (Sec. 2.1), with a linear "ghost" update after density.
 *
 * Conventions (all entry points):
 *  - Every call returns an sph_status.  On failure sph_last_error() gives a
 *    message (thread-local, valid until the next call on the same thread).
 *  - GPU calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL is the legacy default stream).  Pointers named dev_* are device
 *    pointers; pointers named host_* are host pointers.
 *  - The library never allocates the large buffers: the particle store and
 *    the pack/result buffers are caller memory, sized by the *_bytes
 *    queries.  It allocates only the task metadata of an sph_tasks handle
 *    (host and, after sph_tasks_upload, device memory; freed by
 *    sph_tasks_destroy).
 *  - Handles are not thread-safe; use one handle per thread or serialise.
 *  - Particle indices are int64 on the host; on the device a store holds at
 *    most 2^31 - 1 particles and a bundle at most 2^31 - 1 slots.
 */
#ifndef SPH_H
#define SPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_store_s *sph_store;
typedef struct sph_tasks_s *sph_tasks;
typedef struct sph_batch_s *sph_batch;

/* Store layouts of Sec. 3.1. */
enum sph_layout {
    SPH_AOS = 0,                   /* one struct per particle, use order */
    SPH_AOS_RANDOM = 1,            /* AoS with members shuffled (seeded) */
    SPH_SAOS_PACK_GRAD = 2,        /* substruct = the gradient view */
    SPH_SAOS_PACK_FORCE = 3,       /* substruct = the force view */
    SPH_SAOS_PACK_SHARED = 4,      /* shared {x,v,m,h}, {u,rho}, force-only */
    SPH_SAOS_PACK_GRAD_TYPE = 5,   /* pack-gradient split by double/float/int */
    SPH_SAOS_PACK_FORCE_TYPE = 6,  /* pack-force split by type */
    SPH_SAOS_PACK_SHARED_TYPE = 7, /* pack-shared split by type */
    SPH_SOA = 8,                   /* one array per field component */
    SPH_SAOS_PACK_FORCE_REPL = 9,  /* pack-force plus the density view
                                      {x, v, m, h} stored again on its own
                                      (replicated positions, Sec. 5): the
                                      density pack reads only that copy */
    SPH_SAOS_FUSED = 10,           /* fused views: each loop's inputs with the
                                      outputs its unpack writes, in phase order */
    SPH_NUM_LAYOUTS = 11
};

/* Interaction loops of Sec. 2.1. */
enum sph_loop { SPH_DENSITY = 0, SPH_GRADIENT = 1, SPH_FORCE = 2 };

enum sph_status {
    SPH_OK = 0,
    SPH_EINVAL = 1,       /* bad argument (NULL handle, size, index, enum) */
    SPH_ENOMEM = 2,       /* host or device metadata allocation failed */
    SPH_ECUDA = 3,        /* a CUDA runtime call failed */
    SPH_EBOUNDS = 4,      /* a kernel saw an index outside its buffers */
    SPH_ETIMEOUT = 5,     /* a bounded device wait ran out (no current kernel waits) */
    SPH_EUNSUPPORTED = 6  /* valid request the library cannot serve */
};

/* Logical particle fields, one array per field in ORIGINAL particle order.
 * Vector fields (x, v, a, rot_v) hold 3 consecutive components per particle.
 * A NULL pointer means "not transferred". */
typedef struct {
    double *x;          /* positions, FP64 */
    float *v;           /* velocities */
    float *a;           /* accelerations (force loop output) */
    float *mass;
    float *h;           /* smoothing length; kernel support H = kernel_gamma h */
    float *u;           /* internal energy per unit mass */
    float *u_dt;        /* du/dt (force output) */
    float *rho;         /* density (density output, gradient/force input) */
    int8_t *time_bin;   /* force loop activity: active iff time_bin <= bin */
    float *alpha_visc;  /* artificial viscosity coefficient */
    float *alpha_diff;  /* artificial conduction coefficient */
    float *rho_dh;      /* d rho / d H */
    float *wcount;      /* weighted neighbour number (4 pi/3) H^3 sum W */
    float *wcount_dh;   /* d wcount / d H */
    float *div_v;       /* velocity divergence */
    float *rot_v;       /* velocity curl (3 components) */
    float *f_gradh;     /* grad-h factor 1/Omega */
    float *pressure;
    float *soundspeed;
    float *balsara;     /* Balsara switch */
    float *v_sig_grad;  /* signal velocity of the gradient loop */
    float *laplace_u;   /* Laplacian of u */
    float *h_dt;        /* dh/dt (force output) */
    float *v_sig;       /* signal velocity of the force loop */
    int64_t *id;        /* particle id (ballast for the loops) */
} sph_fields;

/* Physical parameters of the loops. */
typedef struct {
    double gamma;         /* adiabatic index, 5/3 */
    double kernel_gamma;  /* H / h of the cubic spline, 1.825742 */
    double beta_visc;     /* signal-velocity factor, 3 */
    double balsara_eps;   /* Balsara regulariser (times c/h), 1e-4 */
    int32_t active_bin;   /* force loop: particle active iff time_bin <= it */
    int32_t reserved;     /* must be 0 */
} sph_params;

/* Cell grid and bundling parameters for sph_tasks_build. */
typedef struct {
    double box[3];             /* periodic box edges (> 0) */
    double kernel_gamma;       /* H / h, as in sph_params */
    int32_t ncell[3];          /* cells per dimension, 0 = octree rule:
                                  halve the edge while the half is >= H_max */
    int32_t reserved;          /* must be 0 */
    int64_t bundle_max_slots;  /* bundle slot budget, <= 0: one bundle */
} sph_grid_params;

/* ---- library ---------------------------------------------------------- */
const char *sph_version(void);
const char *sph_last_error(void);

/* ---- particle store (Sec. 3.1) ----------------------------------------
 * A layout is a sequence of substructs; each substruct is a C struct of its
 * members with natural alignment, and the substruct arrays follow each other
 * in the caller's memory, each starting on a 256-byte boundary.
 * SPH_AOS_RANDOM shuffles the AoS members with a Fisher-Yates shuffle driven
 * by SplitMix64 seeded with `seed`; other layouts ignore `seed`. */

/* Bytes of caller memory a store of n particles needs (0 on bad input). */
size_t sph_store_bytes(int64_t n, int layout, uint64_t seed);

/* Number of substructs of a layout, or -1.  Host only. */
int sph_layout_group_count(int layout, uint64_t seed);

/* Describe substruct `group`: member count, member field ids (the order of
 * sph_fields, 25 = ballast bytes), component (SoA: 0..2, else -1), member
 * byte offsets, record bytes.  Arrays hold >= 26 entries.  Host only. */
int sph_layout_describe(int layout, uint64_t seed, int group, int32_t *nmem,
                        int32_t *field_ids, int32_t *comps, int32_t *offsets,
                        int32_t *record_bytes);

/* Create a store over caller device memory dev_mem (>= sph_store_bytes,
 * 256-byte aligned; owned by the caller and not freed by the library).
 * The memory is zero-filled (synchronously). */
int sph_store_create(int64_t n, int layout, uint64_t seed, void *dev_mem,
                     size_t bytes, sph_store *out);
int sph_store_destroy(sph_store s);

/* Copy logical fields into / out of the store.  Store slot k holds original
 * particle dev_perm[k] (device int64[n]; NULL = identity).  Fields whose
 * pointer is NULL are skipped.  All field pointers are device pointers. */
int sph_store_import(sph_store s, const sph_fields *dev_src,
                     const int64_t *dev_perm, void *stream);
int sph_store_export(sph_store s, const sph_fields *dev_dst,
                     const int64_t *dev_perm, void *stream);

/* ---- end-to-end host I/O ------------------------------------------------
 * A step's inputs live in page-locked host arrays and its results go back to
 * them: the offload cycle of Sec. 2.3 seen from an application whose data
 * stay on the host between steps.  A host I/O handle moves them through a
 * double-buffered device staging area so that, on the caller's streams,
 * step k+1's host-to-device copies and step k-1's device-to-host copies run
 * while step k computes:
 *
 *   sph_hostio_begin(io, host_in, stream)   H2D of every selected input on
 *        copy_in_stream into staging set k%2 (after that set's previous
 *        import finished), then, on `stream`, the import into the store;
 *   ... the step's library calls on `stream` ...
 *   sph_hostio_end(io, host_out, stream)    export into staging set k%2 on
 *        `stream` (after that set's previous D2H copies finished), then the
 *        D2H copies into host_out on copy_out_stream;
 *   sph_hostio_drain(io, stream)            `stream` waits for the last D2H.
 *
 * in_sel / out_sel select the fields: every non-NULL member is selected (its
 * value is not used).  The staging area is caller device memory of
 * sph_hostio_bytes bytes, 256-byte aligned; dev_perm is the store's
 * permutation (as for sph_store_import; the handle keeps the pointer).
 * host_in / host_out must hold exactly the selected fields, in original
 * particle order, each in page-locked host memory (SPH_EINVAL otherwise,
 * before anything is enqueued).  A host array must not be touched by the
 * host until the copies of its step are complete (after sph_hostio_drain and
 * a synchronisation of `stream`, or two steps later).  begin and end
 * alternate, one pair per step.  The handle owns eight CUDA events and
 * nothing else; sph_hostio_info gives the bytes copied per step (in, out)
 * and the steps completed.  Not thread-safe. */
typedef struct sph_hostio_s *sph_hostio;
size_t sph_hostio_bytes(int64_t n, const sph_fields *in_sel, const sph_fields *out_sel);
int sph_hostio_create(sph_store s, const int64_t *dev_perm, const sph_fields *in_sel,
                      const sph_fields *out_sel, void *dev_staging, size_t bytes,
                      void *copy_in_stream, void *copy_out_stream, sph_hostio *out);
int sph_hostio_begin(sph_hostio io, const sph_fields *host_in, void *stream);
int sph_hostio_end(sph_hostio io, const sph_fields *host_out, void *stream);
int sph_hostio_drain(sph_hostio io, void *stream);
int sph_hostio_info(sph_hostio io, int64_t info[3]);
int sph_hostio_destroy(sph_hostio io);

/* Layout conversion between two device stores of the same particles (same
 * count and order): every field of dst, every copy of a replicated one, from
 * src; the ballast bytes too.  One kernel pass.  This is the step a
 * kernel-dependent layout (one layout per algorithmic phase, Sec. 4) pays
 * between phases. */
int sph_store_convert(sph_store dst, sph_store src, void *stream);

/* ---- cells, tasks, bundles (Sec. 2.2-2.3) ------------------------------
 * Host-side builder.  Cells: a uniform grid with edges >= H_max =
 * kernel_gamma * max h (>= 3 cells per dimension).  Particles are sorted by
 * cell (ix fastest) with a stable counting sort; host_perm_out[k] receives
 * the original index of the k-th particle in cell order, to be passed to
 * sph_store_import.  Tasks: per non-empty cell a self task, then a pair
 * task for each of the 13 neighbour offsets after (0,0,0) in the (dz,dy,dx)
 * enumeration of {-1,0,1}^3 whose cell is not empty, the second cell's
 * particles shifted by -1/0/+1 box edges per dimension.  Bundles: greedy
 * consecutive task ranges of at most bundle_max_slots slots. */
int sph_tasks_build(int64_t n, const double *host_x, const float *host_h,
                    const sph_grid_params *gp, int64_t *host_perm_out,
                    sph_tasks *out);

/* Copy the task metadata to the current device (synchronous).  Required
 * before any GPU call that takes the handle. */
int sph_tasks_upload(sph_tasks t);

/* info[0..2] cells per dimension, [3] tasks, [4] bundles, [5] total slots,
 * [6] largest bundle slots, [7] non-empty cells, [8] particles,
 * [9] largest cell population.  Host only. */
int sph_tasks_info(sph_tasks t, int64_t info[10]);

/* Host copies of the task list: ci[ntasks], cj[ntasks] (-1 for self),
 * shift[3 ntasks], cell_start[ncells + 1], bundle_start[nbundles + 1].
 * Any pointer may be NULL.  Host only. */
int sph_tasks_get(sph_tasks t, int32_t *ci, int32_t *cj, int8_t *shift,
                  int64_t *cell_start, int64_t *bundle_start);

/* Largest buffer any bundle needs for `loop`: in_or_out 0 = pack buffer,
 * 1 = result buffer.  Lane k of a bundle of S slots starts at
 * sum_{l<k} round_up(S * size_l, 256) bytes; slots are ordered by task and,
 * inside a pair task, ci's particles then cj's.
 *   density  in : x0 x1 x2 (f64) | {vx vy vz m} (4 f32) | h
 *   gradient in : density in | u | rho
 *   force    in : gradient in | f_gradh | balsara | alpha_visc | alpha_diff |
 *                 time_bin (i8)
 *   density  out: {rho rho_dh wcount wcount_dh} | {div_v rot_x rot_y rot_z}
 *   gradient out: {v_sig_grad laplace_u}
 *   force    out: {ax ay az u_dt} | {h_dt v_sig}
 * Returns 0 on bad input. */
size_t sph_buffer_bytes(sph_tasks t, int loop, int in_or_out);

/* ---- the offload cycle (Sec. 2.3) --------------------------------------
 * For one loop: sph_init, then for every bundle b in order sph_pack ->
 * sph_density|gradient|force -> sph_unpack, then (after density) sph_ghost. */

/* Zero the outputs of `loop` in the store (force: active particles only). */
int sph_init(sph_store s, int loop, const sph_params *p, void *stream);

/* Gather the view of `loop` for bundle b into dev_buf_in.  Positions of a
 * pair task's second cell get x + shift * box in FP64 (Sec. 2.3). */
int sph_pack(sph_store s, sph_tasks t, int loop, int bundle, void *dev_buf_in,
             void *stream);

/* Interaction kernels: one result record per slot.  Slot of particle i in
 * task T holds the sums over the other cell of T (self task: over j != i of
 * the same cell):
 *   density : sum m_j W(r,H_i), sum m_j dW/dH(r,H_i), (4pi/3) H_i^3 sum W,
 *             its H-derivative, -sum m_j v_ij.rhat dW/dr, sum m_j v_ij x rhat
 *             dW/dr  (r < H_i; cubic spline, 8/pi normalisation)
 *   gradient: max_j (c_i + c_j - beta min(0, v_ij.rhat)),
 *             sum 2 m_j (u_i - u_j)/rho_j dW/dr(r,H_i)/r
 *   force   : a_i, du_i/dt, dh_i/dt contributions and max signal velocity
 *             over r < max(H_i, H_j); inactive i write zeros.
 * Positions are FP64 in the buffer; separations are formed in compensated
 * (two-float) arithmetic, the rest in FP32 with a compensated density sum. */
int sph_density(sph_tasks t, int bundle, const void *dev_buf_in,
                void *dev_buf_out, const sph_params *p, void *stream);
int sph_gradient(sph_tasks t, int bundle, const void *dev_buf_in,
                 void *dev_buf_out, const sph_params *p, void *stream);
int sph_force(sph_tasks t, int bundle, const void *dev_buf_in,
              void *dev_buf_out, const sph_params *p, void *stream);

/* Reduce bundle b's result buffer into the store: per particle, its slots in
 * increasing task order (ci before cj) are added to the stored value with
 * Kahan-compensated FP32 summation (compensation starting at 0 for each
 * call); signal velocities take the max.  Deterministic, no atomics. */
int sph_unpack(sph_store s, sph_tasks t, int loop, int bundle,
               const void *dev_buf_out, void *stream);

/* Linear update after `loop` (only SPH_DENSITY has one): add the self
 * contribution, divide div/curl by rho, and set f_gradh = 1/Omega,
 * pressure, sound speed and the Balsara switch. */
int sph_ghost(sph_store s, int after_loop, const sph_params *p, void *stream);

/* Convenience: the whole cycle of one loop over all bundles (init, pack,
 * kernel, unpack per bundle, ghost after density), on caller buffers of
 * sph_buffer_bytes(t, loop, 0/1) bytes. */
int sph_offload_loop(sph_store s, sph_tasks t, int loop, void *dev_buf_in,
                     void *dev_buf_out, const sph_params *p, void *stream);

/* Count the pair interactions of `loop` in bundle b (r < H_i for density and
 * gradient, r < max(H_i, H_j) for force, i active), added to
 * *dev_count (device uint64). */
int sph_count_pairs(sph_tasks t, int loop, int bundle, const void *dev_buf_in,
                    const sph_params *p, unsigned long long *dev_count,
                    void *stream);

/* Host-side fault injection, for tests of the error paths (no device fault
 * is ever caused): the countdown-th library use of `site` from now fails
 * once, as if the CUDA call had failed, and the call reports it (device
 * allocation of plan metadata: SPH_ENOMEM; metadata copy: SPH_ECUDA) after
 * releasing what it had set up.  SPH_FAULT_NONE or countdown 0 disarms.
 * The environment variable SPH_FAULT_INJECT=alloc:N or copy:N arms a site
 * the same way when the library is loaded. */
enum sph_fault_site { SPH_FAULT_NONE = 0, SPH_FAULT_DEVICE_ALLOC = 1, SPH_FAULT_COPY = 2 };
int sph_fault_inject(int site, int countdown);

/* Wait for `stream` and report errors latched by kernels: SPH_EBOUNDS (an
 * index outside its buffers), SPH_ETIMEOUT (a bounded wait ran out),
 * SPH_ENOMEM (a neighbour-list pool ran out). */
int sph_sync(void *stream);

/* ---- host-staged offload (Sec. 2.3, the paper's own setting) ------------
 * The store lives in host memory; pack gathers each bundle's view on the
 * host into a (pinned) host buffer, the buffer crosses the host link, the
 * interaction kernel runs, the results cross back and unpack reduces them
 * into the host store.  Host pack/unpack produce exactly the bytes / values
 * of sph_pack / sph_unpack.  `nthreads` <= 0 uses all OpenMP threads.
 * Device calls (sph_pack, sph_unpack, sph_init, sph_ghost, import/export)
 * reject a host store and the calls below reject a device store. */
int sph_store_create_host(int64_t n, int layout, uint64_t seed, void *host_mem,
                          size_t bytes, sph_store *out);
int sph_store_import_host(sph_store s, const sph_fields *host_src,
                          const int64_t *host_perm, int nthreads);
int sph_store_export_host(sph_store s, const sph_fields *host_dst,
                          const int64_t *host_perm, int nthreads);
int sph_pack_host(sph_store s, sph_tasks t, int loop, int bundle, void *host_buf_in,
                  int nthreads);
int sph_unpack_host(sph_store s, sph_tasks t, int loop, int bundle,
                    const void *host_buf_out, int nthreads);
/* Loop-fission variants of the host pack and unpack (Sec. 3.3): the same
 * bytes as sph_pack_host / sph_unpack_host, with the innermost loop split
 * by store substruct, by field component, by data type, or by substruct and
 * type (SPH_FISSION_NONE: one loop over all components).  The copies use one
 * generic body over component descriptors in every variant, so that only
 * the loop structure differs between them. */
enum sph_fission {
    SPH_FISSION_NONE = 0,
    SPH_FISSION_BY_STRUCT = 1,
    SPH_FISSION_BY_ELEMENT = 2,
    SPH_FISSION_BY_TYPE = 3,
    SPH_FISSION_BY_STRUCT_AND_TYPE = 4
};
int sph_pack_host_fission(sph_store s, sph_tasks t, int loop, int bundle, void *host_buf_in,
                          int fission, int nthreads);
int sph_unpack_host_fission(sph_store s, sph_tasks t, int loop, int bundle,
                            const void *host_buf_out, int fission, int nthreads);
int sph_init_host(sph_store s, int loop, const sph_params *p, int nthreads);
int sph_ghost_host(sph_store s, int after_loop, const sph_params *p, int nthreads);

/* One loop of the host-staged cycle over all bundles, double-buffered on two
 * streams: while bundle b's H2D copy, kernel and D2H copy run on streams[b%2],
 * the host packs bundle b+1 and unpacks bundle b-1.  host_in/host_out/dev_in/
 * dev_out each hold two buffers of sph_buffer_bytes(t, loop, 0 / 1) bytes
 * (host buffers should be pinned for the copies to be asynchronous).
 * Returns after the last unpack (and the ghost after density) on the host. */
int sph_offload_loop_host(sph_store s, sph_tasks t, int loop, void *const host_in[2],
                          void *const host_out[2], void *const dev_in[2],
                          void *const dev_out[2], const sph_params *p,
                          void *const streams[2], int nthreads);

/* The same loop with every stage timed, for the breakdown of the offload
 * time into the host pack, the transfers, the kernels and the host unpack
 * (Sec. 2.3-2.5, Fig. 1).  Host stages are timed on the host clock; the
 * H2D copy, the kernel and the D2H copy of each bundle with CUDA events on
 * its stream (summed over bundles; they overlap the host stages and each
 * other across the two streams, so the parts add up to more than wall_s).
 * stats must be non-NULL.  Costs 4 events per bundle. */
typedef struct {
    double wall_s;         /* the whole call, host clock */
    double host_pack_s;    /* host pack of every bundle */
    double host_unpack_s;  /* host unpack of every bundle (and the ghost after density) */
    double host_wait_s;    /* host blocked on a bundle's device work */
    double h2d_ms;         /* device time of the host-to-device copies */
    double kernel_ms;      /* device time of the interaction kernels */
    double d2h_ms;         /* device time of the device-to-host copies */
    int64_t h2d_bytes;     /* bytes copied host to device */
    int64_t d2h_bytes;     /* bytes copied device to host */
    int64_t bundles;
} sph_staged_stats;
int sph_offload_loop_host_stats(sph_store s, sph_tasks t, int loop, void *const host_in[2],
                                void *const host_out[2], void *const dev_in[2],
                                void *const dev_out[2], const sph_params *p,
                                void *const streams[2], int nthreads, sph_staged_stats *stats);

/* ---- offload cycle without any allocation ------------------------------
 * The paper has no counterpart to this entry point.  It is for callers that
 * cannot allocate device memory while they run: for example a host
 * application whose device memory is entirely reserved by its own pool
 * allocator, or a loop that may not pay the latency and implicit
 * synchronisation of cudaMalloc/cudaFree after start-up.
 *
 * It does what sph_offload_loop does, but the pack and result buffers live in
 * one scratch array of SPH_NOALLOC_SCRATCH_BYTES that the library defines in
 * device memory; every GPU that loads the library holds this array until the
 * process exits.  The caller still provides the store and the uploaded tasks.
 * The call allocates nothing (no cudaMalloc, no cudaFree, no allocating
 * library routine).
 *
 * Limits and behaviour:
 *  - The buffers of the largest bundle of `loop` (sph_buffer_bytes(t, loop,
 *    0) and (t, loop, 1), each rounded up to 256 bytes) must fit in
 *    SPH_NOALLOC_SCRATCH_BYTES together; otherwise the call returns
 *    SPH_EUNSUPPORTED without launching anything.  Choose bundle_max_slots
 *    in sph_tasks_build accordingly (e.g. 300000 slots fit every loop).
 *  - The first call on a device looks up that device's address of the array
 *    (with that device current); make this first call before any stream
 *    capture is started on the device.  The address is kept for the life of
 *    the process: after cudaDeviceReset (or any other teardown of the
 *    device's primary context) the array may live elsewhere, so do not call
 *    this entry point again in that process.
 *  - All calls share the one array and it keeps whatever the last call left
 *    in it.  Nothing in it needs to start at zero: each bundle's pack buffer
 *    is written in full before it is read, and so is its result buffer.
 *  - Calls whose work overlaps on the GPU (for example on two streams, or
 *    from two threads) race on the array and give wrong results; serialise
 *    them. */
#define SPH_NOALLOC_SCRATCH_BYTES (32u << 20)

/* ---- batched (cell-dedup) offload ---------------------------------------
 * The same interactions as the per-task cycle, with the bundling of Sec. 2.3
 * taken further: a bundle is a range of target cells; each cell the range
 * needs (targets and their periodic neighbours) is packed once per bundle
 * (positions already split for the FP32 kernels), and one persistent launch
 * works through (target cell, particle chunk) items in longest-first order,
 * each computing its particles' sums over all the target's neighbour
 * entries (the 27 periodic neighbour cells of the grid plan, or the
 * box-distance entries of the tree plan).  Unpack
 * adds each target particle's single result into the store (no per-slot
 * reduction).  Outputs agree with the per-task cycle to rounding (the sum
 * order over neighbours differs). */
typedef struct {
    int64_t max_target_cells;  /* target cells per bundle, <= 0: all */
    int32_t threads;           /* CTA size of the persistent kernels: 64, 128, 256
                                  (a work item is one warp of 32 particles) */
    int32_t reserved;          /* must be 0 */
} sph_batch_params;

/* Build a batch plan from a task handle's cells (host) and upload it to the
 * current device (allocates the plan's device metadata).
 *
 * A plan (this one or a tree plan) holds for the positions and supports it
 * was built from.  Every cell records the largest support the plan holds
 * for it: here the shortest cell edge (any support up to it keeps every
 * interacting pair in adjacent cells), for a tree plan the leaf's largest
 * support at build time (its neighbour entries were found with it).  Each
 * density pack checks the cell's current supports against that limit; a
 * larger one, whose pairs the plan may miss, is reported by the next
 * sph_sync as SPH_EUNSUPPORTED, and the plan must be rebuilt.  The list
 * build's fixed-point path (sph_batch_list_fixed) is decided from the same
 * supports, so it stays valid while no such report occurs.  Particles that
 * leave their cell also need a new plan; that is the caller's to track. */
int sph_batch_build(sph_tasks t, const sph_batch_params *bp, sph_batch *out);
/* info[0] bundles, [1] largest bundle slots, [2] work items, [3] threads,
 * [4] largest bundle target slots, [5] packed cells (all bundles). */
int sph_batch_info(sph_batch b, int64_t info[6]);
/* Largest buffer of any bundle for `loop` (0 pack, 1 result). */
size_t sph_batch_buffer_bytes(sph_batch b, int loop, int in_or_out);
int sph_batch_pack(sph_store s, sph_batch b, int loop, int bundle, void *dev_buf_in,
                   const sph_params *p, void *stream);
int sph_batch_interact(sph_batch b, int loop, int bundle, const void *dev_buf_in,
                       void *dev_buf_out, const sph_params *p, void *stream);
/* Adds each target particle's result of one bundle into the store (maxima
 * for the signal velocities), as the per-task unpack does; the store's
 * outputs of the loop must be initialised (sph_init) before the first
 * bundle. */
int sph_batch_unpack(sph_store s, sph_batch b, int loop, int bundle, const void *dev_buf_out,
                     const void *dev_buf_in, void *stream);
/* The same result without sph_init: each target particle's outputs are
 * written as the fold onto an initialised store would leave them (0 + v,
 * max(0, v); inactive particles of the force loop keep theirs, which equals
 * the fold for signal velocities >= 0).  Valid because a batched plan holds
 * every particle's cell as a target in exactly one bundle, so one bundle's
 * result is the particle's whole sum.  with_ghost != 0 (density loop only):
 * the bundle's targets also get the ghost, bit for bit as sph_ghost after
 * the last bundle would give, so no separate ghost pass is needed. */
int sph_batch_unpack_write(sph_store s, sph_batch b, int loop, int bundle,
                           const void *dev_buf_out, const void *dev_buf_in, const sph_params *p,
                           int with_ghost, void *stream);
/* Per bundle pack -> interact -> unpack (written, no init pass; after the
 * density loop with the ghost fused); enqueues only (no host
 * synchronisation), so it can be recorded into a CUDA graph after a first
 * call. */
int sph_batch_offload_loop(sph_store s, sph_batch b, int loop, void *dev_buf_in,
                           void *dev_buf_out, const sph_params *p, void *stream);
int sph_batch_destroy(sph_batch b);

/* ---- adaptive plan for clustered particle sets -------------------------
 * A uniform grid needs cell edges >= the largest support, so when h spans
 * decades (clustered sets) its cells hold up to millions of particles.  The
 * tree plan replaces the grid's cells by the leaves of an octree over the
 * particles' Morton keys (21 bits per dimension; positions are clamped into
 * the box the way the grid builder clamps them): a node is split while it
 * holds more than leaf_max particles.  Each leaf's neighbour entries are all
 * (leaf, periodic shift) pairs whose particle bounding boxes are closer than
 * max(H_max of either leaf) + 4e-6 * (largest box edge), found by a pruned
 * walk of the tree; the batched kernels then run unchanged over those lists.
 * host_perm_out[k] receives the original index of the k-th particle in leaf
 * (Morton) order, to be passed to sph_store_import.  Requires every support
 * to be below half the smallest box edge (one periodic image per pair);
 * SPH_EUNSUPPORTED otherwise.  Host inputs, uploads the plan to the current
 * device. */
typedef struct {
    double box[3];
    double kernel_gamma;
    int32_t leaf_max;    /* 8 .. 2048 */
    int32_t rule;        /* 0: split while a node holds > leaf_max particles;
                            1: the octree rule of the cell tree (Sec. 2.2) as well:
                            split only while half the node's edge is >= the
                            largest support of its particles, so leaves can
                            hold far more than leaf_max */
} sph_tree_params;
int sph_batch_build_tree(int64_t n, const double *host_x, const float *host_h,
                         const sph_tree_params *tp, const sph_batch_params *bp,
                         int64_t *host_perm_out, sph_batch *out);
/* The tree plan's leaves and neighbour entries, on the host only (no device
 * call): leaf l holds Morton-ordered particles [leaf_start[l], leaf_start[l+1])
 * (arrays of n + 1 entries suffice), its entries are nb[nb_start[l] ..
 * nb_start[l+1]), each (leaf << 6) | shift code.  *nleaf_out and *nnb_out
 * receive the counts; SPH_EINVAL if nb_cap < *nnb_out (nb may then be NULL:
 * call once to size nb). */
int sph_tree_plan(int64_t n, const double *host_x, const float *host_h,
                  const sph_tree_params *tp, int64_t *host_perm_out,
                  int64_t *host_leaf_start, int64_t *nleaf_out, int64_t *host_nb_start,
                  int32_t *host_nb, int64_t nb_cap, int64_t *nnb_out);
/* info[0] plan kind (0 grid, 1 tree), [1] cells or leaves with particles,
 * [2] largest cell / leaf population, [3] neighbour entries (all cells). */
int sph_batch_plan_info(sph_batch b, int64_t info[4]);
/* The cells one bundle packs, in pack order (host-side copy): *ncells gets
 * their count and, when cells is non-NULL, cells gets three int32 per cell:
 * its first store particle, its particle count and its first bundle slot. */
int sph_batch_cells(sph_batch b, int bundle, int32_t *cells, int64_t *ncells);
/* 1 when the plan's list build decides pairs on 32-bit fixed-point
 * separations (every cell or leaf extent plus the largest support is below
 * half the box, so minimum images are unambiguous), 0 when it uses two-float
 * separations with the entries' periodic shifts; -SPH_EINVAL for NULL. */
int sph_batch_list_fixed(sph_batch b);
/* Pair interactions of `loop` over the plan, decided in FP64 as the loops
 * define them (density and gradient: r < H_i; force: r < max(H_i, H_j),
 * active i only), added to *dev_count (device uint64).  Uses dev_buf_in of
 * sph_batch_buffer_bytes_fp64(b, 0) bytes as scratch. */
int sph_batch_count_pairs(sph_store s, sph_batch b, int loop, void *dev_buf_in,
                          const sph_params *p, unsigned long long *dev_count, void *stream);

/* ---- neighbour-list variant of the batched cycle --------------------------
 * The batched interaction kernels test all candidates of a target's
 * neighbour entries again in each loop.  The list variant tests them once per
 * step: sph_batch_list_build packs the density view of each bundle and
 * stores, for every target particle, the bundle slots of the j with
 * r < max(H_i, H_j) (flagged when r < H_i), decided exactly as the loops
 * decide; sph_batch_offload_loop_list then runs each loop over the lists
 * (pack -> list loop -> unpack per bundle, the ghost fused into the
 * density unpack).  Results
 * equal the batched cycle's up to the rounding order of r^2.
 * The list buffer (caller memory, 256-byte aligned) holds a header, per-item
 * tables and a pool of chunks of 2048 entries; sph_batch_list_bytes(b, c)
 * is the size with room for c chunks.  If the pool runs out, the build marks
 * the buffer, the loops skip their pairs, and sph_sync returns SPH_ENOMEM;
 * sph_batch_list_status (synchronous) then gives the chunks needed.  Lists
 * depend on positions and h only: build once per step, before the density
 * loop, with the same plan. */
size_t sph_batch_list_bytes(sph_batch b, int64_t chunks);
int sph_batch_list_build(sph_store s, sph_batch b, void *dev_buf_in, void *dev_list,
                         size_t list_bytes, const sph_params *p, void *stream);
/* One bundle's part of sph_batch_list_build, from a dev_buf_in that already
 * holds this bundle's density pack (sph_batch_pack_list, loop 0), so the
 * density loop's pack serves the build too.  Bundle 0 resets the list
 * header: build the bundles of a step in order, 0 first. */
int sph_batch_list_build_bundle(sph_store s, sph_batch b, int bundle, const void *dev_buf_in,
                                void *dev_list, size_t list_bytes, const sph_params *p,
                                void *stream);
int sph_batch_list_status(const void *dev_list, int64_t *chunks_needed, int *overflow);
/* The list build tests each cell pair once where the plan allows it (one
 * bundle whose targets are all its cells, the fixed-point path, a symmetric
 * neighbour relation: grid plans of at least 5 cells per dimension): a
 * first pass tests the target's own cell and the cells after it and keeps
 * the hit masks of the latter in the list buffer (sph_batch_list_bytes
 * counts them); a second pass gives each particle the pairs its cell's
 * earlier neighbours found, by transposing their masks.  The lists hold the
 * same pairs either way (in another order).  enable 0 / 1 turns it off / on
 * for later builds, a negative value only asks; returns 1 when later builds
 * of this plan use it, 0 when not, a negative status on error. */
int sph_batch_list_symmetric(sph_batch b, int enable);
/* Measurement variant of sph_batch_list_build_bundle (the paper has no
 * counterpart; it states the list build's work from what it tests): builds
 * the same lists and adds into dev_counts[0..4] (device uint64, 8-byte
 * aligned, zeroed by the caller) the candidates staged, the (particle,
 * candidate) pairs that pass the warp-box cull and are prefiltered, the
 * prefilter's hits, the hits that take the exact test, and the list entries
 * written.  Slower than the build it counts; not for timed runs. */
int sph_batch_list_count(sph_store s, sph_batch b, int bundle, const void *dev_buf_in,
                         void *dev_list, size_t list_bytes, const sph_params *p,
                         unsigned long long *dev_counts, void *stream);
/* The pack of the list loops: the density view as sph_batch_pack, the
 * gradient and force views as compact records (c and P recomputed in the
 * loop from u and rho, so each gathered j record is 48 / 64 bytes). */
int sph_batch_pack_list(sph_store s, sph_batch b, int loop, int bundle, void *dev_buf_in,
                        const sph_params *p, void *stream);
/* One bundle's list loop (after sph_batch_pack_list of the same loop and
 * bundle); results land in dev_buf_out for sph_batch_unpack. */
int sph_batch_list_interact(sph_batch b, int loop, int bundle, const void *dev_buf_in,
                            void *dev_buf_out, const void *dev_list, size_t list_bytes,
                            const sph_params *p, void *stream);
int sph_batch_offload_loop_list(sph_store s, sph_batch b, int loop, void *dev_buf_in,
                                void *dev_buf_out, const void *dev_list, size_t list_bytes,
                                const sph_params *p, void *stream);
/* A whole step of the list cycle in one call: per bundle the density pack,
 * that bundle's list build from it, the density list loop and its unpack
 * with the ghost; then the gradient and force loops as
 * sph_batch_offload_loop_list.
 * Enqueues only.  A list pool that runs out is reported by sph_sync
 * (SPH_ENOMEM) and sph_batch_list_status, as for sph_batch_list_build; the
 * step's loops then skip all pairs. */
int sph_batch_offload_step_list(sph_store s, sph_batch b, void *dev_buf_in, void *dev_buf_out,
                                void *dev_list, size_t list_bytes, const sph_params *p,
                                void *stream);

/* Host-staged batched cycle: a host store (sph_store_create_host, in the
 * plan's particle order) and a batch plan; per bundle, host threads pack
 * the bundle's records (its cells once each, particles of a cell in store
 * order) into host_in[k], which goes H2D into dev_in[k] on streams[k], the
 * batched kernel runs, the results come back D2H into host_out[k] and host
 * threads fold each target particle's result into the store, bundles
 * alternating between the two buffer sets.  init before, ghost after the
 * density loop, on the host.  Buffers: sph_batch_buffer_bytes(b, loop, 0/1)
 * bytes each (pinned host memory for the transfers to overlap). */
int sph_batch_offload_loop_host(sph_store s, sph_batch b, int loop, void *const host_in[2],
                                void *const host_out[2], void *const dev_in[2],
                                void *const dev_out[2], const sph_params *p,
                                void *const streams[2], int nthreads);

/* Precision study (the paper fixes no precision; this is the arrangement
 * that keeps FP64 only where cancellation bites): the list step of
 * sph_batch_offload_step_list with every pair separation in the three loops
 * taken as the difference of the two FP64 positions, its periodic image
 * chosen in FP64, then rounded to FP32; the fields, the pair bodies, the
 * compensated density sum and the lists (decided as in the list step) are
 * unchanged.  dev_x64: caller device memory of sph_batch_x64_bytes(b) bytes,
 * 256-byte aligned, where each pack's slots get their FP64 positions.
 * Slower than the list step: the B300's FP64 pipe runs a small fraction of
 * its FP32 rate. */
size_t sph_batch_x64_bytes(sph_batch b);
int sph_batch_offload_step_list_x64(sph_store s, sph_batch b, void *dev_buf_in,
                                    void *dev_buf_out, void *dev_list, size_t list_bytes,
                                    void *dev_x64, size_t x64_bytes, const sph_params *p,
                                    void *stream);

/* ---- adjoint of density -> ghost -> force (differentiation) --------------
 * Gradient of L = sum_i |a_i|^2 + sum_i (du_i/dt)^2 (active particles) with
 * respect to positions, masses and internal energies, for upstream adjoints
 * dev_abar = dL/da (n x 3) and dev_ebar = dL/d(du/dt) (n), both in ORIGINAL
 * particle order like the outputs dev_gx (n x 3, FP64), dev_gm, dev_gu (n).
 * dev_store_perm is the permutation passed to sph_store_import (NULL for the
 * identity).  Smoothing lengths, velocities and the switches' coefficients
 * are held fixed.  Preconditions: a plan of one bundle, the store holding the
 * results of the list cycle (sph_batch_list_build then the three
 * sph_batch_offload_loop_list calls, or sph_batch_offload_step_list) on the
 * current inputs, and that list
 * buffer.  Scratch: sph_batch_adjoint_bytes(b) bytes (0 when the plan has
 * more than one bundle).  Every particle gathers both directions of its
 * pairs from its list: no atomics, deterministic.  FP32 arithmetic. */
size_t sph_batch_adjoint_bytes(sph_batch b);
int sph_batch_adjoint(sph_store s, sph_batch b, void *dev_buf_in, const void *dev_list,
                      size_t list_bytes, void *dev_scratch, size_t scratch_bytes,
                      const int64_t *dev_store_perm, const float *dev_abar,
                      const float *dev_ebar, double *dev_gx, float *dev_gm, float *dev_gu,
                      const sph_params *p, void *stream);

/* All-FP64 variant of the batched cycle (precision study): the same cells and
 * results, every arithmetic step in FP64 (positions, separations, kernel
 * values, sums, ghost), results rounded to the FP32 store once.  Buffers of
 * sph_batch_buffer_bytes_fp64(b, 0 / 1) bytes. */
size_t sph_batch_buffer_bytes_fp64(sph_batch b, int in_or_out);
int sph_batch_offload_loop_fp64(sph_store s, sph_batch b, int loop, void *dev_buf_in,
                                void *dev_buf_out, const sph_params *p, void *stream);
int sph_offload_loop_noalloc(sph_store s, sph_tasks t, int loop, const sph_params *p,
                             void *stream);


/* ---- measurement utility -------------------------------------------------
 * The paper has no counterpart to this call: it measures the arithmetic
 * peaks that the interaction loops' roofline is stated against (they run on
 * the FP32 CUDA cores; an FP64 separation would use the FP64 pipe).  One
 * launch of 8 CTAs of 256 threads per SM, each thread running 8 independent
 * chains of `iters` x 16 operations: kind 0 FP32 fused multiply-add (2 flops
 * each), 1 FP64 fused multiply-add (2 flops), 2 FP64 add (1 flop).
 * *flops_out gets the launch's flop count; the caller times the launch on
 * `stream` (CUDA events) and divides.  dev_sink: 256-byte aligned device
 * memory of at least 8 bytes, which the kernel may write. */
int sph_peak_run(int kind, int64_t iters, void *dev_sink, void *stream, double *flops_out);

int sph_tasks_destroy(sph_tasks t);

#ifdef __cplusplus
}
#endif
#endif /* SPH_H */
