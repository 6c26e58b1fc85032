/*
 * simlod.h: C ABI of the GB300 incremental octree LOD update.
 *
 * The method is SimLOD's per-batch update (Schuetz, Herzberger, Wimmer,
 * "SimLOD: Simultaneous LOD Generation and Rendering", Section 5): every
 * arriving batch of points is counted into the current leaves, leaves holding
 * more than T points split into 8 children until no leaf spills (Section 5.1),
 * every point samples a voxel in the 128^3 occupancy grid of each inner node
 * on its way down (Section 5.2), chunks are allocated from a pool and a bump
 * allocator (Sections 3.2, 3.4, 5.3) and points and voxels are stored into
 * linked chunks of C records (Section 5.4).
 *
 * Determinism: the result after every batch is a pure function of the point
 * stream. Where the GPU would race, the contract fixes the winner: a voxel
 * takes the colour of the point with the lowest global arrival index (gidx)
 * among the points that reach its empty cell, per node (Section 5.2's "first
 * point"). Orders inside chunks, chunk addresses and pool order are not part
 * of the result; the canonical snapshot sorts them away.
 *
 * Memory: the caller owns one device buffer, the arena, the analogue of the
 * paper's persistent buffer (Section 3.2). The library carves its node table,
 * work buffers and the bump-allocated data region (grids and chunks) out of it
 * and never allocates device memory itself. Host-side state (the handle, a
 * small pinned control-block mirror, CUDA events) is the library's.
 *
 * Errors: every entry point returns an int status, 0 on success and a
 * negative SIMLOD_ERR_* code otherwise. Nothing throws across the ABI and no
 * kernel traps. A device-side capacity failure (arena, nodes, spill, backlog)
 * poisons the handle: later calls return SIMLOD_ERR_POISONED (the sticky
 * cause is in simlod_stats.sticky_status) and simlod_destroy still works.
 *
 * Threading: a handle is not thread-safe; calls on one handle must be
 * serialised by the caller. Different handles are independent.
 */
#ifndef SIMLOD_H
#define SIMLOD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SIMLOD_API __attribute__((visibility("default")))
#else
#define SIMLOD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* A point: int32 coordinates (1 mm units in the workloads here) and RGBA8,
 * 16 bytes, 16-byte aligned in device buffers. The paper's SIM format stores
 * float xyz + RGBA8 in the same 16 bytes (Section 7.1). */
typedef struct {
  int32_t x, y, z;
  uint8_t r, g, b, a;
} simlod_point;

/* Octree parameters. simlod_config_default() fills the paper's values. */
typedef struct {
  int32_t root_min[3];       /* root cube [root_min, root_min + 2^root_log2) per axis */
  uint32_t root_log2;        /* 1..31 */
  uint32_t leaf_capacity;    /* T: a leaf splits when it would hold more (50,000; Section 3.1) */
  uint32_t chunk_points;     /* C: records per chunk (1,000; Section 3.4), 1..65,536 */
  uint32_t grid_log2;        /* G: sampling grid 2^G per axis (7 = 128^3; Section 3.3), 1..7 */
  uint32_t max_expand_iters; /* expansion rounds per update; 0 = root_log2 + 1 (enough) */
  uint64_t max_batch_points; /* largest n accepted by one insert, 1..2^31-1 */
  uint64_t spill_capacity;   /* points re-inserted from split leaves, per update, < 2^31 */
  uint64_t backlog_capacity; /* new voxels per update (10M suggested; Section 5.2) */
  uint64_t max_nodes;        /* node table size (9 .. 2^27) */
  uint32_t flags;            /* reserved, 0 */
  uint32_t reserved;
} simlod_config;

/* Canonical snapshot records (see simlod_snapshot). rgba = r | g<<8 | b<<16 | a<<24. */
typedef struct {
  uint32_t level, is_inner;
  int32_t min[3];
  uint32_t log2size;
  uint64_t n_points, n_voxels, n_chunks;
} simlod_node_rec;

typedef struct {
  int32_t x, y, z;
  uint32_t rgba;
  uint32_t gidx;
} simlod_point_rec;

typedef struct {
  uint32_t cell; /* cx + 2^G (cy + 2^G cz) */
  int32_t x, y, z;
  uint32_t rgba;
} simlod_voxel_rec;

/* Snapshot buffers: caller-owned host arrays and their capacities (in
 * records). Call once with all three pointers NULL to learn the sizes, then
 * again with buffers at least that large. */
typedef struct {
  simlod_node_rec* nodes;
  uint64_t nodes_capacity;
  simlod_point_rec* points;
  uint64_t points_capacity;
  simlod_voxel_rec* voxels;
  uint64_t voxels_capacity;
  uint64_t n_nodes, n_points, n_voxels; /* out */
} simlod_snapshot_t;

typedef struct {
  uint64_t batches, points, rejected_batches;
  uint64_t spilled, splits, voxels, iterations_max;
  uint64_t rounds; /* expansion rounds summed over updates (one control-block read each) */
  uint64_t nodes;
  uint64_t chunks_bumped, chunks_pool;
  uint64_t arena_bytes, data_bytes, data_used;
  /* the last applied update */
  uint64_t last_points, last_spilled, last_splits, last_voxels, last_iterations;
  int32_t sticky_status; /* the error that poisoned the handle, or 0 */
  uint32_t device_error_bits;
  /* the last simlod_render: nodes drawn, points and voxels visited */
  uint64_t render_nodes, render_samples;
  /* compaction (simlod_compact): nodes that are arrays now and the chunks
   * they stand in for; nodes turned into arrays and chunks given back to the
   * pool since create/reset; arrays turned back into chunk lists by inserts */
  uint64_t compact_nodes, compact_chunks, compacted_total, compact_chunks_freed,
      decompacted_total;
} simlod_stats;

/* Per-kernel device time, accumulated while timing is enabled, and the
 * time the fused form spent per phase (measured on the GPU timer between
 * its grid barriers, accumulated since create/reset or the last clear). */
#define SIMLOD_N_KERNELS 8
#define SIMLOD_N_PHASES 8
typedef struct {
  const char* name[SIMLOD_N_KERNELS];
  uint64_t launches[SIMLOD_N_KERNELS];
  double ms[SIMLOD_N_KERNELS];
  const char* phase_name[SIMLOD_N_PHASES];
  double phase_ms[SIMLOD_N_PHASES];
} simlod_timing;

enum {
  SIMLOD_OK = 0,
  SIMLOD_ERR_INVALID_ARG = -1,
  SIMLOD_ERR_OUT_OF_BOUNDS = -2, /* a point outside the root cube: batch rejected, no change */
  SIMLOD_ERR_ARENA_FULL = -3,    /* data region exhausted (grids + chunks) */
  SIMLOD_ERR_BACKLOG_FULL = -4,  /* more new voxels in one update than backlog_capacity */
  SIMLOD_ERR_SPILL_FULL = -5,    /* more re-inserted points than spill_capacity */
  SIMLOD_ERR_ITER_CAP = -6,      /* expansion needed more than max_expand_iters rounds */
  SIMLOD_ERR_TIMEOUT = -7,       /* a bounded device wait gave up */
  SIMLOD_ERR_POISONED = -8,      /* an earlier device error: only destroy/stats/status work */
  SIMLOD_ERR_CUDA = -9,          /* a CUDA runtime call failed */
  SIMLOD_ERR_NODES_FULL = -10,   /* node table exhausted */
  SIMLOD_ERR_TOO_MANY_POINTS = -11 /* 2^32 points per octree (gidx is 32-bit) */
};

/* Fill cfg with the paper's parameters: T = 50,000, C = 1,000, 128^3 grids,
 * a 10M-voxel backlog; root cube [0, 2^20)^3; batches up to 16M points. */
SIMLOD_API void simlod_config_default(simlod_config* cfg);

/* Bytes of arena needed for cfg with a data region of data_bytes (grids and
 * chunks). Returns SIMLOD_ERR_INVALID_ARG for an invalid cfg. */
SIMLOD_API int simlod_arena_bytes(const simlod_config* cfg, uint64_t data_bytes,
                                  uint64_t* arena_bytes);

typedef struct simlod simlod_t; /* opaque handle */

/* Create an octree in the caller's device arena (256-byte aligned,
 * arena_bytes long; it must stay allocated until simlod_destroy). Everything
 * left after the fixed regions becomes the data region. The arena is
 * initialised on `stream` (a cudaStream_t; NULL = the legacy default stream)
 * and the call returns after that work completed. The octree starts as one
 * empty leaf, the root. */
SIMLOD_API int simlod_create(const simlod_config* cfg, void* d_arena, size_t arena_bytes,
                             void* stream, simlod_t** out);

/* Insert one batch of n points (Section 5): d_pts is a device pointer to n
 * 16-byte records (16-byte aligned), read-only for the library. The batch is
 * one complete update: expansion, voxel sampling,
 * chunk allocation and storing. Batches are applied in call order; the k-th
 * point ever accepted gets gidx k. n = 0 is a no-op.
 *
 * The work runs on `stream`, in stream order after earlier work there. The
 * expansion rounds are steered from the host: the call waits for the stream
 * once per round (a read of the control block), then enqueues the final
 * store and returns without waiting for it. d_pts must therefore stay valid
 * and unchanged until `stream` has passed the insert (record an event or
 * synchronise). Returns SIMLOD_ERR_OUT_OF_BOUNDS, with the octree and the
 * gidx counter unchanged, when any point lies outside the root cube. Calls on
 * one handle must be ordered: use one stream, or order the streams. */
SIMLOD_API int simlod_insert_batch(simlod_t* h, const simlod_point* d_pts, uint64_t n,
                                   void* stream);

/* As simlod_insert_batch for a batch in host memory: the points are copied
 * into a staging region of the arena on `stream` first (page-locked host
 * memory makes the copy asynchronous and fast). */
SIMLOD_API int simlod_insert_batch_host(simlod_t* h, const simlod_point* h_pts, uint64_t n,
                                        void* stream);

/* Fused form: apply batches 0 .. n_batches-1 in order, each one complete
 * update as in simlod_insert_batch, all inside one persistent cooperative
 * launch on `stream` (Section 4: persistent threads with grid-wide syncs, the
 * update kernel looping over the batches that have arrived). The phases are
 * separated by grid barriers with a time limit, so no expansion round goes
 * back to the host. Asynchronous: the call returns after enqueueing (it first
 * waits for its own previous batch-table copy) and d_batches[k] (device
 * pointers, 16-byte aligned) must stay valid until `stream` passes the
 * launch. At most 16,384 batches per call. A batch with a point outside the
 * root cube is skipped without change; the next simlod_sync then returns
 * SIMLOD_ERR_OUT_OF_BOUNDS once. Device errors are reported by simlod_sync. */
SIMLOD_API int simlod_insert_batches(simlod_t* h, const simlod_point* const* d_batches,
                                     const uint64_t* counts, uint32_t n_batches, void* stream);

/* Fused form fed from page-locked host memory (the host ingest pipeline;
 * Section 4: the update kernel loops over the batches uploaded so far).
 * Batch k is copied from h_batches[k] (page-locked host memory) to d_dst,
 * the batches packed in order (d_dst: device memory, 16-byte aligned, room
 * for the sum of counts), on copy_stream, and a 4-byte copy then sets
 * d_ready[k] (n_batches words of device memory, cleared on `stream` first).
 * One persistent launch on `stream` applies the batches in order, as
 * simlod_insert_batches does, and starts batch k once d_ready[k] is set, so
 * each copy overlaps the updates of the batches before it. copy_stream must
 * not wait for work enqueued on `stream` after this call: a flag that stays
 * clear for 2 s aborts the launch (simlod_sync then returns
 * SIMLOD_ERR_TIMEOUT and the handle is poisoned). copy_stream may equal
 * `stream` (no overlap). h_batches, d_dst and d_ready must stay valid until
 * `stream` passes the launch. Rejections and errors as in
 * simlod_insert_batches. */
SIMLOD_API int simlod_insert_batches_host(simlod_t* h, const simlod_point* const* h_batches,
                                          const uint64_t* counts, uint32_t n_batches,
                                          simlod_point* d_dst, uint32_t* d_ready, void* stream,
                                          void* copy_stream);

/* Batched form: a plan for a fixed list of uneven batches (device pointers,
 * 16-byte aligned, at most 16,384), run as one CUDA graph (when capture is
 * possible, else as direct launches) of three kernels: a check of every batch
 * against the root cube (a batch with a point outside it is rejected whole,
 * without change, as simlod_insert_batch would; simlod_sync then returns
 * SIMLOD_ERR_OUT_OF_BOUNDS once), a grouping of the valid batches, in order,
 * into updates of up to merge_points points, and one persistent launch that
 * applies the updates (a merged update is first gathered into the handle's
 * staging buffer). Merging consecutive batches leaves the octree unchanged:
 * after any prefix of the stream it does not depend on how the stream was cut
 * into batches (Section 5); gidx follows the order of the list. The plan
 * keeps the pointers: a caller refills the same buffers and runs the plan
 * again. simlod_plan_create allocates a small device table (about 80 bytes per
 * batch, cudaMalloc) that simlod_plan_destroy frees; it waits for the plan's
 * last run. One handle runs one plan or fused launch at a time (stream
 * order). */
typedef struct simlod_plan simlod_plan_t;
typedef struct {
  uint64_t merge_points;  /* merged update size; 0 = one update per batch; at most max_batch_points */
  uint32_t blocks_per_sm; /* persistent blocks per SM: 1 .. the kernel instance's maximum, 0 = all that fit */
  uint32_t use_graph;     /* capture the run in a CUDA graph */
  uint32_t variant;       /* kernel instance, 0 .. SIMLOD_N_VARIANTS - 1 (simlod_variant_info) */
} simlod_plan_params;
SIMLOD_API int simlod_plan_create(simlod_t* h, const simlod_point* const* d_batches,
                                  const uint64_t* counts, uint32_t n_batches,
                                  const simlod_plan_params* params, simlod_plan_t** out);
/* Enqueue one run of the plan on `stream` (asynchronous; errors at simlod_sync). */
SIMLOD_API int simlod_plan_run(simlod_plan_t* plan, void* stream);
/* The parameters in effect (merge_points clamped) and whether runs replay a graph. */
SIMLOD_API int simlod_plan_info(const simlod_plan_t* plan, simlod_plan_params* params,
                                uint32_t* graphed);
SIMLOD_API int simlod_plan_destroy(simlod_plan_t* plan);
/* Autotuner of the batched form (Section 4's persistent update kernel, with
 * its block and tile parameters chosen per workload): times plans for this
 * batch list on `h` itself (reset before every trial and at the end: pass a
 * scratch handle of the same configuration to keep an octree). First every
 * kernel instance (simlod_variant_info) at its largest and half its largest
 * blocks per SM, with updates merged up to max_batch_points; then, for the
 * fastest of those, every merge size (none, 256k, 1M, 2M, 4M, 8M points,
 * max_batch_points; those below max_batch_points). Returns the fastest
 * parameters and their time. The choice is kept per device, configuration
 * and batch list (counts): a later call with the same ones returns it at
 * once without timing anything (best_ms then holds the time measured when
 * it was chosen). */
SIMLOD_API int simlod_plan_autotune(simlod_t* h, const simlod_point* const* d_batches,
                                    const uint64_t* counts, uint32_t n_batches, void* stream,
                                    simlod_plan_params* best, double* best_ms);

/* Kernel instances of the batched form: the same persistent update kernel
 * compiled with other block and tile parameters. */
#define SIMLOD_N_VARIANTS 4
typedef struct {
  uint32_t threads_per_block;
  uint32_t max_blocks_per_sm;  /* that fit on the current device */
  uint32_t node_cache;         /* node-table entries mirrored in shared memory */
  uint32_t store_unroll;       /* records per thread in flight while storing */
  uint32_t descent_group;      /* tree levels whose occupancy words load together */
  uint32_t smem_bytes;         /* dynamic shared memory per block */
} simlod_variant_desc;
/* Parameters of kernel instance `variant` on the current device;
 * SIMLOD_ERR_INVALID_ARG for an unknown instance, SIMLOD_ERR_CUDA when the
 * device cannot run it. */
SIMLOD_API int simlod_variant_info(uint32_t variant, simlod_variant_desc* out);

/* Width of the handle's persistent launches (simlod_insert_batches,
 * simlod_frame_update): blocks_per_sm blocks of 512 threads per SM, from 1 to
 * *max_blocks_per_sm (what fits on an SM; 0 = that maximum, the default).
 * A persistent launch waits at its grid barriers for all of its blocks, so
 * launches of several handles that run at the same time must together fit
 * (for example two handles at 1 block per SM when 2 fit): launches that
 * together need more block slots than the GPU has can wait on each other
 * until their barriers time out (SIMLOD_ERR_TIMEOUT). */
SIMLOD_API int simlod_set_launch_width(simlod_t* h, uint32_t blocks_per_sm,
                                       uint32_t* max_blocks_per_sm);

/* Progress of the handle's persistent launches (simlod_insert_batches,
 * simlod_insert_batches_host, simlod_insert_batches_budget,
 * simlod_frame_update; not the batched form's plans, nor the plain form):
 * *finished = batches those launches have finished (applied or rejected)
 * since create; *submitted = batches handed to them, less the batches that a
 * budget stop dropped (both counted modulo 2^32). Batches finish in the order
 * they were handed over, so a launch that started with *finished = f0 has
 * finished its first k batches once *finished >= f0 + k; when a budget stop
 * ends it early, *finished - f0 after the launch is the number it applied.
 * The kernel writes both counts into page-locked host memory after each
 * batch, so the call only reads them: it neither waits nor synchronises, and
 * may be made while a launch runs (the serving form completes each request
 * when its own batch is finished). Not in the paper: its update kernel has
 * no caller that needs a request's completion before the whole frame's. */
SIMLOD_API int simlod_progress(simlod_t* h, uint64_t* finished, uint64_t* submitted);

/* Time limits of the waits inside the handle's persistent launches (not in
 * the paper, whose kernel waits without a limit): barrier_ns bounds one
 * block's wait at a grid barrier, ready_ns one wait for a batch's ready flag
 * (simlod_insert_batches_host); 0 restores the default of 2 s. A wait that
 * runs out aborts the launch: every block leaves at its next barrier,
 * simlod_sync returns SIMLOD_ERR_TIMEOUT, the handle is poisoned and
 * simlod_reset makes it usable again. The limits apply to launches enqueued
 * after the call (a plan keeps the limits it was created with). */
SIMLOD_API int simlod_set_wait_limits(simlod_t* h, uint64_t barrier_ns, uint64_t ready_ns);

/* Frame-budget update (Section 7.2): as simlod_insert_batches, but before
 * starting batch k > 0 the kernel checks the time since the launch began
 * (the GPU's global timer); once it exceeds budget_ns it stops. Batches are
 * never cut. Waits for the launch; *consumed receives the number of batches
 * handled, and the caller passes the rest in the next frame. */
SIMLOD_API int simlod_frame_update(simlod_t* h, const simlod_point* const* d_batches,
                                   const uint64_t* counts, uint32_t n_batches,
                                   uint64_t budget_ns, void* stream, uint32_t* consumed);

/* Frame-budget update without the wait: as simlod_frame_update (batch k > 0
 * starts only while the launch has run for at most budget_ns on the GPU's
 * global timer; batches are never cut), but asynchronous like
 * simlod_insert_batches. The batches after the stop are dropped: the caller
 * learns how many were applied from simlod_progress once `stream` has passed
 * the launch, and passes the rest again. d_batches[k] must stay valid until
 * then. Rejections and errors as in simlod_insert_batches. (The serving form
 * gives a launch the time left before the next frame is due, so that the
 * frame does not wait for the rest of a long launch.) */
SIMLOD_API int simlod_insert_batches_budget(simlod_t* h, const simlod_point* const* d_batches,
                                            const uint64_t* counts, uint32_t n_batches,
                                            uint64_t budget_ns, void* stream);

/* Empty the octree (one empty root leaf, gidx counter 0) without touching
 * the arena allocation; the handle's poison is cleared. Enqueued on `stream`
 * (it waits only when clearing a poisoned handle). */
SIMLOD_API int simlod_reset(simlod_t* h, void* stream);

/* Wait for the handle's last stream and report a device error, if any. */
SIMLOD_API int simlod_sync(simlod_t* h);

/* Counters since create/reset (synchronises). */
SIMLOD_API int simlod_get_stats(simlod_t* h, simlod_stats* out);

/* Canonical export (synchronises; doubles as a checkpoint). Nodes are sorted
 * by (level, ix, iy, iz) with ix = (min_x - root_min_x) >> log2size; each
 * leaf's points follow in node order sorted by gidx; each inner node's voxels
 * follow in node order sorted by cell. n_chunks is the length of the node's
 * chunk list, ceil(count / C) (Section 5.3). */
SIMLOD_API int simlod_snapshot(simlod_t* h, simlod_snapshot_t* snap);

/* Compaction of cold nodes (Section 8's direction of turning nodes that are
 * no longer modified into non-growable arrays): every node whose records
 * (points of a leaf, voxels of an inner node) fill two or more chunks and
 * that has received none in the last idle_updates updates gets them copied,
 * in order, into one contiguous array in the data region, and its chunks go
 * back to the pool. The octree does not change: snapshots (n_chunks still
 * reports ceil(count / C)), frames and later inserts are the same; an insert
 * that adds records to a compacted node first turns it back into a chunk list
 * (the array's space is not reused). Nodes the data region has no room for
 * stay as they are. Asynchronous on `stream`, ordered after the inserts
 * before it; simlod_get_stats reports the counts. */
SIMLOD_API int simlod_compact(simlod_t* h, uint32_t idle_updates, void* stream);

/* Section 6: draw the octree into a caller-owned device framebuffer of
 * width * height uint64_t entries (row-major, 8-byte aligned), each
 * (float bits of depth) << 32 | rgba; all ones = empty. clear != 0 fills it
 * with all ones first, else the octree is drawn over what is there (so
 * several octrees can share a frame). Node selection: a node is drawn when
 * its cube is in the view frustum, it is a leaf or at most 2^grid_log2
 * pixels on screen, and its parent is larger than that (or it is the root);
 * a drawn leaf splats its points, a drawn inner node its voxels, one pixel
 * each; a pixel keeps the smallest word (the closest sample).
 * view_proj: row-major 4x4, clip = M (x, y, z, 1) with the integer
 * coordinates as float; depth = clip w; a sample is drawn when w > 0 and
 * s = (clip.xy / w * 0.5 + 0.5) * (width, height) lies in [0,width)x[0,height)
 * (pixel floor(s)). A cube is culled when its 8 corners are all outside one
 * of x < -w, x > w, y < -w, y > w, w <= 0; its size on screen is the larger
 * side of its corners' screen box (infinite with a corner at w <= 0). Float
 * operations are single-precision IEEE, one per operator in that order, so
 * the frame is reproducible bit for bit. Asynchronous on `stream`, ordered
 * after the inserts enqueued before it on that stream; the octree is not
 * changed. simlod_get_stats reports the nodes drawn and samples visited. */
SIMLOD_API int simlod_render(simlod_t* h, const float view_proj[16], uint32_t width,
                             uint32_t height, uint64_t* d_framebuffer, int clear, void* stream);

/* Restore a canonical snapshot (as simlod_snapshot writes it, or the same
 * layout from elsewhere) into h, replacing its octree: nodes, their chunk
 * lists (a leaf's points keep their gidx, an inner node's voxels their cell
 * and colour), occupancy grids from the voxel cells, and the gidx counter at
 * the number of points, so that later inserts continue the stream exactly as
 * on the octree the snapshot was taken from. The configuration of h must be
 * the snapshot's (root cube, T, C, G); a snapshot that does not form one
 * octree of it (unsorted or missing nodes, wrong chunk counts, cells off the
 * grid) is rejected with SIMLOD_ERR_INVALID_ARG and h is unchanged;
 * SIMLOD_ERR_NODES_FULL / SIMLOD_ERR_ARENA_FULL when it does not fit. The
 * octree is rebuilt on the host and copied in; the call waits for `stream`
 * and returns when the copies are done. Statistics restart (points and
 * voxels are set to the snapshot's). */
SIMLOD_API int simlod_restore(simlod_t* h, const simlod_snapshot_t* snap, void* stream);

/* Record CUDA events around every kernel launch (on the launching stream)
 * and accumulate per-kernel device time; enable = 0 stops, clear resets. */
SIMLOD_API int simlod_set_timing(simlod_t* h, int enable, int clear);
SIMLOD_API int simlod_get_timing(simlod_t* h, simlod_timing* out);

/* Largest batch simlod_sample_node_noalloc accepts. */
#define SIMLOD_NOALLOC_MAX_POINTS 131072u

/* Voxel sampling of one node with no device allocation at all. The paper has
 * no counterpart: it exists for callers that cannot allocate device memory
 * when they need the step, such as a running real-time frame loop (cudaMalloc
 * and cudaFree can synchronise the device and stall a frame) or code inside
 * another framework that owns every device buffer and passes in only inputs
 * and outputs. It needs no handle and no arena.
 *
 * Computes the voxels that the points d_pts[0..n) create in the 2^grid_log2
 * grid inscribed in the cube [node_min, node_min + 2^log2size) per axis, the
 * same way an update samples an inner node: one voxel per occupied cell, at
 * the floor of the cell centre, coloured by the point with the lowest index.
 * Points outside the cube are ignored. Writes the voxels, in no particular
 * order, to d_voxels and their number to *d_count (both device memory owned
 * by the caller; voxels_capacity >= min(n, 2^(3 grid_log2))). The work is
 * enqueued on `stream`; nothing is waited for.
 *
 * Scratch lives in one fixed array of about 4.5 MiB per device, a file-scope
 * device variable that every GPU loading this library holds until the
 * process exits; hence n is limited to SIMLOD_NOALLOC_MAX_POINTS and larger
 * batches are rejected with SIMLOD_ERR_INVALID_ARG. Every call looks up that
 * array's device address in the current context (a host-side query; the
 * first call in a context also loads the library's device code, so make that
 * first call before any stream capture). Every call clears and reuses the
 * same array, so calls whose work overlaps on the GPU (different streams,
 * other threads) race and must be serialised by the caller. Calls no
 * cudaMalloc, cudaFree or allocating library routine. An error already
 * pending in the CUDA runtime from earlier work is reported as
 * SIMLOD_ERR_CUDA and left in place for the caller to read. */
SIMLOD_API int simlod_sample_node_noalloc(const simlod_point* d_pts, uint64_t n,
                                          const int32_t node_min[3], uint32_t log2size,
                                          uint32_t grid_log2, simlod_voxel_rec* d_voxels,
                                          uint64_t voxels_capacity, uint32_t* d_count,
                                          void* stream);

/* Release host-side state. The arena is the caller's and is not touched. */
SIMLOD_API int simlod_destroy(simlod_t* h);

/* Static text for a status code. */
SIMLOD_API const char* simlod_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif
