/*
 * CPU oracle for the incremental octree LOD update of SimLOD (Schuetz,
 * Herzberger, Wimmer: "SimLOD: Simultaneous LOD Generation and Rendering").
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may include, link or
 * call this code: the tests, the smoke check and the benchmark's CPU-baseline
 * leg are its only users. It shares no code with the CUDA library.
 *
 * Two independent implementations of the update live here (and render.c,
 * the renderer of Section 6, for the frame-budget tests):
 *
 *  - incremental.c: a plain, sequential rendering of the paper's per-batch
 *    update (Section 5): expansion by repeated counting and splitting
 *    (Section 5.1), voxel sampling in arrival order (Section 5.2), chunk
 *    allocation from a pool and a bump allocator (Sections 3.2, 3.4, 5.3),
 *    and storing points and voxels through per-node counters (Section 5.4).
 *  - static.c: the closed form of the octree that the incremental update
 *    reaches after any prefix of the stream, built top-down in one go.
 *
 * Both export the same canonical form: nodes sorted by (level, ix, iy, iz),
 * each leaf's points sorted by global arrival index, each inner node's voxels
 * sorted by cell index.
 *
 * Readings of the paper (where it is silent or loose):
 *  - A leaf splits when its count exceeds the capacity T (Section 5.1) and its
 *    cube side is above one unit; a one-unit leaf keeps all its points.
 *  - The leaf counter of an update starts at the points already stored.
 *  - The "first point" that gives a voxel its colour (Section 5.2) is the one
 *    with the lowest global arrival index; every point continues down to its
 *    leaf after sampling an inner node.
 *  - Cell of p in a node with minimum m and side 2^L on a 2^G grid, per axis:
 *    c = ((p - m) << G) >> L; flattened cx + 2^G (cy + 2^G cz). The voxel sits
 *    at the floor of the cell centre, m + (((2c + 1) << L) >> (G + 1)).
 *  - Child octant = bx | by << 1 | bz << 2 with b = bit L-1 of (p - m).
 *  - The root cube [root_min, root_min + 2^root_log2) is given; a batch with a
 *    point outside it is rejected whole, before anything changes.
 */
#ifndef SIMLOD_ORACLE_H
#define SIMLOD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t x, y, z;
  uint8_t r, g, b, a;
} orc_point;

typedef struct {
  int32_t root_min[3];
  uint32_t root_log2;        /* root cube side 2^root_log2, <= 31 */
  uint32_t leaf_capacity;    /* T: 50,000 in the paper (Section 3.1) */
  uint32_t chunk_points;     /* points or voxels per chunk: 1,000 (Section 3.4) */
  uint32_t grid_log2;        /* sampling grid 2^G per axis: 128 = 2^7 (Section 3.3) */
  uint32_t max_expand_iters; /* 0: no cap */
} orc_config;

/* Canonical node record. */
typedef struct {
  uint32_t level, is_inner;
  int32_t min[3];
  uint32_t log2size;
  uint64_t n_points, n_voxels, n_chunks;
} orc_node;

/* A leaf's point with its global arrival index. rgba = r | g<<8 | b<<16 | a<<24. */
typedef struct {
  int32_t x, y, z;
  uint32_t rgba;
  uint32_t gidx;
} orc_point_rec;

/* An inner node's voxel: its cell index, its position and its colour. */
typedef struct {
  uint32_t cell;
  int32_t x, y, z;
  uint32_t rgba;
} orc_voxel_rec;

typedef struct {
  uint64_t n_nodes, n_points, n_voxels;
} orc_sizes;

typedef struct {
  uint64_t batches, points, spilled, splits, voxels, iterations_max;
  uint64_t chunks_live, chunks_pool, chunks_bumped;
  uint64_t spill_voxels_at_old_inner; /* voxels made by re-inserted points at nodes
                                         that were already inner: always 0 */
} orc_stats;

enum {
  ORC_OK = 0,
  ORC_ERR_INVALID = -1,
  ORC_ERR_OUT_OF_BOUNDS = -2,
  ORC_ERR_NOMEM = -3,
  ORC_ERR_ITER_CAP = -6,
  ORC_ERR_TOO_MANY_POINTS = -11
};

typedef struct orc_inc orc_inc;
int orc_inc_create(const orc_config* cfg, orc_inc** out);
int orc_inc_insert(orc_inc* o, const orc_point* pts, uint64_t n);
void orc_inc_sizes(const orc_inc* o, orc_sizes* s);
int orc_inc_export(const orc_inc* o, orc_node* nodes, orc_point_rec* points,
                   orc_voxel_rec* voxels);
void orc_inc_stats(const orc_inc* o, orc_stats* s);
void orc_inc_destroy(orc_inc* o);

typedef struct orc_static orc_static;
int orc_static_build(const orc_config* cfg, const orc_point* pts, uint64_t n, orc_static** out);
void orc_static_sizes(const orc_static* t, orc_sizes* s);
int orc_static_export(const orc_static* t, orc_node* nodes, orc_point_rec* points,
                      orc_voxel_rec* voxels);
void orc_static_destroy(orc_static* t);

/* render.c: Section 6, the level-of-detail selection and pixel-sized splats
   of a canonical octree (see render.c for the readings). framebuffer holds
   width * height entries ((float bits of depth) << 32 | rgba, all ones =
   empty), drawn one flag per node. */
int orc_render(const orc_config* cfg, const orc_node* nodes, uint64_t n_nodes,
               const orc_point_rec* points, const orc_voxel_rec* voxels, const float view_proj[16],
               uint32_t width, uint32_t height, uint64_t* framebuffer, uint8_t* drawn,
               uint64_t* n_drawn);

#ifdef __cplusplus
}
#endif
#endif
