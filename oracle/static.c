/*
 * Static oracle: the octree the incremental update reaches after a prefix
 * P_k of the stream, computed directly from its definition instead of batch
 * by batch.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h). Written independently of
 * incremental.c: no shared helpers.
 *
 * Definition (from the splitting rule of Section 5.1 and the sampling rule of
 * Section 5.2; counts only grow and nodes never merge, so a node that ever
 * exceeded T is exactly a node that exceeds T now):
 *  - the root is inner iff it holds more than T points of P_k;
 *  - an inner node has all 8 children; a child is inner iff it holds more
 *    than T points of P_k and its side is above one unit, otherwise a leaf;
 *  - a leaf holds exactly the points of P_k inside its cube;
 *  - an inner node has one voxel per occupied cell of its 2^G^3 grid, coloured
 *    by the point of lowest arrival index in that cell;
 *  - a node's chunk count is ceil(count / C) (Section 5.3).
 */
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

typedef struct {
  orc_node info;
  uint64_t first; /* first point (leaf) or voxel (inner) in the output arrays */
} built_node;

struct orc_static {
  orc_config cfg;
  built_node* nodes;
  uint64_t n_nodes, cap_nodes;
  orc_point_rec* points;
  uint64_t n_points, cap_points;
  orc_voxel_rec* voxels;
  uint64_t n_voxels, cap_voxels;
};

typedef struct {
  const orc_point* pts;
  uint32_t* scratch; /* partition buffer, same length as the index array */
  uint8_t* seen;     /* one byte per cell of a grid */
  uint64_t grid_cells;
} build_ctx;

static uint32_t rgba_of(const orc_point* p) {
  return (uint32_t)p->r | ((uint32_t)p->g << 8) | ((uint32_t)p->b << 16) | ((uint32_t)p->a << 24);
}

static int grow(void** buf, uint64_t* cap, uint64_t need, size_t elem) {
  if (need <= *cap) return 0;
  uint64_t c = *cap ? *cap : 256;
  while (c < need) c *= 2;
  void* nb = realloc(*buf, c * elem);
  if (!nb) return -1;
  *buf = nb;
  *cap = c;
  return 0;
}

/* idx[0..n) are the arrival indices of the points inside the cube
 * [mn, mn + 2^L)^3, in ascending order. */
static int build_node(orc_static* t, build_ctx* bc, const int32_t mn[3], uint32_t L,
                      uint32_t level, uint32_t* idx, uint64_t n) {
  const uint32_t G = t->cfg.grid_log2;
  const uint64_t C = t->cfg.chunk_points;
  if (grow((void**)&t->nodes, &t->cap_nodes, t->n_nodes + 1, sizeof(built_node))) return -1;
  uint64_t me = t->n_nodes++;
  orc_node* info = &t->nodes[me].info;
  memset(info, 0, sizeof(*info));
  info->level = level;
  info->min[0] = mn[0];
  info->min[1] = mn[1];
  info->min[2] = mn[2];
  info->log2size = L;

  if (!(n > t->cfg.leaf_capacity && L > 0)) {
    /* leaf: exactly its points, in arrival order */
    if (grow((void**)&t->points, &t->cap_points, t->n_points + n, sizeof(orc_point_rec)))
      return -1;
    t->nodes[me].first = t->n_points;
    for (uint64_t k = 0; k < n; ++k) {
      const orc_point* p = &bc->pts[idx[k]];
      orc_point_rec* r = &t->points[t->n_points + k];
      r->x = p->x;
      r->y = p->y;
      r->z = p->z;
      r->rgba = rgba_of(p);
      r->gidx = idx[k];
    }
    t->n_points += n;
    info->is_inner = 0;
    info->n_points = n;
    info->n_chunks = (n + C - 1) / C;
    return 0;
  }

  /* inner: one voxel per occupied cell, first point (lowest index) wins */
  info->is_inner = 1;
  uint64_t first_voxel = t->n_voxels;
  for (uint64_t k = 0; k < n; ++k) {
    const orc_point* p = &bc->pts[idx[k]];
    const int64_t off[3] = {(int64_t)p->x - mn[0], (int64_t)p->y - mn[1], (int64_t)p->z - mn[2]};
    uint64_t cx = ((uint64_t)off[0] << G) >> L;
    uint64_t cy = ((uint64_t)off[1] << G) >> L;
    uint64_t cz = ((uint64_t)off[2] << G) >> L;
    uint64_t cell = cx + (cy << G) + (cz << (2 * G));
    if (bc->seen[cell]) continue;
    bc->seen[cell] = 1;
    if (grow((void**)&t->voxels, &t->cap_voxels, t->n_voxels + 1, sizeof(orc_voxel_rec)))
      return -1;
    orc_voxel_rec* v = &t->voxels[t->n_voxels++];
    v->cell = (uint32_t)cell;
    /* floor of the cell centre: mn + (c + 1/2) * 2^L / 2^G */
    v->x = mn[0] + (int32_t)(((2 * cx + 1) << L) >> (G + 1));
    v->y = mn[1] + (int32_t)(((2 * cy + 1) << L) >> (G + 1));
    v->z = mn[2] + (int32_t)(((2 * cz + 1) << L) >> (G + 1));
    v->rgba = rgba_of(p);
  }
  uint64_t nv = t->n_voxels - first_voxel;
  for (uint64_t k = first_voxel; k < t->n_voxels; ++k) bc->seen[t->voxels[k].cell] = 0;
  info = &t->nodes[me].info;
  info->n_voxels = nv;
  info->n_chunks = (nv + C - 1) / C;
  t->nodes[me].first = first_voxel;

  /* stable partition of idx into the 8 octants, keeping arrival order */
  uint64_t cnt[8] = {0}, start[8];
  const int64_t half = (int64_t)1 << (L - 1);
  for (uint64_t k = 0; k < n; ++k) {
    const orc_point* p = &bc->pts[idx[k]];
    int o = (((int64_t)p->x - mn[0]) >= half) | ((((int64_t)p->y - mn[1]) >= half) << 1) |
            ((((int64_t)p->z - mn[2]) >= half) << 2);
    cnt[o]++;
  }
  start[0] = 0;
  for (int o = 1; o < 8; ++o) start[o] = start[o - 1] + cnt[o - 1];
  uint64_t pos[8];
  memcpy(pos, start, sizeof(pos));
  for (uint64_t k = 0; k < n; ++k) {
    const orc_point* p = &bc->pts[idx[k]];
    int o = (((int64_t)p->x - mn[0]) >= half) | ((((int64_t)p->y - mn[1]) >= half) << 1) |
            ((((int64_t)p->z - mn[2]) >= half) << 2);
    bc->scratch[pos[o]++] = idx[k];
  }
  memcpy(idx, bc->scratch, n * sizeof(uint32_t));
  for (int o = 0; o < 8; ++o) {
    int32_t cm[3] = {(int32_t)(mn[0] + ((o & 1) ? half : 0)), (int32_t)(mn[1] + ((o & 2) ? half : 0)),
                     (int32_t)(mn[2] + ((o & 4) ? half : 0))};
    if (build_node(t, bc, cm, L - 1, level + 1, idx + start[o], cnt[o])) return -1;
  }
  return 0;
}

int orc_static_build(const orc_config* cfg, const orc_point* pts, uint64_t n, orc_static** out) {
  if (!cfg || !out || cfg->root_log2 > 31 || cfg->leaf_capacity == 0 ||
      cfg->chunk_points == 0 || cfg->grid_log2 == 0 || cfg->grid_log2 > 10 || (n && !pts))
    return ORC_ERR_INVALID;
  if (n > ((uint64_t)1 << 32)) return ORC_ERR_TOO_MANY_POINTS;
  const int64_t side = (int64_t)1 << cfg->root_log2;
  for (uint64_t k = 0; k < n; ++k) {
    int64_t d[3] = {(int64_t)pts[k].x - cfg->root_min[0], (int64_t)pts[k].y - cfg->root_min[1],
                    (int64_t)pts[k].z - cfg->root_min[2]};
    for (int a = 0; a < 3; ++a)
      if (d[a] < 0 || d[a] >= side) return ORC_ERR_OUT_OF_BOUNDS;
  }
  orc_static* t = (orc_static*)calloc(1, sizeof(orc_static));
  if (!t) return ORC_ERR_NOMEM;
  t->cfg = *cfg;
  build_ctx bc;
  bc.pts = pts;
  bc.grid_cells = (uint64_t)1 << (3 * cfg->grid_log2);
  bc.seen = (uint8_t*)calloc(bc.grid_cells, 1);
  uint32_t* idx = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  bc.scratch = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
  int rc = ORC_ERR_NOMEM;
  if (bc.seen && idx && bc.scratch) {
    for (uint64_t k = 0; k < n; ++k) idx[k] = (uint32_t)k;
    rc = build_node(t, &bc, cfg->root_min, cfg->root_log2, 0, idx, n) ? ORC_ERR_NOMEM : ORC_OK;
  }
  free(bc.seen);
  free(idx);
  free(bc.scratch);
  if (rc) {
    orc_static_destroy(t);
    return rc;
  }
  *out = t;
  return ORC_OK;
}

void orc_static_sizes(const orc_static* t, orc_sizes* s) {
  s->n_nodes = t->n_nodes;
  s->n_points = t->n_points;
  s->n_voxels = t->n_voxels;
}

static const orc_static* g_sort_tree; /* qsort has no context argument in C11 */

static int cmp_built(const void* pa, const void* pb) {
  const orc_node* a = &g_sort_tree->nodes[*(const uint64_t*)pa].info;
  const orc_node* b = &g_sort_tree->nodes[*(const uint64_t*)pb].info;
  if (a->level != b->level) return a->level < b->level ? -1 : 1;
  const int32_t* rm = g_sort_tree->cfg.root_min;
  for (int ax = 0; ax < 3; ++ax) {
    uint64_t ia = (uint64_t)((int64_t)a->min[ax] - rm[ax]) >> a->log2size;
    uint64_t ib = (uint64_t)((int64_t)b->min[ax] - rm[ax]) >> b->log2size;
    if (ia != ib) return ia < ib ? -1 : 1;
  }
  return 0;
}

static int cmp_cell(const void* pa, const void* pb) {
  uint32_t a = ((const orc_voxel_rec*)pa)->cell, b = ((const orc_voxel_rec*)pb)->cell;
  return a < b ? -1 : (a > b ? 1 : 0);
}

int orc_static_export(const orc_static* t, orc_node* nodes, orc_point_rec* points,
                      orc_voxel_rec* voxels) {
  uint64_t* order = (uint64_t*)malloc(sizeof(uint64_t) * (t->n_nodes ? t->n_nodes : 1));
  if (!order) return ORC_ERR_NOMEM;
  for (uint64_t k = 0; k < t->n_nodes; ++k) order[k] = k;
  g_sort_tree = t;
  qsort(order, t->n_nodes, sizeof(uint64_t), cmp_built);
  g_sort_tree = NULL;
  uint64_t pp = 0, vv = 0;
  for (uint64_t k = 0; k < t->n_nodes; ++k) {
    const built_node* b = &t->nodes[order[k]];
    nodes[k] = b->info;
    if (b->info.is_inner) {
      memcpy(voxels + vv, t->voxels + b->first, b->info.n_voxels * sizeof(orc_voxel_rec));
      qsort(voxels + vv, b->info.n_voxels, sizeof(orc_voxel_rec), cmp_cell);
      vv += b->info.n_voxels;
    } else {
      /* already in arrival order */
      memcpy(points + pp, t->points + b->first, b->info.n_points * sizeof(orc_point_rec));
      pp += b->info.n_points;
    }
  }
  free(order);
  return ORC_OK;
}

void orc_static_destroy(orc_static* t) {
  if (!t) return;
  free(t->nodes);
  free(t->points);
  free(t->voxels);
  free(t);
}
