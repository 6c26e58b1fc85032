/*
 * Incremental oracle: the per-batch octree update of SimLOD, run
 * sequentially on the CPU, one step after the other in the order the paper
 * gives them (Section 5, Figure "kernel_update").
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h). Slow and plain on purpose.
 */
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define NO_CHILD 0xFFFFFFFFu

/* Section 3.4: a chunk stores up to C records and links to the next chunk. */
typedef struct chunk {
  struct chunk* next;
  orc_point_rec* items; /* C slots; for voxels the gidx field holds the cell */
} chunk;

/* Section 3.1: an octree node. Leaves hold points, inner nodes voxels. */
typedef struct {
  int32_t min[3];
  uint32_t log2size, level;
  int is_leaf;
  uint32_t child0; /* the 8 children are child0 .. child0+7 */
  /* Section 5.1: per-update point counter and "final" mark */
  uint64_t counter;
  int final;
  /* Section 5.4: numPoints / numVoxels */
  uint64_t num_points, num_voxels;
  uint64_t vox_counter; /* voxels created during the current update */
  /* linked list of chunks; `index` mirrors the list for O(1) access */
  chunk* head;
  chunk* tail;
  uint64_t n_chunks, index_cap;
  chunk** index;
  uint8_t* grid; /* Section 3.3: one bit per cell of the 2^G^3 grid */
} node;

typedef struct {
  orc_point p;
  uint32_t gidx;
} item;

typedef struct {
  uint32_t node, cell;
  orc_point voxel;
} backlog_entry;

struct orc_inc {
  orc_config cfg;
  node* nodes;
  uint64_t n_nodes, cap_nodes;
  /* Section 3.4: chunk pool, a stack of freed chunks */
  chunk** pool;
  uint64_t n_pool, cap_pool;
  uint64_t chunks_bumped; /* chunks taken from the persistent buffer */
  uint64_t base;          /* points inserted so far: next global index */
  orc_stats stats;
};

/* --------------------------------------------------------------- helpers */

static int push_node(orc_inc* o, const node* nd) {
  if (o->n_nodes == o->cap_nodes) {
    uint64_t cap = o->cap_nodes ? o->cap_nodes * 2 : 64;
    node* nn = (node*)realloc(o->nodes, cap * sizeof(node));
    if (!nn) return ORC_ERR_NOMEM;
    o->nodes = nn;
    o->cap_nodes = cap;
  }
  o->nodes[o->n_nodes++] = *nd;
  return ORC_OK;
}

static void init_node(node* nd, const int32_t min[3], uint32_t log2size, uint32_t level) {
  memset(nd, 0, sizeof(*nd));
  nd->min[0] = min[0];
  nd->min[1] = min[1];
  nd->min[2] = min[2];
  nd->log2size = log2size;
  nd->level = level;
  nd->is_leaf = 1;
  nd->child0 = NO_CHILD;
}

static int inside_root(const orc_config* c, const orc_point* p) {
  int64_t side = (int64_t)1 << c->root_log2;
  int64_t d[3] = {(int64_t)p->x - c->root_min[0], (int64_t)p->y - c->root_min[1],
                  (int64_t)p->z - c->root_min[2]};
  for (int a = 0; a < 3; ++a)
    if (d[a] < 0 || d[a] >= side) return 0;
  return 1;
}

/* Octant of p inside an inner node: bit (L-1) of (p - min) per axis. */
static uint32_t octant(const node* nd, const orc_point* p) {
  uint32_t h = nd->log2size - 1;
  uint32_t bx = (uint32_t)((((int64_t)p->x - nd->min[0]) >> h) & 1);
  uint32_t by = (uint32_t)((((int64_t)p->y - nd->min[1]) >> h) & 1);
  uint32_t bz = (uint32_t)((((int64_t)p->z - nd->min[2]) >> h) & 1);
  return bx | (by << 1) | (bz << 2);
}

/* Walk from the root to the leaf whose cube contains p. */
static uint32_t descend(const orc_inc* o, const orc_point* p) {
  uint32_t id = 0;
  while (!o->nodes[id].is_leaf) id = o->nodes[id].child0 + octant(&o->nodes[id], p);
  return id;
}

/* Section 3.3: cell of p in the grid inscribed into node nd. */
static uint32_t cell_of(const orc_inc* o, const node* nd, const orc_point* p, uint32_t c[3]) {
  uint32_t G = o->cfg.grid_log2;
  int64_t d[3] = {(int64_t)p->x - nd->min[0], (int64_t)p->y - nd->min[1],
                  (int64_t)p->z - nd->min[2]};
  for (int a = 0; a < 3; ++a) c[a] = (uint32_t)(((uint64_t)d[a] << G) >> nd->log2size);
  return c[0] + (c[1] << G) + (c[2] << (2 * G));
}

/* Section 3.4: the voxel is stored as a point at the cell centre. */
static orc_point voxel_point(const orc_inc* o, const node* nd, const uint32_t c[3],
                             const orc_point* colour) {
  uint32_t G = o->cfg.grid_log2;
  orc_point v = *colour;
  int32_t xyz[3];
  for (int a = 0; a < 3; ++a)
    xyz[a] = nd->min[a] + (int32_t)((((uint64_t)(2 * c[a] + 1)) << nd->log2size) >> (G + 1));
  v.x = xyz[0];
  v.y = xyz[1];
  v.z = xyz[2];
  return v;
}

static uint32_t pack_rgba(const orc_point* p) {
  return (uint32_t)p->r | ((uint32_t)p->g << 8) | ((uint32_t)p->b << 16) | ((uint32_t)p->a << 24);
}

static uint64_t grid_bytes(const orc_config* c) {
  uint64_t bits = (uint64_t)1 << (3 * c->grid_log2);
  return bits >= 8 ? bits / 8 : 1;
}

static int test_bit(const uint8_t* g, uint32_t cell) { return (g[cell >> 3] >> (cell & 7)) & 1; }
static void set_bit(uint8_t* g, uint32_t cell) { g[cell >> 3] |= (uint8_t)(1u << (cell & 7)); }

/* Section 3.4: acquire a chunk from the pool, else from the persistent buffer. */
static chunk* acquire_chunk(orc_inc* o) {
  if (o->n_pool > 0) return o->pool[--o->n_pool];
  chunk* ch = (chunk*)malloc(sizeof(chunk));
  if (!ch) return NULL;
  ch->items = (orc_point_rec*)malloc(sizeof(orc_point_rec) * o->cfg.chunk_points);
  if (!ch->items) {
    free(ch);
    return NULL;
  }
  ch->next = NULL;
  o->chunks_bumped++;
  return ch;
}

static int release_chunk(orc_inc* o, chunk* ch) {
  if (o->n_pool == o->cap_pool) {
    uint64_t cap = o->cap_pool ? o->cap_pool * 2 : 64;
    chunk** np = (chunk**)realloc(o->pool, cap * sizeof(chunk*));
    if (!np) return ORC_ERR_NOMEM;
    o->pool = np;
    o->cap_pool = cap;
  }
  ch->next = NULL;
  o->pool[o->n_pool++] = ch;
  return ORC_OK;
}

/* Link one more chunk at the end of a node's list. */
static int append_chunk(orc_inc* o, uint32_t id) {
  chunk* ch = acquire_chunk(o);
  if (!ch) return ORC_ERR_NOMEM;
  node* nd = &o->nodes[id];
  if (nd->n_chunks == nd->index_cap) {
    uint64_t cap = nd->index_cap ? nd->index_cap * 2 : 4;
    chunk** ni = (chunk**)realloc(nd->index, cap * sizeof(chunk*));
    if (!ni) return ORC_ERR_NOMEM;
    nd->index = ni;
    nd->index_cap = cap;
  }
  ch->next = NULL;
  if (nd->tail) nd->tail->next = ch;
  else nd->head = ch;
  nd->tail = ch;
  nd->index[nd->n_chunks++] = ch;
  return ORC_OK;
}

/* Section 5.4: slot idx of a node lives in chunk idx / C at position idx % C. */
static orc_point_rec* slot(const orc_inc* o, const node* nd, uint64_t idx) {
  uint64_t C = o->cfg.chunk_points;
  return &nd->index[idx / C]->items[idx % C];
}

typedef struct {
  item* v;
  uint64_t n, cap;
} item_vec;

static int item_push(item_vec* s, const orc_point* p, uint32_t gidx) {
  if (s->n == s->cap) {
    uint64_t cap = s->cap ? s->cap * 2 : 1024;
    item* nv = (item*)realloc(s->v, cap * sizeof(item));
    if (!nv) return ORC_ERR_NOMEM;
    s->v = nv;
    s->cap = cap;
  }
  s->v[s->n].p = *p;
  s->v[s->n].gidx = gidx;
  s->n++;
  return ORC_OK;
}

/* Section 5.1, "Splitting": make 8 children with counter 0, move the node's
 * points to the spill buffer, return its chunks to the pool. The node becomes
 * an inner node and gets a zeroed sampling grid (Section 3.3). */
static int split_leaf(orc_inc* o, uint32_t id, item_vec* spill) {
  node* nd = &o->nodes[id];
  uint32_t half_log2 = nd->log2size - 1;
  int64_t half = (int64_t)1 << half_log2;
  int32_t pmin[3] = {nd->min[0], nd->min[1], nd->min[2]};
  uint32_t level = nd->level;
  uint32_t first = (uint32_t)o->n_nodes;
  for (uint32_t k = 0; k < 8; ++k) {
    int32_t cmin[3] = {(int32_t)(pmin[0] + ((k & 1) ? half : 0)),
                       (int32_t)(pmin[1] + ((k & 2) ? half : 0)),
                       (int32_t)(pmin[2] + ((k & 4) ? half : 0))};
    node child;
    init_node(&child, cmin, half_log2, level + 1);
    int rc = push_node(o, &child);
    if (rc) return rc;
  }
  nd = &o->nodes[id]; /* the node array may have moved */
  for (uint64_t i = 0; i < nd->num_points; ++i) {
    orc_point_rec* r = slot(o, nd, i);
    orc_point p = {r->x, r->y, r->z, (uint8_t)r->rgba, (uint8_t)(r->rgba >> 8),
                   (uint8_t)(r->rgba >> 16), (uint8_t)(r->rgba >> 24)};
    int rc = item_push(spill, &p, r->gidx);
    if (rc) return rc;
  }
  for (chunk* ch = nd->head; ch;) {
    chunk* nx = ch->next;
    int rc = release_chunk(o, ch);
    if (rc) return rc;
    ch = nx;
  }
  nd->head = nd->tail = NULL;
  nd->n_chunks = 0;
  nd->num_points = 0;
  nd->counter = 0;
  nd->is_leaf = 0;
  nd->child0 = first;
  nd->grid = (uint8_t*)calloc(grid_bytes(&o->cfg), 1);
  if (!nd->grid) return ORC_ERR_NOMEM;
  o->stats.splits++;
  return ORC_OK;
}

static int cmp_item_gidx(const void* a, const void* b) {
  uint32_t x = ((const item*)a)->gidx, y = ((const item*)b)->gidx;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* --------------------------------------------------------------- public */

int orc_inc_create(const orc_config* cfg, orc_inc** out) {
  if (!cfg || !out || cfg->root_log2 > 31 || cfg->leaf_capacity == 0 ||
      cfg->chunk_points == 0 || cfg->grid_log2 == 0 || cfg->grid_log2 > 10)
    return ORC_ERR_INVALID;
  orc_inc* o = (orc_inc*)calloc(1, sizeof(orc_inc));
  if (!o) return ORC_ERR_NOMEM;
  o->cfg = *cfg;
  node root;
  init_node(&root, cfg->root_min, cfg->root_log2, 0);
  if (push_node(o, &root)) {
    free(o);
    return ORC_ERR_NOMEM;
  }
  *out = o;
  return ORC_OK;
}

int orc_inc_insert(orc_inc* o, const orc_point* pts, uint64_t n) {
  if (!o) return ORC_ERR_INVALID;
  if (n == 0) return ORC_OK;
  if (!pts) return ORC_ERR_INVALID;
  for (uint64_t i = 0; i < n; ++i)
    if (!inside_root(&o->cfg, &pts[i])) return ORC_ERR_OUT_OF_BOUNDS;
  if (o->base + n > ((uint64_t)1 << 32)) return ORC_ERR_TOO_MANY_POINTS;

  const uint64_t T = o->cfg.leaf_capacity, C = o->cfg.chunk_points;
  const uint64_t n_nodes_at_start = o->n_nodes;
  int rc = ORC_OK;
  item_vec spill = {0};
  backlog_entry* backlog = NULL;
  uint64_t n_backlog = 0, cap_backlog = 0;
  char* was_inner = NULL;

  /* Which nodes were inner before this update (for the spill check). */
  was_inner = (char*)malloc(n_nodes_at_start ? n_nodes_at_start : 1);
  if (!was_inner) return ORC_ERR_NOMEM;
  for (uint64_t id = 0; id < n_nodes_at_start; ++id) was_inner[id] = !o->nodes[id].is_leaf;

  /* ---- Section 5.1: expand by counting and splitting until all leaves are final. */
  for (uint64_t id = 0; id < o->n_nodes; ++id) {
    node* nd = &o->nodes[id];
    if (nd->is_leaf) {
      nd->counter = nd->num_points;
      nd->final = 0;
    }
    nd->vox_counter = 0;
  }
  uint64_t iter = 0;
  for (;;) {
    if (o->cfg.max_expand_iters && iter >= o->cfg.max_expand_iters) {
      rc = ORC_ERR_ITER_CAP;
      goto done;
    }
    ++iter;
    /* Counting: every point of the batch and of the spill buffer. */
    for (uint64_t i = 0; i < n; ++i) {
      node* leaf = &o->nodes[descend(o, &pts[i])];
      if (!leaf->final) leaf->counter++;
    }
    for (uint64_t s = 0; s < spill.n; ++s) {
      node* leaf = &o->nodes[descend(o, &spill.v[s].p)];
      if (!leaf->final) leaf->counter++;
    }
    /* Splitting: leaves over the threshold split, the others become final.
     * Children made in this round are left for the next count. */
    int any_split = 0;
    uint64_t n_before = o->n_nodes;
    for (uint64_t id = 0; id < n_before; ++id) {
      node* nd = &o->nodes[id];
      if (!nd->is_leaf || nd->final) continue;
      if (nd->counter > T && nd->log2size > 0) {
        rc = split_leaf(o, (uint32_t)id, &spill);
        if (rc) goto done;
        any_split = 1;
      } else {
        nd->final = 1;
      }
    }
    if (!any_split) break;
  }
  if (iter > o->stats.iterations_max) o->stats.iterations_max = iter;

  /* ---- Section 5.2: voxel sampling. Points go through the tree in arrival
   * order (spilled points are older than the batch), so the first point to
   * reach an empty cell is the one with the lowest global index. */
  qsort(spill.v, spill.n, sizeof(item), cmp_item_gidx);
  for (uint64_t k = 0; k < spill.n + n; ++k) {
    int from_spill = k < spill.n;
    const orc_point* p = from_spill ? &spill.v[k].p : &pts[k - spill.n];
    uint32_t id = 0;
    while (!o->nodes[id].is_leaf) {
      node* nd = &o->nodes[id];
      uint32_t c3[3];
      uint32_t cell = cell_of(o, nd, p, c3);
      if (!test_bit(nd->grid, cell)) {
        set_bit(nd->grid, cell);
        if (n_backlog == cap_backlog) {
          uint64_t cap = cap_backlog ? cap_backlog * 2 : 1024;
          backlog_entry* nb = (backlog_entry*)realloc(backlog, cap * sizeof(backlog_entry));
          if (!nb) {
            rc = ORC_ERR_NOMEM;
            goto done;
          }
          backlog = nb;
          cap_backlog = cap;
        }
        backlog[n_backlog].node = id;
        backlog[n_backlog].cell = cell;
        backlog[n_backlog].voxel = voxel_point(o, nd, c3, p);
        n_backlog++;
        nd->vox_counter++;
        if (from_spill && id < n_nodes_at_start && was_inner[id])
          o->stats.spill_voxels_at_old_inner++;
      }
      id = nd->child0 + octant(nd, p);
    }
  }

  /* ---- Section 5.3: ceil(count / C) chunks per node. */
  for (uint64_t id = 0; id < o->n_nodes; ++id) {
    node* nd = &o->nodes[id];
    uint64_t total = nd->is_leaf ? nd->counter : nd->num_voxels + nd->vox_counter;
    uint64_t need = (total + C - 1) / C;
    while (o->nodes[id].n_chunks < need) {
      rc = append_chunk(o, (uint32_t)id);
      if (rc) goto done;
    }
  }

  /* ---- Section 5.4: store points (numPoints gives the slot), then voxels. */
  for (uint64_t k = 0; k < n + spill.n; ++k) {
    const orc_point* p = k < n ? &pts[k] : &spill.v[k - n].p;
    uint32_t gidx = k < n ? (uint32_t)(o->base + k) : spill.v[k - n].gidx;
    node* leaf = &o->nodes[descend(o, p)];
    orc_point_rec* r = slot(o, leaf, leaf->num_points++);
    r->x = p->x;
    r->y = p->y;
    r->z = p->z;
    r->rgba = pack_rgba(p);
    r->gidx = gidx;
  }
  for (uint64_t b = 0; b < n_backlog; ++b) {
    node* nd = &o->nodes[backlog[b].node];
    orc_point_rec* r = slot(o, nd, nd->num_voxels++);
    r->x = backlog[b].voxel.x;
    r->y = backlog[b].voxel.y;
    r->z = backlog[b].voxel.z;
    r->rgba = pack_rgba(&backlog[b].voxel);
    r->gidx = backlog[b].cell;
  }

  o->base += n;
  o->stats.batches++;
  o->stats.points += n;
  o->stats.spilled += spill.n;
  o->stats.voxels += n_backlog;

done:
  free(spill.v);
  free(backlog);
  free(was_inner);
  return rc;
}

void orc_inc_sizes(const orc_inc* o, orc_sizes* s) {
  s->n_nodes = o->n_nodes;
  s->n_points = 0;
  s->n_voxels = 0;
  for (uint64_t id = 0; id < o->n_nodes; ++id) {
    s->n_points += o->nodes[id].num_points;
    s->n_voxels += o->nodes[id].num_voxels;
  }
}

void orc_inc_stats(const orc_inc* o, orc_stats* s) {
  *s = o->stats;
  uint64_t live = 0;
  for (uint64_t id = 0; id < o->n_nodes; ++id) live += o->nodes[id].n_chunks;
  s->chunks_live = live;
  s->chunks_pool = o->n_pool;
  s->chunks_bumped = o->chunks_bumped;
}

/* ---- canonical export */

typedef struct {
  uint32_t level;
  uint32_t ix, iy, iz;
  uint32_t id;
} node_key;

static int cmp_node_key(const void* pa, const void* pb) {
  const node_key *a = (const node_key*)pa, *b = (const node_key*)pb;
  if (a->level != b->level) return a->level < b->level ? -1 : 1;
  if (a->ix != b->ix) return a->ix < b->ix ? -1 : 1;
  if (a->iy != b->iy) return a->iy < b->iy ? -1 : 1;
  if (a->iz != b->iz) return a->iz < b->iz ? -1 : 1;
  return 0;
}

static int cmp_prec_gidx(const void* pa, const void* pb) {
  uint32_t a = ((const orc_point_rec*)pa)->gidx, b = ((const orc_point_rec*)pb)->gidx;
  return a < b ? -1 : (a > b ? 1 : 0);
}

static int cmp_vrec_cell(const void* pa, const void* pb) {
  uint32_t a = ((const orc_voxel_rec*)pa)->cell, b = ((const orc_voxel_rec*)pb)->cell;
  return a < b ? -1 : (a > b ? 1 : 0);
}

int orc_inc_export(const orc_inc* o, orc_node* nodes, orc_point_rec* points,
                   orc_voxel_rec* voxels) {
  node_key* keys = (node_key*)malloc(sizeof(node_key) * (o->n_nodes ? o->n_nodes : 1));
  if (!keys) return ORC_ERR_NOMEM;
  for (uint64_t id = 0; id < o->n_nodes; ++id) {
    const node* nd = &o->nodes[id];
    keys[id].level = nd->level;
    keys[id].ix = (uint32_t)(((int64_t)nd->min[0] - o->cfg.root_min[0]) >> nd->log2size);
    keys[id].iy = (uint32_t)(((int64_t)nd->min[1] - o->cfg.root_min[1]) >> nd->log2size);
    keys[id].iz = (uint32_t)(((int64_t)nd->min[2] - o->cfg.root_min[2]) >> nd->log2size);
    keys[id].id = (uint32_t)id;
  }
  qsort(keys, o->n_nodes, sizeof(node_key), cmp_node_key);
  uint64_t pp = 0, vv = 0;
  for (uint64_t k = 0; k < o->n_nodes; ++k) {
    const node* nd = &o->nodes[keys[k].id];
    orc_node* out = &nodes[k];
    out->level = nd->level;
    out->is_inner = !nd->is_leaf;
    out->min[0] = nd->min[0];
    out->min[1] = nd->min[1];
    out->min[2] = nd->min[2];
    out->log2size = nd->log2size;
    out->n_points = nd->num_points;
    out->n_voxels = nd->num_voxels;
    out->n_chunks = nd->n_chunks;
    if (nd->is_leaf) {
      for (uint64_t i = 0; i < nd->num_points; ++i) points[pp + i] = *slot(o, nd, i);
      qsort(points + pp, nd->num_points, sizeof(orc_point_rec), cmp_prec_gidx);
      pp += nd->num_points;
    } else {
      for (uint64_t i = 0; i < nd->num_voxels; ++i) {
        const orc_point_rec* r = slot(o, nd, i);
        orc_voxel_rec* v = &voxels[vv + i];
        v->cell = r->gidx;
        v->x = r->x;
        v->y = r->y;
        v->z = r->z;
        v->rgba = r->rgba;
      }
      qsort(voxels + vv, nd->num_voxels, sizeof(orc_voxel_rec), cmp_vrec_cell);
      vv += nd->num_voxels;
    }
  }
  free(keys);
  return ORC_OK;
}

void orc_inc_destroy(orc_inc* o) {
  if (!o) return;
  for (uint64_t id = 0; id < o->n_nodes; ++id) {
    node* nd = &o->nodes[id];
    for (chunk* ch = nd->head; ch;) {
      chunk* nx = ch->next;
      free(ch->items);
      free(ch);
      ch = nx;
    }
    free(nd->index);
    free(nd->grid);
  }
  for (uint64_t k = 0; k < o->n_pool; ++k) {
    free(o->pool[k]->items);
    free(o->pool[k]);
  }
  free(o->pool);
  free(o->nodes);
  free(o);
}
