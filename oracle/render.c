/*
 * CPU oracle of the paper's renderer (Section 6), for the tests only: the
 * level-of-detail node selection and pixel-sized splats that keep the
 * closest sample per pixel. TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Readings of Section 6 (it fixes neither the projection nor "size on
 * screen"):
 *  - clip = M (x, y, z, 1) with M a row-major 4x4 float matrix and x, y, z
 *    the integer coordinates converted to float; the depth of a sample is its
 *    clip w. A sample is drawn when w > 0 and its screen position
 *    s = (clip.xy / w * 0.5 + 0.5) * (width, height) lies in
 *    [0, width) x [0, height); its pixel is floor(s).
 *  - A pixel keeps the minimum of (float bits of w) << 32 | rgba: the
 *    closest sample (ties: the smaller colour word). Empty = all ones.
 *  - A node's cube is culled when all 8 corners lie outside one of the
 *    planes x < -w, x > w, y < -w, y > w, w <= 0 (conservative frustum test).
 *  - A node's size on screen is the larger side of the screen-space box of
 *    its 8 projected corners, or infinite when a corner has w <= 0.
 *  - Selection, as the paper describes it, top down from the root: a node in
 *    the frustum is drawn if it is a leaf or not larger than 2^G pixels (the
 *    voxel resolution of an inner node); an inner node larger than that is
 *    hidden and its children are visited instead.
 *  - Every product, sum and quotient is one IEEE single-precision operation
 *    in the order written (the library is built without contraction), so the
 *    GPU can match it bit for bit.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

typedef struct {
  float cx, cy, cw;
} clip3;

static clip3 project(const float* m, float x, float y, float z) {
  clip3 c;
  c.cx = ((m[0] * x + m[1] * y) + m[2] * z) + m[3];
  c.cy = ((m[4] * x + m[5] * y) + m[6] * z) + m[7];
  c.cw = ((m[12] * x + m[13] * y) + m[14] * z) + m[15];
  return c;
}

static float screen(float c, float w, float extent) { return ((c / w) * 0.5f + 0.5f) * extent; }

/* Frustum test and size on screen of the cube [mn, mn + 2^L). */
static void cube_view(const float* m, const int64_t mn[3], uint32_t L, float W, float H,
                      int* culled, float* size) {
  int out[5] = {0, 0, 0, 0, 0};
  int behind = 0;
  float x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
  for (int k = 0; k < 8; ++k) {
    const float x = (float)(mn[0] + ((int64_t)(k & 1) << L));
    const float y = (float)(mn[1] + ((int64_t)((k >> 1) & 1) << L));
    const float z = (float)(mn[2] + ((int64_t)((k >> 2) & 1) << L));
    const clip3 c = project(m, x, y, z);
    out[0] += c.cx < -c.cw;
    out[1] += c.cx > c.cw;
    out[2] += c.cy < -c.cw;
    out[3] += c.cy > c.cw;
    out[4] += !(c.cw > 0.0f);
    if (!(c.cw > 0.0f)) {
      behind = 1;
      continue;
    }
    const float sx = screen(c.cx, c.cw, W), sy = screen(c.cy, c.cw, H);
    if (sx < x0) x0 = sx;
    if (sx > x1) x1 = sx;
    if (sy < y0) y0 = sy;
    if (sy > y1) y1 = sy;
  }
  *culled = out[0] == 8 || out[1] == 8 || out[2] == 8 || out[3] == 8 || out[4] == 8;
  if (behind) {
    *size = INFINITY;
  } else {
    const float w = x1 - x0, h = y1 - y0;
    *size = w > h ? w : h;
  }
}

static void splat(const float* m, int32_t px_, int32_t py_, int32_t pz_, uint32_t rgba,
                  uint32_t W, uint32_t H, uint64_t* fb) {
  const clip3 c = project(m, (float)px_, (float)py_, (float)pz_);
  if (!(c.cw > 0.0f)) return;
  const float sx = screen(c.cx, c.cw, (float)W), sy = screen(c.cy, c.cw, (float)H);
  if (!(sx >= 0.0f && sx < (float)W && sy >= 0.0f && sy < (float)H)) return;
  const uint32_t px = (uint32_t)sx, py = (uint32_t)sy;
  uint32_t depth;
  memcpy(&depth, &c.cw, 4);
  const uint64_t key = ((uint64_t)depth << 32) | rgba;
  uint64_t* f = fb + (uint64_t)py * W + px;
  if (key < *f) *f = key;
}

typedef struct {
  const orc_config* cfg;
  const orc_node* nodes;
  uint64_t n_nodes;
  const uint64_t* p_off;  /* first point of node k */
  const uint64_t* v_off;  /* first voxel of node k */
  const orc_point_rec* points;
  const orc_voxel_rec* voxels;
  const float* m;
  uint32_t W, H;
  uint64_t* fb;
  uint8_t* drawn;
  uint64_t n_drawn;
} render_ctx;

/* Canonical index of node (level, ix, iy, iz), or -1 (nodes are sorted by
   that key). */
static int64_t find_node(const render_ctx* r, uint32_t level, int64_t ix, int64_t iy, int64_t iz) {
  int64_t lo = 0, hi = (int64_t)r->n_nodes - 1;
  const orc_config* c = r->cfg;
  while (lo <= hi) {
    const int64_t mid = (lo + hi) / 2;
    const orc_node* n = &r->nodes[mid];
    const uint32_t L = n->log2size;
    const int64_t kx = ((int64_t)n->min[0] - c->root_min[0]) >> L;
    const int64_t ky = ((int64_t)n->min[1] - c->root_min[1]) >> L;
    const int64_t kz = ((int64_t)n->min[2] - c->root_min[2]) >> L;
    int cmp;
    if (n->level != level) cmp = n->level < level ? -1 : 1;
    else if (kx != ix) cmp = kx < ix ? -1 : 1;
    else if (ky != iy) cmp = ky < iy ? -1 : 1;
    else if (kz != iz) cmp = kz < iz ? -1 : 1;
    else return mid;
    if (cmp < 0) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

static void draw_node(render_ctx* r, int64_t k) {
  const orc_node* n = &r->nodes[k];
  r->drawn[k] = 1;
  r->n_drawn++;
  if (n->is_inner) {
    for (uint64_t q = 0; q < n->n_voxels; ++q) {
      const orc_voxel_rec* v = &r->voxels[r->v_off[k] + q];
      splat(r->m, v->x, v->y, v->z, v->rgba, r->W, r->H, r->fb);
    }
  } else {
    for (uint64_t q = 0; q < n->n_points; ++q) {
      const orc_point_rec* p = &r->points[r->p_off[k] + q];
      splat(r->m, p->x, p->y, p->z, p->rgba, r->W, r->H, r->fb);
    }
  }
}

static void visit(render_ctx* r, int64_t k) {
  const orc_node* n = &r->nodes[k];
  const int64_t mn[3] = {n->min[0], n->min[1], n->min[2]};
  int culled;
  float size;
  cube_view(r->m, mn, n->log2size, (float)r->W, (float)r->H, &culled, &size);
  if (culled) return;
  const float lod = (float)(1u << r->cfg->grid_log2);
  if (!n->is_inner || !(size > lod)) {
    draw_node(r, k);
    return;
  }
  const orc_config* c = r->cfg;
  const uint32_t L = n->log2size;
  const int64_t ix = ((int64_t)n->min[0] - c->root_min[0]) >> L;
  const int64_t iy = ((int64_t)n->min[1] - c->root_min[1]) >> L;
  const int64_t iz = ((int64_t)n->min[2] - c->root_min[2]) >> L;
  for (int o = 0; o < 8; ++o) {
    const int64_t ch = find_node(r, n->level + 1, 2 * ix + (o & 1), 2 * iy + ((o >> 1) & 1),
                                 2 * iz + ((o >> 2) & 1));
    if (ch >= 0) visit(r, ch);
  }
}

int orc_render(const orc_config* cfg, const orc_node* nodes, uint64_t n_nodes,
               const orc_point_rec* points, const orc_voxel_rec* voxels, const float view_proj[16],
               uint32_t width, uint32_t height, uint64_t* framebuffer, uint8_t* drawn,
               uint64_t* n_drawn) {
  if (!cfg || !framebuffer || !drawn || !view_proj || width == 0 || height == 0)
    return ORC_ERR_INVALID;
  for (uint64_t i = 0; i < (uint64_t)width * height; ++i) framebuffer[i] = ~0ull;
  memset(drawn, 0, n_nodes);
  uint64_t* p_off = malloc(sizeof(uint64_t) * (n_nodes + 1));
  uint64_t* v_off = malloc(sizeof(uint64_t) * (n_nodes + 1));
  if (!p_off || !v_off) {
    free(p_off);
    free(v_off);
    return ORC_ERR_NOMEM;
  }
  p_off[0] = v_off[0] = 0;
  for (uint64_t k = 0; k < n_nodes; ++k) {
    p_off[k + 1] = p_off[k] + nodes[k].n_points;
    v_off[k + 1] = v_off[k] + nodes[k].n_voxels;
  }
  render_ctx r = {cfg, nodes, n_nodes, p_off, v_off, points, voxels, view_proj,
                  width, height, framebuffer, drawn, 0};
  if (n_nodes) visit(&r, 0); /* the root is the first node in canonical order */
  if (n_drawn) *n_drawn = r.n_drawn;
  free(p_off);
  free(v_off);
  return ORC_OK;
}
