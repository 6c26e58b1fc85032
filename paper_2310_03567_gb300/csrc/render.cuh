// The renderer of Section 6: level-of-detail node selection and pixel-sized
// splats that keep the closest sample per pixel with a 64-bit atomicMin on
// (float bits of depth << 32 | rgba), drawn straight from the octree's chunk
// lists. It reads the octree as the update left it (stream order) and
// changes nothing in it.
//
// Selection, per node in parallel: a node is drawn when it is in the view
// frustum, it is a leaf or not larger than 2^G pixels on screen (the voxel
// resolution of an inner node), and its parent is larger than 2^G pixels (or
// it is the root). Because a child's projected box lies inside its parent's,
// this selects exactly the nodes of the paper's top-down rule (an inner node
// larger than 2^G pixels is hidden and its children are drawn instead).
//
// Projection: clip = M (x, y, z, 1) with M row-major; depth = clip w; a
// sample at screen s = (clip.xy / w * 0.5 + 0.5) * (width, height) with w > 0
// and s inside the screen lands in pixel floor(s). A cube is culled when all
// 8 corners are outside one plane of x < -w, x > w, y < -w, y > w, w <= 0;
// its size on screen is the larger side of its corners' screen box
// (infinite when a corner has w <= 0). Every float operation is one IEEE
// single-precision operation in the written order (no contraction), so the
// result is reproducible bit for bit.
#pragma once

#include "device.cuh"

namespace SL_NS {

struct View {
  float m[16];
  float W, H, lod;
  uint32_t width, height;
};

__device__ __forceinline__ float dot4(float a, float x, float b, float y, float c, float z, float d) {
  return __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(a, x), __fmul_rn(b, y)), __fmul_rn(c, z)), d);
}

__device__ __forceinline__ float screen_coord(float c, float w, float extent) {
  return __fmul_rn(__fadd_rn(__fmul_rn(__fdiv_rn(c, w), 0.5f), 0.5f), extent);
}

// Frustum test and size on screen of the cube [mn, mn + 2^L).
__device__ __forceinline__ void cube_view(const View& v, const long long (&mn)[3], uint32_t L,
                                          bool& culled, float& size) {
  int out0 = 0, out1 = 0, out2 = 0, out3 = 0, out4 = 0;
  bool behind = false;
  float x0 = __int_as_float(0x7f800000), x1 = -x0, y0 = x0, y1 = -x0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float x = __ll2float_rn(mn[0] + ((long long)(k & 1) << L));
    const float y = __ll2float_rn(mn[1] + ((long long)((k >> 1) & 1) << L));
    const float z = __ll2float_rn(mn[2] + ((long long)((k >> 2) & 1) << L));
    const float cx = dot4(v.m[0], x, v.m[1], y, v.m[2], z, v.m[3]);
    const float cy = dot4(v.m[4], x, v.m[5], y, v.m[6], z, v.m[7]);
    const float cw = dot4(v.m[12], x, v.m[13], y, v.m[14], z, v.m[15]);
    out0 += cx < -cw;
    out1 += cx > cw;
    out2 += cy < -cw;
    out3 += cy > cw;
    out4 += !(cw > 0.0f);
    if (!(cw > 0.0f)) {
      behind = true;
      continue;
    }
    const float sx = screen_coord(cx, cw, v.W), sy = screen_coord(cy, cw, v.H);
    if (sx < x0) x0 = sx;
    if (sx > x1) x1 = sx;
    if (sy < y0) y0 = sy;
    if (sy > y1) y1 = sy;
  }
  culled = out0 == 8 || out1 == 8 || out2 == 8 || out3 == 8 || out4 == 8;
  if (behind) {
    size = __int_as_float(0x7f800000);
  } else {
    const float w = __fsub_rn(x1, x0), h = __fsub_rn(y1, y0);
    size = w > h ? w : h;
  }
}

__device__ __forceinline__ bool node_drawn(const Ctx& c, const View& v, uint32_t id) {
  const NodeMeta& m = c.meta[id];
  const uint32_t level = m.level;
  const uint32_t L = c.rlog2 - level;
  const long long mn[3] = {m.min[0], m.min[1], m.min[2]};
  bool culled;
  float size;
  cube_view(v, mn, L, culled, size);
  if (culled) return false;
  if (c.child[id] != NONE && size > v.lod) return false;  // hidden: its children are drawn
  if (level == 0) return true;
  long long pmn[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    pmn[a] = c.rmin[a] + (((mn[a] - c.rmin[a]) >> (L + 1)) << (L + 1));
  float psize;
  cube_view(v, pmn, L + 1, culled, psize);
  return psize > v.lod;
}

// One thread per node: list the drawn nodes (warp-aggregated appends).
__global__ void k_render_select(Ctx c, View v, uint32_t* vis) {
  const uint32_t n = vload(&c.ctl->n_nodes);
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b < n; b += stride) {
    const uint64_t id = b + lane;
    const bool d = id < n && id < c.max_nodes && node_drawn(c, v, (uint32_t)id);
    const unsigned mm = __ballot_sync(FULL_MASK, d);
    if (mm == 0u) continue;
    uint32_t o = 0;
    if (lane == 0) o = atomicAdd(&c.ctl->vis_count, (uint32_t)__popc(mm));
    o = __shfl_sync(FULL_MASK, o, 0);
    if (d) vis[o + __popc(mm & ((1u << lane) - 1u))] = (uint32_t)id;
  }
}

__device__ __forceinline__ void splat(const View& v, int4 r, unsigned long long* fb) {
  const float x = (float)r.x, y = (float)r.y, z = (float)r.z;
  const float cw = dot4(v.m[12], x, v.m[13], y, v.m[14], z, v.m[15]);
  if (!(cw > 0.0f)) return;
  const float cx = dot4(v.m[0], x, v.m[1], y, v.m[2], z, v.m[3]);
  const float cy = dot4(v.m[4], x, v.m[5], y, v.m[6], z, v.m[7]);
  const float sx = screen_coord(cx, cw, v.W), sy = screen_coord(cy, cw, v.H);
  if (!(sx >= 0.0f && sx < v.W && sy >= 0.0f && sy < v.H)) return;
  const uint32_t px = __float2uint_rz(sx), py = __float2uint_rz(sy);
  const unsigned long long key =
      ((unsigned long long)__float_as_uint(cw) << 32) | (uint32_t)r.w;
  atomicMin(fb + (uint64_t)py * v.width + px, key);
}

// One warp per drawn node: walk its chunk list (Section 6's chunk loop, with the
// next link loaded before the chunk's records are drawn) and splat every
// point (leaf) or voxel (inner node).
__global__ void k_render_draw(Ctx c, View v, const uint32_t* vis, unsigned long long* fb) {
  const uint32_t nv = vload(&c.ctl->vis_count);
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const uint64_t nwarps = (uint64_t)gridDim.x * blockDim.x / 32;
  for (uint64_t k = warp; k < nv && k < c.max_nodes; k += nwarps) {
    const uint32_t id = vis[k];
    const uint32_t n = c.num[id];
    const NodeMeta& m = c.meta[id];
    if (m.compact) {  // one contiguous array (simlod_compact)
      if (array_ok(c, m.head, n)) {
        const int4* recs = array_recs(c, m.head);
        for (uint32_t q = lane; q < n; q += 32) splat(v, recs[q], fb);
      } else if (lane == 0) {
        set_error(c, E_INTERNAL);
      }
      if (lane == 0) atomicAdd(&c.ctl->render_samples, (unsigned long long)n);
      continue;
    }
    const uint32_t nch = m.n_chunks;
    uint32_t ref = m.head, done = 0;
    for (uint32_t j = 0; j < nch && done < n; ++j) {
      if (!ref_ok(c, ref, c.chunk_bytes)) {
        if (lane == 0) set_error(c, E_INTERNAL);
        break;
      }
      const uint32_t nxt = *chunk_next(c, ref);
      const uint32_t cnt = min(c.C, n - done);
      const int4* recs = chunk_recs(c, ref);
      for (uint32_t q = lane; q < cnt; q += 32) splat(v, recs[q], fb);
      done += cnt;
      ref = nxt;
    }
    if (lane == 0) atomicAdd(&c.ctl->render_samples, (unsigned long long)n);
  }
}

__global__ void k_fb_clear(unsigned long long* fb, uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    fb[i] = ~0ull;
}

}  // namespace SL_NS
