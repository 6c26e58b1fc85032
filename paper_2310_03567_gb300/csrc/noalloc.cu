// Voxel sampling of one node without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need this
// step: a real-time frame loop that forbids allocation once it is running
// (cudaMalloc and cudaFree may synchronise the whole device and stall the
// frame), or code embedded in another framework that owns every device buffer
// and hands out only its inputs and outputs. For them this file keeps the
// step's scratch (the claim table and the list of new cells) in one fixed,
// file-scope device array instead of the caller's arena.
//
// The array is small and fixed: every GPU that loads the library holds it
// until the process exits. Every call reuses it, so a call clears it first,
// and two calls whose kernels overlap on the GPU race on it.
#include <cuda_runtime.h>

#include <cstdint>

#include "simlod.h"

namespace {

constexpr unsigned long long HASH_EMPTY = ~0ull;
constexpr uint32_t FULL_MASK = 0xFFFFFFFFu;

struct HSlot {
  unsigned long long key;  // cell index, HASH_EMPTY when free
  unsigned long long val;  // (point index << 32) | rgba of the best point so far
};

__device__ __forceinline__ unsigned long long fmix64(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

// Cell of an offset r inside a cube of side 2^L on a 2^G grid: (r << G) >> L.
__device__ __forceinline__ uint32_t cell_axis(uint32_t r, uint32_t L, uint32_t G) {
  return (L >= G) ? (r >> (L - G)) : (r << (G - L));
}

__device__ __forceinline__ uint32_t cell_index(uint32_t rx, uint32_t ry, uint32_t rz, uint32_t L,
                                               uint32_t G) {
  return cell_axis(rx, L, G) | (cell_axis(ry, L, G) << G) | (cell_axis(rz, L, G) << (2u * G));
}

constexpr uint32_t NA_TABLE_SLOTS = 1u << 18;                // claim table, load <= 1/2
constexpr uint32_t NA_MAX_POINTS = SIMLOD_NOALLOC_MAX_POINTS; // = max distinct cells
static_assert(2ull * NA_MAX_POINTS <= NA_TABLE_SLOTS, "table too small for the point limit");

struct NaScratch {
  HSlot table[NA_TABLE_SLOTS];   // (cell) -> (index << 32 | rgba), lowest index wins
  uint32_t list[NA_MAX_POINTS];  // table slots of the cells found by this call
  uint32_t count;                // entries in list
  uint32_t pad[63];
};

// 4 MiB + 512 KiB + 256 B per device, for the life of the process.
static __device__ __align__(256) NaScratch g_na_scratch;

// Device address of g_na_scratch in the current context. In host code the
// symbol itself is only a stand-in, not a device address. The address is
// looked up on every call (a host-side query, no stream work): a context
// re-created on the device (after cudaDeviceReset) reloads this module, and
// the array may then sit elsewhere. The first call in a context also loads
// the module's device code.
int na_scratch(NaScratch** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return SIMLOD_ERR_CUDA;
  *out = static_cast<NaScratch*>(p);
  return SIMLOD_OK;
}

__global__ void k_na_clear(NaScratch* s) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < NA_TABLE_SLOTS;
       i += gridDim.x * blockDim.x) {
    s->table[i].key = HASH_EMPTY;
    s->table[i].val = HASH_EMPTY;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) s->count = 0;
}

__device__ __forceinline__ void na_claim(NaScratch* s, unsigned long long key,
                                         unsigned long long val) {
  uint32_t h = (uint32_t)fmix64(key) & (NA_TABLE_SLOTS - 1u);
  for (uint32_t probe = 0; probe < NA_TABLE_SLOTS; ++probe) {
    HSlot* e = s->table + h;
    unsigned long long k = *reinterpret_cast<volatile unsigned long long*>(&e->key);
    if (k == HASH_EMPTY) {
      unsigned long long old = atomicCAS(&e->key, HASH_EMPTY, key);
      if (old == HASH_EMPTY) {
        atomicMin(&e->val, val);
        s->list[atomicAdd(&s->count, 1u)] = h;  // at most NA_MAX_POINTS cells
        return;
      }
      k = old;
    }
    if (k == key) {
      atomicMin(&e->val, val);
      return;
    }
    h = (h + 1u) & (NA_TABLE_SLOTS - 1u);
  }
}

// Every point inside the node claims its cell; the lowest index wins.
__global__ void k_na_claim(NaScratch* s, const int4* pts, uint32_t n, int3 mn, uint32_t L,
                           uint32_t G) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t nwarps = gridDim.x * (blockDim.x / 32);
  for (uint32_t w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; w * 32 < n; w += nwarps) {
    const uint32_t i = w * 32 + lane;
    bool want = false;
    unsigned long long key = 0;
    int4 p = make_int4(0, 0, 0, 0);
    if (i < n) {
      p = __ldg(pts + i);
      const long long side = 1ll << L;
      const long long dx = (long long)p.x - mn.x, dy = (long long)p.y - mn.y,
                      dz = (long long)p.z - mn.z;
      want = dx >= 0 && dy >= 0 && dz >= 0 && dx < side && dy < side && dz < side;
      if (want) key = cell_index((uint32_t)dx, (uint32_t)dy, (uint32_t)dz, L, G);
    }
    const unsigned m = __ballot_sync(FULL_MASK, want);
    if (want) {
      const unsigned grp = __match_any_sync(m, key);
      const unsigned best = __reduce_min_sync(grp, i);
      if (i == best) na_claim(s, key, ((unsigned long long)i << 32) | (uint32_t)p.w);
    }
  }
}

// One voxel per claimed cell, at the floor of the cell centre (Section 3.4).
__global__ void k_na_emit(NaScratch* s, int3 mn, uint32_t L, uint32_t G, simlod_voxel_rec* out,
                          uint32_t* d_count) {
  const uint32_t cnt = s->count;
  const uint32_t amask = (1u << G) - 1u;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
    const HSlot h = s->table[s->list[e]];
    const uint32_t cell = (uint32_t)h.key;
    const uint32_t cx = cell & amask, cy = (cell >> G) & amask, cz = cell >> (2u * G);
    simlod_voxel_rec v;
    v.cell = cell;
    v.x = mn.x + (int32_t)(((2ull * cx + 1ull) << L) >> (G + 1u));
    v.y = mn.y + (int32_t)(((2ull * cy + 1ull) << L) >> (G + 1u));
    v.z = mn.z + (int32_t)(((2ull * cz + 1ull) << L) >> (G + 1u));
    v.rgba = (uint32_t)h.val;
    out[e] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *d_count = cnt;
}

}  // namespace

extern "C" SIMLOD_API int simlod_sample_node_noalloc(const simlod_point* d_pts, uint64_t n,
                                                     const int32_t node_min[3],
                                                     uint32_t log2size, uint32_t grid_log2,
                                                     simlod_voxel_rec* d_voxels,
                                                     uint64_t voxels_capacity, uint32_t* d_count,
                                                     void* stream) {
  if (!node_min || !d_voxels || !d_count || (n && !d_pts) ||
      (reinterpret_cast<uintptr_t>(d_pts) & 15u) || log2size > 31 || grid_log2 < 1 ||
      grid_log2 > 7)
    return SIMLOD_ERR_INVALID_ARG;
  if (n > NA_MAX_POINTS) return SIMLOD_ERR_INVALID_ARG;  // beyond the fixed scratch
  const uint64_t cells = 1ull << (3 * grid_log2);
  if (voxels_capacity < (n < cells ? n : cells)) return SIMLOD_ERR_INVALID_ARG;
  for (int a = 0; a < 3; ++a)
    if ((long long)node_min[a] + (1ll << log2size) - 1 > 0x7FFFFFFFll) return SIMLOD_ERR_INVALID_ARG;
  // an error already pending from earlier work is reported, not cleared
  if (cudaPeekAtLastError() != cudaSuccess) return SIMLOD_ERR_CUDA;
  NaScratch* s = nullptr;
  int rc = na_scratch(&s);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int3 mn = make_int3(node_min[0], node_min[1], node_min[2]);
  // the whole table is cleared on every call: a table left by a context that
  // no longer exists, or by a call that failed half way, may hold anything
  k_na_clear<<<256, 256, 0, st>>>(s);
  if (cudaPeekAtLastError() != cudaSuccess) return SIMLOD_ERR_CUDA;
  if (n) {
    const uint32_t blocks = (uint32_t)((n + 255) / 256);
    k_na_claim<<<blocks, 256, 0, st>>>(s, reinterpret_cast<const int4*>(d_pts), (uint32_t)n, mn,
                                       log2size, grid_log2);
    if (cudaPeekAtLastError() != cudaSuccess) return SIMLOD_ERR_CUDA;
  }
  k_na_emit<<<64, 256, 0, st>>>(s, mn, log2size, grid_log2, d_voxels, d_count);
  return cudaPeekAtLastError() == cudaSuccess ? SIMLOD_OK : SIMLOD_ERR_CUDA;
}
