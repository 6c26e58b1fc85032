// Device-side data layout and the phase functions of one octree update.
//
// The update of one batch follows Section 5 of the paper, re-planned for a
// GPU that can keep the per-update working set in L2:
//
//  count1  every batch point walks from the root to its leaf. At every inner
//          node on the way it tests the node's occupancy bit (Section 3.3);
//          an empty cell makes the point a contender for a new voxel. At the
//          leaf it is counted (Section 5.1, "Counting"); the leaf is kept per
//          point (its cursor).
//  decide  per candidate node: a leaf whose stored + counted points exceed T
//          splits (Section 5.1, "Splitting"): 8 children, a grid, and one
//          spill task per chunk of its stored points. Any other counted node
//          is final and gets its chunks now (Section 5.3).
//  advance points whose cursor node split in the previous round (batch
//          points, and the stored points of split leaves, copied out of their
//          old chunks at their first move) sample that node's grid and move
//          one level down, counting into the child; the grids of the previous
//          round's splits are zeroed alongside. Repeated with decide until
//          nothing splits: the paper's iterative deepening, but each round
//          touches only the points that have to move (mover lists).
//  store   every point goes to its cursor leaf at the next free slot; every
//          new voxel goes to its node (Section 5.4); occupancy bits are set
//          here, after all claims of the update; the chunks of split leaves
//          return to the pool (Section 3.4).
//
// Voxel claims: the paper lets the first point that finds an empty cell win.
// Here all contenders of an update for a (node, cell) meet in an open-
// addressing table with a 64-bit atomicMin on (gidx << 32 | rgba), so the
// lowest arrival index wins regardless of thread timing. The table entries of
// an update are listed (the backlog of Section 5.2) and cleared by store.
//
// Descents read the node table (first child, grid reference) from a copy in
// shared memory of the first NODE_CACHE nodes (the node ids of the upper
// levels are the smallest): the plain form's count / advance kernels load it,
// the persistent kernel loads it once and patches it after every decide
// round with the nodes that split or were created.
// Per-node counters are summed per block in shared memory before they reach
// the global counters (the block tally cache).
#pragma once

#include <cstddef>
#include <cstdint>

#include "simlod.h"

// Namespace of this instance of the device code: the library builds the
// persistent update kernel more than once, with other launch-shape knobs,
// each instance in a namespace of its own (fused_variant.cu).
#ifndef SL_NS
#define SL_NS sl
#endif

namespace SL_NS {

constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr unsigned long long HASH_EMPTY = ~0ull;
constexpr uint32_t FULL_MASK = 0xFFFFFFFFu;
constexpr int MAX_PROBES = 1 << 14;
constexpr uint32_t REF_BYTES = 256;  // chunk, grid and directory references count 256-byte units
constexpr uint32_t CHUNK_HEADER = 16;
// Launch-shape and algorithm knobs (compile-time; -D overrides them).
#ifndef SL_NODE_CACHE
#define SL_NODE_CACHE 4096
#endif
#ifndef SL_DESCENT_GROUP
#define SL_DESCENT_GROUP 2
#endif
#ifndef SL_PHASE_BLOCK
#define SL_PHASE_BLOCK 512
#endif
#ifndef SL_PHASE_MIN_BLOCKS
#define SL_PHASE_MIN_BLOCKS 2
#endif
#ifndef SL_HASH_BUCKET
#define SL_HASH_BUCKET 0
#endif
#ifndef SL_ADVANCE_UNROLL
#define SL_ADVANCE_UNROLL 1
#endif
#ifndef SL_ADVANCE_RUNS
#define SL_ADVANCE_RUNS 0  // 1: the advance phase merges lanes with equal keys first
#endif
#ifndef SL_CTL_VIEW
#define SL_CTL_VIEW 1
#endif
#ifndef SL_CTL_SPREAD
#define SL_CTL_SPREAD 1
#endif
#ifndef SL_STORE_PREFETCH
#define SL_STORE_PREFETCH 1
#endif
#ifndef SL_COUNT_PREFETCH
#define SL_COUNT_PREFETCH 1
#endif
#ifndef SL_COUNT_UNROLL
#define SL_COUNT_UNROLL 1
#endif
#ifndef SL_STORE_UNROLL
#define SL_STORE_UNROLL 2
#endif
#ifndef SL_STORE_BLOCK
#define SL_STORE_BLOCK 1
#endif
#ifndef SL_BLOCK_TALLY
#define SL_BLOCK_TALLY 1
#endif
#ifndef SL_COUNT_CHUNK_MAX
#define SL_COUNT_CHUNK_MAX 2  // log2 of the largest count-phase chunk (4 units)
#endif
#ifndef SL_COUNT_CHUNK_DIV
#define SL_COUNT_CHUNK_DIV 8  // a chunk size keeps at least this many chunks per warp
#endif
constexpr uint32_t NODE_CACHE = SL_NODE_CACHE;         // nodes mirrored in shared memory
constexpr uint32_t NODE_CACHE_BYTES = NODE_CACHE * 8;  // child + grid reference
constexpr uint32_t ZERO_UNIT = 4096;                   // bytes of grid zeroed per warp unit
constexpr int DESCENT_GROUP = SL_DESCENT_GROUP;        // levels whose grid words load together
constexpr int ADVANCE_U = SL_ADVANCE_UNROLL;           // advance units a warp carries at a time
constexpr int COUNT_U = SL_COUNT_UNROLL;               // count units a warp carries at a time
#ifndef SL_WBUF
#define SL_WBUF 128
#endif
constexpr uint32_t WBUF = SL_WBUF;                      // new-cell slots staged per warp
constexpr int PHASE_BLOCK = SL_PHASE_BLOCK;            // threads of count / advance / fused blocks
constexpr int PHASE_MIN_BLOCKS = SL_PHASE_MIN_BLOCKS;  // resident blocks per SM they aim for
// dynamic shared memory of the count / advance / fused blocks
#ifndef SL_MVBUF
#define SL_MVBUF 256
#endif
constexpr uint32_t MVBUF = SL_MVBUF;                    // mover-list entries staged per warp
constexpr uint32_t TALLY_LOG2 = 9;                      // block tally cache: 512 nodes
constexpr uint32_t TALLY_SLOTS = 1u << TALLY_LOG2;
// dynamic shared memory of the count / advance / fused blocks: node cache,
// new-cell staging, mover staging, block tally cache
constexpr uint32_t SMEM_WBUF = 2 * NODE_CACHE;                        // in u32 words
constexpr uint32_t SMEM_MVBUF = SMEM_WBUF + (PHASE_BLOCK / 32) * WBUF;
constexpr uint32_t SMEM_TALLY = SMEM_MVBUF + (PHASE_BLOCK / 32) * MVBUF * 2;
constexpr uint32_t PHASE_SMEM_BYTES = 4 * (SMEM_TALLY + 2 * TALLY_SLOTS);

// Sticky device error bits.
enum : uint32_t {
  E_ARENA = 1u,
  E_NODES = 2u,
  E_SPILL = 4u,
  E_BACKLOG = 8u,
  E_ALLOC_REFS = 16u,
  E_INTERNAL = 32u,
  E_POOL = 64u,
  E_TIMEOUT = 128u,
  E_ITER_CAP = 256u,
};

// Control block at the start of the arena.
// The counters that warps all over the grid change with atomics inside a
// phase (SL_HOT) each start a 128-byte line of their own, so that their
// atomics spread over several L2 slices instead of queueing at one.
#if SL_CTL_SPREAD
#define SL_HOT alignas(128)
#else
#define SL_HOT
#endif
struct Ctl {
  unsigned long long base;                  // gidx of the next accepted point
  SL_HOT unsigned long long bump;           // bytes taken from the data region
  unsigned long long chunks_bumped;         // chunks taken from the data region
  SL_HOT unsigned int n_nodes;
  SL_HOT int pool_top;                      // chunk refs in the pool
  unsigned int error;                       // sticky E_* bits
  unsigned int reject;                      // out-of-cube point seen in this update
  SL_HOT unsigned int spill_count;          // re-inserted points of this update
  SL_HOT unsigned int nkeys;                // new voxels (backlog entries) of this update
  SL_HOT unsigned int alloc_seq;            // alloc_refs entries of this update
  SL_HOT unsigned int split_count;          // split-list entries of this update
  SL_HOT unsigned int ntasks;               // spill tasks (= freed chunks) of this update
  unsigned int vis_count;                   // nodes drawn by the last render
  unsigned long long st_batches, st_points, st_rejected, st_spilled, st_splits, st_voxels,
      st_iter_max, st_rounds;
  unsigned long long last_points, last_spilled, last_splits, last_voxels, last_iters;
  unsigned long long st_rejected_async;  // rejections inside fused launches
  SL_HOT unsigned int mv_count[2];       // entries of the two mover lists
  SL_HOT unsigned long long render_samples;  // points and voxels visited by the last render
  unsigned long long phase_ns[8];        // fused form: time per phase (see PH_*)
  unsigned long long st_compacted;       // nodes turned into arrays (simlod_compact), in all
  unsigned long long st_compact_chunks;  // chunks those nodes gave back to the pool
  unsigned long long st_decompacted;     // arrays turned back into chunk lists by an insert
  unsigned long long compact_now;        // nodes that are arrays now
  unsigned long long compact_chunks_now; // chunks those arrays stand in for
  unsigned long long pad_ctl;
};
#undef SL_HOT
static_assert(sizeof(Ctl) % 16 == 0, "Ctl size");

// Phases of the fused form, for its phase clock.
enum : int { PH_COUNT = 0, PH_DECIDE, PH_ADVANCE, PH_STORE, PH_END, PH_ROLLBACK, PH_LAUNCH, PH_OTHER };

// Per-node metadata that the count/advance hot loops do not touch.
struct NodeMeta {
  int32_t min[3];
  uint32_t level;
  uint32_t n_chunks;
  uint32_t head, tail;  // chunk list (points of a leaf, voxels of an inner node)
  uint32_t dir;         // chunk directory of a leaf (ref), NONE if none
  uint32_t st_nch;      // store map of the current update: chunks before allocation,
  uint32_t st_tail;     //   the tail before allocation,
  uint32_t st_seq;      //   first alloc_refs entry of the newly allocated chunks,
  uint32_t st_base;     //   and the records stored before this update
  uint32_t touched;     // updates applied when the node last received records (1 = the first)
  uint32_t compact;     // 1: the records are one contiguous array (head), not a chunk list
  uint32_t pad[2];
};
static_assert(sizeof(NodeMeta) == 64, "NodeMeta size");
static_assert(offsetof(NodeMeta, st_nch) == 32 && offsetof(NodeMeta, st_base) == 44,
              "the store map is one aligned 16-byte load");

struct __align__(16) HSlot {
  unsigned long long key;  // (node << 3G) | cell, HASH_EMPTY when free
  unsigned long long val;  // (gidx << 32) | rgba of the best contender so far
};

struct SplitEntry {
  uint32_t node;
  uint32_t spill_off;
};

// The stored points of one chunk of a split leaf, re-inserted this update:
// point q of the chunk is spill entry dst + q.
struct SpillTask {
  uint32_t ref;   // the chunk
  uint32_t node;  // the leaf that split
  uint32_t dst;   // first spill entry
  uint32_t n;     // points in the chunk
};

// Everything a phase needs: arena pointers and the configuration.
struct Ctx {
  Ctl* ctl;
  uint32_t* child;    // first child id or NONE (leaf), per node
  uint32_t* gridref;  // occupancy grid ref or NONE, per node
  uint32_t* cnt;      // per-update counter: new points (leaf) or new voxels (inner)
  uint32_t* num;      // stored points (leaf) or voxels (inner)
  NodeMeta* meta;
  uint32_t* pool;
  uint32_t* pending;  // chunk refs freed by this update's splits (one per task)
  uint32_t* alloc_refs;
  SplitEntry* splits;
  SpillTask* tasks;
  uint32_t* sp_cur;   // per spill entry: cursor node (after its first move)
  int4* sp_rec;       // per spill entry: the point, copied at its first move
  uint32_t* sp_gidx;  //   and its gidx
  uint32_t* b_cur;    // per batch point: cursor node
  uint32_t* scur;     // per node: store cursor of the current update
  uint2* mv[2];       // mover lists: points that moved in the last advance round
  HSlot* hash;
  uint32_t* keys;     // backlog: table slots of this update's new cells
  uint8_t* data;
  unsigned long long data_bytes;
  int4* staging;
  int32_t rmin[3];
  uint32_t rlog2, T, C, G;
  uint32_t chunk_bytes, chunk_units, grid_bytes, dir_bytes, dir_cap;
  uint32_t hash_mask;
  uint32_t max_nodes, max_chunks, spill_cap, backlog_cap, max_splits;
  uint64_t max_batch;
  uint64_t mv_cap;  // entries of each mover list (batch + spill capacity)
  unsigned long long* launch_bar;  // barrier word of the persistent launch (abort bit)
  unsigned long long bar_ns;       // persistent launch: time limit of one grid-barrier wait
  unsigned long long ready_ns;     //   and of one wait for a batch's ready flag
  unsigned int* progress;          // persistent launch: host-mapped words, [0] batches finished,
                                   //   [1] batches dropped by budget stops (nullptr: none)
};

// Abort bit of a persistent launch's barrier word: set with the first
// device error, so that every block leaves at its next barrier.
constexpr unsigned long long BAR_ABORT = 1ull << 63;

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned long long fmix64(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ void set_error(const Ctx& c, uint32_t bits) {
  atomicOr(&c.ctl->error, bits);
  atomicOr(c.launch_bar, BAR_ABORT);
}

__device__ __forceinline__ uint8_t* ref_ptr(const Ctx& c, uint32_t ref) {
  return c.data + (size_t)ref * REF_BYTES;
}

__device__ __forceinline__ uint32_t* chunk_next(const Ctx& c, uint32_t ref) {
  return reinterpret_cast<uint32_t*>(ref_ptr(c, ref));
}

__device__ __forceinline__ int4* chunk_recs(const Ctx& c, uint32_t ref) {
  return reinterpret_cast<int4*>(ref_ptr(c, ref) + CHUNK_HEADER);
}

__device__ __forceinline__ uint32_t* chunk_aux(const Ctx& c, uint32_t ref) {
  return reinterpret_cast<uint32_t*>(ref_ptr(c, ref) + CHUNK_HEADER + 16u * c.C);
}

// A compacted node's records: one array in the data region, a chunk header
// (next = NONE, then the capacity) followed by cap records and cap aux words,
// the layout of a chunk of cap records.
__device__ __forceinline__ int4* array_recs(const Ctx& c, uint32_t ref) {
  return reinterpret_cast<int4*>(ref_ptr(c, ref) + CHUNK_HEADER);
}

__device__ __forceinline__ uint32_t* array_aux(const Ctx& c, uint32_t ref, uint32_t cap) {
  return reinterpret_cast<uint32_t*>(ref_ptr(c, ref) + CHUNK_HEADER + 16ull * cap);
}

__device__ __forceinline__ unsigned long long array_bytes(uint32_t cap) {
  return ((CHUNK_HEADER + 20ull * cap) + REF_BYTES - 1) / REF_BYTES * REF_BYTES;
}

// A reference that stays inside the data region for `bytes` bytes.
__device__ __forceinline__ bool ref_ok(const Ctx& c, uint32_t ref, uint32_t bytes) {
  return ref != NONE && (unsigned long long)ref * REF_BYTES + bytes <= c.data_bytes;
}

// An array of cap records at ref stays inside the data region.
__device__ __forceinline__ bool array_ok(const Ctx& c, uint32_t ref, uint32_t cap) {
  return ref != NONE && (unsigned long long)ref * REF_BYTES + array_bytes(cap) <= c.data_bytes;
}

__device__ __forceinline__ uint32_t* grid_words(const Ctx& c, uint32_t ref) {
  return reinterpret_cast<uint32_t*>(ref_ptr(c, ref));
}

__device__ __forceinline__ uint32_t* dir_entries(const Ctx& c, uint32_t ref) {
  return reinterpret_cast<uint32_t*>(ref_ptr(c, ref));
}

// Coordinates relative to the root minimum; false when outside the root cube.
__device__ __forceinline__ bool rel_coords(const Ctx& c, int4 p, uint32_t& rx, uint32_t& ry,
                                           uint32_t& rz) {
  long long dx = (long long)p.x - c.rmin[0];
  long long dy = (long long)p.y - c.rmin[1];
  long long dz = (long long)p.z - c.rmin[2];
  long long side = 1ll << c.rlog2;
  rx = (uint32_t)dx;
  ry = (uint32_t)dy;
  rz = (uint32_t)dz;
  return dx >= 0 && dy >= 0 && dz >= 0 && dx < side && dy < side && dz < side;
}

// Octant of a point inside a node of side 2^L (L >= 1): bit L-1 per axis.
__device__ __forceinline__ uint32_t octant(uint32_t rx, uint32_t ry, uint32_t rz, uint32_t L) {
  uint32_t s = L - 1u;
  return ((rx >> s) & 1u) | (((ry >> s) & 1u) << 1) | (((rz >> s) & 1u) << 2);
}

// Cell of a point in the 2^G grid of a node of side 2^L: per axis
// ((p - min) << G) >> L, where p - min is the low L bits of the root-relative
// coordinate (Section 3.3).
__device__ __forceinline__ uint32_t cell_axis(uint32_t r, uint32_t L, uint32_t G) {
  uint32_t local = (L >= 32u) ? r : (r & ((1u << L) - 1u));
  return (L >= G) ? (local >> (L - G)) : (local << (G - L));
}

__device__ __forceinline__ uint32_t cell_index(uint32_t rx, uint32_t ry, uint32_t rz, uint32_t L,
                                               uint32_t G) {
  return cell_axis(rx, L, G) | (cell_axis(ry, L, G) << G) | (cell_axis(rz, L, G) << (2u * G));
}

// ------------------------------------------------------- node-table cache

// Shared-memory copy of child[] and gridref[] for nodes [0, NODE_CACHE).
struct NodeCache {
  uint32_t* child;
  uint32_t* grid;
  uint32_t n;  // cached nodes
};

// The cache of the first min(n_nodes, NODE_CACHE) nodes in `smem`.
__device__ __forceinline__ NodeCache node_cache_at(uint32_t* smem, uint32_t n_nodes) {
  NodeCache nc;
  nc.child = smem;
  nc.grid = smem + NODE_CACHE;
  nc.n = n_nodes < NODE_CACHE ? n_nodes : NODE_CACHE;
  return nc;
}

// The whole block copies nodes [lo, hi) (those below NODE_CACHE) into the
// cache. The caller synchronises the block before the cache is read.
__device__ __forceinline__ void node_cache_load(const Ctx& c, uint32_t* smem, uint32_t lo,
                                                uint32_t hi) {
  hi = hi < NODE_CACHE ? hi : NODE_CACHE;
  for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    smem[i] = c.child[i];
    smem[NODE_CACHE + i] = c.gridref[i];
  }
}

// The whole block brings the cache up to date after a decide round: the
// nodes of the split entries [s_lo, s_hi) became inner (child and grid set),
// the nodes [n_lo, n_hi) were created (leaves without a grid). Nothing else
// in the node table changes during an update. The caller synchronises.
__device__ __forceinline__ void node_cache_patch(const Ctx& c, uint32_t* smem, uint32_t s_lo,
                                                 uint32_t s_hi, uint32_t n_lo, uint32_t n_hi) {
  for (uint32_t e = s_lo + threadIdx.x; e < s_hi; e += blockDim.x) {
    const uint32_t id = c.splits[e].node;
    if (id < NODE_CACHE) {
      smem[id] = c.child[id];
      smem[NODE_CACHE + id] = c.gridref[id];
    }
  }
  node_cache_load(c, smem, n_lo, n_hi);
}

// The whole block empties the block tally cache (at the start of a phase,
// before a block barrier).
__device__ __forceinline__ void tally_init(uint32_t* smem) {
  for (uint32_t i = threadIdx.x; i < TALLY_SLOTS; i += blockDim.x) {
    smem[SMEM_TALLY + i] = NONE;
    smem[SMEM_TALLY + TALLY_SLOTS + i] = 0;
  }
}

// ------------------------------------------------------ block tally cache
//
// Per-update node counters (points counted into a leaf, new voxels of an
// inner node) are summed per block in shared memory first: a direct-mapped
// table of TALLY_SLOTS (node, count) pairs. A node whose slot holds another
// node goes to the global counter at once. Dense regions send thousands of
// warps to the same few counters; the cache turns their global atomics,
// which serialise at one L2 slice, into one per block and node.

__device__ __forceinline__ void tally_add(const Ctx& c, uint32_t* smem, uint32_t node,
                                          uint32_t k) {
#if SL_BLOCK_TALLY
  const uint32_t slot = (node * 0x9E3779B1u) >> (32u - TALLY_LOG2);
  uint32_t* tn = smem + SMEM_TALLY;
  const uint32_t old = tn[slot] == node ? node : atomicCAS(tn + slot, NONE, node);
  if (old == NONE || old == node) {
    atomicAdd(tn + TALLY_SLOTS + slot, k);
    return;
  }
#endif
  atomicAdd(&c.cnt[node], k);
}

// The whole block calls at the end of a phase: add the cached counts to the
// global counters.
__device__ __forceinline__ void tally_flush(const Ctx& c, uint32_t* smem) {
#if SL_BLOCK_TALLY
  __syncthreads();
  const uint32_t* tn = smem + SMEM_TALLY;
  for (uint32_t i = threadIdx.x; i < TALLY_SLOTS; i += blockDim.x) {
    const uint32_t node = tn[i], k = tn[TALLY_SLOTS + i];
    if (node != NONE && k) atomicAdd(&c.cnt[node], k);
  }
#endif
}

__device__ __forceinline__ uint32_t node_child(const Ctx& c, NodeCache nc, uint32_t id) {
  return id < nc.n ? nc.child[id] : c.child[id];
}

__device__ __forceinline__ uint32_t node_grid(const Ctx& c, NodeCache nc, uint32_t id) {
  return id < nc.n ? nc.grid[id] : c.gridref[id];
}

// -------------------------------------------------------- voxel claims

template <typename T>
__device__ __forceinline__ T vload(const T* p) {
  return *reinterpret_cast<const volatile T*>(p);
}

// Key and value of a claim-table slot in one 16-byte load. Within an update
// a slot's value only decreases once its key is set (the store phase empties
// the slots between updates), so a value read with the key bounds the current
// one from above.
__device__ __forceinline__ ulonglong2 slot_load(const HSlot* s) {
  ulonglong2 kv;
  asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];"
               : "=l"(kv.x), "=l"(kv.y)
               : "l"(s)
               : "memory");
  return kv;
}

// First claim-table slot of a key (node << 3G | cell). By default it is the
// top log2(slots) bits of key * 2^64 / phi (multiplicative hashing: one
// 64-bit multiply instead of the two of a 64-bit finalizer; where a key sits
// does not change which point wins). With SL_HASH_FIB=0 a 64-bit finalizer
// places every key at random, or, with SL_HASH_BUCKET, runs of
// 2^SL_HASH_BUCKET cells along x share one randomly placed bucket of slots,
// so that the neighbouring cells a warp claims fall on a few cache lines.
#ifndef SL_HASH_FIB
#define SL_HASH_FIB 1
#endif
__device__ __forceinline__ uint32_t claim_slot(const Ctx& c, unsigned long long key) {
#if SL_HASH_FIB
  const uint32_t bits = (uint32_t)__popc(c.hash_mask);  // the table has at least 2 slots
  return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64u - bits)) & c.hash_mask;
#elif SL_HASH_BUCKET
  constexpr uint32_t B = SL_HASH_BUCKET;
  return (((uint32_t)fmix64(key >> B) << B) | ((uint32_t)key & ((1u << B) - 1u))) & c.hash_mask;
#else
  return (uint32_t)fmix64(key) & c.hash_mask;
#endif
}

// Probes after the first for `key` (slot h held another key): returns true,
// with the slot in h, when this call put the key into the table (the cell is
// new in this update); a slot already holding the key is lowered to val if
// val is smaller.
__device__ bool hash_claim_rest(const Ctx& c, unsigned long long key, unsigned long long val,
                                uint32_t& h) {
  for (int probe = 1; probe < MAX_PROBES; ++probe) {
    h = (h + 1u) & c.hash_mask;
    HSlot* s = c.hash + h;
    const ulonglong2 kv = slot_load(s);
    unsigned long long k = kv.x;
    if (k == HASH_EMPTY) {
      k = atomicCAS(&s->key, HASH_EMPTY, key);
      if (k == HASH_EMPTY) {
        atomicMin(&s->val, val);
        return true;
      }
      if (k == key) atomicMin(&s->val, val);
      else continue;
      return false;
    }
    if (k == key) {
      if (kv.y > val) atomicMin(&s->val, val);
      return false;
    }
  }
  set_error(c, E_BACKLOG);
  return false;
}

// ------------------------------------------------ lane runs (warp groups)
//
// Lanes that hold the same value in a contiguous run of participating lanes
// form one group: one shuffle and two ballots, instead of a match over the
// whole warp. Equal values in separate runs form separate groups, which every
// caller tolerates (more groups, same result: counts and slot reservations
// add up, claims of one cell meet again in the table). The points a warp
// holds are neighbours in the stream, so equal nodes and cells mostly sit in
// runs.
struct LaneRun {
  bool head;       // this lane starts its run
  uint32_t first;  // the lane that starts this lane's run
  uint32_t end;    // one past the run's last lane
};

__device__ __forceinline__ unsigned lanes_upto(uint32_t lane) {
  return lane == 31u ? FULL_MASK : (2u << lane) - 1u;
}

// All 32 lanes call; lanes without `on` take part in no run.
template <typename T>
__device__ __forceinline__ LaneRun lane_run(bool on, T v) {
  const uint32_t lane = lane_id();
  const unsigned onm = __ballot_sync(FULL_MASK, on);
  const T prev = __shfl_up_sync(FULL_MASK, v, 1);
  const bool head = on && !(lane > 0u && ((onm >> (lane - 1u)) & 1u) && prev == v);
  const unsigned heads = __ballot_sync(FULL_MASK, head);
  LaneRun r;
  r.head = head;
  const unsigned below = heads & lanes_upto(lane);
  r.first = below ? 31u - (uint32_t)__clz(below) : lane;
  const unsigned breaks = (heads | ~onm) & ~lanes_upto(r.first);
  r.end = breaks ? (uint32_t)__ffs(breaks) - 1u : 32u;
  return r;
}

// All 32 lanes call: the minimum of v over this lane and the lanes after it
// in its run (at the run's first lane: the run's minimum).
__device__ __forceinline__ unsigned long long run_min(unsigned long long v, const LaneRun& r) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (uint32_t d = 1; d < 32u; d <<= 1) {
    const unsigned long long o = __shfl_down_sync(FULL_MASK, v, d);
    if (lane + d < r.end && o < v) v = o;
  }
  return v;
}

// Per-warp staging of the table slots of new cells (shared memory), flushed
// to the backlog with one atomic per flush.
struct WarpBuf {
  uint32_t* buf;   // WBUF entries of this warp
  uint32_t n;      // staged entries (the same value in every lane)
  uint32_t* smem;  // the block's dynamic shared memory (tally cache)
};

__device__ __forceinline__ WarpBuf warp_buf(uint32_t* smem) {
  WarpBuf wb;
  wb.buf = smem + SMEM_WBUF + (threadIdx.x / 32) * WBUF;
  wb.n = 0;
  wb.smem = smem;
  return wb;
}

// All 32 lanes call: append the staged slots to the backlog.
__device__ __forceinline__ void warp_flush(const Ctx& c, WarpBuf& wb) {
  if (wb.n == 0u) return;
  __syncwarp();
  uint32_t e0 = 0;
  if (lane_id() == 0) e0 = atomicAdd(&c.ctl->nkeys, wb.n);
  e0 = __shfl_sync(FULL_MASK, e0, 0);
  for (uint32_t k = lane_id(); k < wb.n; k += 32) {
    const uint32_t e = e0 + k;
    if (e < c.backlog_cap) c.keys[e] = wb.buf[k];
    else set_error(c, E_BACKLOG);
  }
  wb.n = 0;
  __syncwarp();
}

// Per-warp staging of mover-list entries (shared memory, after the node cache
// and the new-cell staging), appended to the list with one atomicAdd per
// flush: one reservation per MVBUF movers instead of one per warp unit.
struct MoverBuf {
  uint2* buf;
  uint32_t n;  // staged entries (the same value in every lane)
};

__device__ __forceinline__ MoverBuf mover_buf(uint32_t* smem) {
  MoverBuf mb;
  mb.buf = reinterpret_cast<uint2*>(smem + SMEM_MVBUF) + (threadIdx.x / 32) * MVBUF;
  mb.n = 0;
  return mb;
}

// All 32 lanes call.
__device__ __forceinline__ void mover_flush(const Ctx& c, MoverBuf& mb, int list) {
  if (mb.n == 0u) return;
  __syncwarp();
  uint32_t o0 = 0;
  if (lane_id() == 0) o0 = atomicAdd(&c.ctl->mv_count[list], mb.n);
  o0 = __shfl_sync(FULL_MASK, o0, 0);
  for (uint32_t k = lane_id(); k < mb.n; k += 32) {
    const uint64_t o = (uint64_t)o0 + k;
    if (o < c.mv_cap) c.mv[list][o] = mb.buf[k];
    else set_error(c, E_INTERNAL);
  }
  mb.n = 0;
  __syncwarp();
}

// All 32 lanes call: lanes with `moved` stage entry `ent`.
__device__ __forceinline__ void mover_add(const Ctx& c, MoverBuf& mb, int list, bool moved,
                                          uint2 ent) {
  const unsigned mm = __ballot_sync(FULL_MASK, moved);
  if (mm == 0u) return;
  const uint32_t k = (uint32_t)__popc(mm);
  if (mb.n + k > MVBUF) mover_flush(c, mb, list);
  if (moved) mb.buf[mb.n + __popc(mm & ((1u << lane_id()) - 1u))] = ent;
  mb.n += k;
}

// All 32 lanes call. Lanes with lead[j] offer val[j] for cell key[j] of node
// node[j] to the update's claim table; the lowest value wins. The first
// probes of all N items are issued together (their key loads, then their
// compare-and-swaps), so the items pay about two L2 round trips together. A
// key new in this update is staged for the backlog and counted towards its
// node's new voxels.
template <int N>
__device__ __forceinline__ void warp_claim_global(const Ctx& c, WarpBuf& wb, const bool (&lead)[N],
                                                  const unsigned long long (&key)[N],
                                                  const unsigned long long (&val)[N],
                                                  const uint32_t (&node)[N]) {
  const uint32_t lane = lane_id();
  bool cas[N], inst[N];
  uint32_t h[N];
  unsigned long long k0[N], v0[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    h[j] = claim_slot(c, key[j]);
    k0[j] = v0[j] = 0ull;
    if (lead[j]) {
      const ulonglong2 kv = slot_load(c.hash + h[j]);
      k0[j] = kv.x;
      v0[j] = kv.y;
    }
  }
#pragma unroll
  for (int j = 0; j < N; ++j) {
    cas[j] = lead[j] && k0[j] == HASH_EMPTY;
    if (cas[j]) {
      k0[j] = atomicCAS(&c.hash[h[j]].key, HASH_EMPTY, key[j]);
      v0[j] = HASH_EMPTY;
    }
  }
#pragma unroll
  for (int j = 0; j < N; ++j) {
    inst[j] = false;
    if (lead[j]) {
      if (cas[j] && k0[j] == HASH_EMPTY) {
        inst[j] = true;
        atomicMin(&c.hash[h[j]].val, val[j]);
      } else if (k0[j] == key[j]) {
        if (v0[j] > val[j]) atomicMin(&c.hash[h[j]].val, val[j]);
      } else {
        inst[j] = hash_claim_rest(c, key[j], val[j], h[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const unsigned mi = __ballot_sync(FULL_MASK, inst[j]);
    if (mi == 0u) continue;
    const uint32_t ni = (uint32_t)__popc(mi);
    if (wb.n + ni > WBUF) warp_flush(c, wb);
    const LaneRun r = lane_run(inst[j], node[j]);
    if (inst[j]) {
      wb.buf[wb.n + __popc(mi & ((1u << lane) - 1u))] = h[j];
      if (r.head) tally_add(c, wb.smem, node[j], r.end - lane);
    }
    wb.n += ni;
  }
}

// All 32 lanes call. For each of N items j, lanes with want[j] contend for
// the cell key[j] = (node[j], cell) with val = (gidx << 32 | rgba); the lowest
// gidx wins. Lanes with equal keys in a run are merged first and only the
// run's lowest gidx goes to the global table. SORTED: gidx grows with the
// lane, so a run's first lane holds its lowest gidx.
template <int N, bool SORTED>
__device__ __forceinline__ void warp_claim(const Ctx& c, WarpBuf& wb, const bool (&want)[N],
                                           const unsigned long long (&key)[N],
                                           const uint32_t (&gidx)[N], const uint32_t (&rgba)[N],
                                           const uint32_t (&node)[N]) {
  bool any = false;
#pragma unroll
  for (int j = 0; j < N; ++j) any = any || want[j];
  if (__ballot_sync(FULL_MASK, any) == 0u) return;
  bool lead[N];
  unsigned long long val[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    val[j] = ((unsigned long long)gidx[j] << 32) | rgba[j];
    const LaneRun r = lane_run(want[j], key[j]);
    if (!SORTED) val[j] = run_min(want[j] ? val[j] : ~0ull, r);
    lead[j] = want[j] && r.head;
  }
  warp_claim_global<N>(c, wb, lead, key, val, node);
}

// All 32 lanes call. Lanes with `valid` count one point into `leaf` (one
// addition per run of equal leaves; the slot is given at store).
__device__ __forceinline__ void warp_tally(const Ctx& c, uint32_t* smem, bool valid,
                                           uint32_t leaf) {
  const LaneRun r = lane_run(valid, leaf);
  if (valid && r.head) tally_add(c, smem, leaf, r.end - lane_id());
}

// The k-th 32-item unit of a phase that a warp handles: chunks of 2^chl
// consecutive units are dealt out to the warps in turn (chunk q to warp q mod
// nwarps), so that a warp's units are neighbours in the stream while the work
// stays spread over the grid.
__device__ __forceinline__ uint64_t warp_unit(uint64_t warp0, uint64_t nwarps, uint64_t k,
                                              uint32_t chl) {
  return ((warp0 + (k >> chl) * nwarps) << chl) + (k & ((1ull << chl) - 1ull));
}

// log2 of the count phase's chunk for `units` units: the largest power of two
// up to 2^SL_COUNT_CHUNK_MAX that still leaves SL_COUNT_CHUNK_DIV chunks per
// warp. Chunks of neighbouring points let a warp's descents and claims share
// nodes and cells (measured on the clustered stream: 15.1 against 18.7 ms of
// count phase with chunks of 4); batches too small to give every warp several
// chunks keep single units (1M-point batches slowed down with chunks of 8).
__device__ __forceinline__ uint32_t count_chunk_log2(uint64_t units, uint64_t nwarps) {
  uint32_t chl = 0;
  while (chl < SL_COUNT_CHUNK_MAX && units >= (nwarps * SL_COUNT_CHUNK_DIV) << (chl + 1)) ++chl;
  return chl;
}

// ------------------------------------------------------------ phase: count1

// Iteration 1 for the batch points [0, n): descend, claim, count. `smem`
// holds PHASE_SMEM_BYTES of dynamic shared memory; n_nodes is the node count.
__device__ void phase_count1(const Ctx& c, uint32_t* smem, const NodeCache nc, const int4* pts,
                             uint64_t n, unsigned long long base, uint64_t warp0,
                             uint64_t nwarps) {
  constexpr int U = COUNT_U, D = DESCENT_GROUP;
  tally_init(smem);
  __syncthreads();  // also publishes the caller's node-cache writes
  WarpBuf wb = warp_buf(smem);
  const uint32_t lane = lane_id();
  // each warp carries U units of 32 points (warp_unit k, k + 1, ...) at a
  // time so that their L2 round trips overlap; the next units' points are
  // loaded while the current ones descend
  const uint32_t chl = count_chunk_log2((n + 31) / 32, nwarps);
#if SL_COUNT_PREFETCH
  int4 pn[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const uint64_t i = warp_unit(warp0, nwarps, j, chl) * 32 + lane;
    pn[j] = i < n ? __ldcg(pts + i) : make_int4(0, 0, 0, 0);
  }
#endif
  for (uint64_t k0 = 0; warp_unit(warp0, nwarps, k0, chl) * 32 < n; k0 += U) {
    bool valid[U], walking[U];
    int4 p[U];
    uint32_t rx[U], ry[U], rz[U], node[U], L[U], gidx[U];
    uint64_t iu[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const uint64_t i = warp_unit(warp0, nwarps, k0 + j, chl) * 32 + lane;
      iu[j] = i;
      valid[j] = i < n;
#if SL_COUNT_PREFETCH
      p[j] = pn[j];
      const uint64_t inext = warp_unit(warp0, nwarps, k0 + j + U, chl) * 32 + lane;
      pn[j] = inext < n ? __ldcg(pts + inext) : make_int4(0, 0, 0, 0);
#else
      p[j] = valid[j] ? __ldcg(pts + i) : make_int4(0, 0, 0, 0);
#endif
      gidx[j] = (uint32_t)(base + i);
    }
#pragma unroll
    for (int j = 0; j < U; ++j) {
      rx[j] = ry[j] = rz[j] = 0;
      if (valid[j] && !rel_coords(c, p[j], rx[j], ry[j], rz[j])) {
        atomicOr(&c.ctl->reject, 1u);
        valid[j] = false;
      }
      node[j] = 0;
      L[j] = c.rlog2;
      walking[j] = valid[j];
    }
    for (;;) {
      bool any = false;
#pragma unroll
      for (int j = 0; j < U; ++j) any = any || walking[j];
      if (!__any_sync(FULL_MASK, any)) break;
      // Walk up to D levels through the node table first and issue their
      // grid-word loads together (their addresses do not depend on each
      // other), then test the bits and claim all of them at once.
      uint32_t gnode[U * D], gcell[U * D], gword[U * D];
      bool ginner[U * D];
#pragma unroll
      for (int j = 0; j < U; ++j) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const int s = j * D + k;
          ginner[s] = false;
          gnode[s] = node[j];
          gcell[s] = 0;
          gword[s] = 0;
          if (walking[j]) {
            const uint32_t ch = node_child(c, nc, node[j]);
            if (ch == NONE) {
              walking[j] = false;
            } else {
              const uint32_t gref = node_grid(c, nc, node[j]);
              const uint32_t cell = cell_index(rx[j], ry[j], rz[j], L[j], c.G);
              const uint32_t nxt = ch + octant(rx[j], ry[j], rz[j], L[j]);
              if (!ref_ok(c, gref, c.grid_bytes) || nxt >= c.max_nodes) {
                set_error(c, E_INTERNAL);
                walking[j] = false;
              } else {
                ginner[s] = true;
                gcell[s] = cell;
                gword[s] = grid_words(c, gref)[cell >> 5];
                node[j] = nxt;
                --L[j];
              }
            }
          }
        }
      }
      bool want[U * D];
      unsigned long long key[U * D];
      uint32_t gg[U * D], gc[U * D];
#pragma unroll
      for (int s = 0; s < U * D; ++s) {
        want[s] = ginner[s] && ((gword[s] >> (gcell[s] & 31u)) & 1u) == 0u;
        key[s] = ((unsigned long long)gnode[s] << (3u * c.G)) | gcell[s];
        gg[s] = gidx[s / D];
        gc[s] = (uint32_t)p[s / D].w;
      }
      warp_claim<U * D, true>(c, wb, want, key, gg, gc, gnode);
    }
#pragma unroll
    for (int j = 0; j < U; ++j) {
      warp_tally(c, smem, valid[j], node[j]);
      if (valid[j]) c.b_cur[iu[j]] = node[j];
    }
  }
  warp_flush(c, wb);
  tally_flush(c, smem);
}

// ----------------------------------------------------------- phase: advance

// U items per lane whose cursor node split in the previous round (moving[j]:
// the cursor cur[j], at level lvl[j], has children ch[j]) sample that node's
// grid (empty until store, so every point contends) and move one level down,
// counting into the child. cur[j] then holds the new cursor.
template <int U>
__device__ __forceinline__ void advance_items(const Ctx& c, WarpBuf& wb, const bool (&moving)[U],
                                              const int4 (&p)[U], const uint32_t (&gidx)[U],
                                              const uint32_t (&lvl)[U], const uint32_t (&ch)[U],
                                              uint32_t (&cur)[U]) {
  uint32_t nxt[U], rgba[U];
  unsigned long long key[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    uint32_t rx = 0, ry = 0, rz = 0, cell = 0;
    nxt[j] = cur[j];
    if (moving[j]) {
      rel_coords(c, p[j], rx, ry, rz);
      const uint32_t L = c.rlog2 - lvl[j];
      cell = cell_index(rx, ry, rz, L, c.G);
      nxt[j] = ch[j] + octant(rx, ry, rz, L);
    }
    key[j] = ((unsigned long long)cur[j] << (3u * c.G)) | cell;
    rgba[j] = (uint32_t)p[j].w;
  }
#if SL_ADVANCE_RUNS
  warp_claim<U, false>(c, wb, moving, key, gidx, rgba, cur);
#else
  // Every moving lane offers its own value: the movers of one warp rarely
  // share a cell (lane runs merged 1.4 % of these claims), so the run and
  // its 64-bit segmented minimum would cost more than they save. Lanes with
  // the same key meet in the table, where one compare-and-swap puts the key
  // in and every lower value lowers the slot.
  bool any = false;
#pragma unroll
  for (int j = 0; j < U; ++j) any = any || moving[j];
  if (__ballot_sync(FULL_MASK, any) != 0u) {
    unsigned long long val[U];
#pragma unroll
    for (int j = 0; j < U; ++j) val[j] = ((unsigned long long)gidx[j] << 32) | rgba[j];
    warp_claim_global<U>(c, wb, moving, key, val, cur);
  }
#endif
#pragma unroll
  for (int j = 0; j < U; ++j) {
    warp_tally(c, wb.smem, moving[j], nxt[j]);
    cur[j] = nxt[j];
  }
}

// A mover-list entry (8 bytes) is a point whose cursor moved in the last
// advance round: x = MV_SPILL | spill entry, or a batch point index; y = its
// cursor node (MV_NODE_BITS bits) | that node's level << MV_NODE_BITS.
constexpr uint32_t MV_SPILL = 1u << 31;
constexpr uint32_t MV_NODE_BITS = 27;  // node ids below 2^27 (the node table limit)
constexpr uint32_t MV_NODE_MASK = (1u << MV_NODE_BITS) - 1u;

// Advance round r of the expansion (r >= 2 counts decide rounds): zero the
// grids of the splits [s_lo, s_hi) of the previous decide, then move every
// point whose cursor node split there one level down (advance_items), and
// list the points that moved in mover list out_list.
//
// Only nodes created in the previous round can split in a later one (every
// leaf that existed before the update was decided in the first round), so
// only points that moved in the previous round can move again: the first
// round (in_list < 0) scans every batch cursor and every point of the spill
// tasks [0, t_hi) (all created by the first decide; their points still sit
// in the split leaf's chunks and are copied to the spill records here), later
// rounds only the n_in entries of mover list in_list, which carry cursor and
// level. Points are cut into 32-item warp units (a unit of a task never
// crosses into the next task).
__device__ void phase_advance(const Ctx& c, uint32_t* smem, const NodeCache nc, const int4* pts,
                              uint64_t n, unsigned long long base, uint32_t t_hi, uint32_t s_lo,
                              uint32_t s_hi, int in_list, uint32_t n_in, int out_list,
                              uint64_t warp0, uint64_t nwarps) {
  tally_init(smem);
  __syncthreads();  // also publishes the caller's node-cache writes
  WarpBuf wb = warp_buf(smem);
  MoverBuf mb = mover_buf(smem);
  const uint32_t lane = lane_id();
  const uint32_t zpg = (c.grid_bytes + ZERO_UNIT - 1) / ZERO_UNIT;  // zero units per grid
  const uint64_t uz = (uint64_t)(s_hi - s_lo) * zpg;
  for (uint64_t w = warp0; w < uz; w += nwarps) {
    const uint32_t id = c.splits[s_lo + (uint32_t)(w / zpg)].node;
    const uint32_t gref = id < c.max_nodes ? c.gridref[id] : NONE;
    if (!ref_ok(c, gref, c.grid_bytes)) {
      if (lane == 0) set_error(c, E_INTERNAL);
      continue;
    }
    const uint32_t lo = (uint32_t)(w % zpg) * ZERO_UNIT;
    const uint32_t hi = min(lo + ZERO_UNIT, c.grid_bytes);
    int4* g = reinterpret_cast<int4*>(grid_words(c, gref));
    for (uint32_t b = lo / 16 + lane; b < hi / 16; b += 32) g[b] = make_int4(0, 0, 0, 0);
  }
  const uint32_t parts = (c.C + 31) / 32;  // units per task
  const bool first = in_list < 0;
  const uint64_t ub = first ? (n + 31) / 32 : 0;
  const uint64_t units = first ? ub + (uint64_t)t_hi * parts : ((uint64_t)n_in + 31) / 32;
  const uint2* in = first ? nullptr : c.mv[in_list];
  constexpr int AU = ADVANCE_U;
  // each warp carries AU units (w, w + nwarps, ...) at a time so that their
  // L2 round trips overlap (chunks of neighbouring units measured slower
  // here: the movers of dense regions then load few warps)
  for (uint64_t k0 = 0; warp_unit(warp0, nwarps, k0, 0) < units; k0 += AU) {
    bool valid[AU], spill[AU], have_p[AU], mv[AU];
    uint32_t idx[AU], cur[AU], lvl[AU], g[AU], ch[AU];  // idx: batch point index or spill entry
    int4 p[AU];
#pragma unroll
    for (int j = 0; j < AU; ++j) {
      const uint64_t w = warp_unit(warp0, nwarps, k0 + j, 0);
      valid[j] = spill[j] = have_p[j] = false;
      idx[j] = cur[j] = lvl[j] = g[j] = 0;
      p[j] = make_int4(0, 0, 0, 0);
      if (w >= units) {
        // past the end: nothing
      } else if (first && w < ub) {
        const uint64_t i = w * 32 + lane;
        valid[j] = i < n;
        idx[j] = (uint32_t)i;
        cur[j] = valid[j] ? c.b_cur[i] : 0u;
      } else if (first) {
        const uint64_t u = w - ub;
        const uint32_t t = (uint32_t)(u / parts), q = (uint32_t)(u % parts) * 32u + lane;
        const SpillTask tk = c.tasks[t];
        const bool task_ok = ref_ok(c, tk.ref, c.chunk_bytes) && tk.n <= c.C &&
                             (unsigned long long)tk.dst + tk.n <= c.spill_cap;
        if (!task_ok && lane == 0) set_error(c, E_INTERNAL);
        valid[j] = task_ok && q < tk.n;
        spill[j] = true;
        idx[j] = tk.dst + q;
        cur[j] = tk.node;
        if (valid[j]) {
          // the point leaves its chunk (which returns to the pool at store)
          p[j] = chunk_recs(c, tk.ref)[q];
          g[j] = chunk_aux(c, tk.ref)[q];
          c.sp_rec[idx[j]] = p[j];
          c.sp_gidx[idx[j]] = g[j];
          have_p[j] = true;
        }
      } else {
        const uint64_t k = w * 32 + lane;
        if (k < n_in) {
          const uint2 ent = in[k];
          valid[j] = true;
          spill[j] = (ent.x & MV_SPILL) != 0u;
          idx[j] = ent.x & ~MV_SPILL;
          cur[j] = ent.y & MV_NODE_MASK;
          lvl[j] = ent.y >> MV_NODE_BITS;
          if (spill[j] ? idx[j] >= c.spill_cap : idx[j] >= n) {
            set_error(c, E_INTERNAL);
            valid[j] = false;
          }
        }
      }
      if (valid[j] && cur[j] >= c.max_nodes) {
        set_error(c, E_INTERNAL);
        valid[j] = false;
      }
    }
#pragma unroll
    for (int j = 0; j < AU; ++j) {
      // read a point only when its cursor node split (it moves)
      ch[j] = valid[j] ? node_child(c, nc, cur[j]) : NONE;
      mv[j] = ch[j] != NONE && ch[j] + 8u <= c.max_nodes;
      if (mv[j]) {
        if (first) lvl[j] = c.meta[cur[j]].level;
        if (!have_p[j]) {
          if (spill[j]) {
            p[j] = c.sp_rec[idx[j]];
            g[j] = c.sp_gidx[idx[j]];
          } else {
            p[j] = __ldcg(pts + idx[j]);
            g[j] = (uint32_t)(base + idx[j]);
          }
        }
      }
    }
    advance_items<AU>(c, wb, mv, p, g, lvl, ch, cur);
#pragma unroll
    for (int j = 0; j < AU; ++j) {
      if (mv[j]) {
        if (spill[j]) c.sp_cur[idx[j]] = cur[j];
        else c.b_cur[idx[j]] = cur[j];
      }
      mover_add(c, mb, out_list, mv[j],
                make_uint2(spill[j] ? (idx[j] | MV_SPILL) : idx[j],
                           cur[j] | ((lvl[j] + 1u) << MV_NODE_BITS)));
    }
  }
  warp_flush(c, wb);
  mover_flush(c, mb, out_list);
  tally_flush(c, smem);
}

// ------------------------------------------------------------ phase: decide

// Take up to k refs from the pool; returns how many and the first index.
// One atomicSub per allocation: the top may go below zero while the pool is
// empty; store and end clamp it at zero.
__device__ __forceinline__ uint32_t pool_take(const Ctx& c, uint32_t k, int* first) {
  const int t = atomicSub(&c.ctl->pool_top, (int)k);
  if (t <= 0) return 0;
  const int take = t < (int)k ? t : (int)k;
  *first = t - take;
  return (uint32_t)take;
}

// Section 5.3, all 32 lanes of a warp call with the same arguments: give
// node `id` ceil(total / C) chunks, pool first, then the bump allocator; link
// them, note them in a leaf's directory and record the store map for this
// update. Lane 0 takes the allocator atomics; the lanes link the new chunks
// in parallel (chunk q's successor is chunk q + 1 of the same allocation).
__device__ void alloc_chunks(const Ctx& c, uint32_t id, uint32_t total, bool leaf) {
  const uint32_t lane = lane_id();
  NodeMeta& m = c.meta[id];
  const uint32_t have = m.n_chunks, tail = m.tail, mdir = m.dir;
  const uint32_t need = (uint32_t)(((unsigned long long)total + c.C - 1) / c.C);
  const uint32_t k = need > have ? need - have : 0u;
  uint32_t seq = 0, from_pool = 0, ok = 1;
  int pfirst = 0;
  unsigned long long off = 0;
  if (lane == 0 && k) {
    seq = atomicAdd(&c.ctl->alloc_seq, k);
    if ((unsigned long long)seq + k > c.max_chunks) {
      set_error(c, E_ALLOC_REFS);
      ok = 0;
    } else {
      from_pool = pool_take(c, k, &pfirst);
      const uint32_t rest = k - from_pool;
      if (rest) {
        off = atomicAdd(&c.ctl->bump, (unsigned long long)rest * c.chunk_bytes);
        if (off + (unsigned long long)rest * c.chunk_bytes > c.data_bytes) {
          set_error(c, E_ARENA);
          ok = 0;
        } else {
          atomicAdd(&c.ctl->chunks_bumped, (unsigned long long)rest);
        }
      }
    }
  }
  seq = __shfl_sync(FULL_MASK, seq, 0);
  from_pool = __shfl_sync(FULL_MASK, from_pool, 0);
  pfirst = __shfl_sync(FULL_MASK, pfirst, 0);
  off = __shfl_sync(FULL_MASK, off, 0);
  ok = __shfl_sync(FULL_MASK, ok, 0);
  if (lane == 0) {
    m.st_nch = have;
    m.st_tail = tail;
    m.st_seq = k ? seq : 0u;
    m.st_base = c.num[id];
    m.touched = (uint32_t)c.ctl->st_batches + 1u;
    c.scur[id] = 0;
  }
  if (!k || !ok) return;
  uint32_t* dir = (leaf && ref_ok(c, mdir, c.dir_bytes)) ? dir_entries(c, mdir) : nullptr;
  const uint32_t bump_ref = (uint32_t)(off / REF_BYTES);
  auto ref_of = [&](uint32_t q) -> uint32_t {
    return q < from_pool ? c.pool[pfirst + (int)q] : bump_ref + (q - from_pool) * c.chunk_units;
  };
  for (uint32_t q = lane; q < k; q += 32) {
    const uint32_t ref = ref_of(q);
    const uint32_t nxt = q + 1u < k ? ref_of(q + 1u) : NONE;
    c.alloc_refs[seq + q] = ref;
    *chunk_next(c, ref) = nxt;
    if (dir && have + q < c.dir_cap) dir[have + q] = ref;
    if (q == 0) {
      if (tail == NONE) m.head = ref;
      else *chunk_next(c, tail) = ref;
    }
    if (q + 1u == k) m.tail = ref;
  }
  if (lane == 0) m.n_chunks = need;
}

// Section 5.1, all 32 lanes of a warp call: split leaf `id` whose count
// exceeds T: 8 children (with chunk directories), a grid for the node (zeroed
// in the next round), and one spill task per chunk of its stored points;
// those chunks return to the pool at the end of the update.
__device__ void split_leaf(const Ctx& c, uint32_t id) {
  const uint32_t lane = lane_id();
  NodeMeta& m = c.meta[id];
  const uint32_t stored = c.num[id], nch = m.n_chunks, mdir = m.dir;
  uint32_t c0 = 0, s0 = 0, t0 = 0, e = 0, ok = 1;
  unsigned long long dbase = 0, g = 0;
  if (lane == 0) {
    c0 = atomicAdd(&c.ctl->n_nodes, 8u);
    dbase = atomicAdd(&c.ctl->bump, 8ull * c.dir_bytes + c.grid_bytes);
    g = dbase + 8ull * c.dir_bytes;
    s0 = atomicAdd(&c.ctl->spill_count, stored);
    t0 = atomicAdd(&c.ctl->ntasks, nch);
    e = atomicAdd(&c.ctl->split_count, 1u);
    if ((unsigned long long)c0 + 8 > c.max_nodes || e >= c.max_splits) {
      set_error(c, E_NODES);
      ok = 0;
    } else if (g + c.grid_bytes > c.data_bytes) {
      set_error(c, E_ARENA);
      ok = 0;
    } else if ((unsigned long long)s0 + stored > c.spill_cap) {
      set_error(c, E_SPILL);
      ok = 0;
    } else if ((unsigned long long)t0 + nch > c.max_chunks || nch > c.dir_cap ||
               (nch && !ref_ok(c, mdir, c.dir_bytes))) {
      set_error(c, E_INTERNAL);
      ok = 0;
    }
  }
  if (!__shfl_sync(FULL_MASK, ok, 0)) return;
  c0 = __shfl_sync(FULL_MASK, c0, 0);
  s0 = __shfl_sync(FULL_MASK, s0, 0);
  t0 = __shfl_sync(FULL_MASK, t0, 0);
  e = __shfl_sync(FULL_MASK, e, 0);
  dbase = __shfl_sync(FULL_MASK, dbase, 0);
  g = __shfl_sync(FULL_MASK, g, 0);
  if (lane < 8) {
    const uint32_t k = lane;
    const uint32_t Lc = c.rlog2 - m.level - 1u;  // children's log2 size
    NodeMeta cm;
    cm.min[0] = m.min[0] + (int32_t)((k & 1u) << Lc);
    cm.min[1] = m.min[1] + (int32_t)(((k >> 1) & 1u) << Lc);
    cm.min[2] = m.min[2] + (int32_t)(((k >> 2) & 1u) << Lc);
    cm.level = m.level + 1u;
    cm.n_chunks = 0;
    cm.head = cm.tail = NONE;
    cm.dir = (uint32_t)((dbase + (unsigned long long)k * c.dir_bytes) / REF_BYTES);
    cm.st_nch = 0;
    cm.st_tail = NONE;
    cm.st_seq = 0;
    cm.st_base = 0;
    cm.touched = 0;
    cm.compact = 0;
    cm.pad[0] = cm.pad[1] = 0;
    c.meta[c0 + k] = cm;
    c.child[c0 + k] = NONE;
    c.gridref[c0 + k] = NONE;
    c.cnt[c0 + k] = 0;
    c.num[c0 + k] = 0;
  }
  const uint32_t* dir = nch ? dir_entries(c, mdir) : nullptr;
  for (uint32_t j = lane; j < nch; j += 32) {
    const uint32_t ref = dir[j];
    const uint32_t first = j * c.C;
    c.tasks[t0 + j] = SpillTask{ref, id, s0 + first, min(c.C, stored - first)};
    c.pending[t0 + j] = ref;
  }
  __syncwarp();  // every lane has read m before lane 0 rewrites it
  if (lane == 0) {
    c.splits[e] = SplitEntry{id, s0};
    c.gridref[id] = (uint32_t)(g / REF_BYTES);
    m.n_chunks = 0;
    m.head = m.tail = NONE;
    m.dir = NONE;
    c.num[id] = 0;
    c.cnt[id] = 0;
    c.child[id] = c0;
  }
}

// All 32 lanes of a warp call: a compacted node (simlod_compact) that receives
// records again goes back to a chunk list first: ceil(n / C) chunks, pool
// first then bump, linked and noted in the leaf's directory, with its n
// records copied in. The array's space is not reused.
__device__ void restore_chunks(const Ctx& c, uint32_t id, bool leaf) {
  NodeMeta& m = c.meta[id];
  const uint32_t n = c.num[id], arr = m.head;
  if (!array_ok(c, arr, n)) {
    if (lane_id() == 0) set_error(c, E_INTERNAL);
    return;
  }
  __syncwarp();
  if (lane_id() == 0) {
    m.n_chunks = 0;
    m.head = m.tail = NONE;
  }
  __syncwarp();
  alloc_chunks(c, id, n, leaf);
  __syncwarp();
  const uint32_t seq = m.st_seq, nch = m.n_chunks;
  if (nch != (n + c.C - 1) / c.C || (unsigned long long)seq + nch > c.max_chunks) {
    if (lane_id() == 0) set_error(c, E_INTERNAL);  // the allocation failed (error already set)
    return;
  }
  const int4* src = array_recs(c, arr);
  const uint32_t* sax = array_aux(c, arr, n);
  for (uint32_t i = lane_id(); i < n; i += 32u) {
    const uint32_t ref = c.alloc_refs[seq + i / c.C], q = i % c.C;
    chunk_recs(c, ref)[q] = src[i];
    chunk_aux(c, ref)[q] = sax[i];
  }
  __syncwarp();
  if (lane_id() == 0) {
    m.compact = 0;
    atomicAdd(&c.ctl->st_decompacted, 1ull);
    atomicAdd(&c.ctl->compact_now, ~0ull);  // minus one
    atomicAdd(&c.ctl->compact_chunks_now, 0ull - nch);
  }
  __syncwarp();
}

// All 32 lanes of a warp call for one candidate node.
__device__ __forceinline__ void decide_node(const Ctx& c, uint32_t id) {
  const uint32_t k = c.cnt[id];
  if (k == 0) return;
  if (c.meta[id].compact) restore_chunks(c, id, c.child[id] == NONE);
  const uint32_t num = c.num[id];
  if (c.child[id] == NONE) {
    const uint32_t total = num + k;
    const uint32_t L = c.rlog2 - c.meta[id].level;
    if (total > c.T && L > 0) {
      split_leaf(c, id);
      return;
    }
    alloc_chunks(c, id, total, true);
    __syncwarp();
    if (lane_id() == 0) c.num[id] = total;
  } else {
    alloc_chunks(c, id, num + k, false);
    __syncwarp();
    if (lane_id() == 0) c.num[id] = num + k;
  }
  if (lane_id() == 0) c.cnt[id] = 0;
}

// Candidates, one warp each: the nodes split in the previous round (their
// voxels are now all claimed) and the node id range [n_lo, n_hi).
// zero_list >= 0: also empty that mover list (the next advance round fills
// it; the round before last was its reader).
__device__ void phase_decide(const Ctx& c, uint32_t s_lo, uint32_t s_hi, uint32_t n_lo,
                             uint32_t n_hi, int zero_list, uint64_t warp0, uint64_t nwarps) {
  const uint64_t ns = s_hi - s_lo, nn = n_hi - n_lo;
  if (zero_list >= 0 && warp0 == 0 && lane_id() == 0) c.ctl->mv_count[zero_list] = 0;
  for (uint64_t w = warp0; w < ns + nn; w += nwarps) {
    const uint32_t id = w < ns ? c.splits[s_lo + w].node : (uint32_t)(n_lo + (w - ns));
    decide_node(c, id);
  }
}

// The batch was rejected (a point outside the root cube): undo the counts
// and claims of its count round, nodes [0, n_nodes), so nothing changed.
__device__ void phase_rollback(const Ctx& c, uint32_t n_nodes, uint64_t t0, uint64_t nthreads) {
  for (uint64_t t = t0; t < n_nodes; t += nthreads) c.cnt[t] = 0;
  const uint32_t nk = min(*reinterpret_cast<volatile unsigned int*>(&c.ctl->nkeys), c.backlog_cap);
  for (uint64_t t = t0; t < nk; t += nthreads) {
    HSlot* s = c.hash + c.keys[t];
    s->key = HASH_EMPTY;
    s->val = HASH_EMPTY;
  }
}

// -------------------------------------------------------------- phase: store

// All 32 lanes call with U items each (warp-uniform). Every valid item gets
// the next free slot of its node in this update: the node's records before
// the update (st_base) + a running per-node cursor, one atomicAdd per
// distinct node per warp and item index; the store map then turns the slot
// into (chunk ref, index in chunk). The map (st_nch, st_tail, st_seq,
// st_base) is one 16-byte load per item, issued with the cursor atomics.
// Invalid items, and items whose slot has no chunk, get ref NONE (the latter
// raise E_INTERNAL).
template <int U>
__device__ __forceinline__ void warp_place(const Ctx& c, const bool (&valid)[U],
                                           const uint32_t (&node)[U], uint32_t (&ref)[U],
                                           uint32_t (&q)[U]) {
  const uint32_t lane = lane_id();
  uint4 map[U];
  uint32_t rank[U], cur[U];
  int leader[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    map[j] = valid[j] ? *reinterpret_cast<const uint4*>(&c.meta[node[j]].st_nch)
                      : make_uint4(0, NONE, 0, 0);
  }
  // exact groups here (a match over the warp): the cursor atomics return a
  // value, and in dense regions the lanes of one node are not contiguous, so
  // one reservation per lane run would queue many more of them on one counter
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const unsigned m = __ballot_sync(FULL_MASK, valid[j]);
    leader[j] = 0;
    rank[j] = 0;
    cur[j] = 0;
    if (valid[j]) {
      const unsigned grp = __match_any_sync(m, node[j]);
      leader[j] = __ffs(grp) - 1;
      rank[j] = __popc(grp & ((1u << lane) - 1u));
      if ((int)lane == leader[j]) cur[j] = atomicAdd(&c.scur[node[j]], (uint32_t)__popc(grp));
    }
  }
#pragma unroll
  for (int j = 0; j < U; ++j) {
    cur[j] = __shfl_sync(FULL_MASK, cur[j], leader[j]);
    ref[j] = NONE;
    q[j] = 0;
    if (valid[j]) {
      const uint32_t slot = map[j].w + cur[j] + rank[j];
      const uint32_t k = slot / c.C;
      q[j] = slot - k * c.C;
      if (k + 1u == map[j].x) {
        ref[j] = map[j].y;
      } else if (k >= map[j].x) {
        const unsigned long long at = (unsigned long long)map[j].z + (k - map[j].x);
        if (at < c.max_chunks) ref[j] = c.alloc_refs[at];
      }
    }
  }
#pragma unroll
  for (int j = 0; j < U; ++j) {
    if (valid[j] && !ref_ok(c, ref[j], c.chunk_bytes)) {
      set_error(c, E_INTERNAL);
      ref[j] = NONE;
    }
  }
}

// Block form of warp_place (all threads of the block call; loops are
// block-uniform): items of the whole block reserve their slots per node in a
// shared-memory table first (256 slots, direct-mapped, in the tally region),
// then one thread per table entry takes the node's range with one global
// atomicAdd. In dense regions many warps of a block store into the same few
// nodes; their returning atomics on one counter would queue at one L2 slice.
// Items whose table slot holds another node take the warp path.
constexpr uint32_t PLACE_SLOTS = 256;

template <int U>
__device__ __forceinline__ void block_place(const Ctx& c, uint32_t* smem, const bool (&valid)[U],
                                            const uint32_t (&node)[U], uint32_t (&ref)[U],
                                            uint32_t (&q)[U]) {
  const uint32_t lane = lane_id();
  uint32_t* tn = smem + SMEM_TALLY;  // node of each table slot
  uint32_t* tc = tn + PLACE_SLOTS;   // items of the block for it
  uint32_t* tb = tc + PLACE_SLOTS;   // the range it got
  uint4 map[U];
  uint32_t sl[U], rank[U], cur[U];
  int leader[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    map[j] = valid[j] ? *reinterpret_cast<const uint4*>(&c.meta[node[j]].st_nch)
                      : make_uint4(0, NONE, 0, 0);
    sl[j] = NONE;
    rank[j] = 0;
    if (valid[j]) {
      const uint32_t h = (node[j] * 0x9E3779B1u) >> 24;  // PLACE_SLOTS = 2^8
      const uint32_t old = tn[h] == node[j] ? node[j] : atomicCAS(tn + h, NONE, node[j]);
      if (old == NONE || old == node[j]) {
        sl[j] = h;
        rank[j] = atomicAdd(tc + h, 1u);
      }
    }
  }
  // items without a table slot: exact groups of the warp, one global atomic each
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const bool fb = valid[j] && sl[j] == NONE;
    const unsigned m = __ballot_sync(FULL_MASK, fb);
    leader[j] = 0;
    cur[j] = 0;
    if (fb) {
      const unsigned grp = __match_any_sync(m, node[j]);
      leader[j] = __ffs(grp) - 1;
      rank[j] = __popc(grp & ((1u << lane) - 1u));
      if ((int)lane == leader[j]) cur[j] = atomicAdd(&c.scur[node[j]], (uint32_t)__popc(grp));
    }
    cur[j] = __shfl_sync(FULL_MASK, cur[j], leader[j]);
  }
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < PLACE_SLOTS; t += blockDim.x) {
    const uint32_t nd = tn[t];
    if (nd != NONE) tb[t] = atomicAdd(&c.scur[nd], tc[t]);
    tn[t] = NONE;  // every thread has passed its table lookups (barrier above)
    tc[t] = 0;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < U; ++j) {
    ref[j] = NONE;
    q[j] = 0;
    if (valid[j]) {
      const uint32_t slot = map[j].w + (sl[j] != NONE ? tb[sl[j]] : cur[j]) + rank[j];
      const uint32_t k = slot / c.C;
      q[j] = slot - k * c.C;
      if (k + 1u == map[j].x) {
        ref[j] = map[j].y;
      } else if (k >= map[j].x) {
        const unsigned long long at = (unsigned long long)map[j].z + (k - map[j].x);
        if (at < c.max_chunks) ref[j] = c.alloc_refs[at];
      }
      if (!ref_ok(c, ref[j], c.chunk_bytes)) {
        set_error(c, E_INTERNAL);
        ref[j] = NONE;
      }
    }
  }
}

// All threads of the block call: an empty block placement table.
__device__ __forceinline__ void block_place_init(uint32_t* smem) {
  for (uint32_t t = threadIdx.x; t < PLACE_SLOTS; t += blockDim.x) {
    smem[SMEM_TALLY + t] = NONE;
    smem[SMEM_TALLY + PLACE_SLOTS + t] = 0;
  }
  __syncthreads();
}

__device__ __forceinline__ void put_rec(const Ctx& c, uint32_t ref, uint32_t q, int4 rec,
                                        uint32_t aux) {
  if (ref == NONE) return;
  chunk_recs(c, ref)[q] = rec;
  chunk_aux(c, ref)[q] = aux;
}

constexpr int STORE_U = SL_STORE_UNROLL;
static_assert(3 * 256 <= 2 * TALLY_SLOTS, "the block placement table fits the tally region");

// Store the batch points, the n_spill re-inserted points (from the spill
// records) and the n_keys new voxels, each at the next free slot of its node;
// hand the n_tasks chunks of split leaves (one per task) to the pool above
// pool_top (the caller then raises pool_top). Loops are warp-uniform so that the
// lanes of a warp share one slot reservation per node; each lane carries
// STORE_U items at a time so that their L2 round trips overlap.
__device__ void phase_store(const Ctx& c, uint32_t* smem, const int4* pts, uint64_t n,
                            unsigned long long base, uint32_t n_spill, uint32_t n_tasks,
                            uint32_t n_keys, int pool_top, uint64_t t0, uint64_t nthreads) {
  constexpr int U = STORE_U;
  const uint32_t lane = lane_id();
  // block-uniform loops: item j of thread t in round b is b + j * nthreads + t
  const uint64_t blk = t0 - threadIdx.x, stride = nthreads;
  const uint64_t me = threadIdx.x;
  auto place = [&](const bool (&valid)[U], const uint32_t (&node)[U], uint32_t (&ref)[U],
                   uint32_t (&q)[U]) {
#if SL_STORE_BLOCK
    if (smem) {
      block_place<U>(c, smem, valid, node, ref, q);
      return;
    }
#endif
    warp_place<U>(c, valid, node, ref, q);
  };
#if SL_STORE_BLOCK
  if (smem) block_place_init(smem);
#endif
#if SL_STORE_PREFETCH
  // the next round's cursors and points load while this round is placed
  uint32_t node_n[U];
  int4 p_n[U];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const uint64_t i = blk + j * stride + me;
    node_n[j] = i < n ? c.b_cur[i] : 0u;
    p_n[j] = i < n ? __ldcg(pts + i) : make_int4(0, 0, 0, 0);
  }
#endif
  for (uint64_t b0 = blk; b0 < n; b0 += U * stride) {
    bool valid[U];
    uint32_t node[U], ref[U], q[U];
    int4 p[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const uint64_t i = b0 + j * stride + me;
      valid[j] = i < n;
#if SL_STORE_PREFETCH
      node[j] = node_n[j];
      p[j] = p_n[j];
      const uint64_t inext = i + (uint64_t)U * stride;
      node_n[j] = inext < n ? c.b_cur[inext] : 0u;
      p_n[j] = inext < n ? __ldcg(pts + inext) : make_int4(0, 0, 0, 0);
#else
      node[j] = valid[j] ? c.b_cur[i] : 0u;
      p[j] = valid[j] ? __ldcg(pts + i) : make_int4(0, 0, 0, 0);
#endif
      if (valid[j] && node[j] >= c.max_nodes) {
        set_error(c, E_INTERNAL);
        valid[j] = false;
      }
    }
    place(valid, node, ref, q);
#pragma unroll
    for (int j = 0; j < U; ++j) put_rec(c, ref[j], q[j], p[j], (uint32_t)(base + b0 + j * stride + me));
  }
  for (uint64_t b0 = blk; b0 < n_spill; b0 += U * stride) {
    bool valid[U];
    uint32_t node[U], ref[U], q[U], g[U];
    int4 r[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const uint64_t e = b0 + j * stride + me;
      valid[j] = e < n_spill;
      node[j] = valid[j] ? c.sp_cur[e] : 0u;
      r[j] = valid[j] ? c.sp_rec[e] : make_int4(0, 0, 0, 0);
      g[j] = valid[j] ? c.sp_gidx[e] : 0u;
      if (valid[j] && node[j] >= c.max_nodes) {
        set_error(c, E_INTERNAL);
        valid[j] = false;
      }
    }
    place(valid, node, ref, q);
#pragma unroll
    for (int j = 0; j < U; ++j) put_rec(c, ref[j], q[j], r[j], g[j]);
  }
  const uint32_t G = c.G, cmask = (1u << (3u * G)) - 1u, amask = (1u << G) - 1u;
  for (uint64_t b0 = blk; b0 < n_keys; b0 += U * stride) {
    bool valid[U];
    uint32_t node[U], ref[U], q[U], cell[U], gref[U], rgba[U];
    HSlot* sl[U];
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const uint64_t e = b0 + j * stride + me;
      valid[j] = e < n_keys;
      sl[j] = valid[j] ? c.hash + c.keys[e] : nullptr;
    }
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const ulonglong2 kv = valid[j] ? *reinterpret_cast<const ulonglong2*>(sl[j])
                                     : make_ulonglong2(0ull, 0ull);
      rgba[j] = (uint32_t)kv.y;
      node[j] = (uint32_t)(kv.x >> (3u * G));
      cell[j] = (uint32_t)kv.x & cmask;
    }
    int4 nm[U];  // the node's min corner and level (voxel centre), loaded with its grid ref
#pragma unroll
    for (int j = 0; j < U; ++j) {
      const bool in = valid[j] && node[j] < c.max_nodes;
      gref[j] = in ? c.gridref[node[j]] : NONE;
      nm[j] = in ? *reinterpret_cast<const int4*>(&c.meta[node[j]].min[0]) : make_int4(0, 0, 0, 0);
      const bool ok = valid[j] && ref_ok(c, gref[j], c.grid_bytes);
      if (valid[j] && !ok) set_error(c, E_INTERNAL);
      valid[j] = ok;
    }
    place(valid, node, ref, q);
#pragma unroll
    for (int j = 0; j < U; ++j) {
      if (!valid[j]) continue;
      const uint32_t L = c.rlog2 - (uint32_t)nm[j].w;
      const uint32_t cx = cell[j] & amask, cy = (cell[j] >> G) & amask, cz = cell[j] >> (2u * G);
      // Section 3.4: the voxel is a point at the (floor of the) cell centre
      int4 v;
      v.x = nm[j].x + (int32_t)(((2ull * cx + 1ull) << L) >> (G + 1u));
      v.y = nm[j].y + (int32_t)(((2ull * cy + 1ull) << L) >> (G + 1u));
      v.z = nm[j].z + (int32_t)(((2ull * cz + 1ull) << L) >> (G + 1u));
      v.w = (int32_t)rgba[j];
      put_rec(c, ref[j], q[j], v, cell[j]);
      atomicOr(grid_words(c, gref[j]) + (cell[j] >> 5), 1u << (cell[j] & 31u));
      sl[j]->key = HASH_EMPTY;
      sl[j]->val = HASH_EMPTY;
    }
  }
  (void)lane;
  const int top = pool_top > 0 ? pool_top : 0;
  if ((unsigned long long)top + n_tasks > c.max_chunks) {
    if (t0 == 0) set_error(c, E_POOL);
    return;
  }
  for (uint64_t q = t0; q < n_tasks; q += nthreads) c.pool[top + q] = c.pending[q];
}

// One thread: close an applied update (advance gidx, return the freed
// chunks to the pool, fold the update into the stats, clear the per-update
// counters).
__device__ void phase_end(const Ctx& c, uint64_t n, uint32_t iters) {
  Ctl* t = c.ctl;
  const unsigned long long nk =
      min((unsigned long long)t->nkeys, (unsigned long long)c.backlog_cap);
  t->base += n;
  const int top = t->pool_top > 0 ? t->pool_top : 0;
  t->pool_top = ((unsigned long long)top + t->ntasks <= c.max_chunks) ? top + (int)t->ntasks : top;
  t->st_batches += 1;
  t->st_points += n;
  t->st_spilled += t->spill_count;
  t->st_splits += t->split_count;
  t->st_voxels += nk;
  if (iters > t->st_iter_max) t->st_iter_max = iters;
  t->st_rounds += iters;
  t->last_points = n;
  t->last_spilled = t->spill_count;
  t->last_splits = t->split_count;
  t->last_voxels = nk;
  t->last_iters = iters;
  t->spill_count = 0;
  t->nkeys = 0;
  t->alloc_seq = 0;
  t->split_count = 0;
  t->ntasks = 0;
  t->mv_count[0] = 0;
  t->mv_count[1] = 0;
}

// One thread: close a rejected update (the rollback undid its counters).
__device__ void phase_end_rejected(const Ctx& c) {
  Ctl* t = c.ctl;
  t->reject = 0;
  t->nkeys = 0;
  t->st_rejected += 1;
}

}  // namespace SL_NS
