// Kernels and host API of the C ABI in include/simlod.h (plain form: one
// kernel per phase, expansion rounds steered from the host).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "device.cuh"
#include "fused.cuh"
#include "render.cuh"
#include "simlod.h"
#include "variant.h"

using namespace sl;

// ================================================================= kernels

namespace {

constexpr int BLOCK = 256;
constexpr int PBLOCK = PHASE_BLOCK;  // count / advance kernels (one node-table cache per block)

__global__ void k_init(Ctx c) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Ctl* t = c.ctl;
    unsigned long long phase_ns[8];  // diagnostics survive a reset
    for (int k = 0; k < 8; ++k) phase_ns[k] = t->phase_ns[k];
    memset(t, 0, sizeof(Ctl));
    for (int k = 0; k < 8; ++k) t->phase_ns[k] = phase_ns[k];
    t->n_nodes = 1;
    t->bump = c.dir_bytes;  // the root's chunk directory is the first data ref
    NodeMeta m;
    memset(&m, 0, sizeof(m));
    m.min[0] = c.rmin[0];
    m.min[1] = c.rmin[1];
    m.min[2] = c.rmin[2];
    m.level = 0;
    m.head = m.tail = NONE;
    m.dir = 0;
    m.st_tail = NONE;
    c.meta[0] = m;
    c.child[0] = NONE;
    c.gridref[0] = NONE;
    c.cnt[0] = 0;
    c.num[0] = 0;
  }
}

__global__ void k_fill_hash(HSlot* h, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    h[i].key = HASH_EMPTY;
    h[i].val = HASH_EMPTY;
  }
}

__global__ void __launch_bounds__(PBLOCK, PHASE_MIN_BLOCKS) k_count1(Ctx c, const int4* pts, uint64_t n,
                                                    unsigned long long base, uint32_t n_nodes) {
  extern __shared__ uint32_t smem[];
  const uint64_t warps_per_block = blockDim.x / 32;
  node_cache_load(c, smem, 0, n_nodes);
  phase_count1(c, smem, node_cache_at(smem, n_nodes), pts, n, base,
               blockIdx.x * warps_per_block + threadIdx.x / 32,
               (uint64_t)gridDim.x * warps_per_block);
}

// Decide / allocate; after the first count round of a rejected batch (no
// thread changes the reject flag during this kernel) undo that round instead.
__global__ void __launch_bounds__(BLOCK) k_decide(Ctx c, uint32_t s_lo, uint32_t s_hi,
                                                   uint32_t n_lo, uint32_t n_hi, int zero_list) {
  const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
  if (*reinterpret_cast<volatile unsigned int*>(&c.ctl->reject)) {
    phase_rollback(c, n_hi, t0, nt);
    return;
  }
  phase_decide(c, s_lo, s_hi, n_lo, n_hi, zero_list, t0 / 32, nt / 32);
}

__global__ void __launch_bounds__(PBLOCK, PHASE_MIN_BLOCKS) k_advance(Ctx c, const int4* pts, uint64_t n,
                                                     unsigned long long base, uint32_t n_nodes,
                                                     uint32_t t_hi, uint32_t s_lo, uint32_t s_hi,
                                                     int in_list, uint32_t n_in, int out_list) {
  extern __shared__ uint32_t smem[];
  const uint64_t warps_per_block = blockDim.x / 32;
  node_cache_load(c, smem, 0, n_nodes);
  phase_advance(c, smem, node_cache_at(smem, n_nodes), pts, n, base, t_hi, s_lo, s_hi, in_list,
                n_in, out_list,
                blockIdx.x * warps_per_block + threadIdx.x / 32,
                (uint64_t)gridDim.x * warps_per_block);
}

__global__ void __launch_bounds__(BLOCK) k_store(Ctx c, const int4* pts, uint64_t n,
                                                  unsigned long long base, uint32_t n_spill,
                                                  uint32_t n_tasks, uint32_t n_keys, int pool_top) {
  phase_store(c, nullptr, pts, n, base, n_spill, n_tasks, n_keys, pool_top,
              blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, (uint64_t)gridDim.x * blockDim.x);
}

// Compaction of cold nodes (the paper's closing direction: nodes that are no
// longer modified become non-growable arrays). One warp per node: a node with
// records in two or more chunks that has received none in the last `idle`
// updates gets one contiguous array (records, then aux words) from the data
// region, its records are copied over in order, and its chunks go back to
// the pool. Space the data region cannot give is skipped without an error.
__global__ void k_compact(Ctx c, uint32_t idle) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const uint64_t nwarps = (uint64_t)gridDim.x * blockDim.x / 32;
  const uint32_t n_nodes = min(vload(&c.ctl->n_nodes), c.max_nodes);
  const unsigned long long now = vload(&c.ctl->st_batches);
  for (uint64_t id = warp; id < n_nodes; id += nwarps) {
    NodeMeta& m = c.meta[id];
    const uint32_t n = c.num[id], nch = m.n_chunks;
    if (m.compact || n == 0 || nch < 2 || (unsigned long long)m.touched + idle > now) continue;
    const unsigned long long bytes = array_bytes(n);
    unsigned long long off = ~0ull;
    int p0 = 0;
    if (lane == 0) {
      unsigned long long b = vload(&c.ctl->bump);
      while (b + bytes <= c.data_bytes) {
        const unsigned long long seen = atomicCAS(&c.ctl->bump, b, b + bytes);
        if (seen == b) {
          off = b;
          break;
        }
        b = seen;
      }
      if (off != ~0ull) {
        p0 = atomicAdd(&c.ctl->pool_top, (int)nch);
        if (p0 < 0 || (unsigned long long)p0 + nch > c.max_chunks) {
          set_error(c, E_POOL);
          off = ~0ull;
        }
      }
    }
    off = __shfl_sync(FULL_MASK, off, 0);
    p0 = __shfl_sync(FULL_MASK, p0, 0);
    if (off == ~0ull) continue;
    const uint32_t arr = (uint32_t)(off / REF_BYTES);
    int4* drec = array_recs(c, arr);
    uint32_t* daux = array_aux(c, arr, n);
    uint32_t ref = m.head, idx = 0;
    for (uint32_t j = 0; j < nch && idx < n; ++j) {
      if (!ref_ok(c, ref, c.chunk_bytes)) {
        if (lane == 0) set_error(c, E_INTERNAL);
        break;
      }
      const uint32_t nxt = *chunk_next(c, ref);
      const uint32_t cnt = min(c.C, n - idx);
      const int4* srec = chunk_recs(c, ref);
      const uint32_t* saux = chunk_aux(c, ref);
      for (uint32_t q = lane; q < cnt; q += 32) {
        drec[idx + q] = srec[q];
        daux[idx + q] = saux[q];
      }
      if (lane == 0) c.pool[p0 + (int)j] = ref;
      idx += cnt;
      ref = nxt;
    }
    __syncwarp();
    if (lane == 0) {
      uint32_t* hdr = reinterpret_cast<uint32_t*>(ref_ptr(c, arr));
      hdr[0] = NONE;  // no next chunk
      hdr[1] = n;     // capacity
      m.head = m.tail = arr;
      m.compact = 1;
      atomicAdd(&c.ctl->st_compacted, 1ull);
      atomicAdd(&c.ctl->st_compact_chunks, (unsigned long long)nch);
      atomicAdd(&c.ctl->compact_now, 1ull);
      atomicAdd(&c.ctl->compact_chunks_now, (unsigned long long)nch);
    }
  }
}

__global__ void k_end(Ctx c, uint64_t n, uint32_t iters) { phase_end(c, n, iters); }

__global__ void k_end_rejected(Ctx c) { phase_end_rejected(c); }

// Kernel instance 0: the k_fused of this file (the header's knobs).
int fused_info_0(sl_variant_info* out) {
  out->block = FUSED_BLOCK;
  out->min_blocks = PHASE_MIN_BLOCKS;
  out->node_cache = NODE_CACHE;
  out->store_unroll = STORE_U;
  out->descent_group = DESCENT_GROUP;
  out->smem_bytes = PHASE_SMEM_BYTES;
  out->max_per_sm = 0;
  if (cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           PHASE_SMEM_BYTES) != cudaSuccess)
    return 1;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fused, FUSED_BLOCK,
                                                    PHASE_SMEM_BYTES) != cudaSuccess)
    return 1;
  out->max_per_sm = n;
  return 0;
}

int fused_launch_0(const sl_fused_launch* a) {
  if (a->ctx_bytes != sizeof(Ctx)) return (int)cudaErrorInvalidValue;
  Ctx c;
  memcpy(&c, a->ctx, sizeof(Ctx));
  const BatchDesc* bt = static_cast<const BatchDesc*>(a->batches);
  uint32_t n = a->n_batches;
  FusedCtl* f = static_cast<FusedCtl*>(a->fctl);
  unsigned long long budget = a->budget_ns;
  uint32_t max_iters = a->max_iters;
  const unsigned int* n_dev = a->n_dev;
  const PlanSeg* segs = static_cast<const PlanSeg*>(a->segs);
  const unsigned int* ready = a->ready;
  void* args[] = {&c, &bt, &n, &f, &budget, &max_iters, &n_dev, &segs, &ready};
  return (int)cudaLaunchCooperativeKernel((const void*)k_fused, dim3(a->grid), dim3(FUSED_BLOCK),
                                          args, PHASE_SMEM_BYTES,
                                          static_cast<cudaStream_t>(a->stream));
}

}  // namespace

// The other kernel instances (fused_variant.cu, one object per instance).
extern "C" {
int sl_fused_variant_info_1(sl_variant_info* out);
int sl_fused_variant_launch_1(const sl_fused_launch* a);
int sl_fused_variant_info_2(sl_variant_info* out);
int sl_fused_variant_launch_2(const sl_fused_launch* a);
int sl_fused_variant_info_3(sl_variant_info* out);
int sl_fused_variant_launch_3(const sl_fused_launch* a);
}

namespace {

struct VariantFns {
  int (*info)(sl_variant_info*);
  int (*launch)(const sl_fused_launch*);
};
static_assert(SL_N_VARIANTS == SIMLOD_N_VARIANTS, "kernel instances");
const VariantFns kVariants[SL_N_VARIANTS] = {
    {fused_info_0, fused_launch_0},
    {sl_fused_variant_info_1, sl_fused_variant_launch_1},
    {sl_fused_variant_info_2, sl_fused_variant_launch_2},
    {sl_fused_variant_info_3, sl_fused_variant_launch_3},
};

}  // namespace

// ================================================================ host side

enum KernelId { K_COUNT = 0, K_DECIDE, K_ADVANCE, K_STORE, K_END, K_FUSED, K_INIT, K_RENDER };
static const char* const kKernelNames[SIMLOD_N_KERNELS] = {
    "count1", "decide", "advance", "store", "end", "fused_update", "init", "render"};

struct Layout {
  size_t ctl, fctl, batches, child, gridref, cnt, num, meta, pool, pending, alloc_refs, splits,
      tasks, sp_cur, sp_rec, sp_gidx, b_cur, mv0, mv1, scur, vis, hash, keys, staging, data, end;
  uint64_t hash_slots, max_chunks, max_splits, data_bytes;
};

struct simlod {
  simlod_config cfg;
  Ctx ctx;
  Layout lay;
  uint8_t* arena;
  size_t arena_bytes;
  Ctl* ctl_host;  // pinned mirror of the control block
  unsigned long long base;  // host copy of the gidx counter
  uint32_t n_nodes;         // host copy of the node count
  int sticky;               // poison status
  cudaStream_t last_stream;
  int sm_count;
  // fused form
  int fused_grid;           // blocks of k_fused launches
  int fused_max_per_sm;     // co-resident k_fused blocks per SM
  sl_variant_info var[SL_N_VARIANTS];  // kernel instances of the batched form
  bool mirror_stale;        // a fused launch ran since the last control-block read
  unsigned long long rejected_async_seen;  // fused-launch rejections already reported
  BatchDesc* desc_host;     // pinned staging of the batch table
  cudaEvent_t desc_done;    // the last batch-table copy has finished
  FusedCtl* fctl_host;      // pinned mirror of the fused control words
  uint32_t* one_host;       // pinned word holding 1: the source of ready-flag copies
  uint32_t* prog_host;      // mapped pinned words: [0] batches of persistent launches
  uint32_t* prog_dev;       //   finished, [1] batches dropped by budget stops; device address
  uint32_t prog_submitted;  // batches handed to persistent launches (simlod_progress)
  cudaEvent_t flags_clear;  // the ready flags of the last host-fed launch are cleared
  FusedCtl* fctl_dev;
  BatchDesc* batches_dev;
  // timing
  bool timing;
  std::vector<cudaEvent_t> ev_pool;
  struct Pending {
    int kernel;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  uint64_t launches[SIMLOD_N_KERNELS];
  double ms[SIMLOD_N_KERNELS];
  unsigned long long phase_ns_cleared[SIMLOD_N_PHASES];
};

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

uint64_t next_pow2(uint64_t v) {
  uint64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

bool valid_config(const simlod_config* c) {
  if (!c) return false;
  if (c->root_log2 < 1 || c->root_log2 > 31) return false;
  if (c->leaf_capacity < 1 || c->chunk_points < 1 || c->chunk_points > 65536) return false;
  if (c->grid_log2 < 1 || c->grid_log2 > 7) return false;
  // mover-list entries name a batch point or a spill entry in 31 bits
  if (c->max_batch_points < 1 || c->max_batch_points >= (1ull << 31)) return false;
  if (c->spill_capacity >= (1ull << 31) || c->backlog_capacity < 1 ||
      c->backlog_capacity > (1ull << 31))
    return false;
  if (c->max_nodes < 9 || c->max_nodes > (1ull << MV_NODE_BITS)) return false;
  if ((c->leaf_capacity + (uint64_t)c->chunk_points - 1) / c->chunk_points > (1u << 18))
    return false;  // chunk directories of at most 1 MiB
  for (int a = 0; a < 3; ++a) {
    long long hi = (long long)c->root_min[a] + (1ll << c->root_log2) - 1;
    if (hi > 0x7FFFFFFFll) return false;
  }
  return true;
}

uint32_t chunk_bytes_of(const simlod_config* c) {
  return (uint32_t)align_up(CHUNK_HEADER + 20ull * c->chunk_points, REF_BYTES);
}

// A leaf's chunk directory holds one ref per chunk; a leaf that can still
// split holds at most T points, so ceil(T / C) + 1 entries suffice.
uint32_t dir_cap_of(const simlod_config* c) {
  return (uint32_t)((c->leaf_capacity + (uint64_t)c->chunk_points - 1) / c->chunk_points + 1);
}

uint32_t dir_bytes_of(const simlod_config* c) {
  return (uint32_t)align_up(4ull * dir_cap_of(c), REF_BYTES);
}

uint32_t grid_bytes_of(const simlod_config* c) {
  uint64_t bits = 1ull << (3 * c->grid_log2);
  return (uint32_t)align_up(std::max<uint64_t>(bits / 8, 1), REF_BYTES);
}

// Place every region; the data region (grids and chunks) takes what is left
// and pool / pending / alloc_refs hold one entry per chunk that fits in it.
bool plan_layout(const simlod_config* c, size_t arena_bytes, Layout* L) {
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = align_up(o, 256);
    o = at + bytes;
    return at;
  };
  const uint64_t N = c->max_nodes, B = c->max_batch_points, S = c->spill_capacity;
  L->max_splits = N / 8 + 1;
  L->hash_slots = next_pow2(2 * c->backlog_capacity);
  L->ctl = take(sizeof(Ctl));
  L->fctl = take(sizeof(FusedCtl));
  L->batches = take(sizeof(BatchDesc) * MAX_FUSED_BATCHES);
  L->child = take(4 * N);
  L->gridref = take(4 * N);
  L->cnt = take(4 * N);
  L->num = take(4 * N);
  L->meta = take(sizeof(NodeMeta) * N);
  L->splits = take(sizeof(SplitEntry) * L->max_splits);
  L->sp_cur = take(4 * S);
  L->b_cur = take(4 * B);
  L->mv0 = take(8 * (B + S));
  L->mv1 = take(8 * (B + S));
  L->sp_rec = take(16 * S);
  L->sp_gidx = take(4 * S);
  L->scur = take(4 * N);
  L->vis = take(4 * N);
  L->hash = take(sizeof(HSlot) * L->hash_slots);
  L->keys = take(sizeof(uint32_t) * c->backlog_capacity);
  L->staging = take(16 * B);
  const size_t fixed = align_up(o, 256);
  if (arena_bytes < fixed) return false;
  const uint64_t cb = chunk_bytes_of(c);
  // per chunk of the data region: pool, pending, alloc_refs (4 B each) and a task (16 B)
  uint64_t max_chunks = (arena_bytes - fixed) / (cb + 28);
  if (max_chunks > 0xFFFFFFF0ull) max_chunks = 0xFFFFFFF0ull;
  L->max_chunks = max_chunks;
  L->pool = take(4 * max_chunks);
  L->pending = take(4 * max_chunks);
  L->alloc_refs = take(4 * max_chunks);
  L->tasks = take(sizeof(SpillTask) * max_chunks);
  L->data = align_up(o, 256);
  if (arena_bytes < L->data) return false;
  L->data_bytes = (arena_bytes - L->data) / REF_BYTES * REF_BYTES;
  if (L->data_bytes / REF_BYTES > 0xFFFFFFFFull) L->data_bytes = 0xFFFFFFFFull * REF_BYTES;
  L->end = L->data + L->data_bytes;
  return true;
}

void make_ctx(simlod_t* h) {
  Ctx& c = h->ctx;
  const Layout& L = h->lay;
  uint8_t* a = h->arena;
  c.ctl = reinterpret_cast<Ctl*>(a + L.ctl);
  h->fctl_dev = reinterpret_cast<FusedCtl*>(a + L.fctl);
  c.launch_bar = &h->fctl_dev->bar;
  h->batches_dev = reinterpret_cast<BatchDesc*>(a + L.batches);
  c.child = reinterpret_cast<uint32_t*>(a + L.child);
  c.gridref = reinterpret_cast<uint32_t*>(a + L.gridref);
  c.cnt = reinterpret_cast<uint32_t*>(a + L.cnt);
  c.num = reinterpret_cast<uint32_t*>(a + L.num);
  c.meta = reinterpret_cast<NodeMeta*>(a + L.meta);
  c.pool = reinterpret_cast<uint32_t*>(a + L.pool);
  c.pending = reinterpret_cast<uint32_t*>(a + L.pending);
  c.alloc_refs = reinterpret_cast<uint32_t*>(a + L.alloc_refs);
  c.splits = reinterpret_cast<SplitEntry*>(a + L.splits);
  c.tasks = reinterpret_cast<SpillTask*>(a + L.tasks);
  c.sp_cur = reinterpret_cast<uint32_t*>(a + L.sp_cur);
  c.b_cur = reinterpret_cast<uint32_t*>(a + L.b_cur);
  c.mv[0] = reinterpret_cast<uint2*>(a + L.mv0);
  c.mv[1] = reinterpret_cast<uint2*>(a + L.mv1);
  c.sp_rec = reinterpret_cast<int4*>(a + L.sp_rec);
  c.sp_gidx = reinterpret_cast<uint32_t*>(a + L.sp_gidx);
  c.scur = reinterpret_cast<uint32_t*>(a + L.scur);
  c.hash = reinterpret_cast<HSlot*>(a + L.hash);
  c.keys = reinterpret_cast<uint32_t*>(a + L.keys);
  c.staging = reinterpret_cast<int4*>(a + L.staging);
  c.data = a + L.data;
  c.data_bytes = L.data_bytes;
  const simlod_config& g = h->cfg;
  for (int k = 0; k < 3; ++k) c.rmin[k] = g.root_min[k];
  c.rlog2 = g.root_log2;
  c.T = g.leaf_capacity;
  c.C = g.chunk_points;
  c.G = g.grid_log2;
  c.chunk_bytes = chunk_bytes_of(&g);
  c.chunk_units = c.chunk_bytes / REF_BYTES;
  c.grid_bytes = grid_bytes_of(&g);
  c.dir_bytes = dir_bytes_of(&g);
  c.dir_cap = dir_cap_of(&g);
  c.hash_mask = (uint32_t)(L.hash_slots - 1);
  c.max_nodes = (uint32_t)g.max_nodes;
  c.max_chunks = (uint32_t)L.max_chunks;
  c.spill_cap = (uint32_t)g.spill_capacity;
  c.backlog_cap = (uint32_t)g.backlog_capacity;
  c.max_splits = (uint32_t)L.max_splits;
  c.max_batch = g.max_batch_points;
  c.mv_cap = g.max_batch_points + g.spill_capacity;
  c.bar_ns = FUSED_BARRIER_NS;
  c.ready_ns = FUSED_READY_NS;
  c.progress = nullptr;  // set per persistent launch (launch_fused)
}

int error_from_bits(uint32_t e) {
  if (e & E_ITER_CAP) return SIMLOD_ERR_ITER_CAP;
  if (e & E_ARENA) return SIMLOD_ERR_ARENA_FULL;
  if (e & E_NODES) return SIMLOD_ERR_NODES_FULL;
  if (e & E_SPILL) return SIMLOD_ERR_SPILL_FULL;
  if (e & E_BACKLOG) return SIMLOD_ERR_BACKLOG_FULL;
  if (e & (E_ALLOC_REFS | E_POOL)) return SIMLOD_ERR_ARENA_FULL;
  if (e & E_TIMEOUT) return SIMLOD_ERR_TIMEOUT;
  return SIMLOD_ERR_CUDA;
}

int poison(simlod_t* h, int status) {
  if (!h->sticky) h->sticky = status;
  return status;
}

cudaEvent_t take_event(simlod_t* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Fold finished timing pairs into the per-kernel totals (after a sync).
void harvest_timing(simlod_t* h) {
  for (auto& p : h->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      h->ms[p.kernel] += ms;
      h->launches[p.kernel] += 1;
    }
    h->ev_pool.push_back(p.a);
    h->ev_pool.push_back(p.b);
  }
  h->pending.clear();
}

template <typename Launch>
int launch(simlod_t* h, int kernel, cudaStream_t s, Launch&& fn) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (h->timing) {
    a = take_event(h);
    cudaEventRecord(a, s);
  }
  fn();
  cudaError_t err = cudaGetLastError();
  if (h->timing) {
    b = take_event(h);
    cudaEventRecord(b, s);
    h->pending.push_back({kernel, a, b});
  }
  return err == cudaSuccess ? SIMLOD_OK : SIMLOD_ERR_CUDA;
}

unsigned grid_for(const simlod_t* h, uint64_t work, uint64_t per_block) {
  uint64_t blocks = (work + per_block - 1) / per_block;
  uint64_t cap = (uint64_t)h->sm_count * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (unsigned)blocks;
}

// Read the control block (waits for the stream).
int read_ctl(simlod_t* h, cudaStream_t s) {
  if (cudaMemcpyAsync(h->ctl_host, h->ctx.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return SIMLOD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return SIMLOD_ERR_CUDA;
  if (h->timing) harvest_timing(h);
  if (h->mirror_stale) {
    h->base = h->ctl_host->base;
    h->n_nodes = h->ctl_host->n_nodes;
    h->mirror_stale = false;
  }
  return SIMLOD_OK;
}

int insert_device(simlod_t* h, const int4* pts, uint64_t n, cudaStream_t s) {
  if (h->mirror_stale) {
    int r0 = read_ctl(h, h->last_stream);
    if (r0) return poison(h, r0);
    if (h->ctl_host->error) return poison(h, error_from_bits(h->ctl_host->error));
  }
  h->last_stream = s;
  const Ctx& c = h->ctx;
  const unsigned long long base = h->base;
  const uint32_t nodes0 = h->n_nodes;
  const unsigned gp = std::max(1u, std::min<unsigned>(grid_for(h, n, PBLOCK), (unsigned)PHASE_MIN_BLOCKS * h->sm_count));
  int rc;
  rc = launch(h, K_COUNT, s, [&] {
    k_count1<<<gp, PBLOCK, PHASE_SMEM_BYTES, s>>>(c, pts, n, base, nodes0);
  });
  if (rc) return poison(h, rc);
  rc = launch(h, K_DECIDE, s, [&] {
    k_decide<<<grid_for(h, 32ull * nodes0, BLOCK), BLOCK, 0, s>>>(c, 0, 0, 0, nodes0, -1);
  });
  if (rc) return poison(h, rc);
  if ((rc = read_ctl(h, s))) return poison(h, rc);
  const Ctl& t = *h->ctl_host;
  if (t.error) return poison(h, error_from_bits(t.error));
  if (t.reject) {
    rc = launch(h, K_END, s, [&] { k_end_rejected<<<1, 1, 0, s>>>(c); });
    if (rc) return poison(h, rc);
    return SIMLOD_ERR_OUT_OF_BOUNDS;
  }
  const uint32_t max_iters = h->cfg.max_expand_iters ? h->cfg.max_expand_iters
                                                      : h->cfg.root_log2 + 1;
  // s: split-list range of the previous round, n: nodes it created,
  // t_hi: spill tasks (all made by the first decide round)
  uint32_t s_lo = 0, s_hi = t.split_count, n_lo = nodes0, n_hi = t.n_nodes,
           t_hi = t.ntasks, iters = 1;
  while (s_hi > s_lo) {
    if (iters >= max_iters) return poison(h, SIMLOD_ERR_ITER_CAP);
    const int in_list = iters >= 2 ? (int)((iters - 2) & 1u) : -1;
    const int out_list = (int)((iters - 1) & 1u);
    const uint32_t n_in = in_list >= 0 ? h->ctl_host->mv_count[in_list] : 0u;
    const uint64_t units = (in_list < 0 ? (n + 31) / 32 + (uint64_t)t_hi * ((c.C + 31) / 32)
                                        : ((uint64_t)n_in + 31) / 32) +
                           (uint64_t)(s_hi - s_lo) * 64;
    const unsigned ga =
        std::max(1u, std::min<unsigned>(grid_for(h, units * 32, PBLOCK), (unsigned)PHASE_MIN_BLOCKS * h->sm_count));
    const uint32_t nn = n_hi;
    rc = launch(h, K_ADVANCE, s, [&] {
      k_advance<<<ga, PBLOCK, PHASE_SMEM_BYTES, s>>>(c, pts, n, base, nn, t_hi, s_lo, s_hi,
                                                     in_list, n_in, out_list);
    });
    if (rc) return poison(h, rc);
    ++iters;
    const uint64_t cand = (uint64_t)(s_hi - s_lo) + (n_hi - n_lo);
    const int zero_list = iters >= 3 ? (int)((iters - 1) & 1u) : -1;
    rc = launch(h, K_DECIDE, s, [&] {
      k_decide<<<grid_for(h, 32 * cand, BLOCK), BLOCK, 0, s>>>(c, s_lo, s_hi, n_lo, n_hi,
                                                              zero_list);
    });
    if (rc) return poison(h, rc);
    if ((rc = read_ctl(h, s))) return poison(h, rc);
    if (h->ctl_host->error) return poison(h, error_from_bits(h->ctl_host->error));
    if (h->ctl_host->ntasks != t_hi) return poison(h, SIMLOD_ERR_CUDA);
    s_lo = s_hi;
    s_hi = h->ctl_host->split_count;
    n_lo = n_hi;
    n_hi = h->ctl_host->n_nodes;
  }
  const uint32_t n_tasks = h->ctl_host->ntasks;
  const uint32_t n_spill = std::min<uint32_t>(h->ctl_host->spill_count, c.spill_cap);
  const uint32_t n_keys = std::min<uint32_t>(h->ctl_host->nkeys, c.backlog_cap);
  const int pool_top = h->ctl_host->pool_top;
  const uint64_t work =
      std::max<uint64_t>(std::max<uint64_t>(std::max<uint64_t>(n, n_spill), n_tasks), n_keys);
  rc = launch(h, K_STORE, s, [&] {
    k_store<<<grid_for(h, work, BLOCK), BLOCK, 0, s>>>(c, pts, n, base, n_spill, n_tasks,
                                                      n_keys, pool_top);
  });
  if (rc) return poison(h, rc);
  rc = launch(h, K_END, s, [&] { k_end<<<1, 1, 0, s>>>(c, n, iters); });
  if (rc) return poison(h, rc);
  h->base += n;
  h->n_nodes = h->ctl_host->n_nodes;
  return SIMLOD_OK;
}

// Enqueue one fused launch over n batches (device pointers + counts).
int launch_fused(simlod_t* h, const simlod_point* const* d_batches, const uint64_t* counts,
                 uint32_t n, unsigned long long budget_ns, cudaStream_t s,
                 const unsigned int* ready = nullptr) {
  if (h->fused_grid < 1) return SIMLOD_ERR_CUDA;
  uint64_t total = 0;
  for (uint32_t k = 0; k < n; ++k) {
    if (counts[k] > h->cfg.max_batch_points) return SIMLOD_ERR_INVALID_ARG;
    if (counts[k] && (!d_batches[k] || (reinterpret_cast<uintptr_t>(d_batches[k]) & 15u)))
      return SIMLOD_ERR_INVALID_ARG;
    total += counts[k];
  }
  if (h->base + total > (1ull << 32)) return SIMLOD_ERR_TOO_MANY_POINTS;
  // the staging table may still feed the previous copy
  if (cudaEventSynchronize(h->desc_done) != cudaSuccess) return poison(h, SIMLOD_ERR_CUDA);
  for (uint32_t k = 0; k < n; ++k)
    h->desc_host[k] = BatchDesc{reinterpret_cast<const int4*>(d_batches[k]), counts[k], 0, 0};
  h->last_stream = s;
  if (cudaMemcpyAsync(h->batches_dev, h->desc_host, sizeof(BatchDesc) * n,
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaEventRecord(h->desc_done, s) != cudaSuccess ||
      cudaMemsetAsync(h->fctl_dev, 0, sizeof(FusedCtl), s) != cudaSuccess)
    return poison(h, SIMLOD_ERR_CUDA);
  Ctx c = h->ctx;
  c.progress = h->prog_dev;
  const BatchDesc* bt = h->batches_dev;
  FusedCtl* f = h->fctl_dev;
  uint32_t max_iters = h->cfg.max_expand_iters ? h->cfg.max_expand_iters : h->cfg.root_log2 + 1;
  const unsigned int* n_dev = nullptr;
  const PlanSeg* segs = nullptr;
  void* args[] = {&c, &bt, &n, &f, &budget_ns, &max_iters, &n_dev, &segs, &ready};
  cudaError_t le = cudaSuccess;
  int rc = launch(h, K_FUSED, s, [&] {
    le = cudaLaunchCooperativeKernel((const void*)k_fused, dim3(h->fused_grid),
                                     dim3(FUSED_BLOCK), args, PHASE_SMEM_BYTES, s);
  });
  if (rc || le != cudaSuccess) return poison(h, SIMLOD_ERR_CUDA);
  h->base += total;  // upper bound until the next control-block read
  h->mirror_stale = true;
  h->prog_submitted += n;
  return SIMLOD_OK;
}

// After a fused launch: wait, fold rejected batches into the status.
int finish_fused(simlod_t* h, uint32_t* consumed) {
  cudaStream_t s = h->last_stream;
  if (cudaMemcpyAsync(h->fctl_host, h->fctl_dev, sizeof(FusedCtl), cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return poison(h, SIMLOD_ERR_CUDA);
  int rc = read_ctl(h, s);
  if (rc) return poison(h, rc);
  if (h->ctl_host->error) return poison(h, error_from_bits(h->ctl_host->error));
  if (consumed) *consumed = h->fctl_host->consumed;
  const unsigned long long rej = h->ctl_host->st_rejected_async;
  const bool fresh = rej > h->rejected_async_seen;
  h->rejected_async_seen = rej;
  return fresh ? SIMLOD_ERR_OUT_OF_BOUNDS : SIMLOD_OK;
}

int init_octree(simlod_t* h, cudaStream_t s, bool clear_hash, bool wait) {
  const Ctx& c = h->ctx;
  if (clear_hash) {
    k_fill_hash<<<grid_for(h, h->lay.hash_slots, BLOCK), BLOCK, 0, s>>>(c.hash, h->lay.hash_slots);
    if (cudaGetLastError() != cudaSuccess) return SIMLOD_ERR_CUDA;
  }
  k_init<<<1, 1, 0, s>>>(c);
  if (cudaGetLastError() != cudaSuccess) return SIMLOD_ERR_CUDA;
  if (wait && cudaStreamSynchronize(s) != cudaSuccess) return SIMLOD_ERR_CUDA;
  h->base = 0;
  h->n_nodes = 1;
  h->sticky = 0;
  h->rejected_async_seen = 0;
  h->mirror_stale = false;
  h->last_stream = s;
  return SIMLOD_OK;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

SIMLOD_API void simlod_config_default(simlod_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->root_log2 = 20;
  cfg->leaf_capacity = 50000;
  cfg->chunk_points = 1000;
  cfg->grid_log2 = 7;
  cfg->max_expand_iters = 0;
  cfg->max_batch_points = 16ull << 20;
  cfg->spill_capacity = 8ull << 20;
  cfg->backlog_capacity = 10000000ull;
  cfg->max_nodes = 1ull << 20;
}

SIMLOD_API int simlod_arena_bytes(const simlod_config* cfg, uint64_t data_bytes,
                                  uint64_t* arena_bytes) {
  if (!valid_config(cfg) || !arena_bytes) return SIMLOD_ERR_INVALID_ARG;
  Layout L;
  plan_layout(cfg, 0, &L);  // fixed part only
  size_t o = L.staging + 16 * cfg->max_batch_points;
  uint64_t chunks = data_bytes / chunk_bytes_of(cfg) + 1;
  o = align_up(o, 256) + align_up(4 * chunks, 256) * 3 + align_up(16 * chunks, 256) + 256;
  *arena_bytes = align_up(o + data_bytes, 256) + 256;
  return SIMLOD_OK;
}

SIMLOD_API int simlod_create(const simlod_config* cfg, void* d_arena, size_t arena_bytes,
                             void* stream, simlod_t** out) {
  if (!out) return SIMLOD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!valid_config(cfg) || !d_arena || (reinterpret_cast<uintptr_t>(d_arena) & 255u))
    return SIMLOD_ERR_INVALID_ARG;
  simlod_t* h = new (std::nothrow) simlod_t();
  if (!h) return SIMLOD_ERR_INVALID_ARG;
  h->cfg = *cfg;
  h->arena = static_cast<uint8_t*>(d_arena);
  h->arena_bytes = arena_bytes;
  if (!plan_layout(cfg, arena_bytes, &h->lay) || h->lay.max_chunks < 1) {
    delete h;
    return SIMLOD_ERR_INVALID_ARG;
  }
  make_ctx(h);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&h->ctl_host), sizeof(Ctl)) != cudaSuccess) {
    delete h;
    return SIMLOD_ERR_CUDA;
  }
  memset(h->ctl_host, 0, sizeof(Ctl));
  if (cudaFuncSetAttribute(k_count1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           PHASE_SMEM_BYTES) != cudaSuccess ||
      cudaFuncSetAttribute(k_advance, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           PHASE_SMEM_BYTES) != cudaSuccess ||
      cudaFuncSetAttribute(k_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           PHASE_SMEM_BYTES) != cudaSuccess) {
    cudaFreeHost(h->ctl_host);
    delete h;
    return SIMLOD_ERR_CUDA;
  }
#ifdef SL_CARVEOUT
  // shared-memory share of the unified L1/shared storage, in percent
  cudaFuncSetAttribute(k_fused, cudaFuncAttributePreferredSharedMemoryCarveout, SL_CARVEOUT);
  cudaFuncSetAttribute(k_count1, cudaFuncAttributePreferredSharedMemoryCarveout, SL_CARVEOUT);
  cudaFuncSetAttribute(k_advance, cudaFuncAttributePreferredSharedMemoryCarveout, SL_CARVEOUT);
  cudaGetLastError();
#endif
  int coop = 0, bpsm = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpsm, k_fused, FUSED_BLOCK,
                                                             PHASE_SMEM_BYTES) == cudaSuccess)
  {
    h->fused_max_per_sm = std::min(bpsm, 4);
    h->fused_grid = h->fused_max_per_sm * h->sm_count;
  }
  for (int k = 0; k < SL_N_VARIANTS; ++k) {
    if (kVariants[k].info(&h->var[k]) != 0) h->var[k].max_per_sm = 0;
    if (!coop) h->var[k].max_per_sm = 0;
  }
  cudaGetLastError();  // an instance this device cannot run is simply never used
  if (cudaMallocHost(reinterpret_cast<void**>(&h->desc_host),
                     sizeof(BatchDesc) * MAX_FUSED_BATCHES) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&h->fctl_host), sizeof(FusedCtl)) != cudaSuccess ||
      cudaMallocHost(reinterpret_cast<void**>(&h->one_host), sizeof(uint32_t)) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->desc_done, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->flags_clear, cudaEventDisableTiming) != cudaSuccess) {
    simlod_destroy(h);
    return SIMLOD_ERR_CUDA;
  }
  *h->one_host = 1u;
  // progress of persistent launches: a word the kernel writes in host memory
  if (cudaHostAlloc(reinterpret_cast<void**>(&h->prog_host), 2 * sizeof(uint32_t),
                    cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->prog_dev), h->prog_host, 0) !=
          cudaSuccess) {
    simlod_destroy(h);
    return SIMLOD_ERR_CUDA;
  }
  h->prog_host[0] = h->prog_host[1] = 0u;
  h->prog_submitted = 0u;
  // the arena is the caller's memory: start from a zeroed control block
  if (cudaMemsetAsync(h->ctx.ctl, 0, sizeof(Ctl), static_cast<cudaStream_t>(stream)) !=
      cudaSuccess) {
    simlod_destroy(h);
    return SIMLOD_ERR_CUDA;
  }
  int rc = init_octree(h, static_cast<cudaStream_t>(stream), true, true);
  if (rc) {
    simlod_destroy(h);
    return rc;
  }
  *out = h;
  return SIMLOD_OK;
}

SIMLOD_API int simlod_insert_batch(simlod_t* h, const simlod_point* d_pts, uint64_t n,
                                   void* stream) {
  if (!h) return SIMLOD_ERR_INVALID_ARG;
  if (h->sticky) return SIMLOD_ERR_POISONED;
  if (n == 0) return SIMLOD_OK;
  if (!d_pts || (reinterpret_cast<uintptr_t>(d_pts) & 15u) || n > h->cfg.max_batch_points)
    return SIMLOD_ERR_INVALID_ARG;
  if (h->base + n > (1ull << 32)) return SIMLOD_ERR_TOO_MANY_POINTS;
  return insert_device(h, reinterpret_cast<const int4*>(d_pts), n,
                       static_cast<cudaStream_t>(stream));
}

SIMLOD_API int simlod_insert_batch_host(simlod_t* h, const simlod_point* h_pts, uint64_t n,
                                        void* stream) {
  if (!h) return SIMLOD_ERR_INVALID_ARG;
  if (h->sticky) return SIMLOD_ERR_POISONED;
  if (n == 0) return SIMLOD_OK;
  if (!h_pts || n > h->cfg.max_batch_points) return SIMLOD_ERR_INVALID_ARG;
  if (h->base + n > (1ull << 32)) return SIMLOD_ERR_TOO_MANY_POINTS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(h->ctx.staging, h_pts, n * sizeof(simlod_point), cudaMemcpyHostToDevice,
                      s) != cudaSuccess)
    return poison(h, SIMLOD_ERR_CUDA);
  return insert_device(h, h->ctx.staging, n, s);
}

SIMLOD_API int simlod_insert_batches(simlod_t* h, const simlod_point* const* d_batches,
                                     const uint64_t* counts, uint32_t n_batches, void* stream) {
  if (!h || (n_batches && (!d_batches || !counts)) || n_batches > MAX_FUSED_BATCHES)
    return SIMLOD_ERR_INVALID_ARG;
  if (h->sticky) return SIMLOD_ERR_POISONED;
  if (n_batches == 0) return SIMLOD_OK;
  return launch_fused(h, d_batches, counts, n_batches, NO_BUDGET,
                      static_cast<cudaStream_t>(stream));
}

SIMLOD_API int simlod_insert_batches_host(simlod_t* h, const simlod_point* const* h_batches,
                                          const uint64_t* counts, uint32_t n_batches,
                                          simlod_point* d_dst, uint32_t* d_ready, void* stream,
                                          void* copy_stream) {
  if (!h || (n_batches && (!h_batches || !counts || !d_dst || !d_ready)) ||
      n_batches > MAX_FUSED_BATCHES || (reinterpret_cast<uintptr_t>(d_dst) & 15u) ||
      (reinterpret_cast<uintptr_t>(d_ready) & 3u))
    return SIMLOD_ERR_INVALID_ARG;
  if (h->sticky) return SIMLOD_ERR_POISONED;
  if (n_batches == 0) return SIMLOD_OK;
  std::vector<const simlod_point*> dst(n_batches);
  uint64_t off = 0;
  for (uint32_t k = 0; k < n_batches; ++k) {
    if (counts[k] > h->cfg.max_batch_points || (counts[k] && !h_batches[k]))
      return SIMLOD_ERR_INVALID_ARG;
    dst[k] = d_dst + off;
    off += counts[k];
  }
  if (h->base + off > (1ull << 32)) return SIMLOD_ERR_TOO_MANY_POINTS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStream_t cs = static_cast<cudaStream_t>(copy_stream);
  // flags cleared on `stream` before the launch, and before any copy sets one
  if (cudaMemsetAsync(d_ready, 0, sizeof(uint32_t) * n_batches, s) != cudaSuccess ||
      cudaEventRecord(h->flags_clear, s) != cudaSuccess ||
      cudaStreamWaitEvent(cs, h->flags_clear, 0) != cudaSuccess)
    return poison(h, SIMLOD_ERR_CUDA);
  // one copy per batch, then a 4-byte copy of 1 into its flag: copies of one
  // stream run in order, so the flag is set after the batch is in place
  for (uint32_t k = 0; k < n_batches; ++k) {
    if (counts[k] &&
        cudaMemcpyAsync(const_cast<simlod_point*>(dst[k]), h_batches[k],
                        sizeof(simlod_point) * counts[k], cudaMemcpyHostToDevice,
                        cs) != cudaSuccess)
      return poison(h, SIMLOD_ERR_CUDA);
    if (cudaMemcpyAsync(d_ready + k, h->one_host, sizeof(uint32_t), cudaMemcpyHostToDevice, cs) !=
        cudaSuccess)
      return poison(h, SIMLOD_ERR_CUDA);
  }
  return launch_fused(h, dst.data(), counts, n_batches, NO_BUDGET, s, d_ready);
}

SIMLOD_API int simlod_frame_update(simlod_t* h, const simlod_point* const* d_batches,
                                   const uint64_t* counts, uint32_t n_batches,
                                   uint64_t budget_ns, void* stream, uint32_t* consumed) {
  if (!h || !consumed || (n_batches && (!d_batches || !counts)) ||
      n_batches > MAX_FUSED_BATCHES)
    return SIMLOD_ERR_INVALID_ARG;
  *consumed = 0;
  if (h->sticky) return SIMLOD_ERR_POISONED;
  if (n_batches == 0) return SIMLOD_OK;
  const unsigned long long budget = budget_ns >= NO_BUDGET ? NO_BUDGET - 1 : budget_ns;
  int rc = launch_fused(h, d_batches, counts, n_batches, budget, static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  return finish_fused(h, consumed);
}

SIMLOD_API int simlod_insert_batches_budget(simlod_t* h, const simlod_point* const* d_batches,
                                            const uint64_t* counts, uint32_t n_batches,
                                            uint64_t budget_ns, void* stream) {
  if (!h || (n_batches && (!d_batches || !counts)) || n_batches > MAX_FUSED_BATCHES)
    return SIMLOD_ERR_INVALID_ARG;
  if (h->sticky) return SIMLOD_ERR_POISONED;
  if (n_batches == 0) return SIMLOD_OK;
  const unsigned long long budget = budget_ns >= NO_BUDGET ? NO_BUDGET - 1 : budget_ns;
  return launch_fused(h, d_batches, counts, n_batches, budget, static_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------ batched form

struct simlod_plan {
  simlod_t* h;
  simlod_plan_params p;
  uint32_t n;           // input batches
  uint64_t total;       // their points
  uint32_t units;       // 4,096-point validation units
  unsigned grid;        // blocks of the persistent launch
  void* dmem;           // the plan's device tables (one cudaMalloc)
  PlanInput* in;
  uint32_t* tile0;
  unsigned int* bad;
  BatchDesc* groups;
  PlanSeg* segs;
  unsigned int* n_groups;
  cudaStream_t cap;     // capture stream
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool graphed;
  cudaStream_t last;    // stream of the last run
};

namespace {

// The launch sequence of one run: validate, group, fused update.
int plan_enqueue(simlod_plan_t* P, cudaStream_t s) {
  simlod_t* h = P->h;
  Ctx c = h->ctx;
  if (cudaMemsetAsync(P->bad, 0, 4ull * P->n, s) != cudaSuccess ||
      cudaMemsetAsync(P->n_groups, 0, sizeof(unsigned int), s) != cudaSuccess)
    return SIMLOD_ERR_CUDA;
  const unsigned vg = std::max(1u, std::min<unsigned>(P->units, (unsigned)h->sm_count * 8));
  k_plan_validate<<<vg, BLOCK, 0, s>>>(c, P->in, P->tile0, P->n, P->bad);
  k_plan_groups<<<1, 1, 0, s>>>(c, P->in, P->n, P->bad, P->p.merge_points, P->groups, P->segs,
                                P->n_groups);
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemsetAsync(h->fctl_dev, 0, sizeof(FusedCtl), s) != cudaSuccess)
    return SIMLOD_ERR_CUDA;
  sl_fused_launch a;
  a.ctx = &c;
  a.ctx_bytes = sizeof(Ctx);
  a.batches = P->groups;
  a.n_batches = P->n;
  a.fctl = h->fctl_dev;
  a.budget_ns = NO_BUDGET;
  a.max_iters = h->cfg.max_expand_iters ? h->cfg.max_expand_iters : h->cfg.root_log2 + 1;
  a.n_dev = P->n_groups;
  a.segs = P->segs;
  a.ready = nullptr;
  a.grid = P->grid;
  a.stream = s;
  if (kVariants[P->p.variant].launch(&a) != (int)cudaSuccess) return SIMLOD_ERR_CUDA;
  return SIMLOD_OK;
}

}  // namespace

SIMLOD_API int simlod_plan_create(simlod_t* h, const simlod_point* const* d_batches,
                                  const uint64_t* counts, uint32_t n_batches,
                                  const simlod_plan_params* params, simlod_plan_t** out) {
  if (!h || !out || !params || (n_batches && (!d_batches || !counts)) ||
      n_batches > MAX_FUSED_BATCHES || params->variant >= SL_N_VARIANTS)
    return SIMLOD_ERR_INVALID_ARG;
  *out = nullptr;
  const int vmax = h->var[params->variant].max_per_sm;
  if (params->blocks_per_sm > (uint32_t)std::max(vmax, 0)) return SIMLOD_ERR_INVALID_ARG;
  if (h->sticky) return SIMLOD_ERR_POISONED;
  if (vmax < 1) return SIMLOD_ERR_CUDA;
  uint64_t total = 0;
  std::vector<PlanInput> in(n_batches);
  std::vector<uint32_t> tile0(n_batches + 1, 0);
  for (uint32_t k = 0; k < n_batches; ++k) {
    if (counts[k] > h->cfg.max_batch_points) return SIMLOD_ERR_INVALID_ARG;
    if (counts[k] && (!d_batches[k] || (reinterpret_cast<uintptr_t>(d_batches[k]) & 15u)))
      return SIMLOD_ERR_INVALID_ARG;
    in[k] = PlanInput{reinterpret_cast<const int4*>(d_batches[k]), counts[k]};
    total += counts[k];
    tile0[k + 1] = tile0[k] + (uint32_t)((counts[k] + 4095) / 4096);
  }
  auto* P = new simlod_plan();
  P->h = h;
  P->p = *params;
  P->p.merge_points = std::min<uint64_t>(params->merge_points, h->cfg.max_batch_points);
  P->n = n_batches;
  P->total = total;
  P->units = tile0[n_batches];
  P->grid = (unsigned)h->sm_count *
            (params->blocks_per_sm ? params->blocks_per_sm : (unsigned)vmax);
  P->last = h->last_stream;
  const size_t nb = std::max<uint32_t>(n_batches, 1);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = align_up(o, 256);
    o = at + bytes;
    return at;
  };
  const size_t o_in = take(sizeof(PlanInput) * nb), o_t0 = take(4 * (nb + 1)),
               o_bad = take(4 * nb), o_g = take(sizeof(BatchDesc) * nb),
               o_s = take(sizeof(PlanSeg) * nb), o_ng = take(16);
  if (cudaMalloc(&P->dmem, o) != cudaSuccess) {
    delete P;
    return SIMLOD_ERR_CUDA;
  }
  uint8_t* d = static_cast<uint8_t*>(P->dmem);
  P->in = reinterpret_cast<PlanInput*>(d + o_in);
  P->tile0 = reinterpret_cast<uint32_t*>(d + o_t0);
  P->bad = reinterpret_cast<unsigned int*>(d + o_bad);
  P->groups = reinterpret_cast<BatchDesc*>(d + o_g);
  P->segs = reinterpret_cast<PlanSeg*>(d + o_s);
  P->n_groups = reinterpret_cast<unsigned int*>(d + o_ng);
  if ((n_batches && cudaMemcpy(P->in, in.data(), sizeof(PlanInput) * n_batches,
                               cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(P->tile0, tile0.data(), 4ull * (n_batches + 1), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    cudaFree(P->dmem);
    delete P;
    return SIMLOD_ERR_CUDA;
  }
  if (params->use_graph && n_batches) {
    // capture the launch sequence once; replays skip the per-launch host work
    bool ok = cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      const int rc = plan_enqueue(P, P->cap);
      const bool ended = cudaStreamEndCapture(P->cap, &P->graph) == cudaSuccess;
      ok = rc == SIMLOD_OK && ended && P->graph &&
           cudaGraphInstantiate(&P->exec, P->graph, 0) == cudaSuccess;
    }
    cudaGetLastError();  // a failed capture leaves no error behind: runs launch directly
    P->graphed = ok;
  }
  *out = P;
  return SIMLOD_OK;
}

SIMLOD_API int simlod_plan_run(simlod_plan_t* P, void* stream) {
  if (!P) return SIMLOD_ERR_INVALID_ARG;
  simlod_t* h = P->h;
  if (h->sticky) return SIMLOD_ERR_POISONED;
  if (P->n == 0) return SIMLOD_OK;
  if (h->base + P->total > (1ull << 32)) return SIMLOD_ERR_TOO_MANY_POINTS;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  P->last = s;
  int rc = SIMLOD_OK;
  const int lr = launch(h, K_FUSED, s, [&] {
    if (P->graphed) {
      if (cudaGraphLaunch(P->exec, s) != cudaSuccess) rc = SIMLOD_ERR_CUDA;
    } else {
      rc = plan_enqueue(P, s);
    }
  });
  if (rc || lr) return poison(h, SIMLOD_ERR_CUDA);
  h->base += P->total;  // upper bound until the next control-block read
  h->mirror_stale = true;
  return SIMLOD_OK;
}

SIMLOD_API int simlod_plan_info(const simlod_plan_t* P, simlod_plan_params* params,
                                uint32_t* graphed) {
  if (!P) return SIMLOD_ERR_INVALID_ARG;
  if (params) *params = P->p;
  if (graphed) *graphed = P->graphed ? 1u : 0u;
  return SIMLOD_OK;
}

SIMLOD_API int simlod_plan_destroy(simlod_plan_t* P) {
  if (!P) return SIMLOD_ERR_INVALID_ARG;
  cudaStreamSynchronize(P->last);
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  if (P->cap) cudaStreamDestroy(P->cap);
  if (P->dmem) cudaFree(P->dmem);
  delete P;
  return SIMLOD_OK;
}

namespace {

// Autotuner choices, per device, configuration and batch list.
struct TuneKey {
  int device, sm_count;
  std::vector<uint64_t> words;  // configuration fields and the batch counts
  bool operator<(const TuneKey& o) const {
    if (device != o.device) return device < o.device;
    if (sm_count != o.sm_count) return sm_count < o.sm_count;
    return words < o.words;
  }
};
struct TuneChoice {
  simlod_plan_params p;
  double ms;
};
std::mutex g_tune_mutex;
std::map<TuneKey, TuneChoice> g_tune_cache;

TuneKey tune_key(const simlod_t* h, const uint64_t* counts, uint32_t n) {
  TuneKey k;
  k.device = 0;
  cudaGetDevice(&k.device);
  k.sm_count = h->sm_count;
  const simlod_config& c = h->cfg;
  k.words = {(uint64_t)(uint32_t)c.root_min[0], (uint64_t)(uint32_t)c.root_min[1],
             (uint64_t)(uint32_t)c.root_min[2], c.root_log2, c.leaf_capacity, c.chunk_points,
             c.grid_log2, c.max_expand_iters, c.max_batch_points, c.spill_capacity,
             c.backlog_capacity, c.max_nodes, h->lay.data_bytes};
  k.words.insert(k.words.end(), counts, counts + n);
  return k;
}

}  // namespace

SIMLOD_API int simlod_plan_autotune(simlod_t* h, const simlod_point* const* d_batches,
                                    const uint64_t* counts, uint32_t n_batches, void* stream,
                                    simlod_plan_params* best, double* best_ms) {
  if (!h || !best || (n_batches && (!d_batches || !counts))) return SIMLOD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const TuneKey key = tune_key(h, counts, n_batches);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *best = it->second.p;
      if (best_ms) *best_ms = it->second.ms;
      return simlod_reset(h, s);
    }
  }
  const uint64_t mb = h->cfg.max_batch_points;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
    return SIMLOD_ERR_CUDA;
  double best_t = -1.0;
  auto trial = [&](const simlod_plan_params& p) {
    simlod_plan_t* P = nullptr;
    if (simlod_reset(h, s) != SIMLOD_OK) return;
    if (simlod_plan_create(h, d_batches, counts, n_batches, &p, &P) != SIMLOD_OK) return;
    auto ran = [&] {  // rejected batches are fine; device errors are not
      const int r = simlod_sync(h);
      return r == SIMLOD_OK || r == SIMLOD_ERR_OUT_OF_BOUNDS;
    };
    float ms = -1.0f;
    if (simlod_plan_run(P, s) == SIMLOD_OK && ran() && simlod_reset(h, s) == SIMLOD_OK &&
        cudaEventRecord(a, s) == cudaSuccess && simlod_plan_run(P, s) == SIMLOD_OK &&
        cudaEventRecord(b, s) == cudaSuccess && ran())
      cudaEventElapsedTime(&ms, a, b);
    simlod_plan_destroy(P);
    if (ms >= 0.0f && (best_t < 0.0 || ms < best_t)) {
      best_t = ms;
      *best = p;
    }
  };
  // stage 1: every kernel instance at its largest and half its largest
  // width, updates merged up to the largest batch the octree takes
  for (uint32_t v = 0; v < SL_N_VARIANTS; ++v) {
    const int mx = h->var[v].max_per_sm;
    if (mx < 1) continue;
    trial(simlod_plan_params{mb, (uint32_t)mx, 1, v});
    if (mx >= 2) trial(simlod_plan_params{mb, (uint32_t)(mx / 2), 1, v});
  }
  // stage 2: every merge size for the fastest instance and width
  if (best_t >= 0.0) {
    const simlod_plan_params top = *best;
    for (uint64_t m : {0ull, 1ull << 18, 1ull << 20, 1ull << 21, 1ull << 22, 1ull << 23})
      if (m < mb) trial(simlod_plan_params{m, top.blocks_per_sm, 1, top.variant});
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  const int rr = simlod_reset(h, s);
  if (best_t < 0.0) return SIMLOD_ERR_CUDA;
  if (best_ms) *best_ms = best_t;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = TuneChoice{*best, best_t};
  }
  return rr;
}

SIMLOD_API int simlod_variant_info(uint32_t variant, simlod_variant_desc* out) {
  if (!out || variant >= SL_N_VARIANTS) return SIMLOD_ERR_INVALID_ARG;
  sl_variant_info v;
  const int rc = kVariants[variant].info(&v);
  cudaGetLastError();
  out->threads_per_block = v.block;
  out->max_blocks_per_sm = rc == 0 && v.max_per_sm > 0 ? (uint32_t)v.max_per_sm : 0u;
  out->node_cache = v.node_cache;
  out->store_unroll = v.store_unroll;
  out->descent_group = v.descent_group;
  out->smem_bytes = v.smem_bytes;
  return out->max_blocks_per_sm ? SIMLOD_OK : SIMLOD_ERR_CUDA;
}

SIMLOD_API int simlod_set_launch_width(simlod_t* h, uint32_t blocks_per_sm,
                                       uint32_t* max_blocks_per_sm) {
  if (!h) return SIMLOD_ERR_INVALID_ARG;
  if (max_blocks_per_sm) *max_blocks_per_sm = (uint32_t)h->fused_max_per_sm;
  if (h->fused_max_per_sm < 1) return SIMLOD_ERR_CUDA;
  if (blocks_per_sm > (uint32_t)h->fused_max_per_sm) return SIMLOD_ERR_INVALID_ARG;
  const int bps = blocks_per_sm ? (int)blocks_per_sm : h->fused_max_per_sm;
  h->fused_grid = bps * h->sm_count;
  return SIMLOD_OK;
}

SIMLOD_API int simlod_progress(simlod_t* h, uint64_t* finished, uint64_t* submitted) {
  if (!h || !finished) return SIMLOD_ERR_INVALID_ARG;
  // the kernel writes the dropped count before its release store of the
  // finished count: an acquire load of the latter makes the former visible
  const uint32_t fin = __atomic_load_n(&h->prog_host[0], __ATOMIC_ACQUIRE);
  const uint32_t dropped = __atomic_load_n(&h->prog_host[1], __ATOMIC_RELAXED);
  *finished = fin;
  if (submitted) *submitted = (uint32_t)(h->prog_submitted - dropped);
  return SIMLOD_OK;
}

SIMLOD_API int simlod_set_wait_limits(simlod_t* h, uint64_t barrier_ns, uint64_t ready_ns) {
  if (!h) return SIMLOD_ERR_INVALID_ARG;
  h->ctx.bar_ns = barrier_ns ? barrier_ns : FUSED_BARRIER_NS;
  h->ctx.ready_ns = ready_ns ? ready_ns : FUSED_READY_NS;
  return SIMLOD_OK;
}

// ----------------------------------------------------------------- restore

SIMLOD_API int simlod_restore(simlod_t* h, const simlod_snapshot_t* snap, void* stream) {
  if (!h || !snap || !snap->nodes || snap->n_nodes == 0 || (snap->n_points && !snap->points) ||
      (snap->n_voxels && !snap->voxels))
    return SIMLOD_ERR_INVALID_ARG;
  const simlod_config& g = h->cfg;
  const uint64_t n = snap->n_nodes;
  if (n > g.max_nodes) return SIMLOD_ERR_NODES_FULL;
  if (snap->n_points > (1ull << 32)) return SIMLOD_ERR_TOO_MANY_POINTS;
  const simlod_node_rec* nodes = snap->nodes;
  const uint32_t C = g.chunk_points, G = g.grid_log2;
  // canonical key (level, ix, iy, iz) of a record; records must be sorted by it
  struct Key {
    uint64_t level, ix, iy, iz;
    bool operator<(const Key& o) const {
      if (level != o.level) return level < o.level;
      if (ix != o.ix) return ix < o.ix;
      if (iy != o.iy) return iy < o.iy;
      return iz < o.iz;
    }
    bool operator==(const Key& o) const {
      return level == o.level && ix == o.ix && iy == o.iy && iz == o.iz;
    }
  };
  std::vector<Key> keys(n);
  std::vector<uint64_t> po(n + 1, 0), vo(n + 1, 0);
  for (uint64_t k = 0; k < n; ++k) {
    const simlod_node_rec& r = nodes[k];
    if (r.level > g.root_log2 || r.log2size != g.root_log2 - r.level) return SIMLOD_ERR_INVALID_ARG;
    const uint32_t L = r.log2size;
    uint64_t ijk[3];
    for (int a = 0; a < 3; ++a) {
      const long long rel = (long long)r.min[a] - g.root_min[a];
      if (rel < 0 || (rel & ((1ll << L) - 1)) || (rel >> g.root_log2)) return SIMLOD_ERR_INVALID_ARG;
      ijk[a] = (uint64_t)(rel >> L);
    }
    keys[k] = Key{r.level, ijk[0], ijk[1], ijk[2]};
    if (k && !(keys[k - 1] < keys[k])) return SIMLOD_ERR_INVALID_ARG;
    const uint64_t cnt = r.is_inner ? r.n_voxels : r.n_points;
    if ((r.is_inner ? r.n_points : r.n_voxels) != 0 || r.n_chunks != (cnt + C - 1) / C ||
        (r.is_inner && L == 0))
      return SIMLOD_ERR_INVALID_ARG;
    po[k + 1] = po[k] + r.n_points;
    vo[k + 1] = vo[k] + r.n_voxels;
  }
  if (po[n] != snap->n_points || vo[n] != snap->n_voxels || keys[0].level != 0)
    return SIMLOD_ERR_INVALID_ARG;
  auto find = [&](const Key& k) -> int64_t {
    auto it = std::lower_bound(keys.begin(), keys.end(), k);
    return (it != keys.end() && *it == k) ? (int64_t)(it - keys.begin()) : -1;
  };
  // node ids: the children of a node are 8 consecutive ids in octant order
  std::vector<uint32_t> rec_of;
  std::vector<uint32_t> first_child(n, NONE);
  rec_of.reserve(n);
  rec_of.push_back(0);
  for (size_t q = 0; q < rec_of.size(); ++q) {
    const uint32_t r = rec_of[q];
    if (!nodes[r].is_inner) continue;
    first_child[q] = (uint32_t)rec_of.size();
    const Key& pk = keys[r];
    for (uint32_t o = 0; o < 8; ++o) {
      const int64_t c = find(Key{pk.level + 1, 2 * pk.ix + (o & 1), 2 * pk.iy + ((o >> 1) & 1),
                                 2 * pk.iz + ((o >> 2) & 1)});
      if (c < 0 || rec_of.size() >= n) return SIMLOD_ERR_INVALID_ARG;
      rec_of.push_back((uint32_t)c);
    }
  }
  if (rec_of.size() != n) return SIMLOD_ERR_INVALID_ARG;  // nodes outside the tree
  // host image of the node arrays and of the used data region (bump order)
  const uint64_t cb = chunk_bytes_of(&g), gb = grid_bytes_of(&g), db = dir_bytes_of(&g);
  const uint32_t dcap = dir_cap_of(&g);
  uint64_t bytes = 0, chunks = 0;
  for (uint64_t k = 0; k < n; ++k) {
    bytes += nodes[k].is_inner ? gb : db;
    bytes += nodes[k].n_chunks * cb;
    chunks += nodes[k].n_chunks;
  }
  if (bytes > h->lay.data_bytes) return SIMLOD_ERR_ARENA_FULL;
  if (chunks > h->lay.max_chunks) return SIMLOD_ERR_ARENA_FULL;
  std::vector<uint8_t> data;
  try {
    data.assign(bytes, 0);
  } catch (const std::bad_alloc&) {
    return SIMLOD_ERR_INVALID_ARG;
  }
  std::vector<uint32_t> child(n), gridref(n), num(n), zeros(n, 0);
  std::vector<NodeMeta> meta(n);
  uint64_t bump = 0;
  auto take = [&](uint64_t b) {
    const uint64_t at = bump;
    bump += b;
    return at;
  };
  for (uint64_t id = 0; id < n; ++id) {
    const uint32_t r = rec_of[id];
    const simlod_node_rec& rec = nodes[r];
    NodeMeta m;
    memset(&m, 0, sizeof(m));
    for (int a = 0; a < 3; ++a) m.min[a] = rec.min[a];
    m.level = rec.level;
    m.st_tail = NONE;
    m.head = m.tail = NONE;
    uint32_t* dir = nullptr;
    if (rec.is_inner) {
      const uint64_t go = take(gb);
      uint32_t* words = reinterpret_cast<uint32_t*>(data.data() + go);
      for (uint64_t q = vo[r]; q < vo[r + 1]; ++q) {
        const uint32_t cell = snap->voxels[q].cell;
        if (cell >> (3 * G)) return SIMLOD_ERR_INVALID_ARG;
        words[cell >> 5] |= 1u << (cell & 31u);
      }
      gridref[id] = (uint32_t)(go / REF_BYTES);
      child[id] = first_child[id];
      num[id] = (uint32_t)rec.n_voxels;
      m.dir = NONE;
    } else {
      const uint64_t d = take(db);
      dir = reinterpret_cast<uint32_t*>(data.data() + d);
      gridref[id] = NONE;
      child[id] = NONE;
      num[id] = (uint32_t)rec.n_points;
      m.dir = (uint32_t)(d / REF_BYTES);
    }
    const uint64_t cnt = rec.is_inner ? rec.n_voxels : rec.n_points;
    uint32_t prev = NONE;
    for (uint64_t j = 0; j < rec.n_chunks; ++j) {
      const uint64_t co = take(cb);
      const uint32_t ref = (uint32_t)(co / REF_BYTES);
      uint8_t* ch = data.data() + co;
      *reinterpret_cast<uint32_t*>(ch) = NONE;
      int4* recs = reinterpret_cast<int4*>(ch + CHUNK_HEADER);
      uint32_t* aux = reinterpret_cast<uint32_t*>(ch + CHUNK_HEADER + 16ull * C);
      for (uint64_t q = 0; q < C && j * C + q < cnt; ++q) {
        if (rec.is_inner) {
          const simlod_voxel_rec& v = snap->voxels[vo[r] + j * C + q];
          recs[q] = make_int4(v.x, v.y, v.z, (int)v.rgba);
          aux[q] = v.cell;
        } else {
          const simlod_point_rec& p = snap->points[po[r] + j * C + q];
          recs[q] = make_int4(p.x, p.y, p.z, (int)p.rgba);
          aux[q] = p.gidx;
        }
      }
      if (prev == NONE) m.head = ref;
      else *reinterpret_cast<uint32_t*>(data.data() + (uint64_t)prev * REF_BYTES) = ref;
      if (dir && j < dcap) dir[j] = ref;
      prev = ref;
    }
    m.tail = prev;
    m.n_chunks = (uint32_t)rec.n_chunks;
    meta[id] = m;
  }
  // start from an empty octree (clears a poisoned state and the claim table)
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool dirty = h->sticky != 0;
  if (dirty) cudaStreamSynchronize(h->last_stream);
  h->sticky = 0;
  int rc = init_octree(h, s, true, false);
  if (rc) return poison(h, rc);
  if (cudaStreamSynchronize(s) != cudaSuccess) return poison(h, SIMLOD_ERR_CUDA);
  Ctl t;
  if (cudaMemcpy(&t, h->ctx.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess)
    return poison(h, SIMLOD_ERR_CUDA);
  t.base = snap->n_points;
  t.n_nodes = (unsigned int)n;
  t.bump = bump;
  t.chunks_bumped = chunks;
  t.pool_top = 0;
  t.st_points = snap->n_points;
  t.st_voxels = snap->n_voxels;
  const Ctx& c = h->ctx;
  if (cudaMemcpy(c.child, child.data(), 4 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c.gridref, gridref.data(), 4 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c.num, num.data(), 4 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c.cnt, zeros.data(), 4 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c.scur, zeros.data(), 4 * n, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c.meta, meta.data(), sizeof(NodeMeta) * n, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      (bump && cudaMemcpy(c.data, data.data(), bump, cudaMemcpyHostToDevice) != cudaSuccess) ||
      cudaMemcpy(c.ctl, &t, sizeof(Ctl), cudaMemcpyHostToDevice) != cudaSuccess)
    return poison(h, SIMLOD_ERR_CUDA);
  h->base = snap->n_points;
  h->n_nodes = (uint32_t)n;
  h->mirror_stale = false;
  h->rejected_async_seen = 0;
  h->last_stream = s;
  return SIMLOD_OK;
}

SIMLOD_API int simlod_reset(simlod_t* h, void* stream) {
  if (!h) return SIMLOD_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // a poisoned update may have left claims in the table
  const bool dirty = h->sticky != 0;
  if (dirty) cudaStreamSynchronize(h->last_stream);
  return init_octree(h, s, dirty, dirty);
}

SIMLOD_API int simlod_sync(simlod_t* h) {
  if (!h) return SIMLOD_ERR_INVALID_ARG;
  if (h->sticky) return SIMLOD_ERR_POISONED;
  return finish_fused(h, nullptr);
}

SIMLOD_API int simlod_get_stats(simlod_t* h, simlod_stats* out) {
  if (!h || !out) return SIMLOD_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  int rc = read_ctl(h, h->last_stream);
  if (rc) return rc;
  const Ctl& t = *h->ctl_host;
  out->batches = t.st_batches;
  out->points = t.st_points;
  out->rejected_batches = t.st_rejected;
  out->spilled = t.st_spilled;
  out->splits = t.st_splits;
  out->voxels = t.st_voxels;
  out->iterations_max = t.st_iter_max;
  out->rounds = t.st_rounds;
  out->nodes = t.n_nodes;
  out->chunks_bumped = t.chunks_bumped;
  out->chunks_pool = t.pool_top > 0 ? (uint64_t)t.pool_top : 0;
  out->arena_bytes = h->arena_bytes;
  out->data_bytes = h->lay.data_bytes;
  out->data_used = t.bump;
  out->last_points = t.last_points;
  out->last_spilled = t.last_spilled;
  out->last_splits = t.last_splits;
  out->last_voxels = t.last_voxels;
  out->last_iterations = t.last_iters;
  out->sticky_status = h->sticky;
  out->device_error_bits = t.error;
  out->render_nodes = t.vis_count;
  out->render_samples = t.render_samples;
  out->compact_nodes = t.compact_now;
  out->compact_chunks = t.compact_chunks_now;
  out->compacted_total = t.st_compacted;
  out->compact_chunks_freed = t.st_compact_chunks;
  out->decompacted_total = t.st_decompacted;
  return SIMLOD_OK;
}

SIMLOD_API int simlod_compact(simlod_t* h, uint32_t idle_updates, void* stream) {
  if (!h) return SIMLOD_ERR_INVALID_ARG;
  if (h->sticky) return SIMLOD_ERR_POISONED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  h->last_stream = s;
  const Ctx& c = h->ctx;
  k_compact<<<(unsigned)h->sm_count * 4, BLOCK, 0, s>>>(c, idle_updates);
  return cudaGetLastError() == cudaSuccess ? SIMLOD_OK : poison(h, SIMLOD_ERR_CUDA);
}

SIMLOD_API int simlod_render(simlod_t* h, const float view_proj[16], uint32_t width,
                             uint32_t height, uint64_t* d_framebuffer, int clear,
                             void* cuda_stream) {
  if (!h || !view_proj || !d_framebuffer || width == 0 || height == 0 ||
      (reinterpret_cast<uintptr_t>(d_framebuffer) & 7u) ||
      (uint64_t)width * height > (1ull << 32))
    return SIMLOD_ERR_INVALID_ARG;
  if (h->sticky) return SIMLOD_ERR_POISONED;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  h->last_stream = s;
  View v;
  for (int k = 0; k < 16; ++k) v.m[k] = view_proj[k];
  v.W = (float)width;
  v.H = (float)height;
  v.lod = (float)(1u << h->cfg.grid_log2);
  v.width = width;
  v.height = height;
  const Ctx& c = h->ctx;
  uint32_t* vis = reinterpret_cast<uint32_t*>(h->arena + h->lay.vis);
  unsigned long long* fb = reinterpret_cast<unsigned long long*>(d_framebuffer);
  if (cudaMemsetAsync(&c.ctl->vis_count, 0, sizeof(unsigned int), s) != cudaSuccess ||
      cudaMemsetAsync(&c.ctl->render_samples, 0, sizeof(unsigned long long), s) != cudaSuccess)
    return SIMLOD_ERR_CUDA;
  const unsigned grid = (unsigned)h->sm_count * 4;
  return launch(h, K_RENDER, s, [&] {
    if (clear) k_fb_clear<<<grid, BLOCK, 0, s>>>(fb, (uint64_t)width * height);
    k_render_select<<<grid, BLOCK, 0, s>>>(c, v, vis);
    k_render_draw<<<grid * 2, BLOCK, 0, s>>>(c, v, vis, fb);
  });
}

SIMLOD_API int simlod_snapshot(simlod_t* h, simlod_snapshot_t* snap) {
  if (!h || !snap) return SIMLOD_ERR_INVALID_ARG;
  if (h->sticky) return SIMLOD_ERR_POISONED;
  cudaStream_t s = h->last_stream;
  int rc = read_ctl(h, s);
  if (rc) return poison(h, rc);
  const Ctl t = *h->ctl_host;
  if (t.error) return poison(h, error_from_bits(t.error));
  const uint32_t n = t.n_nodes;
  std::vector<uint32_t> child(n), num(n);
  std::vector<NodeMeta> meta(n);
  std::vector<uint8_t> data(t.bump);
  const Ctx& c = h->ctx;
  if (cudaMemcpy(child.data(), c.child, 4ull * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(num.data(), c.num, 4ull * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(meta.data(), c.meta, sizeof(NodeMeta) * n, cudaMemcpyDeviceToHost) !=
          cudaSuccess ||
      (t.bump && cudaMemcpy(data.data(), c.data, t.bump, cudaMemcpyDeviceToHost) != cudaSuccess))
    return poison(h, SIMLOD_ERR_CUDA);
  uint64_t np = 0, nv = 0;
  for (uint32_t i = 0; i < n; ++i) (child[i] == NONE ? np : nv) += num[i];
  snap->n_nodes = n;
  snap->n_points = np;
  snap->n_voxels = nv;
  if (!snap->nodes && !snap->points && !snap->voxels) return SIMLOD_OK;
  if (!snap->nodes || snap->nodes_capacity < n || (np && (!snap->points ||
      snap->points_capacity < np)) || (nv && (!snap->voxels || snap->voxels_capacity < nv)))
    return SIMLOD_ERR_INVALID_ARG;
  const uint32_t C = h->cfg.chunk_points, G = h->cfg.grid_log2;
  struct Key {
    uint32_t level, ix, iy, iz, id;
  };
  std::vector<Key> keys(n);
  for (uint32_t i = 0; i < n; ++i) {
    const uint32_t L = h->cfg.root_log2 - meta[i].level;
    keys[i] = {meta[i].level,
               (uint32_t)(((long long)meta[i].min[0] - h->cfg.root_min[0]) >> L),
               (uint32_t)(((long long)meta[i].min[1] - h->cfg.root_min[1]) >> L),
               (uint32_t)(((long long)meta[i].min[2] - h->cfg.root_min[2]) >> L), i};
  }
  std::sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
    if (a.level != b.level) return a.level < b.level;
    if (a.ix != b.ix) return a.ix < b.ix;
    if (a.iy != b.iy) return a.iy < b.iy;
    return a.iz < b.iz;
  });
  const uint64_t chunk_bytes = chunk_bytes_of(&h->cfg);
  uint64_t po = 0, vo = 0;
  int bad = 0;
  for (uint32_t k = 0; k < n; ++k) {
    const uint32_t i = keys[k].id;
    const NodeMeta& m = meta[i];
    const bool inner = child[i] != NONE;
    simlod_node_rec& r = snap->nodes[k];
    r.level = m.level;
    r.is_inner = inner ? 1u : 0u;
    r.min[0] = m.min[0];
    r.min[1] = m.min[1];
    r.min[2] = m.min[2];
    r.log2size = h->cfg.root_log2 - m.level;
    r.n_points = inner ? 0 : num[i];
    r.n_voxels = inner ? num[i] : 0;
    uint64_t walked = 0, idx = 0;
    if (m.compact) {  // one contiguous array (simlod_compact)
      const uint64_t off = (uint64_t)m.head * REF_BYTES;
      const uint64_t cap = num[i];
      if (m.head == NONE || off + CHUNK_HEADER + 20 * cap > data.size()) {
        bad = 1;
      } else {
        const int4* recs = reinterpret_cast<const int4*>(data.data() + off + CHUNK_HEADER);
        const uint32_t* aux =
            reinterpret_cast<const uint32_t*>(data.data() + off + CHUNK_HEADER + 16 * cap);
        for (; idx < cap; ++idx) {
          const int4 v = recs[idx];
          if (inner) {
            snap->voxels[vo + idx] = simlod_voxel_rec{aux[idx], v.x, v.y, v.z, (uint32_t)v.w};
          } else {
            snap->points[po + idx] = simlod_point_rec{v.x, v.y, v.z, (uint32_t)v.w, aux[idx]};
          }
        }
      }
      walked = (num[i] + C - 1) / C;  // the chunks the node would take
    }
    // walk the linked list, as a renderer would (Section 6)
    for (uint32_t ref = m.compact ? NONE : m.head; ref != NONE && walked <= m.n_chunks;
         ++walked) {
      const uint64_t off = (uint64_t)ref * REF_BYTES;
      if (off + chunk_bytes > data.size()) {
        bad = 1;
        break;
      }
      const uint8_t* ch = data.data() + off;
      const int4* recs = reinterpret_cast<const int4*>(ch + CHUNK_HEADER);
      const uint32_t* aux = reinterpret_cast<const uint32_t*>(ch + CHUNK_HEADER + 16ull * C);
      for (uint32_t q = 0; q < C && idx < num[i]; ++q, ++idx) {
        const int4 v = recs[q];
        if (inner) {
          snap->voxels[vo + idx] = simlod_voxel_rec{aux[q], v.x, v.y, v.z, (uint32_t)v.w};
        } else {
          snap->points[po + idx] = simlod_point_rec{v.x, v.y, v.z, (uint32_t)v.w, aux[q]};
        }
      }
      ref = *reinterpret_cast<const uint32_t*>(ch);
    }
    if (idx != num[i]) bad = 1;
    r.n_chunks = walked;
    if (inner) {
      std::sort(snap->voxels + vo, snap->voxels + vo + num[i],
                [](const simlod_voxel_rec& a, const simlod_voxel_rec& b) { return a.cell < b.cell; });
      vo += num[i];
    } else {
      std::sort(snap->points + po, snap->points + po + num[i],
                [](const simlod_point_rec& a, const simlod_point_rec& b) { return a.gidx < b.gidx; });
      po += num[i];
    }
  }
  (void)G;
  return bad ? SIMLOD_ERR_CUDA : SIMLOD_OK;
}

SIMLOD_API int simlod_set_timing(simlod_t* h, int enable, int clear) {
  if (!h) return SIMLOD_ERR_INVALID_ARG;
  if (clear) {
    cudaStreamSynchronize(h->last_stream);
    harvest_timing(h);
    memset(h->launches, 0, sizeof(h->launches));
    memset(h->ms, 0, sizeof(h->ms));
    if (read_ctl(h, h->last_stream) == SIMLOD_OK)
      for (int k = 0; k < SIMLOD_N_PHASES; ++k) h->phase_ns_cleared[k] = h->ctl_host->phase_ns[k];
  }
  h->timing = enable != 0;
  return SIMLOD_OK;
}

SIMLOD_API int simlod_get_timing(simlod_t* h, simlod_timing* out) {
  if (!h || !out) return SIMLOD_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(h->last_stream) != cudaSuccess) return SIMLOD_ERR_CUDA;
  harvest_timing(h);
  for (int k = 0; k < SIMLOD_N_KERNELS; ++k) {
    out->name[k] = kKernelNames[k];
    out->launches[k] = h->launches[k];
    out->ms[k] = h->ms[k];
  }
  static const char* const kPhaseNames[SIMLOD_N_PHASES] = {
      "count", "decide", "advance", "store", "end", "rollback", "launch", "other"};
  int rc = read_ctl(h, h->last_stream);
  if (rc) return rc;
  for (int k = 0; k < SIMLOD_N_PHASES; ++k) {
    out->phase_name[k] = kPhaseNames[k];
    out->phase_ms[k] = (h->ctl_host->phase_ns[k] - h->phase_ns_cleared[k]) * 1e-6;
  }
  return SIMLOD_OK;
}

SIMLOD_API int simlod_destroy(simlod_t* h) {
  if (!h) return SIMLOD_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->last_stream);
  harvest_timing(h);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->ctl_host) cudaFreeHost(h->ctl_host);
  if (h->desc_host) cudaFreeHost(h->desc_host);
  if (h->fctl_host) cudaFreeHost(h->fctl_host);
  if (h->one_host) cudaFreeHost(h->one_host);
  if (h->prog_host) cudaFreeHost(h->prog_host);
  if (h->desc_done) cudaEventDestroy(h->desc_done);
  if (h->flags_clear) cudaEventDestroy(h->flags_clear);
  delete h;
  return SIMLOD_OK;
}

SIMLOD_API const char* simlod_status_string(int status) {
  switch (status) {
    case SIMLOD_OK: return "ok";
    case SIMLOD_ERR_INVALID_ARG: return "invalid argument";
    case SIMLOD_ERR_OUT_OF_BOUNDS: return "point outside the root cube: batch rejected";
    case SIMLOD_ERR_ARENA_FULL: return "arena data region exhausted";
    case SIMLOD_ERR_BACKLOG_FULL: return "voxel backlog capacity exceeded";
    case SIMLOD_ERR_SPILL_FULL: return "spill buffer capacity exceeded";
    case SIMLOD_ERR_ITER_CAP: return "expansion iteration cap reached";
    case SIMLOD_ERR_TIMEOUT: return "bounded device wait timed out";
    case SIMLOD_ERR_POISONED: return "handle poisoned by an earlier device error";
    case SIMLOD_ERR_CUDA: return "CUDA runtime error";
    case SIMLOD_ERR_NODES_FULL: return "node table exhausted";
    case SIMLOD_ERR_TOO_MANY_POINTS: return "more than 2^32 points in one octree";
    default: return "unknown status";
  }
}

}  // extern "C"
