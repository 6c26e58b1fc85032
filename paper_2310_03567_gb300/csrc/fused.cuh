// Fused form of the update: one persistent cooperative launch runs every
// phase of every batch in a list, with grid-wide barriers between phases
// instead of kernel boundaries and host round trips. This is the paper's
// own kernel organisation (Section 4: persistent threads and grid syncs,
// the update kernel looping over the batches uploaded so far), with the
// phases of device.cuh.
//
// Barriers are bounded: a block that waits longer than the handle's barrier
// limit (Ctx::bar_ns, 2 s unless the caller sets another) marks the launch
// aborted and returns, the others see the abort flag (or time out themselves)
// and return as well; the host then reads a TIMEOUT status. Nothing spins
// without a limit.
#pragma once

#include "device.cuh"

namespace SL_NS {

constexpr unsigned long long FUSED_BARRIER_NS = 2000000000ull;  // default barrier limit: 2 s
constexpr unsigned long long FUSED_READY_NS = 2000000000ull;    // default ready limit: 2 s per batch
constexpr int FUSED_BLOCK = PHASE_BLOCK;
constexpr unsigned long long NO_BUDGET = ~0ull;
constexpr uint32_t MAX_FUSED_BATCHES = 16384;

// One update of the fused launch: n points at pts, or, with nseg > 0, the
// segments [seg0, seg0 + nseg) of the segment table, gathered into the
// staging buffer first (a merged update of several batches).
struct BatchDesc {
  const int4* pts;
  unsigned long long n;
  uint32_t seg0, nseg;
};

// A batch inside a merged update: n points at src go to staging[dst, dst + n).
struct PlanSeg {
  const int4* src;
  uint32_t n, dst;
};

// Per-launch control words of the fused kernel (arena).
struct FusedCtl {
  // block arrivals at grid barriers since the launch began (gridDim.x per
  // barrier); bit 63 (BAR_ABORT) aborts the launch
  unsigned long long bar;
  unsigned int consumed;  // batches fully handled (applied or rejected)
  unsigned int stop;      // the frame budget ran out
  unsigned int rejected;  // batches rejected in this launch
  unsigned int pad[11];
};
static_assert(sizeof(FusedCtl) == 64, "FusedCtl size");

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier with a time limit. Thread 0 of each block publishes the
// block's writes (fence, then one atomic add on the launch's arrival count)
// and waits until the count reaches the end of this barrier's generation;
// the last block to arrive waits for nothing. A device error sets the abort
// bit of the same word (set_error), so a waiting block sees it in the value
// it polls and an arriving block in the value its add returns: every block
// leaves at its next barrier, and all blocks that run a phase have seen the
// previous phase complete. Returns false when the launch was aborted.
//
// view != nullptr: thread 0 also reads the control values that the code after
// this barrier needs (all written before it, none written again before the
// next one) into the block's shared copy, so that one load per block, not
// one per warp, reaches the control block's L2 lines.
struct CtlView {
  unsigned long long base;
  uint32_t n_nodes, reject, split_count, ntasks, spill_count, nkeys, stop;
  int pool_top;
  uint32_t mv_count[2];
};

__device__ __forceinline__ bool grid_barrier(const Ctx& c, FusedCtl* f, CtlView* view = nullptr) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long* w = &f->bar;
    unsigned long long v;
    asm volatile(
        "fence.acq_rel.gpu;\n\t"
        "atom.relaxed.gpu.global.add.u64 %0, [%1], 1;"
        : "=l"(v)
        : "l"(w)
        : "memory");
    const unsigned long long g = gridDim.x;
    const unsigned long long target = ((v & ~BAR_ABORT) / g + 1ull) * g;
    int ok = (v & BAR_ABORT) == 0ull;
    if (ok && (v & ~BAR_ABORT) + 1ull < target) {
      const unsigned long long t0 = globaltimer_ns();
      for (uint32_t k = 1;; ++k) {
        asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(w) : "memory");
        if (v & BAR_ABORT) {
          ok = 0;
          break;
        }
        if (v >= target) break;
        if ((k & 15u) == 0u && globaltimer_ns() - t0 > c.bar_ns) {
          set_error(c, E_TIMEOUT);  // also sets the abort bit
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
#if SL_CTL_VIEW
    if (ok && view) {
      view->base = vload(&c.ctl->base);
      view->n_nodes = vload(&c.ctl->n_nodes);
      view->reject = vload(&c.ctl->reject);
      view->split_count = vload(&c.ctl->split_count);
      view->ntasks = vload(&c.ctl->ntasks);
      view->spill_count = vload(&c.ctl->spill_count);
      view->nkeys = vload(&c.ctl->nkeys);
      view->pool_top = vload(&c.ctl->pool_top);
      view->mv_count[0] = vload(&c.ctl->mv_count[0]);
      view->mv_count[1] = vload(&c.ctl->mv_count[1]);
      view->stop = vload(&f->stop);
    }
#endif
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Wait until a batch is ready: *flag != 0, written by a copy on another
// stream after the batch's own copy (Section 4: the update kernel handles the
// batches uploaded so far). Thread 0 of each block polls, bounded by
// Ctx::ready_ns; the abort bit ends the wait too. Returns false when the
// launch was aborted.
__device__ __forceinline__ bool wait_ready(const Ctx& c, FusedCtl* f, const unsigned int* flag) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
    if (v == 0u) {
      const unsigned long long t0 = globaltimer_ns();
      for (uint32_t k = 1;; ++k) {
        __nanosleep(128);
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v != 0u) break;
        if (vload(&f->bar) & BAR_ABORT) {
          ok = 0;
          break;
        }
        if ((k & 15u) == 0u && globaltimer_ns() - t0 > c.ready_ns) {
          set_error(c, E_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Phase clock (block 0, thread 0): charge the time since the previous tick
// to `phase`. Called right after a barrier, so it covers the phase and the
// barrier that closed it.
struct PhaseClock {
  unsigned long long t;
  __device__ __forceinline__ void tick(const Ctx& c, int phase) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const unsigned long long now = globaltimer_ns();
      atomicAdd(&c.ctl->phase_ns[phase], now - t);
      t = now;
    }
  }
};

// All batches of `batches`, in order, each one complete update. Before a
// batch other than the first, stop once more than budget_ns has passed since
// the launch began (Section 7.2's frame budget; batches are never cut);
// NO_BUDGET disables the check.
//
// n_dev != nullptr: the number of updates is read from the device (written by
// the planning kernel before this launch) instead of n_batches.
//
// ready != nullptr: update b starts once ready[b] != 0 (its points were copied
// by another stream, which then set the flag).
__global__ void __launch_bounds__(FUSED_BLOCK, PHASE_MIN_BLOCKS) k_fused(Ctx c, const BatchDesc* batches,
                                                        uint32_t n_batches, FusedCtl* f,
                                                        unsigned long long budget_ns,
                                                        uint32_t max_iters,
                                                        const unsigned int* n_dev,
                                                        const PlanSeg* segs,
                                                        const unsigned int* ready) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t warp0 = tid / 32, nwarps = nthreads / 32;
  const unsigned long long t_begin = globaltimer_ns();
  extern __shared__ uint32_t smem[];  // node-table cache (PHASE_SMEM_BYTES)
  PhaseClock clk{t_begin};
  const uint32_t nb = n_dev ? min(vload(n_dev), n_batches) : n_batches;
  // the node-table cache is loaded once and patched after every decide round
  node_cache_load(c, smem, 0, vload(&c.ctl->n_nodes));
#if SL_CTL_VIEW
  __shared__ CtlView cv;  // control values after the last barrier that filled it
  CtlView* const vw = &cv;
#define SL_CV(field, addr) (cv.field)
#else
  CtlView* const vw = nullptr;
#define SL_CV(field, addr) vload(addr)
#endif
  for (uint32_t b = 0; b < nb; ++b) {
    // every value read here was written before the last barrier and is not
    // written again before the next one, so all threads decide alike (the
    // first batch reads them directly: no barrier has filled the view yet)
    if (b ? SL_CV(stop, &f->stop) : vload(&f->stop)) return;
    if (ready && !wait_ready(c, f, ready + b)) return;
    BatchDesc bd = batches[b];
    const unsigned long long base = b ? SL_CV(base, &c.ctl->base) : vload(&c.ctl->base);
    const uint32_t nodes0 = b ? SL_CV(n_nodes, &c.ctl->n_nodes) : vload(&c.ctl->n_nodes);
    bool rejected = false;
    if (bd.nseg && bd.n) {
      // merged update: gather its batches into the staging buffer
      if (bd.n > c.max_batch) {
        if (tid == 0) set_error(c, E_INTERNAL);
        return;
      }
      for (uint32_t k = 0; k < bd.nseg; ++k) {
        const PlanSeg sg = segs[bd.seg0 + k];
        if ((unsigned long long)sg.dst + sg.n > bd.n) continue;
        for (uint64_t i = tid; i < sg.n; i += nthreads) c.staging[sg.dst + i] = __ldg(sg.src + i);
      }
      if (!grid_barrier(c, f)) return;
      clk.tick(c, PH_OTHER);
      bd.pts = c.staging;
    }
    if (bd.n) {
      phase_count1(c, smem, node_cache_at(smem, nodes0), bd.pts, bd.n, base, warp0, nwarps);
      if (!grid_barrier(c, f, vw)) return;
      clk.tick(c, PH_COUNT);
      rejected = SL_CV(reject, &c.ctl->reject) != 0u;  // set only by the count round
      if (rejected) {
        phase_rollback(c, nodes0, tid, nthreads);
        if (!grid_barrier(c, f)) return;  // all have read the flag before it is cleared
        clk.tick(c, PH_ROLLBACK);
        if (tid == 0) {
          phase_end_rejected(c);
          c.ctl->st_rejected_async += 1;
          f->rejected += 1;
        }
      } else {
        // s: split-list range of the previous round, n: nodes it created,
        // t_hi: spill tasks (all made by the first decide round)
        uint32_t s_lo = 0, s_hi = 0, n_lo = 0, n_hi = nodes0, t_hi = 0, iters = 1;
        for (;;) {
          phase_decide(c, s_lo, s_hi, n_lo, n_hi, iters >= 3 ? (int)((iters - 1) & 1u) : -1,
                       warp0, nwarps);
          if (!grid_barrier(c, f, vw)) return;
          clk.tick(c, PH_DECIDE);
          const uint32_t sc = SL_CV(split_count, &c.ctl->split_count);
          const uint32_t nn = SL_CV(n_nodes, &c.ctl->n_nodes);
          const uint32_t nt = SL_CV(ntasks, &c.ctl->ntasks);
          node_cache_patch(c, smem, s_hi, sc, n_hi, nn);  // this round's splits and new nodes
          if (iters == 1) t_hi = nt;
          else if (nt != t_hi && tid == 0) set_error(c, E_INTERNAL);
          if (sc == s_hi) break;
          if (iters >= max_iters) {
            if (tid == 0) set_error(c, E_ITER_CAP);
            return;
          }
          s_lo = s_hi;
          s_hi = sc;
          n_lo = n_hi;
          n_hi = nn;
          const int in_list = iters >= 2 ? (int)((iters - 2) & 1u) : -1;
          const uint32_t n_in =
              in_list >= 0 ? SL_CV(mv_count[in_list], &c.ctl->mv_count[in_list]) : 0u;
          phase_advance(c, smem, node_cache_at(smem, nn), bd.pts, bd.n, base, t_hi, s_lo, s_hi,
                        in_list, n_in, (int)((iters - 1) & 1u), warp0, nwarps);
          ++iters;
          if (!grid_barrier(c, f)) return;
          clk.tick(c, PH_ADVANCE);
        }
        // (the last decide round's barrier filled the view)
        const uint32_t n_tasks = SL_CV(ntasks, &c.ctl->ntasks);
        const uint32_t n_spill = min(SL_CV(spill_count, &c.ctl->spill_count), c.spill_cap);
        const uint32_t n_keys = min(SL_CV(nkeys, &c.ctl->nkeys), c.backlog_cap);
        const int pool_top = SL_CV(pool_top, &c.ctl->pool_top);
        phase_store(c, smem, bd.pts, bd.n, base, n_spill, n_tasks, n_keys, pool_top, tid,
                    nthreads);
        if (!grid_barrier(c, f)) return;
        clk.tick(c, PH_STORE);
        if (tid == 0) phase_end(c, bd.n, iters);
      }
    }
    if (tid == 0) {
      f->consumed = b + 1;
      const bool stop = budget_ns != NO_BUDGET && globaltimer_ns() - t_begin > budget_ns;
      if (stop) f->stop = 1;
      if (c.progress) {
        // the host's counts: only this handle's launches write them, and they
        // run one after another, so thread 0 adds to them by load and store
        if (stop && b + 1u < nb) {
          // the batches after b are dropped for good
          unsigned int d;
          asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(d) : "l"(c.progress + 1)
                       : "memory");
          d += nb - b - 1u;
          asm volatile("st.relaxed.sys.global.u32 [%0], %1;" : : "l"(c.progress + 1), "r"(d)
                       : "memory");
        }
        // batch b is applied (or rejected); the release also publishes the
        // dropped count above
        unsigned int done;
        asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(done) : "l"(c.progress)
                     : "memory");
        asm volatile("st.release.sys.global.u32 [%0], %1;" : : "l"(c.progress), "r"(done + 1u)
                     : "memory");
      }
    }
    if (!grid_barrier(c, f, vw)) return;  // the next batch reads stop, base and n_nodes
    clk.tick(c, PH_END);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    atomicAdd(&c.ctl->phase_ns[PH_LAUNCH], globaltimer_ns() - t_begin);
#undef SL_CV
}

// ------------------------------------------------------------ batched form
//
// Planning of a list of uneven batches on the device, before the fused
// launch: every batch is checked against the root cube (a batch with a point
// outside it is rejected whole, as simlod_insert_batch would), then the valid
// batches are merged, in order, into updates of up to `merge` points. Merging
// consecutive batches gives the octree they would give one by one (the
// octree after a prefix of the stream does not depend on how it was cut into
// batches; Section 5), with fewer expansion rounds and grid barriers.

struct PlanInput {
  const int4* pts;
  unsigned long long n;
};

// Units of 4,096 points over all batches; tile0[k] = first unit of batch k
// (n_in + 1 entries). Sets bad[k] when batch k has a point outside the cube.
__global__ void k_plan_validate(Ctx c, const PlanInput* in, const uint32_t* tile0, uint32_t n_in,
                                unsigned int* bad) {
  const uint32_t units = tile0[n_in];
  for (uint32_t u = blockIdx.x; u < units; u += gridDim.x) {
    uint32_t lo = 0, hi = n_in;  // batch k with tile0[k] <= u < tile0[k + 1]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) / 2;
      if (tile0[mid] <= u) lo = mid;
      else hi = mid;
    }
    const uint32_t k = lo;
    const PlanInput b = in[k];
    const uint64_t first = (uint64_t)(u - tile0[k]) * 4096;
    bool out = false;
    for (uint64_t i = first + threadIdx.x; i < b.n && i < first + 4096; i += blockDim.x) {
      uint32_t rx, ry, rz;
      out |= !rel_coords(c, __ldg(b.pts + i), rx, ry, rz);
    }
    if (__syncthreads_or(out) && threadIdx.x == 0) bad[k] = 1u;
  }
}

// One thread: group the valid batches into updates, count the rejected ones.
__global__ void k_plan_groups(Ctx c, const PlanInput* in, uint32_t n_in, const unsigned int* bad,
                              unsigned long long merge, BatchDesc* groups, PlanSeg* segs,
                              unsigned int* n_groups) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  uint32_t ng = 0, ns = 0, rejected = 0;
  BatchDesc g{nullptr, 0, 0, 0};
  auto close = [&]() {
    if (g.n == 0) return;
    if (g.nseg == 1) {  // a single batch is read in place
      g.pts = segs[g.seg0].src;
      g.nseg = 0;
    }
    groups[ng++] = g;
    g = BatchDesc{nullptr, 0, ns, 0};
  };
  g.seg0 = 0;
  for (uint32_t k = 0; k < n_in; ++k) {
    if (bad[k]) {
      ++rejected;
      continue;
    }
    const unsigned long long n = in[k].n;
    if (n == 0) continue;
    if (g.n && g.n + n > merge) close();
    if (g.nseg == 0) g.seg0 = ns;
    segs[ns++] = PlanSeg{in[k].pts, (uint32_t)n, (uint32_t)g.n};
    g.n += n;
    ++g.nseg;
  }
  close();
  *n_groups = ng;
  if (rejected) {
    c.ctl->st_rejected += rejected;
    c.ctl->st_rejected_async += rejected;
  }
}

}  // namespace SL_NS
