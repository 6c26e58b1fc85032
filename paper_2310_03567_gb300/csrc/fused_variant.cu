// One more instance of the persistent update kernel (k_fused), compiled with
// other launch-shape knobs than the instance built into simlod.cu: threads
// per block, resident blocks per SM, node-cache entries, store unroll and
// descent group (SL_PHASE_BLOCK, SL_PHASE_MIN_BLOCKS, SL_NODE_CACHE,
// SL_STORE_UNROLL, SL_DESCENT_GROUP). The build compiles this file once per
// instance with those values, a namespace of its own (SL_NS) and the names of
// its two entry points (SL_VARIANT_INFO, SL_VARIANT_LAUNCH); the host code of
// simlod.cu calls them through variant.h. The arithmetic is the same in every
// instance, so every instance builds the same octree.
#if !defined(SL_NS) || !defined(SL_VARIANT_INFO) || !defined(SL_VARIANT_LAUNCH)
#error "fused_variant.cu is built once per kernel instance, with SL_NS and its entry names"
#endif

#include <cuda_runtime.h>

#include <cstring>

#include "fused.cuh"
#include "variant.h"

using namespace SL_NS;

extern "C" int SL_VARIANT_INFO(sl_variant_info* out) {
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

extern "C" int SL_VARIANT_LAUNCH(const sl_fused_launch* a) {
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
