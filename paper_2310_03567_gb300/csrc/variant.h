// Internal interface between the host code (simlod.cu) and the instances of
// the persistent update kernel (k_fused). Every instance is the same kernel
// compiled with other launch-shape knobs; the batched form's autotuner times
// them on the caller's batch list (simlod_plan_autotune). Instance 0 is the
// one built into simlod.cu, the others come from fused_variant.cu, built once
// per instance with its knobs. None of this is part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>

// Knobs and resources of one instance.
struct sl_variant_info {
  uint32_t block;          // threads per block
  uint32_t min_blocks;     // resident blocks per SM the registers are sized for
  uint32_t node_cache;     // node-table entries mirrored in shared memory
  uint32_t store_unroll;   // items per thread in flight in the store phase
  uint32_t descent_group;  // tree levels whose grid words load together
  uint32_t smem_bytes;     // dynamic shared memory per block
  int32_t max_per_sm;      // blocks per SM that fit on this device (0 = none)
};

// Arguments of one k_fused launch; ctx points at a Ctx (ctx_bytes long:
// every instance checks that its Ctx has that size), batches at the device
// batch table, fctl at the launch's control words.
struct sl_fused_launch {
  const void* ctx;
  size_t ctx_bytes;
  const void* batches;
  uint32_t n_batches;
  void* fctl;
  unsigned long long budget_ns;
  uint32_t max_iters;
  const unsigned int* n_dev;
  const void* segs;
  const unsigned int* ready;
  unsigned grid;
  void* stream;
};

// Every instance k (1 .. SL_N_VARIANTS - 1) defines, with C linkage:
//   int sl_fused_variant_info_k(sl_variant_info* out);   // also sets the
//       kernel's shared-memory limit; returns 0 on success
//   int sl_fused_variant_launch_k(const sl_fused_launch* a);  // cooperative
//       launch on a->stream; returns a cudaError_t value
#define SL_N_VARIANTS 4
