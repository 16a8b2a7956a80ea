// hb_hash_kernels.cuh -- the hashing kernels (fixed-algorithm and persistent
// ragged), the table of launch shapes they are instantiated for, and the
// functions that map a shape index to a kernel.  Each instantiation table is
// compiled in its own translation unit (hb_inst_*.cu) so the library builds
// in parallel; hb_kernels.cu launches them.
#pragma once

#include <cstdint>

#include "hb_launch.h"
#include "hb_pipeline.cuh"

namespace hb {

// ---------------------------------------------------------------------------
// Fixed-algorithm kernel.

template <int ALG, int WARPS, int STAGES, int KB, bool COOP>
__global__ void __launch_bounds__(WARPS * 32) hb_plain_kernel(KernelArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  if (a.abort_flag && *a.abort_flag) return;
  uint8_t* wsm = smem + warp * WarpSmem<STAGES, KB>::kBytes;
  const uint64_t gwarp = (uint64_t)blockIdx.x * WARPS + warp;
  const uint64_t nwarps = (uint64_t)gridDim.x * WARPS;
  StaticSource<ALG> src(a, gwarp, nwarps, lane);
  warp_pipeline<STAGES, KB, COOP, ALG, false, false>(src, wsm, a, lane);
}

// The fused kernel's relay form (few long messages): persistent; warps take
// (segment, chunk) items and pass chains on between segments (RelaySource).
template <int WARPS, int STAGES, int KB, bool COOP>
__global__ void __launch_bounds__(WARPS * 32) hb_relay_kernel(KernelArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  if (a.abort_flag && *a.abort_flag) return;
  uint8_t* wsm = smem + warp * WarpSmem<STAGES, KB, false, true>::kBytes;
  RelaySource src(a, lane);
  warp_pipeline<STAGES, KB, COOP, HB_ALL, false, false, true>(src, wsm, a, lane);
}

// SEG: messages arrive as segments (a.seg), see hb_pipeline.cuh.
template <int WARPS, int STAGES, int KB, bool COOP, bool SEG>
__global__ void __launch_bounds__(WARPS * 32) hb_mixed_kernel(KernelArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warp = threadIdx.x >> 5;
  if (a.abort_flag && *a.abort_flag) return;
  uint8_t* wsm = smem + warp * WarpSmem<STAGES, KB, SEG>::kBytes;
  DynamicSource<SEG> src(a, lane, (uint64_t)blockIdx.x * WARPS + warp);
  warp_pipeline<STAGES, KB, COOP, HB_MD5, true, SEG>(src, wsm, a, lane);
}

// Launch shapes: (warps per block, stages in flight per warp, blocks per
// stage, cooperative copies).  The table is the single list every kernel is
// instantiated for.
#define HB_SHAPES(X)     \
  X(0, 4, 4, 1, false)   \
  X(1, 4, 2, 1, false)   \
  X(2, 8, 3, 1, false)   \
  X(3, 1, 4, 1, false)   \
  X(4, 2, 3, 1, false)   \
  X(5, 16, 2, 1, false)  \
  X(6, 8, 2, 4, false)   \
  X(7, 4, 3, 4, false)   \
  X(8, 8, 2, 2, false)   \
  X(9, 4, 2, 4, false)   \
  X(10, 4, 3, 4, true)   \
  X(11, 8, 2, 4, true)   \
  X(12, 16, 2, 1, true)  \
  X(13, 4, 4, 1, true)   \
  X(14, 8, 2, 2, true)   \
  X(15, 8, 3, 2, true)   \
  X(16, 4, 3, 2, true)   \
  X(17, 4, 4, 2, true)   \
  X(18, 1, 3, 4, true)   \
  X(19, 1, 2, 4, true)   \
  X(20, 1, 4, 2, true)   \
  X(21, 1, 2, 2, true)   \
  X(22, 1, 3, 2, true)   \
  X(23, 2, 2, 2, true)   \
  X(24, 4, 2, 4, true)   \
  X(25, 2, 2, 4, true)

struct ShapeDesc {
  int warps, stages, kb;
  bool coop;
};
#define HB_SHAPE_DESC(i, w, st, kb, co) {w, st, kb, co},

using KernelFn = void (*)(KernelArgs);

// Kernel of launch shape `shape` for one algorithm (HB_ALL: the fused
// kernel), nullptr outside the table.
template <int ALG>
KernelFn plain_fn(int shape) {
#define HB_PLAIN_CASE(i, w, st, kb, co) \
  case i: return hb_plain_kernel<ALG, w, st, kb, co>;
  switch (shape) {
    HB_SHAPES(HB_PLAIN_CASE)
    default: return nullptr;
  }
#undef HB_PLAIN_CASE
}

// The relay form of the fused kernel of launch shape `shape` (hb_inst_relay.cu).
KernelFn relay_fn(int shape);

// The persistent ragged kernel of launch shape `shape` (SEG: over segments).
template <bool SEG>
KernelFn mixed_fn(int shape) {
#define HB_MIXED_CASE(i, w, st, kb, co) \
  case i: return hb_mixed_kernel<w, st, kb, co, SEG>;
  switch (shape) {
    HB_SHAPES(HB_MIXED_CASE)
    default: return nullptr;
  }
#undef HB_MIXED_CASE
}

}  // namespace hb
