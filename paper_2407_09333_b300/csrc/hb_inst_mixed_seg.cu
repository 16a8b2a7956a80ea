// hb_inst_mixed_seg.cu -- instantiates the persistent ragged kernels over segments for every launch shape.
#include "hb_hash_kernels.cuh"

namespace hb {
template KernelFn mixed_fn<true>(int);
}  // namespace hb
