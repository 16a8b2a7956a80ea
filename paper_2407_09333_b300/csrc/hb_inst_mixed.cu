// hb_inst_mixed.cu -- instantiates the persistent ragged kernels for every launch shape.
#include "hb_hash_kernels.cuh"

namespace hb {
template KernelFn mixed_fn<false>(int);
}  // namespace hb
