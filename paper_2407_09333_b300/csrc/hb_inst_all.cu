// hb_inst_all.cu -- instantiates the fused three-algorithm kernels for every launch shape.
#include "hb_hash_kernels.cuh"

namespace hb {
template KernelFn plain_fn<HB_ALL>(int);
}  // namespace hb
