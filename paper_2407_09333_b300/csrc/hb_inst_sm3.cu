// hb_inst_sm3.cu -- instantiates the SM3 kernels for every launch shape.
#include "hb_hash_kernels.cuh"

namespace hb {
template KernelFn plain_fn<HB_SM3>(int);
}  // namespace hb
