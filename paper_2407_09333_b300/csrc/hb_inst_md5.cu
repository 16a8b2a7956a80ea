// hb_inst_md5.cu -- instantiates the MD5 kernels for every launch shape.
#include "hb_hash_kernels.cuh"

namespace hb {
template KernelFn plain_fn<HB_MD5>(int);
}  // namespace hb
