// hb_inst_sha1.cu -- instantiates the SHA-1 kernels for every launch shape.
#include "hb_hash_kernels.cuh"

namespace hb {
template KernelFn plain_fn<HB_SHA1>(int);
}  // namespace hb
