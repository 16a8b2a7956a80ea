// hb_inst_relay.cu -- instantiates the relay form of the fused kernel for every launch shape.
#include "hb_hash_kernels.cuh"

namespace hb {

KernelFn relay_fn(int shape) {
#define HB_RELAY_CASE(i, w, st, kb, co) \
  case i: return hb_relay_kernel<w, st, kb, co>;
  switch (shape) {
    HB_SHAPES(HB_RELAY_CASE)
    default: return nullptr;
  }
#undef HB_RELAY_CASE
}

}  // namespace hb
