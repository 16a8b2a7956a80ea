// hb_noalloc.cu -- hash_batch_mixed_noalloc: the ragged (per-message
// algorithm) path for callers that cannot allocate device memory.
//
// Who needs it.  hash_batch_mixed grows a scratch area with cudaMalloc the
// first time it sees a larger batch, and keeps a per-device context that is
// itself allocated on first use.  Some callers cannot let that happen: a
// process whose device memory is handed out by another owner under a fixed
// budget (an allocation outside that owner would fail or break its
// accounting), or a latency-critical loop that must never hit the implicit
// device-wide synchronisation a cudaMalloc/cudaFree can cause.  This entry
// point does the same work with a fixed scratch area compiled into the
// library instead: a file-scope __device__ array that every GPU which loads
// the library holds until the process exits.  It never calls cudaMalloc,
// cudaFree or any allocating routine.
//
// The array is shared by every call on a device and keeps whatever the last
// call left in it; the bucketing step clears the counters it needs at the
// start of each call, and every permutation entry is rewritten before it is
// read.  Calls whose work overlaps on the GPU (for example on two streams
// without ordering between them) use the same array and race: order them.
//
// Device-detected errors.  The kernels record HB_DEV_* bits in a status word
// at the start of the array (the library's per-device status word lives in a
// context that is allocated on first use, so this path cannot use it).
// hash_device_status() reads that word with a plain device-to-host copy, ORs
// it into what it returns and clears it, so a caller sees these bits where it
// sees every other entry point's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "hashbatch.h"
#include "hb_launch.h"

namespace {

constexpr uint64_t kMaxMessages = HB_NOALLOC_MAX_MESSAGES;
constexpr int kShape = hb::kDefaultMixedShape;  // launch shape; digests do not depend on it
constexpr size_t kStatusBytes = 256;  // status word, kept in its own 256-byte line
constexpr size_t kScratchBytes =
    kStatusBytes + sizeof(hb::MixedWorkspace) + (kMaxMessages + 31ull * hb::kGroups) * sizeof(uint32_t);

// The scratch area.  Host code must not use this name as an address: on the
// host it is only a stand-in for the symbol; its device address comes from
// cudaGetSymbolAddress, below.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
  bool ready = false;
  uint8_t* scratch = nullptr;  // device address of g_noalloc_scratch
  int sms = 0;
  int blocks_per_sm = 0;       // occupancy of the persistent kernel
};

std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

// Once per device, with that device current: look up the device address of
// the scratch array and the launch limits.  None of these calls allocates.
int setup_current_device(DeviceSetup** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HB_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
      return HB_ERR_CUDA;
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return HB_ERR_CUDA;
    if (hb::prepare_kernel(true, 0, kShape, &occ) != cudaSuccess) return HB_ERR_CUDA;
    s.scratch = static_cast<uint8_t*>(p);
    s.sms = sms;
    int warps = 0, stages = 0;
    hb::shape_desc(kShape, &warps, &stages);
    s.blocks_per_sm = std::max(1, std::min(occ, hb::kDefaultMixedWarpsPerSm / warps));
    s.ready = true;
  }
  *out = &s;
  return HB_OK;
}

}  // namespace

namespace hb {
cudaError_t noalloc_take_status(int* bits) {
  *bits = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  const DeviceSetup& s = g_setup[dev];
  if (!s.ready) return cudaSuccess;  // never ran here: nothing recorded
  int v = 0;
  e = cudaMemcpy(&v, s.scratch, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v != 0) e = cudaMemset(s.scratch, 0, sizeof(int));
  if (e == cudaSuccess) *bits = v;
  return e;
}
}  // namespace hb

extern "C" int hash_batch_mixed_noalloc(const uint8_t* algs, const uint8_t* packed_bytes,
                                        const uint64_t* offsets, const uint32_t* lengths,
                                        uint64_t n, uint8_t* digests_out, void* stream) {
  if (n == 0) return HB_OK;
  if (n > kMaxMessages) return HB_ERR_TOO_LARGE;
  if (!algs || !packed_bytes || !offsets || !lengths || !digests_out) return HB_ERR_NULL;
  if (reinterpret_cast<uintptr_t>(digests_out) & 15u) return HB_ERR_ALIGN;
  DeviceSetup* s = nullptr;
  int rc = setup_current_device(&s);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  int* status = reinterpret_cast<int*>(s->scratch);
  hb::MixedWorkspace* ws = reinterpret_cast<hb::MixedWorkspace*>(s->scratch + kStatusBytes);
  uint32_t* perm = reinterpret_cast<uint32_t*>(s->scratch + kStatusBytes + sizeof(hb::MixedWorkspace));

  hb::MixedArgs m{};
  m.cfg = hb::kDefaultBuckets;
  m.algs = algs;
  m.lengths = lengths;
  m.n = n;
  m.n_dev = nullptr;
  m.digests = digests_out;
  m.ws = ws;
  m.perm = perm;
  const uint64_t need = (n + 255) / 256;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)s->sms * 8));
  // Zeroes the group counters, then bucketing; the scan step resets the
  // cursors and the chunk counter, the scatter and scan steps rewrite every
  // permutation entry that the hashing kernel reads.
  if (hb::launch_bucketing(m, grid, st) != cudaSuccess) return HB_ERR_CUDA;

  hb::KernelArgs a{};
  a.packed = packed_bytes;
  a.offsets = offsets;
  a.lengths = lengths;
  a.algs = algs;
  a.perm = perm;
  a.chunk_counter = &ws->chunk_counter;
  a.nchunks = &ws->nchunks;
  a.early = ws->early;
  a.n = n;
  a.digests = digests_out;
  a.status = status;
  a.abort_flag = nullptr;
  a.wait_limit_ns = hb::wait_limit_ns();
  a.mc = hb::make_mul_consts();
  if (hb::launch_hash(true, 0, kShape, s->sms * s->blocks_per_sm, a, st) != cudaSuccess)
    return HB_ERR_CUDA;
  return HB_OK;
}
