// hb_capi.cu -- the C-ABI of libhashbatch.so (declared in include/hashbatch.h):
// argument checks, the per-device context, launch-shape selection, the
// host-buffer path and the captured-graph plans of the ragged path.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "hashbatch.h"
#include "hb_launch.h"

using hb::KernelArgs;
using hb::MixedArgs;
using hb::MixedWorkspace;

namespace {

constexpr int kMaxDevices = 64;
constexpr int kMaxShapes = 64;  // capacity of the per-shape occupancy cache
constexpr uint64_t kMaxPlainN = 1ull << 40;
constexpr uint64_t kMaxMixedN = 1ull << 31;
// Host path: the packed bytes go over in up to kHostChunks pieces of at least
// kHostChunkMin bytes, so hashing and the copy-out overlap the copy-in.
constexpr int kHostChunks = 16;
constexpr uint64_t kHostChunkMin = 8ull << 20;

struct DeviceBuf {
  void* p = nullptr;
  size_t cap = 0;
  // Grows to at least `bytes`; the old contents are not kept.
  cudaError_t reserve(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) {
      cudaError_t e = cudaFree(p);  // synchronises the device
      if (e != cudaSuccess) return e;
      p = nullptr;
      cap = 0;
    }
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    cap = want;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

struct Ctx {
  int device = -1;
  int sms = 0;
  int* status = nullptr;                 // device word of HB_DEV_* bits
  int occ_plain[HB_ALL + 1][kMaxShapes] = {};  // resident blocks per SM, 0 = not prepared
  int occ_mixed[kMaxShapes] = {};
  int occ_mixed_seg[kMaxShapes] = {};    // segment-aware variant
  int tune_plain[HB_ALL + 1] = {0, 0, 0, 0, 0};  // index HB_ALL: the fused kernel
  int tune_mixed = hb::kDefaultMixedShape;
  int mixed_warps_per_sm = hb::kDefaultMixedWarpsPerSm;  // 0 = full occupancy
  hb::BucketCfg buckets = hb::kDefaultBuckets;
  DeviceBuf ws;                          // ragged-path scratch
  cudaEvent_t ws_event = nullptr;        // last use of `ws`
  bool ws_used = false;
  // relay form of the fused kernel: item counter and longest length (16
  // bytes, allocated with the context), its last use, segment blocks (0 = off)
  uint32_t* relay = nullptr;
  cudaEvent_t relay_event = nullptr;
  bool relay_used = false;
  int occ_relay[kMaxShapes] = {};
  int relay_seg_blocks = (int)hb::kDefaultRelaySegBlocks;
  // host-buffer path
  DeviceBuf h_packed, h_off, h_len, h_algs, h_dig, h_flag, h_cmp;
  int* flag_host = nullptr;              // pinned: [0] bounds, [1] ends not monotone
  // pipelined host path: hashing and copy-out streams, per-chunk events
  cudaStream_t host_hash = nullptr, host_out = nullptr;
  cudaEvent_t ev_meta = nullptr, ev_end = nullptr;
  cudaEvent_t ev_in[kHostChunks] = {}, ev_hashed[kHostChunks] = {};
  // windowed host path: two windows, each one device buffer
  DeviceBuf win[2];
  cudaEvent_t ev_win_out[2] = {};
};

std::mutex g_mu;
Ctx* g_ctx[kMaxDevices] = {};
uint64_t g_wait_limit_ns = 2000000000ull;
uint64_t g_host_limit = 0;  // device bytes the host path may use; 0 = no limit

thread_local cudaError_t g_last_cuda_error = cudaSuccess;

int cuda_fail(cudaError_t e) {
  g_last_cuda_error = e;
  return e == cudaErrorMemoryAllocation ? HB_ERR_NOMEM : HB_ERR_CUDA;
}

// The current device's context, created on first use (this first call
// allocates and must not happen inside a stream capture).
int get_ctx(Ctx** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return cuda_fail(cudaGetLastError());
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ctx[dev]) {
    Ctx* c = new Ctx();
    c->device = dev;
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaMalloc(&c->status, sizeof(int)) != cudaSuccess ||
        cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->relay, 4 * sizeof(uint32_t)) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ws_event, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->relay_event, cudaEventDisableTiming) != cudaSuccess ||
        cudaHostAlloc(&c->flag_host, 2 * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
      delete c;
      return cuda_fail(cudaGetLastError());
    }
    g_ctx[dev] = c;
  }
  *out = g_ctx[dev];
  return HB_OK;
}

int occupancy(Ctx* c, bool mixed, int alg, int shape, int* occ, bool seg = false) {
  if (shape < 0 || shape >= kMaxShapes || shape >= hb::num_shapes()) return HB_ERR_ARG;
  seg = seg && mixed;
  int& slot = seg ? c->occ_mixed_seg[shape] : mixed ? c->occ_mixed[shape] : c->occ_plain[alg][shape];
  if (slot == 0) {
    int b = 0;
    cudaError_t e = hb::prepare_kernel(mixed, alg, shape, &b, seg);
    if (e != cudaSuccess) return cuda_fail(e);
    slot = b > 0 ? b : 1;
  }
  *occ = slot;
  return HB_OK;
}

int check_common(const void* packed, const uint64_t* offsets, const uint32_t* lengths,
                 uint64_t n, const uint8_t* digests) {
  if (!packed || !offsets || !lengths || !digests) return HB_ERR_NULL;
  if (reinterpret_cast<uintptr_t>(digests) & 15u) return HB_ERR_ALIGN;
  (void)n;
  return HB_OK;
}

int launch_plain(Ctx* c, int alg, int shape, int grid, const KernelArgs& a, cudaStream_t s) {
  if (shape < 0 || shape >= hb::num_shapes()) return HB_ERR_ARG;
  int occ = 0;
  int rc = occupancy(c, false, alg, shape, &occ);
  if (rc) return rc;
  int warps = 0, stages = 0;
  hb::shape_desc(shape, &warps, &stages);
  const uint64_t ntasks = (a.n + 31) / 32;
  const uint64_t need = (ntasks + warps - 1) / warps;
  if (grid <= 0) grid = (int)std::min<uint64_t>(need, (uint64_t)c->sms * occ);
  cudaError_t e = hb::launch_hash(false, alg, shape, grid, a, s);
  return e == cudaSuccess ? HB_OK : cuda_fail(e);
}

int grid_for_elementwise(Ctx* c, uint64_t n) {
  const uint64_t need = (n + 255) / 256;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)c->sms * 8));
}

// The relay form of the fused kernel (hb_pipeline.cuh, RelaySource) for a
// batch of between half and eight times as many 32-message chunks as the GPU
// has SM sub-partitions: too few for a grid-stride split to load them evenly.
// Not inside a stream capture (the item counter is per-device scratch,
// ordered between streams by an event).  Returns 1 when it launched, 0 when
// the batch takes the grid-stride kernel, or an HB_ERR_* code.
bool relay_window(const Ctx* c, uint64_t n) {
  const uint64_t nchunks = (n + 31) / 32;
  const uint64_t smsps = 4ull * (uint64_t)c->sms;
  return c->relay_seg_blocks > 0 && nchunks * 2 >= smsps && nchunks <= 8 * smsps;
}

int launch_all_relay(Ctx* c, int shape, const KernelArgs& base, cudaStream_t s) {
  if (shape < 0 || shape >= kMaxShapes || !relay_window(c, base.n)) return 0;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (cap != cudaStreamCaptureStatusNone) return 0;
  int& occ = c->occ_relay[shape];
  if (occ == 0) {
    int b = 0;
    cudaError_t e = hb::prepare_relay(shape, &b);
    if (e != cudaSuccess) return cuda_fail(e);
    occ = b > 0 ? b : 1;
  }
  if (c->relay_used && cudaStreamWaitEvent(s, c->relay_event, 0) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  KernelArgs a = base;
  a.relay = c->relay;
  a.relay_seg_blocks = (uint32_t)c->relay_seg_blocks;
  cudaError_t e = hb::launch_relay_setup(base.lengths, base.n, a.relay_seg_blocks * 64u,
                                         base.digests, c->relay, grid_for_elementwise(c, base.n), s);
  if (e == cudaSuccess) e = hb::launch_relay(shape, c->sms * occ, a, s);
  if (e == cudaSuccess) e = cudaEventRecord(c->relay_event, s);
  if (e != cudaSuccess) return cuda_fail(e);
  c->relay_used = true;
  return 1;
}

// Ragged path on a given workspace (bucketing + persistent kernel).
struct Completion {
  const uint32_t* msg_req = nullptr;
  uint32_t* remaining = nullptr;
  volatile uint32_t* done = nullptr;
};

int launch_mixed(Ctx* c, int shape, int grid, const uint8_t* algs, const uint8_t* packed,
                 const uint64_t* offsets, const uint32_t* lengths, uint64_t n, uint8_t* digests,
                 void* ws, const int* abort_flag, cudaStream_t s, const uint64_t* n_dev = nullptr,
                 const hb::BucketCfg* buckets = nullptr, int warps_per_sm = -1,
                 const Completion* comp = nullptr, const uint64_t* seg = nullptr,
                 const uint32_t* slot_index = nullptr) {
  if (shape < 0 || shape >= hb::num_shapes()) return HB_ERR_ARG;
  MixedArgs m{};
  m.cfg = buckets ? *buckets : c->buckets;
  m.slot_index = slot_index;
  m.algs = algs;
  m.lengths = lengths;
  m.n = n;
  m.n_dev = n_dev;
  m.digests = digests;
  m.ws = static_cast<MixedWorkspace*>(ws);
  m.perm = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + sizeof(MixedWorkspace));
  cudaError_t e = hb::launch_bucketing(m, grid_for_elementwise(c, n), s);
  if (e != cudaSuccess) return cuda_fail(e);
  int occ = 0;
  int rc = occupancy(c, true, 0, shape, &occ, seg != nullptr);
  if (rc) return rc;
  KernelArgs a{};
  a.seg = seg;
  a.slot_index = seg ? slot_index : nullptr;
  a.packed = packed;
  a.offsets = offsets;
  a.lengths = lengths;
  a.algs = algs;
  a.perm = m.perm;
  a.chunk_counter = &m.ws->chunk_counter;
  a.nchunks = &m.ws->nchunks;
  a.early = m.ws->early;
  a.n = n;
  a.digests = digests;
  a.status = c->status;
  a.abort_flag = abort_flag;
  a.wait_limit_ns = g_wait_limit_ns;
  a.mc = hb::make_mul_consts();
  if (comp) {
    a.msg_req = comp->msg_req;
    a.req_remaining = comp->remaining;
    a.req_done = comp->done;
  }
  if (warps_per_sm < 0) warps_per_sm = c->mixed_warps_per_sm;
  if (grid <= 0) {
    int per_sm = occ;
    if (warps_per_sm > 0) {
      int warps = 0, stages = 0;
      hb::shape_desc(shape, &warps, &stages);
      per_sm = std::min(occ, std::max(1, warps_per_sm / warps));
    }
    grid = c->sms * per_sm;
  }
  e = hb::launch_hash(true, 0, shape, grid, a, s);
  return e == cudaSuccess ? HB_OK : cuda_fail(e);
}

int reserve_ws(Ctx* c, uint64_t n) {
  const size_t need = hb::mixed_workspace_bytes(n);
  if (need > c->ws.cap && c->ws_used) {
    if (cudaEventSynchronize(c->ws_event) != cudaSuccess) return cuda_fail(cudaGetLastError());
  }
  cudaError_t e = c->ws.reserve(need);
  return e == cudaSuccess ? HB_OK : cuda_fail(e);
}

}  // namespace

extern "C" {

size_t hash_digest_size(int alg) {
  switch (alg) {
    case HB_MD5: return 16;
    case HB_SHA1: return 20;
    case HB_SM3: return 32;
    default: return 0;
  }
}

const char* hash_strerror(int code) {
  switch (code) {
    case HB_OK: return "ok";
    case HB_ERR_INVALID_ALG: return "invalid algorithm code";
    case HB_ERR_NULL: return "null pointer";
    case HB_ERR_TOO_LARGE: return "size exceeds a documented limit";
    case HB_ERR_CUDA: return "CUDA runtime or launch error";
    case HB_ERR_NOMEM: return "device or pinned memory allocation failed";
    case HB_ERR_TIMEOUT: return "a device-side wait timed out";
    case HB_ERR_ALIGN: return "digests_out is not 16-byte aligned";
    case HB_ERR_BOUNDS: return "a message lies outside the packed buffer";
    case HB_ERR_BUDGET: return "request exceeds the memory budget";
    case HB_ERR_ARG: return "invalid argument";
    default: return "unknown error code";
  }
}

int hash_batch_all_shape(const uint8_t* packed_bytes, const uint64_t* offsets,
                         const uint32_t* lengths, uint64_t n, uint8_t* records_out,
                         int shape_index, int grid_blocks, void* stream);

int hash_batch_shape(int alg, const uint8_t* packed_bytes, const uint64_t* offsets,
                     const uint32_t* lengths, uint64_t n, uint8_t* digests_out, int shape_index,
                     int grid_blocks, void* stream) {
  if (alg == HB_ALL)
    return hash_batch_all_shape(packed_bytes, offsets, lengths, n, digests_out, shape_index,
                                grid_blocks, stream);
  if (hash_digest_size(alg) == 0) return HB_ERR_INVALID_ALG;
  if (n == 0) return HB_OK;
  if (n >= kMaxPlainN) return HB_ERR_TOO_LARGE;
  int rc = check_common(packed_bytes, offsets, lengths, n, digests_out);
  if (rc) return rc;
  Ctx* c = nullptr;
  if ((rc = get_ctx(&c))) return rc;
  if (shape_index < 0) shape_index = c->tune_plain[alg];
  KernelArgs a{};
  a.packed = packed_bytes;
  a.offsets = offsets;
  a.lengths = lengths;
  a.n = n;
  a.digests = digests_out;
  a.status = c->status;
  a.wait_limit_ns = g_wait_limit_ns;
  a.mc = hb::make_mul_consts();
  return launch_plain(c, alg, shape_index, grid_blocks, a, static_cast<cudaStream_t>(stream));
}

int hash_batch_all_shape(const uint8_t* packed_bytes, const uint64_t* offsets,
                         const uint32_t* lengths, uint64_t n, uint8_t* records_out,
                         int shape_index, int grid_blocks, void* stream) {
  if (n == 0) return HB_OK;
  if (n >= kMaxPlainN) return HB_ERR_TOO_LARGE;
  int rc = check_common(packed_bytes, offsets, lengths, n, records_out);
  if (rc) return rc;
  Ctx* c = nullptr;
  if ((rc = get_ctx(&c))) return rc;
  if (shape_index < 0) shape_index = c->tune_plain[HB_ALL];
  KernelArgs a{};
  a.packed = packed_bytes;
  a.offsets = offsets;
  a.lengths = lengths;
  a.n = n;
  a.digests = records_out;
  a.status = c->status;
  a.wait_limit_ns = g_wait_limit_ns;
  a.mc = hb::make_mul_consts();
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (grid_blocks <= 0) {
    rc = launch_all_relay(c, shape_index, a, s);
    if (rc < 0) return rc;
    if (rc == 1) return HB_OK;
  }
  return launch_plain(c, HB_ALL, shape_index, grid_blocks, a, s);
}

int hash_batch_all(const uint8_t* packed_bytes, const uint64_t* offsets, const uint32_t* lengths,
                   uint64_t n, uint8_t* records_out, void* stream) {
  return hash_batch_all_shape(packed_bytes, offsets, lengths, n, records_out, -1, 0, stream);
}

int hash_batch(int alg, const uint8_t* packed_bytes, const uint64_t* offsets,
               const uint32_t* lengths, uint64_t n, uint8_t* digests_out, void* stream) {
  return hash_batch_shape(alg, packed_bytes, offsets, lengths, n, digests_out, -1, 0, stream);
}

}  // extern "C"

namespace {

// hash_batch_mixed(_shape) and hash_batch_segments: the ragged path on the
// per-device scratch.
int mixed_on_ctx(const uint8_t* algs, const uint8_t* packed_bytes, const uint64_t* offsets,
                 const uint32_t* lengths, const uint64_t* seg, const uint32_t* slot_index,
                 uint64_t n, uint8_t* digests_out, int shape_index, int grid_blocks,
                 void* stream) {
  if (n == 0) return HB_OK;
  if (n >= kMaxMixedN) return HB_ERR_TOO_LARGE;
  int rc = check_common(packed_bytes, offsets, lengths, n, digests_out);
  if (rc) return rc;
  if (!algs) return HB_ERR_NULL;
  Ctx* c = nullptr;
  if ((rc = get_ctx(&c))) return rc;
  if (shape_index < 0) shape_index = c->tune_mixed;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = reserve_ws(c, n))) return rc;
  if (c->ws_used && cudaStreamWaitEvent(s, c->ws_event, 0) != cudaSuccess) return cuda_fail(cudaGetLastError());
  rc = launch_mixed(c, shape_index, grid_blocks, algs, packed_bytes, offsets, lengths, n,
                    digests_out, c->ws.p, nullptr, s, nullptr, nullptr, -1, nullptr, seg,
                    slot_index);
  if (rc) return rc;
  if (cudaEventRecord(c->ws_event, s) != cudaSuccess) return cuda_fail(cudaGetLastError());
  c->ws_used = true;
  return HB_OK;
}

}  // namespace

namespace hb {
int* current_status_word() {
  Ctx* c = nullptr;
  return get_ctx(&c) == HB_OK ? c->status : nullptr;
}

uint64_t wait_limit_ns() {
  std::lock_guard<std::mutex> lock(g_mu);
  return g_wait_limit_ns;
}
}  // namespace hb

extern "C" {

int hash_batch_mixed_shape(const uint8_t* algs, const uint8_t* packed_bytes,
                           const uint64_t* offsets, const uint32_t* lengths, uint64_t n,
                           uint8_t* digests_out, int shape_index, int grid_blocks, void* stream) {
  return mixed_on_ctx(algs, packed_bytes, offsets, lengths, nullptr, nullptr, n, digests_out,
                      shape_index, grid_blocks, stream);
}

int hash_batch_segments(const uint8_t* algs, const uint8_t* packed_bytes,
                        const uint64_t* offsets, const uint32_t* lengths, const uint64_t* seg,
                        const uint32_t* slot_index, uint64_t n, uint8_t* slots_inout,
                        void* stream) {
  if (n == 0) return HB_OK;
  if (!seg) return HB_ERR_NULL;
  return mixed_on_ctx(algs, packed_bytes, offsets, lengths, seg, slot_index, n, slots_inout, -1,
                      0, stream);
}

int hash_batch_mixed(const uint8_t* algs, const uint8_t* packed_bytes, const uint64_t* offsets,
                     const uint32_t* lengths, uint64_t n, uint8_t* digests_out, void* stream) {
  return hash_batch_mixed_shape(algs, packed_bytes, offsets, lengths, n, digests_out, -1, 0,
                                stream);
}

int hash_batch_check_bounds(const uint64_t* offsets, const uint32_t* lengths, uint64_t n,
                            uint64_t packed_len, int* status_dev, void* stream) {
  if (!status_dev) return HB_ERR_NULL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(status_dev, 0, sizeof(int), s) != cudaSuccess) return cuda_fail(cudaGetLastError());
  if (n == 0) return HB_OK;
  if (!offsets || !lengths) return HB_ERR_NULL;
  Ctx* c = nullptr;
  int rc = get_ctx(&c);
  if (rc) return rc;
  cudaError_t e = hb::launch_bounds(offsets, lengths, n, packed_len, status_dev, c->status,
                                    grid_for_elementwise(c, n), s);
  return e == cudaSuccess ? HB_OK : cuda_fail(e);
}

}  // extern "C"

namespace {

int host_streams(Ctx* c) {
  if (c->host_hash) return HB_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&c->host_hash, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->host_out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_meta, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_end, cudaEventDisableTiming);
  for (int k = 0; e == cudaSuccess && k < kHostChunks; ++k) {
    e = cudaEventCreateWithFlags(&c->ev_in[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_hashed[k], cudaEventDisableTiming);
  }
  for (int j = 0; e == cudaSuccess && j < 2; ++j)
    e = cudaEventCreateWithFlags(&c->ev_win_out[j], cudaEventDisableTiming);
  return e == cudaSuccess ? HB_OK : cuda_fail(e);
}

// Hashes messages [first, first + count) of the device copies on stream s.
int host_hash_range(Ctx* c, int alg, const uint8_t* d_algs, const uint8_t* d_packed,
                    const uint64_t* d_off, const uint32_t* d_len, uint64_t first, uint64_t count,
                    uint8_t* d_dig, const int* abort_flag, cudaStream_t s) {
  if (count == 0) return HB_OK;
  const uint64_t rec = alg == HB_ALL ? HB_ALL_RECORD_BYTES : HB_SLOT_BYTES;
  if (d_algs)
    return launch_mixed(c, c->tune_mixed, 0, d_algs + first, d_packed, d_off + first,
                        d_len + first, count, d_dig + first * HB_SLOT_BYTES, c->ws.p, abort_flag, s);
  KernelArgs a{};
  a.packed = d_packed;
  a.offsets = d_off + first;
  a.lengths = d_len + first;
  a.n = count;
  a.digests = d_dig + first * rec;
  a.status = c->status;
  a.abort_flag = abort_flag;
  a.wait_limit_ns = g_wait_limit_ns;
  a.mc = hb::make_mul_consts();
  return launch_plain(c, alg, c->tune_plain[alg], 0, a, s);
}

// Device bytes a window needs per message: offset, length, algorithm code,
// digest slot.
constexpr uint64_t kWinMsgBytes = 8 + 4 + 1 + HB_ALL_RECORD_BYTES;  // largest record

uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// Host bytes per message in the packed digest layout.
uint64_t packed_digest_bytes(int alg) {
  return alg == HB_ALL ? HB_ALL_DIGEST_BYTES : hash_digest_size(alg);
}

// Batches larger than the host-path limit: windows of consecutive messages
// whose bytes (from the previous window's last message end to their own last
// end) and metadata fit half the limit go through two alternating device
// buffers; copy-in, hashing and copy-out of different windows overlap.
// Needs message ends in non-decreasing index order with no message starting
// before the previous window's last end (a back-to-back layout, gaps
// allowed); each window is checked on the device.
int host_windowed(Ctx* c, int alg, const uint8_t* algs_host, const uint8_t* packed_host,
                  uint64_t packed_len, const uint64_t* offsets_host,
                  const uint32_t* lengths_host, uint64_t n, uint8_t* digests_host,
                  cudaStream_t s, bool pack, bool* layout_failed) {
  *layout_failed = false;
  const uint64_t rec = (alg == HB_ALL && !algs_host) ? HB_ALL_RECORD_BYTES : HB_SLOT_BYTES;
  const uint64_t orec = pack ? packed_digest_bytes(alg) : rec;  // host bytes per message
  const uint64_t msg_bytes = kWinMsgBytes + (pack ? orec : 0);
  const uint64_t B = g_host_limit / 2;  // bytes per window buffer
  const uint64_t max_msgs = B / (2 * msg_bytes);
  if (max_msgs == 0) return HB_ERR_TOO_LARGE;
  auto end_of = [&](uint64_t i) { return offsets_host[i] + lengths_host[i]; };
  cudaError_t e;
  for (int j = 0; j < 2; ++j)
    if ((e = c->win[j].reserve(B)) != cudaSuccess) return cuda_fail(e);
  if (algs_host) {
    int rc = reserve_ws(c, max_msgs);
    if (rc) return rc;
  }
  if ((e = c->h_flag.reserve(2 * sizeof(int))) != cudaSuccess) return cuda_fail(e);
  int* d_flag = static_cast<int*>(c->h_flag.p);
  cudaStream_t sh = c->host_hash, so = c->host_out;
  auto fail = [&]() { return cuda_fail(cudaGetLastError()); };
  if (cudaMemsetAsync(d_flag, 0, 2 * sizeof(int), s) || cudaEventRecord(c->ev_meta, s) ||
      cudaStreamWaitEvent(sh, c->ev_meta, 0))
    return fail();
  uint64_t m = 0, rs = 0;
  int k = 0;
  while (m < n) {
    // largest window [m, m2) whose bytes [rs, end(m2-1)) plus metadata fit B
    uint64_t lo = m + 1, hi = std::min<uint64_t>(n, m + max_msgs);
    auto fits = [&](uint64_t x) {
      const uint64_t re = std::max<uint64_t>(end_of(x - 1), rs);
      return align_up(re - rs, 256) + msg_bytes * (x - m) + 1024 <= B;
    };
    if (!fits(lo)) {
      // nothing may still be writing the caller's buffers when we return
      cudaStreamSynchronize(s);
      cudaStreamSynchronize(sh);
      cudaStreamSynchronize(so);
      if (offsets_host[m] > packed_len || lengths_host[m] > packed_len - offsets_host[m])
        return HB_ERR_BOUNDS;
      if (align_up(lengths_host[m], 256) + msg_bytes + 1024 > B)
        return HB_ERR_TOO_LARGE;  // one message larger than a window
      *layout_failed = true;
      return HB_ERR_ARG;          // the message lies too far past the previous window
    }
    while (lo < hi) {
      const uint64_t mid = lo + (hi - lo + 1) / 2;
      if (fits(mid)) lo = mid; else hi = mid - 1;
    }
    const uint64_t m2 = lo, cnt = m2 - m;
    const uint64_t re = std::min<uint64_t>(std::max<uint64_t>(end_of(m2 - 1), rs), packed_len);
    const int j = k & 1;
    uint8_t* base = static_cast<uint8_t*>(c->win[j].p);
    uint8_t* d_packed = base;
    uint64_t* d_off = reinterpret_cast<uint64_t*>(base + align_up(re - rs + 16, 256));
    uint32_t* d_len = reinterpret_cast<uint32_t*>(d_off + cnt);
    uint8_t* d_dig = reinterpret_cast<uint8_t*>(align_up(reinterpret_cast<uint64_t>(d_len + cnt), 256));
    uint8_t* d_algs = d_dig + cnt * rec;
    uint8_t* d_cmp = reinterpret_cast<uint8_t*>(align_up(reinterpret_cast<uint64_t>(d_algs + cnt), 256));
    // this window's buffer is free once the window two back has been copied out
    if (k >= 2 && cudaStreamWaitEvent(s, c->ev_win_out[j], 0)) return fail();
    if ((re > rs && cudaMemcpyAsync(d_packed, packed_host + rs, re - rs, cudaMemcpyHostToDevice, s)) ||
        cudaMemcpyAsync(d_off, offsets_host + m, cnt * sizeof(uint64_t), cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(d_len, lengths_host + m, cnt * sizeof(uint32_t), cudaMemcpyHostToDevice, s) ||
        (algs_host && cudaMemcpyAsync(d_algs, algs_host + m, cnt, cudaMemcpyHostToDevice, s)) ||
        cudaEventRecord(c->ev_in[k % kHostChunks], s) ||
        cudaStreamWaitEvent(sh, c->ev_in[k % kHostChunks], 0))
      return fail();
    const int g = grid_for_elementwise(c, cnt);
    e = hb::launch_rebase(d_off, cnt, rs, g, sh);
    if (e == cudaSuccess) e = hb::launch_bounds(d_off, d_len, cnt, re - rs, d_flag, nullptr, g, sh);
    if (e != cudaSuccess) return cuda_fail(e);
    int rc = host_hash_range(c, alg, algs_host ? d_algs : nullptr, d_packed, d_off, d_len, 0, cnt,
                             d_dig, d_flag, sh);
    if (rc) return rc;
    if (pack && (e = hb::launch_pack(d_dig, (uint32_t)rec, cnt, d_cmp, (uint32_t)orec,
                                     grid_for_elementwise(c, cnt * (orec / 4)), sh)))
      return cuda_fail(e);
    if (cudaEventRecord(c->ev_hashed[k % kHostChunks], sh) ||
        cudaStreamWaitEvent(so, c->ev_hashed[k % kHostChunks], 0) ||
        cudaMemcpyAsync(digests_host + m * orec, pack ? d_cmp : d_dig, cnt * (size_t)orec,
                        cudaMemcpyDeviceToHost, so) ||
        cudaEventRecord(c->ev_win_out[j], so))
      return fail();
    m = m2;
    rs = re;
    ++k;
  }
  if (cudaMemcpyAsync(c->flag_host, d_flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, so) ||
      cudaEventRecord(c->ev_end, so) || cudaStreamWaitEvent(s, c->ev_end, 0))
    return fail();
  if (algs_host) {
    if (cudaEventRecord(c->ws_event, sh) != cudaSuccess) return fail();
    c->ws_used = true;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail();
  if (c->flag_host[0]) {
    // a window saw a message outside its bytes: either the message is out of
    // the buffer (a caller error) or the layout does not stream
    for (uint64_t i = 0; i < n; ++i)
      if (offsets_host[i] > packed_len || lengths_host[i] > packed_len - offsets_host[i])
        return HB_ERR_BOUNDS;
    *layout_failed = true;
    return HB_ERR_ARG;
  }
  return HB_OK;
}

}  // namespace

extern "C" {

uint64_t hash_set_host_memory_limit(uint64_t bytes) {
  std::lock_guard<std::mutex> lock(g_mu);
  const uint64_t old = g_host_limit;
  g_host_limit = bytes;
  return old;
}

// Pipeline: the caller's stream copies the metadata, then the packed bytes in
// chunks [b_k, b_k+1); the hashing stream, after the bounds check, hashes the
// messages whose last byte lies in chunk k as soon as chunk k has arrived;
// the copy-out stream brings their digest slots back while later chunks are
// still coming in.  Which messages end in which chunk is found on the host by
// binary search, assuming message ends (offset + length) never decrease with
// the index -- true of any back-to-back layout.  A device check confirms
// that; when it fails, every message is hashed again once all bytes are in,
// so the result never depends on the layout.
// PACK: digests_host takes the digest bytes back to back (packed on the
// device before the copy back) instead of 32-byte slots / 96-byte records.
static int host_call(int alg, const uint8_t* algs_host, const uint8_t* packed_host,
                     uint64_t packed_len, const uint64_t* offsets_host,
                     const uint32_t* lengths_host, uint64_t n, uint8_t* digests_host,
                     void* stream, bool pack) {
  if (!algs_host && alg != HB_ALL && hash_digest_size(alg) == 0) return HB_ERR_INVALID_ALG;
  if (n == 0) return HB_OK;
  if (n >= (algs_host ? kMaxMixedN : kMaxPlainN)) return HB_ERR_TOO_LARGE;
  // digest bytes per message on the device: one slot, or (HB_ALL) a
  // three-slot record; on the host the same, or the packed digest bytes
  const uint64_t rec = (alg == HB_ALL && !algs_host) ? HB_ALL_RECORD_BYTES : HB_SLOT_BYTES;
  const uint64_t orec = pack ? packed_digest_bytes(alg) : rec;
  if (!offsets_host || !lengths_host || !digests_host || (!packed_host && packed_len))
    return HB_ERR_NULL;
  Ctx* c = nullptr;
  int rc = get_ctx(&c);
  if (rc) return rc;
  if ((rc = host_streams(c))) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Make sure no earlier call on another stream still uses the buffers.
  if (cudaDeviceSynchronize() != cudaSuccess) return cuda_fail(cudaGetLastError());
  const size_t pbytes = ((size_t)packed_len + 15) / 16 * 16 + 16;
  const uint64_t footprint = pbytes + n * (kWinMsgBytes + 4 + (pack ? orec : 0));
  if (g_host_limit && footprint > g_host_limit) {
    bool layout_failed = false;
    return host_windowed(c, alg, algs_host, packed_host, packed_len, offsets_host, lengths_host,
                         n, digests_host, s, pack, &layout_failed);
  }
  cudaError_t e;
  if ((e = c->h_packed.reserve(pbytes)) != cudaSuccess ||
      (e = c->h_off.reserve(n * sizeof(uint64_t))) != cudaSuccess ||
      (e = c->h_len.reserve(n * sizeof(uint32_t))) != cudaSuccess ||
      (e = c->h_dig.reserve(n * (size_t)rec)) != cudaSuccess ||
      (e = c->h_flag.reserve(2 * sizeof(int))) != cudaSuccess ||
      (algs_host && (e = c->h_algs.reserve(n)) != cudaSuccess) ||
      (pack && (e = c->h_cmp.reserve(n * (size_t)orec)) != cudaSuccess))
    return cuda_fail(e);
  if (algs_host && (rc = reserve_ws(c, n))) return rc;
  uint8_t* d_packed = static_cast<uint8_t*>(c->h_packed.p);
  uint64_t* d_off = static_cast<uint64_t*>(c->h_off.p);
  uint32_t* d_len = static_cast<uint32_t*>(c->h_len.p);
  uint8_t* d_dig = static_cast<uint8_t*>(c->h_dig.p);
  int* d_flag = static_cast<int*>(c->h_flag.p);
  uint8_t* d_algs = algs_host ? static_cast<uint8_t*>(c->h_algs.p) : nullptr;
  uint8_t* d_cmp = pack ? static_cast<uint8_t*>(c->h_cmp.p) : nullptr;
  // the bytes copied back for messages [m, m + cnt), packed first if asked
  auto out_range = [&](uint64_t m, uint64_t cnt, cudaStream_t st) -> const uint8_t* {
    if (!pack) return d_dig + m * rec;
    e = hb::launch_pack(d_dig + m * rec, (uint32_t)rec, cnt, d_cmp + m * orec, (uint32_t)orec,
                        grid_for_elementwise(c, cnt * (orec / 4)), st);
    return e == cudaSuccess ? d_cmp + m * orec : nullptr;
  };
  cudaStream_t sh = c->host_hash, so = c->host_out;
  auto fail = [&]() { return cuda_fail(cudaGetLastError()); };

  // metadata, then the checks on the hashing stream
  if (cudaMemcpyAsync(d_off, offsets_host, n * sizeof(uint64_t), cudaMemcpyHostToDevice, s) ||
      cudaMemcpyAsync(d_len, lengths_host, n * sizeof(uint32_t), cudaMemcpyHostToDevice, s) ||
      (algs_host && cudaMemcpyAsync(d_algs, algs_host, n, cudaMemcpyHostToDevice, s)) ||
      cudaEventRecord(c->ev_meta, s) || cudaStreamWaitEvent(sh, c->ev_meta, 0) ||
      cudaMemsetAsync(d_flag, 0, 2 * sizeof(int), sh))
    return fail();
  // bounds first: the hashing kernels skip all work when it failed
  e = hb::launch_bounds(d_off, d_len, n, packed_len, d_flag, nullptr, grid_for_elementwise(c, n), sh);
  if (e == cudaSuccess) e = hb::launch_monotone(d_off, d_len, n, d_flag + 1, grid_for_elementwise(c, n), sh);
  if (e != cudaSuccess) return cuda_fail(e);

  // chunks of the packed bytes and the messages ending in each
  int K = (int)std::min<uint64_t>(kHostChunks, std::max<uint64_t>(1, packed_len / kHostChunkMin));
  uint64_t prev_b = 0, prev_m = 0;
  for (int k = 0; k < K; ++k) {
    const uint64_t b = (k == K - 1) ? packed_len : packed_len / K * (k + 1);
    // first message whose end lies past b (ends assumed non-decreasing)
    uint64_t lo = prev_m, hi = n;
    if (k == K - 1) {
      lo = n;
    } else {
      while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (offsets_host[mid] + lengths_host[mid] <= b) lo = mid + 1; else hi = mid;
      }
    }
    if (b > prev_b && cudaMemcpyAsync(d_packed + prev_b, packed_host + prev_b, b - prev_b,
                                      cudaMemcpyHostToDevice, s))
      return fail();
    if (cudaEventRecord(c->ev_in[k], s) || cudaStreamWaitEvent(sh, c->ev_in[k], 0)) return fail();
    if ((rc = host_hash_range(c, alg, d_algs, d_packed, d_off, d_len, prev_m, lo - prev_m, d_dig,
                              d_flag, sh)))
      return rc;
    const uint8_t* src = out_range(prev_m, lo - prev_m, sh);
    if (!src) return cuda_fail(e);
    if (cudaEventRecord(c->ev_hashed[k], sh) || cudaStreamWaitEvent(so, c->ev_hashed[k], 0))
      return fail();
    if (lo > prev_m && cudaMemcpyAsync(digests_host + prev_m * orec, src,
                                       (lo - prev_m) * (size_t)orec,
                                       cudaMemcpyDeviceToHost, so))
      return fail();
    prev_b = b;
    prev_m = lo;
  }
  if (cudaMemcpyAsync(c->flag_host, d_flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, so) ||
      cudaEventRecord(c->ev_end, so) || cudaStreamWaitEvent(s, c->ev_end, 0))
    return fail();
  if (algs_host) {
    if (cudaEventRecord(c->ws_event, sh) != cudaSuccess) return fail();
    c->ws_used = true;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail();
  if (c->flag_host[0]) return HB_ERR_BOUNDS;
  if (c->flag_host[1]) {
    // ends decrease somewhere: every byte is in now, hash everything again
    if ((rc = host_hash_range(c, alg, d_algs, d_packed, d_off, d_len, 0, n, d_dig, d_flag, s)))
      return rc;
    const uint8_t* src = out_range(0, n, s);
    if (!src) return cuda_fail(e);
    if (cudaMemcpyAsync(digests_host, src, n * (size_t)orec, cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
      return fail();
  }
  return HB_OK;
}

int hash_batch_host(int alg, const uint8_t* algs_host, const uint8_t* packed_host,
                    uint64_t packed_len, const uint64_t* offsets_host,
                    const uint32_t* lengths_host, uint64_t n, uint8_t* digests_host,
                    void* stream) {
  return host_call(alg, algs_host, packed_host, packed_len, offsets_host, lengths_host, n,
                   digests_host, stream, false);
}

int hash_batch_host_packed(int alg, const uint8_t* packed_host, uint64_t packed_len,
                           const uint64_t* offsets_host, const uint32_t* lengths_host, uint64_t n,
                           uint8_t* digests_host, void* stream) {
  return host_call(alg, nullptr, packed_host, packed_len, offsets_host, lengths_host, n,
                   digests_host, stream, true);
}

int hash_digits(int alg, uint64_t first, uint64_t count, uint8_t* digests_out, void* stream) {
  if (hash_digest_size(alg) == 0) return HB_ERR_INVALID_ALG;
  if (count == 0) return HB_OK;
  if (first >= HB_DIGITS_COUNT || count > HB_DIGITS_COUNT - first) return HB_ERR_TOO_LARGE;
  if (!digests_out) return HB_ERR_NULL;
  if (reinterpret_cast<uintptr_t>(digests_out) & 15u) return HB_ERR_ALIGN;
  Ctx* c = nullptr;
  int rc = get_ctx(&c);
  if (rc) return rc;
  const uint64_t runs = (first + count + 9) / 10 - first / 10;
  const uint64_t need = (runs + 255) / 256;
  const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)c->sms * 8));
  cudaError_t e = hb::launch_digits(alg, first, count, digests_out, grid,
                                    static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? HB_OK : cuda_fail(e);
}

int hash_device_status(void* stream, int* status_out) {
  if (!status_out) return HB_ERR_NULL;
  Ctx* c = nullptr;
  int rc = get_ctx(&c);
  if (rc) return rc;
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return cuda_fail(cudaGetLastError());
  int v = 0, na = 0;
  if (cudaMemcpy(&v, c->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess)
    return cuda_fail(cudaGetLastError());
  // bits of the no-allocation entry point, whose word is in its own scratch
  cudaError_t e = hb::noalloc_take_status(&na);
  if (e != cudaSuccess) return cuda_fail(e);
  *status_out = v | na;
  return HB_OK;
}

int hash_release_device(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return cuda_fail(cudaGetLastError());
  std::lock_guard<std::mutex> lock(g_mu);
  Ctx* c = g_ctx[dev];
  if (!c) return HB_OK;
  cudaDeviceSynchronize();
  c->ws.release();
  c->h_packed.release();
  c->h_off.release();
  c->h_len.release();
  c->h_algs.release();
  c->h_dig.release();
  c->h_flag.release();
  if (c->status) cudaFree(c->status);
  if (c->relay) cudaFree(c->relay);
  if (c->ws_event) cudaEventDestroy(c->ws_event);
  if (c->relay_event) cudaEventDestroy(c->relay_event);
  if (c->flag_host) cudaFreeHost(c->flag_host);
  if (c->host_hash) cudaStreamDestroy(c->host_hash);
  if (c->host_out) cudaStreamDestroy(c->host_out);
  for (cudaEvent_t ev : {c->ev_meta, c->ev_end})
    if (ev) cudaEventDestroy(ev);
  for (int k = 0; k < kHostChunks; ++k) {
    if (c->ev_in[k]) cudaEventDestroy(c->ev_in[k]);
    if (c->ev_hashed[k]) cudaEventDestroy(c->ev_hashed[k]);
  }
  for (int j = 0; j < 2; ++j) {
    c->win[j].release();
    if (c->ev_win_out[j]) cudaEventDestroy(c->ev_win_out[j]);
  }
  delete c;
  g_ctx[dev] = nullptr;
  return HB_OK;
}

const char* hash_last_cuda_error(void) {
  return g_last_cuda_error == cudaSuccess ? "no CUDA error recorded" : cudaGetErrorString(g_last_cuda_error);
}

int hash_tune_shapes(void) { return hb::num_shapes(); }

int hash_tune_shape(int index, int* warps_per_block, int* stages, int* blocks_per_stage,
                    int* cooperative) {
  if (!warps_per_block || !stages || !blocks_per_stage || !cooperative) return HB_ERR_NULL;
  return hb::shape_desc(index, warps_per_block, stages, blocks_per_stage, cooperative) ? HB_OK
                                                                                        : HB_ERR_ARG;
}

int hash_tune_set(int alg, int shape_index) {
  if (shape_index < 0 || shape_index >= hb::num_shapes()) return HB_ERR_ARG;
  if (alg != HB_TUNE_MIXED && alg != HB_ALL && hash_digest_size(alg) == 0) return HB_ERR_INVALID_ALG;
  Ctx* c = nullptr;
  int rc = get_ctx(&c);
  if (rc) return rc;
  if (alg == HB_TUNE_MIXED)
    c->tune_mixed = shape_index;
  else
    c->tune_plain[alg] = shape_index;
  return HB_OK;
}

int hash_tune_get(int alg) {
  Ctx* c = nullptr;
  if (get_ctx(&c)) return cuda_fail(cudaGetLastError());
  if (alg == HB_TUNE_MIXED) return c->tune_mixed;
  if (alg != HB_ALL && hash_digest_size(alg) == 0) return HB_ERR_INVALID_ALG;
  return c->tune_plain[alg];
}

int hash_all_uses_relay(uint64_t n) {
  Ctx* c = nullptr;
  int rc = get_ctx(&c);
  if (rc) return rc;
  return relay_window(c, n) ? 1 : 0;
}

int hash_tune_relay(int segment_blocks) {
  if (segment_blocks < 0 || segment_blocks > (1 << 20)) return HB_ERR_ARG;
  Ctx* c = nullptr;
  int rc = get_ctx(&c);
  if (rc) return rc;
  c->relay_seg_blocks = segment_blocks;
  return HB_OK;
}

int hash_tune_mixed_warps(int warps_per_sm) {
  if (warps_per_sm < 0 || warps_per_sm > 64) return HB_ERR_ARG;
  Ctx* c = nullptr;
  int rc = get_ctx(&c);
  if (rc) return rc;
  c->mixed_warps_per_sm = warps_per_sm;
  return HB_OK;
}

int hash_tune_buckets(int sub_log2, int alg_major) {
  if (sub_log2 < 0 || sub_log2 > (int)hb::kMaxSubLog2 || alg_major < 0 || alg_major > 2)
    return HB_ERR_ARG;
  Ctx* c = nullptr;
  int rc = get_ctx(&c);
  if (rc) return rc;
  c->buckets.sub_log2 = (uint32_t)sub_log2;
  c->buckets.alg_major = (uint32_t)alg_major;
  return HB_OK;
}

int hash_tune_occupancy(int alg, int shape_index) {
  if (shape_index < 0 || shape_index >= hb::num_shapes()) return HB_ERR_ARG;
  const bool mixed = alg == HB_TUNE_MIXED;
  if (!mixed && alg != HB_ALL && hash_digest_size(alg) == 0) return HB_ERR_INVALID_ALG;
  Ctx* c = nullptr;
  int rc = get_ctx(&c);
  if (rc) return rc;
  int occ = 0;
  if ((rc = occupancy(c, mixed, mixed ? 0 : alg, shape_index, &occ))) return rc;
  return occ;
}

int hash_int_peak(int op_class, int blocks, int threads, int iters, uint64_t* cycles_out_dev,
                  uint32_t* sink_dev, void* stream) {
  if (!cycles_out_dev || !sink_dev) return HB_ERR_NULL;
  if (blocks <= 0 || threads <= 0 || threads > 1024 || iters <= 0) return HB_ERR_ARG;
  cudaError_t e = hb::launch_int_peak(op_class, blocks, threads, iters,
                                      reinterpret_cast<unsigned long long*>(cycles_out_dev),
                                      sink_dev, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? HB_OK : (e == cudaErrorInvalidValue ? HB_ERR_ARG : HB_ERR_CUDA);
}

int hash_int_peak_ops_per_iter(void) { return 32; }

int hash_selftest_wait_timeout(uint64_t timeout_ns, void* stream) {
  Ctx* c = nullptr;
  int rc = get_ctx(&c);
  if (rc) return rc;
  cudaError_t e = hb::launch_selftest_wait(timeout_ns, c->status, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? HB_OK : HB_ERR_CUDA;
}

uint64_t hash_set_wait_limit_ns(uint64_t limit_ns) {
  std::lock_guard<std::mutex> lock(g_mu);
  const uint64_t old = g_wait_limit_ns;
  if (limit_ns) g_wait_limit_ns = limit_ns;
  return old;
}

int hash_gather(const hb_copy* copies_dev, uint32_t count, void* stream) {
  if (count == 0) return HB_OK;
  if (!copies_dev) return HB_ERR_NULL;
  Ctx* c = nullptr;
  int rc = get_ctx(&c);
  if (rc) return rc;
  const int grid = (int)std::min<uint32_t>(count, (uint32_t)c->sms * 4);
  cudaError_t e = hb::launch_gather(copies_dev, count, grid, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? HB_OK : cuda_fail(e);
}

// ---------------------------------------------------------------------------
// Plans: the ragged path with private scratch, and its captured graph.

struct hb_plan {
  int device = -1;
  uint64_t max_n = 0;
  void* ws = nullptr;          // bucketing scratch for up to max_n messages
  uint64_t* n_dev = nullptr;   // message count read by the captured graph
  int shape = 0;
  int warps_per_sm = 0;
  hb::BucketCfg buckets = hb::kDefaultBuckets;
  Completion completion;
  const uint64_t* seg = nullptr;  // segment descriptors (hash_plan_set_segments)
  const uint32_t* slot_index = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

int hash_plan_configure(hb_plan* p, int shape_index, int warps_per_sm) {
  if (!p) return HB_ERR_NULL;
  if (shape_index >= hb::num_shapes() || warps_per_sm > 64) return HB_ERR_ARG;
  if (p->exec) return HB_ERR_ARG;  // configure before capturing
  if (shape_index >= 0) p->shape = shape_index;
  if (warps_per_sm >= 0) p->warps_per_sm = warps_per_sm;
  return HB_OK;
}

int hash_plan_set_completion(hb_plan* p, const uint32_t* msg_req_dev, uint32_t* remaining_dev,
                             uint32_t* done_flags) {
  if (!p) return HB_ERR_NULL;
  if (p->exec) return HB_ERR_ARG;  // before capturing
  const bool any = msg_req_dev || remaining_dev || done_flags;
  const bool all = msg_req_dev && remaining_dev && done_flags;
  if (any && !all) return HB_ERR_NULL;
  uint32_t* done_dev = nullptr;
  if (done_flags) {
    // The flags are host memory written by the kernel: take the device-side
    // address the runtime maps for it, and refuse memory that is not mapped.
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, done_flags) != cudaSuccess ||
        attr.type != cudaMemoryTypeHost) {
      cudaGetLastError();
      return HB_ERR_ARG;
    }
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, done_flags, 0) != cudaSuccess || d == nullptr) {
      cudaGetLastError();
      return HB_ERR_ARG;
    }
    done_dev = static_cast<uint32_t*>(d);
  }
  p->completion.msg_req = msg_req_dev;
  p->completion.remaining = remaining_dev;
  p->completion.done = done_dev;
  return HB_OK;
}

int hash_plan_set_segments(hb_plan* p, const uint64_t* seg_dev, const uint32_t* slot_index_dev) {
  if (!p) return HB_ERR_NULL;
  if (p->exec) return HB_ERR_ARG;  // before capturing
  if (slot_index_dev && !seg_dev) return HB_ERR_NULL;
  p->seg = seg_dev;
  p->slot_index = slot_index_dev;
  return HB_OK;
}

int hash_plan_create(uint64_t max_n, hb_plan** plan_out) {
  if (!plan_out) return HB_ERR_NULL;
  *plan_out = nullptr;
  if (max_n == 0) return HB_ERR_ARG;
  if (max_n >= kMaxMixedN) return HB_ERR_TOO_LARGE;
  Ctx* c = nullptr;
  int rc = get_ctx(&c);
  if (rc) return rc;
  hb_plan* p = new hb_plan();
  p->device = c->device;
  p->max_n = max_n;
  p->shape = c->tune_mixed;
  p->warps_per_sm = c->mixed_warps_per_sm;
  p->buckets = c->buckets;
  cudaError_t e = cudaMalloc(&p->ws, hb::mixed_workspace_bytes(max_n));
  if (e == cudaSuccess) e = cudaMalloc(&p->n_dev, sizeof(uint64_t));
  if (e != cudaSuccess) {
    hash_plan_destroy(p);
    return cuda_fail(e);
  }
  *plan_out = p;
  return HB_OK;
}

int hash_plan_destroy(hb_plan* p) {
  if (!p) return HB_OK;
  if (p->ws || p->n_dev || p->exec) cudaDeviceSynchronize();
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->ws) cudaFree(p->ws);
  if (p->n_dev) cudaFree(p->n_dev);
  delete p;
  return HB_OK;
}

int hash_plan_run(hb_plan* p, const uint8_t* algs, const uint8_t* packed_bytes,
                  const uint64_t* offsets, const uint32_t* lengths, uint64_t n,
                  uint8_t* digests_out, int grid_blocks, void* stream) {
  if (!p) return HB_ERR_NULL;
  if (n == 0) return HB_OK;
  if (n > p->max_n) return HB_ERR_TOO_LARGE;
  int rc = check_common(packed_bytes, offsets, lengths, n, digests_out);
  if (rc) return rc;
  if (!algs) return HB_ERR_NULL;
  Ctx* c = nullptr;
  if ((rc = get_ctx(&c))) return rc;
  if (c->device != p->device) return HB_ERR_ARG;
  return launch_mixed(c, p->shape, grid_blocks, algs, packed_bytes, offsets, lengths, n,
                      digests_out, p->ws, nullptr, static_cast<cudaStream_t>(stream), nullptr,
                      &p->buckets, p->warps_per_sm, &p->completion, p->seg, p->slot_index);
}

int hash_plan_capture(hb_plan* p, const uint8_t* algs, const uint8_t* packed_bytes,
                      const uint64_t* offsets, const uint32_t* lengths, uint8_t* digests_out,
                      int grid_blocks) {
  if (!p) return HB_ERR_NULL;
  int rc = check_common(packed_bytes, offsets, lengths, 1, digests_out);
  if (rc) return rc;
  if (!algs) return HB_ERR_NULL;
  Ctx* c = nullptr;
  if ((rc = get_ctx(&c))) return rc;
  if (c->device != p->device) return HB_ERR_ARG;
  int occ = 0;
  if ((rc = occupancy(c, true, 0, p->shape, &occ, p->seg != nullptr))) return rc;  // set-up before capture
  if (p->exec) {
    cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
  }
  if (p->graph) {
    cudaGraphDestroy(p->graph);
    p->graph = nullptr;
  }
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    // Grids of the grid-stride bucketing kernels are sized for max_n; the
    // kernels read the actual count from n_dev when the graph runs.
    rc = launch_mixed(c, p->shape, grid_blocks, algs, packed_bytes, offsets, lengths, p->max_n,
                      digests_out, p->ws, nullptr, s, p->n_dev, &p->buckets, p->warps_per_sm,
                      &p->completion, p->seg, p->slot_index);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &g);
    if (rc == HB_OK && e2 != cudaSuccess) rc = cuda_fail(e2);
    if (rc == HB_OK) {
      e = cudaGraphInstantiate(&p->exec, g, 0);
      if (e != cudaSuccess) rc = cuda_fail(e);
    }
    if (rc == HB_OK)
      p->graph = g;
    else if (g)
      cudaGraphDestroy(g);
  } else {
    rc = cuda_fail(e);
  }
  cudaStreamDestroy(s);
  return rc;
}

int hash_plan_replay(hb_plan* p, uint64_t n, void* stream) {
  if (!p) return HB_ERR_NULL;
  if (!p->exec) return HB_ERR_ARG;
  if (n > p->max_n) return HB_ERR_TOO_LARGE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = hb::launch_set_count(p->n_dev, n, s);
  if (e == cudaSuccess) e = cudaGraphLaunch(p->exec, s);
  return e == cudaSuccess ? HB_OK : cuda_fail(e);
}

}  // extern "C"
