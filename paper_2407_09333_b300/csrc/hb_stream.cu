// hb_stream.cu -- streaming rounds (hash_round_*): the device side of a
// serving loop over a ring of message entries.
//
// One round is a captured CUDA graph of five steps on one stream:
//   hb_round_claim_kernel    READY entries of the window become BUSY and get
//                            a place in the round's batch and staging area
//   hb_round_copy_kernel     segment bytes: message source -> staging
//   bucketing + hb_mixed_kernel<SEG>   the ragged path over the segments,
//                            slots indexed by ring entry
//   hb_round_advance_kernel  progress, READY/FREE, per-request completion
// The batch size is only known on the device; the bucketing kernels and the
// copy and advance kernels read it from the round's control block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "hashbatch.h"
#include "hb_launch.h"

namespace hb {
namespace {

constexpr int kClaimThreads = 256;
constexpr uint64_t kCountShift = 40;  // reservation word: count << 40 | bytes
constexpr uint64_t kBytesMask = (1ull << kCountShift) - 1;

// Per-launch control block (device).  head/tail are set by the begin kernel;
// the rest is zeroed there and filled by the claim kernel.
struct RoundCtl {
  uint64_t head, tail;
  unsigned long long resv;        // reservations attempted: count << 40 | bytes
  unsigned long long n_valid;     // segments in the batch
  unsigned long long bytes_valid; // staging bytes they use
  uint64_t pad[3];
};

struct RoundArgs {
  // ring
  uint64_t mask;
  const uint64_t* src;
  uint64_t* prior;
  const uint32_t* len;
  const uint32_t* req;
  const uint8_t* alg;
  uint32_t* state;
  uint32_t* req_remaining;
  volatile uint32_t* req_done;   // device view of mapped host memory
  uint64_t req_capacity;
  int* status;                   // HB_DEV_* bits
  // round
  RoundCtl* ctl;
  uint32_t max_msgs;
  uint8_t* staging;              // nullptr: hash in place from the sources
  uint64_t in_place_base;        // in place: offsets are relative to this address
  uint64_t staging_bytes;
  uint32_t segment_bytes[4];     // per algorithm code (index 3: unknown codes)
  uint8_t* b_algs;
  uint64_t* b_offsets;
  uint32_t* b_lengths;
  uint64_t* b_seg;
  uint32_t* b_slot;
  HbCopy* b_copies;
  volatile unsigned long long* report;  // device view of mapped host memory
};

__device__ __forceinline__ uint32_t ld_cg_u32(const uint32_t* p) { return __ldcg(p); }
__device__ __forceinline__ uint64_t ld_cg_u64(const uint64_t* p) { return __ldcg(p); }

__global__ void hb_round_begin_kernel(RoundCtl* ctl, uint64_t head, uint64_t tail) {
  ctl->head = head;
  ctl->tail = tail;
  ctl->resv = 0;
  ctl->n_valid = 0;
  ctl->bytes_valid = 0;
}

// Warp w takes window positions [32 i, 32 i + 32) for i = w, w + W, ...; a
// warp reserves batch places and staging bytes for its claimed entries with
// one 64-bit atomic.  Reservations grow monotonically, so the ones that fit
// form a prefix of the reservation order: the batch has no holes, and a
// warp whose reservation does not fit releases its claims and stops (every
// later reservation would not fit either).
__global__ void __launch_bounds__(kClaimThreads) hb_round_claim_kernel(RoundArgs r) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t head = r.ctl->head;
  const uint64_t window = r.ctl->tail - head;
  for (uint64_t base = warp * 32; base < window; base += nwarps * 32) {
    // stop early once the batch is full (lane 0 reads, the warp follows)
    unsigned long long seen = 0;
    if (lane == 0) seen = *(volatile unsigned long long*)&r.ctl->resv;
    seen = __shfl_sync(0xFFFFFFFFu, seen, 0);
    if ((seen >> kCountShift) >= r.max_msgs || (seen & kBytesMask) >= r.staging_bytes) break;
    const uint64_t j = base + lane;
    const uint64_t k = (head + j) & r.mask;
    bool claimed = false;
    if (j < window && ld_cg_u32(r.state + k) == HB_RING_READY)
      claimed = atomicCAS(r.state + k, HB_RING_READY, HB_RING_BUSY) == HB_RING_READY;
    uint64_t prior = 0, seg = 0, from = 0;
    bool more = false;
    if (claimed) {
      prior = ld_cg_u64(r.prior + k);
      const uint32_t code = __ldcg(r.alg + k);
      const uint64_t S = r.segment_bytes[code < 3u ? code : 3u];
      const uint64_t rem = (uint64_t)ld_cg_u32(r.len + k) - prior;
      more = rem > S;
      seg = more ? S : rem;
      from = ld_cg_u64(r.src + k) + prior;  // the segment's first byte
    }
    const uint32_t mask = __ballot_sync(0xFFFFFFFFu, claimed);
    if (mask == 0) continue;
    // A staged segment keeps its source's position within a 16-byte granule
    // (it starts `lead` bytes into its 16-byte aligned staging span), so the
    // copy moves aligned 16-byte vectors whatever the client's alignment.
    const uint64_t lead = r.staging ? (from & 15u) : 0u;
    const uint64_t b16 = claimed ? (lead + seg + 15) & ~15ull : 0;
    uint64_t incl = b16;  // inclusive scan of staged bytes
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t v = __shfl_up_sync(0xFFFFFFFFu, incl, d);
      if (lane >= (uint32_t)d) incl += v;
    }
    const uint64_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    const uint32_t cnt = __popc(mask);
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(&r.ctl->resv, ((unsigned long long)cnt << kCountShift) | total);
    old = __shfl_sync(0xFFFFFFFFu, old, 0);
    const uint64_t old_cnt = old >> kCountShift, old_bytes = old & kBytesMask;
    const bool fits = old_cnt + cnt <= r.max_msgs && old_bytes + total <= r.staging_bytes;
    if (!fits) {
      if (claimed) atomicExch(r.state + k, HB_RING_READY);
      break;
    }
    if (claimed) {
      const uint64_t i = old_cnt + __popc(mask & ((1u << lane) - 1u));
      const uint64_t off = old_bytes + incl - b16 + lead;
      r.b_algs[i] = (uint8_t)__ldcg(r.alg + k);
      // staged: offset into the staging area; in place: the source itself
      r.b_offsets[i] = r.staging ? off : from - r.in_place_base;
      r.b_lengths[i] = (uint32_t)seg;
      r.b_seg[i] = prior | (more ? HB_SEG_MORE : 0ull);
      r.b_slot[i] = (uint32_t)k;
      HbCopy c;
      c.src = from;
      c.dst = reinterpret_cast<uint64_t>(r.staging) + off;
      c.bytes = seg;
      r.b_copies[i] = c;
    }
    if (lane == 0) {
      atomicMax(&r.ctl->n_valid, (unsigned long long)(old_cnt + cnt));
      atomicMax(&r.ctl->bytes_valid, (unsigned long long)(old_bytes + total));
    }
  }
}

// One warp per segment.  Source and destination have the same position
// within a 16-byte granule (the claim places staged segments so): the bytes
// up to the first granule boundary go one per lane, the rest as 16-byte
// vectors, the tail one byte per lane.  Other pairs fall back to 4-byte
// words when both are 4-byte aligned, else bytes.
__global__ void hb_round_copy_kernel(const HbCopy* copies, const RoundCtl* ctl) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t n = ctl->n_valid;
  for (uint64_t rec = warp; rec < n; rec += nwarps) {
    const HbCopy c = copies[rec];
    const uint8_t* src = reinterpret_cast<const uint8_t*>(c.src);
    uint8_t* dst = reinterpret_cast<uint8_t*>(c.dst);
    uint64_t done = 0;
    if (((c.src ^ c.dst) & 15u) == 0) {
      const uint64_t head = (16u - (c.src & 15u)) & 15u;
      done = head < c.bytes ? head : c.bytes;
      if (lane < done) dst[lane] = __ldg(src + lane);
      const uint64_t nv = (c.bytes - done) >> 4;
      const uint4* s4 = reinterpret_cast<const uint4*>(src + done);
      uint4* d4 = reinterpret_cast<uint4*>(dst + done);
      uint64_t v = lane;
      for (; v + 96 < nv; v += 128) {
        const uint4 a = __ldg(s4 + v), b = __ldg(s4 + v + 32), x = __ldg(s4 + v + 64),
                    y = __ldg(s4 + v + 96);
        d4[v] = a;
        d4[v + 32] = b;
        d4[v + 64] = x;
        d4[v + 96] = y;
      }
      for (; v < nv; v += 32) d4[v] = __ldg(s4 + v);
      done += nv << 4;
    } else if (((c.src | c.dst) & 3u) == 0) {
      const uint64_t nw = c.bytes >> 2;
      const uint32_t* s1 = reinterpret_cast<const uint32_t*>(src);
      uint32_t* d1 = reinterpret_cast<uint32_t*>(dst);
      for (uint64_t v = lane; v < nw; v += 32) d1[v] = __ldg(s1 + v);
      done = nw << 2;
    }
    for (uint64_t b = done + lane; b < c.bytes; b += 32) dst[b] = __ldg(src + b);
  }
}

__global__ void hb_round_advance_kernel(RoundArgs r) {
  const uint64_t n = r.ctl->n_valid;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t k = r.b_slot[i];
    const uint64_t sg = r.b_seg[i];
    r.prior[k] = (sg & ~HB_SEG_MORE) + r.b_lengths[i];
    __threadfence();  // progress is visible before the entry can be claimed again
    if (sg & HB_SEG_MORE) {
      atomicExch(r.state + k, HB_RING_READY);
    } else {
      atomicExch(r.state + k, HB_RING_FREE);
      const uint32_t q = ld_cg_u32(r.req + k);
      if (q >= r.req_capacity) {  // a request index outside the table: report, skip
        atomicOr(r.status, HB_DEV_BOUNDS);
      } else if (atomicSub(r.req_remaining + q, 1u) == 1u) {
        __threadfence_system();
        r.req_done[q] = 1u;
      }
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    r.report[0] = n;
    r.report[1] = r.ctl->bytes_valid;
  }
}

template <class T>
cudaError_t dev_alloc(T** p, size_t count) {
  return cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(count, 1) * sizeof(T));
}

}  // namespace
}  // namespace hb

struct hb_round {
  int device = -1;
  hb::RoundArgs args{};
  hb::RoundCtl* ctl = nullptr;
  unsigned long long* report_host = nullptr;  // pinned, mapped
  void* ws = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" {

int hash_round_destroy(hb_round* p) {
  if (!p) return HB_OK;
  cudaDeviceSynchronize();
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  cudaFree(p->ctl);
  cudaFree(p->ws);
  cudaFree(p->args.b_algs);
  cudaFree(p->args.b_offsets);
  cudaFree(p->args.b_lengths);
  cudaFree(p->args.b_seg);
  cudaFree(p->args.b_slot);
  cudaFree(p->args.b_copies);
  if (p->report_host) cudaFreeHost(p->report_host);
  delete p;
  return HB_OK;
}

int hash_round_create(const hb_ring* ring, uint32_t max_msgs, uint8_t* staging,
                      uint64_t staging_bytes, const uint32_t* segment_bytes, int shape_index,
                      int warps_per_sm, hb_round** round_out) {
  using namespace hb;
  if (!ring || !round_out || !segment_bytes) return HB_ERR_NULL;
  *round_out = nullptr;
  if (!ring->src || !ring->prior || !ring->len || !ring->req || !ring->alg || !ring->state ||
      !ring->slots || !ring->req_remaining || !ring->req_done)
    return HB_ERR_NULL;
  const uint64_t cap = ring->capacity;
  if (cap == 0 || (cap & (cap - 1)) || cap > (1ull << 32)) return HB_ERR_ARG;
  if (ring->req_capacity == 0) return HB_ERR_ARG;
  if (max_msgs == 0 || max_msgs >= (1u << 23)) return HB_ERR_TOO_LARGE;
  for (int i = 0; i < 3; ++i)
    if (segment_bytes[i] == 0 || (segment_bytes[i] & 63u)) return HB_ERR_ARG;
  if (staging_bytes == 0 || staging_bytes >= (1ull << 39)) return HB_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(staging) & 15u) return HB_ERR_ALIGN;
  if (reinterpret_cast<uintptr_t>(ring->slots) & 15u) return HB_ERR_ALIGN;
  if (shape_index < 0) shape_index = kDefaultMixedShape;
  if (shape_index >= num_shapes() || warps_per_sm < 0 || warps_per_sm > 64) return HB_ERR_ARG;

  int dev = 0, sms = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HB_ERR_CUDA;
  int* status = current_status_word();
  if (!status) return HB_ERR_CUDA;
  // request flags: the device-side address of the caller's mapped memory
  cudaPointerAttributes attr;
  void* done_dev = nullptr;
  if (cudaPointerGetAttributes(&attr, ring->req_done) != cudaSuccess ||
      attr.type != cudaMemoryTypeHost ||
      cudaHostGetDevicePointer(&done_dev, ring->req_done, 0) != cudaSuccess || !done_dev) {
    cudaGetLastError();
    return HB_ERR_ARG;
  }
  if (prepare_kernel(true, 0, shape_index, &occ, true) != cudaSuccess) return HB_ERR_CUDA;

  hb_round* p = new hb_round();
  p->device = dev;
  RoundArgs& a = p->args;
  a.mask = cap - 1;
  a.src = ring->src;
  a.prior = ring->prior;
  a.len = ring->len;
  a.req = ring->req;
  a.alg = ring->alg;
  a.state = ring->state;
  a.req_remaining = ring->req_remaining;
  a.req_done = static_cast<volatile uint32_t*>(done_dev);
  a.req_capacity = ring->req_capacity;
  a.status = status;
  a.max_msgs = max_msgs;
  a.staging = staging;
  a.in_place_base = reinterpret_cast<uint64_t>(ring->slots);
  a.staging_bytes = staging_bytes;
  for (int i = 0; i < 3; ++i) a.segment_bytes[i] = segment_bytes[i];
  a.segment_bytes[3] = *std::max_element(segment_bytes, segment_bytes + 3);
  void* report_dev = nullptr;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = dev_alloc(&p->ctl, 1);
  if (e == cudaSuccess) e = dev_alloc(&a.b_algs, max_msgs);
  if (e == cudaSuccess) e = dev_alloc(&a.b_offsets, max_msgs);
  if (e == cudaSuccess) e = dev_alloc(&a.b_lengths, max_msgs);
  if (e == cudaSuccess) e = dev_alloc(&a.b_seg, max_msgs);
  if (e == cudaSuccess) e = dev_alloc(&a.b_slot, max_msgs);
  if (e == cudaSuccess) e = dev_alloc(&a.b_copies, max_msgs);
  if (e == cudaSuccess) e = cudaMalloc(&p->ws, mixed_workspace_bytes(max_msgs));
  if (e == cudaSuccess)
    e = cudaHostAlloc(reinterpret_cast<void**>(&p->report_host), 2 * sizeof(unsigned long long),
                      cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&report_dev, p->report_host, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    hash_round_destroy(p);
    return e == cudaErrorMemoryAllocation ? HB_ERR_NOMEM : HB_ERR_CUDA;
  }
  p->report_host[0] = p->report_host[1] = 0;
  a.ctl = p->ctl;
  a.report = static_cast<volatile unsigned long long*>(report_dev);

  // bucketing and hashing of the batch, sized from the control block
  MixedArgs m{};
  m.cfg = kDefaultBuckets;
  m.algs = a.b_algs;
  m.lengths = a.b_lengths;
  m.n = max_msgs;
  m.n_dev = reinterpret_cast<const uint64_t*>(&p->ctl->n_valid);
  m.digests = ring->slots;
  m.ws = static_cast<MixedWorkspace*>(p->ws);
  m.perm = reinterpret_cast<uint32_t*>(static_cast<char*>(p->ws) + sizeof(MixedWorkspace));
  m.slot_index = a.b_slot;
  KernelArgs k{};
  // in place, any valid device address serves as the base (message
  // addresses are base + offset; the base also feeds zero-byte copies)
  k.packed = staging ? staging : ring->slots;
  k.offsets = a.b_offsets;
  k.lengths = a.b_lengths;
  k.algs = a.b_algs;
  k.perm = m.perm;
  k.chunk_counter = &m.ws->chunk_counter;
  k.nchunks = &m.ws->nchunks;
  k.early = m.ws->early;
  k.n = max_msgs;
  k.digests = ring->slots;
  k.status = status;
  k.wait_limit_ns = wait_limit_ns();
  k.mc = make_mul_consts();
  k.seg = a.b_seg;
  k.slot_index = a.b_slot;
  int warps = 0, stages = 0;
  shape_desc(shape_index, &warps, &stages);
  const int per_sm = warps_per_sm > 0 ? std::min(occ, std::max(1, warps_per_sm / warps)) : occ;
  const int hash_grid = sms * std::max(1, per_sm);
  const int elem_grid = sms * 8;

  cudaStream_t s = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    hb_round_claim_kernel<<<elem_grid, kClaimThreads, 0, s>>>(a);
    if (staging) hb_round_copy_kernel<<<elem_grid, 256, 0, s>>>(a.b_copies, p->ctl);
    cudaError_t e1 = launch_bucketing(m, elem_grid, s);
    if (e1 == cudaSuccess) e1 = launch_hash(true, 0, shape_index, hash_grid, k, s);
    hb_round_advance_kernel<<<elem_grid, 256, 0, s>>>(a);
    if (e1 == cudaSuccess) e1 = cudaGetLastError();
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (e1 != cudaSuccess) e = e1;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, g, 0);
    if (e == cudaSuccess)
      p->graph = g;
    else if (g)
      cudaGraphDestroy(g);
  }
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    hash_round_destroy(p);
    return e == cudaErrorMemoryAllocation ? HB_ERR_NOMEM : HB_ERR_CUDA;
  }
  *round_out = p;
  return HB_OK;
}

int hash_round_launch(hb_round* p, uint64_t head, uint64_t tail, void* stream) {
  if (!p) return HB_ERR_NULL;
  if (tail < head || tail - head > p->args.mask + 1) return HB_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  hb::hb_round_begin_kernel<<<1, 1, 0, s>>>(p->ctl, head, tail);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaGraphLaunch(p->exec, s);
  return e == cudaSuccess ? HB_OK : HB_ERR_CUDA;
}

int hash_round_report(hb_round* p, uint64_t* segments, uint64_t* bytes) {
  if (!p) return HB_ERR_NULL;
  volatile unsigned long long* r = p->report_host;
  if (segments) *segments = r[0];
  if (bytes) *bytes = r[1];
  return HB_OK;
}

}  // extern "C"
