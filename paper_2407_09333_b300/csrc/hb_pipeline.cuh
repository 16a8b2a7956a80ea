// hb_pipeline.cuh -- the per-warp staging pipeline shared by the fixed-
// algorithm and the ragged (mixed-algorithm) kernels.
//
// Unit of work.  A warp owns a "task" of 32 messages, one per lane, and walks
// them block by block (64-byte blocks of the padded message).  An "item" is
// one block step of one task: for each lane, the 64-byte window of its
// message at that block.
//
// Staging.  Every lane stages its own window into a private 80-byte slot of
// shared memory with one 1-D bulk copy (cp.async.bulk, TMA engine, never
// multicast): the copy covers the 16-byte aligned granules that hold message
// bytes of the window, so the window's first byte lands at slot + (addr & 15).
// Completion is counted in transaction bytes on one mbarrier per stage; lane 0
// arms it with the warp's total byte count.  STAGES items are in flight: the
// warp issues item j + STAGES - 1 before it waits for item j, so the copies
// run under the compression of earlier blocks.  An item record (message
// index, length, block number, alignment, algorithm) travels with each stage
// in shared memory, so the consuming side needs no global metadata loads.
//
// Padding (RFC 1321 Sec. 3.1-3.2, FIPS 180-4 Sec. 5.1.1, GB/T 32905 Sec. 5.2)
// is done in the lane's own slot: the byte after the message becomes 0x80,
// the rest of the window is zeroed; a block past the message end is all zero;
// the final block's last two words are replaced by the 64-bit bit length in
// registers.  Words are read with 32-bit shared loads and realigned with one
// PRMT each, which also applies the big-endian byte swap for SHA-1 and SM3.
//
// Waits are bounded (hb_device.cuh): a wait that times out sets
// HB_DEV_TIMEOUT in the status word and the warp drains and returns.
#pragma once

#include <cstdint>

#include "hb_algs.cuh"
#include "hb_device.cuh"
#include "hb_launch.h"

namespace hb {

constexpr int kSlotBytes = 80;   // 64-byte window + up to 15 lead bytes, rounded to 16
constexpr int kItemBytes = 16;   // item record per lane per stage
constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kNoBlock = 0xFFFFFFFFu;

template <int STAGES>
struct WarpSmem {
  static constexpr int kSlots = STAGES * 32 * kSlotBytes;
  static constexpr int kItems = STAGES * 32 * kItemBytes;
  static constexpr int kBars = ((STAGES * 8 + 127) / 128) * 128;
  static constexpr int kBytes = kSlots + kItems + kBars;  // multiple of 128
};

// Padded block count: message + 0x80 + 8 length bytes, rounded up to 64.
__device__ __forceinline__ uint32_t padded_blocks(uint32_t len) {
  return (uint32_t)(((uint64_t)len + 72u) >> 6);
}

// Per-lane description of the task the issuing side is walking.
struct LaneTask {
  uint64_t msg;    // message index (digest slot); meaningful when nb > 0
  uint64_t addr;   // absolute address of the message's first byte
  uint32_t len;    // message length in bytes
  uint32_t nb;     // padded block count, 0 for an idle lane
  uint32_t alg;    // algorithm code
};


// ---------------------------------------------------------------------------
// Task sources.  A source hands the issuing side one task after another, with
// the per-lane metadata of the next task already requested from memory.

// Fixed algorithm, static grid-stride over tasks of 32 consecutive messages.
template <int ALG>
struct StaticSource {
  const uint8_t* packed;
  const uint64_t* offsets;
  const uint32_t* lengths;
  uint64_t n, ntasks, stride, next;  // warp-uniform
  uint32_t lane;
  bool pf_ok;
  uint64_t pf_msg, pf_off;
  uint32_t pf_len;

  __device__ StaticSource(const KernelArgs& args, uint64_t first, uint64_t stride_, uint32_t lane_)
      : packed(args.packed),
        offsets(args.offsets),
        lengths(args.lengths),
        n(args.n),
        ntasks((args.n + 31) / 32),
        stride(stride_),
        next(first),
        lane(lane_) {
    prefetch();
  }

  __device__ __forceinline__ void prefetch() {
    pf_ok = next < ntasks;
    pf_msg = next * 32 + lane;
    pf_off = 0;
    pf_len = 0;
    if (pf_ok && pf_msg < n) {
      pf_off = ldg_nc_u64(offsets + pf_msg);
      pf_len = ldg_nc_u32(lengths + pf_msg);
    }
    next += stride;
  }

  // Move to the next task; false when the source is exhausted.
  __device__ __forceinline__ bool take(LaneTask& t) {
    if (!pf_ok) return false;
    const bool valid = pf_msg < n;
    t.msg = pf_msg;
    t.addr = reinterpret_cast<uint64_t>(packed) + pf_off;
    t.len = pf_len;
    t.nb = valid ? padded_blocks(pf_len) : 0u;
    t.alg = ALG;
    prefetch();
    return true;
  }
};

// Mixed algorithms: chunks of 32 bucketed messages popped from a shared
// counter in order (longest estimated cost first).  Three-deep prefetch:
// popped chunk id -> permutation entry -> message metadata.
struct DynamicSource {
  const uint8_t* packed;
  const uint64_t* offsets;
  const uint32_t* lengths;
  const uint8_t* algs;
  const uint32_t* perm;
  uint32_t* counter;
  uint32_t lane, nchunks;
  uint32_t pf_chunk;        // popped id, perm entry not yet loaded
  uint32_t pf_perm_chunk;   // chunk whose perm entry is in pf_msg
  uint32_t pf_msg;          // perm entry of pf_perm_chunk
  uint32_t pf_meta_chunk;   // chunk whose metadata is in pf_*
  uint32_t pf_msg2;
  uint64_t pf_off;
  uint32_t pf_len, pf_alg;

  __device__ __forceinline__ uint32_t pop() {
    uint32_t c = 0;
    if (lane == 0) c = atomicAdd(counter, 1u);
    return __shfl_sync(kFull, c, 0);
  }

  __device__ __forceinline__ uint32_t load_perm(uint32_t chunk) {
    return chunk < nchunks ? ldg_nc_u32(perm + (uint64_t)chunk * 32 + lane) : 0xFFFFFFFFu;
  }

  __device__ __forceinline__ void load_meta(uint32_t chunk, uint32_t msg) {
    pf_meta_chunk = chunk;
    pf_msg2 = msg;
    pf_off = 0;
    pf_len = 0;
    pf_alg = 0;
    if (chunk < nchunks && msg != 0xFFFFFFFFu) {
      pf_off = ldg_nc_u64(offsets + msg);
      pf_len = ldg_nc_u32(lengths + msg);
      pf_alg = __ldg(algs + msg);
    }
  }

  __device__ DynamicSource(const KernelArgs& args, uint32_t lane_)
      : packed(args.packed),
        offsets(args.offsets),
        lengths(args.lengths),
        algs(args.algs),
        perm(args.perm),
        counter(args.chunk_counter),
        lane(lane_) {
    nchunks = *args.nchunks;
    const uint32_t c0 = pop();
    load_meta(c0, load_perm(c0));
    pf_perm_chunk = pop();
    pf_msg = load_perm(pf_perm_chunk);
    pf_chunk = pop();
  }

  __device__ __forceinline__ bool take(LaneTask& t) {
    if (pf_meta_chunk >= nchunks) return false;
    const bool valid = pf_msg2 != 0xFFFFFFFFu;
    t.msg = pf_msg2;
    t.addr = reinterpret_cast<uint64_t>(packed) + pf_off;
    t.len = pf_len;
    t.nb = valid ? padded_blocks(pf_len) : 0u;
    // Codes outside {0,1,2} were excluded by the bucketing step; the chunk's
    // algorithm is that of lane 0 (every chunk starts with a real message).
    t.alg = __shfl_sync(kFull, pf_alg, 0);
    load_meta(pf_perm_chunk, pf_msg);
    pf_perm_chunk = pf_chunk;
    pf_msg = load_perm(pf_chunk);
    pf_chunk = pf_chunk < nchunks ? pop() : pf_chunk;
    return true;
  }
};

// ---------------------------------------------------------------------------
// Consuming side: one block of one message per lane.

template <bool BE>
__device__ __forceinline__ void read_block_words(uint32_t slot, uint32_t s, uint32_t (&w)[16]) {
  // The window starts at byte s of the slot (a 16-byte aligned shared
  // address); read the 17 aligned words that cover it and realign with PRMT
  // (bytes r..r+3 of each word pair; reversed for big-endian word order).
  const uint32_t r = s & 3u;
  const uint32_t p = slot + (s & ~3u);
  const uint32_t sel = BE ? (0x0123u + 0x1111u * r) : (0x3210u + 0x1111u * r);
  uint32_t x[17];
#pragma unroll
  for (int k = 0; k < 17; ++k) x[k] = lds32(p + 4 * k);
#pragma unroll
  for (int i = 0; i < 16; ++i) w[i] = prmt(x[i], x[i + 1], sel);
}

// Write the 0x80 marker at window byte `rem` (0 <= rem < 64) and zero the
// rest of the window, in the lane's own slot.
__device__ __forceinline__ void pad_tail_in_slot(uint32_t slot, uint32_t s, uint32_t rem) {
  const uint32_t pos = slot + s + rem;
  const uint32_t wa = pos & ~3u;
  const uint32_t bi = pos & 3u;
  const uint32_t keep = bi ? (0xFFFFFFFFu >> (32u - 8u * bi)) : 0u;
  sts32(wa, (lds32(wa) & keep) | (0x80u << (8u * bi)));
  const uint32_t end = slot + s + 64u;  // words starting below this are read
#pragma unroll 1
  for (uint32_t a = wa + 4; a < end; a += 4) sts32(a, 0u);
  fence_proxy_async_smem();  // order these writes before the slot's next bulk copy
}

template <int ALG>
__device__ __forceinline__ void process_block(uint32_t (&st)[8], uint32_t slot, uint32_t s, uint32_t len, uint32_t b, uint64_t msg,
                                              uint8_t* digests) {
  constexpr bool BE = AlgTraits<ALG>::kBigEndian;
  const int64_t rem = (int64_t)len - 64 * (int64_t)b;
  uint32_t w[16];
  if (rem >= 64) {
    read_block_words<BE>(slot, s, w);
  } else if (rem >= 0) {
    pad_tail_in_slot(slot, s, (uint32_t)rem);
    read_block_words<BE>(slot, s, w);
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) w[i] = 0u;
  }
  const bool final_block = rem <= 55;
  if (final_block) {
    const uint32_t lo = len << 3, hi = len >> 29;  // bit length mod 2^64
    w[14] = BE ? hi : lo;
    w[15] = BE ? lo : hi;
  }
  if (b == 0) alg_init<ALG>(st);
  alg_compress<ALG>(st, w);
  if (final_block) {
    uint32_t o[8];
    alg_digest_words<ALG>(st, o);
    uint8_t* dst = digests + msg * HB_SLOT_BYTES;
    stg128_cs(dst, o[0], o[1], o[2], o[3]);
    stg128_cs(dst + 16, o[4], o[5], o[6], o[7]);
  }
}

// ---------------------------------------------------------------------------
// The warp loop.  MIXED selects the algorithm per item (warp-uniform);
// otherwise ALG is fixed.

template <int STAGES, int ALG, bool MIXED, class Source>
__device__ __forceinline__ void warp_pipeline(Source& src, uint8_t* wsm, const KernelArgs& a,
                                              uint32_t lane) {
  using L = WarpSmem<STAGES>;
  const uint32_t slots = smem_addr(wsm);
  const uint32_t items = slots + L::kSlots;
  const uint32_t bars = items + L::kItems;

  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < STAGES; ++i) mbar_init(bars + 8 * i, 1);
    fence_barrier_init();
  }
  fence_proxy_async_smem();
  __syncwarp();

  // Issuing side state (warp-uniform except the LaneTask fields).
  LaneTask t;
  bool have = src.take(t);
  uint32_t maxnb = have ? __reduce_max_sync(kFull, t.nb) : 0u;
  uint32_t ib = 0;  // next block of the current task to issue
  int is = 0;       // stage the next issue goes to

  // Consuming side state.
  int cs = 0;
  uint32_t cpar = 0;
  uint32_t st[8];
  int inflight = 0;
  bool failed = false;

  auto issue = [&]() {
    uint32_t bytes = 0;
    uint64_t lo = 0;
    const bool act = ib < t.nb;
    if (act) {
      const uint64_t A = t.addr + 64ull * ib;
      const uint64_t end = t.addr + t.len;
      if (A < end) {
        lo = A & ~15ull;
        const uint64_t e = (A + 64 < end) ? A + 64 : end;
        bytes = (uint32_t)(((e + 15) & ~15ull) - lo);
      }
    }
    uint4 rec;
    rec.x = (uint32_t)t.msg;
    rec.y = (uint32_t)(t.msg >> 32) | ((uint32_t)(t.addr & 15u) << 24) | (t.alg << 28);
    rec.z = t.len;
    rec.w = act ? ib : kNoBlock;
    sts128(items + (is * 32 + lane) * kItemBytes, rec);
    const uint32_t total = __reduce_add_sync(kFull, bytes);
    if (lane == 0) mbar_arrive_expect_tx(bars + 8 * is, total);
    if (bytes) bulk_copy_g2s(slots + (is * 32 + lane) * kSlotBytes,
                             reinterpret_cast<const void*>(lo), bytes, bars + 8 * is);
    ++inflight;
    is = (is + 1 == STAGES) ? 0 : is + 1;
    if (++ib >= maxnb) {
      have = src.take(t);
      maxnb = have ? __reduce_max_sync(kFull, t.nb) : 0u;
      ib = 0;
    }
  };

#pragma unroll 1
  for (int k = 0; k < STAGES - 1 && have; ++k) issue();

#pragma unroll 1
  while (inflight > 0) {
    if (have && !failed) issue();
    const bool ok = !failed && mbar_wait_bounded(bars + 8 * cs, cpar, a.wait_limit_ns, a.status);
    if (!ok) {
      // Drain: give every copy still in flight a bounded chance to land
      // before the warp leaves (a copy must not outlive its shared memory).
      failed = true;
      mbar_wait_bounded(bars + 8 * cs, cpar, a.wait_limit_ns, nullptr);
    } else {
      const uint4 rec = lds128(items + (cs * 32 + lane) * kItemBytes);
      if (rec.w != kNoBlock) {
        const uint64_t msg = (uint64_t)rec.x | ((uint64_t)(rec.y & 0x00FFFFFFu) << 32);
        const uint32_t s = (rec.y >> 24) & 15u;
        const uint32_t slot = slots + (cs * 32 + lane) * kSlotBytes;
        if constexpr (MIXED) {
          const uint32_t alg = rec.y >> 28;
          if (alg == HB_MD5)
            process_block<HB_MD5>(st, slot, s, rec.z, rec.w, msg, a.digests);
          else if (alg == HB_SHA1)
            process_block<HB_SHA1>(st, slot, s, rec.z, rec.w, msg, a.digests);
          else
            process_block<HB_SM3>(st, slot, s, rec.z, rec.w, msg, a.digests);
        } else {
          process_block<ALG>(st, slot, s, rec.z, rec.w, msg, a.digests);
        }
      }
    }
    __syncwarp();  // every lane is done with stage cs before it is re-armed
    --inflight;
    cs = (cs + 1 == STAGES) ? 0 : cs + 1;
    cpar ^= (cs == 0) ? 1u : 0u;
  }
}

}  // namespace hb
