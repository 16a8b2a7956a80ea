// hb_pipeline.cuh -- the per-warp staging pipeline shared by the fixed-
// algorithm and the ragged (mixed-algorithm) kernels.
//
// Unit of work.  A warp owns a "task" of 32 messages, one per lane, and walks
// them block by block (64-byte blocks of the padded message).  An "item"
// (stage) is KB block steps of one task: for each lane, the window of its
// message covering those KB blocks.
//
// Staging.  Every lane stages its own window of KB blocks (64*KB bytes) into a
// private slot of 64*KB + 16 bytes of shared memory with 4*KB or 4*KB + 1
// asynchronous 16-byte copies (cp.async, LDGSTS): the copies cover the
// 16-byte aligned granules that hold the window, so the window's first byte
// lands at slot + (addr & 15).  Larger KB means fewer, larger requests per
// lane, which matters when the 32 lanes of a warp read 32 distant places.  Granules
// are zero-filled past the message end by the copy itself (src-size), so a
// window that runs past the end of its message already holds zeros there.
// STAGES items are in flight: the warp issues item j + STAGES - 1 before it
// waits for item j (cp.async.wait_group), so the copies run under the
// compression of earlier blocks.  Every lane reads only what it copied
// itself, so no cross-lane synchronisation is needed.  An item record
// (message index, length, block number, alignment, algorithm) travels with
// each stage in shared memory, so the consuming side needs no global
// metadata loads.
//
// Padding (RFC 1321 Sec. 3.1-3.2, FIPS 180-4 Sec. 5.1.1, GB/T 32905 Sec. 5.2):
// the zero-filled window gives the zero bytes; the lane stores the 0x80
// marker after the last message byte into its own slot; the final block's
// last two words are replaced by the 64-bit bit length in registers.  Words
// are read with 32-bit shared loads and realigned with one PRMT each, which
// also applies the big-endian byte swap for SHA-1 and SM3.
//
// Segments (SEG, mixed path only): a message may arrive in pieces over
// several launches.  A piece that is not the last is a whole number of
// blocks and gets no padding; its last block's chaining value is stored raw
// in the message's 32-byte slot.  A later piece starts from that value
// instead of the initial one: the issuing lane copies it into shared memory
// together with the piece's first window, so the consumer never waits on a
// global load.  The last piece is padded with the whole message's length.
#pragma once

#include <cstdint>

#include "hb_algs.cuh"
#include "hb_device.cuh"
#include "hb_launch.h"

namespace hb {

// A stage holds KB consecutive blocks of each lane's message: a window of
// 64*KB bytes plus up to 15 lead bytes, rounded to 16.
template <int KB>
struct Slot {
  static constexpr int kBytes = 64 * KB + 16;
};
constexpr int kItemBytes = 16;   // item record per lane per stage
constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kNoBlock = 0xFFFFFFFFu;

template <int STAGES, int KB, bool SEG = false, bool RELAY = false>
struct WarpSmem {
  static constexpr int kSlots = STAGES * 32 * Slot<KB>::kBytes;
  static constexpr int kItems = STAGES * 32 * kItemBytes;
  static constexpr int kTable = 32 * 16;  // per-lane copy descriptors (cooperative copies)
  // segments: a second item record (prior bytes, more flag) and a staged
  // chaining value per lane per stage (relay: the record only, the chaining
  // value is read when the stage is consumed)
  static constexpr int kSegItems = (SEG || RELAY) ? STAGES * 32 * kItemBytes : 0;
  static constexpr int kStates = SEG ? STAGES * 32 * HB_SLOT_BYTES : 0;
  static constexpr int kBytes = kSlots + kItems + kTable + kSegItems + kStates;  // multiple of 128
};

// Padded block count: message + 0x80 + 8 length bytes, rounded up to 64.
__device__ __forceinline__ uint32_t padded_blocks(uint32_t len) {
  return (uint32_t)(((uint64_t)len + 72u) >> 6);
}

// Chaining state a lane carries across the blocks of its message: one
// algorithm's words, or (HB_ALL) all three algorithms' side by side.
struct AllState {
  uint32_t md5[8], sha1[8], sm3[8];
};
template <int ALG>
struct StateFor {
  using type = uint32_t[8];
};
template <>
struct StateFor<HB_ALL> {
  using type = AllState;
};

// Per-lane description of the task the issuing side is walking.
struct LaneTask {
  uint64_t msg;    // message index (digest slot); meaningful when nb > 0
  uint64_t addr;   // absolute address of the message's first byte
  uint32_t len;    // message length in bytes
  uint32_t nb;     // padded block count, 0 for an idle lane
  uint32_t alg;    // algorithm code
  uint64_t seg;    // segments only: prior bytes | HB_SEG_MORE
  uint32_t slot;   // segments only: the message's 32-byte slot
};

// Blocks of a segment: whole blocks only when more segments follow, else
// the padded count.  A segment that breaks the multiple-of-64 rules gets 0
// blocks and raises HB_DEV_SEGMENT.
__device__ __forceinline__ uint32_t segment_blocks(uint32_t len, uint64_t seg, int* status) {
  const bool more = (seg & HB_SEG_MORE) != 0;
  const uint64_t prior = seg & ~HB_SEG_MORE;
  if ((prior & 63u) != 0 || (more && (len & 63u) != 0)) {
    atomicOr(status, HB_DEV_SEGMENT);
    return 0u;
  }
  return more ? (len >> 6) : padded_blocks(len);
}


// ---------------------------------------------------------------------------
// Task sources.  A source hands the issuing side one task after another, with
// the per-lane metadata of the next task already requested from memory.

// Fixed algorithm, static grid-stride over tasks of 32 consecutive messages.
// The per-lane metadata (offset, length) of the next DEPTH tasks is in
// flight while the warp issues the current one.  For one-block messages a
// task lasts about one DRAM round trip, so the single-algorithm kernels look
// two tasks ahead (one left them waiting on these loads); the fused kernel
// spends three algorithms' work on each task and keeps one, which spares it
// registers.
template <int ALG, int DEPTH = (ALG == HB_ALL ? 1 : 2)>
struct StaticSource {
  const uint8_t* packed;
  const uint64_t* offsets;
  const uint32_t* lengths;
  uint64_t n, ntasks, stride, next;  // warp-uniform
  uint32_t lane;
  bool pf_ok[DEPTH];
  uint64_t pf_msg[DEPTH], pf_off[DEPTH];
  uint32_t pf_len[DEPTH];

  __device__ StaticSource(const KernelArgs& args, uint64_t first, uint64_t stride_, uint32_t lane_)
      : packed(args.packed),
        offsets(args.offsets),
        lengths(args.lengths),
        n(args.n),
        ntasks((args.n + 31) / 32),
        stride(stride_),
        next(first),
        lane(lane_) {
#pragma unroll
    for (int k = 0; k < DEPTH; ++k) prefetch(k);
  }

  __device__ __forceinline__ void prefetch(int k) {
    pf_ok[k] = next < ntasks;
    pf_msg[k] = next * 32 + lane;
    pf_off[k] = 0;
    pf_len[k] = 0;
    if (pf_ok[k] && pf_msg[k] < n) {
      pf_off[k] = ldg_nc_u64(offsets + pf_msg[k]);
      pf_len[k] = ldg_nc_u32(lengths + pf_msg[k]);
    }
    next += stride;
  }

  __device__ __forceinline__ void hint(uint32_t) {}

  // Move to the next task; false when the source is exhausted.
  __device__ __forceinline__ bool take(LaneTask& t) {
    if (!pf_ok[0]) return false;
    const bool valid = pf_msg[0] < n;
    t.msg = pf_msg[0];
    t.addr = reinterpret_cast<uint64_t>(packed) + pf_off[0];
    t.len = pf_len[0];
    t.nb = valid ? padded_blocks(pf_len[0]) : 0u;
    t.alg = ALG;
    t.seg = 0;
    t.slot = 0;
#pragma unroll
    for (int k = 0; k + 1 < DEPTH; ++k) {
      pf_ok[k] = pf_ok[k + 1];
      pf_msg[k] = pf_msg[k + 1];
      pf_off[k] = pf_off[k + 1];
      pf_len[k] = pf_len[k + 1];
    }
    prefetch(DEPTH - 1);
    return true;
  }
};

// Mixed algorithms: chunks of 32 bucketed messages popped from a shared
// counter in order (longest estimated cost first).  A warp reserves its next
// chunk only while it issues the last items of the current one, so no chunk
// is tied to a warp long before the warp can start it: the pop, the
// permutation load and the metadata loads are spread over the last three
// items (hint), and `take` finishes whatever is still outstanding.
template <bool SEG = false>
struct DynamicSource {
  const uint8_t* packed;
  const uint64_t* offsets;
  const uint32_t* lengths;
  const uint8_t* algs;
  const uint32_t* perm;
  const uint64_t* segs;
  const uint32_t* slot_index;
  int* status;
  uint32_t* counter;
  uint32_t* early_counter;
  uint32_t lane, nchunks;
  uint32_t early_first, early_count;  // the early queue (bucketing mode 2)
  bool early_ok;     // this warp serves the early queue first (lane 0's view)
  bool main_ok;      // the main queue may still hold work (lane 0's view)
  bool early_left;   // the early queue may still hold work (lane 0's view)
  int stage;         // 0 nothing reserved, 1 popped, 2 perm loaded, 3 metadata loaded
  uint32_t chunk;    // reserved chunk id (stage >= 1)
  uint32_t msg;      // this lane's message in it (stage >= 2)
  uint64_t off;      // stage 3
  uint32_t len, alg;
  uint64_t seg;      // stage 3, segments only
  uint32_t slot;     // stage 3, segments only

  // gwarp: the warp's index in the grid; odd warps serve the early queue
  // first (the even ones start the main queue's longest work beside them).
  __device__ DynamicSource(const KernelArgs& args, uint32_t lane_, uint64_t gwarp)
      : packed(args.packed),
        offsets(args.offsets),
        lengths(args.lengths),
        algs(args.algs),
        perm(args.perm),
        segs(args.seg),
        slot_index(args.slot_index),
        status(args.status),
        counter(args.chunk_counter),
        early_counter(args.early + 2),
        lane(lane_),
        stage(0) {
    nchunks = *args.nchunks;
    early_first = args.early[0];
    early_count = args.early[1];
    early_ok = early_count != 0 && (gwarp & 1u);
    main_ok = true;
    early_left = true;
  }

  // One more step towards having the next chunk ready (warp-uniform).
  __device__ __forceinline__ void advance() {
    if (stage == 0) {
      uint32_t c = 0;
      if (lane == 0) {
        // odd warps serve the early queue first, even warps the main queue;
        // each turns to the other queue once its own is empty, so no warp
        // stops while either queue holds work
        bool got = false;
        if (early_ok) {
          const uint32_t e = atomicAdd(early_counter, 1u);
          got = e < early_count;
          if (got) c = early_first + e;
          else early_ok = false;  // the early queue is empty: main queue from now on
        }
        if (!got && main_ok) {
          // the main queue holds every chunk outside the early range
          const uint32_t v = atomicAdd(counter, 1u);
          c = v < early_first ? v : v + early_count;
          got = c < nchunks;
          if (!got) main_ok = false;
        }
        if (!got && early_count != 0 && early_left) {
          const uint32_t e = atomicAdd(early_counter, 1u);
          got = e < early_count;
          if (got) c = early_first + e;
          else early_left = false;
        }
        if (!got) c = nchunks;  // both queues empty
      }
      chunk = __shfl_sync(kFull, c, 0);
      stage = 1;
    } else if (stage == 1) {
      msg = chunk < nchunks ? ldg_nc_u32(perm + (uint64_t)chunk * 32 + lane) : 0xFFFFFFFFu;
      stage = 2;
    } else if (stage == 2) {
      off = 0;
      len = 0;
      alg = 0;
      seg = 0;
      slot = msg;
      if (chunk < nchunks && msg != 0xFFFFFFFFu) {
        off = ldg_nc_u64(offsets + msg);
        len = ldg_nc_u32(lengths + msg);
        alg = __ldg(algs + msg);
        if constexpr (SEG) {
          seg = ldg_nc_u64(segs + msg);
          if (slot_index) slot = ldg_nc_u32(slot_index + msg);
        }
      }
      stage = 3;
    }
  }

  // Called after each issued item with the items left in the current task.
  __device__ __forceinline__ void hint(uint32_t items_left) {
    if (items_left <= 3) advance();
  }

  __device__ __forceinline__ bool take(LaneTask& t) {
    while (stage < 3) advance();
    stage = 0;
    if (chunk >= nchunks) {
      stage = 3;  // exhausted: stays exhausted
      return false;
    }
    const bool valid = msg != 0xFFFFFFFFu;
    // Codes outside {0,1,2} were excluded by the bucketing step; the chunk's
    // algorithm is that of lane 0 (every chunk starts with a real message).
    t.alg = __shfl_sync(kFull, alg, 0);
    // Lane order: a lane reads its window at word (addr / 4) % 4 of its
    // first 16-byte granule, and the slots of eight consecutive lanes start
    // in eight different groups of four banks.  Lanes whose messages share
    // that word offset are therefore put next to each other (messages in
    // order of the offset, idle lanes last): up to eight of them read
    // distinct banks, so a warp's shared loads take ceil(largest class / 8)
    // wavefronts instead of colliding wherever two lanes eight apart share
    // the offset.
    const uint64_t addr = reinterpret_cast<uint64_t>(packed) + off;
    const uint32_t cls = valid ? (uint32_t)(addr >> 2) & 3u : 4u;
    const uint32_t b0 = __ballot_sync(kFull, cls == 0u), b1 = __ballot_sync(kFull, cls == 1u);
    const uint32_t b2 = __ballot_sync(kFull, cls == 2u), b3 = __ballot_sync(kFull, cls == 3u);
    const uint32_t s1 = __popc(b0), s2 = s1 + __popc(b1), s3 = s2 + __popc(b2);
    const uint32_t s4 = s3 + __popc(b3);
    // this lane takes the message of the k-th lane (in lane order) of its class
    const uint32_t c = (lane >= s1) + (lane >= s2) + (lane >= s3) + (lane >= s4);
    const uint32_t mask = c == 0 ? b0 : c == 1 ? b1 : c == 2 ? b2 : c == 3 ? b3 : ~(b0 | b1 | b2 | b3);
    const uint32_t start = c == 0 ? 0u : c == 1 ? s1 : c == 2 ? s2 : c == 3 ? s3 : s4;
    const uint32_t from = __fns(mask, 0u, (int)(lane - start) + 1);
    const uint32_t nb = valid ? (SEG ? segment_blocks(len, seg, status) : padded_blocks(len)) : 0u;
    t.msg = __shfl_sync(kFull, (uint64_t)msg, from);
    t.addr = __shfl_sync(kFull, addr, from);
    t.len = __shfl_sync(kFull, len, from);
    t.nb = __shfl_sync(kFull, nb, from);
    if constexpr (SEG) {
      t.seg = __shfl_sync(kFull, seg, from);
      t.slot = __shfl_sync(kFull, slot, from);
    } else {
      t.seg = 0;
      t.slot = 0;
    }
    return true;
  }
};

// Relay (fused kernel): few long messages.  Tasks of 32 consecutive messages
// ("chunks") are cut into segments of seg_blocks blocks, and the warps of a
// persistent grid take (segment, chunk) items from one counter, segment by
// segment: item i is segment i / nchunks of chunk i % nchunks.  A chunk's
// chains thus move from warp to warp between segments, so every SM
// sub-partition ends up with the same share of the work even when the
// chunks are fewer than four times the sub-partitions (a grid-stride split of
// 2048 chunks over 592 sub-partitions leaves some with four and some with
// three, and the step lasts as long as the fours).  A segment that is not its
// message's last is pure message data (a whole number of blocks, no padding).
// Between segments a message's chaining values wait in its own 96-byte
// record (MD5's state in the first slot, SHA-1's in the second, SM3's in the
// third), and word 4 of the record -- spare until the final digests
// overwrite it with zeros -- counts the message's blocks done so far (zero
// before the launch).  The next segment's lane waits for that count before
// it reads the values.  Items are taken in order and each waits only on an
// item taken before it, so the earliest unfinished item can always run.
struct RelaySource {
  const uint8_t* packed;
  const uint64_t* offsets;
  const uint32_t* lengths;
  unsigned long long* counter;
  uint64_t n, nitems;
  uint32_t nchunks, seg_bytes, lane;

  __device__ RelaySource(const KernelArgs& args, uint32_t lane_)
      : packed(args.packed),
        offsets(args.offsets),
        lengths(args.lengths),
        counter(reinterpret_cast<unsigned long long*>(args.relay)),
        n(args.n),
        nchunks((uint32_t)((args.n + 31) / 32)),
        seg_bytes(args.relay_seg_blocks * 64u),
        lane(lane_) {
    // segments of the longest message: no chunk has more
    const uint32_t longest = args.relay[2];
    const uint64_t nseg = longest > seg_bytes ? ((uint64_t)longest + seg_bytes - 1) / seg_bytes : 1u;
    nitems = nseg * nchunks;
  }

  __device__ __forceinline__ void hint(uint32_t) {}

  __device__ __forceinline__ bool take(LaneTask& t) {
    while (true) {
      unsigned long long i = 0;
      if (lane == 0) i = atomicAdd(counter, 1ull);
      i = __shfl_sync(kFull, i, 0);
      if (i >= nitems) return false;
      const uint32_t chunk = (uint32_t)(i % nchunks);
      const uint32_t segment = (uint32_t)(i / nchunks);
      const uint64_t msg = (uint64_t)chunk * 32 + lane;
      uint64_t off = 0;
      uint32_t len = 0;
      bool act = false;
      if (msg < n) {
        off = ldg_nc_u64(offsets + msg);
        len = ldg_nc_u32(lengths + msg);
        // segments of this message: ceil(len / seg_bytes), at least one
        const uint32_t nseg =
            len > seg_bytes ? (uint32_t)(((uint64_t)len + seg_bytes - 1) / seg_bytes) : 1u;
        act = segment < nseg;
      }
      // an item no lane has part in (its messages are all shorter) is skipped
      if (!__any_sync(kFull, act)) continue;
      const uint64_t prior = (uint64_t)segment * seg_bytes;
      const bool more = act && prior + seg_bytes < len;
      t.msg = msg;
      t.addr = reinterpret_cast<uint64_t>(packed) + off + prior;
      t.len = act ? (more ? seg_bytes : len - (uint32_t)prior) : 0u;
      t.nb = act ? (more ? seg_bytes >> 6 : padded_blocks(t.len)) : 0u;
      t.alg = HB_ALL;
      t.seg = prior | (more ? HB_SEG_MORE : 0ull);
      t.slot = (uint32_t)msg;
      return true;
    }
  }
};

// Relay: waits, warp-uniformly, until every lane with `need` sees its
// message's block count (word 4 of its record) reach `blocks`; gives up
// after limit_ns and records HB_DEV_TIMEOUT.  The counts are read with
// acquire semantics, so the chaining values stored before them are visible.
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void relay_wait(const uint32_t* count, uint32_t blocks, bool need,
                                           uint64_t limit_ns, int* status, uint32_t lane) {
  bool ok = !need || ld_acquire_u32(count) >= blocks;
  if (__all_sync(kFull, ok)) return;
  const uint64_t t0 = global_timer_ns();
  uint32_t ns = 32;
  while (true) {
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
    if (!ok) ok = ld_acquire_u32(count) >= blocks;
    if (__all_sync(kFull, ok)) return;
    // one decision for the whole warp
    if (__any_sync(kFull, global_timer_ns() - t0 > limit_ns)) {
      if (lane == 0) atomicOr(status, HB_DEV_TIMEOUT);
      return;
    }
  }
}

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

// Per-request completion for the serving path: counts down the request's
// messages and raises its host-visible flag after the last one.
__device__ __forceinline__ void note_message_done(const KernelArgs& a, uint64_t msg) {
  if (a.msg_req == nullptr) return;
  __threadfence();  // this message's digest is visible before the count drops
  const uint32_t r = a.msg_req[msg];
  if (atomicSub(&a.req_remaining[r], 1u) == 1u) {
    __threadfence_system();
    a.req_done[r] = 1u;
  }
}

// Segment context of the block being consumed (SEG only): the bytes hashed
// by earlier segments, whether more follow, and the staged chaining value.
struct SegCtx {
  uint64_t prior;
  bool more;
  uint32_t state;  // shared address of the staged chaining value
  uint32_t slot;   // the message's 32-byte slot
};

// Where block b of a message stands (all 32-bit: b < nb <= 2^26 + 2):
//   the 0x80 marker goes into block len / 64, at byte len % 64 (the block
//   holding the message's end, or the first padding block when len is a
//   multiple of 64); the bit length fills the last two words of block nb - 1.
// A segment that is not its message's last (`more`) has neither: its last
// block (nb - 1, nb = len / 64) ends by storing the chaining value instead.

// One block of a message for all three algorithms (HB_ALL): the staged
// words feed MD5 as loaded and SHA-1 / SM3 byte-swapped; the final block
// writes the message's 96-byte record.  RELAY: the block belongs to a
// segment starting `prior` bytes into its message; a segment followed by
// more (`more`) has no padding and ends by storing the raw chaining values
// in the record, then the message's blocks done in word 4 (release).
template <bool RELAY = false>
__device__ __forceinline__ void process_block_all(AllState& st, uint32_t slot, uint32_t s,
                                                  uint32_t len, uint32_t b, uint32_t nb,
                                                  uint64_t msg, uint8_t* records,
                                                  const MulConsts& mc, bool more = false,
                                                  uint64_t prior = 0) {
  if (!(RELAY && more) && b == (len >> 6)) sts8(slot + s + (len & 63u), 0x80u);
  // One copy of the words is live at a time: MD5 takes them as loaded, then
  // they are byte-swapped in place for SHA-1 and SM3.
  uint32_t w[16];
  read_block_words<false>(slot, s, w);
  const bool last = b + 1 == nb;
  const bool final_block = last && !(RELAY && more);
  // bit length of the whole message mod 2^64
  const uint64_t bits = RELAY ? (prior + len) << 3 : (uint64_t)len << 3;
  const uint32_t lo = (uint32_t)bits, hi = (uint32_t)(bits >> 32);
  if (final_block) {
    w[14] = lo;
    w[15] = hi;
  }
#if HB_FUSED_INTERLEAVE
  uint32_t y[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) y[i] = bswap32(w[i]);
  if (final_block) {
    y[14] = hi;
    y[15] = lo;
  }
  sha1_compress(st.sha1, y, mc);
  md5_sm3_compress<kMd5FusedFma>(st.md5, st.sm3, w, y, mc);
#else
  md5_compress<kMd5FusedFma, kMd5FusedXt>(st.md5, w, mc);
#pragma unroll
  for (int i = 0; i < 16; ++i) w[i] = bswap32(w[i]);
  if (final_block) {
    w[14] = hi;
    w[15] = lo;
  }
  sha1_compress(st.sha1, w, mc);
  sm3_compress<HB_SM3_ROLLED != 0, kSm3FusedS0Fma>(st.sm3, w, mc);
#endif
  if (final_block) {
    uint8_t* dst = records + msg * HB_ALL_RECORD_BYTES;
    uint32_t o[8];
    alg_digest_words<HB_MD5>(st.md5, o);
    stg128_cs(dst, o[0], o[1], o[2], o[3]);
    stg128_cs(dst + 16, o[4], o[5], o[6], o[7]);
    alg_digest_words<HB_SHA1>(st.sha1, o);
    stg128_cs(dst + 32, o[0], o[1], o[2], o[3]);
    stg128_cs(dst + 48, o[4], o[5], o[6], o[7]);
    alg_digest_words<HB_SM3>(st.sm3, o);
    stg128_cs(dst + 64, o[0], o[1], o[2], o[3]);
    stg128_cs(dst + 80, o[4], o[5], o[6], o[7]);
  } else if (RELAY && more && last) {
    uint8_t* dst = records + msg * HB_ALL_RECORD_BYTES;
    stg128_cs(dst, st.md5[0], st.md5[1], st.md5[2], st.md5[3]);
    stg128_cs(dst + 32, st.sha1[0], st.sha1[1], st.sha1[2], st.sha1[3]);
    stg128_cs(dst + 48, st.sha1[4], 0u, 0u, 0u);
    stg128_cs(dst + 64, st.sm3[0], st.sm3[1], st.sm3[2], st.sm3[3]);
    stg128_cs(dst + 80, st.sm3[4], st.sm3[5], st.sm3[6], st.sm3[7]);
    const uint32_t done = (uint32_t)((prior + len) >> 6);
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(dst + 16), "r"(done) : "memory");
  }
}

template <int ALG, bool SEG = false>
__device__ __forceinline__ void process_block(uint32_t (&st)[8], uint32_t slot, uint32_t s,
                                              uint32_t len, uint32_t b, uint32_t nb, uint64_t msg,
                                              uint8_t* digests, const MulConsts& mc,
                                              const KernelArgs& a, const SegCtx& sc = SegCtx{}) {
  constexpr bool BE = AlgTraits<ALG>::kBigEndian;
  const bool more = SEG && sc.more;
  if (!more && b == (len >> 6)) sts8(slot + s + (len & 63u), 0x80u);
  uint32_t w[16];
  read_block_words<BE>(slot, s, w);
  const bool last = b + 1 == nb;
  const bool final_block = !more && last;
  if (final_block) {
    // bit length of the whole message mod 2^64
    const uint64_t bits = SEG ? (sc.prior + len) << 3 : (uint64_t)len << 3;
    const uint32_t lo = (uint32_t)bits, hi = (uint32_t)(bits >> 32);
    w[14] = BE ? hi : lo;
    w[15] = BE ? lo : hi;
  }
  alg_compress<ALG>(st, w, mc);
  if (final_block) {
    uint32_t o[8];
    alg_digest_words<ALG>(st, o);
    uint8_t* dst = digests + (SEG ? (uint64_t)sc.slot : msg) * HB_SLOT_BYTES;
    stg128_cs(dst, o[0], o[1], o[2], o[3]);
    stg128_cs(dst + 16, o[4], o[5], o[6], o[7]);
    note_message_done(a, msg);
  } else if (more && last) {
    // last block of a segment that is not the message's last: keep the
    // chaining value (words past the algorithm's state are zero)
    constexpr int kW = AlgTraits<ALG>::kStateWords;
    uint8_t* dst = digests + (uint64_t)sc.slot * HB_SLOT_BYTES;
    stg128_cs(dst, st[0], st[1], st[2], st[3]);
    stg128_cs(dst + 16, kW > 4 ? st[4] : 0u, kW > 5 ? st[5] : 0u, kW > 6 ? st[6] : 0u,
              kW > 7 ? st[7] : 0u);
  }
}

// ---------------------------------------------------------------------------
// The warp loop.  MIXED selects the algorithm per item (warp-uniform);
// otherwise ALG is fixed.

// Consumes the KB blocks of one stage for one lane (blocks past the
// message's padded length are skipped).  A message's chain starts in the
// stage that holds its block 0: from the algorithm's initial value, or, for
// a later segment, from the chaining value staged with it (SEG) or left in
// the message's record by the warp that ran the previous segment (RELAY;
// read through L2 after relay_wait).
template <int ALG, int KB, bool SEG = false, bool RELAY = false>
__device__ __forceinline__ void process_stage(typename StateFor<ALG>::type& st, uint32_t slot,
                                              uint32_t s, uint32_t len, uint32_t b0, uint64_t msg,
                                              const KernelArgs& a, const SegCtx& sc = SegCtx{}) {
  const uint32_t nb = ((SEG || RELAY) && sc.more) ? (len >> 6) : padded_blocks(len);
  if (b0 == 0) {
    if constexpr (ALG == HB_ALL) {
      if (RELAY && sc.prior != 0) {
        const uint4* r = reinterpret_cast<const uint4*>(a.digests + msg * HB_ALL_RECORD_BYTES);
        const uint4 m = __ldcg(r), h0 = __ldcg(r + 2), h1 = __ldcg(r + 3);
        const uint4 s0 = __ldcg(r + 4), s1 = __ldcg(r + 5);
        st.md5[0] = m.x; st.md5[1] = m.y; st.md5[2] = m.z; st.md5[3] = m.w;
        st.sha1[0] = h0.x; st.sha1[1] = h0.y; st.sha1[2] = h0.z; st.sha1[3] = h0.w;
        st.sha1[4] = h1.x;
        st.sm3[0] = s0.x; st.sm3[1] = s0.y; st.sm3[2] = s0.z; st.sm3[3] = s0.w;
        st.sm3[4] = s1.x; st.sm3[5] = s1.y; st.sm3[6] = s1.z; st.sm3[7] = s1.w;
      } else {
        md5_init(st.md5);
        sha1_init(st.sha1);
        sm3_init(st.sm3);
      }
    } else if (SEG && sc.prior != 0) {
      const uint4 v0 = lds128(sc.state), v1 = lds128(sc.state + 16);
      st[0] = v0.x; st[1] = v0.y; st[2] = v0.z; st[3] = v0.w;
      st[4] = v1.x; st[5] = v1.y; st[6] = v1.z; st[7] = v1.w;
    } else {
      alg_init<ALG>(st);
    }
  }
  const uint32_t nj = nb - b0 < (uint32_t)KB ? nb - b0 : (uint32_t)KB;
#pragma unroll 1
  for (uint32_t j = 0; j < nj; ++j) {
    if constexpr (ALG == HB_ALL)
      process_block_all<RELAY>(st, slot + 64 * j, s, len, b0 + j, nb, msg, a.digests, a.mc,
                               sc.more, sc.prior);
    else
      process_block<ALG, SEG>(st, slot + 64 * j, s, len, b0 + j, nb, msg, a.digests, a.mc, a, sc);
  }
}

// COOP selects the copy mapping.  false: every lane copies the granules of
// its own window (one instruction touches 32 messages).  true: the warp copies
// window after window, consecutive lanes taking consecutive granules of the
// same message, so one instruction touches two or three messages -- far fewer
// distinct pages per instruction when the messages lie far apart.  Lanes then
// read windows that other lanes copied, so the warp synchronises after the
// copy wait and before a stage is reused.
// RELAY (with ALG == HB_ALL and a RelaySource): items are segments whose
// chaining values come from other warps, see RelaySource.
template <int STAGES, int KB, bool COOP, int ALG, bool MIXED, bool SEG, bool RELAY = false,
          class Source>
__device__ __forceinline__ void warp_pipeline(Source& src, uint8_t* wsm, const KernelArgs& a,
                                              uint32_t lane) {
  static_assert(!RELAY || (ALG == HB_ALL && !MIXED && !SEG), "relay: fused kernel only");
  using L = WarpSmem<STAGES, KB, SEG, RELAY>;
  constexpr int kSlotBytes = Slot<KB>::kBytes;
  constexpr int kGranules = 4 * KB + 1;
  const uint32_t slots = smem_addr(wsm);
  const uint32_t items = slots + L::kSlots;
  const uint32_t table = items + L::kItems;
  const uint32_t seg_items = table + L::kTable;      // SEG or RELAY
  const uint32_t states = seg_items + L::kSegItems;  // SEG only
  const uint64_t safe_src = reinterpret_cast<uint64_t>(a.packed) & ~15ull;

  // Issuing side state (warp-uniform except the LaneTask fields).
  LaneTask t;
  bool have = src.take(t);
  uint32_t maxnb = have ? __reduce_max_sync(kFull, t.nb) : 0u;
  uint32_t ib = 0;  // first block of the next stage to issue
  int is = 0;       // stage the next issue goes to

  // Consuming side state.
  int cs = 0;
  typename StateFor<MIXED ? HB_MD5 : ALG>::type st;
  int inflight = 0;

  auto issue = [&]() {
    const bool act = ib < t.nb;
    uint4 rec;
    rec.x = (uint32_t)t.msg;
    rec.y = (uint32_t)(t.msg >> 32) | ((uint32_t)(t.addr & 15u) << 24) | (t.alg << 28);
    rec.z = t.len;
    rec.w = act ? ib : kNoBlock;
    sts128(items + (is * 32 + lane) * kItemBytes, rec);
    if constexpr (SEG || RELAY) {
      sts128(seg_items + (is * 32 + lane) * kItemBytes,
             make_uint4((uint32_t)t.seg, (uint32_t)(t.seg >> 32), t.slot, 0u));
      // a continued message's first item also stages its chaining value
      // (SEG: written by an earlier launch; a relay's comes from a warp of
      // this launch and is read when the stage is consumed)
      if (SEG && act && ib == 0 && (t.seg & ~HB_SEG_MORE) != 0) {
        const uint8_t* cv = a.digests + (uint64_t)t.slot * HB_SLOT_BYTES;
        const uint32_t dst = states + (is * 32 + lane) * HB_SLOT_BYTES;
        cp_async16_zfill(dst, cv, 16u);
        cp_async16_zfill(dst + 16, cv + 16, 16u);
      }
    }
    // This lane's window: first granule and message bytes from there on.
    uint64_t g0 = 0;
    int32_t avail = 0;
    if (act) {
      const uint64_t A = t.addr + 64ull * ib;            // window start
      g0 = A & ~15ull;                                   // first granule
      const uint64_t end = t.addr + t.len;               // one past the last message byte
      const uint64_t left = end > g0 ? end - g0 : 0ull;  // message bytes from g0 on
      avail = left > (uint64_t)kSlotBytes ? kSlotBytes : (int32_t)left;
    }
    if constexpr (!COOP) {
      if (act) {
        const uint32_t dst = slots + (is * 32 + lane) * kSlotBytes;
        const bool extra = (t.addr & 15u) != 0u;  // unaligned window needs one more granule
        if (avail == kSlotBytes) {
          // the whole slot lies inside the message (the usual case in a long
          // message): every granule is a full one
#pragma unroll
          for (int g = 0; g < kGranules; ++g)
            if (g < kGranules - 1 || extra)
              cp_async16_zfill(dst + 16 * g, reinterpret_cast<const void*>(g0 + 16ull * g), 16u);
        } else {
#pragma unroll
          for (int g = 0; g < kGranules; ++g) {
            const int32_t v = avail - 16 * g;
            const uint32_t nbytes = v <= 0 ? 0u : (v >= 16 ? 16u : (uint32_t)v);
            const uint64_t from = nbytes ? g0 + 16ull * g : safe_src;
            if (g < kGranules - 1 || extra)
              cp_async16_zfill(dst + 16 * g, reinterpret_cast<const void*>(from), nbytes);
          }
        }
      }
    } else {
      // Publish this lane's window, then copy the 32 windows message-major:
      // each round copies the 4*KB aligned granules of 32 / (4*KB) windows,
      // lane l taking granule l % (4*KB) of window r * 32/(4*KB) + l / (4*KB);
      // a last round copies each lane's own trailing granule (present only
      // when its window is not 16-byte aligned).
      sts128(table + lane * 16, make_uint4((uint32_t)g0, (uint32_t)(g0 >> 32), (uint32_t)avail, 0u));
      __syncwarp();
      constexpr int kMain = 4 * KB;            // granules every window has
      constexpr int kPerRound = 32 / kMain;    // windows per round
      const uint32_t gi = lane % kMain;
      const uint32_t mlo = lane / kMain;
      const uint32_t tab = table + mlo * 16;
      const uint32_t dst0 = slots + (is * 32 + mlo) * kSlotBytes + 16 * gi;
      if (__all_sync(kFull, avail == kSlotBytes)) {
        // every lane's whole slot lies inside its message (the usual case in
        // long messages): full granules, no clamping
#pragma unroll
        for (int r = 0; r < kMain; ++r) {
          const uint4 e = lds128(tab + 16 * kPerRound * r);
          const uint64_t from = (((uint64_t)e.y << 32) | e.x) + 16ull * gi;
          cp_async16_zfill(dst0 + kPerRound * kSlotBytes * r, reinterpret_cast<const void*>(from),
                           16u);
        }
        if ((t.addr & 15u) != 0u)
          cp_async16_zfill(slots + (is * 32 + lane) * kSlotBytes + 16 * kMain,
                           reinterpret_cast<const void*>(g0 + 16ull * kMain), 16u);
      } else {
#pragma unroll
        for (int r = 0; r < kMain; ++r) {
          const uint4 e = lds128(tab + 16 * kPerRound * r);
          const int32_t v = (int32_t)e.z - 16 * (int32_t)gi;
          const uint32_t nbytes = v <= 0 ? 0u : (v >= 16 ? 16u : (uint32_t)v);
          const uint64_t from = nbytes ? (((uint64_t)e.y << 32) | e.x) + 16ull * gi : safe_src;
          cp_async16_zfill(dst0 + kPerRound * kSlotBytes * r, reinterpret_cast<const void*>(from),
                           nbytes);
        }
        if (act && (t.addr & 15u) != 0u) {
          const int32_t v = avail - 16 * kMain;
          const uint32_t nbytes = v <= 0 ? 0u : (v >= 16 ? 16u : (uint32_t)v);
          const uint64_t from = nbytes ? g0 + 16ull * kMain : safe_src;
          cp_async16_zfill(slots + (is * 32 + lane) * kSlotBytes + 16 * kMain,
                           reinterpret_cast<const void*>(from), nbytes);
        }
      }
    }
    ++inflight;
    is = (is + 1 == STAGES) ? 0 : is + 1;
    ib += KB;
    src.hint(ib >= maxnb ? 0u : (maxnb - ib + KB - 1) / KB);
    if (ib >= maxnb) {
      have = src.take(t);
      maxnb = have ? __reduce_max_sync(kFull, t.nb) : 0u;
      ib = 0;
    }
  };

#pragma unroll 1
  for (int k = 0; k < STAGES - 1; ++k) {
    if (have) issue();
    cp_async_commit();
  }

#pragma unroll 1
  while (inflight > 0) {
    if (have) issue();
    cp_async_commit();
    cp_async_wait<STAGES - 1>();  // this lane's copies of item `cs` have landed
    if constexpr (COOP) __syncwarp();  // ... and every other lane's
    const uint4 rec = lds128(items + (cs * 32 + lane) * kItemBytes);
    uint64_t r_prior = 0;
    bool r_more = false;
    if constexpr (RELAY) {
      // a continued segment's first stage: wait for the previous segment's
      // chaining values (every lane of the warp takes part)
      const uint4 r2 = lds128(seg_items + (cs * 32 + lane) * kItemBytes);
      const uint64_t sg = (uint64_t)r2.x | ((uint64_t)r2.y << 32);
      r_prior = sg & ~HB_SEG_MORE;
      r_more = (sg & HB_SEG_MORE) != 0;
      const bool need = rec.w == 0 && r_prior != 0;
      if (__any_sync(kFull, need)) {
        const uint64_t m = (uint64_t)rec.x | ((uint64_t)(rec.y & 0x00FFFFFFu) << 32);
        const uint32_t* count =
            reinterpret_cast<const uint32_t*>(a.digests + m * HB_ALL_RECORD_BYTES + 16);
        relay_wait(count, (uint32_t)(r_prior >> 6), need, a.wait_limit_ns, a.status, lane);
      }
    }
    if (rec.w != kNoBlock) {
      const uint64_t msg = (uint64_t)rec.x | ((uint64_t)(rec.y & 0x00FFFFFFu) << 32);
      const uint32_t s = (rec.y >> 24) & 15u;
      const uint32_t slot = slots + (cs * 32 + lane) * kSlotBytes;
      if constexpr (MIXED) {
        const uint32_t alg = rec.y >> 28;
        SegCtx sc{};
        if constexpr (SEG) {
          const uint4 r2 = lds128(seg_items + (cs * 32 + lane) * kItemBytes);
          const uint64_t sg = (uint64_t)r2.x | ((uint64_t)r2.y << 32);
          sc.prior = sg & ~HB_SEG_MORE;
          sc.more = (sg & HB_SEG_MORE) != 0;
          sc.state = states + (cs * 32 + lane) * HB_SLOT_BYTES;
          sc.slot = r2.z;
        }
        if (alg == HB_MD5)
          process_stage<HB_MD5, KB, SEG>(st, slot, s, rec.z, rec.w, msg, a, sc);
        else if (alg == HB_SHA1)
          process_stage<HB_SHA1, KB, SEG>(st, slot, s, rec.z, rec.w, msg, a, sc);
        else
          process_stage<HB_SM3, KB, SEG>(st, slot, s, rec.z, rec.w, msg, a, sc);
      } else if constexpr (RELAY) {
        SegCtx sc{};
        sc.prior = r_prior;
        sc.more = r_more;
        process_stage<ALG, KB, false, true>(st, slot, s, rec.z, rec.w, msg, a, sc);
      } else {
        process_stage<ALG, KB>(st, slot, s, rec.z, rec.w, msg, a);
      }
    }
    --inflight;
    cs = (cs + 1 == STAGES) ? 0 : cs + 1;
    if constexpr (COOP) __syncwarp();  // stage cs - 1 is free for the next copies
  }
}

}  // namespace hb
