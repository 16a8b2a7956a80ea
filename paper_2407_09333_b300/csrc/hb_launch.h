// hb_launch.h -- internal interface between the kernels (hb_kernels.cu) and
// the C-ABI layer (hb_capi.cu).  Not installed; not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "hashbatch.h"

namespace hb {

// Factors for moving adds and rotations onto the multiply-add pipe (see
// hb_device.cuh): one = 1, pow2[s] = 2^s.  Passed as kernel arguments so the
// compiler cannot fold them.
struct MulConsts {
  uint32_t one;
  uint32_t pow2[32];
};

inline MulConsts make_mul_consts() {
  MulConsts m;
  m.one = 1u;
  for (int s = 0; s < 32; ++s) m.pow2[s] = 1u << s;
  return m;
}

// Kernel arguments for the hashing kernels (plain and mixed).
struct KernelArgs {
  const uint8_t* packed;
  const uint64_t* offsets;
  const uint32_t* lengths;
  const uint8_t* algs;        // mixed path only
  const uint32_t* perm;       // mixed path only: chunk slot -> message index
  uint32_t* chunk_counter;    // mixed path only
  const uint32_t* nchunks;    // mixed path only
  uint32_t* early;            // mixed path only: MixedWorkspace::early
  uint64_t n;
  uint8_t* digests;
  int* status;                // per-device status word (HB_DEV_* bits)
  const int* abort_flag;      // optional: skip all work when *abort_flag != 0
  uint64_t wait_limit_ns;
  MulConsts mc;
  // Optional per-request completion (serving): message i belongs to request
  // msg_req[i]; the lane that finishes a request's last message sets
  // req_done[request] = 1 (host-visible memory) after its digests are stored.
  const uint32_t* msg_req;
  uint32_t* req_remaining;
  volatile uint32_t* req_done;
  // Optional segments (mixed path): seg[i] = bytes of message i hashed by
  // earlier calls (a multiple of 64) | HB_SEG_MORE when more segments follow.
  // Between segments the message's 32-byte slot carries its chaining value.
  const uint64_t* seg;
  // Optional with segments: message i's slot is slot_index[i] instead of i.
  const uint32_t* slot_index;
  // Relay (fused kernel, hb_pipeline.cuh): relay[0..1] is the 64-bit count of
  // (segment, chunk) items taken, relay[2] the longest message length, both
  // set before the launch; nullptr for the grid-stride kernels.
  uint32_t* relay;
  uint32_t relay_seg_blocks;  // blocks per segment (a multiple of the stage's blocks)
};

// Ragged-path bucketing: groups are (cost bucket, algorithm) pairs ordered
// from the most to the least expensive estimated work per message.  Cost
// buckets split each octave of estimated cost into 2^sub_log2 parts
// (sub_log2 <= 6, so at most 32 * 64 buckets): the finer the buckets, the
// closer the lengths of a chunk's 32 messages, and the fewer lanes idle
// while the chunk's longest message finishes.  With alg_major the order is
// all SM3 groups, then SHA-1, then MD5 (each longest first), so that warps
// running at the same time mostly run the same algorithm; otherwise the
// algorithms interleave bucket by bucket (strict longest-first).
constexpr uint32_t kMaxSubLog2 = 6;
constexpr uint32_t kCostBuckets = 32u << kMaxSubLog2;
constexpr uint32_t kGroups = kCostBuckets * 3;

struct BucketCfg {
  uint32_t sub_log2;   // 0..kMaxSubLog2
  uint32_t alg_major;  // 0 interleaved, 1 algorithm-major, 2 algorithm-major with MD5's
                       // two longest octaves served early (MixedWorkspace::early)
};

constexpr BucketCfg kDefaultBuckets = {6u, 2u};

// Default launch of the persistent ragged kernel: shape 19 (1-warp blocks, 2
// stages of 4 blocks, cooperative copies) with 8 resident warps per SM, i.e.
// two per SM sub-partition.  A long message is a serial chain of blocks; with
// more co-resident warps its warp gets a smaller share of the sub-partition's
// issue slots and the longest chains finish last (MD5 saturates a
// sub-partition at about four warps, SHA-1 and SM3 at two).
constexpr int kDefaultMixedShape = 19;
constexpr int kDefaultMixedWarpsPerSm = 8;

// Device scratch of the ragged path; followed in memory by the permutation
// array of (n + 31 * kGroups) uint32 entries.
struct MixedWorkspace {
  uint32_t counts[kGroups];
  uint32_t cursor[kGroups];
  uint32_t chunk_counter;
  uint32_t nchunks;
  // alg_major == 2: chunks [early[0], early[0] + early[1]) -- MD5's two
  // longest octaves -- form a second queue (pop counter early[2]) that every other
  // warp serves first, so those chains start with the SM3 phase instead of
  // after every SM3 and SHA-1 chunk (where they would end the launch late)
  uint32_t early[3];
  uint32_t pad[27];
};

inline size_t mixed_workspace_bytes(uint64_t n) {
  return sizeof(MixedWorkspace) + (size_t)(n + 31ull * kGroups) * sizeof(uint32_t);
}

struct MixedArgs {
  BucketCfg cfg;
  const uint8_t* algs;
  const uint32_t* lengths;
  uint64_t n;
  const uint64_t* n_dev;  // when set, the message count is read from here (captured graphs)
  uint8_t* digests;
  MixedWorkspace* ws;
  uint32_t* perm;
  const uint32_t* slot_index;  // optional (segments): slot of message i
};

int num_shapes();
bool shape_desc(int shape, int* warps, int* stages, int* kb = nullptr, int* coop = nullptr);
int shape_smem_bytes(int shape, bool seg = false);

// Sets the kernel's shared-memory attribute and returns its occupancy.  `seg`
// selects the segment-aware variant of the mixed kernel.
cudaError_t prepare_kernel(bool mixed, int alg, int shape, int* blocks_per_sm, bool seg = false);
// The mixed path launches the segment-aware variant when a.seg is set.
cudaError_t launch_hash(bool mixed, int alg, int shape, int grid, const KernelArgs& a,
                        cudaStream_t stream);
cudaError_t launch_bucketing(const MixedArgs& m, int grid, cudaStream_t stream);
// The fused kernel's relay form (a.relay set): shared-memory attribute and
// occupancy, the launch, and the setup before it (item counter zeroed, the
// longest length into relay[2], the blocks-done word of every record whose
// message spans more than one segment zeroed).
constexpr uint32_t kDefaultRelaySegBlocks = 64;
cudaError_t prepare_relay(int shape, int* blocks_per_sm);
cudaError_t launch_relay(int shape, int grid, const KernelArgs& a, cudaStream_t stream);
cudaError_t launch_relay_setup(const uint32_t* lengths, uint64_t n, uint32_t seg_bytes,
                               uint8_t* records, uint32_t* relay, int grid, cudaStream_t stream);
cudaError_t launch_bounds(const uint64_t* offsets, const uint32_t* lengths, uint64_t n,
                          uint64_t packed_len, int* status_dev, int* ctx_status, int grid,
                          cudaStream_t stream);
// Digests of the 9-character decimal strings of first .. first + count - 1.
cudaError_t launch_digits(int alg, uint64_t first, uint64_t count, uint8_t* digests, int grid,
                          cudaStream_t stream);
// offsets[i] -= base for i < n.
// Packs n slots of `rec` bytes (32, or 96 for three-algorithm records) into
// n x dsz bytes of digest (dsz = 16, 20, 32, or 68 for a record).
cudaError_t launch_pack(const uint8_t* slots, uint32_t rec, uint64_t n, uint8_t* out, uint32_t dsz,
                        int grid, cudaStream_t stream);
cudaError_t launch_rebase(uint64_t* offsets, uint64_t n, uint64_t base, int grid,
                          cudaStream_t stream);
// flag = 1 when offsets[i] + lengths[i] decreases anywhere in index order.
cudaError_t launch_monotone(const uint64_t* offsets, const uint32_t* lengths, uint64_t n, int* flag,
                            int grid, cudaStream_t stream);
cudaError_t launch_int_peak(int op, int blocks, int threads, int iters, unsigned long long* cycles,
                            uint32_t* sink, cudaStream_t stream);
cudaError_t launch_selftest_wait(uint64_t limit_ns, int* status, cudaStream_t stream);
// Request-packing copies of the serving path (hash_gather).
using HbCopy = hb_copy;
cudaError_t launch_gather(const HbCopy* copies, uint32_t count, int grid, cudaStream_t stream);
// Writes the message count a captured ragged graph reads (one tiny kernel).
cudaError_t launch_set_count(uint64_t* n_dev, uint64_t n, cudaStream_t stream);

// The current device's status word (HB_DEV_* bits, read by
// hash_device_status); creates the device context on first use.  nullptr
// when that fails.
int* current_status_word();

// Device-side wait limit of the hashing kernels (hash_set_wait_limit_ns).
uint64_t wait_limit_ns();

// HB_DEV_* bits recorded by hash_batch_mixed_noalloc's kernels on the current
// device since the last call (its status word lives in its fixed scratch
// array, not in the device context), cleared as they are read.  Synchronous;
// allocates nothing.  0 when that entry point has not run on this device.
cudaError_t noalloc_take_status(int* bits);

}  // namespace hb
