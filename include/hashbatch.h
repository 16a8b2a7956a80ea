/*
 * hashbatch.h -- C-ABI of libhashbatch.so: MD5, SHA-1 and SM3 digests of a
 * large batch of independent messages on one NVIDIA B300 (sm_103a).
 *
 * What is computed.  The "parallel scenario" hash operations of the paper
 * (Sec. IV-B: digests of many messages computed at once; Sec. V-D: every
 * input message and every output digest sits in its own array location, so
 * the work is free of data races).  Each digest is the standard one:
 *   HB_MD5   RFC 1321                      16-byte digest
 *   HB_SHA1  FIPS 180-4 Sec. 6.1           20-byte digest
 *   HB_SM3   GB/T 32905-2016               32-byte digest
 * Messages are byte strings of 0 .. 2^32-1 bytes; padding (0x80, zeros,
 * 64-bit bit length) is done on the device.
 *
 * Layout (all entry points).
 *   packed_bytes  message bytes; message i is
 *                 packed_bytes[offsets[i] .. offsets[i] + lengths[i]).
 *                 Messages may start at any byte and may overlap (they are
 *                 only read).  Reads are done in 16-byte aligned granules:
 *                 up to 15 bytes before a message's first byte and after its
 *                 last byte are read (never used), so those bytes must lie in
 *                 mapped device memory -- always true inside one cudaMalloc
 *                 allocation, whose granularity is far above 16 bytes.
 *   offsets       uint64 per message (byte offsets into packed_bytes).
 *   lengths       uint32 per message (byte counts).
 *   algs          uint8 per message (HB_MD5 / HB_SHA1 / HB_SM3), mixed calls.
 *   digests_out   HB_SLOT_BYTES (32) bytes per message, 16-byte aligned:
 *                 slot i holds hash_digest_size(alg) digest bytes in the
 *                 standard's output byte order, then zero bytes.
 *
 * Ownership.  Every pointer is owned by the caller.  Unless an entry point
 * says "host", pointers are CUDA device pointers of the current device.  The
 * library keeps a small per-device context (status word, scratch for the
 * mixed path, captured graphs) created on first use and freed at process
 * exit or by hash_release_device().
 *
 * Asynchrony.  Device calls are enqueued on `stream` (a cudaStream_t; NULL
 * is the legacy default stream) and return without waiting.  The return
 * value reports argument and launch errors only.  Errors found by a kernel
 * (a bounded wait that timed out, a bounds violation seen by the checker,
 * a malformed segment) are OR-ed into a per-device status word read by hash_device_status().
 *
 * Errors.  0 is success; negative values are the HB_ERR_* codes below;
 * hash_strerror() names them.  n == 0 is a successful no-op.
 */
#ifndef HASHBATCH_H
#define HASHBATCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Algorithm codes (the same codes appear in the per-message `algs` array). */
#define HB_MD5 0
#define HB_SHA1 1
#define HB_SM3 2

#define HB_SLOT_BYTES 32
/* All three algorithms on every message (hash_batch_all): one 96-byte record
 * per message holding the MD5, SHA-1 and SM3 slots in that order.  Also the
 * tuning code of the fused kernel (hash_tune_set / get / occupancy). */
#define HB_ALL 4
#define HB_ALL_RECORD_BYTES 96

/* Return codes. */
#define HB_OK 0
#define HB_ERR_INVALID_ALG (-1)   /* algorithm code not 0, 1 or 2            */
#define HB_ERR_NULL (-2)          /* a required pointer is NULL with n > 0   */
#define HB_ERR_TOO_LARGE (-3)     /* n or a size exceeds a documented limit  */
#define HB_ERR_CUDA (-4)          /* a CUDA runtime call or launch failed    */
#define HB_ERR_NOMEM (-5)         /* device or pinned workspace allocation   */
#define HB_ERR_TIMEOUT (-6)       /* a device-side wait gave up (status)     */
#define HB_ERR_ALIGN (-7)         /* digests_out not 16-byte aligned         */
#define HB_ERR_BOUNDS (-8)        /* a message lies outside packed_len       */
#define HB_ERR_BUDGET (-9)        /* request exceeds the serving budget      */
#define HB_ERR_ARG (-10)          /* any other invalid argument              */

/* Device status bits (hash_device_status). */
#define HB_DEV_TIMEOUT 0x1        /* a kernel's bounded wait expired         */
#define HB_DEV_BOUNDS 0x2         /* hash_batch_check_bounds found a message
                                     outside [0, packed_len), or a streaming
                                     round met a request index outside its
                                     table                                   */
#define HB_DEV_SEGMENT 0x4        /* a segment that is not the last was not a
                                     whole number of 64-byte blocks, or its
                                     prior byte count was not (message skipped) */

/* Digest size in bytes of an algorithm (16, 20, 32); 0 for an unknown code. */
size_t hash_digest_size(int alg);

/* Static description of a return code. */
const char *hash_strerror(int code);

/* The CUDA runtime's description of the last CUDA failure that made an entry
 * point return HB_ERR_CUDA or HB_ERR_NOMEM on the calling thread. */
const char *hash_last_cuda_error(void);

/*
 * hash_batch -- one algorithm for the whole batch (paper Sec. IV-B, parallel
 * op; Sec. V-D, separate slots).  One message per GPU thread; each warp stages
 * the next 64-byte blocks of its 32 messages into shared memory with
 * asynchronous 16-byte copies while it compresses the current ones.
 * Returns HB_OK, HB_ERR_INVALID_ALG, HB_ERR_NULL, HB_ERR_ALIGN, HB_ERR_CUDA.
 * Limits: n < 2^40.
 */
int hash_batch(int alg, const uint8_t *packed_bytes, const uint64_t *offsets,
               const uint32_t *lengths, uint64_t n, uint8_t *digests_out,
               void *stream);

/*
 * hash_batch_all -- MD5, SHA-1 and SM3 of every message in one pass: each
 * message's bytes are staged once and every staged block feeds the three
 * compression functions (little-endian words for MD5, byte-swapped words for
 * SHA-1 and SM3).  records_out is a device array of n 96-byte records
 * (16-byte aligned): record i holds message i's MD5, SHA-1 and SM3 slots, each
 * laid out as hash_batch writes it.  Same results as three hash_batch calls,
 * one read of the input instead of three.  Returns as hash_batch.
 * A batch of between 2 and 8 x 32 messages per SM sub-partition (4 per SM)
 * runs, outside stream capture, as a relay (hash_tune_relay): long messages
 * are hashed in segments whose chains pass from warp to warp, so that every
 * sub-partition gets the same share; between segments a message's chaining
 * values are kept in its own record.  Such a call also uses 16 bytes of
 * per-device scratch, ordered with other relay calls by an event.
 */
int hash_batch_all(const uint8_t *packed_bytes, const uint64_t *offsets,
                   const uint32_t *lengths, uint64_t n, uint8_t *records_out, void *stream);

/*
 * hash_batch_mixed -- per-message algorithm, for ragged batches: messages are
 * bucketed on the device by (estimated cost, algorithm), longest first, and
 * one persistent launch hashes 32-message chunks popped from a shared
 * counter.  Uses a per-device scratch area owned by the library (grown on
 * demand with cudaMalloc; calls on different streams are ordered through an
 * event so they never share it concurrently).  Algorithm codes outside
 * {0,1,2} leave their slot zeroed and set nothing else.
 * Limits: n < 2^31.  Returns as hash_batch, plus HB_ERR_NOMEM / HB_ERR_TOO_LARGE.
 */
int hash_batch_mixed(const uint8_t *algs, const uint8_t *packed_bytes,
                     const uint64_t *offsets, const uint32_t *lengths, uint64_t n,
                     uint8_t *digests_out, void *stream);

/*
 * hash_batch_segments -- hash_batch_mixed over pieces ("segments") of
 * messages, so that a long message can be hashed over several calls with only
 * its current piece in device memory (the serving loop streams long messages
 * this way).  The iterated compression of RFC 1321 Sec. 3.4, FIPS 180-4
 * Sec. 6.1.2 / the SHA-1 loop, and GB/T 32905 Sec. 5.3 only needs the chaining
 * value between blocks; it travels from one segment to the next in the
 * message's 32-byte slot.
 *   seg[i] = P | (more ? HB_SEG_MORE : 0): P = bytes of message i hashed by
 *   earlier calls (a multiple of 64, below 2^61); HB_SEG_MORE marks a segment
 *   that is not the message's last.  packed_bytes + offsets[i] holds the
 *   segment's lengths[i] bytes.
 *   - P == 0: the chain starts from the algorithm's initial value.
 *     P > 0: slots_inout[i] must hold what the call with the previous
 *     segment left in its slot (copy the 32 bytes if the index changes).
 *   - more: lengths[i] must be a multiple of 64; afterwards slot i holds the
 *     chaining value (internal format, 32 bytes; pass it back unchanged).
 *   - last: slot i receives the digest of the whole message (P + lengths[i]
 *     bytes), exactly as hash_batch_mixed would for the whole message.
 *   A segment that breaks a multiple-of-64 rule is skipped and sets
 *   HB_DEV_SEGMENT in the device status (hash_device_status).
 *   slot_index (optional, device uint32): message i uses slot
 *   slots_inout + 32 * slot_index[i] instead of slot i, so a message can keep
 *   one slot while its position changes from call to call.  NULL = slot i.
 * Consecutive segments of one message must be ordered (same stream, or an
 * event between the calls).  Limits and return codes as hash_batch_mixed.
 */
#define HB_SEG_MORE (1ull << 63)
int hash_batch_segments(const uint8_t *algs, const uint8_t *packed_bytes,
                        const uint64_t *offsets, const uint32_t *lengths,
                        const uint64_t *seg, const uint32_t *slot_index, uint64_t n,
                        uint8_t *slots_inout, void *stream);

/*
 * hash_batch_mixed_noalloc -- hash_batch_mixed for callers that cannot
 * allocate device memory.  The paper has no counterpart: it exists because
 * hash_batch_mixed may call cudaMalloc (its scratch area and the per-device
 * context grow on demand), which some callers must avoid -- a process whose
 * device memory belongs to another owner under a fixed budget, or a
 * latency-critical loop that must not meet the device-wide synchronisation
 * an allocation can cause.  This variant allocates nothing: its bucketing
 * scratch is a fixed array of about 5.01 MB compiled into the library, held
 * by every GPU that loads the library until the process exits.
 *   - n must be at most HB_NOALLOC_MAX_MESSAGES; larger batches return
 *     HB_ERR_TOO_LARGE without touching the GPU.  n == 0 is a no-op.
 *   - The first call on a device looks up the array's device address and
 *     the kernel's launch limits (no allocation); make that first call on
 *     each device before any stream capture.
 *   - All calls on a device share the array.  Each call clears what must
 *     start at zero, but calls whose work overlaps on the GPU race on it:
 *     order them (one stream, or events).
 *   - Device-detected errors go to a status word inside the array;
 *     hash_device_status() ORs it into the bits it returns and clears it
 *     (that read is a plain copy and allocates nothing once the library's
 *     context exists).  The kernels honour hash_set_wait_limit_ns().
 * Arguments, layout and results are those of hash_batch_mixed; the digests
 * are identical.  Returns HB_OK, HB_ERR_TOO_LARGE, HB_ERR_NULL, HB_ERR_ALIGN
 * or HB_ERR_CUDA.
 */
#define HB_NOALLOC_MAX_MESSAGES (1u << 20)
int hash_batch_mixed_noalloc(const uint8_t *algs, const uint8_t *packed_bytes,
                             const uint64_t *offsets, const uint32_t *lengths, uint64_t n,
                             uint8_t *digests_out, void *stream);

/*
 * Plans: the ragged path (as hash_batch_mixed) with scratch owned by the
 * plan, so that batches on different streams run concurrently, and its
 * launch sequence (bucketing + persistent kernel) captured once as a CUDA
 * graph and replayed for batches of any size up to max_n.
 *
 * hash_plan_create  -- allocates the plan's scratch for up to max_n < 2^31
 *                      messages (cudaMalloc) and takes the current device's
 *                      tuning (shape, warps per SM, bucketing).
 * hash_plan_run     -- one ragged batch of n <= max_n messages on `stream`
 *                      with the plan's scratch; grid_blocks 0 = tuned size.
 * hash_plan_capture -- records the ragged launch sequence for these buffer
 *                      pointers as a graph (replaces an earlier capture).
 *                      The buffers must stay valid while the graph is used.
 * hash_plan_replay  -- sets the message count n <= max_n (a one-thread
 *                      kernel on `stream`) and launches the graph on
 *                      `stream`; the messages are the first n entries of the
 *                      captured algs/offsets/lengths arrays.
 * hash_plan_configure -- overrides the plan's launch shape (-1 keeps it) and
 *                      resident warps per SM (-1 keeps it, 0 = as many as
 *                      fit) before the first capture; HB_ERR_ARG after.
 * hash_plan_set_completion -- per-request completion for serving: message i
 *                      of a batch belongs to request msg_req_dev[i] (device
 *                      uint32); remaining_dev[r] (device uint32) must hold
 *                      request r's message count when the batch starts; the
 *                      lane that finishes request r's last message stores 1
 *                      to done_flags[r] (host memory the device can write:
 *                      pinned memory on a unified-addressing system) after
 *                      the request's digests are stored.  All three or none
 *                      (NULL = off); before the first capture.  done_flags
 *                      must be page-locked host memory mapped for the device
 *                      (cudaHostAlloc); other memory returns HB_ERR_ARG.
 * hash_plan_set_segments -- the plan's batches are segments as in
 *                      hash_batch_segments: seg_dev[i] (device uint64) describes
 *                      message i of a batch, slot_index_dev (optional) maps
 *                      it to its slot, and the slots carry chaining values
 *                      between segments.  seg_dev NULL = whole messages.
 *                      Before the first capture; HB_ERR_ARG after.
 * hash_plan_destroy -- synchronises the device and frees the plan.
 * A plan's scratch is used by one batch at a time: order the runs and
 * replays of one plan (same stream, or events); different plans overlap.
 */
typedef struct hb_plan hb_plan;

/*
 * hash_gather -- packs byte ranges on the device: record i copies
 * copies[i].bytes bytes from device address copies[i].src to copies[i].dst
 * (one thread block per record; 16-byte vector copies when both addresses
 * are 16-byte aligned).  copies_dev is a device array of `count` records.
 * The serving loop uses it to move admitted requests into its arena with
 * one launch per batch.  Ranges must not overlap.
 */
typedef struct hb_copy {
  uint64_t src;
  uint64_t dst;
  uint64_t bytes;
} hb_copy;
int hash_gather(const hb_copy *copies_dev, uint32_t count, void *stream);
int hash_plan_create(uint64_t max_n, hb_plan **plan_out);
int hash_plan_run(hb_plan *plan, const uint8_t *algs, const uint8_t *packed_bytes,
                  const uint64_t *offsets, const uint32_t *lengths, uint64_t n,
                  uint8_t *digests_out, int grid_blocks, void *stream);
int hash_plan_capture(hb_plan *plan, const uint8_t *algs, const uint8_t *packed_bytes,
                      const uint64_t *offsets, const uint32_t *lengths, uint8_t *digests_out,
                      int grid_blocks);
int hash_plan_replay(hb_plan *plan, uint64_t n, void *stream);
int hash_plan_configure(hb_plan *plan, int shape_index, int warps_per_sm);
int hash_plan_set_completion(hb_plan *plan, const uint32_t *msg_req_dev, uint32_t *remaining_dev,
                             uint32_t *done_flags);
int hash_plan_set_segments(hb_plan *plan, const uint64_t *seg_dev,
                           const uint32_t *slot_index_dev);
int hash_plan_destroy(hb_plan *plan);

/*
 * Streaming rounds -- the device side of a serving loop whose messages arrive
 * over time and may be long.  The caller keeps a ring of message entries in
 * device memory (hb_ring, all arrays caller-owned); a round, launched on a
 * stream, does on the device:
 *   1. claim: every entry of the window [head, tail) (counters taken modulo
 *      capacity) in state HB_RING_READY, oldest first, becomes HB_RING_BUSY
 *      while its next segment fits the round's limits (max_msgs segments,
 *      staging_bytes of staging; a staged segment takes its own 16-byte
 *      aligned span and sits in it at its source's offset within a 16-byte
 *      granule, so sources may have any alignment and still copy as 16-byte
 *      vectors).  A segment is the next min(len - prior, segment_bytes[alg])
 *      bytes;
 *   2. copy: the segments' bytes go from src + prior to the staging area
 *      (with staging NULL, none: step 3 reads them where they are, and
 *      staging_bytes only caps the bytes one round claims);
 *   3. hash: the ragged path over the segments (hash_batch_segments with
 *      slot_index = the entry), so each entry's 32-byte slot carries its
 *      chaining value between rounds and finally its digest;
 *   4. advance: prior grows by the segment; a finished message's entry
 *      becomes HB_RING_FREE and request req[k]'s counter req_remaining drops
 *      by one -- the lane that drops it to zero stores 1 to req_done[req]
 *      (page-locked host memory mapped for the device, after the digests);
 *      an unfinished entry becomes HB_RING_READY again.
 * So only the segments of a round occupy staging memory: a long message
 * holds segment_bytes of it at a time however long its serial chain runs.
 * Rounds on different streams may run at the same time over one ring: the
 * claim is atomic, so a message is in at most one round at a time.
 * The caller fills an entry (src, len, req, alg, prior = 0, its request's
 * counter) before it sets the entry READY, orders those writes before the
 * round that covers the entry (same stream or an event), and reuses an entry
 * only when it is FREE and its digest has been read.
 *
 * hash_round_create -- allocates the round's batch arrays and scratch
 *   (cudaMalloc) and captures its launch sequence as a CUDA graph.
 *   segment_bytes[3]: per algorithm code, multiples of 64 (a cheaper
 *   algorithm can take longer segments for the same chain time);
 *   max_msgs < 2^23; staging must be 16-byte aligned, or NULL for the
 *   in-place mode.  Sets up every kernel first: call it outside any capture.
 * hash_round_launch -- runs one round for the window [head, tail)
 *   (tail - head <= capacity) on `stream`.  Do not launch a round again until
 *   its previous launch has finished.
 * hash_round_report -- segments and staged bytes the last finished launch
 *   claimed (call after that launch completed).
 * hash_round_destroy -- synchronises the device and frees the round.
 * The paper has no counterpart; it is the serving loop's device side.
 */
#define HB_RING_FREE 0u
#define HB_RING_READY 1u
#define HB_RING_BUSY 2u
typedef struct hb_ring {
  uint64_t capacity;        /* entries, a power of two                       */
  const uint64_t *src;      /* device address of each message's first byte  */
  uint64_t *prior;          /* bytes of each message hashed so far           */
  const uint32_t *len;      /* message length                                */
  const uint32_t *req;      /* request of each message (< req_capacity)      */
  const uint8_t *alg;       /* algorithm code 0, 1 or 2                      */
  uint32_t *state;          /* HB_RING_FREE / READY / BUSY                   */
  uint8_t *slots;           /* capacity * 32 bytes: chaining value, digest   */
  uint32_t *req_remaining;  /* device: messages of the request not finished  */
  uint32_t *req_done;       /* mapped host memory: 1 once the request is done */
  uint64_t req_capacity;
} hb_ring;
typedef struct hb_round hb_round;
int hash_round_create(const hb_ring *ring, uint32_t max_msgs, uint8_t *staging,
                      uint64_t staging_bytes, const uint32_t *segment_bytes,
                      int shape_index, int warps_per_sm, hb_round **round_out);
int hash_round_launch(hb_round *round, uint64_t head, uint64_t tail, void *stream);
int hash_round_report(hb_round *round, uint64_t *segments, uint64_t *bytes);
int hash_round_destroy(hb_round *round);

/*
 * hash_digits -- the paper's workload generated on the device (Sec. V-A.2):
 * message i is the 9-character decimal string of i with leading zeros
 * ("000000000" .. "999999999"); digests_out[k] (32-byte slot) receives the
 * digest of message first + k, for k < count.  No input bytes are read: the
 * strings are built in registers.  first + count <= HB_DIGITS_COUNT (10^9);
 * digests_out is a device array of count slots, 16-byte aligned.
 * Returns HB_OK, HB_ERR_INVALID_ALG, HB_ERR_TOO_LARGE, HB_ERR_NULL,
 * HB_ERR_ALIGN or HB_ERR_CUDA.
 */
#define HB_DIGITS_COUNT 1000000000ull
int hash_digits(int alg, uint64_t first, uint64_t count, uint8_t *digests_out, void *stream);

/*
 * hash_batch_check_bounds -- checks on the device that every message lies in
 * [0, packed_len): offsets[i] + lengths[i] <= packed_len, computed without
 * overflow.  Writes 0 to *status_dev when all messages are in bounds, else
 * HB_DEV_BOUNDS (status_dev is a device int owned by the caller); also ORs
 * the result into the per-device status word.  Never traps.
 */
int hash_batch_check_bounds(const uint64_t *offsets, const uint32_t *lengths, uint64_t n,
                            uint64_t packed_len, int *status_dev, void *stream);

/*
 * hash_batch_host -- the same computation from HOST buffers: copies the packed
 * bytes, offsets and lengths to device memory owned by the library, hashes
 * them, copies the digest slots back to digests_host, and waits for the
 * stream.  The packed bytes go over in chunks; the messages whose last byte
 * is in a chunk are hashed, and their slots copied back, while later chunks
 * are still coming in (two library streams besides `stream`).  This assumes
 * message ends (offset + length) do not decrease with the index, as in any
 * back-to-back layout; a device check confirms it, and otherwise every
 * message is hashed again once all bytes are in (same result, slower).
 *
 * Device memory: by default the call keeps the whole batch on the device.
 * After hash_set_host_memory_limit(bytes) (0 = no limit, the default),
 * batches whose device footprint would exceed the limit stream through two
 * device windows of at most bytes/2 each: consecutive messages whose bytes
 * and metadata fit a window are copied in, checked, hashed and copied out
 * while the other window is in flight, so batches larger than the device
 * (or than a budget) hash at copy speed.  This needs message ends in
 * non-decreasing index order and no message starting before the end of an
 * earlier window's last message (back-to-back, gaps allowed); otherwise the
 * call returns HB_ERR_ARG (HB_ERR_BOUNDS for a message outside packed_len,
 * HB_ERR_TOO_LARGE for a message that does not fit a window).  Host buffers should be pinned (cudaHostAlloc / cudaHostRegister)
 * for full copy speed; pageable memory works but is slower.  algs_host may be
 * NULL (single `alg`, or HB_ALL for hash_batch_all's 96-byte records) or a
 * host array of per-message codes (mixed path).
 * After the copies, every message is checked against packed_len on the
 * device before any message byte is read; when one is out of bounds the
 * hashing kernels skip all work and the call returns HB_ERR_BOUNDS.  The
 * device buffers are reused across calls; the call synchronises the device
 * before reusing them.  Returns as hash_batch / hash_batch_mixed, plus
 * HB_ERR_BOUNDS.
 */
uint64_t hash_set_host_memory_limit(uint64_t bytes);
int hash_batch_host(int alg, const uint8_t *algs_host, const uint8_t *packed_host,
                    uint64_t packed_len, const uint64_t *offsets_host,
                    const uint32_t *lengths_host, uint64_t n, uint8_t *digests_host,
                    void *stream);

/*
 * hash_batch_host_packed -- hash_batch_host with the digests packed back to
 * back on the host: message i's digest (RFC 1321 Sec. 3.5, FIPS 180-4
 * Sec. 6.1.2, GB/T 32905 Sec. 5.4: 16, 20 or 32 bytes in the standard's byte
 * order) at digests_host + i * hash_digest_size(alg), no zero fill; for
 * HB_ALL, i * HB_ALL_DIGEST_BYTES holds the MD5, SHA-1 and SM3 digests in
 * that order.  The slots are packed on the device before the copy back, so
 * the copy carries digest bytes only (the host path is bound by the PCIe
 * link, and for one-block messages the 96-byte records are most of what it
 * moves).  One algorithm or HB_ALL (there is no per-message algorithm array:
 * the sizes would vary).  digests_host holds n times that many bytes.
 * Otherwise, including device memory, windows and errors, as hash_batch_host.
 */
#define HB_ALL_DIGEST_BYTES 68
int hash_batch_host_packed(int alg, const uint8_t *packed_host, uint64_t packed_len,
                           const uint64_t *offsets_host, const uint32_t *lengths_host,
                           uint64_t n, uint8_t *digests_host, void *stream);

/*
 * hash_device_status -- synchronises `stream`, then returns the OR of the
 * HB_DEV_* bits recorded on the current device since the last call, and
 * clears them.  *status_out receives the bits.  The bits include those of
 * hash_batch_mixed_noalloc, whose status word lives in its fixed scratch.
 */
int hash_device_status(void *stream, int *status_out);

/* hash_release_device -- frees the current device's library context. */
int hash_release_device(void);

/*
 * Tuning.  The hashing kernels are instantiated for a few launch shapes
 * (warps per block x copy stages in flight per warp x 64-byte blocks staged
 * per lane and stage x copy mapping: each lane copying its own message, or
 * the warp copying message after message with consecutive lanes on
 * consecutive 16-byte pieces, which keeps one copy instruction within two or
 * three messages).  hash_tune_set
 * selects the shape that hash_batch uses for `alg`, or that the ragged path
 * uses when alg == HB_TUNE_MIXED; hash_tune_get reads the selection;
 * hash_tune_shape describes shape `index` and hash_tune_occupancy returns
 * its resident blocks per SM.  An index outside [0, hash_tune_shapes()) is
 * rejected with HB_ERR_ARG.  The Python autotuner drives these and keeps its
 * results in a JSON cache keyed by device, SM count, algorithm and length.
 */
#define HB_TUNE_MIXED 3
int hash_tune_shapes(void);
int hash_tune_shape(int index, int *warps_per_block, int *stages, int *blocks_per_stage,
                    int *cooperative);
int hash_tune_set(int alg, int shape_index);
int hash_tune_get(int alg);
int hash_tune_occupancy(int alg, int shape_index);

/*
 * hash_tune_buckets -- bucketing of the ragged path on the current device:
 * each octave of estimated per-message cost (padded blocks x relative cost of
 * the algorithm's block) is split into 2^sub_log2 buckets (0 <= sub_log2 <=
 * 6; finer buckets give chunks of more equal length), and with alg_major = 1
 * the chunk order runs through all SM3 messages, then SHA-1, then MD5, each
 * longest first, instead of interleaving the algorithms.  alg_major = 2 is
 * that order with MD5's two longest octaves of messages taken out into a second
 * queue that every other warp serves first, so those chains run beside the
 * SM3 phase instead of starting after it and the SHA-1 phase (0 <= alg_major
 * <= 2).  Digests do not depend on any of these choices.  Defaults:
 * sub_log2 = 6, alg_major = 2.
 */
int hash_tune_buckets(int sub_log2, int alg_major);

/*
 * hash_tune_relay -- segment length, in 64-byte blocks, of hash_batch_all's
 * relay form on the current device (0 = never relay; default 64).  Every
 * message longer than one segment is hashed one segment per item; items are
 * taken in order, segment by segment, by the warps of a persistent grid, and
 * each waits (bounded by hash_set_wait_limit_ns, else HB_DEV_TIMEOUT) for
 * its message's previous segment.  Digests do not depend on the choice.
 * Returns HB_ERR_ARG outside [0, 2^20].
 */
int hash_tune_relay(int segment_blocks);

/*
 * hash_all_uses_relay -- 1 when hash_batch_all of n messages on the current
 * device (default grid, outside stream capture) takes the relay form, else
 * 0; or an HB_ERR_* code.
 */
int hash_all_uses_relay(uint64_t n);

/*
 * hash_tune_mixed_warps -- resident warps per SM of the persistent ragged
 * kernel on the current device (0 = as many as fit).  A long message is a
 * serial chain of blocks, so the warp that holds it should not share its SM
 * sub-partition with many other busy warps; default 8 (two per
 * sub-partition).  Returns HB_ERR_ARG outside [0, 64].
 */
int hash_tune_mixed_warps(int warps_per_sm);

/*
 * hash_batch_shape / hash_batch_mixed_shape -- hash_batch / hash_batch_mixed
 * with an explicit launch shape (-1 = the tuned one) and grid size (0 = the
 * library's choice: enough blocks for the work, at most one full wave of
 * resident blocks); used by the autotuner and the benchmarks.
 */
int hash_batch_all_shape(const uint8_t *packed_bytes, const uint64_t *offsets,
                         const uint32_t *lengths, uint64_t n, uint8_t *records_out,
                         int shape_index, int grid_blocks, void *stream);
int hash_batch_shape(int alg, const uint8_t *packed_bytes, const uint64_t *offsets,
                     const uint32_t *lengths, uint64_t n, uint8_t *digests_out,
                     int shape_index, int grid_blocks, void *stream);
int hash_batch_mixed_shape(const uint8_t *algs, const uint8_t *packed_bytes,
                           const uint64_t *offsets, const uint32_t *lengths, uint64_t n,
                           uint8_t *digests_out, int shape_index, int grid_blocks,
                           void *stream);

/*
 * Integer-issue microbenchmark (measurement only; not part of the hashing
 * path): runs `iters` iterations of eight independent chains per thread of
 * one operation class on every thread of the launch -- 0 LOP3, 1 IADD3,
 * 2 SHF funnel rotate, 3 PRMT, 4 LOP3/IADD3/SHF in rotation, 5 IMAD x*y+z,
 * 6 LOP3/IMAD, 7 IADD3/IMAD, 8 SHF/IMAD, 9 LOP3/FFMA, 10 IMAD x*1+y (an add
 * on the multiply-add pipe), 11 LOP3/(x*1+y), 12 LOP3/SHF/IADD3/(x*1+y),
 * 13 IMAD.HI, 14 LOP3/IMAD.HI, 15 LOP3 + a rotation done as IMAD.HI of an
 * IMAD (three operations per pair of steps), 16 a rotation done on the
 * multiply-add pipe as the two halves of a widening multiply by 2^s added
 * together (two instructions per step), 17 LOP3 / that rotation,
 * 18 SHF / that rotation --
 * and writes the SM cycles each block took to cycles_out_dev[blocks]
 * (device) and a sink word to sink_dev.  The number of 32-bit operations
 * executed is blocks * threads * iters * hash_int_peak_ops_per_iter().
 */
int hash_int_peak(int op_class, int blocks, int threads, int iters, uint64_t *cycles_out_dev,
                  uint32_t *sink_dev, void *stream);
int hash_int_peak_ops_per_iter(void);

/*
 * Failure-detection self test: launches one warp that waits, with the same
 * bounded wait the hashing kernels use, on a barrier phase that nothing
 * completes.  After timeout_ns the wait gives up, records HB_DEV_TIMEOUT in
 * the per-device status word and the kernel returns normally.
 */
int hash_selftest_wait_timeout(uint64_t timeout_ns, void *stream);

/* Device-side wait limit used by the hashing kernels, in nanoseconds
 * (default 2 s).  Returns the previous value. */
uint64_t hash_set_wait_limit_ns(uint64_t limit_ns);

#ifdef __cplusplus
}
#endif

#endif /* HASHBATCH_H */
