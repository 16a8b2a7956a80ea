// hb_kernels.cu -- the library's kernels other than the hashing kernels,
// and the host-side launchers of all of them.
//
//   hb_plain_kernel    (hb_hash_kernels.cuh) one algorithm (or all three,
//                      HB_ALL), one message per thread, static grid-stride
//                      over 32-message tasks (hash_batch, hash_batch_all)
//   hb_hist_kernel     ragged path, step 1: histogram of (cost bucket, alg)
//   hb_scan_kernel     ragged path, step 2: group starts, padding, counters
//   hb_scatter_kernel  ragged path, step 3: message ids into their group
//   hb_mixed_kernel    (hb_hash_kernels.cuh) ragged path, step 4:
//                      persistent, chunks popped from a counter
//                      longest-first (hash_batch_mixed)
//   hb_digits_kernel   the paper's nine-digit workload generated in registers
//   hb_bounds_kernel   offsets/lengths against the packed buffer size
//   hb_monotone_kernel, hb_rebase_kernel, hb_pack_kernel   host-path helpers
//                      (chunk check, window-relative offsets, digests packed
//                      back to back for the copy to the host)
//   hb_set_count_kernel, hb_gather_kernel  batch size for captured graphs,
//                      byte-range packing
//   hb_int_peak_kernel integer-issue microbenchmark (measurement only)
//   hb_selftest_wait_kernel  bounded-wait failure test
// (The streaming-round kernels live in hb_stream.cu.)
#include <cuda_runtime.h>

#include <cstdint>

#include "hb_launch.h"
#include "hb_hash_kernels.cuh"
#include "hb_pipeline.cuh"

namespace hb {

// ---------------------------------------------------------------------------
// Ragged path: bucketing by estimated cost, then the persistent kernel.

// Relative cost of one block: MD5 : SHA-1 : SM3 ~ 4 : 7 : 17 (their counted
// 32-bit operations per block, about 330 : 610 : 1410).
__device__ __forceinline__ uint32_t cost_group(uint32_t len, uint32_t alg, BucketCfg cfg) {
  const uint32_t w = alg == HB_MD5 ? 4u : alg == HB_SHA1 ? 7u : 17u;
  const uint32_t c = padded_blocks(len) * w;  // < 2^27 * 17 < 2^32
  const int e = 31 - __clz(c);                // floor(log2 c), c >= 4
  const int sub = (int)cfg.sub_log2;
  const uint32_t mask = (1u << sub) - 1u;
  // the `sub` bits below the leading one
  const uint32_t frac = e >= sub ? (c >> (e - sub)) & mask : (c << (sub - e)) & mask;
  const uint32_t bucket = ((uint32_t)e << sub) + frac;  // < kCostBuckets
  const uint32_t desc = kCostBuckets - 1u - bucket;     // most expensive first
  if (cfg.alg_major) {
    const uint32_t rank = alg == HB_SM3 ? 0u : alg == HB_SHA1 ? 1u : 2u;
    return rank * kCostBuckets + desc;
  }
  return desc * 3u + alg;
}

__device__ __forceinline__ uint64_t batch_size(const MixedArgs& m) {
  return m.n_dev ? *m.n_dev : m.n;
}

__global__ void hb_hist_kernel(MixedArgs m) {
  __shared__ uint32_t counts[kGroups];
  for (uint32_t g = threadIdx.x; g < kGroups; g += blockDim.x) counts[g] = 0;
  __syncthreads();
  const uint64_t n = batch_size(m);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t alg = m.algs[i];
    if (alg <= HB_SM3) {
      atomicAdd(&counts[cost_group(m.lengths[i], alg, m.cfg)], 1u);
    } else {
      // Unknown code: the slot stays all zero and the message is not hashed.
      uint8_t* dst = m.digests + (m.slot_index ? (uint64_t)m.slot_index[i] : i) * HB_SLOT_BYTES;
      stg128_cs(dst, 0, 0, 0, 0);
      stg128_cs(dst + 16, 0, 0, 0, 0);
    }
  }
  __syncthreads();
  for (uint32_t g = threadIdx.x; g < kGroups; g += blockDim.x)
    if (counts[g]) atomicAdd(&m.ws->counts[g], counts[g]);
}

// One block of kScanThreads threads, kScanPer consecutive groups each.
// Every chunk of 32 permutation entries must hold a single algorithm and start
// with a real message.  In algorithm-major order (alg_major 1, 2) each
// algorithm's groups are adjacent, so they are laid out back to back and
// only each algorithm's end is padded to a multiple of 32: a chunk may hold
// the cheapest messages of one cost bucket and the costliest of the next,
// instead of a group's last chunk running part-empty.  With the algorithms
// interleaved (alg_major 0) every group is padded.  An exclusive prefix sum
// of the (padded) counts, per thread and then across the block's warps,
// gives each group's first permutation entry.
constexpr uint32_t kScanThreads = 512;
constexpr uint32_t kScanPer = kGroups / kScanThreads;
static_assert(kGroups % kScanThreads == 0, "scan covers every group");

__global__ void __launch_bounds__(kScanThreads) hb_scan_kernel(MixedArgs m) {
  __shared__ uint32_t warp_sums[kScanThreads / 32];
  __shared__ uint32_t gstart[kGroups + 1];
  __shared__ uint32_t md5_top;  // first non-empty MD5 group (alg_major 2)
  const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
  const bool per_alg = m.cfg.alg_major != 0;
  uint32_t cnt[kScanPer], pad[kScanPer], own = 0;
#pragma unroll
  for (uint32_t k = 0; k < kScanPer; ++k) {
    cnt[k] = m.ws->counts[t * kScanPer + k];
    pad[k] = per_alg ? cnt[k] : (cnt[k] + 31u) & ~31u;
    own += pad[k];
  }
  uint32_t incl = own;  // inclusive scan within the warp
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t v = __shfl_up_sync(kFull, incl, d);
    if (lane >= (uint32_t)d) incl += v;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  uint32_t before = 0, total = 0;
  for (uint32_t w = 0; w < kScanThreads / 32; ++w) {
    const uint32_t v = warp_sums[w];
    before += w < warp ? v : 0u;
    total += v;
  }
  uint32_t start = before + incl - own;
#pragma unroll
  for (uint32_t k = 0; k < kScanPer; ++k) {
    gstart[t * kScanPer + k] = start;
    start += pad[k];
  }
  if (t == 0) md5_top = kGroups;
  __syncthreads();
  // Algorithm-major: algorithm rank r (groups [r, r + 1) * kCostBuckets)
  // moves up by the padding of the ranks before it.
  uint32_t all[3] = {0u, 0u, 0u}, shift[3] = {0u, 0u, 0u}, padded_total = total;
  if (per_alg) {
    const uint32_t e1 = gstart[kCostBuckets], e2 = gstart[2 * kCostBuckets];
    all[0] = e1;
    all[1] = e2 - e1;
    all[2] = total - e2;
    shift[1] = ((all[0] + 31u) & ~31u) - all[0];
    shift[2] = shift[1] + ((all[1] + 31u) & ~31u) - all[1];
    padded_total = total + shift[2] + ((all[2] + 31u) & ~31u) - all[2];
  }
  __syncthreads();  // every raw start has been read
#pragma unroll
  for (uint32_t k = 0; k < kScanPer; ++k) {
    const uint32_t g = t * kScanPer + k;
    const uint32_t sg = gstart[g] + (per_alg ? shift[g / kCostBuckets] : 0u);
    m.ws->cursor[g] = sg;
    gstart[g] = sg;
    if (!per_alg)
      for (uint32_t e = sg + cnt[k]; e < sg + pad[k]; ++e) m.perm[e] = 0xFFFFFFFFu;
    if (cnt[k] && g >= 2 * kCostBuckets) atomicMin(&md5_top, g);  // MD5 groups, rank 2
  }
  if (per_alg && t < 3) {
    // the padding after algorithm rank t
    const uint32_t first = t == 0 ? 0u : (t == 1 ? all[0] + shift[1] : all[0] + all[1] + shift[2]);
    for (uint32_t e = first + all[t]; e < first + ((all[t] + 31u) & ~31u); ++e)
      m.perm[e] = 0xFFFFFFFFu;
  }
  if (t == 0) gstart[kGroups] = padded_total;
  __syncthreads();
  if (t == 0) {
    m.ws->nchunks = padded_total / 32u;
    m.ws->chunk_counter = 0u;
    uint32_t first = 0, count = 0;
    if (m.cfg.alg_major == 2 && md5_top < kGroups) {
      // the chunks holding two octaves of MD5 cost buckets from its longest
      // non-empty one (MD5's first chunk starts there: the groups before it
      // are empty)
      const uint32_t span = 2u << m.cfg.sub_log2;
      const uint32_t end = md5_top + span < kGroups ? md5_top + span : kGroups;
      first = gstart[md5_top] / 32u;
      count = (gstart[end] + 31u) / 32u - first;
    }
    m.ws->early[0] = first;
    m.ws->early[1] = count;
    m.ws->early[2] = 0u;
  }
}

// Each block places a contiguous range of the messages: it counts its
// messages per group in shared memory, reserves each group's places with one
// global atomic (the group's cursor), and hands them out with shared-memory
// atomics.  Any order within a group is as good as another; what matters is
// that the global atomics are few (one per non-empty group per block, where
// a warp-aggregated reservation still met about 31 distinct groups per warp).
constexpr int kScatterThreads = 1024;

__global__ void __launch_bounds__(kScatterThreads) hb_scatter_kernel(MixedArgs m) {
  __shared__ uint32_t next[kGroups];
  const uint64_t n = batch_size(m);
  const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint64_t lo = (uint64_t)blockIdx.x * per;
  const uint64_t hi = lo + per < n ? lo + per : n;
  for (uint32_t g = threadIdx.x; g < kGroups; g += blockDim.x) next[g] = 0;
  __syncthreads();
  for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const uint32_t alg = m.algs[i];
    if (alg <= HB_SM3) atomicAdd(&next[cost_group(m.lengths[i], alg, m.cfg)], 1u);
  }
  __syncthreads();
  for (uint32_t g = threadIdx.x; g < kGroups; g += blockDim.x) {
    const uint32_t c = next[g];
    if (c) next[g] = atomicAdd(&m.ws->cursor[g], c);
  }
  __syncthreads();
  for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const uint32_t alg = m.algs[i];
    if (alg <= HB_SM3) m.perm[atomicAdd(&next[cost_group(m.lengths[i], alg, m.cfg)], 1u)] = (uint32_t)i;
  }
}

// ---------------------------------------------------------------------------
// The paper's workload, generated on the device (Sec. V-A.2): message i is
// the 9-character decimal string of i with leading zeros, "000000000" ..
// "999999999", built in registers -- no input bytes are read.  Each string
// is one padded block: 9 characters, 0x80, zeros, the bit length 72.  A
// thread hashes the ten strings 10q .. 10q+9, which share their first eight
// characters, so the digits of q are worked out once per ten messages.

// Message words of the strings 10q .. 10q+9 except word 2 (the last digit,
// then the 0x80 marker), in the algorithm's word order.
template <bool BE>
__device__ __forceinline__ void digit_words(uint64_t q, uint32_t (&w)[16]) {
  uint32_t c[8];  // characters of q, most significant first
  uint32_t v = (uint32_t)q;
#pragma unroll
  for (int k = 7; k >= 0; --k) {
    c[k] = '0' + v % 10u;
    v /= 10u;
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) w[k] = 0u;
  if (BE) {
    w[0] = (c[0] << 24) | (c[1] << 16) | (c[2] << 8) | c[3];
    w[1] = (c[4] << 24) | (c[5] << 16) | (c[6] << 8) | c[7];
    w[15] = 72u;
  } else {
    w[0] = c[0] | (c[1] << 8) | (c[2] << 16) | (c[3] << 24);
    w[1] = c[4] | (c[5] << 8) | (c[6] << 16) | (c[7] << 24);
    w[14] = 72u;
  }
}

template <bool BE>
__device__ __forceinline__ uint32_t digit_word2(uint32_t d) {
  const uint32_t ch = '0' + d;
  return BE ? ((ch << 24) | (0x80u << 16)) : (ch | (0x80u << 8));
}

constexpr int kDigitsThreads = 256;

template <int ALG>
__global__ void __launch_bounds__(kDigitsThreads) hb_digits_kernel(uint64_t first, uint64_t count,
                                                                   uint8_t* digests, MulConsts mc) {
  constexpr bool BE = AlgTraits<ALG>::kBigEndian;
  const uint64_t end = first + count;
  const uint64_t q_end = (end + 9) / 10;
  if constexpr (ALG == HB_MD5) {
    // MD5 is quick enough that lane-strided 16-byte stores (each lane's ten
    // slots are 320 bytes apart from the next lane's) bound it.  A warp takes
    // 32 consecutive runs -- 320 consecutive messages -- keeps their digests
    // in shared memory, and writes the 10 KB of slots in order: each store
    // instruction covers 512 consecutive bytes.
    __shared__ uint4 staged[kDigitsThreads / 32][320];
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t wib = threadIdx.x >> 5;
    uint4* mine = staged[wib];
    const uint64_t warps = (uint64_t)gridDim.x * (kDigitsThreads / 32);
    for (uint64_t qw = first / 10 + ((uint64_t)blockIdx.x * (kDigitsThreads / 32) + wib) * 32;
         qw < q_end; qw += warps * 32) {  // warp-uniform
      const uint64_t q = qw + lane;
      if (q < q_end) {
        uint32_t w[16];
        digit_words<BE>(q, w);
#pragma unroll 1
        for (uint32_t d = 0; d < 10; ++d) {
          uint32_t x[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) x[k] = w[k];
          x[2] = digit_word2<BE>(d);
          // keep the words that vary opaque, so that their sums with MD5's
          // constants are not hoisted out of this loop into extra registers
          asm volatile("" : "+r"(x[0]), "+r"(x[1]));
          uint32_t st[8];
          alg_init<ALG>(st);
          alg_compress<ALG>(st, x, mc);
          mine[lane * 10 + d] = make_uint4(st[0], st[1], st[2], st[3]);
        }
      }
      __syncwarp();
      // 16-byte piece c of the warp's 320 slots: the digest (even c) or the
      // zero fill (odd c) of message 10 qw + c / 2
#pragma unroll 1
      for (uint32_t c = lane; c < 640; c += 32) {
        const uint64_t m = qw * 10 + c / 2;
        if (m >= first && m < end) {
          const uint4 v = (c & 1u) ? make_uint4(0u, 0u, 0u, 0u) : mine[c / 2];
          stg128_cs(digests + (m - first) * HB_SLOT_BYTES + 16 * (c & 1u), v.x, v.y, v.z, v.w);
        }
      }
      __syncwarp();
    }
  } else {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q = first / 10 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < q_end;
         q += stride) {
      uint32_t w[16];
      digit_words<BE>(q, w);
#pragma unroll 1
      for (uint32_t d = 0; d < 10; ++d) {
        const uint64_t i = q * 10 + d;
        if (i < first || i >= end) continue;
        w[2] = digit_word2<BE>(d);
        uint32_t st[8];
        alg_init<ALG>(st);
        alg_compress<ALG>(st, w, mc);
        uint32_t o[8];
        alg_digest_words<ALG>(st, o);
        uint8_t* dst = digests + (i - first) * HB_SLOT_BYTES;
        stg128_cs(dst, o[0], o[1], o[2], o[3]);
        stg128_cs(dst + 16, o[4], o[5], o[6], o[7]);
      }
    }
  }
}

cudaError_t launch_digits(int alg, uint64_t first, uint64_t count, uint8_t* digests, int grid,
                          cudaStream_t stream) {
  const MulConsts mc = make_mul_consts();
  switch (alg) {
    case HB_MD5: hb_digits_kernel<HB_MD5><<<grid, kDigitsThreads, 0, stream>>>(first, count, digests, mc); break;
    case HB_SHA1: hb_digits_kernel<HB_SHA1><<<grid, kDigitsThreads, 0, stream>>>(first, count, digests, mc); break;
    case HB_SM3: hb_digits_kernel<HB_SM3><<<grid, kDigitsThreads, 0, stream>>>(first, count, digests, mc); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Bounds check (never traps; reports through status words).

__global__ void hb_bounds_kernel(const uint64_t* offsets, const uint32_t* lengths, uint64_t n,
                                 uint64_t packed_len, int* status_dev, int* ctx_status) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t o = offsets[i];
    const uint64_t l = lengths[i];
    bad |= (o > packed_len) || (l > packed_len - o);
  }
  if (bad) {
    if (status_dev) atomicOr(status_dev, HB_DEV_BOUNDS);
    if (ctx_status) atomicOr(ctx_status, HB_DEV_BOUNDS);
  }
}

// Whether message ends (offset + length) are non-decreasing in index order;
// sets *flag = 1 when they are not.  The pipelined host path relies on it to
// hash a message once the packed bytes up to its end have arrived.
__global__ void hb_monotone_kernel(const uint64_t* offsets, const uint32_t* lengths, uint64_t n,
                                   int* flag) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i + 1 < n; i += stride)
    bad |= offsets[i] + lengths[i] > offsets[i + 1] + lengths[i + 1];
  if (bad) atomicExch(flag, 1);
}

// ---------------------------------------------------------------------------
// Integer issue microbenchmark: eight independent chains per thread, four
// unrolled steps per iteration, one 32-bit operation per chain per step.
// `one` is a kernel argument equal to 1, so x * one + y stays a multiply-add
// (IMAD) that the compiler cannot turn back into a plain add.
//   0 LOP3   1 IADD3   2 SHF   3 PRMT   4 LOP3/IADD3/SHF   5 IMAD x*y+z
//   6 LOP3/IMAD   7 IADD3/IMAD   8 SHF/IMAD   9 LOP3/FFMA   10 IMAD x*1+y
//   11 LOP3/(x*1+y)   12 LOP3/SHF/IADD3/(x*1+y)   13 IMAD.HI x*2^7+y
//   14 LOP3/IMAD.HI   15 LOP3 + rotation as IMAD.HI(x, 2^7, IMAD(x, 2^7, 0))
//   16 rotation on the multiply-add pipe: {lo, hi} = x*2^7 (IMAD.WIDE),
//      then lo*1 + hi (IMAD): two instructions per counted step
//   17 LOP3 / rotation as in 16   18 SHF / rotation as in 16

template <int OP>
__device__ __forceinline__ uint32_t peak_step(int u, uint32_t x, uint32_t y, uint32_t z, uint32_t one) {
  if constexpr (OP == 0) return lop3<0x96>(x, y, z);
  else if constexpr (OP == 1) return x + y + z;
  else if constexpr (OP == 2) return __funnelshift_l(x, y, 7);
  else if constexpr (OP == 3) return __byte_perm(x, y, 0x6351);
  else if constexpr (OP == 4) {
    const int m = u % 3;
    return m == 0 ? lop3<0x96>(x, y, z) : m == 1 ? x + y + z : __funnelshift_l(x, y, 7);
  } else if constexpr (OP == 5) return x * y + z;
  else if constexpr (OP == 6) return (u & 1) ? x * y + z : lop3<0x96>(x, y, z);
  else if constexpr (OP == 7) return (u & 1) ? x * y + z : x + y + z;
  else if constexpr (OP == 8) return (u & 1) ? x * y + z : __funnelshift_l(x, y, 7);
  else if constexpr (OP == 9) {
    if (u & 1) return __float_as_uint(fmaf(__uint_as_float(x), 1.0001f, __uint_as_float(z)));
    return lop3<0x96>(x, y, z);
  } else if constexpr (OP == 10) return x * one + y;
  else if constexpr (OP == 11) return (u & 1) ? x * one + y : lop3<0x96>(x, y, z);
  else if constexpr (OP == 13) {
    uint32_t d;
    asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(one << 7), "r"(y));
    return d;
  } else if constexpr (OP == 14) {
    if (!(u & 1)) return lop3<0x96>(x, y, z);
    uint32_t d;
    asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(one << 7), "r"(y));
    return d;
  } else if constexpr (OP == 15) {
    // one LOP3 and one two-IMAD rotation per pair of chain steps
    if (!(u & 1)) return lop3<0x96>(x, y, z);
    uint32_t lo, d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(lo) : "r"(x), "r"(one << 7), "r"(0u));
    asm("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(one << 7), "r"(lo));
    return d;
  }
  else if constexpr (OP >= 16 && OP <= 18) {
    if (OP == 17 && !(u & 1)) return lop3<0x96>(x, y, z);
    if (OP == 18 && !(u & 1)) return __funnelshift_l(x, y, 7);
    uint64_t w;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(w) : "r"(x), "r"(one << 7));
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"((uint32_t)w), "r"(one), "r"((uint32_t)(w >> 32)));
    return d;
  }
  else {
    const int m = u & 3;
    return m == 0 ? lop3<0x96>(x, y, z) : m == 1 ? __funnelshift_l(x, y, 7)
         : m == 2 ? x + y + z : x * one + y;
  }
}

template <int OP>
__global__ void hb_int_peak_kernel(int iters, uint32_t one, unsigned long long* cycles, uint32_t* sink) {
  uint32_t x[8];
  const uint32_t seed = threadIdx.x * 2654435761u + blockIdx.x;
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = seed ^ (0x9e3779b9u * (k + 1));
  const uint32_t z = seed | 1u;
  __syncthreads();
  const unsigned long long t0 = clock64();
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = peak_step<OP>(u * 8 + k, x[k], x[(k + 1) & 7], z, one);
    }
  }
  __syncthreads();
  const unsigned long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) acc ^= x[k];
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
  if (acc == 0x12345678u) sink[0] = acc;  // keeps the chains alive
}

// ---------------------------------------------------------------------------
// Failure-detection self test: a wait on a barrier phase nobody completes.

__global__ void hb_selftest_wait_kernel(uint64_t limit_ns, int* status) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t addr = smem_addr(&bar);
  if (threadIdx.x == 0) {
    mbar_init(addr, 1);
    fence_barrier_init();
  }
  __syncwarp();
  mbar_wait_bounded(addr, 0, limit_ns, status);
}

// ---------------------------------------------------------------------------
// Launch shapes and host launchers.

static const ShapeDesc kShapes[] = {HB_SHAPES(HB_SHAPE_DESC)};
static constexpr int kNumShapes = sizeof(kShapes) / sizeof(kShapes[0]);

// The kernels' instantiation tables are compiled in their own translation
// units (hb_inst_*.cu), in parallel.
extern template KernelFn plain_fn<HB_MD5>(int);
extern template KernelFn plain_fn<HB_SHA1>(int);
extern template KernelFn plain_fn<HB_SM3>(int);
extern template KernelFn plain_fn<HB_ALL>(int);
extern template KernelFn mixed_fn<false>(int);
extern template KernelFn mixed_fn<true>(int);

static int shape_smem(int shape, bool seg) {
#define HB_SMEM_CASE(i, w, st, kb, co) \
  case i: return w * (seg ? WarpSmem<st, kb, true>::kBytes : WarpSmem<st, kb, false>::kBytes);
  switch (shape) {
    HB_SHAPES(HB_SMEM_CASE)
    default: return 0;
  }
#undef HB_SMEM_CASE
}

int num_shapes() { return kNumShapes; }

bool shape_desc(int shape, int* warps, int* stages, int* kb, int* coop) {
  if (shape < 0 || shape >= kNumShapes) return false;
  *warps = kShapes[shape].warps;
  *stages = kShapes[shape].stages;
  if (kb) *kb = kShapes[shape].kb;
  if (coop) *coop = kShapes[shape].coop ? 1 : 0;
  return true;
}

int shape_smem_bytes(int shape, bool seg) { return shape_smem(shape, seg); }

static int shape_smem_relay(int shape) {
#define HB_SMEM_RELAY_CASE(i, w, st, kb, co) \
  case i: return w * WarpSmem<st, kb, false, true>::kBytes;
  switch (shape) {
    HB_SHAPES(HB_SMEM_RELAY_CASE)
    default: return 0;
  }
#undef HB_SMEM_RELAY_CASE
}

cudaError_t prepare_relay(int shape, int* blocks_per_sm) {
  KernelFn fn = relay_fn(shape);
  if (!fn) return cudaErrorInvalidValue;
  const int smem = shape_smem_relay(shape);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kShapes[shape].warps * 32,
                                                       smem);
}

cudaError_t launch_relay(int shape, int grid, const KernelArgs& a, cudaStream_t stream) {
  KernelFn fn = relay_fn(shape);
  if (!fn || grid <= 0 || !a.relay) return cudaErrorInvalidValue;
  fn<<<grid, kShapes[shape].warps * 32, shape_smem_relay(shape), stream>>>(a);
  return cudaGetLastError();
}

// Before a relay: relay[2] = the longest length (relay[0..3] zeroed before),
// and word 4 of every record whose message spans more than one segment
// (the blocks-done count its later segments wait on) set to zero.
__global__ void hb_relay_setup_kernel(const uint32_t* lengths, uint64_t n, uint32_t seg_bytes,
                                      uint8_t* records, uint32_t* relay) {
  uint32_t m = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t len = lengths[i];
    m = max(m, len);
    if (len > seg_bytes) *reinterpret_cast<uint32_t*>(records + i * HB_ALL_RECORD_BYTES + 16) = 0u;
  }
  m = __reduce_max_sync(0xFFFFFFFFu, m);
  if ((threadIdx.x & 31u) == 0 && m) atomicMax(relay + 2, m);
}

cudaError_t launch_relay_setup(const uint32_t* lengths, uint64_t n, uint32_t seg_bytes,
                               uint8_t* records, uint32_t* relay, int grid, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(relay, 0, 4 * sizeof(uint32_t), stream);
  if (e != cudaSuccess) return e;
  hb_relay_setup_kernel<<<grid, 256, 0, stream>>>(lengths, n, seg_bytes, records, relay);
  return cudaGetLastError();
}

static KernelFn pick(bool mixed, int alg, int shape, bool seg) {
  if (mixed) return seg ? mixed_fn<true>(shape) : mixed_fn<false>(shape);
  switch (alg) {
    case HB_MD5: return plain_fn<HB_MD5>(shape);
    case HB_SHA1: return plain_fn<HB_SHA1>(shape);
    case HB_SM3: return plain_fn<HB_SM3>(shape);
    case HB_ALL: return plain_fn<HB_ALL>(shape);
    default: return nullptr;
  }
}

cudaError_t prepare_kernel(bool mixed, int alg, int shape, int* blocks_per_sm, bool seg) {
  KernelFn fn = pick(mixed, alg, shape, seg && mixed);
  if (!fn) return cudaErrorInvalidValue;
  const int smem = shape_smem(shape, seg && mixed);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kShapes[shape].warps * 32,
                                                       smem);
}

cudaError_t launch_hash(bool mixed, int alg, int shape, int grid, const KernelArgs& a,
                        cudaStream_t stream) {
  const bool seg = mixed && a.seg != nullptr;
  KernelFn fn = pick(mixed, alg, shape, seg);
  if (!fn || grid <= 0) return cudaErrorInvalidValue;
  fn<<<grid, kShapes[shape].warps * 32, shape_smem(shape, seg), stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bucketing(const MixedArgs& m, int grid, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(m.ws->counts, 0, sizeof(m.ws->counts), stream);
  if (e != cudaSuccess) return e;
  hb_hist_kernel<<<grid, 256, 0, stream>>>(m);
  hb_scan_kernel<<<1, kScanThreads, 0, stream>>>(m);
  // `grid` is at most 8 blocks of 256 threads per SM: the scatter takes an
  // eighth of it in 1024-thread blocks (at most one per SM), since the fewer
  // blocks, the fewer global reservations
  hb_scatter_kernel<<<(grid + 7) / 8, kScatterThreads, 0, stream>>>(m);
  return cudaGetLastError();
}

cudaError_t launch_bounds(const uint64_t* offsets, const uint32_t* lengths, uint64_t n,
                          uint64_t packed_len, int* status_dev, int* ctx_status, int grid,
                          cudaStream_t stream) {
  hb_bounds_kernel<<<grid, 256, 0, stream>>>(offsets, lengths, n, packed_len, status_dev,
                                             ctx_status);
  return cudaGetLastError();
}

// offsets[i] -= base (a window's messages, relative to the window's bytes;
// an offset below base wraps to a huge value that the bounds check rejects).
__global__ void hb_rebase_kernel(uint64_t* offsets, uint64_t n, uint64_t base) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    offsets[i] -= base;
}

cudaError_t launch_rebase(uint64_t* offsets, uint64_t n, uint64_t base, int grid,
                          cudaStream_t stream) {
  hb_rebase_kernel<<<grid, 256, 0, stream>>>(offsets, n, base);
  return cudaGetLastError();
}

// Digest bytes of 32-byte slots (or 96-byte records of the three algorithms)
// packed back to back: out word w is word k = w mod q of message i = w / q,
// q = dsz / 4; in a record, words 0-3 are MD5's, 8-12 SHA-1's, 16-23 SM3's.
// One thread per output word, so the stores are coalesced.
__global__ void hb_pack_kernel(const uint32_t* __restrict__ slots, uint32_t rec_words,
                               uint64_t n, uint32_t* __restrict__ out, uint32_t q, int all) {
  const uint64_t total = n * q;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += stride) {
    const uint64_t i = w / q;
    const uint32_t k = (uint32_t)(w - i * q);
    const uint32_t src = !all ? k : k < 4 ? k : k < 9 ? 8 + (k - 4) : 16 + (k - 9);
    out[w] = slots[i * rec_words + src];
  }
}

cudaError_t launch_pack(const uint8_t* slots, uint32_t rec, uint64_t n, uint8_t* out, uint32_t dsz,
                        int grid, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  hb_pack_kernel<<<grid, 256, 0, stream>>>(reinterpret_cast<const uint32_t*>(slots), rec / 4, n,
                                           reinterpret_cast<uint32_t*>(out), dsz / 4,
                                           rec == HB_ALL_RECORD_BYTES ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_monotone(const uint64_t* offsets, const uint32_t* lengths, uint64_t n, int* flag,
                            int grid, cudaStream_t stream) {
  hb_monotone_kernel<<<grid, 256, 0, stream>>>(offsets, lengths, n, flag);
  return cudaGetLastError();
}

template <int OP>
static void int_peak_launch(int blocks, int threads, int iters, unsigned long long* cycles,
                            uint32_t* sink, cudaStream_t stream) {
  hb_int_peak_kernel<OP><<<blocks, threads, 0, stream>>>(iters, 1u, cycles, sink);
}

cudaError_t launch_int_peak(int op, int blocks, int threads, int iters, unsigned long long* cycles,
                            uint32_t* sink, cudaStream_t stream) {
  using Fn = void (*)(int, int, int, unsigned long long*, uint32_t*, cudaStream_t);
  static const Fn table[] = {int_peak_launch<0>, int_peak_launch<1>, int_peak_launch<2>,
                             int_peak_launch<3>, int_peak_launch<4>, int_peak_launch<5>,
                             int_peak_launch<6>, int_peak_launch<7>, int_peak_launch<8>,
                             int_peak_launch<9>, int_peak_launch<10>, int_peak_launch<11>,
                             int_peak_launch<12>, int_peak_launch<13>, int_peak_launch<14>,
                             int_peak_launch<15>, int_peak_launch<16>, int_peak_launch<17>,
                             int_peak_launch<18>};
  if (op < 0 || op >= (int)(sizeof(table) / sizeof(table[0]))) return cudaErrorInvalidValue;
  table[op](blocks, threads, iters, cycles, sink, stream);
  return cudaGetLastError();
}

__global__ void hb_set_count_kernel(uint64_t* n_dev, uint64_t n) { *n_dev = n; }

// Byte copies described by {src, dst, bytes} records, one block per record
// (grid-stride over records): 16-byte vector copies when both ends are
// 16-byte aligned, byte copies otherwise and for the tail.
__global__ void hb_gather_kernel(const HbCopy* copies, uint32_t count) {
  for (uint32_t r = blockIdx.x; r < count; r += gridDim.x) {
    const HbCopy c = copies[r];
    const uint8_t* src = reinterpret_cast<const uint8_t*>(c.src);
    uint8_t* dst = reinterpret_cast<uint8_t*>(c.dst);
    uint64_t done = 0;
    if (((c.src | c.dst) & 15u) == 0) {
      const uint64_t nv = c.bytes / 16;
      const uint4* s4 = reinterpret_cast<const uint4*>(src);
      uint4* d4 = reinterpret_cast<uint4*>(dst);
      for (uint64_t k = threadIdx.x; k < nv; k += blockDim.x) d4[k] = __ldg(s4 + k);
      done = nv * 16;
    }
    for (uint64_t k = done + threadIdx.x; k < c.bytes; k += blockDim.x) dst[k] = src[k];
  }
}

cudaError_t launch_gather(const HbCopy* copies, uint32_t count, int grid, cudaStream_t stream) {
  if (count == 0) return cudaSuccess;
  hb_gather_kernel<<<grid, 256, 0, stream>>>(copies, count);
  return cudaGetLastError();
}

cudaError_t launch_set_count(uint64_t* n_dev, uint64_t n, cudaStream_t stream) {
  hb_set_count_kernel<<<1, 1, 0, stream>>>(n_dev, n);
  return cudaGetLastError();
}

cudaError_t launch_selftest_wait(uint64_t limit_ns, int* status, cudaStream_t stream) {
  hb_selftest_wait_kernel<<<1, 32, 0, stream>>>(limit_ns, status);
  return cudaGetLastError();
}

}  // namespace hb
