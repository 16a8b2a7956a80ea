// hb_device.cuh -- sm_103a device primitives used by the hashing kernels:
// integer ops pinned to single instructions (LOP3, SHF, PRMT), moves of adds
// and rotations to the multiply-add pipe, shared-memory and cp.async staging
// primitives, and the bounded mbarrier wait that reports a timeout instead of
// hanging.
#pragma once

#include <cstdint>

#include "hashbatch.h"
#include "hb_launch.h"

namespace hb {

// ---------------------------------------------------------------------------
// Integer building blocks.

// Three-input Boolean function as one LOP3; LUT is the function's truth table
// evaluated on the canonical operands a = 0xF0, b = 0xCC, c = 0xAA.
template <uint32_t LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
  return d;
}

// Truth tables, computed from the Boolean definitions on the canonical inputs.
constexpr uint32_t kA = 0xF0, kB = 0xCC, kC = 0xAA;
constexpr uint32_t LUT_XOR3 = (kA ^ kB ^ kC) & 0xFF;                         // x^y^z
constexpr uint32_t LUT_CHOOSE = ((kA & kB) | (~kA & kC)) & 0xFF;             // x?y:z
constexpr uint32_t LUT_MAJ = ((kA & kB) | (kA & kC) | (kB & kC)) & 0xFF;     // majority
constexpr uint32_t LUT_MD5_G = ((kA & kC) | (kB & ~kC)) & 0xFF;              // (x&z)|(y&~z)
constexpr uint32_t LUT_MD5_I = (kB ^ (kA | ~kC)) & 0xFF;                     // y^(x|~z)

// Left rotation as a funnel shift (SHF.L.W).
template <int S>
__device__ __forceinline__ uint32_t rotl(uint32_t x) {
  return __funnelshift_l(x, x, S);
}

// ---------------------------------------------------------------------------
// Work for the multiply-add pipe.  The SM's 32-bit integer ALU pipe (LOP3,
// IADD3, SHF, LEA, PRMT) retires 64 results per clock per SM; the multiply-add
// (FMA) pipe retires another 64 IMAD results per clock at the same time.  A
// two-input add becomes x * 1 + y, and a rotate-and-add splits into one ALU
// and one FMA instruction:
//   rotl(x, s) + y = x * 2^s + ((x >> (32 - s)) + y)       (s = 1..31)
// because x * 2^s mod 2^32 = x << s and the two parts of the rotation do not
// overlap; the shift-and-add is one LEA.HI.  The factors 1 and 2^s are kernel
// arguments, so the compiler cannot turn the multiplications back into ALU
// adds and shifts.  Standalone rotations stay one SHF on the ALU: moving one
// to the FMA pipe takes an IMAD.HI, which retires at a quarter of IMAD's rate.
// Each algorithm chooses (template argument F) whether its adds go to the
// FMA pipe; HB_FMA_OFFLOAD=0 forces the plain ALU forms everywhere.
#ifndef HB_FMA_OFFLOAD
#define HB_FMA_OFFLOAD 1
#endif

__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// x + y, on the FMA pipe when F.
template <bool F>
__device__ __forceinline__ uint32_t add_f(uint32_t x, uint32_t y, const MulConsts& m) {
  if constexpr (F && HB_FMA_OFFLOAD) return mad_lo(x, m.one, y);
  else return x + y;
}

// rotl(x, S) + y; when F, one ALU shift-and-add and one FMA multiply-add.
template <int S, bool F>
__device__ __forceinline__ uint32_t rotl_add_f(uint32_t x, uint32_t y, const MulConsts& m) {
  if constexpr (F && HB_FMA_OFFLOAD) return mad_lo(x, m.pow2[S], (x >> (32 - S)) + y);
  else return __funnelshift_l(x, x, S) + y;
}

// rotl(x, S) entirely on the FMA pipe: the 64-bit product x * 2^S holds
// x << S in its low word and x >> (32 - S) in its high word; their bits do not
// overlap, so their sum is the rotation (one IMAD.WIDE, one IMAD).
template <int S>
__device__ __forceinline__ uint32_t rotl_fma(uint32_t x, const MulConsts& m) {
  uint64_t w;
  asm("mul.wide.u32 %0, %1, %2;" : "=l"(w) : "r"(x), "r"(m.pow2[S]));
  return mad_lo((uint32_t)w, m.one, (uint32_t)(w >> 32));
}

// rotl(x, S) on the ALU pipe (one SHF) or, when F, on the FMA pipe.
template <int S, bool F>
__device__ __forceinline__ uint32_t rotl_f(uint32_t x, const MulConsts& m) {
  if constexpr (F && HB_FMA_OFFLOAD) return rotl_fma<S>(x, m);
  else return __funnelshift_l(x, x, S);
}

// Byte permute (PRMT): bytes of the 64-bit value {hi:lo} picked by `sel`.
__device__ __forceinline__ uint32_t prmt(uint32_t lo, uint32_t hi, uint32_t sel) {
  return __byte_perm(lo, hi, sel);
}

// Byte-reverse of one word.
__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

// ---------------------------------------------------------------------------
// Shared-memory, mbarrier and bulk-copy wrappers (PTX ISA, sm_90+).

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Make an mbarrier's initialisation visible before it is waited on.
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of an mbarrier to complete, giving up after
// `limit_ns` nanoseconds.  On timeout, records HB_DEV_TIMEOUT in *status and
// returns false; the caller stops issuing work.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns,
                                                  int* status) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 > limit_ns) {
      if (status) atomicOr(status, HB_DEV_TIMEOUT);
      return false;
    }
  }
}

// Shared-memory accesses by 32-bit shared-window address.  They are
// `volatile` so they keep their order relative to the cp.async waits and to
// each other at the source level, but carry no memory clobber, so the
// compiler still schedules the surrounding arithmetic freely.
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}

__device__ __forceinline__ uint4 lds128(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr));
  return v;
}

__device__ __forceinline__ void sts128(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w));
}

__device__ __forceinline__ void sts8(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.u8 [%0], %1;" ::"r"(addr), "r"(v));
}

// Asynchronous 16-byte global -> shared copy (LDGSTS, L2 only) of the first
// `src_bytes` (0..16) bytes at `src`; the rest of the 16 destination bytes are
// zero-filled.  Both addresses must be 16-byte aligned.
__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Wait until at most N of this thread's committed copy groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Read-only global loads of the per-message metadata.
__device__ __forceinline__ uint64_t ldg_nc_u64(const uint64_t* p) { return __ldg(p); }
__device__ __forceinline__ uint32_t ldg_nc_u32(const uint32_t* p) { return __ldg(p); }

// Streaming 16-byte global store (digest slots are written once).
__device__ __forceinline__ void stg128_cs(void* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.global.cs.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

}  // namespace hb
