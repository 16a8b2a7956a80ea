// hb_algs.cuh -- the three compression functions on one 64-byte block held in
// registers, fully unrolled: MD5 (RFC 1321 Sec. 3.4), SHA-1 (FIPS 180-4
// Sec. 6.1.2) and SM3 (GB/T 32905-2016 Sec. 5.3).  Boolean functions are one
// LOP3 each, rotations one funnel shift, sums fold into IADD3.  Work is split
// between the ALU pipe (LOP3, IADD3, SHF) and the multiply-add pipe (adds as
// x*1+y, rotations as the two halves of x*2^s; hb_device.cuh) so that both
// pipes carry about the same number of instructions per round.
//
// Word order on entry: MD5 takes the block's words little-endian; SHA-1 and
// SM3 take them big-endian (the staging code byte-swaps with PRMT).
#pragma once

#include <cstdint>

#include "hb_device.cuh"
#include "hb_md5_table.h"

namespace hb {

// Algorithm descriptors -------------------------------------------------------

// Whether an algorithm moves its adds to the FMA pipe (hb_device.cuh).  SHA-1
// and SM3 are bound by the ALU pipe and gain; MD5's round is one long chain of
// dependent operations, and at a few warps per SM sub-partition (long
// messages) the IMAD's longer latency costs more than the freed ALU slots.
constexpr bool kMd5Fma = false;
constexpr bool kSha1Fma = true;
constexpr bool kSm3Fma = true;

// The fused three-algorithm kernel: whether its MD5 adds go to the FMA pipe,
// and whether MD5 and SM3 run interleaved step by step (md5_sm3_compress).
// Both are off by default; measured on B300, neither is faster (the MD5 chain
// pays the IMAD latency, and the interleaved code is as large as the two
// unrolled functions).
#ifndef HB_MD5_FUSED_FMA
#define HB_MD5_FUSED_FMA 0
#endif
// X[k] + T[i] of MD5's steps as one IMAD on the FMA pipe in the fused kernel
// (off MD5's dependent chain; 64 ALU instructions fewer per block, +1% there;
// the MD5-only kernel measured mixed: +4% at 16 KiB, -4% at 55 B).
#ifndef HB_MD5_FUSED_XT
#define HB_MD5_FUSED_XT 1
#endif
constexpr bool kMd5FusedXt = HB_MD5_FUSED_XT != 0;
// SM3's SS1 sum as two IMADs in the fused kernel (sm3_round_t's S0F): +1.5%
// there; the SM3-only kernel measured 7-8% slower with it and keeps the IADD3.
#ifndef HB_SM3_FUSED_S0_FMA
#define HB_SM3_FUSED_S0_FMA 1
#endif
constexpr bool kSm3FusedS0Fma = HB_SM3_FUSED_S0_FMA != 0;
#ifndef HB_FUSED_INTERLEAVE
#define HB_FUSED_INTERLEAVE 0
#endif
constexpr bool kMd5FusedFma = HB_MD5_FUSED_FMA != 0;

// SM3 rotations that run on the FMA pipe (rotl_fma), one bit per site:
//   1 C <- B<<<9   2 G <- F<<<19   4 A<<<12   8 (A<<<12 + E + T)<<<7
//   16 both rotations of P0   32 W<<<15 in the expansion   64 W<<<7 in the
//   expansion   128 both rotations of P1   256 A<<<12 + E + T as two IMADs
#ifndef HB_SM3_FMA_ROT
#define HB_SM3_FMA_ROT 0
#endif
constexpr unsigned kSm3Rot = HB_SM3_FMA_ROT;

template <int ALG>
struct AlgTraits;

template <>
struct AlgTraits<HB_MD5> {
  static constexpr int kStateWords = 4;
  static constexpr int kDigestWords = 4;
  static constexpr bool kBigEndian = false;
};
template <>
struct AlgTraits<HB_SHA1> {
  static constexpr int kStateWords = 5;
  static constexpr int kDigestWords = 5;
  static constexpr bool kBigEndian = true;
};
template <>
struct AlgTraits<HB_SM3> {
  static constexpr int kStateWords = 8;
  static constexpr int kDigestWords = 8;
  static constexpr bool kBigEndian = true;
};

// ---------------------------------------------------------------------------
// MD5 (RFC 1321).

__device__ __forceinline__ void md5_init(uint32_t (&st)[8]) {
  // Sec. 3.3: A, B, C, D whose bytes, low-order first, are 01 23 45 67,
  // 89 ab cd ef, fe dc ba 98, 76 54 32 10.
  st[0] = 0x67452301u;
  st[1] = 0xefcdab89u;
  st[2] = 0x98badcfeu;
  st[3] = 0x10325476u;
}

// Step J of the 64 (RFC 1321 Sec. 3.4): a = b + ((a + g(b,c,d) + X[k] + T[J])
// <<< s), with g, the word index k and the shift s fixed by the round J / 16:
//   round 1  F = (x & y) | (~x & z)   k = j           s = 7 12 17 22
//   round 2  G = (x & z) | (y & ~z)   k = 1 + 5j      s = 5 9 14 20
//   round 3  H = x ^ y ^ z            k = 5 + 3j      s = 4 11 16 23
//   round 4  I = y ^ (x | ~z)         k = 7j          s = 6 10 15 21
// (j = J mod 16, k mod 16).  The four registers rotate one place per step:
// step J updates the one at position -J mod 4 of (A, B, C, D).  The sum
// a + X[k] + T[J] does not depend on b, c, d and is one IADD3.  F selects
// whether the adds run on the FMA pipe; the rotate-and-add alternates between
// its two equivalent forms, which differ only there.
template <int J>
struct Md5Step {
  static constexpr int kRound = J / 16;
  static constexpr int kJ = J % 16;
  static constexpr int kWord = kRound == 0   ? kJ
                               : kRound == 1 ? (1 + 5 * kJ) % 16
                               : kRound == 2 ? (5 + 3 * kJ) % 16
                                             : (7 * kJ) % 16;
  static constexpr int kShift = (kRound == 0   ? 0x16110c07
                                 : kRound == 1 ? 0x140e0905
                                 : kRound == 2 ? 0x17100b04
                                               : 0x150f0a06) >> (8 * (J % 4)) & 0xff;
  static constexpr uint32_t kLut = kRound == 0   ? LUT_CHOOSE
                                   : kRound == 1 ? LUT_MD5_G
                                   : kRound == 2 ? LUT_XOR3
                                                 : LUT_MD5_I;
  static constexpr int kA = (4 - J % 4) % 4;  // the register this step updates
};

template <int J, bool F, bool XT = false>
__device__ __forceinline__ void md5_step(uint32_t (&r)[4], const uint32_t (&X)[16],
                                         const MulConsts& mc) {
  using S = Md5Step<J>;
  constexpr uint32_t T[64] = {HB_MD5_T_TABLE};
  uint32_t& a = r[S::kA];
  const uint32_t b = r[(S::kA + 1) % 4], c = r[(S::kA + 2) % 4], d = r[(S::kA + 3) % 4];
  if constexpr (XT && !F) {
    // X[k] + T[J] does not depend on the chain: one IMAD on the FMA pipe,
    // then one IADD3, one SHF and one add on the ALU
    const uint32_t xt = mad_lo(X[S::kWord], mc.one, T[J]);
    a = a + xt + lop3<S::kLut>(b, c, d);
    a = rotl<S::kShift>(a) + b;
  } else {
    a += X[S::kWord] + T[J];
    a = add_f<F>(lop3<S::kLut>(b, c, d), a, mc);
    if constexpr (J % 2 == 0)
      a = rotl_add_f<S::kShift, F>(a, b, mc);
    else
      a = add_f<F>(rotl<S::kShift>(a), b, mc);
  }
}

template <int J, bool F, bool XT = false>
__device__ __forceinline__ void md5_steps(uint32_t (&r)[4], const uint32_t (&X)[16],
                                          const MulConsts& mc) {
  if constexpr (J < 64) {
    md5_step<J, F, XT>(r, X, mc);
    md5_steps<J + 1, F, XT>(r, X, mc);
  }
}

// F: the adds on the FMA pipe.  XT (when not F): only X[k] + T[i] there.
template <bool F = kMd5Fma, bool XT = false>
__device__ __forceinline__ void md5_compress(uint32_t (&st)[8], const uint32_t (&X)[16],
                                             const MulConsts& mc) {
  uint32_t r[4] = {st[0], st[1], st[2], st[3]};
  md5_steps<0, F, XT>(r, X, mc);
#pragma unroll
  for (int i = 0; i < 4; ++i) st[i] = add_f<F>(st[i], r[i], mc);
}

// ---------------------------------------------------------------------------
// SHA-1 (FIPS 180-4).

__device__ __forceinline__ void sha1_init(uint32_t (&st)[8]) {
  // Sec. 5.3.1
  st[0] = 0x67452301u;
  st[1] = 0xefcdab89u;
  st[2] = 0x98badcfeu;
  st[3] = 0x10325476u;
  st[4] = 0xc3d2e1f0u;
}

template <int T>
__device__ __forceinline__ uint32_t sha1_f(uint32_t x, uint32_t y, uint32_t z) {
  // Sec. 4.1.1: Ch, Parity, Maj, Parity over t = 0-19, 20-39, 40-59, 60-79.
  if constexpr (T < 20) return lop3<LUT_CHOOSE>(x, y, z);
  else if constexpr (T < 40) return lop3<LUT_XOR3>(x, y, z);
  else if constexpr (T < 60) return lop3<LUT_MAJ>(x, y, z);
  else return lop3<LUT_XOR3>(x, y, z);
}

template <int T>
__device__ __forceinline__ constexpr uint32_t sha1_k() {
  // Sec. 4.2.1
  return T < 20 ? 0x5a827999u : T < 40 ? 0x6ed9eba1u : T < 60 ? 0x8f1bbcdcu : 0xca62c1d6u;
}

// Rounds T .. 79 by compile-time recursion; W is the 16-word schedule ring.
// Split per round: the schedule word (two LOP3 and a rotate), f, ROTL30(b)
// and the shift-and-add half of ROTL5(a) + sum on the ALU; the adds
// e + W, + K, + f and the multiply half of ROTL5(a) + sum on the FMA pipe
// (ALU 6, FMA 4 while the schedule runs).
template <int T>
__device__ __forceinline__ void sha1_rounds(uint32_t& a, uint32_t& b, uint32_t& c, uint32_t& d,
                                            uint32_t& e, uint32_t (&W)[16], const MulConsts& mc) {
  if constexpr (T < 80) {
    // The round constant as a register operand of an IMAD (one MOV per group
    // of twenty rounds after the compiler hoists it).
    uint32_t k = sha1_k<T>();
    asm("" : "+r"(k));
    if constexpr (T >= 16) {
      W[T & 15] = rotl<1>(lop3<LUT_XOR3>(W[(T - 3) & 15], W[(T - 8) & 15], W[(T - 14) & 15]) ^
                          W[T & 15]);
    }
    const uint32_t ewk = add_f<kSha1Fma>(add_f<kSha1Fma>(e, W[T & 15], mc), k, mc);
    const uint32_t t = rotl_add_f<5, kSha1Fma>(a, add_f<kSha1Fma>(sha1_f<T>(b, c, d), ewk, mc), mc);
    e = d;
    d = c;
    c = rotl<30>(b);
    b = a;
    a = t;
    sha1_rounds<T + 1>(a, b, c, d, e, W, mc);
  }
}

__device__ __forceinline__ void sha1_compress(uint32_t (&st)[8], const uint32_t (&X)[16],
                                              const MulConsts& mc) {
  uint32_t W[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) W[i] = X[i];
  uint32_t a = st[0], b = st[1], c = st[2], d = st[3], e = st[4];
  sha1_rounds<0>(a, b, c, d, e, W, mc);
  st[0] = add_f<kSha1Fma>(st[0], a, mc);
  st[1] = add_f<kSha1Fma>(st[1], b, mc);
  st[2] = add_f<kSha1Fma>(st[2], c, mc);
  st[3] = add_f<kSha1Fma>(st[3], d, mc);
  st[4] = add_f<kSha1Fma>(st[4], e, mc);
}

// ---------------------------------------------------------------------------
// SM3 (GB/T 32905-2016).

__device__ __forceinline__ void sm3_init(uint32_t (&st)[8]) {
  // Sec. 4.1
  st[0] = 0x7380166fu;
  st[1] = 0x4914b2b9u;
  st[2] = 0x172442d7u;
  st[3] = 0xda8a0600u;
  st[4] = 0xa96f30bcu;
  st[5] = 0x163138aau;
  st[6] = 0xe38dee4du;
  st[7] = 0xb0fb0e4eu;
}

// T_j <<< (j mod 32), Sec. 4.2 and 5.3.3, folded at compile time.
__host__ __device__ constexpr uint32_t sm3_t_rot(int j) {
  const uint32_t t = j < 16 ? 0x79cc4519u : 0x7a879d8au;
  const int s = j % 32;
  return s == 0 ? t : (uint32_t)((t << s) | (t >> (32 - s)));
}
template <int J>
__device__ __forceinline__ constexpr uint32_t sm3_tj_rot() {
  return sm3_t_rot(J);
}

__device__ __forceinline__ uint32_t sm3_p0(uint32_t x, const MulConsts& mc) {
  constexpr bool F = (kSm3Rot & 16u) != 0;
  return lop3<LUT_XOR3>(x, rotl_f<9, F>(x, mc), rotl_f<17, F>(x, mc));
}
__device__ __forceinline__ uint32_t sm3_p1(uint32_t x, const MulConsts& mc) {
  constexpr bool F = (kSm3Rot & 128u) != 0;
  return lop3<LUT_XOR3>(x, rotl_f<15, F>(x, mc), rotl_f<23, F>(x, mc));
}

// Rounds J .. 63.  W is a 16-word ring holding W_{J} .. W_{J+3} (and older
// words still needed); round J first extends it with W_{J+4} (Sec. 5.3.2),
// so that W'_J = W_J ^ W_{J+4} is available.  Split per round: rotations,
// the Boolean functions, P0 and SS1's sum on the ALU; the six adds of TT1 and
// TT2 on the FMA pipe; the expansion (three LOP3, four rotations) on the ALU.
// S0F: SS1's sum A<<<12 + E + T_j as two IMADs on the FMA pipe instead of
// one IADD3 (the fused kernel's choice).
template <int J, bool S0F = false>
__device__ __forceinline__ void sm3_round_t(uint32_t (&v)[8], uint32_t (&W)[16], const MulConsts& mc,
                                            uint32_t tj) {
  {
    constexpr int M = J + 4;  // index of the word produced this round
    if constexpr (M >= 16 && M < 68) {
      const uint32_t x = lop3<LUT_XOR3>(W[(M - 16) & 15], W[(M - 9) & 15],
                                        rotl_f<15, (kSm3Rot & 32u) != 0>(W[(M - 3) & 15], mc));
      W[M & 15] = lop3<LUT_XOR3>(sm3_p1(x, mc), rotl_f<7, (kSm3Rot & 64u) != 0>(W[(M - 13) & 15], mc),
                                 W[(M - 6) & 15]);
    }
    uint32_t& A = v[0];
    uint32_t& B = v[1];
    uint32_t& C = v[2];
    uint32_t& D = v[3];
    uint32_t& E = v[4];
    uint32_t& F = v[5];
    uint32_t& G = v[6];
    uint32_t& H = v[7];
    const uint32_t wj = W[J & 15];
    const uint32_t wpj = wj ^ W[M & 15];
    const uint32_t a12 = rotl_f<12, (kSm3Rot & 4u) != 0>(A, mc);
    uint32_t s0;
    if constexpr (S0F || (kSm3Rot & 256u) != 0)
      s0 = add_f<true>(a12, add_f<true>(E, tj, mc), mc);
    else
      s0 = a12 + E + tj;
    const uint32_t ss1 = rotl_f<7, (kSm3Rot & 8u) != 0>(s0, mc);
    const uint32_t ss2 = ss1 ^ a12;
    uint32_t ff, gg;
    if constexpr (J < 16) {
      ff = lop3<LUT_XOR3>(A, B, C);
      gg = lop3<LUT_XOR3>(E, F, G);
    } else {
      ff = lop3<LUT_MAJ>(A, B, C);
      gg = lop3<LUT_CHOOSE>(E, F, G);
    }
    const uint32_t tt1 = add_f<kSm3Fma>(ss2, add_f<kSm3Fma>(ff, add_f<kSm3Fma>(D, wpj, mc), mc), mc);
    const uint32_t tt2 = add_f<kSm3Fma>(ss1, add_f<kSm3Fma>(gg, add_f<kSm3Fma>(H, wj, mc), mc), mc);
    D = C;
    C = rotl_f<9, (kSm3Rot & 1u) != 0>(B, mc);
    B = A;
    A = tt1;
    H = G;
    G = rotl_f<19, (kSm3Rot & 2u) != 0>(F, mc);
    F = E;
    E = sm3_p0(tt2, mc);
  }
}

template <int J, bool S0F = false>
__device__ __forceinline__ void sm3_round(uint32_t (&v)[8], uint32_t (&W)[16], const MulConsts& mc) {
  sm3_round_t<J, S0F>(v, W, mc, sm3_tj_rot<J>());
}

template <int J, int END = 64, bool S0F = false>
__device__ __forceinline__ void sm3_rounds(uint32_t (&v)[8], uint32_t (&W)[16], const MulConsts& mc) {
  if constexpr (J < END) {
    sm3_round<J, S0F>(v, W, mc);
    sm3_rounds<J + 1, END, S0F>(v, W, mc);
  }
}

// The rolled form of rounds 16-63: every round from 16 on has the same shape
// (Boolean functions, expansion) and the ring positions repeat every 16
// rounds, so rounds 16-31, 32-47 and 48-63 are one 16-round body run three
// times.  Only the constant T_j <<< (j mod 32) changes between passes; the
// body reads it from a constant-memory table at a warp-uniform index.  The
// rolled code is half the size: worth it where the three algorithms
// share one kernel (its instruction footprint is what the SM's instruction
// cache has to hold), not in the SM3-only kernel, whose unrolled form lets
// the scheduler overlap rounds across pass boundaries.
//   HB_SM3_ROLLED  0: unrolled everywhere  1: rolled in the three-algorithm
//                  kernel only (default)  2: rolled everywhere
#ifndef HB_SM3_ROLLED
#define HB_SM3_ROLLED 1
#endif

// T_j <<< (j mod 32) for j = 16..63 (Sec. 4.2, 5.3.3), for the rolled form.
struct Sm3TTable {
  uint32_t t[48];
};
__host__ __device__ constexpr Sm3TTable make_sm3_t_table() {
  Sm3TTable tb{};
  for (int j = 16; j < 64; ++j) tb.t[j - 16] = sm3_t_rot(j);
  return tb;
}
static __constant__ Sm3TTable kSm3TRot = make_sm3_t_table();

// Rounds 16 + 16 * pass + R .. 16 + 16 * pass + 15.
template <int R, bool S0F = false>
__device__ __forceinline__ void sm3_pass(uint32_t (&v)[8], uint32_t (&W)[16], const MulConsts& mc,
                                         int pass) {
  if constexpr (R < 16) {
    sm3_round_t<16 + R, S0F>(v, W, mc, kSm3TRot.t[16 * pass + R]);
    sm3_pass<R + 1, S0F>(v, W, mc, pass);
  }
}

template <bool ROLLED = (HB_SM3_ROLLED == 2), bool S0F = false>
__device__ __forceinline__ void sm3_compress(uint32_t (&st)[8], const uint32_t (&X)[16],
                                             const MulConsts& mc) {
  uint32_t W[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) W[i] = X[i];
  uint32_t v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = st[i];
  if constexpr (ROLLED) {
    sm3_rounds<0, 16, S0F>(v, W, mc);
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) sm3_pass<0, S0F>(v, W, mc, pass);
  } else {
    sm3_rounds<0, 64, S0F>(v, W, mc);
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) st[i] ^= v[i];
}

// ---------------------------------------------------------------------------
// MD5 and SM3 of the same block, step J of one beside round J of the other.
// Both run 64 steps; MD5's is one dependent chain, SM3's round has several
// independent parts, so issuing them side by side gives the scheduler work
// for the MD5 chain's latency.  X holds the block's words as MD5 reads them
// (little-endian), Y the same words big-endian for SM3.

template <int J, bool F>
__device__ __forceinline__ void md5_sm3_steps(uint32_t (&r)[4], const uint32_t (&X)[16],
                                              uint32_t (&v)[8], uint32_t (&W)[16],
                                              const MulConsts& mc) {
  if constexpr (J < 64) {
    md5_step<J, F>(r, X, mc);
    sm3_round<J>(v, W, mc);
    md5_sm3_steps<J + 1, F>(r, X, v, W, mc);
  }
}

template <bool F>
__device__ __forceinline__ void md5_sm3_compress(uint32_t (&md5)[8], uint32_t (&sm3)[8],
                                                 const uint32_t (&X)[16], const uint32_t (&Y)[16],
                                                 const MulConsts& mc) {
  uint32_t r[4] = {md5[0], md5[1], md5[2], md5[3]};
  uint32_t W[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) W[i] = Y[i];
  uint32_t v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = sm3[i];
  md5_sm3_steps<0, F>(r, X, v, W, mc);
#pragma unroll
  for (int i = 0; i < 4; ++i) md5[i] = add_f<F>(md5[i], r[i], mc);
#pragma unroll
  for (int i = 0; i < 8; ++i) sm3[i] ^= v[i];
}

// ---------------------------------------------------------------------------
// Uniform entry points.

template <int ALG>
__device__ __forceinline__ void alg_init(uint32_t (&st)[8]) {
  if constexpr (ALG == HB_MD5) md5_init(st);
  else if constexpr (ALG == HB_SHA1) sha1_init(st);
  else sm3_init(st);
}

template <int ALG>
__device__ __forceinline__ void alg_compress(uint32_t (&st)[8], const uint32_t (&X)[16],
                                             const MulConsts& mc) {
  if constexpr (ALG == HB_MD5) md5_compress<>(st, X, mc);
  else if constexpr (ALG == HB_SHA1) sha1_compress(st, X, mc);
  else sm3_compress<>(st, X, mc);
}

// Digest words in memory order for the 32-byte slot (zero fill after the
// digest): MD5 words little-endian as held, SHA-1 and SM3 byte-swapped.
template <int ALG>
__device__ __forceinline__ void alg_digest_words(const uint32_t (&st)[8], uint32_t (&out)[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    if (i < AlgTraits<ALG>::kDigestWords)
      out[i] = AlgTraits<ALG>::kBigEndian ? bswap32(st[i]) : st[i];
    else
      out[i] = 0u;
  }
}

}  // namespace hb
