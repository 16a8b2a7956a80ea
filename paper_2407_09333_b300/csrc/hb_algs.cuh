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

// One operation a = b + ((a + g(b,c,d) + X[k] + T[i]) <<< s).  The sum
// a + X[k] + T[i] does not depend on b, c, d and is one IADD3.  (V selects
// between two equivalent forms of the rotate-and-add; they differ only when
// the adds go to the FMA pipe.)
#define HB_MD5_OP(LUT, a, b, c, d, xk, t, s, V)           \
  do {                                                   \
    a += (xk) + (t);                                     \
    a = add_f<kMd5Fma>(lop3<LUT>(b, c, d), a, mc);       \
    if (V)                                               \
      a = rotl_add_f<s, kMd5Fma>(a, b, mc);              \
    else                                                 \
      a = add_f<kMd5Fma>(rotl<s>(a), b, mc);             \
  } while (0)

// Round 2's G(x,y,z) = (x & z) | (y & ~z): LUT built with x->a, y->b, z->c.
__device__ __forceinline__ void md5_compress(uint32_t (&st)[8], const uint32_t (&X)[16],
                                             const MulConsts& mc) {
  constexpr uint32_t T[64] = {HB_MD5_T_TABLE};
  uint32_t a = st[0], b = st[1], c = st[2], d = st[3];
  // Round 1: F, words in order, shifts 7 12 17 22.
  HB_MD5_OP(LUT_CHOOSE, a, b, c, d, X[0], T[0], 7, 1);
  HB_MD5_OP(LUT_CHOOSE, d, a, b, c, X[1], T[1], 12, 0);
  HB_MD5_OP(LUT_CHOOSE, c, d, a, b, X[2], T[2], 17, 1);
  HB_MD5_OP(LUT_CHOOSE, b, c, d, a, X[3], T[3], 22, 0);
  HB_MD5_OP(LUT_CHOOSE, a, b, c, d, X[4], T[4], 7, 1);
  HB_MD5_OP(LUT_CHOOSE, d, a, b, c, X[5], T[5], 12, 0);
  HB_MD5_OP(LUT_CHOOSE, c, d, a, b, X[6], T[6], 17, 1);
  HB_MD5_OP(LUT_CHOOSE, b, c, d, a, X[7], T[7], 22, 0);
  HB_MD5_OP(LUT_CHOOSE, a, b, c, d, X[8], T[8], 7, 1);
  HB_MD5_OP(LUT_CHOOSE, d, a, b, c, X[9], T[9], 12, 0);
  HB_MD5_OP(LUT_CHOOSE, c, d, a, b, X[10], T[10], 17, 1);
  HB_MD5_OP(LUT_CHOOSE, b, c, d, a, X[11], T[11], 22, 0);
  HB_MD5_OP(LUT_CHOOSE, a, b, c, d, X[12], T[12], 7, 1);
  HB_MD5_OP(LUT_CHOOSE, d, a, b, c, X[13], T[13], 12, 0);
  HB_MD5_OP(LUT_CHOOSE, c, d, a, b, X[14], T[14], 17, 1);
  HB_MD5_OP(LUT_CHOOSE, b, c, d, a, X[15], T[15], 22, 0);
  // Round 2: G, words 1 + 5j mod 16, shifts 5 9 14 20.
  HB_MD5_OP(LUT_MD5_G, a, b, c, d, X[1], T[16], 5, 1);
  HB_MD5_OP(LUT_MD5_G, d, a, b, c, X[6], T[17], 9, 0);
  HB_MD5_OP(LUT_MD5_G, c, d, a, b, X[11], T[18], 14, 1);
  HB_MD5_OP(LUT_MD5_G, b, c, d, a, X[0], T[19], 20, 0);
  HB_MD5_OP(LUT_MD5_G, a, b, c, d, X[5], T[20], 5, 1);
  HB_MD5_OP(LUT_MD5_G, d, a, b, c, X[10], T[21], 9, 0);
  HB_MD5_OP(LUT_MD5_G, c, d, a, b, X[15], T[22], 14, 1);
  HB_MD5_OP(LUT_MD5_G, b, c, d, a, X[4], T[23], 20, 0);
  HB_MD5_OP(LUT_MD5_G, a, b, c, d, X[9], T[24], 5, 1);
  HB_MD5_OP(LUT_MD5_G, d, a, b, c, X[14], T[25], 9, 0);
  HB_MD5_OP(LUT_MD5_G, c, d, a, b, X[3], T[26], 14, 1);
  HB_MD5_OP(LUT_MD5_G, b, c, d, a, X[8], T[27], 20, 0);
  HB_MD5_OP(LUT_MD5_G, a, b, c, d, X[13], T[28], 5, 1);
  HB_MD5_OP(LUT_MD5_G, d, a, b, c, X[2], T[29], 9, 0);
  HB_MD5_OP(LUT_MD5_G, c, d, a, b, X[7], T[30], 14, 1);
  HB_MD5_OP(LUT_MD5_G, b, c, d, a, X[12], T[31], 20, 0);
  // Round 3: H, words 5 + 3j mod 16, shifts 4 11 16 23.
  HB_MD5_OP(LUT_XOR3, a, b, c, d, X[5], T[32], 4, 1);
  HB_MD5_OP(LUT_XOR3, d, a, b, c, X[8], T[33], 11, 0);
  HB_MD5_OP(LUT_XOR3, c, d, a, b, X[11], T[34], 16, 1);
  HB_MD5_OP(LUT_XOR3, b, c, d, a, X[14], T[35], 23, 0);
  HB_MD5_OP(LUT_XOR3, a, b, c, d, X[1], T[36], 4, 1);
  HB_MD5_OP(LUT_XOR3, d, a, b, c, X[4], T[37], 11, 0);
  HB_MD5_OP(LUT_XOR3, c, d, a, b, X[7], T[38], 16, 1);
  HB_MD5_OP(LUT_XOR3, b, c, d, a, X[10], T[39], 23, 0);
  HB_MD5_OP(LUT_XOR3, a, b, c, d, X[13], T[40], 4, 1);
  HB_MD5_OP(LUT_XOR3, d, a, b, c, X[0], T[41], 11, 0);
  HB_MD5_OP(LUT_XOR3, c, d, a, b, X[3], T[42], 16, 1);
  HB_MD5_OP(LUT_XOR3, b, c, d, a, X[6], T[43], 23, 0);
  HB_MD5_OP(LUT_XOR3, a, b, c, d, X[9], T[44], 4, 1);
  HB_MD5_OP(LUT_XOR3, d, a, b, c, X[12], T[45], 11, 0);
  HB_MD5_OP(LUT_XOR3, c, d, a, b, X[15], T[46], 16, 1);
  HB_MD5_OP(LUT_XOR3, b, c, d, a, X[2], T[47], 23, 0);
  // Round 4: I, words 7j mod 16, shifts 6 10 15 21.
  HB_MD5_OP(LUT_MD5_I, a, b, c, d, X[0], T[48], 6, 1);
  HB_MD5_OP(LUT_MD5_I, d, a, b, c, X[7], T[49], 10, 0);
  HB_MD5_OP(LUT_MD5_I, c, d, a, b, X[14], T[50], 15, 1);
  HB_MD5_OP(LUT_MD5_I, b, c, d, a, X[5], T[51], 21, 0);
  HB_MD5_OP(LUT_MD5_I, a, b, c, d, X[12], T[52], 6, 1);
  HB_MD5_OP(LUT_MD5_I, d, a, b, c, X[3], T[53], 10, 0);
  HB_MD5_OP(LUT_MD5_I, c, d, a, b, X[10], T[54], 15, 1);
  HB_MD5_OP(LUT_MD5_I, b, c, d, a, X[1], T[55], 21, 0);
  HB_MD5_OP(LUT_MD5_I, a, b, c, d, X[8], T[56], 6, 1);
  HB_MD5_OP(LUT_MD5_I, d, a, b, c, X[15], T[57], 10, 0);
  HB_MD5_OP(LUT_MD5_I, c, d, a, b, X[6], T[58], 15, 1);
  HB_MD5_OP(LUT_MD5_I, b, c, d, a, X[13], T[59], 21, 0);
  HB_MD5_OP(LUT_MD5_I, a, b, c, d, X[4], T[60], 6, 1);
  HB_MD5_OP(LUT_MD5_I, d, a, b, c, X[11], T[61], 10, 0);
  HB_MD5_OP(LUT_MD5_I, c, d, a, b, X[2], T[62], 15, 1);
  HB_MD5_OP(LUT_MD5_I, b, c, d, a, X[9], T[63], 21, 0);
  st[0] = add_f<kMd5Fma>(st[0], a, mc);
  st[1] = add_f<kMd5Fma>(st[1], b, mc);
  st[2] = add_f<kMd5Fma>(st[2], c, mc);
  st[3] = add_f<kMd5Fma>(st[3], d, mc);
}
#undef HB_MD5_OP

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
template <int J>
__device__ __forceinline__ constexpr uint32_t sm3_tj_rot() {
  constexpr uint32_t t = J < 16 ? 0x79cc4519u : 0x7a879d8au;
  constexpr int s = J % 32;
  return s == 0 ? t : (uint32_t)((t << s) | (t >> (32 - s)));
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
template <int J>
__device__ __forceinline__ void sm3_rounds(uint32_t (&v)[8], uint32_t (&W)[16], const MulConsts& mc) {
  if constexpr (J < 64) {
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
    if constexpr ((kSm3Rot & 256u) != 0)
      s0 = add_f<true>(a12, add_f<true>(E, sm3_tj_rot<J>(), mc), mc);
    else
      s0 = a12 + E + sm3_tj_rot<J>();
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
    sm3_rounds<J + 1>(v, W, mc);
  }
}

__device__ __forceinline__ void sm3_compress(uint32_t (&st)[8], const uint32_t (&X)[16],
                                             const MulConsts& mc) {
  uint32_t W[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) W[i] = X[i];
  uint32_t v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = st[i];
  sm3_rounds<0>(v, W, mc);
#pragma unroll
  for (int i = 0; i < 8; ++i) st[i] ^= v[i];
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
  if constexpr (ALG == HB_MD5) md5_compress(st, X, mc);
  else if constexpr (ALG == HB_SHA1) sha1_compress(st, X, mc);
  else sm3_compress(st, X, mc);
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
