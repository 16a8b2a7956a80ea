/*
 * sha1.c -- SHA-1 as defined in FIPS 180-4, written out step by step.
 *
 * TEST INFRASTRUCTURE ONLY (see hash_oracle.h).
 *
 * Sec. 5.1.1  padding, 64-bit big-endian length (padding.c)
 * Sec. 5.2.1  the padded message is parsed into 512-bit blocks of sixteen
 *             32-bit big-endian words
 * Sec. 5.3.1  initial hash value H(0)
 * Sec. 4.1.1  f_t: Ch for t = 0..19, Parity for 20..39, Maj for 40..59,
 *             Parity for 60..79
 * Sec. 4.2.1  constants K_t for the same four ranges
 * Sec. 6.1.2  message schedule W_0..W_79, eighty rounds of
 *             T = ROTL5(a) + f_t(b,c,d) + e + K_t + W_t and the shift
 *             e=d, d=c, c=ROTL30(b), b=a, a=T; then H(i) = H(i-1) + (a..e)
 */
#include "oracle_internal.h"

static uint32_t sha1_Ch(uint32_t x, uint32_t y, uint32_t z) { return (x & y) ^ (~x & z); }
static uint32_t sha1_Parity(uint32_t x, uint32_t y, uint32_t z) { return x ^ y ^ z; }
static uint32_t sha1_Maj(uint32_t x, uint32_t y, uint32_t z) { return (x & y) ^ (x & z) ^ (y & z); }

static uint32_t sha1_f(unsigned t, uint32_t x, uint32_t y, uint32_t z)
{
    if (t < 20) return sha1_Ch(x, y, z);
    if (t < 40) return sha1_Parity(x, y, z);
    if (t < 60) return sha1_Maj(x, y, z);
    return sha1_Parity(x, y, z);
}

/* Sec. 4.2.1.  The four values are the integer parts of 2^30 times
 * sqrt 2, sqrt 3, sqrt 5 and sqrt 10; the test-suite re-derives them with an
 * integer square root. */
static uint32_t sha1_K(unsigned t)
{
    if (t < 20) return 0x5a827999u;
    if (t < 40) return 0x6ed9eba1u;
    if (t < 60) return 0x8f1bbcdcu;
    return 0xca62c1d6u;
}

uint32_t oracle_sha1_K(unsigned t) { return sha1_K(t); }

int oracle_sha1(const uint8_t *msg, uint64_t len, uint8_t out[20])
{
    /* Sec. 5.3.1 */
    uint32_t H[5] = {0x67452301u, 0xefcdab89u, 0x98badcfeu, 0x10325476u, 0xc3d2e1f0u};

    uint64_t nblocks = oracle_padded_blocks(len);
    uint8_t block[64];
    for (uint64_t q = 0; q < nblocks; ++q) {
        oracle_padded_block(msg, len, q, /*length_big_endian=*/1, block);

        uint32_t W[80];
        for (unsigned t = 0; t < 16; ++t)
            W[t] = ((uint32_t)block[4 * t] << 24) | ((uint32_t)block[4 * t + 1] << 16) |
                   ((uint32_t)block[4 * t + 2] << 8) | (uint32_t)block[4 * t + 3];
        for (unsigned t = 16; t < 80; ++t)
            W[t] = oracle_rotl32(W[t - 3] ^ W[t - 8] ^ W[t - 14] ^ W[t - 16], 1);

        uint32_t a = H[0], b = H[1], c = H[2], d = H[3], e = H[4];
        for (unsigned t = 0; t < 80; ++t) {
            uint32_t T = oracle_rotl32(a, 5) + sha1_f(t, b, c, d) + e + sha1_K(t) + W[t];
            e = d;
            d = c;
            c = oracle_rotl32(b, 30);
            b = a;
            a = T;
        }
        H[0] += a;
        H[1] += b;
        H[2] += c;
        H[3] += d;
        H[4] += e;
    }

    /* The digest is H0..H4, each high-order byte first. */
    for (unsigned w = 0; w < 5; ++w)
        for (unsigned k = 0; k < 4; ++k)
            out[4 * w + k] = (uint8_t)(H[w] >> (24 - 8 * k));
    return 0;
}
