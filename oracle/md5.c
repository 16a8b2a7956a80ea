/*
 * md5.c -- MD5 as defined in RFC 1321, written out step by step.
 *
 * TEST INFRASTRUCTURE ONLY (see hash_oracle.h).
 *
 * Sec. 3.1-3.2  padding and length (little-endian), in padding.c
 * Sec. 3.3      buffer A, B, C, D initialised to the words whose bytes,
 *               low-order first, are 01 23 45 67 / 89 ab cd ef /
 *               fe dc ba 98 / 76 54 32 10
 * Sec. 3.4      per 16-word block X: four rounds of sixteen operations
 *               a = b + ((a + g(b,c,d) + X[k] + T[i]) <<< s), where the
 *               roles of a, b, c, d rotate after every operation, g is
 *               F, G, H, I in rounds 1..4, and T[i] = floor(2^32 |sin i|);
 *               then A += AA etc.
 * Sec. 3.5      output A, B, C, D, each low-order byte first.
 */
#include <math.h>
#include <pthread.h>
#include <string.h>

#include "oracle_internal.h"

/* The four auxiliary functions of Sec. 3.4. */
static uint32_t md5_F(uint32_t x, uint32_t y, uint32_t z) { return (x & y) | (~x & z); }
static uint32_t md5_G(uint32_t x, uint32_t y, uint32_t z) { return (x & z) | (y & ~z); }
static uint32_t md5_H(uint32_t x, uint32_t y, uint32_t z) { return x ^ y ^ z; }
static uint32_t md5_I(uint32_t x, uint32_t y, uint32_t z) { return y ^ (x | ~z); }

/* T[i], i = 1..64 (stored at index i-1): the integer part of
 * 4294967296 * |sin(i)|, i in radians.  Computed in long double (64-bit
 * significand); the test-suite checks every entry against a 50-digit
 * evaluation of the same formula. */
static uint32_t md5_T[64];
static pthread_once_t md5_T_once = PTHREAD_ONCE_INIT;

static void md5_build_T(void)
{
    for (int i = 1; i <= 64; ++i) {
        long double v = 4294967296.0L * fabsl(sinl((long double)i));
        md5_T[i - 1] = (uint32_t)floorl(v);
    }
}

void oracle_md5_sine_table(uint32_t out[64])
{
    pthread_once(&md5_T_once, md5_build_T);
    memcpy(out, md5_T, sizeof(md5_T));
}

/* Message word index k and shift s of operation j (0..15) in round r (0..3),
 * as listed in Sec. 3.4: round 1 takes the words in order, round 2 steps
 * by 5 from word 1, round 3 by 3 from word 5, round 4 by 7 from word 0. */
static unsigned md5_word_index(unsigned r, unsigned j)
{
    switch (r) {
    case 0: return j;
    case 1: return (1u + 5u * j) % 16u;
    case 2: return (5u + 3u * j) % 16u;
    default: return (7u * j) % 16u;
    }
}

static unsigned md5_shift(unsigned r, unsigned j)
{
    static const unsigned s[4][4] = {
        {7, 12, 17, 22}, {5, 9, 14, 20}, {4, 11, 16, 23}, {6, 10, 15, 21}};
    return s[r][j % 4u];
}

static uint32_t md5_round_fn(unsigned r, uint32_t x, uint32_t y, uint32_t z)
{
    switch (r) {
    case 0: return md5_F(x, y, z);
    case 1: return md5_G(x, y, z);
    case 2: return md5_H(x, y, z);
    default: return md5_I(x, y, z);
    }
}

int oracle_md5(const uint8_t *msg, uint64_t len, uint8_t out[16])
{
    pthread_once(&md5_T_once, md5_build_T);

    /* Sec. 3.3: initial buffer, bytes listed low-order first. */
    uint32_t A = 0x67452301u, B = 0xefcdab89u, C = 0x98badcfeu, D = 0x10325476u;

    uint64_t nblocks = oracle_padded_blocks(len);
    uint8_t block[64];
    for (uint64_t q = 0; q < nblocks; ++q) {
        oracle_padded_block(msg, len, q, /*length_big_endian=*/0, block);

        /* Copy block q into X: word j is bytes 4j..4j+3, low-order first. */
        uint32_t X[16];
        for (unsigned j = 0; j < 16; ++j)
            X[j] = (uint32_t)block[4 * j] | ((uint32_t)block[4 * j + 1] << 8) |
                   ((uint32_t)block[4 * j + 2] << 16) | ((uint32_t)block[4 * j + 3] << 24);

        uint32_t AA = A, BB = B, CC = C, DD = D;
        uint32_t a = A, b = B, c = C, d = D;
        for (unsigned r = 0; r < 4; ++r) {
            for (unsigned j = 0; j < 16; ++j) {
                unsigned i = 16u * r + j; /* T index, 0-based */
                uint32_t sum = a + md5_round_fn(r, b, c, d) + X[md5_word_index(r, j)] + md5_T[i];
                uint32_t nb = b + oracle_rotl32(sum, md5_shift(r, j));
                /* [abcd] -> [dabc]: the next operation's a is this d, etc. */
                a = d;
                d = c;
                c = b;
                b = nb;
            }
        }
        A = a + AA;
        B = b + BB;
        C = c + CC;
        D = d + DD;
    }

    /* Sec. 3.5: A, B, C, D, each low-order byte first. */
    const uint32_t words[4] = {A, B, C, D};
    for (unsigned w = 0; w < 4; ++w)
        for (unsigned k = 0; k < 4; ++k)
            out[4 * w + k] = (uint8_t)(words[w] >> (8 * k));
    return 0;
}
