/*
 * padding.c -- Merkle-Damgard padding, one byte at a time.
 *
 * TEST INFRASTRUCTURE ONLY (see hash_oracle.h).
 *
 * All three standards pad the same way and differ only in the byte order of
 * the appended length (RFC 1321 Sec. 3.1-3.2: low-order byte first;
 * FIPS 180-4 Sec. 5.1.1 and GB/T 32905-2016 Sec. 5.2: high-order byte first):
 *   padded = message || 0x80 || 0x00 ... 0x00 || (8*L mod 2^64, 8 bytes)
 * with the smallest number of zero bytes that makes the total a multiple of
 * 64 bytes.  Nothing here is blocked or vectorised: the oracle asks for the
 * padded message byte by byte.
 */
#include "oracle_internal.h"

uint64_t oracle_padded_blocks(uint64_t len)
{
    /* message + one 0x80 byte + 8 length bytes, rounded up to 64 bytes */
    return (len + 1 + 8 + 63) / 64;
}

uint8_t oracle_padded_byte(const uint8_t *msg, uint64_t len, uint64_t p,
                           int length_big_endian)
{
    uint64_t total = 64 * oracle_padded_blocks(len);
    if (p < len)
        return msg[p];
    if (p == len)
        return 0x80;
    if (p >= total - 8) {
        uint64_t bits = len * 8u; /* unsigned wrap: the bit length mod 2^64 */
        unsigned k = (unsigned)(p - (total - 8)); /* 0..7 within the field */
        unsigned shift = length_big_endian ? 8u * (7u - k) : 8u * k;
        return (uint8_t)(bits >> shift);
    }
    return 0;
}

void oracle_padded_block(const uint8_t *msg, uint64_t len, uint64_t block,
                         int length_big_endian, uint8_t out[64])
{
    for (unsigned j = 0; j < 64; ++j)
        out[j] = oracle_padded_byte(msg, len, 64 * block + j, length_big_endian);
}
