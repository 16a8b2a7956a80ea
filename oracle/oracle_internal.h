/*
 * oracle_internal.h -- helpers shared by the oracle's own C files.
 *
 * TEST INFRASTRUCTURE ONLY (see hash_oracle.h).  Not visible to, and not
 * used by, the CUDA library.
 */
#ifndef ORACLE_INTERNAL_H
#define ORACLE_INTERNAL_H

#include "hash_oracle.h"

/* Number of 64-byte blocks after padding a message of `len` bytes. */
uint64_t oracle_padded_blocks(uint64_t len);

/* Byte p (0 <= p < 64 * oracle_padded_blocks(len)) of the padded message. */
uint8_t oracle_padded_byte(const uint8_t *msg, uint64_t len, uint64_t p,
                           int length_big_endian);

/* The 64 bytes of padded block number `block`. */
void oracle_padded_block(const uint8_t *msg, uint64_t len, uint64_t block,
                         int length_big_endian, uint8_t out[64]);

/* Left rotation of a 32-bit word by s bits, 0 <= s < 32. */
static inline uint32_t oracle_rotl32(uint32_t x, unsigned s)
{
    s &= 31u;
    return s ? (uint32_t)((x << s) | (x >> (32u - s))) : x;
}

#endif
