/*
 * hash_oracle.h -- plain, slow CPU reference for the batched-hash hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no header, table or helper with the
 * CUDA library; the two are compared digest by digest.
 *
 * What it computes (paper Sec. IV-B: the "parallel scenario" crypto ops, one
 * digest per message, each message and each digest in its own array slot as
 * in Sec. V-D):
 *   MD5    -- RFC 1321 (Sec. 3.1-3.5), 16-byte digest, little-endian words.
 *   SHA-1  -- FIPS 180-4 (Sec. 5.1.1 padding, 5.3.1 IV, 6.1.2 hash), 20 bytes.
 *   SM3    -- GB/T 32905-2016 (Sec. 5.2 padding, 5.3 expansion and
 *             compression), 32-byte digest.
 * Messages are byte strings; the bit length is 8*L mod 2^64.
 *
 * Batch layout: message i is packed[offsets[i] .. offsets[i]+lengths[i]);
 * its digest goes to out[32*i .. 32*i+32): digest bytes first, zero fill
 * after.  Messages may overlap and start at any byte.
 */
#ifndef HASH_ORACLE_H
#define HASH_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORACLE_MD5 = 0, ORACLE_SHA1 = 1, ORACLE_SM3 = 2 };

#define ORACLE_SLOT_BYTES 32

/* Digest size in bytes for an algorithm code, 0 for an unknown code. */
size_t oracle_digest_size(int alg);

/* One message, one digest.  `out` receives oracle_digest_size(alg) bytes.
 * Returns 0, or -1 for an unknown algorithm. */
int oracle_md5(const uint8_t *msg, uint64_t len, uint8_t out[16]);
int oracle_sha1(const uint8_t *msg, uint64_t len, uint8_t out[20]);
int oracle_sm3(const uint8_t *msg, uint64_t len, uint8_t out[32]);
int oracle_digest(int alg, const uint8_t *msg, uint64_t len, uint8_t *out);

/* The 64 MD5 additive constants T[1..64] of RFC 1321 Sec. 3.4, as computed by
 * the oracle from their definition floor(2^32 * |sin(i)|). */
void oracle_md5_sine_table(uint32_t out[64]);

/* The SHA-1 round constant K_t of FIPS 180-4 Sec. 4.2.1, t = 0..79. */
uint32_t oracle_sha1_K(unsigned t);

/* Batch of n messages with one algorithm (alg >= 0) or with a per-message
 * algorithm array (algs != NULL, alg ignored).  packed_len bounds every
 * message.  Work is split over `threads` POSIX threads (<= 0: one).
 * Returns 0; -1 bad algorithm; -2 message outside packed_len; -3 null
 * pointer with n > 0. */
int oracle_hash_batch(int alg, const uint8_t *algs, const uint8_t *packed,
                      uint64_t packed_len, const uint64_t *offsets,
                      const uint32_t *lengths, uint64_t n, uint8_t *out,
                      int threads);

#ifdef __cplusplus
}
#endif

#endif
