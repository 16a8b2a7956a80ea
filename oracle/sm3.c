/*
 * sm3.c -- SM3 as defined in GB/T 32905-2016, written out step by step.
 *
 * TEST INFRASTRUCTURE ONLY (see hash_oracle.h).
 *
 * Sec. 4.1  initial value IV (eight 32-bit words)
 * Sec. 4.2  constants T_j: 79cc4519 for j = 0..15, 7a879d8a for 16..63
 * Sec. 4.3  Boolean functions FF_j, GG_j (XOR of three for j < 16, majority
 *           and choose for j >= 16)
 * Sec. 4.4  permutations P0(X) = X ^ (X<<<9) ^ (X<<<17),
 *           P1(X) = X ^ (X<<<15) ^ (X<<<23)
 * Sec. 5.2  padding with a 64-bit big-endian bit length (padding.c)
 * Sec. 5.3.2 message expansion into W_0..W_67 and W'_0..W'_63
 * Sec. 5.3.3 compression CF(V, B): 64 rounds over registers A..H, then
 *           V(i+1) = ABCDEFGH xor V(i)
 * Sec. 5.4  the digest is V(n), each word high-order byte first
 */
#include "oracle_internal.h"

static uint32_t sm3_T(unsigned j) { return j < 16 ? 0x79cc4519u : 0x7a879d8au; }

static uint32_t sm3_FF(unsigned j, uint32_t X, uint32_t Y, uint32_t Z)
{
    if (j < 16) return X ^ Y ^ Z;
    return (X & Y) | (X & Z) | (Y & Z);
}

static uint32_t sm3_GG(unsigned j, uint32_t X, uint32_t Y, uint32_t Z)
{
    if (j < 16) return X ^ Y ^ Z;
    return (X & Y) | (~X & Z);
}

static uint32_t sm3_P0(uint32_t X) { return X ^ oracle_rotl32(X, 9) ^ oracle_rotl32(X, 17); }
static uint32_t sm3_P1(uint32_t X) { return X ^ oracle_rotl32(X, 15) ^ oracle_rotl32(X, 23); }

int oracle_sm3(const uint8_t *msg, uint64_t len, uint8_t out[32])
{
    uint32_t V[8] = {0x7380166fu, 0x4914b2b9u, 0x172442d7u, 0xda8a0600u,
                     0xa96f30bcu, 0x163138aau, 0xe38dee4du, 0xb0fb0e4eu};

    uint64_t nblocks = oracle_padded_blocks(len);
    uint8_t block[64];
    for (uint64_t q = 0; q < nblocks; ++q) {
        oracle_padded_block(msg, len, q, /*length_big_endian=*/1, block);

        /* Sec. 5.3.2: expansion. */
        uint32_t W[68], Wp[64];
        for (unsigned j = 0; j < 16; ++j)
            W[j] = ((uint32_t)block[4 * j] << 24) | ((uint32_t)block[4 * j + 1] << 16) |
                   ((uint32_t)block[4 * j + 2] << 8) | (uint32_t)block[4 * j + 3];
        for (unsigned j = 16; j < 68; ++j)
            W[j] = sm3_P1(W[j - 16] ^ W[j - 9] ^ oracle_rotl32(W[j - 3], 15)) ^
                   oracle_rotl32(W[j - 13], 7) ^ W[j - 6];
        for (unsigned j = 0; j < 64; ++j)
            Wp[j] = W[j] ^ W[j + 4];

        /* Sec. 5.3.3: compression. */
        uint32_t A = V[0], B = V[1], C = V[2], D = V[3];
        uint32_t E = V[4], F = V[5], G = V[6], H = V[7];
        for (unsigned j = 0; j < 64; ++j) {
            uint32_t SS1 = oracle_rotl32(oracle_rotl32(A, 12) + E + oracle_rotl32(sm3_T(j), j % 32u), 7);
            uint32_t SS2 = SS1 ^ oracle_rotl32(A, 12);
            uint32_t TT1 = sm3_FF(j, A, B, C) + D + SS2 + Wp[j];
            uint32_t TT2 = sm3_GG(j, E, F, G) + H + SS1 + W[j];
            D = C;
            C = oracle_rotl32(B, 9);
            B = A;
            A = TT1;
            H = G;
            G = oracle_rotl32(F, 19);
            F = E;
            E = sm3_P0(TT2);
        }
        V[0] ^= A;
        V[1] ^= B;
        V[2] ^= C;
        V[3] ^= D;
        V[4] ^= E;
        V[5] ^= F;
        V[6] ^= G;
        V[7] ^= H;
    }

    for (unsigned w = 0; w < 8; ++w)
        for (unsigned k = 0; k < 4; ++k)
            out[4 * w + k] = (uint8_t)(V[w] >> (24 - 8 * k));
    return 0;
}
