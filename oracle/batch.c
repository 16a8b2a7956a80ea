/*
 * batch.c -- the batch form of the oracle: one digest per message, each in
 * its own 32-byte slot (paper Sec. IV-B, parallel crypto ops; Sec. V-D, each
 * input message and each output hash value in separate array locations).
 *
 * TEST INFRASTRUCTURE ONLY (see hash_oracle.h).
 *
 * The loop over messages is the definition: slot i is the digest of message
 * i followed by zero bytes.  Threads only split the index range; they do not
 * change what any slot holds.
 */
#include <pthread.h>
#include <string.h>

#include "oracle_internal.h"

size_t oracle_digest_size(int alg)
{
    switch (alg) {
    case ORACLE_MD5: return 16;
    case ORACLE_SHA1: return 20;
    case ORACLE_SM3: return 32;
    default: return 0;
    }
}

int oracle_digest(int alg, const uint8_t *msg, uint64_t len, uint8_t *out)
{
    switch (alg) {
    case ORACLE_MD5: return oracle_md5(msg, len, out);
    case ORACLE_SHA1: return oracle_sha1(msg, len, out);
    case ORACLE_SM3: return oracle_sm3(msg, len, out);
    default: return -1;
    }
}

struct batch_job {
    int alg;
    const uint8_t *algs;
    const uint8_t *packed;
    const uint64_t *offsets;
    const uint32_t *lengths;
    uint8_t *out;
    uint64_t begin, end;
    int status;
};

static void *batch_worker(void *arg)
{
    struct batch_job *job = (struct batch_job *)arg;
    for (uint64_t i = job->begin; i < job->end; ++i) {
        int alg = job->algs ? (int)job->algs[i] : job->alg;
        uint8_t *slot = job->out + (uint64_t)ORACLE_SLOT_BYTES * i;
        memset(slot, 0, ORACLE_SLOT_BYTES);
        if (oracle_digest(alg, job->packed + job->offsets[i], job->lengths[i], slot) != 0) {
            job->status = -1;
            return NULL;
        }
    }
    return NULL;
}

int oracle_hash_batch(int alg, const uint8_t *algs, const uint8_t *packed,
                      uint64_t packed_len, const uint64_t *offsets,
                      const uint32_t *lengths, uint64_t n, uint8_t *out,
                      int threads)
{
    if (n == 0)
        return 0;
    if (!offsets || !lengths || !out || (!packed && packed_len > 0))
        return -3;
    /* Reject bad inputs before writing anything. */
    for (uint64_t i = 0; i < n; ++i) {
        int a = algs ? (int)algs[i] : alg;
        if (oracle_digest_size(a) == 0)
            return -1;
        if (offsets[i] > packed_len || lengths[i] > packed_len - offsets[i])
            return -2;
    }

    if (threads < 1)
        threads = 1;
    if ((uint64_t)threads > n)
        threads = (int)n;

    struct batch_job jobs[256];
    pthread_t tids[256];
    if (threads > 256)
        threads = 256;
    for (int t = 0; t < threads; ++t) {
        jobs[t].alg = alg;
        jobs[t].algs = algs;
        jobs[t].packed = packed;
        jobs[t].offsets = offsets;
        jobs[t].lengths = lengths;
        jobs[t].out = out;
        jobs[t].begin = n * (uint64_t)t / (uint64_t)threads;
        jobs[t].end = n * (uint64_t)(t + 1) / (uint64_t)threads;
        jobs[t].status = 0;
    }
    if (threads == 1) {
        batch_worker(&jobs[0]);
        return jobs[0].status;
    }
    for (int t = 0; t < threads; ++t)
        pthread_create(&tids[t], NULL, batch_worker, &jobs[t]);
    int status = 0;
    for (int t = 0; t < threads; ++t) {
        pthread_join(tids[t], NULL);
        if (jobs[t].status)
            status = jobs[t].status;
    }
    return status;
}
