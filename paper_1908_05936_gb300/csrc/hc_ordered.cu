// hc_ordered.cu -- the lowest index wins among equal keys of one batch.
//
// Section 4 leaves which of several equal keys of one concurrent insert
// stores itself (and, for maps, its value) to the scheduler.  The ordered
// calls fix it: every occurrence of a key finds the lowest index at which the
// key occurs in the batch (its leader) through a scratch hash table of
// indices, only leaders probe the container, and the other occurrences take
// the result a sequential pass in index order gives them: EXISTS after their
// leader's insert (OVERFLOW if the leader overflowed), NOT_FOUND after their
// leader's erase.
//
// Scratch: `aux`, a power of two P >= 2n of int64 indices (-1 = empty slot),
// probed linearly from a hash of the key; an entry's key is the key at its
// index in the caller's array, so entries need no key field and a slot's key
// never changes (atomicMin replaces an index only by a smaller index of the
// same key).  Then `lead` (n int64 leader indices) and `skip` (n bytes).
#include <cstdint>

#include "hc_core.cuh"
#include "hc_internal.h"

namespace hc {

namespace {

__device__ __forceinline__ unsigned long long aux_hash(unsigned long long k) {
    return fmix64(k ^ 0xD6E8FEB86659FD93ull);
}

template <class Key>
__global__ void __launch_bounds__(256) k_claim_leaders(const Key *keys, long long n, long long *aux,
                                                       unsigned long long mask, unsigned *err) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const Key k = keys[i];
        unsigned long long h = aux_hash((unsigned long long)k) & mask;
        bool done = false;
        for (unsigned long long p = 0; p <= mask && !done; ++p) {
            long long cur = *((volatile long long *)&aux[h]);
            if (cur < 0) {
                cur = (long long)atomicCAS(reinterpret_cast<unsigned long long *>(&aux[h]), ~0ull,
                                           (unsigned long long)i);
                if (cur < 0) { done = true; break; }
            }
            if (keys[cur] == k) {
                atomicMin(&aux[h], i);
                done = true;
                break;
            }
            h = (h + 1) & mask;
        }
        if (!done) atomicOr(err, ERR_PROBE_BOUND);   // cannot happen with P >= 2n
    }
}

template <class Key>
__global__ void __launch_bounds__(256) k_mark_followers(const Key *keys, long long n, const long long *aux,
                                                        unsigned long long mask, long long *lead, uint8_t *skip) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const Key k = keys[i];
        unsigned long long h = aux_hash((unsigned long long)k) & mask;
        long long leader = i;
        for (unsigned long long p = 0; p <= mask; ++p) {
            const long long cur = aux[h];
            if (cur < 0) break;                         // cannot happen: the key was claimed
            if (keys[cur] == k) {
                leader = cur;
                break;
            }
            h = (h + 1) & mask;
        }
        lead[i] = leader;
        skip[i] = leader != i;
    }
}

__global__ void __launch_bounds__(256) k_follow_insert(long long n, const long long *lead, const uint8_t *skip,
                                                       uint8_t *status) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && skip[i]) status[i] = status[lead[i]] == ST_OVERFLOW ? (uint8_t)ST_OVERFLOW : (uint8_t)ST_EXISTS;
}

// One thread per key and as many 256-thread blocks as the keys need: short
// blocks let an SM refill as soon as its slowest probes finish.
unsigned grid_of(long long n, int) {
    const long long g = (n + 255) / 256;
    return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

unsigned long long ordered_aux_slots(long long n) {
    unsigned long long p = 64;
    while (p < 2ull * (unsigned long long)n) p <<= 1;
    return p;
}

cudaError_t ordered_leaders(const void *keys, int key_bytes, long long n, void *scratch, unsigned *err, int sms,
                            cudaStream_t s) {
    const unsigned long long P = ordered_aux_slots(n);
    long long *aux = static_cast<long long *>(scratch);
    long long *lead = aux + P;
    uint8_t *skip = reinterpret_cast<uint8_t *>(lead + n);
    cudaError_t e = cudaMemsetAsync(aux, 0xFF, P * sizeof(long long), s);
    if (e != cudaSuccess) return e;
    const unsigned g = grid_of(n, sms);
    if (key_bytes == 4) {
        k_claim_leaders<uint32_t><<<g, 256, 0, s>>>((const uint32_t *)keys, n, aux, P - 1, err);
        k_mark_followers<uint32_t><<<g, 256, 0, s>>>((const uint32_t *)keys, n, aux, P - 1, lead, skip);
    } else {
        k_claim_leaders<unsigned long long><<<g, 256, 0, s>>>((const unsigned long long *)keys, n, aux, P - 1, err);
        k_mark_followers<unsigned long long><<<g, 256, 0, s>>>((const unsigned long long *)keys, n, aux, P - 1,
                                                                lead, skip);
    }
    return cudaGetLastError();
}

cudaError_t ordered_follow_insert(long long n, void *scratch, uint8_t *status, int sms, cudaStream_t s) {
    const unsigned long long P = ordered_aux_slots(n);
    const long long *lead = static_cast<const long long *>(scratch) + P;
    const uint8_t *skip = reinterpret_cast<const uint8_t *>(lead + n);
    k_follow_insert<<<grid_of(n, sms), 256, 0, s>>>(n, lead, skip, status);
    return cudaGetLastError();
}

const uint8_t *ordered_skip(long long n, const void *scratch) {
    const unsigned long long P = ordered_aux_slots(n);
    return reinterpret_cast<const uint8_t *>(static_cast<const long long *>(scratch) + P + n);
}

}  // namespace hc
