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
// Scratch: `aux`, a power of two P >= 2n of 16-byte entries (key bits,
// index), probed linearly from a hash of the key.  An empty entry is all ones
// (index -1); a claimed entry's index is >= 0, so no claimed entry looks
// empty, whatever its key.  A key claims an empty entry with one 16-byte
// compare-and-swap that writes key and index together, so a probe compares
// keys without reading the caller's array again, and a later occurrence
// lowers the index with atomicMin (an entry's key never changes).  Then
// `lead` (n int64 leader indices) and `skip` (n bytes).
#include <cstdint>

#include "hc_core.cuh"
#include "hc_internal.h"

namespace hc {

namespace {

__device__ __forceinline__ unsigned long long aux_hash(unsigned long long k) {
    return fmix64(k ^ 0xD6E8FEB86659FD93ull);
}

struct AuxEntry {
    unsigned long long key;
    long long idx;
};

__device__ __forceinline__ AuxEntry load_entry(const AuxEntry *e) {
    AuxEntry r;
    asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(r.key), "=l"(r.idx) : "l"(e));
    return r;
}

// 16-byte compare-and-swap of an empty entry (all ones) to (key, idx);
// returns the entry as it was.
__device__ __forceinline__ AuxEntry claim_entry(AuxEntry *e, unsigned long long key, long long idx) {
    AuxEntry r;
    asm volatile("{\n\t.reg .b128 c, v, d;\n\t"
                 "mov.b128 c, {%2, %2};\n\t"
                 "mov.b128 v, {%3, %4};\n\t"
                 "atom.global.cas.b128 d, [%5], c, v;\n\t"
                 "mov.b128 {%0, %1}, d;\n\t}"
                 : "=l"(r.key), "=l"(r.idx)
                 : "l"(~0ull), "l"(key), "l"(idx), "l"(e)
                 : "memory");
    return r;
}

template <class Key>
__global__ void __launch_bounds__(256) k_claim_leaders(const Key *keys, long long n, AuxEntry *aux,
                                                       unsigned long long mask, unsigned *err) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const unsigned long long k = (unsigned long long)keys[i];
        unsigned long long h = aux_hash(k) & mask;
        bool done = false;
        for (unsigned long long p = 0; p <= mask && !done; ++p) {
            AuxEntry cur = load_entry(aux + h);
            // an empty entry is claimed; an entry whose key reads as all ones
            // goes through the swap too, which returns it whole (a read that
            // overlapped a claim could pair the new index with the old key)
            if (cur.idx < 0 || cur.key == ~0ull) {
                cur = claim_entry(aux + h, k, i);
                if (cur.idx < 0) { done = true; break; }
            }
            if (cur.key == k) {
                if (i < cur.idx) atomicMin(&aux[h].idx, i);
                done = true;
                break;
            }
            h = (h + 1) & mask;
        }
        if (!done) atomicOr(err, ERR_PROBE_BOUND);   // cannot happen with P >= 2n
    }
}

template <class Key>
__global__ void __launch_bounds__(256) k_mark_followers(const Key *keys, long long n, const AuxEntry *aux,
                                                        unsigned long long mask, long long *lead, uint8_t *skip) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const unsigned long long k = (unsigned long long)keys[i];
        unsigned long long h = aux_hash(k) & mask;
        long long leader = i;
        for (unsigned long long p = 0; p <= mask; ++p) {
            const AuxEntry cur = load_entry(aux + h);
            if (cur.idx < 0) break;                     // cannot happen: the key was claimed
            if (cur.key == k) {
                leader = cur.idx;
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

long long ordered_scratch_bytes(long long n) {
    const unsigned long long P = ordered_aux_slots(n);
    return (long long)((P * sizeof(AuxEntry) + (unsigned long long)n * 9ull + 255ull) / 256ull * 256ull);
}

cudaError_t ordered_leaders(const void *keys, int key_bytes, long long n, void *scratch, unsigned *err, int sms,
                            cudaStream_t s) {
    const unsigned long long P = ordered_aux_slots(n);
    AuxEntry *aux = static_cast<AuxEntry *>(scratch);
    long long *lead = reinterpret_cast<long long *>(aux + P);
    uint8_t *skip = reinterpret_cast<uint8_t *>(lead + n);
    cudaError_t e = cudaMemsetAsync(aux, 0xFF, P * sizeof(AuxEntry), s);
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
    const long long *lead = reinterpret_cast<const long long *>(static_cast<const AuxEntry *>(scratch) + P);
    const uint8_t *skip = reinterpret_cast<const uint8_t *>(lead + n);
    k_follow_insert<<<grid_of(n, sms), 256, 0, s>>>(n, lead, skip, status);
    return cudaGetLastError();
}

const uint8_t *ordered_skip(long long n, const void *scratch) {
    const unsigned long long P = ordered_aux_slots(n);
    return reinterpret_cast<const uint8_t *>(reinterpret_cast<const long long *>(static_cast<const AuxEntry *>(scratch) + P) + n);
}

}  // namespace hc
