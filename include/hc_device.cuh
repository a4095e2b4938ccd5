// hc_device.cuh -- in-kernel function form of the hash containers.
//
// Section 4.1 of "stdgpu: Efficient STL-like Data Structures on the GPU"
// gives the containers two interfaces: range calls over whole arrays
// (include/hc.h) and per-thread functions that custom kernels call on a
// container passed to them by value (a shallow copy, Section 3.7): insert
// returns where the key is stored and whether this call stored it, find
// returns where it is stored or end, contains and erase report presence and
// removal.  This header is that second interface.  A kernel receives the
// hc_device_view of a table (hc_device_view_get) by value and wraps it:
//
//     __global__ void k(hc_device_view dv, const uint64_t *keys, int64_t n) {
//         hcd::Table<HC_SET_U64> set(dv);
//         const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
//         if (i < n) set.insert(keys[i]);
//     }
//
// Every function is called by single threads, in divergent code if need
// be; no warp-wide participation is required.  Layout, hashing and probing
// are those of the library's own kernels (this header includes their device
// core), so range calls and device functions see the same table.
//
// Concurrency (Section 4: modifications are thread-safe, lookups need no
// lock, and every operation may run concurrently with every other; capacity
// overflow is the only failure):
//   insert   probes from the key's first bucket; stops at the key (EXISTS)
//            or at the first bucket holding an EMPTY slot and claims the
//            first EMPTY slot in a key-dependent order.  Only EMPTY slots
//            are claimed, never tombstones.  Slots never become EMPTY again
//            while kernels run, so every insert of one key reaches the same
//            bucket and the same slot, and a key is stored at most once.
//            Sets claim with one compare-and-swap of the key.  Maps claim
//            the slot with a compare-and-swap to the CLAIM marker, store the
//            value, fence, then store the key, so a reader that sees the key
//            sees its value; no lock is taken.  An insert that meets a claim
//            in progress where its own key could be going (before the first
//            EMPTY slot of its scan order) reads the bucket again until the
//            claim resolves.  No EMPTY slot on the whole probe sequence:
//            OVERFLOW.
//   find     probes to the key or to a bucket holding EMPTY; takes no lock
//            and never waits (a claim in progress is not yet its key).
//   erase    finds the key and swaps it for a tombstone.
// Per key, the results of concurrent calls are those of some serial order
// of them.  Counters (size) move with one atomic per group of threads that
// finish an operation together.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hc.h"
#include "hc_core.cuh"

namespace hcd {

enum : uint32_t { INSERTED = 0, EXISTS = 1, OVERFLOW = 2, ERASED = 3, NOT_FOUND = 4 };

// The end position: returned by find for an absent key.
constexpr long long END = -1;

// Result of insert (the function form's pair of position and success):
// `slot` is where the key is stored (END on overflow), `status` INSERTED when
// this call stored it, EXISTS when it was there, OVERFLOW when it cannot be
// stored.
struct Inserted {
    long long slot;
    uint32_t status;
};

namespace detail {

using hc::Header;
using hc::View;

// Bounds every wait and retry (claim in progress, side lock held, compare-and-swap lost); a
// correct table never reaches it.
constexpr uint32_t kMaxRetries = hc::kMaxRestarts;

__device__ __forceinline__ unsigned lane_id() {
    unsigned l;
    asm("mov.u32 %0, %%laneid;" : "=r"(l));
    return l;
}

// Counter updates of the threads that reach this point together: one atomic
// per counter per group.
__device__ __forceinline__ void count(Header *h, uint32_t ins, uint32_t del, uint32_t used) {
    const unsigned m = __activemask();
    const uint32_t a = __reduce_add_sync(m, ins);
    const uint32_t d = __reduce_add_sync(m, del);
    const uint32_t u = __reduce_add_sync(m, used);
    if (lane_id() == (unsigned)(__ffs(m) - 1)) {
        const long long net = (long long)a - (long long)d;
        if (net) atomicAdd(&h->live, (unsigned long long)net);
        if (u) atomicAdd(&h->used, (unsigned long long)u);
    }
}

// First set bit of `mask` at or after position `rot`, wrapping around.
template <int SPB>
__device__ __forceinline__ int first_from(uint32_t mask, int rot) {
    constexpr uint32_t ALL = SPB >= 32 ? 0xFFFFFFFFu : ((1u << SPB) - 1u);
    const uint32_t hi = mask & (ALL & ~((1u << rot) - 1u));
    return __ffs(hi ? hi : mask) - 1;
}

// Slots that come before the first set bit of `empty` in the scan order that
// starts at `rot` and wraps around (every slot when `empty` is 0).
template <int SPB>
__device__ __forceinline__ uint32_t before_first(uint32_t empty, int rot) {
    constexpr uint32_t ALL = SPB >= 32 ? 0xFFFFFFFFu : ((1u << SPB) - 1u);
    if (!empty) return ALL;
    const int q = first_from<SPB>(empty, rot);
    const uint32_t from_rot = ALL & ~((1u << rot) - 1u);
    const uint32_t below_q = (1u << q) - 1u;
    return q >= rot ? (from_rot & below_q) : (from_rot | below_q);
}

template <int KIND, int BB>
__device__ __forceinline__ void scan(const View &v, unsigned long long b, typename hc::Traits<KIND>::Key k,
                                     uint32_t &match, uint32_t &empty, uint32_t &claim) {
    using S = hc::Slots<KIND, BB>;
    hc::LaneWords<S::KRB> lw;
    lw.load(hc::bucket_at<BB>(v, b));
    match = 0;
    empty = 0;
    claim = 0;
#pragma unroll
    for (int q = 0; q < S::SPB; ++q) {
        const auto ks = hc::slot_key<KIND, S::KRB>(lw, q);
        match |= (uint32_t)(ks == k) << q;
        empty |= (uint32_t)(ks == hc::Traits<KIND>::EMPTY) << q;
        claim |= (uint32_t)(ks == hc::Traits<KIND>::CLAIM) << q;
    }
}

template <int KIND, int BB>
__device__ __forceinline__ void scan(const View &v, unsigned long long b, typename hc::Traits<KIND>::Key k,
                                     uint32_t &match, uint32_t &empty) {
    uint32_t claim;
    scan<KIND, BB>(v, b, k, match, empty, claim);
}

// Where the stored key equal to CLAIM is (1 + slot position), 0 if none.
__device__ __forceinline__ unsigned long long claim_key_at(const View &v) {
    return *((volatile unsigned long long *)&v.hdr->claim_key_at);
}

// Whether a map insert scanning bucket b from slot `rot` must read it again:
// `claim` holds the slots showing the CLAIM pattern, `empty` the EMPTY ones.
// The stored key equal to CLAIM is not a claim; a claim in progress before
// the first EMPTY slot of the scan order could be an insert of the same key.
// Out of line: claim patterns are rare, and the common path keeps its
// registers.
template <int SPB>
__device__ __noinline__ bool must_wait(const View &v, unsigned long long b, uint32_t claim, uint32_t empty, int rot) {
    const unsigned long long at = claim_key_at(v);
    if (at && (at - 1) / SPB == b) claim &= ~(1u << (int)((at - 1) % SPB));
    return (claim & before_first<SPB>(empty, rot)) != 0;
}

template <int KIND>
__device__ __forceinline__ void store_key(unsigned char *slot, typename hc::Traits<KIND>::Key k) {
    if constexpr (sizeof(k) == 4) atomicExch(reinterpret_cast<unsigned int *>(slot), (unsigned int)k);
    else atomicExch(reinterpret_cast<unsigned long long *>(slot), (unsigned long long)k);
}

// Keys equal to the EMPTY / TOMBSTONE bit patterns live in the header's side
// slots; their positions are nb * SPB + side.
template <int KIND>
__device__ Inserted insert_side(const View &v, int side, unsigned long long val, long long pos) {
    using T = hc::Traits<KIND>;
    Header *h = v.hdr;
    Inserted r{pos, EXISTS};
    uint32_t ins = 0;
    if constexpr (T::MAP) {
        uint32_t tries = 0;
        const uint32_t bit = 1u << side;
        while (true) {
            if (*((volatile unsigned int *)&h->side_present[side])) break;       // present: EXISTS
            if (!(atomicOr(&h->side_lock, bit) & bit)) {
                __threadfence();
                if (!*((volatile unsigned int *)&h->side_present[side])) {
                    *((volatile unsigned long long *)&h->side_val[side]) = val;
                    __threadfence();
                    atomicExch(&h->side_present[side], 1u);
                    r.status = INSERTED;
                    ins = 1;
                }
                __threadfence();
                atomicAnd(&h->side_lock, ~bit);
                break;
            }
            if (++tries > kMaxRetries) {
                atomicOr(&h->err, hc::ERR_PROBE_BOUND);
                r = Inserted{END, OVERFLOW};
                break;
            }
        }
    } else {
        if (atomicCAS(&h->side_present[side], 0u, 1u) == 0u) {
            r.status = INSERTED;
            ins = 1;
        }
    }
    count(h, ins, 0, 0);
    return r;
}

// The key word of slot position pos (a regular slot), read from L2.
template <int KIND, int BB>
__device__ __forceinline__ typename hc::Traits<KIND>::Key slot_word(const View &v, unsigned long long pos) {
    using S = hc::Slots<KIND, BB>;
    const unsigned char *p = S::key(v, pos / S::SPB, (int)(pos % S::SPB));
    return *reinterpret_cast<const volatile typename hc::Traits<KIND>::Key *>(p);
}

// Map insert of the key whose bit pattern equals CLAIM.  Such inserts take
// turns on a header bit, so at most one of them probes at a time; under it
// the header's record says whether the key is stored, and a new one is
// stored in the first EMPTY slot of its scan order: claimed with the
// pattern itself, the value stored, then the record set, which is what makes
// it visible to in-kernel finds and erases.
template <int KIND, int BB>
__device__ __noinline__ Inserted insert_claim_key(const View &v, unsigned long long val) {
    using T = hc::Traits<KIND>;
    using S = hc::Slots<KIND, BB>;
    constexpr int SPB = S::SPB;
    constexpr uint32_t bit = 4u;
    Header *h = v.hdr;
    Inserted r{END, OVERFLOW};
    uint32_t ins = 0, tries = 0;
    bool bound = false;
    while (atomicOr(&h->side_lock, bit) & bit) {
        if (++tries > kMaxRetries) { bound = true; break; }
    }
    if (!bound) {
        __threadfence();
        const unsigned long long at = claim_key_at(v);
        if (at && slot_word<KIND, BB>(v, at - 1) == T::CLAIM) {
            r = Inserted{(long long)(at - 1), EXISTS};
        } else {
            const int rot = hc::slot_rotation<SPB>((unsigned long long)T::CLAIM);
            unsigned long long b = hc::first_bucket(v, (unsigned long long)T::CLAIM);
            for (unsigned long long p = 0; p < v.nb;) {
                uint32_t lm, le;
                scan<KIND, BB>(v, b, T::CLAIM, lm, le);
                if (!le) {
                    b = hc::next_bucket(v, b);
                    ++p;
                    continue;
                }
                const int q = first_from<SPB>(le, rot);
                if (hc::cas_key<KIND>(S::key(v, b, q), T::EMPTY, T::CLAIM) != T::EMPTY) {
                    if (++tries > kMaxRetries) { bound = true; break; }
                    continue;                          // another key took it: read the bucket again
                }
                hc::store_val<KIND, BB>(v, b, q, val);
                __threadfence();                       // the value before the record
                const long long pos = (long long)(b * SPB) + q;
                atomicExch(&h->claim_key_at, (unsigned long long)pos + 1ull);
                r = Inserted{pos, INSERTED};
                ins = 1;
                break;
            }
        }
        __threadfence();
        atomicAnd(&h->side_lock, ~bit);
    }
    if (r.status == OVERFLOW) atomicOr(&h->err, bound ? (hc::ERR_PROBE_BOUND | hc::ERR_OVERFLOW) : hc::ERR_OVERFLOW);
    count(h, ins, 0, ins);
    return r;
}

template <int KIND, int BB>
__device__ Inserted insert(const View &v, typename hc::Traits<KIND>::Key k, unsigned long long val) {
    using T = hc::Traits<KIND>;
    using S = hc::Slots<KIND, BB>;
    constexpr int SPB = S::SPB;
    const int side = hc::side_index<KIND>(k);
    if (side >= 0) return insert_side<KIND>(v, side, val, (long long)(v.nb * SPB) + side);
    if constexpr (T::MAP) {
        if (k == T::CLAIM) return insert_claim_key<KIND, BB>(v, val);
    }
    const int rot = hc::slot_rotation<SPB>((unsigned long long)k);
    unsigned long long b = hc::first_bucket(v, (unsigned long long)k);
    Inserted r{END, OVERFLOW};
    uint32_t ins = 0, retries = 0;
    bool bound = false;
    for (unsigned long long p = 0; p < v.nb;) {
        uint32_t lm, le, lc;
        scan<KIND, BB>(v, b, k, lm, le, lc);
        if (lm) {
            r = Inserted{(long long)(b * SPB) + (__ffs(lm) - 1), EXISTS};
            break;
        }
        if constexpr (T::MAP) {
            // CLAIM patterns: the stored key, or claims in progress; a claim
            // where an insert of this key would also have gone: wait
            if (lc && must_wait<SPB>(v, b, lc, le, rot)) {
                if (++retries > kMaxRetries) { bound = true; break; }
                __nanosleep(64);
                continue;
            }
        }
        if (!le) {
            b = hc::next_bucket(v, b);
            ++p;
            continue;
        }
        const int q = first_from<SPB>(le, rot);
        if constexpr (T::MAP) {
            if (hc::cas_key<KIND>(S::key(v, b, q), T::EMPTY, T::CLAIM) != T::EMPTY) {
                if (++retries > kMaxRetries) { bound = true; break; }
                continue;                              // lost the slot: read the bucket again
            }
            hc::store_val<KIND, BB>(v, b, q, val);
            __threadfence();                           // the value before the key
            store_key<KIND>(S::key(v, b, q), k);
            r = Inserted{(long long)(b * SPB) + q, INSERTED};
            ins = 1;
            break;
        } else {
            const auto old = hc::cas_key<KIND>(S::key(v, b, q), T::EMPTY, k);
            if (old == T::EMPTY) {
                r = Inserted{(long long)(b * SPB) + q, INSERTED};
                ins = 1;
                break;
            }
            if (old == k) {
                r = Inserted{(long long)(b * SPB) + q, EXISTS};
                break;
            }
            // another key took the slot: the same bucket is read again (an
            // equal key can only have gone to this bucket or a later one)
            if (++retries > kMaxRetries) { bound = true; break; }
        }
    }
    if (r.status == OVERFLOW) atomicOr(&v.hdr->err, bound ? (hc::ERR_PROBE_BOUND | hc::ERR_OVERFLOW) : hc::ERR_OVERFLOW);
    count(v.hdr, ins, 0, ins);
    return r;
}

template <int KIND, int BB>
__device__ long long find(const View &v, typename hc::Traits<KIND>::Key k) {
    using T = hc::Traits<KIND>;
    using S = hc::Slots<KIND, BB>;
    constexpr int SPB = S::SPB;
    const int side = hc::side_index<KIND>(k);
    if (side >= 0)
        return *((volatile unsigned int *)&v.hdr->side_present[side]) ? (long long)(v.nb * SPB) + side : END;
    if constexpr (T::MAP) {
        if (k == T::CLAIM) {                           // stored where the header's record says
            const unsigned long long at = claim_key_at(v);
            return (at && slot_word<KIND, BB>(v, at - 1) == T::CLAIM) ? (long long)(at - 1) : END;
        }
    }
    unsigned long long b = hc::first_bucket(v, (unsigned long long)k);
    for (unsigned long long p = 0; p < v.nb; ++p) {
        uint32_t lm, le;
        scan<KIND, BB>(v, b, k, lm, le);
        if (lm) return (long long)(b * SPB) + (__ffs(lm) - 1);
        if (le) return END;
        b = hc::next_bucket(v, b);
    }
    return END;
}

template <int KIND, int BB>
__device__ uint32_t erase(const View &v, typename hc::Traits<KIND>::Key k) {
    using T = hc::Traits<KIND>;
    using S = hc::Slots<KIND, BB>;
    constexpr int SPB = S::SPB;
    uint32_t del = 0;
    const int side = hc::side_index<KIND>(k);
    if (side >= 0) {
        del = atomicCAS(&v.hdr->side_present[side], 1u, 0u) == 1u;
    } else {
        const long long pos = find<KIND, BB>(v, k);
        if (pos != END) {
            const unsigned long long b = (unsigned long long)pos / SPB;
            const int q = (int)((unsigned long long)pos % SPB);
            // a failed swap means a concurrent erase of the same key won
            del = hc::cas_key<KIND>(S::key(v, b, q), k, T::TOMB) == k;
            if constexpr (T::MAP) {
                // the record goes unless a new insert of the key has set it
                if (del && k == T::CLAIM) atomicCAS(&v.hdr->claim_key_at, (unsigned long long)pos + 1ull, 0ull);
            }
        }
    }
    count(v.hdr, 0, del, 0);
    return del ? ERASED : NOT_FOUND;
}

template <int KIND, int BB>
__device__ typename hc::Traits<KIND>::Val value_at(const View &v, long long pos) {
    using T = hc::Traits<KIND>;
    using S = hc::Slots<KIND, BB>;
    __threadfence();                                   // after the load that found the key
    const unsigned long long phys = v.nb * S::SPB;
    if ((unsigned long long)pos >= phys)
        return (typename T::Val) * ((volatile unsigned long long *)&v.hdr->side_val[pos - (long long)phys]);
    return (typename T::Val)hc::load_val<KIND, BB>(v, (unsigned long long)pos / S::SPB, (int)(pos % S::SPB));
}

template <int KIND, int BB>
__device__ typename hc::Traits<KIND>::Key key_at(const View &v, long long pos) {
    using T = hc::Traits<KIND>;
    using S = hc::Slots<KIND, BB>;
    const unsigned long long phys = v.nb * S::SPB;
    if ((unsigned long long)pos >= phys) return pos - (long long)phys == 0 ? T::EMPTY : T::TOMB;
    const unsigned char *p = S::key(v, (unsigned long long)pos / S::SPB, (int)(pos % S::SPB));
    return *reinterpret_cast<const volatile typename T::Key *>(p);
}

}  // namespace detail

// A table of kind KIND (HC_SET_U32, HC_SET_U64, HC_MAP_I64_I32,
// HC_MAP_U64_U64) seen from a kernel.  Keys and values are the bit patterns
// of the kind's types (int64 keys and int32 values as uint64 / uint32).
template <int KIND>
class Table {
public:
    using Key = typename hc::Traits<KIND>::Key;
    using Val = typename hc::Traits<KIND>::Val;
    static constexpr bool is_map = hc::Traits<KIND>::MAP;

    __host__ __device__ explicit Table(const hc_device_view &d) : bb_(d.bucket_bytes) {
        v_.buckets = static_cast<unsigned char *>(d.buckets);
        v_.hdr = static_cast<hc::Header *>(d.header);
        v_.nb = d.nb;
        v_.seed = d.seed;
        v_.hash_mode = d.hash_mode;
        v_.pad_from = d.pad_from;
        v_.rotate = 1;
        v_.reserved = 0;
    }

    // Stores `key` (with `value` for maps) unless it is present.
    __device__ Inserted insert(Key key, Val value = Val()) const {
        switch (bb_) {
            case 32: return detail::insert<KIND, 32>(v_, key, (unsigned long long)value);
            case 64: return detail::insert<KIND, 64>(v_, key, (unsigned long long)value);
            default: return detail::insert<KIND, 128>(v_, key, (unsigned long long)value);
        }
    }
    // Position of `key`, or END.
    __device__ long long find(Key key) const {
        switch (bb_) {
            case 32: return detail::find<KIND, 32>(v_, key);
            case 64: return detail::find<KIND, 64>(v_, key);
            default: return detail::find<KIND, 128>(v_, key);
        }
    }
    __device__ bool contains(Key key) const { return find(key) != END; }
    // ERASED when this call removed `key`, NOT_FOUND otherwise.
    __device__ uint32_t erase(Key key) const {
        switch (bb_) {
            case 32: return detail::erase<KIND, 32>(v_, key);
            case 64: return detail::erase<KIND, 64>(v_, key);
            default: return detail::erase<KIND, 128>(v_, key);
        }
    }
    // The value stored at a position that find or insert returned (maps).
    __device__ Val value(long long pos) const {
        switch (bb_) {
            case 32: return detail::value_at<KIND, 32>(v_, pos);
            case 64: return detail::value_at<KIND, 64>(v_, pos);
            default: return detail::value_at<KIND, 128>(v_, pos);
        }
    }
    // The key stored at a position that find or insert returned.
    __device__ Key key(long long pos) const {
        switch (bb_) {
            case 32: return detail::key_at<KIND, 32>(v_, pos);
            case 64: return detail::key_at<KIND, 64>(v_, pos);
            default: return detail::key_at<KIND, 128>(v_, pos);
        }
    }

    __host__ __device__ int bucket_bytes() const { return bb_; }
    __host__ __device__ const hc::View &view() const { return v_; }

    // Number of positions: every slot of the table, then the two side slots.
    __device__ long long positions() const { return (long long)(v_.nb * (unsigned long long)spb()) + 2; }

    // Whether position `pos` holds a stored key; if so, *k (and *val for maps,
    // when not NULL) receive it.  Meant for ranges over the stored entries while
    // no insert or erase runs on the table.
    __device__ bool entry(long long pos, Key *k, Val *val = nullptr) const {
        using T = hc::Traits<KIND>;
        const unsigned long long phys = v_.nb * (unsigned long long)spb();
        if ((unsigned long long)pos >= phys) {
            const int side = (int)((unsigned long long)pos - phys);
            if (!*((volatile unsigned int *)&v_.hdr->side_present[side])) return false;
            *k = side == 0 ? T::EMPTY : T::TOMB;
            if constexpr (T::MAP) {
                if (val) *val = (Val) * ((volatile unsigned long long *)&v_.hdr->side_val[side]);
            }
            return true;
        }
        const Key key = this->key(pos);
        if (key == T::EMPTY || key == T::TOMB) return false;
        *k = key;
        if constexpr (T::MAP) {
            if (val) *val = value_plain(pos);
        }
        return true;
    }

private:
    __device__ int spb() const {
        switch (bb_) {
            case 32: return hc::Slots<KIND, 32>::SPB;
            case 64: return hc::Slots<KIND, 64>::SPB;
            default: return hc::Slots<KIND, 128>::SPB;
        }
    }
    __device__ Val value_plain(long long pos) const {
        switch (bb_) {
            case 32: return (Val)hc::load_val<KIND, 32>(v_, pos / hc::Slots<KIND, 32>::SPB, (int)(pos % hc::Slots<KIND, 32>::SPB));
            case 64: return (Val)hc::load_val<KIND, 64>(v_, pos / hc::Slots<KIND, 64>::SPB, (int)(pos % hc::Slots<KIND, 64>::SPB));
            default:
                return (Val)hc::load_val<KIND, 128>(v_, pos / hc::Slots<KIND, 128>::SPB,
                                                    (int)(pos % hc::Slots<KIND, 128>::SPB));
        }
    }

    hc::View v_;
    int bb_;
};

namespace detail {

// Keys (and values) of a block tile of J * blockDim.x consecutive slot
// positions: thread t holds positions t, t + blockDim.x, ...; the matches
// of the tile are numbered by a block-wide prefix sum and appended with one
// atomic add on *size.
template <int KIND, int BB, class Pred>
__device__ void copy_if_bb(const View &v, Pred pred, typename hc::Traits<KIND>::Key *keys_out,
                           typename hc::Traits<KIND>::Val *vals_out, unsigned long long cap, unsigned long long *size) {
    using T = hc::Traits<KIND>;
    using Key = typename T::Key;
    using Val = typename T::Val;
    using S = hc::Slots<KIND, BB>;
    constexpr int J = 8;
    __shared__ unsigned warp_sum[32];
    __shared__ unsigned long long tile_base;
    const unsigned lane = lane_id();
    const unsigned warp = threadIdx.x / 32;
    const unsigned nwarps = blockDim.x / 32;
    const unsigned long long phys = v.nb * (unsigned long long)S::SPB;
    const unsigned long long tile = (unsigned long long)blockDim.x * J;
    for (unsigned long long t0 = (unsigned long long)blockIdx.x * tile; t0 < phys; t0 += (unsigned long long)gridDim.x * tile) {
        Key k[J];
        Val val[J];
        uint32_t hit = 0;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const unsigned long long pos = t0 + (unsigned long long)j * blockDim.x + threadIdx.x;
            val[j] = Val();
            if (pos < phys) {
                const unsigned long long b = pos / S::SPB;
                const int q = (int)(pos % S::SPB);
                k[j] = __ldcs(reinterpret_cast<const Key *>(S::key(v, b, q)));
                if (k[j] != T::EMPTY && k[j] != T::TOMB) {
                    if constexpr (T::MAP) val[j] = __ldcs(reinterpret_cast<const Val *>(S::val(v, b, q)));
                    hit |= (uint32_t)pred(k[j], val[j]) << j;
                }
            }
        }
        // exclusive offset of this thread's matches inside the tile
        const unsigned mine = __popc(hit);
        unsigned incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= (unsigned)d) incl += y;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned run = 0;
            for (unsigned w = 0; w < nwarps; ++w) {
                const unsigned c = warp_sum[w];
                warp_sum[w] = run;
                run += c;
            }
            tile_base = run ? atomicAdd(size, (unsigned long long)run) : 0ull;
        }
        __syncthreads();
        unsigned long long at = tile_base + warp_sum[warp] + (incl - mine);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if (hit >> j & 1u) {
                if (at < cap) {
                    keys_out[at] = k[j];
                    if constexpr (T::MAP) {
                        if (vals_out) vals_out[at] = val[j];
                    }
                }
                ++at;
            }
        }
        __syncthreads();                               // warp_sum and tile_base are reused
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {         // the two side slots
        for (int side = 0; side < 2; ++side) {
            if (!*((volatile unsigned int *)&v.hdr->side_present[side])) continue;
            const Key k = side == 0 ? T::EMPTY : T::TOMB;
            const Val val = T::MAP ? (Val) * ((volatile unsigned long long *)&v.hdr->side_val[side]) : Val();
            if (!pred(k, val)) continue;
            const unsigned long long at = atomicAdd(size, 1ull);
            if (at < cap) {
                keys_out[at] = k;
                if constexpr (T::MAP) {
                    if (vals_out) vals_out[at] = val;
                }
            }
        }
    }
}

}  // namespace detail

// Selection over the stored entries (Section 3.6's block selection: a range
// over a container, copied with a predicate through a back inserter into a
// vector).  Appends every stored (key, value) with pred(key, value) true to
// keys_out / vals_out (vals_out may be NULL; sets pass NULL) through *size,
// the output vector's element count: an entry's position is the count before
// it, entries at positions >= cap are counted but not written.  Every thread
// of every block of the calling grid calls it with the same arguments (it
// synchronises the block); blocks are one-dimensional, whole warps, at most
// 1024 threads.  A block walks tiles of 8 * blockDim.x slot positions and
// appends a tile's matches with one atomic add.  No insert or erase may run
// on the table meanwhile.
template <int KIND, class Pred>
__device__ void copy_if(const Table<KIND> &t, Pred pred, typename Table<KIND>::Key *keys_out,
                        typename Table<KIND>::Val *vals_out, unsigned long long cap, unsigned long long *size) {
    switch (t.bucket_bytes()) {
        case 32: detail::copy_if_bb<KIND, 32>(t.view(), pred, keys_out, vals_out, cap, size); break;
        case 64: detail::copy_if_bb<KIND, 64>(t.view(), pred, keys_out, vals_out, cap, size); break;
        default: detail::copy_if_bb<KIND, 128>(t.view(), pred, keys_out, vals_out, cap, size); break;
    }
}

}  // namespace hcd
