// hc_core.cuh -- device side of the GB300 hash containers.
//
// Layout.  A table is nb buckets of BB bytes (32, 64 or 128), aligned to
// their size, so a bucket is one, two or four 32-byte sectors inside one
// 128-byte L2 line.  A bucket holds SPB slots as SPB keys followed, for maps,
// by their SPB values:
//   set<u32>       BB/4 keys          set<u64>  BB/8 keys
//   map<u64,u64>   BB/16 keys + BB/16 values
//   map<i64,i32>   the largest power of two of 12-byte slots that fits
//                  (2, 4 or 8 keys + values, the rest padding)
// On GB300 a random read of any size brings a whole 128-byte line from HBM
// (3.83 DRAM sectors per random 32-byte read, for every load flavour), so the
// cost of an operation is the number of lines it touches: keeping a key and
// its value in one line makes a map lookup or insert touch one line.
// A key slot is EMPTY (all ones), a TOMBSTONE (all ones minus one) or holds a
// key.  The two keys whose bit patterns equal those markers live in two side
// slots of the header (every bit pattern is a valid key: the paper avoids
// placeholder keys, Section 5.1).  Slots past the requested capacity in the
// last bucket are padding: they hold TOMBSTONE and inserts never claim them,
// so a table stores at most `capacity` keys in slots (fixed capacity,
// Section 4).
//
// CLAIM (all ones minus two) is the key pattern an in-kernel map insert
// (include/hc_device.cuh) writes into the EMPTY slot it claims before it
// stores the value and then the key, so that a concurrent reader never sees
// a key without its value.  A stored key with that bit pattern is an
// ordinary key held in a slot; the header records its position (claim_key_at)
// so that in-kernel map inserts tell it from a claim in progress.  Every
// path that stores or erases it in a map keeps that record; range kernels run
// between in-kernel ones and never see a claim in progress.
//
// Probing.  A key hashes to a first bucket; buckets are visited in order,
// wrapping around, at most nb of them.  A group of G = KRB / LB lanes reads the
// bucket's key region (KRB bytes) together, each lane LB bytes (16, 32, 64
// or 128) with vector loads; G = 1 is one thread per key.  The lanes combine
// their findings with __ballot_sync.  Each group may work on KPT keys at once,
// issuing all their bucket loads before examining any.
//
//   insert: stop at the key (EXISTS) or at the first bucket holding an EMPTY
//           slot; claim the first free slot (EMPTY or TOMBSTONE, not padding)
//           seen on the way with a compare-and-swap of the key, then store
//           the value; a lost race restarts the probe.  No free slot in nb
//           buckets gives OVERFLOW, the only failure (Section 4).
//   find:   stop at the key or at a bucket holding an EMPTY slot; no lock
//           (lookups are non-blocking, Section 4).
//   erase:  find, then swap the key for a TOMBSTONE with a compare-and-swap.
// Slots go EMPTY -> key and TOMBSTONE -> key during inserts and key ->
// TOMBSTONE during erases, never back to EMPTY (until clear or rehash); this
// is the invariant that lets a lookup stop at the first bucket holding EMPTY
// and lets equal keys racing in one insert batch end in one slot.
//
// Counters.  The header's live / used counters move by one atomic add per
// warp (__reduce_add_sync of the lanes' counts).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hc {

enum : int { KIND_SET_U32 = 0, KIND_SET_U64 = 1, KIND_MAP_I64_I32 = 2, KIND_MAP_U64_U64 = 3 };
enum : uint32_t { ST_INSERTED = 0, ST_EXISTS = 1, ST_OVERFLOW = 2, ST_ERASED = 3, ST_NOT_FOUND = 4 };
enum : uint32_t { ERR_OVERFLOW = 1u, ERR_PROBE_BOUND = 2u, ERR_DEBUG_BOUNDS = 4u };
enum : int { HASH_MIX64 = 0, HASH_TESCHNER = 1, HASH_TESCHNER_SHORT3 = 2 };

// Restarts of an insert probe after lost compare-and-swap races.  Each lost
// race means another key took a slot, so a correct table never reaches this
// bound; it only keeps every loop finite.
constexpr uint32_t kMaxRestarts = 1u << 16;

// Device-resident table header (256 bytes, in front of the key array).
struct alignas(256) Header {
    unsigned long long live;             // stored keys, side slots included
    unsigned long long used;             // slots that are not EMPTY (keys + tombstones), padding excluded
    unsigned int err;                    // sticky ERR_* bits
    unsigned int side_present[2];        // [0]: all-ones key, [1]: all-ones-minus-one key
    unsigned int side_lock;              // bits 0/1: side slot held by an in-kernel map insert; bit 2: CLAIM-key insert
    unsigned long long side_val[2];
    unsigned long long dump_count;       // output cursor of the dump kernel
    unsigned long long reinserted;       // counter of the rehash kernel
    unsigned long long claim_key_at;     // maps: 1 + slot position of the stored key equal to CLAIM, 0 if none
};
static_assert(sizeof(Header) == 256, "header is one 256-byte block");

// What a kernel needs to reach a table; passed by value (Section 3.7: a
// shallow copy of a device object can be handed to kernels).
struct View {
    unsigned char *buckets;      // nb * BB bytes
    Header *hdr;
    unsigned long long nb;       // buckets
    unsigned long long seed;
    int hash_mode;
    int pad_from;                // slots at positions >= pad_from of the last bucket are padding
    int rotate;                  // inserts scan a bucket from a key-dependent slot (set per call)
    int reserved;
};

template <int KIND> struct Traits;
template <> struct Traits<KIND_SET_U32> {
    using Key = uint32_t;
    using Val = uint32_t;
    static constexpr bool MAP = false;
    static constexpr Key EMPTY = 0xFFFFFFFFu, TOMB = 0xFFFFFFFEu, CLAIM = 0xFFFFFFFDu;
};
template <> struct Traits<KIND_SET_U64> {
    using Key = unsigned long long;
    using Val = unsigned long long;
    static constexpr bool MAP = false;
    static constexpr Key EMPTY = ~0ull, TOMB = ~0ull - 1, CLAIM = ~0ull - 2;
};
template <> struct Traits<KIND_MAP_I64_I32> {
    using Key = unsigned long long;   // int64 keys are handled as bit patterns
    using Val = uint32_t;             // int32 values likewise
    static constexpr bool MAP = true;
    static constexpr Key EMPTY = ~0ull, TOMB = ~0ull - 1, CLAIM = ~0ull - 2;
};
template <> struct Traits<KIND_MAP_U64_U64> {
    using Key = unsigned long long;
    using Val = unsigned long long;
    static constexpr bool MAP = true;
    static constexpr Key EMPTY = ~0ull, TOMB = ~0ull - 1, CLAIM = ~0ull - 2;
};

// ------------------------------------------------------------------ hash ---

// MurmurHash3's 64-bit finaliser (Appleby, public domain).
__device__ __forceinline__ unsigned long long fmix64(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

// Spatial hash of Section 4.1 on a key packing three signed 21-bit block
// coordinates (x | y << 21 | z << 42).  The products are taken in unsigned
// 64-bit wrap-around arithmetic, which is defined for every coordinate.
__device__ __forceinline__ unsigned long long teschner(unsigned long long key) {
    auto coord = [](unsigned long long v) -> unsigned long long {
        long long c = (long long)(v & 0x1FFFFFull);
        c = (c ^ 0x100000ll) - 0x100000ll;  // sign-extend 21 bits
        return (unsigned long long)c;
    };
    unsigned long long x = coord(key), y = coord(key >> 21), z = coord(key >> 42);
    return (x * 73856093ull) ^ (y * 19349669ull) ^ (z * 83492791ull);
}

// The same hash on the paper's own key type, a short3 of signed 16-bit
// coordinates packed as (uint16)x | (uint16)y << 16 | (uint16)z << 32.
__device__ __forceinline__ unsigned long long teschner_short3(unsigned long long key) {
    const unsigned long long x = (unsigned long long)(long long)(short)(key & 0xFFFFull);
    const unsigned long long y = (unsigned long long)(long long)(short)((key >> 16) & 0xFFFFull);
    const unsigned long long z = (unsigned long long)(long long)(short)((key >> 32) & 0xFFFFull);
    return (x * 73856093ull) ^ (y * 19349669ull) ^ (z * 83492791ull);
}

__device__ __forceinline__ unsigned long long first_bucket(const View &v, unsigned long long key) {
    if (v.hash_mode == HASH_TESCHNER) return teschner(key) % v.nb;
    if (v.hash_mode == HASH_TESCHNER_SHORT3) return teschner_short3(key) % v.nb;
    return __umul64hi(fmix64(key ^ v.seed), v.nb);
}

// Key-dependent starting slot of an insert's scan inside a bucket of SPB
// slots (low bits of a 64-bit mix; the bucket index uses the high bits).
template <int SPB>
__device__ __forceinline__ int slot_rotation(unsigned long long key) {
    return (int)(fmix64(key ^ 0x9E3779B97F4A7C15ull) & (unsigned long long)(SPB - 1));
}

__device__ __forceinline__ unsigned long long next_bucket(const View &v, unsigned long long b) {
    ++b;
    return b == v.nb ? 0ull : b;
}

// Debug bounds build (-DHC_DEBUG): an index outside the table, or a key
// range outside the caller's array, records ERR_DEBUG_BOUNDS in the table
// header; a bad bucket or slot is replaced by bucket 0, slot 0, so nothing is
// accessed out of bounds and nothing traps.  The normal build compiles the
// checks away.
__device__ __forceinline__ void debug_bucket(const View &v, unsigned long long &b) {
#ifdef HC_DEBUG
    if (b >= v.nb) {
        atomicOr(&v.hdr->err, ERR_DEBUG_BOUNDS);
        b = 0;
    }
#else
    (void)v;
    (void)b;
#endif
}

__device__ __forceinline__ void debug_range(const View &v, long long first, long long count, long long n) {
#ifdef HC_DEBUG
    if (first < 0 || count < 0 || first + count > n) atomicOr(&v.hdr->err, ERR_DEBUG_BOUNDS);
#else
    (void)v;
    (void)first;
    (void)count;
    (void)n;
#endif
}

// Address of bucket b (checked in the debug build).
template <int BB>
__device__ __forceinline__ unsigned char *bucket_at(const View &v, unsigned long long b) {
    debug_bucket(v, b);
    return v.buckets + b * BB;
}

// --------------------------------------------------------------- memory ---

// One lane's share of a bucket: LB bytes in 32-byte vector loads cached in L2
// only (the slots are shared by all SMs and modified by atomics; an L1 copy
// could be stale after a lost compare-and-swap).
template <int LB> struct LaneWords {
    static_assert(LB == 16 || LB == 32 || LB == 64 || LB == 128, "lane bytes");
    unsigned long long w[LB / 8];
    __device__ __forceinline__ void load(const unsigned char *p) {
        if constexpr (LB == 16) {
            asm volatile("ld.global.cg.v2.u64 {%0,%1}, [%2];" : "=l"(w[0]), "=l"(w[1]) : "l"(p));
        } else {
#pragma unroll
            for (int q = 0; q < LB / 32; ++q)
                asm volatile("ld.global.cg.v4.u64 {%0,%1,%2,%3}, [%4];"
                             : "=l"(w[4 * q]), "=l"(w[4 * q + 1]), "=l"(w[4 * q + 2]), "=l"(w[4 * q + 3])
                             : "l"(p + 32 * q));
        }
    }
};

template <int KIND, int LB>
__device__ __forceinline__ typename Traits<KIND>::Key slot_key(const LaneWords<LB> &lw, int s) {
    using Key = typename Traits<KIND>::Key;
    if constexpr (sizeof(Key) == 4) return (Key)(lw.w[s >> 1] >> ((s & 1) * 32));
    else return lw.w[s];
}

// 32- or 64-bit compare-and-swap on a key slot.
template <int KIND>
__device__ __forceinline__ typename Traits<KIND>::Key cas_key(unsigned char *slot, typename Traits<KIND>::Key expect,
                                                             typename Traits<KIND>::Key desired) {
    if constexpr (sizeof(typename Traits<KIND>::Key) == 4)
        return atomicCAS(reinterpret_cast<unsigned int *>(slot), expect, desired);
    else
        return atomicCAS(reinterpret_cast<unsigned long long *>(slot), expect, desired);
}

// Where slot s of bucket b keeps its key and value (see the layout above).
template <int KIND, int BB> struct Slots {
    using T = Traits<KIND>;
    static constexpr int KB = (int)sizeof(typename T::Key);
    static constexpr int VB = T::MAP ? (int)sizeof(typename T::Val) : 0;
    static constexpr int fit(int n) { return n >= 16 ? 16 : n >= 8 ? 8 : n >= 4 ? 4 : n >= 2 ? 2 : 1; }
    static constexpr int SPB = T::MAP ? fit(BB / (KB + VB)) : BB / KB;   // slots per bucket
    static constexpr int KRB = SPB * KB;                                 // key region bytes
    static_assert(KRB + SPB * VB <= BB, "bucket overflow");
    __device__ __forceinline__ static unsigned char *key(const View &v, unsigned long long b, int s) {
        check(v, b, s);
        return v.buckets + b * BB + (size_t)s * KB;
    }
    __device__ __forceinline__ static unsigned char *val(const View &v, unsigned long long b, int s) {
        check(v, b, s);
        return v.buckets + b * BB + KRB + (size_t)s * VB;
    }
    __device__ __forceinline__ static void check(const View &v, unsigned long long &b, int &s) {
        debug_bucket(v, b);
#ifdef HC_DEBUG
        if (s < 0 || s >= SPB) {
            atomicOr(&v.hdr->err, ERR_DEBUG_BOUNDS);
            s = 0;
        }
#endif
    }
};

template <int KIND, int BB>
__device__ __forceinline__ void store_val(const View &v, unsigned long long b, int s, unsigned long long val) {
    using T = Traits<KIND>;
    if constexpr (T::MAP) *reinterpret_cast<typename T::Val *>(Slots<KIND, BB>::val(v, b, s)) = (typename T::Val)val;
}

template <int KIND, int BB>
__device__ __forceinline__ unsigned long long load_val(const View &v, unsigned long long b, int s) {
    using T = Traits<KIND>;
    if constexpr (T::MAP)
        return (unsigned long long)__ldcg(reinterpret_cast<const typename T::Val *>(Slots<KIND, BB>::val(v, b, s)));
    else return 0ull;
}

// Streaming loads/stores of the caller's arrays (evict-first: they are read
// or written once, and should not push table buckets out of L2).
template <class T> __device__ __forceinline__ T ld_stream(const T *p) { return __ldcs(p); }
__device__ __forceinline__ void st_stream(uint8_t *p, uint8_t v) { __stcs(reinterpret_cast<signed char *>(p), (signed char)v); }
__device__ __forceinline__ void st_stream(uint32_t *p, uint32_t v) { __stcs(reinterpret_cast<unsigned int *>(p), v); }
__device__ __forceinline__ void st_stream(unsigned long long *p, unsigned long long v) { __stcs(p, v); }

// ------------------------------------------------------------ group ops ---

// A group is G consecutive lanes of a warp (G = 1, 2 or 4).
template <int G> struct Group {
    unsigned mask;   // lanes of this group
    int base;        // first lane of the group
    int sub;         // this lane's index inside the group
    __device__ __forceinline__ Group() {
        const int lane = threadIdx.x & 31;
        base = lane & ~(G - 1);
        sub = lane & (G - 1);
        mask = ((1u << G) - 1u) << base;
    }
    // Bits [0, G) = pred of the group's lanes.
    __device__ __forceinline__ unsigned ballot(bool pred) const {
        if constexpr (G == 1) return pred ? 1u : 0u;
        else return (__ballot_sync(mask, pred) >> base) & ((1u << G) - 1u);
    }
    template <class T> __device__ __forceinline__ T bcast(T v, int src_sub) const {
        if constexpr (G == 1) return v;
        else return __shfl_sync(mask, v, base + src_sub);
    }
};

// Slot-layout constants of a (kind, bucket, lane) combination.
// FULL (maps, LB == BB): one thread reads the whole bucket, keys and values,
// so a lookup that finds its key has the value without a second load.
template <int KIND, int BB, int LB> struct Layout {
    using S = Slots<KIND, BB>;
    static constexpr int KB = S::KB;
    static constexpr int SPB = S::SPB;                       // slots per bucket
    static constexpr bool FULL = Traits<KIND>::MAP && LB == BB;
    static constexpr int G = FULL ? 1 : S::KRB / LB;         // lanes per key
    static constexpr int SPL = FULL ? SPB : LB / KB;         // key slots per lane (<= 32)
    static constexpr uint32_t ALL = SPL == 32 ? 0xffffffffu : ((1u << SPL) - 1u);
    static_assert(FULL || (LB <= S::KRB && S::KRB % LB == 0), "lane bytes must divide the key region");
    static_assert(SPL <= 32, "lane masks are 32 bits");
};

// Value of slot s from a FULL lane's words (values follow the KRB key bytes).
template <int KIND, int BB, int LB>
__device__ __forceinline__ unsigned long long word_val(const LaneWords<LB> &lw, int s) {
    using T = Traits<KIND>;
    constexpr int KRB = Slots<KIND, BB>::KRB;
    if constexpr (sizeof(typename T::Val) == 8) return lw.w[KRB / 8 + s];
    else return (uint32_t)(lw.w[(KRB + 4 * s) / 8] >> (((KRB + 4 * s) % 8) * 8));
}

// Keys handled by a warp per tile: (32 / G) groups of KPT keys.
template <int KIND, int BB, int LB, int KPT> struct Shape {
    static constexpr int G = Layout<KIND, BB, LB>::G;
    static constexpr int GROUPS = 32 / G;
    static constexpr int TILE = GROUPS * KPT;
};

// Load the KPT keys of this group (tile position `first`), vectorised when the
// whole run is inside [0, n) and aligned.
template <int KPT, class K>
__device__ __forceinline__ void load_keys(const K *keys, long long first, long long n, K (&k)[KPT], uint32_t &valid) {
    valid = 0;
    if constexpr (KPT * sizeof(K) >= 8) {
        constexpr int VB = KPT * sizeof(K) >= 16 ? 16 : 8;
        const bool vec = first + KPT <= n &&
                         ((reinterpret_cast<uintptr_t>(keys + first) & (VB - 1)) == 0);
        if (vec) {
            if constexpr (VB == 16) {
#pragma unroll
                for (int q = 0; q < (int)(KPT * sizeof(K)) / 16; ++q) {
                    uint4 u = __ldcs(reinterpret_cast<const uint4 *>(keys + first) + q);
                    K tmp[16 / sizeof(K)];
                    memcpy(tmp, &u, 16);
#pragma unroll
                    for (int e = 0; e < (int)(16 / sizeof(K)); ++e) k[q * (16 / sizeof(K)) + e] = tmp[e];
                }
            } else {
                uint2 u = __ldcs(reinterpret_cast<const uint2 *>(keys + first));
                memcpy(&k[0], &u, 8);
            }
            valid = (1u << KPT) - 1u;
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        if (first + j < n) {
            k[j] = ld_stream(keys + first + j);
            valid |= 1u << j;
        } else {
            k[j] = 0;
        }
    }
}

template <int KIND>
__device__ __forceinline__ int side_index(typename Traits<KIND>::Key k) {
    using T = Traits<KIND>;
    return k == T::EMPTY ? 0 : (k == T::TOMB ? 1 : -1);
}

// The header's record of a stored key equal to CLAIM (maps): called when a
// range or rehash kernel has stored key k at slot position pos, or erased it
// (pos < 0).  No in-kernel insert runs meanwhile.
template <int KIND>
__device__ __forceinline__ void note_claim_key(Header *h, typename Traits<KIND>::Key k, long long pos) {
    using T = Traits<KIND>;
    if constexpr (T::MAP) {
        if (k == T::CLAIM) h->claim_key_at = pos < 0 ? 0ull : (unsigned long long)pos + 1ull;
    } else {
        (void)h;
        (void)k;
        (void)pos;
    }
}

// Per-key results of a tile before they are written.
template <int KPT> struct TileResult {
    uint32_t st[KPT];
    unsigned long long val[KPT];
};

// Duplicate folding inside a warp (__match_any_sync over the valid keys of
// slot j of every group).  leader[j] = the lane whose group leads key j, or -1
// if this lane's group leads.  All 32 lanes must call it.
template <int KIND, int G, int KPT>
__device__ __forceinline__ void fold_duplicates(const typename Traits<KIND>::Key (&k)[KPT], uint32_t valid,
                                                int (&leader)[KPT]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        const bool v = (valid >> j) & 1u;
        const unsigned act = __ballot_sync(0xffffffffu, v);
        leader[j] = -1;
        if (v) {
            const unsigned peers = __match_any_sync(act, k[j]);
            const int first = __ffs(peers) - 1;
            // lanes of one group share a key, so the lowest peer lane is in
            // the leading group; a lane leads if that lane is in its group
            if ((first & ~(G - 1)) != (lane & ~(G - 1))) leader[j] = first;
        }
    }
}

// Slots of this lane that are not padding in bucket b (padding exists only in
// the last bucket).
template <int KIND, int BB, int LB>
__device__ __forceinline__ uint32_t claimable(const View &v, unsigned long long b, int sub) {
    using Lay = Layout<KIND, BB, LB>;
    if (b != v.nb - 1) return Lay::ALL;
    const int lim = v.pad_from - sub * Lay::SPL;
    if (lim >= Lay::SPL) return Lay::ALL;
    return lim <= 0 ? 0u : ((1u << lim) - 1u);
}

// ---------------------------------------------------------- insert core ---

template <int KIND, int BB, int LB, int KPT>
__device__ __forceinline__ void insert_group(const View &v, const typename Traits<KIND>::Key (&k)[KPT],
                                             const unsigned long long (&val)[KPT], uint32_t todo,
                                             TileResult<KPT> &res, uint32_t &n_ins, uint32_t &n_new_slot) {
    using T = Traits<KIND>;
    using Key = typename T::Key;
    using Lay = Layout<KIND, BB, LB>;
    constexpr int G = Lay::G;
    constexpr int SPL = Lay::SPL;
    const Group<G> grp;

    unsigned long long b[KPT], b0[KPT], ffb[KPT];
    uint32_t probes[KPT], restarts[KPT], ffs_slot[KPT];
    bool ff_empty[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        b0[j] = b[j] = (todo >> j & 1u) ? first_bucket(v, (unsigned long long)k[j]) : 0ull;
        probes[j] = 0;
        restarts[j] = 0;
        ffb[j] = ~0ull;
        ffs_slot[j] = 0;
        ff_empty[j] = false;
    }
    uint32_t active = todo;
    while (active) {
        LaneWords<LB> lw[KPT];
#pragma unroll
        for (int j = 0; j < KPT; ++j)
            if (active >> j & 1u) lw[j].load(bucket_at<BB>(v, b[j]) + grp.sub * LB);
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            if (!(active >> j & 1u)) continue;
            uint32_t lm = 0, le = 0, lt = 0;
#pragma unroll
            for (int s = 0; s < SPL; ++s) {
                const Key ks = slot_key<KIND, LB>(lw[j], s);
                lm |= (uint32_t)(ks == k[j]) << s;
                le |= (uint32_t)(ks == T::EMPTY) << s;
                lt |= (uint32_t)(ks == T::TOMB) << s;
            }
            if (grp.ballot(lm != 0)) {           // already stored
                res.st[j] = ST_EXISTS;
                active &= ~(1u << j);
                continue;
            }
            const unsigned ge = grp.ballot(le != 0);
            if (ffb[j] == ~0ull) {               // remember the first free slot
                // With v.rotate, slots are scanned in an order rotated by a
                // key-dependent offset: every inserter of one key follows the
                // same order (so equal keys still meet in one slot), while
                // different keys aiming at one bucket spread over its free
                // slots instead of all racing for the lowest one.  The host
                // turns it on when a call carries more keys than the table
                // has buckets (several inserters per bucket).
                lt &= claimable<KIND, BB, LB>(v, b[j], grp.sub);
                const uint32_t lf = le | lt;
                const int rot = v.rotate ? slot_rotation<Lay::SPB>(k[j]) : 0;
                const int lo = rot - grp.sub * SPL;          // this lane's first slot at or after rot
                const uint32_t at_or_after = lo <= 0 ? Lay::ALL : (lo >= SPL ? 0u : (Lay::ALL & ~((1u << lo) - 1u)));
                const uint32_t f_hi = lf & at_or_after;
                const unsigned gh = grp.ballot(f_hi != 0);
                const unsigned gf = gh ? gh : grp.ballot(lf != 0);
                if (gf) {
                    const int owner = __ffs(gf) - 1;
                    const uint32_t pick = grp.bcast(gh ? f_hi : lf, owner);
                    const uint32_t lemp = grp.bcast(le, owner);
                    const int s = __ffs(pick) - 1;
                    ffb[j] = b[j];
                    ffs_slot[j] = owner * SPL + s;
                    ff_empty[j] = (lemp >> s) & 1u;
                }
            }
            bool claim = ge != 0;
            if (!claim) {
                ++probes[j];
                if (probes[j] >= v.nb) {
                    if (ffb[j] == ~0ull) {       // no free slot anywhere
                        res.st[j] = ST_OVERFLOW;
                        active &= ~(1u << j);
                        continue;
                    }
                    claim = true;                // only tombstones were free
                } else {
                    b[j] = next_bucket(v, b[j]);
                    continue;
                }
            }
            // claim the first free slot seen on this probe
            const int owner = ffs_slot[j] / SPL;
            const Key expect = ff_empty[j] ? T::EMPTY : T::TOMB;
            Key old = expect;
            if (grp.sub == owner) {
                old = cas_key<KIND>(Slots<KIND, BB>::key(v, ffb[j], ffs_slot[j]), expect, k[j]);
                if (old == expect) {
                    store_val<KIND, BB>(v, ffb[j], ffs_slot[j], val[j]);
                    note_claim_key<KIND>(v.hdr, k[j], (long long)(ffb[j] * Lay::SPB) + ffs_slot[j]);
                }
            }
            old = grp.bcast(old, owner);
            if (old == expect) {
                res.st[j] = ST_INSERTED;
                if (grp.sub == 0) {
                    ++n_ins;
                    n_new_slot += ff_empty[j] ? 1u : 0u;
                }
                active &= ~(1u << j);
            } else if (old == k[j]) {
                res.st[j] = ST_EXISTS;           // an equal key won the race
                active &= ~(1u << j);
            } else if (++restarts[j] > kMaxRestarts) {
                if (grp.sub == 0) atomicOr(&v.hdr->err, ERR_PROBE_BOUND);
                res.st[j] = ST_OVERFLOW;
                active &= ~(1u << j);
            } else {                             // lost the slot to another key
                b[j] = b0[j];
                probes[j] = 0;
                ffb[j] = ~0ull;
            }
        }
    }
}

// ------------------------------------------------------------ find core ---

template <int KIND, int BB, int LB, int KPT>
__device__ __forceinline__ void find_group(const View &v, const typename Traits<KIND>::Key (&k)[KPT], uint32_t todo,
                                           TileResult<KPT> &res) {
    using T = Traits<KIND>;
    using Key = typename T::Key;
    using Lay = Layout<KIND, BB, LB>;
    constexpr int G = Lay::G;
    constexpr int SPL = Lay::SPL;
    const Group<G> grp;

    unsigned long long b[KPT];
    uint32_t probes[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        b[j] = (todo >> j & 1u) ? first_bucket(v, (unsigned long long)k[j]) : 0ull;
        probes[j] = 0;
    }
    uint32_t active = todo;
    while (active) {
        LaneWords<LB> lw[KPT];
#pragma unroll
        for (int j = 0; j < KPT; ++j)
            if (active >> j & 1u) lw[j].load(bucket_at<BB>(v, b[j]) + grp.sub * LB);
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            if (!(active >> j & 1u)) continue;
            uint32_t lm = 0, le = 0;
#pragma unroll
            for (int s = 0; s < SPL; ++s) {
                const Key ks = slot_key<KIND, LB>(lw[j], s);
                lm |= (uint32_t)(ks == k[j]) << s;
                le |= (uint32_t)(ks == T::EMPTY) << s;
            }
            const unsigned gm = grp.ballot(lm != 0);
            if (gm) {
                const int owner = __ffs(gm) - 1;
                unsigned long long val = 0;
                if constexpr (T::MAP) {
                    if constexpr (Lay::FULL) val = word_val<KIND, BB, LB>(lw[j], __ffs(lm) - 1);
                    else if (grp.sub == owner) val = load_val<KIND, BB>(v, b[j], owner * SPL + (__ffs(lm) - 1));
                    val = grp.bcast(val, owner);
                }
                res.st[j] = 1;
                res.val[j] = val;
                active &= ~(1u << j);
            } else if (grp.ballot(le != 0) || ++probes[j] >= v.nb) {
                res.st[j] = 0;
                res.val[j] = 0;
                active &= ~(1u << j);
            } else {
                b[j] = next_bucket(v, b[j]);
            }
        }
    }
}

// ----------------------------------------------------------- erase core ---

template <int KIND, int BB, int LB, int KPT>
__device__ __forceinline__ void erase_group(const View &v, const typename Traits<KIND>::Key (&k)[KPT], uint32_t todo,
                                            TileResult<KPT> &res, uint32_t &n_del) {
    using T = Traits<KIND>;
    using Key = typename T::Key;
    using Lay = Layout<KIND, BB, LB>;
    constexpr int G = Lay::G;
    constexpr int SPL = Lay::SPL;
    const Group<G> grp;

    unsigned long long b[KPT];
    uint32_t probes[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        b[j] = (todo >> j & 1u) ? first_bucket(v, (unsigned long long)k[j]) : 0ull;
        probes[j] = 0;
    }
    uint32_t active = todo;
    while (active) {
        LaneWords<LB> lw[KPT];
#pragma unroll
        for (int j = 0; j < KPT; ++j)
            if (active >> j & 1u) lw[j].load(bucket_at<BB>(v, b[j]) + grp.sub * LB);
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            if (!(active >> j & 1u)) continue;
            uint32_t lm = 0, le = 0;
#pragma unroll
            for (int s = 0; s < SPL; ++s) {
                const Key ks = slot_key<KIND, LB>(lw[j], s);
                lm |= (uint32_t)(ks == k[j]) << s;
                le |= (uint32_t)(ks == T::EMPTY) << s;
            }
            const unsigned gm = grp.ballot(lm != 0);
            if (gm) {
                const int owner = __ffs(gm) - 1;
                Key old = T::TOMB;
                if (grp.sub == owner) {
                    old = cas_key<KIND>(Slots<KIND, BB>::key(v, b[j], owner * SPL + (__ffs(lm) - 1)), k[j], T::TOMB);
                    if (old == k[j]) note_claim_key<KIND>(v.hdr, k[j], -1);
                }
                old = grp.bcast(old, owner);
                // a failed swap means an equal key in this batch erased it first
                res.st[j] = old == k[j] ? ST_ERASED : ST_NOT_FOUND;
                if (old == k[j] && grp.sub == 0) ++n_del;
                active &= ~(1u << j);
            } else if (grp.ballot(le != 0) || ++probes[j] >= v.nb) {
                res.st[j] = ST_NOT_FOUND;
                active &= ~(1u << j);
            } else {
                b[j] = next_bucket(v, b[j]);
            }
        }
    }
}

// ------------------------------------------------------------ warp tiles ---
// One warp processes keys [tile_base, tile_base + TILE) of a call.  The keys
// (and values, skip flags) of a tile are loaded into a TileIn first, so a
// persistent kernel can load the next tile while the current one probes.
// These are shared by the range kernels and the batched persistent kernel.

template <class V> __device__ __forceinline__ unsigned long long widen(V x) { return (unsigned long long)x; }

template <int KIND, int KPT> struct TileIn {
    typename Traits<KIND>::Key k[KPT];
    unsigned long long val[KPT];
    uint32_t valid;     // keys inside [0, n)
    uint32_t present;   // keys a preceding find reported as stored (skip flags)
};

// First key index of this lane's group in a tile.
template <int KIND, int BB, int LB, int KPT>
__device__ __forceinline__ long long group_first(long long tile_base) {
    return tile_base + (long long)((threadIdx.x & 31) / Shape<KIND, BB, LB, KPT>::G) * KPT;
}

template <int KIND, int KPT>
__device__ __forceinline__ void load_tile(TileIn<KIND, KPT> &in, const typename Traits<KIND>::Key *keys,
                                          const typename Traits<KIND>::Val *vals, const uint8_t *skip, long long first,
                                          long long n) {
    using T = Traits<KIND>;
    load_keys<KPT>(keys, first, n, in.k, in.valid);
    in.present = 0;
    if (skip) {
#pragma unroll
        for (int j = 0; j < KPT; ++j)
            if ((in.valid >> j & 1u) && ld_stream(skip + first + j)) in.present |= 1u << j;
    }
#pragma unroll
    for (int j = 0; j < KPT; ++j)
        in.val[j] = (T::MAP && vals && (in.valid >> j & 1u) && !(in.present >> j & 1u))
                        ? widen(ld_stream(vals + first + j)) : 0ull;
}

// Per-thread counts of an insert or erase, added to the header by flush_counts.
struct Counts {
    uint32_t ins = 0, new_slot = 0, del = 0, over = 0;
};

// One atomic per warp per counter.  All 32 lanes must call it.
__device__ __forceinline__ void flush_counts(const View &v, Counts &c) {
    __syncwarp();
    const uint32_t w_ins = __reduce_add_sync(0xffffffffu, c.ins);
    const uint32_t w_new = __reduce_add_sync(0xffffffffu, c.new_slot);
    const uint32_t w_del = __reduce_add_sync(0xffffffffu, c.del);
    const uint32_t w_over = __reduce_or_sync(0xffffffffu, c.over);
    if ((threadIdx.x & 31) == 0) {
        const long long d = (long long)w_ins - (long long)w_del;
        if (d) atomicAdd(&v.hdr->live, (unsigned long long)d);
        if (w_new) atomicAdd(&v.hdr->used, (unsigned long long)w_new);
        if (w_over) atomicOr(&v.hdr->err, ERR_OVERFLOW);
    }
    c = Counts();
}

template <int KIND, int BB, int LB, int KPT>
__device__ __forceinline__ void insert_tile(const View &v, const TileIn<KIND, KPT> &in, long long first,
                                            uint8_t *status, bool fold, Counts &cnt) {
    using T = Traits<KIND>;
    using S = Shape<KIND, BB, LB, KPT>;
    const int lane = threadIdx.x & 31;
    const bool lead_lane = (lane & (S::G - 1)) == 0;

    int leader[KPT];
    if (fold) fold_duplicates<KIND, S::G, KPT>(in.k, in.valid, leader);
    else {
#pragma unroll
        for (int j = 0; j < KPT; ++j) leader[j] = -1;
    }

    TileResult<KPT> res;
    uint32_t todo = 0, n_ins = 0, n_new = 0;
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        res.st[j] = ST_EXISTS;
        if (!(in.valid >> j & 1u) || leader[j] >= 0 || (in.present >> j & 1u)) continue;
        const int side = side_index<KIND>(in.k[j]);
        if (side >= 0) {                         // key equal to a marker: side slot
            uint32_t won = 0;
            if (lead_lane) {
                won = atomicCAS(&v.hdr->side_present[side], 0u, 1u) == 0u;
                if (won) v.hdr->side_val[side] = in.val[j];
                n_ins += won;
            }
            res.st[j] = Group<S::G>().bcast(won, 0) ? ST_INSERTED : ST_EXISTS;
            continue;
        }
        todo |= 1u << j;
    }
    insert_group<KIND, BB, LB, KPT>(v, in.k, in.val, todo, res, n_ins, n_new);

    if (fold) {
        __syncwarp();
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            const uint32_t ls = __shfl_sync(0xffffffffu, res.st[j], leader[j] < 0 ? lane : leader[j]);
            if (leader[j] >= 0) res.st[j] = ls == ST_OVERFLOW ? ST_OVERFLOW : ST_EXISTS;
        }
    }
    if (lead_lane) {
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            if (!(in.valid >> j & 1u)) continue;
            cnt.over |= res.st[j] == ST_OVERFLOW;
            if (status) st_stream(status + first + j, (uint8_t)res.st[j]);
        }
    }
    cnt.ins += n_ins;
    cnt.new_slot += n_new;
}

template <int KIND, int BB, int LB, int KPT>
__device__ __forceinline__ void find_tile(const View &v, const TileIn<KIND, KPT> &in, long long first, uint8_t *found,
                                          typename Traits<KIND>::Val *vals_out) {
    using T = Traits<KIND>;
    using S = Shape<KIND, BB, LB, KPT>;
    const bool lead_lane = ((threadIdx.x & 31) & (S::G - 1)) == 0;
    TileResult<KPT> res;
    uint32_t todo = 0;
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        res.st[j] = 0;
        res.val[j] = 0;
        if (!(in.valid >> j & 1u)) continue;
        const int side = side_index<KIND>(in.k[j]);
        if (side >= 0) {
            res.st[j] = *((volatile unsigned int *)&v.hdr->side_present[side]) ? 1u : 0u;
            res.val[j] = res.st[j] ? *((volatile unsigned long long *)&v.hdr->side_val[side]) : 0ull;
            continue;
        }
        todo |= 1u << j;
    }
    find_group<KIND, BB, LB, KPT>(v, in.k, todo, res);
    if (lead_lane) {
#pragma unroll
        for (int j = 0; j < KPT; ++j) {
            if (!(in.valid >> j & 1u)) continue;
            if (found) st_stream(found + first + j, (uint8_t)res.st[j]);
            if constexpr (T::MAP) {
                if (vals_out) st_stream(vals_out + first + j, (typename T::Val)res.val[j]);
            }
        }
    }
}

template <int KIND, int BB, int LB, int KPT>
__device__ __forceinline__ void erase_tile(const View &v, const TileIn<KIND, KPT> &in, long long first,
                                           uint8_t *status, bool fold, Counts &cnt) {
    using S = Shape<KIND, BB, LB, KPT>;
    const bool lead_lane = ((threadIdx.x & 31) & (S::G - 1)) == 0;
    int leader[KPT];
    if (fold) fold_duplicates<KIND, S::G, KPT>(in.k, in.valid, leader);
    else {
#pragma unroll
        for (int j = 0; j < KPT; ++j) leader[j] = -1;
    }
    TileResult<KPT> res;
    uint32_t todo = 0, n_del = 0;
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
        res.st[j] = ST_NOT_FOUND;
        if (!(in.valid >> j & 1u) || leader[j] >= 0) continue;
        const int side = side_index<KIND>(in.k[j]);
        if (side >= 0) {
            uint32_t won = 0;
            if (lead_lane) {
                won = atomicCAS(&v.hdr->side_present[side], 1u, 0u) == 1u;
                n_del += won;
            }
            res.st[j] = Group<S::G>().bcast(won, 0) ? ST_ERASED : ST_NOT_FOUND;
            continue;
        }
        todo |= 1u << j;
    }
    erase_group<KIND, BB, LB, KPT>(v, in.k, todo, res, n_del);
    if (lead_lane && status) {
#pragma unroll
        for (int j = 0; j < KPT; ++j)
            if (in.valid >> j & 1u) st_stream(status + first + j, (uint8_t)res.st[j]);
    }
    cnt.del += n_del;
}

// The keys [k0, k1) of one call processed by one warp, tile after tile, with
// the next tile's inputs loaded before the current tile probes.  Used by the
// range kernels (one warp-strided sweep over the call) and by the batched
// kernel (one chunk).  OP: 0 insert, 1 find, 2 erase.
template <int KIND, int BB, int LB, int KPT, int OP>
__device__ __forceinline__ void run_tiles(const View &v, const typename Traits<KIND>::Key *keys,
                                          const typename Traits<KIND>::Val *vals, const uint8_t *skip, uint8_t *out,
                                          typename Traits<KIND>::Val *vals_out, long long n, long long t0,
                                          long long t_end, long long t_step, bool fold, Counts &cnt) {
    constexpr int TILE = Shape<KIND, BB, LB, KPT>::TILE;
    if (t0 >= t_end) return;
    TileIn<KIND, KPT> cur, nxt;
    long long first = group_first<KIND, BB, LB, KPT>(t0 * TILE);
    load_tile<KIND, KPT>(cur, keys, OP == 0 ? vals : nullptr, OP == 0 ? skip : nullptr, first, n);
    for (long long t = t0; t < t_end; t += t_step) {
        const long long tn = t + t_step;
        const long long first_n = group_first<KIND, BB, LB, KPT>(tn * TILE);
        if (tn < t_end) load_tile<KIND, KPT>(nxt, keys, OP == 0 ? vals : nullptr, OP == 0 ? skip : nullptr, first_n, n);
        if constexpr (OP == 0) insert_tile<KIND, BB, LB, KPT>(v, cur, first, out, fold, cnt);
        else if constexpr (OP == 1) find_tile<KIND, BB, LB, KPT>(v, cur, first, out, vals_out);
        else erase_tile<KIND, BB, LB, KPT>(v, cur, first, out, fold, cnt);
        cur = nxt;
        first = first_n;
    }
}

}  // namespace hc
