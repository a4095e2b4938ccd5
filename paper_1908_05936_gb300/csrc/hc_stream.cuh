// hc_stream.cuh -- the streaming range kernels: a block stages its chunk of
// keys (and values) in shared memory with coalesced 16-byte loads, so the key
// load leaves each key's chain of dependent reads.  Every thread then keeps S
// probes in flight and refills a slot from the chunk as soon as its probe
// finishes (instead of moving its keys in lock-step rounds); a key is hashed
// when its slot takes it, while the other slots' reads are in flight.
// Results go to shared memory and leave in coalesced stores.  One thread per
// key, reading the bucket's key region (KRB bytes) per probe.
#pragma once

#include "hc_core.cuh"

// Minimum resident 256-thread blocks per SM requested from the compiler
// (__launch_bounds__), i.e. a register cap of 65536 / (256 * MINB) per
// thread; build options.
#ifndef HC_STREAM_FIND_MINB
#define HC_STREAM_FIND_MINB 1
#endif
#ifndef HC_STREAM_INSERT_MINB
#define HC_STREAM_INSERT_MINB 1
#endif
#ifndef HC_STREAM_ERASE_MINB
#define HC_STREAM_ERASE_MINB 1
#endif

// Lookups read buckets through L1 (the read-only path) when 1: a lookup
// never runs together with a modifying call on its table, so the line a
// probe brings into L1 is still valid when a matching key's value is read
// from it right after.  0: L2 only, as the modifying kernels read.
#ifndef HC_FIND_L1
#define HC_FIND_L1 0
#endif

namespace hc {

// The staging of one array of a block chunk (m <= blockDim.x * KPT elements)
// into shared memory, in two steps so that a thread issues the loads of all
// its pieces of every staged array before it stores any: load() reads
// 16-byte pieces tid, tid + nt, ... when src is 16-byte aligned (element by
// element otherwise, and for a tail shorter than 16 bytes) into registers;
// store() writes them to dst (shared, 16-byte aligned), `map` applied to
// every element on the way (the skip flags become result bytes).
template <class T, int KPT>
struct Stage {
    static constexpr int E = 16 / (int)sizeof(T);          // elements per 16-byte piece
    static constexpr int J = (KPT + E - 1) / E;            // pieces per thread
    uint4 piece[J];
    T elem[KPT];
    bool vec;

    __device__ __forceinline__ void load(const T *src, int m) {
        const int nt = blockDim.x, tid = threadIdx.x;
        vec = (reinterpret_cast<uintptr_t>(src) & 15) == 0;
        if (vec) {
            const int nv = m / E;
            const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int u = tid + j * nt;
                if (u < nv) piece[j] = __ldcs(s4 + u);
            }
            const int i = nv * E + tid;                     // the tail: fewer than E elements
            if (i < m) elem[0] = ld_stream(src + i);
        } else {
#pragma unroll
            for (int j = 0; j < KPT; ++j) {
                const int i = tid + j * nt;
                if (i < m) elem[j] = ld_stream(src + i);
            }
        }
    }

    template <class F>
    __device__ __forceinline__ void store(T *dst, int m, F map) const {
        const int nt = blockDim.x, tid = threadIdx.x;
        if (vec) {
            const int nv = m / E;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                const int u = tid + j * nt;
                if (u < nv) {
                    T t[E];
                    memcpy(t, &piece[j], 16);
#pragma unroll
                    for (int e = 0; e < E; ++e) t[e] = map(t[e]);
                    uint4 w;
                    memcpy(&w, t, 16);
                    reinterpret_cast<uint4 *>(dst)[u] = w;
                }
            }
            const int i = nv * E + tid;
            if (i < m) dst[i] = map(elem[0]);
        } else {
#pragma unroll
            for (int j = 0; j < KPT; ++j) {
                const int i = tid + j * nt;
                if (i < m) dst[i] = map(elem[j]);
            }
        }
    }
    __device__ __forceinline__ void store(T *dst, int m) const {
        store(dst, m, [](T x) { return x; });
    }
};

// Dynamic shared memory of the streaming kernels for a chunk of `chunk`
// keys: per key its key, value (vb bytes; 0 for erase) and result byte.
__host__ __device__ __forceinline__ size_t stream_smem(long long chunk, int kb, int vb) {
    return (size_t)chunk * (kb + vb + 1);
}

template <int LB>
__device__ __forceinline__ void load_find(LaneWords<LB> &lw, const unsigned char *p) {
    if constexpr (HC_FIND_L1 && LB >= 32) {
#pragma unroll
        for (int q = 0; q < LB / 32; ++q)
            asm volatile("ld.global.nc.v4.u64 {%0,%1,%2,%3}, [%4];"
                         : "=l"(lw.w[4 * q]), "=l"(lw.w[4 * q + 1]), "=l"(lw.w[4 * q + 2]), "=l"(lw.w[4 * q + 3])
                         : "l"(p + 32 * q));
    } else {
        lw.load(p);
    }
}

template <int KIND, int BB>
__device__ __forceinline__ unsigned long long load_find_val(const View &v, unsigned long long b, int s) {
    using T = Traits<KIND>;
    if constexpr (HC_FIND_L1 && T::MAP)
        return (unsigned long long)__ldg(reinterpret_cast<const typename T::Val *>(Slots<KIND, BB>::val(v, b, s)));
    else
        return load_val<KIND, BB>(v, b, s);
}

template <int KIND, int BB, int KPT, int S>
__device__ __forceinline__ void find_stream_chunk(const View &v, const typename Traits<KIND>::Key *keys, long long c0, int m,
                                                  uint8_t *found, typename Traits<KIND>::Val *vals_out) {
    using T = Traits<KIND>;
    using Key = typename T::Key;
    using Val = typename T::Val;
    using Sl = Slots<KIND, BB>;
    constexpr int LB = Sl::KRB;              // one thread reads the whole key region
    constexpr int SPL = Sl::SPB;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nt = blockDim.x;
    const int chunk = nt * KPT;
    Key *sk = reinterpret_cast<Key *>(smem);
    Val *sv = reinterpret_cast<Val *>(smem + (size_t)chunk * sizeof(Key));
    uint8_t *sf = smem + (size_t)chunk * (sizeof(Key) + sizeof(Val));

    Stage<Key, KPT> gk;
    gk.load(keys + c0, m);
    __syncthreads();                         // the staging of a previous chunk is no longer read
    gk.store(sk, m);
    __syncthreads();

    // this thread's keys: threadIdx.x + j * nt, j < KPT
    int idx[S];
    Key key[S];
    unsigned long long b[S];
    uint32_t probes[S];
    int next = 0;
    uint32_t active = 0;
    auto take = [&](int s) {
        while (next < KPT) {
            const int i = threadIdx.x + (next++) * nt;
            if (i >= m) { next = KPT; break; }
            const Key k = sk[i];
            const int side = side_index<KIND>(k);
            if (side >= 0) {
                const uint32_t pres = *((volatile unsigned int *)&v.hdr->side_present[side]);
                sf[i] = pres ? 1 : 0;
                if constexpr (T::MAP) sv[i] = pres ? (Val) * ((volatile unsigned long long *)&v.hdr->side_val[side]) : (Val)0;
                continue;
            }
            idx[s] = i;
            key[s] = k;
            b[s] = first_bucket(v, (unsigned long long)k);
            probes[s] = 0;
            active |= 1u << s;
            return;
        }
    };
#pragma unroll
    for (int s = 0; s < S; ++s) take(s);
    while (active) {
        LaneWords<LB> lw[S];
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (active >> s & 1u) load_find<LB>(lw[s], bucket_at<BB>(v, b[s]));
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (!(active >> s & 1u)) continue;
            uint32_t lm = 0, le = 0;
#pragma unroll
            for (int q = 0; q < SPL; ++q) {
                const Key ks = slot_key<KIND, LB>(lw[s], q);
                lm |= (uint32_t)(ks == key[s]) << q;
                le |= (uint32_t)(ks == T::EMPTY) << q;
            }
            bool done = false;
            if (lm) {
                sf[idx[s]] = 1;
                if constexpr (T::MAP) sv[idx[s]] = (Val)load_find_val<KIND, BB>(v, b[s], __ffs(lm) - 1);
                done = true;
            } else if (le || ++probes[s] >= v.nb) {
                sf[idx[s]] = 0;
                if constexpr (T::MAP) sv[idx[s]] = (Val)0;
                done = true;
            } else {
                b[s] = next_bucket(v, b[s]);
            }
            if (done) {
                active &= ~(1u << s);
                take(s);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += nt) {
        if (found) st_stream(found + c0 + i, sf[i]);
        if constexpr (T::MAP) {
            if (vals_out) st_stream(vals_out + c0 + i, sv[i]);
        }
    }
}

template <int KIND, int BB, int KPT, int S>
__global__ void __launch_bounds__(256, HC_STREAM_FIND_MINB)
k_find_stream(View v, const typename Traits<KIND>::Key *keys, long long n, uint8_t *found,
              typename Traits<KIND>::Val *vals_out) {
    const long long chunk = (long long)blockDim.x * KPT;
    const long long c0 = (long long)blockIdx.x * chunk;
    const int m = (int)(n - c0 < chunk ? n - c0 : chunk);
    debug_range(v, c0, m, n);
    find_stream_chunk<KIND, BB, KPT, S>(v, keys, c0, m, found, vals_out);
}

// Streaming map lookup by lane pairs: the two lanes of a pair handle one key.
// The first probe reads the key's first bucket in one instruction, the even
// lane its key region (the first BB/2 bytes), the odd lane its values (the
// rest): one request for one line, and a match there (most present keys) has
// its value without a second, dependent request.  Later probes read the key
// regions of two consecutive buckets at once (even lane: b, odd lane: b + 1),
// so a probe chain advances two buckets per round; a match found there reads
// its value separately.  The pair keeps identical state and control flow and
// exchanges the comparison masks with shuffles.
template <int KIND, int BB, int KPT, int S>
__global__ void __launch_bounds__(256, HC_STREAM_FIND_MINB)
k_find_pair(View v, const typename Traits<KIND>::Key *keys, long long n, uint8_t *found,
            typename Traits<KIND>::Val *vals_out) {
    using T = Traits<KIND>;
    using Key = typename T::Key;
    using Val = typename T::Val;
    using Sl = Slots<KIND, BB>;
    constexpr int HB = BB / 2;                    // bytes per lane
    constexpr int SPL = Sl::SPB;
    static_assert(T::MAP && Sl::KRB == HB, "a pair splits a map bucket into keys and values");
    extern __shared__ __align__(16) unsigned char smem[];
    const int pairs = blockDim.x / 2;
    const int chunk = pairs * KPT;
    Key *sk = reinterpret_cast<Key *>(smem);
    Val *sv = reinterpret_cast<Val *>(smem + (size_t)chunk * sizeof(Key));
    uint8_t *sf = smem + (size_t)chunk * (sizeof(Key) + sizeof(Val));

    const long long c0 = (long long)blockIdx.x * chunk;
    const int m = (int)(n - c0 < chunk ? n - c0 : chunk);
    Stage<Key, KPT> gk;
    gk.load(keys + c0, m);
    gk.store(sk, m);
    __syncthreads();

    const unsigned lane = threadIdx.x & 31;
    const bool odd = lane & 1u;
    const unsigned pmask = 3u << (lane & 30u);
    const int pair = threadIdx.x >> 1;
    int idx[S];
    Key key[S];
    unsigned long long b[S];
    uint32_t probes[S];
    bool first[S];
    int next = 0;
    uint32_t active = 0;
    auto take = [&](int s) {
        while (next < KPT) {
            const int i = pair + (next++) * pairs;
            if (i >= m) { next = KPT; break; }
            const Key k = sk[i];
            const int side = side_index<KIND>(k);
            if (side >= 0) {
                if (!odd) {
                    const uint32_t pres = *((volatile unsigned int *)&v.hdr->side_present[side]);
                    sf[i] = pres ? 1 : 0;
                    sv[i] = pres ? (Val) * ((volatile unsigned long long *)&v.hdr->side_val[side]) : (Val)0;
                }
                continue;
            }
            idx[s] = i;
            key[s] = k;
            b[s] = first_bucket(v, (unsigned long long)k);
            probes[s] = 0;
            first[s] = true;
            active |= 1u << s;
            return;
        }
    };
#pragma unroll
    for (int s = 0; s < S; ++s) take(s);
    while (active) {
        LaneWords<HB> lw[S];
        // first probe of a key: keys (even lane) and values (odd lane) of its
        // first bucket; later probes: the key regions of two buckets, b (even
        // lane) and the next one (odd lane)
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (!(active >> s & 1u)) continue;
            const unsigned long long bb = (odd && !first[s]) ? next_bucket(v, b[s]) : b[s];
            load_find<HB>(lw[s], bucket_at<BB>(v, bb) + ((odd && first[s]) ? HB : 0));
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (!(active >> s & 1u)) continue;
            uint32_t lm = 0, le = 0;
            if (!odd || !first[s]) {
#pragma unroll
                for (int q = 0; q < SPL; ++q) {
                    const Key ks = slot_key<KIND, HB>(lw[s], q);
                    lm |= (uint32_t)(ks == key[s]) << q;
                    le |= (uint32_t)(ks == T::EMPTY) << q;
                }
            }
            const uint32_t lm0 = __shfl_sync(pmask, lm, lane & 30u), le0 = __shfl_sync(pmask, le, lane & 30u);
            const uint32_t lm1 = __shfl_sync(pmask, lm, lane | 1u), le1 = __shfl_sync(pmask, le, lane | 1u);
            int hit = -1;                      // bucket offset (0 or 1) of a match
            bool absent = false;
            if (first[s]) {
                if (lm0) {
                    const int q = __ffs(lm0) - 1;
                    if (odd) {
                        Val val = 0;           // select the word without indexing registers at run time
#pragma unroll
                        for (int qq = 0; qq < SPL; ++qq) {
                            if constexpr (sizeof(Val) == 8) {
                                if (qq == q) val = (Val)lw[s].w[qq];
                            } else {
                                if (qq == q) val = (Val)(uint32_t)(lw[s].w[qq >> 1] >> ((qq & 1) * 32));
                            }
                        }
                        sv[idx[s]] = val;
                    } else {
                        sf[idx[s]] = 1;
                    }
                    hit = 2;                   // resolved with its value
                } else if (le0 || ++probes[s] >= v.nb) {
                    absent = true;
                } else {
                    b[s] = next_bucket(v, b[s]);
                    first[s] = false;
                }
            } else {
                if (lm0) hit = 0;
                else if (le0 || ++probes[s] >= v.nb) absent = true;
                else if (lm1) hit = 1;
                else if (le1 || ++probes[s] >= v.nb) absent = true;
                else b[s] = next_bucket(v, next_bucket(v, b[s]));
                if (hit >= 0 && !odd) {        // a later bucket: the value needs its own read
                    const unsigned long long hb = hit ? next_bucket(v, b[s]) : b[s];
                    sf[idx[s]] = 1;
                    sv[idx[s]] = (Val)load_find_val<KIND, BB>(v, hb, __ffs(hit ? lm1 : lm0) - 1);
                }
            }
            if (absent && !odd) {
                sf[idx[s]] = 0;
                sv[idx[s]] = (Val)0;
            }
            if (hit >= 0 || absent) {
                active &= ~(1u << s);
                take(s);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        if (found) st_stream(found + c0 + i, sf[i]);
        if (vals_out) st_stream(vals_out + c0 + i, sv[i]);
    }
}

// Streaming insert: the same staging and refilling as k_find_stream.  Within
// one round every slot first decides whether it claims, then all claiming
// slots issue their compare-and-swap together, so the atomics of different
// keys overlap.  Statuses collect in shared memory and leave in coalesced
// stores; counters leave with one atomic per warp.  Equal keys inside a warp
// are not folded here (folding is a lock-step option).
template <int KIND, int BB, int KPT, int S>
__device__ __forceinline__ void insert_stream_chunk(const View &v, const typename Traits<KIND>::Key *keys,
                                                    const typename Traits<KIND>::Val *vals, long long c0, int m,
                                                    uint8_t *status, const uint8_t *skip) {
    using T = Traits<KIND>;
    using Key = typename T::Key;
    using Val = typename T::Val;
    using Sl = Slots<KIND, BB>;
    using Lay = Layout<KIND, BB, Sl::KRB>;
    constexpr int LB = Sl::KRB;
    constexpr int SPL = Sl::SPB;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nt = blockDim.x;
    const int chunk = nt * KPT;
    Key *sk = reinterpret_cast<Key *>(smem);
    Val *sv = reinterpret_cast<Val *>(smem + (size_t)chunk * sizeof(Key));
    uint8_t *ss = smem + (size_t)chunk * (sizeof(Key) + sizeof(Val));

    Stage<Key, KPT> gk;
    Stage<Val, KPT> gv;
    Stage<uint8_t, KPT> gs;
    gk.load(keys + c0, m);
    if constexpr (T::MAP) gv.load(vals + c0, m);
    if (skip) gs.load(skip + c0, m);
    __syncthreads();                         // the staging of a previous chunk is no longer read
    gk.store(sk, m);
    if constexpr (T::MAP) gv.store(sv, m);
    // result bytes: ST_EXISTS for keys a find reported present, 0xFF (to do)
    if (skip) gs.store(ss, m, [](uint8_t f) { return f ? (uint8_t)ST_EXISTS : (uint8_t)0xFF; });
    else
        for (int i = threadIdx.x; i < m; i += nt) ss[i] = 0xFF;
    __syncthreads();

    Counts cnt;
    int idx[S];
    Key key[S];
    unsigned long long b[S], ffb[S];
    uint32_t probes[S], restarts[S], ffs_slot[S];
    bool ff_empty[S];
    int next = 0;
    uint32_t active = 0;
    auto take = [&](int s) {
        while (next < KPT) {
            const int i = threadIdx.x + (next++) * nt;
            if (i >= m) { next = KPT; break; }
            if (ss[i] != 0xFF) continue;                       // reported present by a find
            const Key k = sk[i];
            const int side = side_index<KIND>(k);
            if (side >= 0) {                                   // key equal to a marker: side slot
                const bool won = atomicCAS(&v.hdr->side_present[side], 0u, 1u) == 0u;
                if (won) {
                    if constexpr (T::MAP) v.hdr->side_val[side] = (unsigned long long)sv[i];
                    ++cnt.ins;
                }
                ss[i] = won ? (uint8_t)ST_INSERTED : (uint8_t)ST_EXISTS;
                continue;
            }
            idx[s] = i;
            key[s] = k;
            b[s] = first_bucket(v, (unsigned long long)k);
            probes[s] = 0;
            restarts[s] = 0;
            ffb[s] = ~0ull;
            active |= 1u << s;
            return;
        }
    };
#pragma unroll
    for (int s = 0; s < S; ++s) take(s);
    while (active) {
        LaneWords<LB> lw[S];
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (active >> s & 1u) lw[s].load(bucket_at<BB>(v, b[s]));
        uint32_t claiming = 0;
        uint32_t finished = 0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (!(active >> s & 1u)) continue;
            uint32_t lm = 0, le = 0, lt = 0;
#pragma unroll
            for (int q = 0; q < SPL; ++q) {
                const Key ks = slot_key<KIND, LB>(lw[s], q);
                lm |= (uint32_t)(ks == key[s]) << q;
                le |= (uint32_t)(ks == T::EMPTY) << q;
                lt |= (uint32_t)(ks == T::TOMB) << q;
            }
            if (lm) {                                           // already stored
                ss[idx[s]] = ST_EXISTS;
                finished |= 1u << s;
                continue;
            }
            if (ffb[s] == ~0ull) {                              // first free slot, rotated scan
                lt &= claimable<KIND, BB, LB>(v, b[s], 0);
                const uint32_t lf = le | lt;
                if (lf) {
                    const int rot = v.rotate ? slot_rotation<Lay::SPB>(key[s]) : 0;
                    const uint32_t hi = lf & (Lay::ALL & ~((1u << rot) - 1u));
                    const int q = __ffs(hi ? hi : lf) - 1;
                    ffb[s] = b[s];
                    ffs_slot[s] = q;
                    ff_empty[s] = (le >> q) & 1u;
                }
            }
            if (le) {
                claiming |= 1u << s;
            } else if (++probes[s] >= v.nb) {
                if (ffb[s] == ~0ull) {                          // no free slot anywhere
                    ss[idx[s]] = ST_OVERFLOW;
                    cnt.over = 1;
                    finished |= 1u << s;
                } else {
                    claiming |= 1u << s;                        // only tombstones were free
                }
            } else {
                b[s] = next_bucket(v, b[s]);
            }
        }
        Key old[S];
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (claiming >> s & 1u)
                old[s] = cas_key<KIND>(Slots<KIND, BB>::key(v, ffb[s], ffs_slot[s]), ff_empty[s] ? T::EMPTY : T::TOMB,
                                       key[s]);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (!(claiming >> s & 1u)) continue;
            const Key expect = ff_empty[s] ? T::EMPTY : T::TOMB;
            if (old[s] == expect) {
                if constexpr (T::MAP) {
                    store_val<KIND, BB>(v, ffb[s], ffs_slot[s], (unsigned long long)sv[idx[s]]);
                    note_claim_key<KIND>(v.hdr, key[s], (long long)(ffb[s] * SPL) + ffs_slot[s]);
                }
                ss[idx[s]] = ST_INSERTED;
                ++cnt.ins;
                cnt.new_slot += ff_empty[s] ? 1u : 0u;
                finished |= 1u << s;
            } else if (old[s] == key[s]) {
                ss[idx[s]] = ST_EXISTS;                         // an equal key won the race
                finished |= 1u << s;
            } else if (++restarts[s] > kMaxRestarts) {
                atomicOr(&v.hdr->err, ERR_PROBE_BOUND);
                ss[idx[s]] = ST_OVERFLOW;
                cnt.over = 1;
                finished |= 1u << s;
            } else {                                            // lost the slot to another key
                b[s] = first_bucket(v, (unsigned long long)key[s]);
                probes[s] = 0;
                ffb[s] = ~0ull;
            }
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (finished >> s & 1u) {
                active &= ~(1u << s);
                take(s);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += nt)
        if (status) st_stream(status + c0 + i, ss[i]);
    flush_counts(v, cnt);
}

template <int KIND, int BB, int KPT, int S>
__global__ void __launch_bounds__(256, HC_STREAM_INSERT_MINB)
k_insert_stream(View v, const typename Traits<KIND>::Key *keys, const typename Traits<KIND>::Val *vals, long long n,
                uint8_t *status, const uint8_t *skip) {
    const long long chunk = (long long)blockDim.x * KPT;
    const long long c0 = (long long)blockIdx.x * chunk;
    const int m = (int)(n - c0 < chunk ? n - c0 : chunk);
    debug_range(v, c0, m, n);
    insert_stream_chunk<KIND, BB, KPT, S>(v, keys, vals, c0, m, status, skip);
}

// Streaming erase: the staging and refilling of k_find_stream; a slot that
// finds its key joins the round's compare-and-swap (key -> TOMB) with the
// other slots that found theirs.  A failed swap means an equal key of the
// same call erased the slot first: that key reports ERASED, this one
// NOT_FOUND, as in the lock-step form.  Keys flagged in `skip` report
// NOT_FOUND without a probe (the later occurrences of a key in the ordered
// erase).
template <int KIND, int BB, int KPT, int S>
__device__ __forceinline__ void erase_stream_chunk(const View &v, const typename Traits<KIND>::Key *keys, long long c0, int m,
                                                   uint8_t *status, const uint8_t *skip) {
    using T = Traits<KIND>;
    using Key = typename T::Key;
    using Sl = Slots<KIND, BB>;
    constexpr int LB = Sl::KRB;
    constexpr int SPL = Sl::SPB;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nt = blockDim.x;
    const int chunk = nt * KPT;
    Key *sk = reinterpret_cast<Key *>(smem);
    uint8_t *ss = smem + (size_t)chunk * sizeof(Key);

    Stage<Key, KPT> gk;
    Stage<uint8_t, KPT> gs;
    gk.load(keys + c0, m);
    if (skip) gs.load(skip + c0, m);
    __syncthreads();                         // the staging of a previous chunk is no longer read
    gk.store(sk, m);
    // result bytes: NOT_FOUND for the later occurrences of a key, 0xFF (to do)
    if (skip) gs.store(ss, m, [](uint8_t f) { return f ? (uint8_t)ST_NOT_FOUND : (uint8_t)0xFF; });
    else
        for (int i = threadIdx.x; i < m; i += nt) ss[i] = 0xFF;
    __syncthreads();

    Counts cnt;
    int idx[S];
    Key key[S];
    unsigned long long b[S];
    uint32_t probes[S], hit_slot[S];
    int next = 0;
    uint32_t active = 0;
    auto take = [&](int s) {
        while (next < KPT) {
            const int i = threadIdx.x + (next++) * nt;
            if (i >= m) { next = KPT; break; }
            if (ss[i] != 0xFF) continue;                       // a later occurrence: NOT_FOUND
            const Key k = sk[i];
            const int side = side_index<KIND>(k);
            if (side >= 0) {                                   // key equal to a marker: side slot
                const bool won = atomicCAS(&v.hdr->side_present[side], 1u, 0u) == 1u;
                cnt.del += won ? 1u : 0u;
                ss[i] = won ? (uint8_t)ST_ERASED : (uint8_t)ST_NOT_FOUND;
                continue;
            }
            idx[s] = i;
            key[s] = k;
            b[s] = first_bucket(v, (unsigned long long)k);
            probes[s] = 0;
            active |= 1u << s;
            return;
        }
    };
#pragma unroll
    for (int s = 0; s < S; ++s) take(s);
    while (active) {
        LaneWords<LB> lw[S];
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (active >> s & 1u) lw[s].load(bucket_at<BB>(v, b[s]));
        uint32_t hitting = 0, finished = 0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (!(active >> s & 1u)) continue;
            uint32_t lm = 0, le = 0;
#pragma unroll
            for (int q = 0; q < SPL; ++q) {
                const Key ks = slot_key<KIND, LB>(lw[s], q);
                lm |= (uint32_t)(ks == key[s]) << q;
                le |= (uint32_t)(ks == T::EMPTY) << q;
            }
            if (lm) {
                hit_slot[s] = __ffs(lm) - 1;
                hitting |= 1u << s;
            } else if (le || ++probes[s] >= v.nb) {
                ss[idx[s]] = ST_NOT_FOUND;
                finished |= 1u << s;
            } else {
                b[s] = next_bucket(v, b[s]);
            }
        }
        Key old[S];
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (hitting >> s & 1u) old[s] = cas_key<KIND>(Sl::key(v, b[s], hit_slot[s]), key[s], T::TOMB);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (!(hitting >> s & 1u)) continue;
            const bool won = old[s] == key[s];
            if (won) note_claim_key<KIND>(v.hdr, key[s], -1);
            ss[idx[s]] = won ? (uint8_t)ST_ERASED : (uint8_t)ST_NOT_FOUND;
            cnt.del += won ? 1u : 0u;
            finished |= 1u << s;
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (finished >> s & 1u) {
                active &= ~(1u << s);
                take(s);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += nt)
        if (status) st_stream(status + c0 + i, ss[i]);
    flush_counts(v, cnt);
}

template <int KIND, int BB, int KPT, int S>
__global__ void __launch_bounds__(256, HC_STREAM_ERASE_MINB)
k_erase_stream(View v, const typename Traits<KIND>::Key *keys, long long n, uint8_t *status, const uint8_t *skip) {
    const long long chunk = (long long)blockDim.x * KPT;
    const long long c0 = (long long)blockIdx.x * chunk;
    const int m = (int)(n - c0 < chunk ? n - c0 : chunk);
    debug_range(v, c0, m, n);
    erase_stream_chunk<KIND, BB, KPT, S>(v, keys, c0, m, status, skip);
}

}  // namespace hc
