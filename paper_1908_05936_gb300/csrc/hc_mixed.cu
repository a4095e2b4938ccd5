// hc_mixed.cu -- free-running mixed batches: inserts, finds and erases of one
// call run at once (Section 4, "Guarantees": concurrency across all
// operations).  Per key, the results are those of some serial order of that
// key's operations; inserts claim EMPTY slots only, and a map insert claims
// its slot with the CLAIM marker, stores the value, then the key, exactly as
// the in-kernel functions of include/hc_device.cuh do (whose waiting rule and
// special keys it shares).
//
// The kernel has the shape of the streaming range kernels: a block stages its
// chunk of operations, keys and values in shared memory with 16-byte loads,
// every thread keeps S operations in flight and refills a slot from the chunk
// as soon as its operation finishes, and in each round all the round's
// compare-and-swaps go out together.  A map insert's claim and its publication
// happen in the same round, around one fence per thread and round that also
// orders the round's lookups of found keys before their value reads; no claim
// is left in progress from one round to the next, so a wait on a claim always
// ends.  Results leave in coalesced stores, counters with one atomic per warp.
#include <algorithm>
#include <cstdint>

#include "hc.h"
#include "hc_device.cuh"
#include "hc_internal.h"
#include "hc_stream.cuh"

namespace hc {

namespace {

constexpr int kMixedBlock = 64;   // threads per block
constexpr int kMixedKPT = 8;      // operations per thread per chunk
constexpr int kMixedS = 2;        // operations in flight per thread

enum : uint8_t { MOP_INSERT = 0, MOP_FIND = 1, MOP_ERASE = 2 };

// The operations on keys that live outside the regular slots' probing: the
// side-slot patterns, and for maps the key equal to CLAIM.  Rare, so they go
// through the in-kernel functions (which count for themselves).
template <int KIND, int BB>
__device__ __noinline__ void special_op(const View &v, uint8_t op, typename Traits<KIND>::Key k,
                                        typename Traits<KIND>::Val *val, uint8_t *st) {
    using T = Traits<KIND>;
    if (op == MOP_INSERT) {
        *st = (uint8_t)hcd::detail::insert<KIND, BB>(v, k, (unsigned long long)*val).status;
        *val = typename T::Val();
    } else if (op == MOP_FIND) {
        const long long pos = hcd::detail::find<KIND, BB>(v, k);
        *st = pos != hcd::END;
        *val = pos != hcd::END ? hcd::detail::value_at<KIND, BB>(v, pos) : typename T::Val();
    } else {
        *st = (uint8_t)hcd::detail::erase<KIND, BB>(v, k);
        *val = typename T::Val();
    }
}

template <int KIND, int BB, int KPT, int S>
__global__ void __launch_bounds__(256)
k_mixed_stream(View v, const uint8_t *ops, const typename Traits<KIND>::Key *keys,
               const typename Traits<KIND>::Val *vals, long long n, uint8_t *status,
               typename Traits<KIND>::Val *vals_out) {
    using T = Traits<KIND>;
    using Key = typename T::Key;
    using Val = typename T::Val;
    using Sl = Slots<KIND, BB>;
    constexpr int LB = Sl::KRB;              // one thread reads the whole key region
    constexpr int SPB = Sl::SPB;
    constexpr int VB = T::MAP ? (int)sizeof(Val) : 0;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nt = blockDim.x;
    const int chunk = nt * KPT;
    const long long c0 = (long long)blockIdx.x * chunk;
    const int m = (int)(n - c0 < chunk ? n - c0 : chunk);
    debug_range(v, c0, m, n);
    Key *sk = reinterpret_cast<Key *>(smem);
    Val *sv = reinterpret_cast<Val *>(smem + (size_t)chunk * sizeof(Key));   // values in, found values out
    uint8_t *so = smem + (size_t)chunk * (sizeof(Key) + VB);                  // operation kinds
    uint8_t *ss = so + chunk;                                                 // results

    Stage<Key, KPT> gk;
    Stage<Val, KPT> gv;
    Stage<uint8_t, KPT> go;
    gk.load(keys + c0, m);
    if constexpr (T::MAP) gv.load(vals + c0, m);
    go.load(ops + c0, m);
    gk.store(sk, m);
    if constexpr (T::MAP) gv.store(sv, m);
    go.store(so, m, [](uint8_t o) { return o == MOP_INSERT ? (uint8_t)MOP_INSERT : (o == MOP_FIND ? (uint8_t)MOP_FIND : (uint8_t)MOP_ERASE); });
    __syncthreads();

    Counts cnt;
    int idx[S];
    Key key[S];
    uint8_t op[S];
    unsigned long long b[S];
    uint32_t probes[S], retries[S];
    int qs[S];
    int next = 0;
    uint32_t active = 0;
    auto take = [&](int s) {
        while (next < KPT) {
            const int i = threadIdx.x + (next++) * nt;
            if (i >= m) { next = KPT; break; }
            const Key k = sk[i];
            const uint8_t o = so[i];
            bool special = side_index<KIND>(k) >= 0;
            if constexpr (T::MAP) special = special || k == T::CLAIM;
            if (special) {
                Val dummy = Val();
                special_op<KIND, BB>(v, o, k, T::MAP ? &sv[i] : &dummy, &ss[i]);
                continue;
            }
            idx[s] = i;
            key[s] = k;
            op[s] = o;
            b[s] = first_bucket(v, (unsigned long long)k);
            probes[s] = 0;
            retries[s] = 0;
            active |= 1u << s;
            return;
        }
    };
    // an operation is over: its result byte is written; a map's value slot
    // keeps a found value (finds) or becomes 0 (inserts, erases)
    auto done = [&](int s, uint8_t st, uint32_t &finished) {
        ss[idx[s]] = st;
        if constexpr (T::MAP) {
            if (op[s] != MOP_FIND || st == 0) sv[idx[s]] = Val();
        }
        finished |= 1u << s;
    };
#pragma unroll
    for (int s = 0; s < S; ++s) take(s);
    while (active) {
        LaneWords<LB> lw[S];
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (active >> s & 1u) lw[s].load(bucket_at<BB>(v, b[s]));
        uint32_t finished = 0, swapping = 0, reading = 0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (!(active >> s & 1u)) continue;
            uint32_t lm = 0, le = 0, lc = 0;
#pragma unroll
            for (int q = 0; q < SPB; ++q) {
                const Key ks = slot_key<KIND, LB>(lw[s], q);
                lm |= (uint32_t)(ks == key[s]) << q;
                le |= (uint32_t)(ks == T::EMPTY) << q;
                if constexpr (T::MAP) lc |= (uint32_t)(ks == T::CLAIM) << q;
            }
            if (op[s] == MOP_FIND) {
                if (lm) {
                    if constexpr (T::MAP) {          // the value is read after this round's fence
                        qs[s] = __ffs(lm) - 1;
                        reading |= 1u << s;
                    } else {
                        done(s, 1, finished);
                    }
                } else if (le || ++probes[s] >= v.nb) {
                    done(s, 0, finished);
                } else {
                    b[s] = next_bucket(v, b[s]);
                }
            } else if (op[s] == MOP_ERASE) {
                if (lm) {
                    qs[s] = __ffs(lm) - 1;
                    swapping |= 1u << s;
                } else if (le || ++probes[s] >= v.nb) {
                    done(s, ST_NOT_FOUND, finished);
                } else {
                    b[s] = next_bucket(v, b[s]);
                }
            } else {
                if (lm) {                            // stored (and, for maps, published with its value)
                    done(s, ST_EXISTS, finished);
                    continue;
                }
                const int rot = slot_rotation<SPB>((unsigned long long)key[s]);
                bool wait = false;
                if constexpr (T::MAP) {              // the stored CLAIM-pattern key, or claims in progress
                    if (lc) wait = hcd::detail::must_wait<SPB>(v, b[s], lc, le, rot);
                }
                if (wait) {                          // read the bucket again next round
                    if (++retries[s] > kMaxRestarts) {
                        atomicOr(&v.hdr->err, ERR_PROBE_BOUND);
                        cnt.over = 1;
                        done(s, ST_OVERFLOW, finished);
                    }
                } else if (!le) {
                    if (++probes[s] >= v.nb) {
                        cnt.over = 1;
                        done(s, ST_OVERFLOW, finished);
                    } else {
                        b[s] = next_bucket(v, b[s]);
                    }
                } else {
                    qs[s] = hcd::detail::first_from<SPB>(le, rot);
                    swapping |= 1u << s;
                }
            }
        }
        Key old[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (!(swapping >> s & 1u)) continue;
            unsigned char *slot = Sl::key(v, b[s], qs[s]);
            if (op[s] == MOP_ERASE) old[s] = cas_key<KIND>(slot, key[s], T::TOMB);
            else old[s] = cas_key<KIND>(slot, T::EMPTY, T::MAP ? T::CLAIM : key[s]);
        }
        uint32_t publishing = 0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            if (!(swapping >> s & 1u)) continue;
            if (op[s] == MOP_ERASE) {
                // a failed swap means a concurrent erase of the same key won
                const bool won = old[s] == key[s];
                cnt.del += won ? 1u : 0u;
                done(s, won ? (uint8_t)ST_ERASED : (uint8_t)ST_NOT_FOUND, finished);
            } else if (old[s] == T::EMPTY) {
                if constexpr (T::MAP) {
                    store_val<KIND, BB>(v, b[s], qs[s], (unsigned long long)sv[idx[s]]);
                    publishing |= 1u << s;
                } else {
                    ++cnt.ins;
                    ++cnt.new_slot;
                    done(s, ST_INSERTED, finished);
                }
            } else if (!T::MAP && old[s] == key[s]) {
                done(s, ST_EXISTS, finished);        // an equal key won the slot
            } else if (++retries[s] > kMaxRestarts) {
                atomicOr(&v.hdr->err, ERR_PROBE_BOUND);
                cnt.over = 1;
                done(s, ST_OVERFLOW, finished);
            }
            // otherwise another key took the slot: the same bucket is read again
        }
        if constexpr (T::MAP) {
            if (publishing | reading) {
                // the claimed slots' values before their keys; the found keys'
                // loads before their values' loads
                __threadfence();
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    if (publishing >> s & 1u) {
                        hcd::detail::store_key<KIND>(Sl::key(v, b[s], qs[s]), key[s]);
                        ++cnt.ins;
                        ++cnt.new_slot;
                        done(s, ST_INSERTED, finished);
                    } else if (reading >> s & 1u) {
                        sv[idx[s]] = (Val)load_val<KIND, BB>(v, b[s], qs[s]);
                        done(s, 1, finished);
                    }
                }
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
    for (int i = threadIdx.x; i < m; i += nt) {
        if (status) st_stream(status + c0 + i, ss[i]);
        if constexpr (T::MAP) {
            if (vals_out) st_stream(vals_out + c0 + i, sv[i]);
        }
    }
    flush_counts(v, cnt);
}

template <int KIND, int BB>
cudaError_t launch_bb(const View &v, const uint8_t *ops, const void *keys, const void *vals, long long n,
                      uint8_t *status, void *vals_out, cudaStream_t s) {
    using T = Traits<KIND>;
    constexpr int chunk = kMixedBlock * kMixedKPT;
    const size_t smem = (size_t)chunk * (sizeof(typename T::Key) + (T::MAP ? sizeof(typename T::Val) : 0) + 2);
    const unsigned grid = (unsigned)((n + chunk - 1) / chunk);
    k_mixed_stream<KIND, BB, kMixedKPT, kMixedS><<<grid, kMixedBlock, smem, s>>>(
        v, ops, (const typename T::Key *)keys, (const typename T::Val *)vals, n, status,
        (typename T::Val *)vals_out);
    return cudaGetLastError();
}

template <int KIND>
cudaError_t launch(const hc_device_view &dv, const uint8_t *ops, const void *keys, const void *vals, long long n,
                   uint8_t *status, void *vals_out, cudaStream_t s) {
    const hcd::Table<KIND> t(dv);
    switch (dv.bucket_bytes) {
        case 32: return launch_bb<KIND, 32>(t.view(), ops, keys, vals, n, status, vals_out, s);
        case 64: return launch_bb<KIND, 64>(t.view(), ops, keys, vals, n, status, vals_out, s);
        default: return launch_bb<KIND, 128>(t.view(), ops, keys, vals, n, status, vals_out, s);
    }
}

}  // namespace

cudaError_t mixed_ops(const hc_device_view &dv, const uint8_t *ops, const void *keys, const void *vals, long long n,
                      uint8_t *status, void *vals_out, cudaStream_t s) {
    switch (dv.kind) {
        case HC_SET_U32: return launch<KIND_SET_U32>(dv, ops, keys, nullptr, n, status, nullptr, s);
        case HC_SET_U64: return launch<KIND_SET_U64>(dv, ops, keys, nullptr, n, status, nullptr, s);
        case HC_MAP_I64_I32: return launch<KIND_MAP_I64_I32>(dv, ops, keys, vals, n, status, vals_out, s);
        default: return launch<KIND_MAP_U64_U64>(dv, ops, keys, vals, n, status, vals_out, s);
    }
}

}  // namespace hc
