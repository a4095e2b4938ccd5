// hc_stream.cuh -- streaming lookup: a block stages its chunk of query keys in
// shared memory with coalesced loads, then every thread keeps S probes in
// flight and refills a slot from the chunk as soon as its probe finishes
// (instead of moving its keys in lock-step rounds).  Found flags and values
// go to shared memory and leave in coalesced stores.  One thread per key,
// reading the bucket's key region (KRB bytes) per probe.
#pragma once

#include "hc_core.cuh"

namespace hc {

template <int KIND, int BB, int KPT, int S>
__global__ void __launch_bounds__(256)
k_find_stream(View v, const typename Traits<KIND>::Key *keys, long long n, uint8_t *found,
              typename Traits<KIND>::Val *vals_out) {
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

    const long long c0 = (long long)blockIdx.x * chunk;
    const int m = (int)(n - c0 < chunk ? n - c0 : chunk);
    for (int i = threadIdx.x; i < m; i += nt) sk[i] = ld_stream(keys + c0 + i);
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
            if (active >> s & 1u) lw[s].load(v.buckets + b[s] * BB);
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
                if constexpr (T::MAP) sv[idx[s]] = (Val)load_val<KIND, BB>(v, b[s], __ffs(lm) - 1);
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

}  // namespace hc
