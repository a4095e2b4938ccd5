// hc_kernels.cuh -- the one-launch-per-call kernels (insert, find, erase,
// clear, rehash) and their launchers, instantiated once per container
// kind by hc_kind_*.cu.
#pragma once

#include "hc_core.cuh"
#include "hc_internal.h"
#include "hc_stream.cuh"

namespace hc {

// ------------------------------------------------------- range kernels ---
// One tile per warp and as many blocks as the call needs: short-lived warps
// let the block scheduler refill an SM as soon as its slowest probes finish.
// (A persistent grid-stride form that prefetched the next tile measured
// 1.3-2x slower on GB300 for every shape.)

// Launch bounds (threads per block[, minimum resident blocks]): a build option,
// since capping registers trades spills for resident warps.
#ifndef HC_INSERT_MAXT
#define HC_INSERT_MAXT 256
#endif
#ifndef HC_INSERT_MINB
#define HC_INSERT_MINB 1
#endif
#ifndef HC_FIND_MAXT
#define HC_FIND_MAXT 256
#endif
#ifndef HC_FIND_MINB
#define HC_FIND_MINB 6   // 40 registers, no spills: +1-7 % for find and erase on GB300
#endif

template <int KIND, int BB, int LB, int KPT>
__global__ void __launch_bounds__(HC_INSERT_MAXT, HC_INSERT_MINB)
k_insert(View v, const typename Traits<KIND>::Key *keys, const typename Traits<KIND>::Val *vals, long long n,
         uint8_t *status, int fold, const uint8_t *skip) {
    constexpr int TILE = Shape<KIND, BB, LB, KPT>::TILE;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    Counts cnt;
    run_tiles<KIND, BB, LB, KPT, 0>(v, keys, vals, skip, status, nullptr, n, warp, (n + TILE - 1) / TILE, warps,
                                    fold != 0, cnt);
    flush_counts(v, cnt);
}

template <int KIND, int BB, int LB, int KPT>
__global__ void __launch_bounds__(HC_FIND_MAXT, HC_FIND_MINB)
k_find(View v, const typename Traits<KIND>::Key *keys, long long n, uint8_t *found,
       typename Traits<KIND>::Val *vals_out) {
    constexpr int TILE = Shape<KIND, BB, LB, KPT>::TILE;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    Counts cnt;
    run_tiles<KIND, BB, LB, KPT, 1>(v, keys, nullptr, nullptr, found, vals_out, n, warp, (n + TILE - 1) / TILE, warps,
                                    false, cnt);
}

template <int KIND, int BB, int LB, int KPT>
__global__ void __launch_bounds__(HC_FIND_MAXT, HC_FIND_MINB)
k_erase(View v, const typename Traits<KIND>::Key *keys, long long n, uint8_t *status, int fold) {
    constexpr int TILE = Shape<KIND, BB, LB, KPT>::TILE;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    Counts cnt;
    run_tiles<KIND, BB, LB, KPT, 2>(v, keys, nullptr, nullptr, status, nullptr, n, warp, (n + TILE - 1) / TILE, warps,
                                    fold != 0, cnt);
    flush_counts(v, cnt);
}

// ---------------------------------------------------------------- clear ---
// Every bucket all-ones bytes (so every key slot is EMPTY; values need no
// initialisation, a value is read only after its key was found), 32-byte
// stores; the header zeroed; then the padding slots of the last bucket become
// tombstones.

static __global__ void __launch_bounds__(256)
k_fill_empty(unsigned char *keys, unsigned long long bytes, Header *hdr) {
    const unsigned long long chunks = bytes / 32;
    const unsigned long long ones = ~0ull;
    for (unsigned long long c = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; c < chunks;
         c += (unsigned long long)gridDim.x * blockDim.x) {
        asm volatile("st.global.v4.u64 [%0], {%1,%1,%1,%1};" ::"l"(keys + c * 32), "l"(ones) : "memory");
    }
    if (blockIdx.x == 0 && threadIdx.x < sizeof(Header) / 8)
        reinterpret_cast<unsigned long long *>(hdr)[threadIdx.x] = 0ull;
}

template <int KIND, int BB>
__global__ void k_pad_tombstones(View v, unsigned long long first, unsigned long long count) {
    using T = Traits<KIND>;
    using S = Slots<KIND, BB>;
    const unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) {
        const unsigned long long slot = first + i;
        *reinterpret_cast<typename T::Key *>(S::key(v, slot / S::SPB, (int)(slot % S::SPB))) = T::TOMB;
    }
}

// --------------------------------------------------------------- rehash ---
// Each stored key of the old arrays goes to the first EMPTY slot of its probe
// sequence in the new arrays (keys are distinct, so no equality test; the new
// table has no tombstones except its padding, which is never EMPTY).

template <int KIND, int BB>
__global__ void __launch_bounds__(256)
k_rehash(View old_v, unsigned long long old_phys, View new_v) {
    using T = Traits<KIND>;
    using Key = typename T::Key;
    using S = Slots<KIND, BB>;
    constexpr int SPB = S::SPB;
    uint32_t moved = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
         base < old_phys; base += stride) {
        const unsigned long long i = base + (threadIdx.x & 31);
        if (i >= old_phys) continue;
        const unsigned long long ob = i / SPB;
        const int os = (int)(i % SPB);
        const Key key = *reinterpret_cast<const Key *>(S::key(old_v, ob, os));
        if (key == T::EMPTY || key == T::TOMB) continue;
        unsigned long long val = 0;
        if constexpr (T::MAP) val = *reinterpret_cast<const typename T::Val *>(S::val(old_v, ob, os));
        unsigned long long b = first_bucket(new_v, (unsigned long long)key);
        bool done = false;
        for (unsigned long long p = 0; p < new_v.nb && !done;) {
            Key *bucket = reinterpret_cast<Key *>(S::key(new_v, b, 0));
            int s = 0;
            for (; s < SPB; ++s) {
                Key ks;
                if constexpr (sizeof(Key) == 4) ks = __ldcg(reinterpret_cast<const unsigned int *>(bucket + s));
                else ks = __ldcg(reinterpret_cast<const unsigned long long *>(bucket + s));
                if (ks == T::EMPTY) break;
            }
            if (s == SPB) {
                b = next_bucket(new_v, b);
                ++p;
                continue;
            }
            if (cas_key<KIND>(reinterpret_cast<unsigned char *>(bucket + s), T::EMPTY, key) == T::EMPTY) {
                store_val<KIND, BB>(new_v, b, s, val);
                note_claim_key<KIND>(new_v.hdr, key, (long long)(b * SPB) + s);
                done = true;
            }
            // a lost race re-reads the same bucket
        }
        if (done) ++moved;
        else atomicOr(&new_v.hdr->err, ERR_PROBE_BOUND);
    }
    const uint32_t w = __reduce_add_sync(0xffffffffu, moved);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&new_v.hdr->reinserted, (unsigned long long)w);
}

// ------------------------------------------------------------ launchers ---

inline unsigned grid_for(long long n, int tile, int block) {
    const long long warps = (n + tile - 1) / tile;                // one tile per warp
    return (unsigned)((warps * 32 + block - 1) / block);
}

template <int KIND, int BB, int LB, int KPT>
cudaError_t launch_range_shape(int op, const View &v, const void *keys, const void *vals, long long n, uint8_t *out,
                               void *vals_out, const LaunchShape &sh, const uint8_t *skip, cudaStream_t s) {
    using T = Traits<KIND>;
    using Key = typename T::Key;
    using Val = typename T::Val;
    constexpr int TILE = Shape<KIND, BB, LB, KPT>::TILE;
    const int block = sh.block;
    if (n <= 0) return cudaSuccess;
    const unsigned grid = grid_for(n, TILE, block);
    if (op == OP_INSERT)
        k_insert<KIND, BB, LB, KPT><<<grid, block, 0, s>>>(v, (const Key *)keys, (const Val *)vals, n, out, sh.fold, skip);
    else if (op == OP_FIND)
        k_find<KIND, BB, LB, KPT><<<grid, block, 0, s>>>(v, (const Key *)keys, n, out, (Val *)vals_out);
    else
        k_erase<KIND, BB, LB, KPT><<<grid, block, 0, s>>>(v, (const Key *)keys, n, out, sh.fold);
    return cudaGetLastError();
}

// A kernel launched with more than the default 48 KB of dynamic shared
// memory (streaming kernels with 256-thread blocks and 8 keys per thread)
// must be allowed it first.
template <class K>
void allow_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) (void)cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Streaming lookup: each thread owns KPT keys of its block's staged chunk and
// keeps S probes in flight (find only, one thread per key).
template <int KIND, int BB, int KPT, int S>
cudaError_t launch_find_stream(const View &v, const void *keys, long long n, uint8_t *out, void *vals_out, int block,
                               cudaStream_t s) {
    using T = Traits<KIND>;
    const long long chunk = (long long)block * KPT;
    const unsigned grid = (unsigned)((n + chunk - 1) / chunk);
    const size_t smem = stream_smem(chunk, sizeof(typename T::Key), sizeof(typename T::Val));
    allow_smem(k_find_stream<KIND, BB, KPT, S>, smem);
    k_find_stream<KIND, BB, KPT, S><<<grid, block, smem, s>>>(v, (const typename T::Key *)keys, n, out,
                                                              (typename T::Val *)vals_out);
    return cudaGetLastError();
}

template <int KIND, int BB, int KPT, int S>
cudaError_t launch_find_pair(const View &v, const void *keys, long long n, uint8_t *out, void *vals_out, int block,
                             cudaStream_t s) {
    using T = Traits<KIND>;
    const long long chunk = (long long)(block / 2) * KPT;
    const unsigned grid = (unsigned)((n + chunk - 1) / chunk);
    const size_t smem = (size_t)chunk * (sizeof(typename T::Key) + sizeof(typename T::Val) + 1);
    k_find_pair<KIND, BB, KPT, S><<<grid, block, smem, s>>>(v, (const typename T::Key *)keys, n, out,
                                                            (typename T::Val *)vals_out);
    return cudaGetLastError();
}

template <int KIND, int BB, int KPT, int S>
cudaError_t launch_insert_stream(const View &v, const void *keys, const void *vals, long long n, uint8_t *out,
                                 const uint8_t *skip, int block, cudaStream_t s) {
    using T = Traits<KIND>;
    const long long chunk = (long long)block * KPT;
    const unsigned grid = (unsigned)((n + chunk - 1) / chunk);
    const size_t smem = stream_smem(chunk, sizeof(typename T::Key), sizeof(typename T::Val));
    allow_smem(k_insert_stream<KIND, BB, KPT, S>, smem);
    k_insert_stream<KIND, BB, KPT, S><<<grid, block, smem, s>>>(v, (const typename T::Key *)keys,
                                                                (const typename T::Val *)vals, n, out, skip);
    return cudaGetLastError();
}

template <int KIND, int BB, int KPT, int S>
cudaError_t launch_erase_stream(const View &v, const void *keys, long long n, uint8_t *out, const uint8_t *skip,
                                int block, cudaStream_t s) {
    using T = Traits<KIND>;
    const long long chunk = (long long)block * KPT;
    const unsigned grid = (unsigned)((n + chunk - 1) / chunk);
    const size_t smem = stream_smem(chunk, sizeof(typename T::Key), 0);
    allow_smem(k_erase_stream<KIND, BB, KPT, S>, smem);
    k_erase_stream<KIND, BB, KPT, S><<<grid, block, smem, s>>>(v, (const typename T::Key *)keys, n, out, skip);
    return cudaGetLastError();
}

template <int KIND, int BB, int LB>
cudaError_t launch_range_kpt(int op, const View &v, const void *keys, const void *vals, long long n, uint8_t *out,
                             void *vals_out, const LaunchShape &sh, const uint8_t *skip, cudaStream_t s) {
    if (sh.keys_per_group >= 4) {       // streaming forms: one thread per key, or a lane pair per map key
        if constexpr (Traits<KIND>::MAP && LB == BB && Slots<KIND, BB>::KRB * 2 == BB) {
            if (n <= 0) return cudaSuccess;
            if (op == OP_FIND) {
                if (sh.keys_per_group == 4) return launch_find_pair<KIND, BB, 4, 2>(v, keys, n, out, vals_out, sh.block, s);
                if (sh.keys_per_group == 8) return launch_find_pair<KIND, BB, 8, 4>(v, keys, n, out, vals_out, sh.block, s);
            }
            return cudaErrorInvalidValue;
        }
        if constexpr (LB == Slots<KIND, BB>::KRB) {
            if (n <= 0) return cudaSuccess;
            if (op == OP_FIND) {
                if (sh.keys_per_group == 4) return launch_find_stream<KIND, BB, 4, 2>(v, keys, n, out, vals_out, sh.block, s);
                if (sh.keys_per_group == 8) return launch_find_stream<KIND, BB, 8, 4>(v, keys, n, out, vals_out, sh.block, s);
            } else if (op == OP_INSERT) {
                if (sh.keys_per_group == 4) return launch_insert_stream<KIND, BB, 4, 2>(v, keys, vals, n, out, skip, sh.block, s);
                if (sh.keys_per_group == 8) return launch_insert_stream<KIND, BB, 8, 4>(v, keys, vals, n, out, skip, sh.block, s);
            } else {
                if (sh.keys_per_group == 4) return launch_erase_stream<KIND, BB, 4, 2>(v, keys, n, out, skip, sh.block, s);
                if (sh.keys_per_group == 8) return launch_erase_stream<KIND, BB, 8, 4>(v, keys, n, out, skip, sh.block, s);
            }
        }
        return cudaErrorInvalidValue;
    }
    switch (sh.keys_per_group) {
        case 1: return launch_range_shape<KIND, BB, LB, 1>(op, v, keys, vals, n, out, vals_out, sh, skip, s);
        case 2: return launch_range_shape<KIND, BB, LB, 2>(op, v, keys, vals, n, out, vals_out, sh, skip, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int KIND, int BB>
cudaError_t launch_range_lb(int op, const View &v, const void *keys, const void *vals, long long n, uint8_t *out,
                            void *vals_out, const LaunchShape &sh, const uint8_t *skip, cudaStream_t s) {
    constexpr int KRB = Slots<KIND, BB>::KRB;
    if constexpr (Traits<KIND>::MAP) {
        if (sh.lane_bytes == 16) return launch_range_kpt<KIND, BB, 16>(op, v, keys, vals, n, out, vals_out, sh, skip, s);
    }
    if constexpr (KRB >= 32)
        if (sh.lane_bytes == 32) return launch_range_kpt<KIND, BB, 32>(op, v, keys, vals, n, out, vals_out, sh, skip, s);
    if constexpr (KRB >= 64)
        if (sh.lane_bytes == 64) return launch_range_kpt<KIND, BB, 64>(op, v, keys, vals, n, out, vals_out, sh, skip, s);
    if constexpr (KRB >= 128)
        if (sh.lane_bytes == 128) return launch_range_kpt<KIND, BB, 128>(op, v, keys, vals, n, out, vals_out, sh, skip, s);
    if constexpr (Traits<KIND>::MAP)   // one thread reads keys and values
        if (sh.lane_bytes == BB) return launch_range_kpt<KIND, BB, BB>(op, v, keys, vals, n, out, vals_out, sh, skip, s);
    return cudaErrorInvalidValue;
}

template <int KIND>
cudaError_t launch_range(int op, const View &v, int bucket_bytes, const void *keys, const void *vals, long long n,
                         uint8_t *out, void *vals_out, const LaunchShape &sh, const uint8_t *skip, cudaStream_t s) {
    switch (bucket_bytes) {
        case 32: return launch_range_lb<KIND, 32>(op, v, keys, vals, n, out, vals_out, sh, skip, s);
        case 64: return launch_range_lb<KIND, 64>(op, v, keys, vals, n, out, vals_out, sh, skip, s);
        case 128: return launch_range_lb<KIND, 128>(op, v, keys, vals, n, out, vals_out, sh, skip, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int KIND, int BB>
cudaError_t launch_clear_bb(const View &v, unsigned long long phys, unsigned long long capacity, int sm_count,
                            cudaStream_t s) {
    const unsigned long long bytes = v.nb * BB;   // whole buckets: a multiple of 32
    const unsigned long long chunks = bytes / 32;
    unsigned grid = (unsigned)std::min<unsigned long long>((chunks + 255) / 256, (unsigned long long)sm_count * 8);
    if (grid == 0) grid = 1;
    k_fill_empty<<<grid, 256, 0, s>>>(v.buckets, bytes, v.hdr);
    if (phys > capacity) {
        const unsigned long long pad = phys - capacity;
        k_pad_tombstones<KIND, BB><<<(unsigned)((pad + 127) / 128), 128, 0, s>>>(v, capacity, pad);
    }
    return cudaGetLastError();
}

template <int KIND>
cudaError_t launch_clear(const View &v, unsigned long long phys, unsigned long long capacity, int bucket_bytes,
                         int sm_count, cudaStream_t s) {
    switch (bucket_bytes) {
        case 32: return launch_clear_bb<KIND, 32>(v, phys, capacity, sm_count, s);
        case 64: return launch_clear_bb<KIND, 64>(v, phys, capacity, sm_count, s);
        case 128: return launch_clear_bb<KIND, 128>(v, phys, capacity, sm_count, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int KIND>
cudaError_t launch_rehash(const View &old_v, unsigned long long old_phys, const View &new_v, int bucket_bytes,
                          int sm_count, cudaStream_t s) {
    unsigned grid = (unsigned)std::min<unsigned long long>((old_phys + 255) / 256, (unsigned long long)sm_count * 16);
    if (grid == 0) grid = 1;
    switch (bucket_bytes) {
        case 32: k_rehash<KIND, 32><<<grid, 256, 0, s>>>(old_v, old_phys, new_v); break;
        case 64: k_rehash<KIND, 64><<<grid, 256, 0, s>>>(old_v, old_phys, new_v); break;
        case 128: k_rehash<KIND, 128><<<grid, 256, 0, s>>>(old_v, old_phys, new_v); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hc

// Explicit per-kind entry points used by the host API.
#define HC_INSTANTIATE_KIND(KIND, NAME)                                                                             \
    namespace hc {                                                                                                  \
    cudaError_t NAME##_range(int op, const View &v, int bb, const void *keys, const void *vals, long long n,        \
                             uint8_t *out, void *vals_out, const LaunchShape &sh, const uint8_t *skip,              \
                             cudaStream_t s) {                                                                      \
        return launch_range<KIND>(op, v, bb, keys, vals, n, out, vals_out, sh, skip, s);                            \
    }                                                                                                               \
    cudaError_t NAME##_clear(const View &v, unsigned long long phys, unsigned long long cap, int bb, int sms,       \
                             cudaStream_t s) {                                                                      \
        return launch_clear<KIND>(v, phys, cap, bb, sms, s);                                                        \
    }                                                                                                               \
    cudaError_t NAME##_rehash(const View &ov, unsigned long long ophys, const View &nv, int bb, int sms,            \
                              cudaStream_t s) {                                                                     \
        return launch_rehash<KIND>(ov, ophys, nv, bb, sms, s);                                                      \
    }                                                                                                               \
    }
