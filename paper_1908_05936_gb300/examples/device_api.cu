// device_api.cu -- user kernels written against include/hc_device.cuh, the
// in-kernel function form of Section 4.1.  They are what a program using the
// containers inside its own kernels looks like, and they are how the tests and
// the benchmark drive that interface:
//
//   hcx_apply       one operation per thread (insert, find or erase, from a
//                   per-thread op array or one op for all), results per thread;
//                   with mixed ops this is free-running concurrency on one table
//   hcx_update_set  Section 4.1's second example: for each voxel block, the
//                   block and its 7 neighbours towards -x, -y, -z that the
//                   block map contains go into an update set (a contains on one
//                   container and an insert into another in the same kernel)
//
// Built into libhc_examples.so; it needs only the two public headers.
#include <cstdint>

#include "hc.h"
#include "hc_device.cuh"

#define HCX_API extern "C" __attribute__((visibility("default")))

namespace {

template <int KIND>
__device__ __forceinline__ void apply_one(hc_device_view dv, const uint8_t *ops, int op_all,
                                          const typename hcd::Table<KIND>::Key *keys,
                                          const typename hcd::Table<KIND>::Val *vals, long long n, uint8_t *status,
                                          typename hcd::Table<KIND>::Val *vals_out, long long *pos_out) {
    using Tab = hcd::Table<KIND>;
    const Tab t(dv);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int op = ops ? ops[i] : op_all;
    const typename Tab::Key k = keys[i];
    long long pos = hcd::END;
    uint8_t st;
    if (op == 0) {
        const hcd::Inserted r = t.insert(k, (Tab::is_map && vals) ? vals[i] : typename Tab::Val());
        pos = r.slot;
        st = (uint8_t)r.status;
    } else if (op == 1) {
        pos = t.find(k);
        st = pos != hcd::END;
        if constexpr (Tab::is_map) {
            if (vals_out) vals_out[i] = st ? t.value(pos) : typename Tab::Val();
        }
    } else {
        st = (uint8_t)t.erase(k);
    }
    if (status) status[i] = st;
    if (pos_out) pos_out[i] = pos;
}

// Sets keep the compiler's register count; maps are held to 40 registers per
// thread, which their insert fits without spilling, for more threads (and
// probes) in flight per SM.
template <int KIND>
__global__ void k_apply_set(hc_device_view dv, const uint8_t *ops, int op_all, const typename hcd::Table<KIND>::Key *keys,
                            const typename hcd::Table<KIND>::Val *vals, long long n, uint8_t *status,
                            typename hcd::Table<KIND>::Val *vals_out, long long *pos_out) {
    apply_one<KIND>(dv, ops, op_all, keys, vals, n, status, vals_out, pos_out);
}

template <int KIND>
__global__ void __maxnreg__(40) k_apply_map(hc_device_view dv, const uint8_t *ops, int op_all,
                                            const typename hcd::Table<KIND>::Key *keys,
                                            const typename hcd::Table<KIND>::Val *vals, long long n, uint8_t *status,
                                            typename hcd::Table<KIND>::Val *vals_out, long long *pos_out) {
    apply_one<KIND>(dv, ops, op_all, keys, vals, n, status, vals_out, pos_out);
}

// Block coordinates packed as three signed 21-bit fields (x | y << 21 | z << 42).
__device__ __forceinline__ long long unpack21(unsigned long long key, int field) {
    const long long c = (long long)((key >> (21 * field)) & 0x1FFFFFull);
    return (c ^ 0x100000ll) - 0x100000ll;
}

__device__ __forceinline__ unsigned long long pack21(long long x, long long y, long long z) {
    constexpr unsigned long long M = 0x1FFFFFull;
    return ((unsigned long long)x & M) | (((unsigned long long)y & M) << 21) | (((unsigned long long)z & M) << 42);
}

__global__ void k_update_set(hc_device_view block_map, hc_device_view update_set, const unsigned long long *blocks,
                             long long n) {
    const hcd::Table<HC_MAP_I64_I32> map(block_map);
    const hcd::Table<HC_SET_U64> set(update_set);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long b = blocks[i];
    const long long x = unpack21(b, 0), y = unpack21(b, 1), z = unpack21(b, 2);
    for (int j = 0; j < 8; ++j) {
        const unsigned long long c = pack21(x - (j & 1), y - ((j >> 1) & 1), z - ((j >> 2) & 1));
        if (map.contains(c)) set.insert(c);
    }
}

}  // namespace

// One operation per thread on the table behind *dv.  ops[i] (or op_all when
// ops is NULL): 0 insert, 1 find, 2 erase.  status[i]: the insert or erase
// status (hcd::INSERTED ... NOT_FOUND), or 1 / 0 for a find that found / did
// not find its key.  vals: map insert values (NULL: zeros).  vals_out: find
// values of maps (0 when absent), may be NULL.  pos_out: the position insert
// or find returned (-1 = end), may be NULL.  All arrays are device arrays of
// n entries.  Returns HC_ERR_ARG for a bad argument, HC_ERR_CUDA if the
// launch fails, else HC_OK (asynchronous on `stream`).
HCX_API hc_rc hcx_apply(const hc_device_view *dv, const uint8_t *ops, int32_t op_all, const void *keys,
                        const void *vals, int64_t n, uint8_t *status, void *vals_out, int64_t *pos_out, int32_t block,
                        void *stream) {
    if (!dv || n < 0 || (n > 0 && !keys) || block < 32 || block > 1024 || block % 32 || op_all < 0 || op_all > 2)
        return HC_ERR_ARG;
    if (n == 0) return HC_OK;
    const unsigned grid = (unsigned)((n + block - 1) / block);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    long long *po = reinterpret_cast<long long *>(pos_out);
    switch (dv->kind) {
        case HC_SET_U32:
            k_apply_set<HC_SET_U32><<<grid, block, 0, s>>>(*dv, ops, op_all, (const uint32_t *)keys, nullptr, n, status,
                                                       nullptr, po);
            break;
        case HC_SET_U64:
            k_apply_set<HC_SET_U64><<<grid, block, 0, s>>>(*dv, ops, op_all, (const unsigned long long *)keys, nullptr, n,
                                                       status, nullptr, po);
            break;
        case HC_MAP_I64_I32:
            k_apply_map<HC_MAP_I64_I32><<<grid, block, 0, s>>>(*dv, ops, op_all, (const unsigned long long *)keys,
                                                           (const uint32_t *)vals, n, status, (uint32_t *)vals_out, po);
            break;
        case HC_MAP_U64_U64:
            k_apply_map<HC_MAP_U64_U64><<<grid, block, 0, s>>>(*dv, ops, op_all, (const unsigned long long *)keys,
                                                           (const unsigned long long *)vals, n, status,
                                                           (unsigned long long *)vals_out, po);
            break;
        default: return HC_ERR_ARG;
    }
    return cudaGetLastError() == cudaSuccess ? HC_OK : HC_ERR_CUDA;
}

// Section 4.1's update-set example: block_map is a map<int64,int32> of voxel
// blocks, update_set a set<uint64>; blocks holds n packed block coordinates
// (device array).  Asynchronous on `stream`.
HCX_API hc_rc hcx_update_set(const hc_device_view *block_map, const hc_device_view *update_set, const int64_t *blocks,
                             int64_t n, void *stream) {
    if (!block_map || !update_set || n < 0 || (n > 0 && !blocks) || block_map->kind != HC_MAP_I64_I32 ||
        update_set->kind != HC_SET_U64)
        return HC_ERR_ARG;
    if (n == 0) return HC_OK;
    const int block = 128;
    k_update_set<<<(unsigned)((n + block - 1) / block), block, 0, static_cast<cudaStream_t>(stream)>>>(
        *block_map, *update_set, reinterpret_cast<const unsigned long long *>(blocks), n);
    return cudaGetLastError() == cudaSuccess ? HC_OK : HC_ERR_CUDA;
}
