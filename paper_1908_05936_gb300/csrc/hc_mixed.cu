// hc_mixed.cu -- free-running mixed batches: inserts, finds and erases of one
// call run at once, one operation per thread, through the in-kernel functions
// of include/hc_device.cuh (Section 4, "Guarantees": concurrency across all
// operations).  Per key, the results are those of some serial order of that
// key's operations; inserts claim EMPTY slots only.
#include <algorithm>
#include <cstdint>

#include "hc.h"
#include "hc_device.cuh"
#include "hc_internal.h"

namespace hc {

namespace {

constexpr int kMixedBlock = 256;

// One block takes kMixedBlock consecutive positions and hands them to its
// threads grouped by operation kind (inserts, then finds, then erases), so a
// warp runs one kind's code path instead of all three one after another.
// The call implies no order across positions, so any assignment of positions
// to threads is a valid schedule.
template <int KIND>
__global__ void __launch_bounds__(kMixedBlock)
k_mixed(hc_device_view dv, const uint8_t *ops, const typename Traits<KIND>::Key *keys,
        const typename Traits<KIND>::Val *vals, long long n, uint8_t *status, typename Traits<KIND>::Val *vals_out) {
    using Tab = hcd::Table<KIND>;
    __shared__ unsigned s_count[3];
    __shared__ unsigned s_pos[kMixedBlock];    // tile offset | kind << 16, grouped by kind
    const long long base = (long long)blockIdx.x * kMixedBlock;
    const int tid = threadIdx.x;
    if (tid < 3) s_count[tid] = 0;
    __syncthreads();
    int kind = -1;
    unsigned slot = 0;
    if (base + tid < n) {
        const uint8_t op = __ldcs(ops + base + tid);
        kind = op == OP_INSERT ? 0 : (op == OP_FIND ? 1 : 2);
        slot = atomicAdd(&s_count[kind], 1u);
    }
    __syncthreads();
    if (kind >= 0) {
        const unsigned off = kind == 0 ? 0u : (kind == 1 ? s_count[0] : s_count[0] + s_count[1]);
        s_pos[off + slot] = (unsigned)tid | ((unsigned)kind << 16);
    }
    __syncthreads();
    if ((unsigned)tid >= s_count[0] + s_count[1] + s_count[2]) return;
    const unsigned e = s_pos[tid];
    const long long i = base + (e & 0xFFFFu);
    const Tab t(dv);
    const typename Tab::Key k = __ldcs(keys + i);
    uint8_t st;
    if ((e >> 16) == 0) {
        st = (uint8_t)t.insert(k, (Tab::is_map && vals) ? __ldcs(vals + i) : typename Tab::Val()).status;
    } else if ((e >> 16) == 1) {
        const long long pos = t.find(k);
        st = pos != hcd::END;
        if constexpr (Tab::is_map) {
            if (vals_out) vals_out[i] = st ? t.value(pos) : typename Tab::Val();
        }
    } else {
        st = (uint8_t)t.erase(k);
    }
    if (status) status[i] = st;
}

template <int KIND>
cudaError_t launch(const hc_device_view &dv, const uint8_t *ops, const void *keys, const void *vals, long long n,
                   uint8_t *status, void *vals_out, cudaStream_t s) {
    using T = Traits<KIND>;
    k_mixed<KIND><<<(unsigned)((n + kMixedBlock - 1) / kMixedBlock), kMixedBlock, 0, s>>>(
        dv, ops, (const typename T::Key *)keys, (const typename T::Val *)vals, n, status,
        (typename T::Val *)vals_out);
    return cudaGetLastError();
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
