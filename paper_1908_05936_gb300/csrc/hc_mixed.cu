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

template <int KIND>
__global__ void __launch_bounds__(256)
k_mixed(hc_device_view dv, const uint8_t *ops, const typename Traits<KIND>::Key *keys,
        const typename Traits<KIND>::Val *vals, long long n, uint8_t *status, typename Traits<KIND>::Val *vals_out) {
    using Tab = hcd::Table<KIND>;
    const Tab t(dv);
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint8_t op = __ldcs(ops + i);
    const typename Tab::Key k = __ldcs(keys + i);
    uint8_t st;
    if (op == OP_INSERT) {
        st = (uint8_t)t.insert(k, (Tab::is_map && vals) ? __ldcs(vals + i) : typename Tab::Val()).status;
    } else if (op == OP_FIND) {
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
    const int block = 128;
    k_mixed<KIND><<<(unsigned)((n + block - 1) / block), block, 0, s>>>(
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
