// hc_select.cu -- selection over the stored entries (Section 3.6): the
// library's predicates applied through hcd::copy_if of the in-kernel header,
// one grid whose blocks walk tiles of slot positions and append a tile's
// matches with one atomic.  hc_dump is the selection of every entry.
#include <algorithm>
#include <cstdint>

#include "hc.h"
#include "hc_device.cuh"
#include "hc_internal.h"

namespace hc {

namespace {

__device__ __forceinline__ long long coord21(unsigned long long key, int field) {
    const long long c = (long long)((key >> (21 * field)) & 0x1FFFFFull);
    return (c ^ 0x100000ll) - 0x100000ll;   // sign-extend 21 bits
}

template <int KIND>
struct Selector {
    using T = Traits<KIND>;
    SelectPred p;

    __device__ bool operator()(typename T::Key k, typename T::Val v) const {
        bool r = true;
        switch (p.kind) {
            case HC_PRED_KEY_RANGE:
                if constexpr (KIND == KIND_MAP_I64_I32) r = (long long)k >= p.lo && (long long)k <= p.hi;
                else if constexpr (KIND == KIND_SET_U32) r = k >= (uint32_t)p.lo && k <= (uint32_t)p.hi;
                else r = k >= (unsigned long long)p.lo && k <= (unsigned long long)p.hi;
                break;
            case HC_PRED_VALUE_RANGE:
                if constexpr (KIND == KIND_MAP_I64_I32) r = (long long)(int32_t)v >= p.lo && (long long)(int32_t)v <= p.hi;
                else r = (unsigned long long)v >= (unsigned long long)p.lo && (unsigned long long)v <= (unsigned long long)p.hi;
                break;
            case HC_PRED_KEY_MASK:
                r = ((unsigned long long)k & (unsigned long long)p.lo) == (unsigned long long)p.hi;
                break;
            case HC_PRED_BLOCK_BOX: {
                const long long x = coord21(k, 0), y = coord21(k, 1), z = coord21(k, 2);
                r = x >= p.box[0] && x <= p.box[1] && y >= p.box[2] && y <= p.box[3] && z >= p.box[4] && z <= p.box[5];
                break;
            }
            case HC_PRED_SHORT3_BOX: {
                const long long x = (short)((unsigned long long)k & 0xFFFFull);
                const long long y = (short)(((unsigned long long)k >> 16) & 0xFFFFull);
                const long long z = (short)(((unsigned long long)k >> 32) & 0xFFFFull);
                r = x >= p.box[0] && x <= p.box[1] && y >= p.box[2] && y <= p.box[3] && z >= p.box[4] && z <= p.box[5];
                break;
            }
            default: break;   // HC_PRED_ALL
        }
        return r != (p.negate != 0);
    }
};

template <int KIND>
__global__ void __launch_bounds__(256)
k_select(hc_device_view dv, Selector<KIND> sel, typename Traits<KIND>::Key *keys_out,
         typename Traits<KIND>::Val *vals_out, unsigned long long cap, unsigned long long *count) {
    const hcd::Table<KIND> t(dv);
    hcd::copy_if(t, sel, keys_out, vals_out, cap, count);
}

template <int KIND>
cudaError_t launch(const hc_device_view &dv, const SelectPred &p, void *ko, void *vo, unsigned long long cap,
                   unsigned long long *count, unsigned long long positions, int sms, cudaStream_t s) {
    using T = Traits<KIND>;
    const unsigned long long tiles = (positions + 2047) / 2048;   // 8 positions per thread of a 256-thread block
    const unsigned grid = (unsigned)std::max<unsigned long long>(
        1ull, std::min<unsigned long long>(tiles, (unsigned long long)sms * 8));
    k_select<KIND><<<grid, 256, 0, s>>>(dv, Selector<KIND>{p}, (typename T::Key *)ko, (typename T::Val *)vo, cap,
                                        count);
    return cudaGetLastError();
}

}  // namespace

namespace {

__global__ void __launch_bounds__(256) k_pack_short3(const int16_t *xyz, long long n, long long *keys) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long x = (uint16_t)xyz[3 * i], y = (uint16_t)xyz[3 * i + 1], z = (uint16_t)xyz[3 * i + 2];
        keys[i] = (long long)(x | (y << 16) | (z << 32));
    }
}

__global__ void __launch_bounds__(256) k_unpack_short3(const long long *keys, long long n, int16_t *xyz) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const unsigned long long k = (unsigned long long)keys[i];
        xyz[3 * i] = (int16_t)(k & 0xFFFFull);
        xyz[3 * i + 1] = (int16_t)((k >> 16) & 0xFFFFull);
        xyz[3 * i + 2] = (int16_t)((k >> 32) & 0xFFFFull);
    }
}

unsigned grid_for_items(long long n, int sms) {
    const long long g = (n + 255) / 256;
    return (unsigned)std::max<long long>(1, std::min<long long>(g, (long long)sms * 8));
}

}  // namespace

cudaError_t pack_short3(const int16_t *xyz, long long n, long long *keys, int sms, cudaStream_t s) {
    k_pack_short3<<<grid_for_items(n, sms), 256, 0, s>>>(xyz, n, keys);
    return cudaGetLastError();
}

cudaError_t unpack_short3(const long long *keys, long long n, int16_t *xyz, int sms, cudaStream_t s) {
    k_unpack_short3<<<grid_for_items(n, sms), 256, 0, s>>>(keys, n, xyz);
    return cudaGetLastError();
}

cudaError_t select_entries(const hc_device_view &dv, const SelectPred &p, void *ko, void *vo, unsigned long long cap,
                           unsigned long long *count, unsigned long long positions, int sms, cudaStream_t s) {
    switch (dv.kind) {
        case HC_SET_U32: return launch<KIND_SET_U32>(dv, p, ko, vo, cap, count, positions, sms, s);
        case HC_SET_U64: return launch<KIND_SET_U64>(dv, p, ko, vo, cap, count, positions, sms, s);
        case HC_MAP_I64_I32: return launch<KIND_MAP_I64_I32>(dv, p, ko, vo, cap, count, positions, sms, s);
        default: return launch<KIND_MAP_U64_U64>(dv, p, ko, vo, cap, count, positions, sms, s);
    }
}

}  // namespace hc
