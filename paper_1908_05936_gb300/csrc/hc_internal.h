// hc_internal.h -- declarations shared by the host API and the per-kind
// kernel translation units.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "hc.h"

namespace hc {

struct View;
struct Header;

enum : int { OP_INSERT = 0, OP_FIND = 1, OP_ERASE = 2 };

struct LaunchShape {
    int lane_bytes;       // 16 (maps), 32, 64 or 128
    int keys_per_group;   // 1 or 2
    int block;            // threads per block
    int fold;             // 1 = fold equal keys inside a warp
    int sms;              // multiprocessors of the table's device (grid sizing)
};

#define HC_DECLARE_KIND(NAME)                                                                                       \
    cudaError_t NAME##_range(int op, const View &v, int bb, const void *keys, const void *vals, long long n,        \
                             uint8_t *out, void *vals_out, const LaunchShape &sh, const uint8_t *skip,              \
                             cudaStream_t s);                                                                       \
    cudaError_t NAME##_clear(const View &v, unsigned long long phys, unsigned long long cap, int bb, int sms,       \
                             cudaStream_t s);                                                                       \
    cudaError_t NAME##_rehash(const View &ov, unsigned long long ophys, const View &nv, int bb, int sms,            \
                              cudaStream_t s);

HC_DECLARE_KIND(set_u32)
HC_DECLARE_KIND(set_u64)
HC_DECLARE_KIND(map_i64_i32)
HC_DECLARE_KIND(map_u64_u64)

#undef HC_DECLARE_KIND

// hc_predicate as the selection kernel takes it.
struct SelectPred {
    int kind, negate;
    long long lo, hi;
    int box[6];
};

// Ordered calls (hc_ordered.cu): scratch layout and the leader passes.
unsigned long long ordered_aux_slots(long long n);
long long ordered_scratch_bytes(long long n);
cudaError_t ordered_leaders(const void *keys, int key_bytes, long long n, void *scratch, unsigned *err, int sms,
                            cudaStream_t s);
cudaError_t ordered_follow_insert(long long n, void *scratch, uint8_t *status, int sms, cudaStream_t s);
const uint8_t *ordered_skip(long long n, const void *scratch);

// hc_batch_run with the descriptors written into caller-owned page-locked
// staging of batch_desc_bytes(n_items) (hc_batch.cu).
hc_rc batch_run_pinned(const hc_batch_item *items, int64_t n_items, const hc_batch_config *cfg, void *d_scratch,
                       int64_t scratch_bytes, void *h_pinned, void *stream);
size_t batch_desc_bytes(int64_t n_items);

// One free-running launch of per-thread insert / find / erase (hc_mixed.cu).
cudaError_t mixed_ops(const hc_device_view &dv, const uint8_t *ops, const void *keys, const void *vals, long long n,
                      uint8_t *status, void *vals_out, cudaStream_t s);

// short3 keys <-> packed int64 keys (hc_select.cu).
cudaError_t pack_short3(const int16_t *xyz, long long n, long long *keys, int sms, cudaStream_t s);
cudaError_t unpack_short3(const long long *keys, long long n, int16_t *xyz, int sms, cudaStream_t s);

// Appends the stored entries of the table behind dv that satisfy p (hc_select).
cudaError_t select_entries(const hc_device_view &dv, const SelectPred &p, void *ko, void *vo, unsigned long long cap,
                           unsigned long long *count, unsigned long long positions, int sms, cudaStream_t s);

}  // namespace hc
