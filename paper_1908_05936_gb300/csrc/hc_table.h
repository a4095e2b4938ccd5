// hc_table.h -- host-side record behind the opaque hc_table handle.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hc_core.cuh"
#include "hc_internal.h"

#define HC_TABLE_MAGIC 0x48435442u   // "HCTB"
#define HC_STAGE_CHUNK (1ll << 22)   // keys per staged chunk of the host-buffer calls

struct hc_table {
    uint32_t magic;
    int kind;
    int device;
    int bucket_bytes;
    long long capacity;   // slots as requested
    long long phys;       // slots allocated (whole buckets)
    long long bytes;      // device bytes (header + slots)
    void *d_mem;          // header followed by the slots
    hc::View view;
    hc::LaunchShape shape[3];
    bool shape_set[3] = {false, false, false};   // hc_set_launch was called for the op
    // staging for the host-buffer calls (allocated on first use)
    void *stage_mem = nullptr;
    cudaStream_t copy_stream = nullptr;
    struct Stage {
        void *keys, *vals, *vals_out;
        uint8_t *out;
        cudaEvent_t h2d_done, done;
    } stage[2];
};
