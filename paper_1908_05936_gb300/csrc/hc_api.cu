// hc_api.cu -- host side of the C ABI declared in include/hc.h: argument
// checks (the contracts of Section 3.3 become return codes), table creation
// and destruction (Section 3.7), dispatch of the range calls to the per-kind
// kernels, counters, clear, dump, rehash and the host-buffer forms.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/hc.h"
#include "hc_core.cuh"
#include "hc_internal.h"
#include "hc_table.h"

namespace {

thread_local std::string g_last_error;

hc_rc fail(hc_rc rc, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return rc;
}

hc_rc cuda_fail(cudaError_t e, const char *what) {
    return fail(HC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define HC_CUDA(call, what)                          \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool valid_kind(int kind) { return kind >= HC_SET_U32 && kind <= HC_MAP_U64_U64; }
bool is_map(int kind) { return kind == HC_MAP_I64_I32 || kind == HC_MAP_U64_U64; }
int key_bytes(int kind) { return kind == HC_SET_U32 ? 4 : 8; }
int val_bytes(int kind) { return kind == HC_MAP_I64_I32 ? 4 : (kind == HC_MAP_U64_U64 ? 8 : 0); }
// bytes a slot holds: key plus value
int slot_bytes(int kind) { return valid_kind(kind) ? key_bytes(kind) + val_bytes(kind) : 0; }
// slots per bucket of bb bytes: keys only for sets; for maps the largest
// power of two of (key, value) slots that fits (same rule as the kernels)
int slots_per_bucket(int kind, int bb) {
    if (!is_map(kind)) return bb / key_bytes(kind);
    int n = bb / slot_bytes(kind), p = 1;
    while (p * 2 <= n && p < 16) p *= 2;
    return p;
}
// bytes of a bucket's key region (what a probe reads)
int key_region_bytes(int kind, int bb) { return slots_per_bucket(kind, bb) * key_bytes(kind); }

int sm_count_of(int dev) {
    static std::mutex mu;
    static int cache[64] = {0};
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64) return 148;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        cache[dev] = n;
    }
    return cache[dev];
}

long long l2_bytes_of(int dev) {
    static std::mutex mu;
    static long long cache[64] = {0};
    std::lock_guard<std::mutex> g(mu);
    if (dev < 0 || dev >= 64) return 128ll << 20;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrL2CacheSize, dev) != cudaSuccess || n <= 0) n = 128 << 20;
        cache[dev] = n;
    }
    return cache[dev];
}

hc_rc check_config(int kind, const hc_config *cfg, int *bb, int *hash_mode, unsigned long long *seed) {
    *bb = 32;
    *hash_mode = HC_HASH_MIX64;
    *seed = 0;
    if (cfg) {
        if (cfg->bucket_bytes) *bb = cfg->bucket_bytes;
        *hash_mode = cfg->hash_mode;
        *seed = cfg->seed;
    }
    if (*bb != 32 && *bb != 64 && *bb != 128) return fail(HC_ERR_ARG, "bucket_bytes must be 32, 64 or 128 (got %d)", *bb);
    if (*hash_mode != HC_HASH_MIX64 && *hash_mode != HC_HASH_TESCHNER && *hash_mode != HC_HASH_TESCHNER_SHORT3)
        return fail(HC_ERR_ARG, "unknown hash_mode %d", *hash_mode);
    if (*hash_mode != HC_HASH_MIX64 && kind != HC_MAP_I64_I32)
        return fail(HC_ERR_ARG, "the spatial hash applies to packed int64 block keys (HC_MAP_I64_I32) only");
    return HC_OK;
}

// Device memory of a table: [header 256 B][nb buckets of bb bytes].
struct Geometry {
    long long nb, phys, bytes;
    int pad_from;
};

Geometry geometry(int kind, long long slots, int bb) {
    const long long spb = slots_per_bucket(kind, bb);
    Geometry g;
    g.nb = (slots + spb - 1) / spb;
    g.phys = g.nb * spb;
    g.pad_from = (int)(spb - (g.phys - slots));
    g.bytes = (long long)sizeof(hc::Header) + (g.nb * bb + 255) / 256 * 256;
    return g;
}

hc::View make_view(void *mem, const Geometry &g, unsigned long long seed, int hash_mode) {
    hc::View v;
    v.hdr = static_cast<hc::Header *>(mem);
    v.buckets = static_cast<unsigned char *>(mem) + sizeof(hc::Header);
    v.nb = g.nb;
    v.seed = seed;
    v.hash_mode = hash_mode;
    v.pad_from = g.pad_from;
    v.rotate = 0;
    v.reserved = 0;
    return v;
}

cudaError_t dispatch_range(int kind, int op, const hc::View &v, int bb, const void *keys, const void *vals, long long n,
                           uint8_t *out, void *vals_out, const hc::LaunchShape &sh, const uint8_t *skip,
                           cudaStream_t s) {
    switch (kind) {
        case HC_SET_U32: return hc::set_u32_range(op, v, bb, keys, vals, n, out, vals_out, sh, skip, s);
        case HC_SET_U64: return hc::set_u64_range(op, v, bb, keys, vals, n, out, vals_out, sh, skip, s);
        case HC_MAP_I64_I32: return hc::map_i64_i32_range(op, v, bb, keys, vals, n, out, vals_out, sh, skip, s);
        default: return hc::map_u64_u64_range(op, v, bb, keys, vals, n, out, vals_out, sh, skip, s);
    }
}

cudaError_t dispatch_clear(const hc_table *t, const hc::View &v, long long phys, long long cap, cudaStream_t s) {
    const int sms = sm_count_of(t->device);
    switch (t->kind) {
        case HC_SET_U32: return hc::set_u32_clear(v, phys, cap, t->bucket_bytes, sms, s);
        case HC_SET_U64: return hc::set_u64_clear(v, phys, cap, t->bucket_bytes, sms, s);
        case HC_MAP_I64_I32: return hc::map_i64_i32_clear(v, phys, cap, t->bucket_bytes, sms, s);
        default: return hc::map_u64_u64_clear(v, phys, cap, t->bucket_bytes, sms, s);
    }
}

__global__ void k_set_u64(unsigned long long *p, unsigned long long v) { *p = v; }

__global__ void k_rehash_finish(hc::Header *old_h, hc::Header *new_h) {
    new_h->live = old_h->live;
    new_h->used = new_h->reinserted;
    new_h->err |= old_h->err;
    new_h->side_present[0] = old_h->side_present[0];
    new_h->side_present[1] = old_h->side_present[1];
    new_h->side_val[0] = old_h->side_val[0];
    new_h->side_val[1] = old_h->side_val[1];
}

__global__ void k_clear_err(hc::Header *h) { h->err = 0u; }

hc_rc read_header(hc_table *t, hc::Header *out, cudaStream_t s) {
    HC_CUDA(cudaMemcpyAsync(out, t->d_mem, sizeof(hc::Header), cudaMemcpyDeviceToHost, s), "reading the table header");
    HC_CUDA(cudaStreamSynchronize(s), "synchronising the stream");
    return HC_OK;
}

hc_rc check_table(const hc_table *t) {
    if (!t || t->magic != HC_TABLE_MAGIC) return fail(HC_ERR_ARG, "invalid table handle");
    return HC_OK;
}

hc_rc check_array(const void *p, int align, const char *name) {
    if (!p) return fail(HC_ERR_ARG, "%s is NULL", name);
    if (reinterpret_cast<uintptr_t>(p) % align) return fail(HC_ERR_ARG, "%s is not aligned to %d bytes", name, align);
    return HC_OK;
}

hc_rc range_checks(const hc_table *t, int op, const void *keys, const void *vals, long long n, const void *out,
                   const void *vals_out) {
    hc_rc rc = check_table(t);
    if (rc != HC_OK) return rc;
    if (n < 0) return fail(HC_ERR_ARG, "n must be >= 0 (got %lld)", n);
    if (n == 0) return HC_OK;
    if ((rc = check_array(keys, key_bytes(t->kind), "keys")) != HC_OK) return rc;
    if (op == hc::OP_INSERT && is_map(t->kind) && (rc = check_array(vals, val_bytes(t->kind), "values")) != HC_OK)
        return rc;
    if (op == hc::OP_FIND && !out) return fail(HC_ERR_ARG, "found flags array is NULL");
    if (op == hc::OP_FIND && vals_out && is_map(t->kind) &&
        (rc = check_array(vals_out, val_bytes(t->kind), "values output")) != HC_OK)
        return rc;
    return HC_OK;
}

hc_rc run_range(hc_table *t, int op, const void *keys, const void *vals, long long n, uint8_t *out, void *vals_out,
                cudaStream_t s, const uint8_t *skip = nullptr) {
    hc_rc rc = range_checks(t, op, keys, vals, n, out, vals_out);
    if (rc != HC_OK || n == 0) return rc;
    hc::LaunchShape sh = t->shape[op];
    sh.sms = sm_count_of(t->device);
    hc::View v = t->view;
    v.rotate = n > (long long)v.nb ? 1 : 0;        // several inserters per bucket: spread them
    // Default shape, a plain insert too small to fill the GPU with 4 keys per
    // thread, into a table larger than L2 with at most one inserter per
    // bucket: one key per thread in lock step, which keeps more probes in
    // flight there (measured on a 4 GiB map: +5-12 % for 2^16-2^20 keys).
    // Crowded or L2-resident inserts and inserts that skip keys keep the
    // streaming form (an 8 MiB set<u32> took 2.4x as long in lock step).
    if (op == hc::OP_INSERT && !t->shape_set[op] && !skip && !v.rotate && n < (long long)sh.sms * 8192 &&
        (long long)v.nb * t->bucket_bytes > l2_bytes_of(t->device))
        sh.keys_per_group = 1;
    cudaError_t e = dispatch_range(t->kind, op, v, t->bucket_bytes, keys, is_map(t->kind) ? vals : nullptr, n,
                                   out, is_map(t->kind) ? vals_out : nullptr, sh, skip, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the range kernel");
    return HC_OK;
}

// Host-buffer forms: chunked copies through two staging buffer sets, the
// copy of chunk i+1 overlapping the kernel of chunk i.
hc_rc ensure_staging(hc_table *t) {
    if (t->stage_mem) return HC_OK;
    const long long C = HC_STAGE_CHUNK;
    const long long per = C * (key_bytes(t->kind) + 2 * 8 + 1) + 1024;
    HC_CUDA(cudaMalloc(&t->stage_mem, 2 * per), "allocating host-call staging buffers");
    for (int i = 0; i < 2; ++i) {
        unsigned char *base = static_cast<unsigned char *>(t->stage_mem) + i * per;
        t->stage[i].keys = base;
        t->stage[i].vals = base + C * key_bytes(t->kind);
        t->stage[i].vals_out = base + C * (key_bytes(t->kind) + 8);
        t->stage[i].out = reinterpret_cast<uint8_t *>(base + C * (key_bytes(t->kind) + 16));
        HC_CUDA(cudaEventCreateWithFlags(&t->stage[i].h2d_done, cudaEventDisableTiming), "creating events");
        HC_CUDA(cudaEventCreateWithFlags(&t->stage[i].done, cudaEventDisableTiming), "creating events");
    }
    HC_CUDA(cudaStreamCreateWithFlags(&t->copy_stream, cudaStreamNonBlocking), "creating the copy stream");
    return HC_OK;
}

// The device address of a page-locked host buffer (registered or allocated by
// CUDA), or nullptr for pageable memory.
void *mapped(const void *h) {
    if (!h) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

hc_rc run_host(hc_table *t, int op, const void *h_keys, const void *h_vals, long long n, uint8_t *h_out,
               void *h_vals_out, cudaStream_t s) {
    hc_rc rc = check_table(t);
    if (rc != HC_OK) return rc;
    if (n < 0) return fail(HC_ERR_ARG, "n must be >= 0 (got %lld)", n);
    if (n == 0) return HC_OK;
    if (!h_keys) return fail(HC_ERR_ARG, "keys is NULL");
    if (op == hc::OP_INSERT && is_map(t->kind) && !h_vals) return fail(HC_ERR_ARG, "values is NULL");
    if (op == hc::OP_FIND && !h_out) return fail(HC_ERR_ARG, "found flags array is NULL");
    {
        // Page-locked buffers: the kernels read the keys and write the results
        // in host memory directly (over NVLink-C2C on GB300), one launch for
        // the whole call, no staging copies.
        const bool want_vals = op == hc::OP_FIND && is_map(t->kind) && h_vals_out;
        void *dk = mapped(h_keys);
        void *dv = (op == hc::OP_INSERT && is_map(t->kind)) ? mapped(h_vals) : nullptr;
        void *dout = mapped(h_out);
        void *dvo = want_vals ? mapped(h_vals_out) : nullptr;
        const bool ok = dk && (op != hc::OP_INSERT || !is_map(t->kind) || dv) && (!h_out || dout) &&
                        (!want_vals || dvo);
        if (ok) {
            if ((rc = run_range(t, op, dk, dv, n, static_cast<uint8_t *>(dout), dvo, s)) != HC_OK) return rc;
            HC_CUDA(cudaStreamSynchronize(s), "synchronising the stream");
            return HC_OK;
        }
    }
    if ((rc = ensure_staging(t)) != HC_OK) return rc;
    const int kb = key_bytes(t->kind), vb = val_bytes(t->kind);
    const long long C = HC_STAGE_CHUNK;
    for (long long off = 0, i = 0; off < n; off += C, ++i) {
        auto &st = t->stage[i & 1];
        const long long m = std::min(C, n - off);
        if (i >= 2) HC_CUDA(cudaStreamWaitEvent(t->copy_stream, st.done, 0), "ordering the staging buffers");
        HC_CUDA(cudaMemcpyAsync(st.keys, static_cast<const unsigned char *>(h_keys) + off * kb, m * kb,
                                cudaMemcpyHostToDevice, t->copy_stream), "copying keys to the device");
        if (op == hc::OP_INSERT && vb)
            HC_CUDA(cudaMemcpyAsync(st.vals, static_cast<const unsigned char *>(h_vals) + off * vb, m * vb,
                                    cudaMemcpyHostToDevice, t->copy_stream), "copying values to the device");
        HC_CUDA(cudaEventRecord(st.h2d_done, t->copy_stream), "recording an event");
        HC_CUDA(cudaStreamWaitEvent(s, st.h2d_done, 0), "ordering the copy before the kernel");
        const bool want_out = h_out != nullptr;
        const bool want_vals = op == hc::OP_FIND && vb && h_vals_out;
        rc = run_range(t, op, st.keys, st.vals, m, want_out ? st.out : nullptr, want_vals ? st.vals_out : nullptr, s);
        if (rc != HC_OK) return rc;
        if (want_out)
            HC_CUDA(cudaMemcpyAsync(h_out + off, st.out, m, cudaMemcpyDeviceToHost, s), "copying results to the host");
        if (want_vals)
            HC_CUDA(cudaMemcpyAsync(static_cast<unsigned char *>(h_vals_out) + off * vb, st.vals_out, m * vb,
                                    cudaMemcpyDeviceToHost, s), "copying values to the host");
        HC_CUDA(cudaEventRecord(st.done, s), "recording an event");
    }
    HC_CUDA(cudaStreamSynchronize(s), "synchronising the stream");
    return HC_OK;
}

}  // namespace

hc_rc hc_internal_fail(hc_rc rc, const char *msg) {
    g_last_error = msg;
    return rc;
}

extern "C" {

int32_t hc_abi_version(void) { return HC_ABI_VERSION; }

const char *hc_last_error(void) { return g_last_error.c_str(); }

hc_rc hc_table_bytes(int32_t kind, int64_t slots, const hc_config *cfg, int64_t *bytes) {
    if (!valid_kind(kind)) return fail(HC_ERR_ARG, "unknown kind %d", kind);
    if (slots < 1) return fail(HC_ERR_ARG, "slots must be >= 1 (got %lld)", (long long)slots);
    if (!bytes) return fail(HC_ERR_ARG, "bytes is NULL");
    int bb, hm;
    unsigned long long seed;
    hc_rc rc = check_config(kind, cfg, &bb, &hm, &seed);
    if (rc != HC_OK) return rc;
    *bytes = geometry(kind, slots, bb).bytes;
    return HC_OK;
}

hc_rc hc_create(hc_table **out, int32_t kind, int64_t slots, const hc_config *cfg, void *stream) {
    if (!out) return fail(HC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!valid_kind(kind)) return fail(HC_ERR_ARG, "unknown kind %d", kind);
    if (slots < 1) return fail(HC_ERR_ARG, "slots must be >= 1 (got %lld)", (long long)slots);
    int bb, hm;
    unsigned long long seed;
    hc_rc rc = check_config(kind, cfg, &bb, &hm, &seed);
    if (rc != HC_OK) return rc;
    const Geometry g = geometry(kind, slots, bb);
    hc_table *t = new hc_table();
    t->magic = HC_TABLE_MAGIC;
    t->kind = kind;
    t->capacity = slots;
    t->phys = g.phys;
    t->bytes = g.bytes;
    t->bucket_bytes = bb;
    HC_CUDA(cudaGetDevice(&t->device), "cudaGetDevice");
    cudaError_t e = cudaMalloc(&t->d_mem, g.bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        delete t;
        return fail(HC_ERR_OOM, "cudaMalloc of %lld bytes failed: %s", (long long)g.bytes, cudaGetErrorString(e));
    }
    t->view = make_view(t->d_mem, g, seed, hm);
    // the streaming kernels, one thread per key reading the bucket's keys,
    // 4 keys per thread with 2 probes in flight, 64-thread blocks: the best
    // shape of the sweeps on GB300 for uniform keys, for every kind and op.
    for (int op = 0; op < 3; ++op) t->shape[op] = hc::LaunchShape{key_region_bytes(kind, bb), 4, 64, 0, 0};
    e = dispatch_clear(t, t->view, t->phys, t->capacity, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        cudaFree(t->d_mem);
        delete t;
        return cuda_fail(e, "initialising the table");
    }
    *out = t;
    return HC_OK;
}

hc_rc hc_destroy(hc_table *t) {
    if (!t) return HC_OK;
    hc_rc rc = check_table(t);
    if (rc != HC_OK) return rc;
    t->magic = 0;
    cudaError_t e = cudaFree(t->d_mem);   // cudaFree waits for work queued on the device
    if (t->stage_mem) {
        cudaFree(t->stage_mem);
        for (int i = 0; i < 2; ++i) {
            cudaEventDestroy(t->stage[i].h2d_done);
            cudaEventDestroy(t->stage[i].done);
        }
        cudaStreamDestroy(t->copy_stream);
    }
    delete t;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFree");
    return HC_OK;
}

hc_rc hc_set_launch(hc_table *t, int32_t op, const hc_launch *shape) {
    hc_rc rc = check_table(t);
    if (rc != HC_OK) return rc;
    if (op < 0 || op > 2 || !shape) return fail(HC_ERR_ARG, "bad op or NULL shape");
    hc::LaunchShape sh = t->shape[op];
    if (shape->lane_bytes) sh.lane_bytes = shape->lane_bytes;
    if (shape->keys_per_group) sh.keys_per_group = shape->keys_per_group;
    if (shape->block) sh.block = shape->block;
    if (shape->fold_duplicates) sh.fold = shape->fold_duplicates == 1 ? 1 : 0;
    const int krb = key_region_bytes(t->kind, t->bucket_bytes);
    const bool full = is_map(t->kind) && sh.lane_bytes == t->bucket_bytes;   // keys and values in one read
    const bool lb_ok = (sh.lane_bytes == 16 && is_map(t->kind)) || sh.lane_bytes == 32 || sh.lane_bytes == 64 ||
                       sh.lane_bytes == 128;
    if (!full && (!lb_ok || sh.lane_bytes > krb))
        return fail(HC_ERR_ARG,
                    "lane_bytes must be 32, 64 or 128 (16 for maps) and at most the %d-byte key region, or the whole "
                    "bucket for maps", krb);
    if (sh.keys_per_group != 1 && sh.keys_per_group != 2 &&
        !((sh.keys_per_group == 4 || sh.keys_per_group == 8) &&
          (sh.lane_bytes == krb || (op == hc::OP_FIND && is_map(t->kind) && sh.lane_bytes == t->bucket_bytes &&
                                    2 * krb == t->bucket_bytes))))
        return fail(HC_ERR_ARG,
                    "keys_per_group must be 1 or 2 (4 or 8: streaming, lane = the key region, or the whole bucket for map lookups)");
    if (sh.block < 64 || sh.block > 256 || sh.block % 32)
        return fail(HC_ERR_ARG, "block must be a multiple of 32 in [64, 256]");
    t->shape[op] = sh;
    if (shape->lane_bytes || shape->keys_per_group || shape->block || shape->fold_duplicates) t->shape_set[op] = true;
    return HC_OK;
}

hc_rc hc_get_launch(const hc_table *t, int32_t op, hc_launch *shape) {
    hc_rc rc = check_table(t);
    if (rc != HC_OK) return rc;
    if (op < 0 || op > 2 || !shape) return fail(HC_ERR_ARG, "bad op or NULL shape");
    const hc::LaunchShape &sh = t->shape[op];
    shape->lane_bytes = sh.lane_bytes;
    shape->keys_per_group = sh.keys_per_group;
    shape->block = sh.block;
    shape->fold_duplicates = sh.fold ? 1 : 2;
    return HC_OK;
}

hc_rc hc_insert(hc_table *t, const void *d_keys, const void *d_vals, int64_t n, uint8_t *d_status, void *stream) {
    return run_range(t, hc::OP_INSERT, d_keys, d_vals, n, d_status, nullptr, static_cast<cudaStream_t>(stream));
}

hc_rc hc_insert_if_absent(hc_table *t, const void *d_keys, const void *d_vals, const uint8_t *d_found, int64_t n,
                          uint8_t *d_status, void *stream) {
    if (n > 0 && !d_found) return fail(HC_ERR_ARG, "found flags array is NULL");
    return run_range(t, hc::OP_INSERT, d_keys, d_vals, n, d_status, nullptr, static_cast<cudaStream_t>(stream),
                     d_found);
}

hc_rc hc_find(hc_table *t, const void *d_keys, int64_t n, uint8_t *d_found, void *d_vals_out, void *stream) {
    return run_range(t, hc::OP_FIND, d_keys, nullptr, n, d_found, d_vals_out, static_cast<cudaStream_t>(stream));
}

hc_rc hc_erase(hc_table *t, const void *d_keys, int64_t n, uint8_t *d_status, void *stream) {
    return run_range(t, hc::OP_ERASE, d_keys, nullptr, n, d_status, nullptr, static_cast<cudaStream_t>(stream));
}

hc_rc hc_insert_host(hc_table *t, const void *h_keys, const void *h_vals, int64_t n, uint8_t *h_status, void *stream) {
    return run_host(t, hc::OP_INSERT, h_keys, h_vals, n, h_status, nullptr, static_cast<cudaStream_t>(stream));
}

hc_rc hc_find_host(hc_table *t, const void *h_keys, int64_t n, uint8_t *h_found, void *h_vals_out, void *stream) {
    return run_host(t, hc::OP_FIND, h_keys, nullptr, n, h_found, h_vals_out, static_cast<cudaStream_t>(stream));
}

hc_rc hc_erase_host(hc_table *t, const void *h_keys, int64_t n, uint8_t *h_status, void *stream) {
    return run_host(t, hc::OP_ERASE, h_keys, nullptr, n, h_status, nullptr, static_cast<cudaStream_t>(stream));
}

hc_rc hc_stats(hc_table *t, hc_stats_t *out, void *stream) {
    hc_rc rc = check_table(t);
    if (rc != HC_OK) return rc;
    if (!out) return fail(HC_ERR_ARG, "out is NULL");
    hc::Header h;
    if ((rc = read_header(t, &h, static_cast<cudaStream_t>(stream))) != HC_OK) return rc;
    out->live = (int64_t)h.live;
    out->used = (int64_t)h.used;
    out->capacity = t->capacity;
    out->slot_bytes = slot_bytes(t->kind);
    out->table_bytes = t->bytes;
    out->error_bits = h.err;
    out->reserved = 0;
    return HC_OK;
}

hc_rc hc_size(hc_table *t, int64_t *live, void *stream) {
    if (!live) return fail(HC_ERR_ARG, "live is NULL");
    hc_stats_t st;
    hc_rc rc = hc_stats(t, &st, stream);
    if (rc == HC_OK) *live = st.live;
    return rc;
}

hc_rc hc_status(hc_table *t, void *stream) {
    hc_stats_t st;
    hc_rc rc = hc_stats(t, &st, stream);
    if (rc != HC_OK) return rc;
    if (st.error_bits) {
        k_clear_err<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(t->view.hdr);
        HC_CUDA(cudaGetLastError(), "clearing the error bits");
        HC_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)), "synchronising the stream");
    }
    if (st.error_bits & hc::ERR_DEBUG_BOUNDS) return fail(HC_ERR_STATE, "a debug bounds check failed");
    if (st.error_bits & hc::ERR_PROBE_BOUND) return fail(HC_ERR_STATE, "a device-side probe bound was reached");
    if (st.error_bits & hc::ERR_OVERFLOW) return fail(HC_ERR_OVERFLOW, "an insert found the table full");
    return HC_OK;
}

hc_rc hc_clear(hc_table *t, void *stream) {
    hc_rc rc = check_table(t);
    if (rc != HC_OK) return rc;
    cudaError_t e = dispatch_clear(t, t->view, t->phys, t->capacity, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "clearing the table");
    return HC_OK;
}

hc_rc hc_rehash(hc_table *t, int64_t new_slots, void *stream) {
    hc_rc rc = check_table(t);
    if (rc != HC_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (new_slots < 1) return fail(HC_ERR_ARG, "new_slots must be >= 1");
    hc::Header h;
    if ((rc = read_header(t, &h, s)) != HC_OK) return rc;
    const long long regular = (long long)h.live - (long long)h.side_present[0] - (long long)h.side_present[1];
    if (new_slots < regular)
        return fail(HC_ERR_ARG, "new_slots %lld is below the %lld stored keys", (long long)new_slots, regular);
    const Geometry g = geometry(t->kind, new_slots, t->bucket_bytes);
    void *mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, g.bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(HC_ERR_OOM, "cudaMalloc of %lld bytes failed: %s", (long long)g.bytes, cudaGetErrorString(e));
    }
    hc::View nv = make_view(mem, g, t->view.seed, t->view.hash_mode);
    e = dispatch_clear(t, nv, g.phys, new_slots, s);
    const int sms = sm_count_of(t->device);
    if (e == cudaSuccess) {
        switch (t->kind) {
            case HC_SET_U32: e = hc::set_u32_rehash(t->view, t->phys, nv, t->bucket_bytes, sms, s); break;
            case HC_SET_U64: e = hc::set_u64_rehash(t->view, t->phys, nv, t->bucket_bytes, sms, s); break;
            case HC_MAP_I64_I32: e = hc::map_i64_i32_rehash(t->view, t->phys, nv, t->bucket_bytes, sms, s); break;
            default: e = hc::map_u64_u64_rehash(t->view, t->phys, nv, t->bucket_bytes, sms, s); break;
        }
    }
    if (e == cudaSuccess) {
        k_rehash_finish<<<1, 1, 0, s>>>(t->view.hdr, nv.hdr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(mem);
        return cuda_fail(e, "rehashing");
    }
    cudaFree(t->d_mem);
    t->d_mem = mem;
    t->view = nv;
    t->capacity = new_slots;
    t->phys = g.phys;
    t->bytes = g.bytes;
    return HC_OK;
}

static void fill_view(const hc_table *t, hc_device_view *out);

hc_rc hc_dump(hc_table *t, void *d_keys_out, void *d_vals_out, int64_t cap, int64_t *n_out, void *stream) {
    hc_rc rc = check_table(t);
    if (rc != HC_OK) return rc;
    if (!n_out) return fail(HC_ERR_ARG, "n_out is NULL");
    if (cap < 0) return fail(HC_ERR_ARG, "cap must be >= 0");
    if (cap > 0 && (rc = check_array(d_keys_out, key_bytes(t->kind), "keys output")) != HC_OK) return rc;
    if (cap > 0 && d_vals_out && is_map(t->kind) &&
        (rc = check_array(d_vals_out, val_bytes(t->kind), "values output")) != HC_OK)
        return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_set_u64<<<1, 1, 0, s>>>(&t->view.hdr->dump_count, 0ull);
    HC_CUDA(cudaGetLastError(), "resetting the dump cursor");
    // the selection of every stored entry, appended through the header's cursor
    hc_device_view dv{};
    fill_view(t, &dv);
    const hc::SelectPred all{HC_PRED_ALL, 0, 0, 0, {}};
    const cudaError_t e = hc::select_entries(dv, all, d_keys_out, is_map(t->kind) ? d_vals_out : nullptr,
                                             (unsigned long long)cap, &t->view.hdr->dump_count,
                                             (unsigned long long)t->phys + 2ull, sm_count_of(t->device), s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the dump kernel");
    hc::Header h;
    if ((rc = read_header(t, &h, s)) != HC_OK) return rc;
    *n_out = (int64_t)h.dump_count;
    if ((long long)h.dump_count > cap)
        return fail(HC_ERR_ARG, "%lld stored keys do not fit the %lld output entries", (long long)h.dump_count,
                    (long long)cap);
    return HC_OK;
}


int64_t hc_ordered_scratch_bytes(int64_t n) {
    if (n < 0) return -1;
    return (int64_t)hc::ordered_scratch_bytes(n);
}

static hc_rc ordered_checks(const hc_table *t, int op, const void *keys, const void *vals, long long n,
                            const void *scratch, int64_t scratch_bytes) {
    hc_rc rc = range_checks(t, op, keys, vals, n, nullptr, nullptr);
    if (rc != HC_OK || n == 0) return rc;
    if (!scratch) return fail(HC_ERR_ARG, "scratch is NULL");
    if ((rc = check_array(scratch, 256, "scratch")) != HC_OK) return rc;
    if (scratch_bytes < hc_ordered_scratch_bytes(n))
        return fail(HC_ERR_ARG, "scratch of %lld bytes is below the %lld that %lld keys need", (long long)scratch_bytes,
                    (long long)hc_ordered_scratch_bytes(n), n);
    return HC_OK;
}

hc_rc hc_insert_ordered(hc_table *t, const void *d_keys, const void *d_vals, int64_t n, uint8_t *d_status,
                        void *d_scratch, int64_t scratch_bytes, void *stream) {
    hc_rc rc = ordered_checks(t, hc::OP_INSERT, d_keys, d_vals, n, d_scratch, scratch_bytes);
    if (rc != HC_OK || n == 0) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int sms = sm_count_of(t->device);
    cudaError_t e = hc::ordered_leaders(d_keys, key_bytes(t->kind), n, d_scratch, &t->view.hdr->err, sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "finding the first occurrences");
    if ((rc = run_range(t, hc::OP_INSERT, d_keys, d_vals, n, d_status, nullptr, s, hc::ordered_skip(n, d_scratch))) !=
        HC_OK)
        return rc;
    if (d_status) {
        e = hc::ordered_follow_insert(n, d_scratch, d_status, sms, s);
        if (e != cudaSuccess) return cuda_fail(e, "copying the first occurrences' results");
    }
    return HC_OK;
}

hc_rc hc_erase_ordered(hc_table *t, const void *d_keys, int64_t n, uint8_t *d_status, void *d_scratch,
                       int64_t scratch_bytes, void *stream) {
    hc_rc rc = ordered_checks(t, hc::OP_ERASE, d_keys, nullptr, n, d_scratch, scratch_bytes);
    if (rc != HC_OK || n == 0) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int sms = sm_count_of(t->device);
    cudaError_t e = hc::ordered_leaders(d_keys, key_bytes(t->kind), n, d_scratch, &t->view.hdr->err, sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "finding the first occurrences");
    // the streaming erase takes the skip flags (later occurrences: NOT_FOUND)
    hc::LaunchShape sh{key_region_bytes(t->kind, t->bucket_bytes), 4, 64, 0, sms};
    e = dispatch_range(t->kind, hc::OP_ERASE, t->view, t->bucket_bytes, d_keys, nullptr, n, d_status, nullptr, sh,
                       hc::ordered_skip(n, d_scratch), s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the erase kernel");
    return HC_OK;
}

hc_rc hc_select(hc_table *t, const hc_predicate *pred, void *d_keys_out, void *d_vals_out, int64_t cap,
                int64_t *d_count, void *stream) {
    hc_rc rc = check_table(t);
    if (rc != HC_OK) return rc;
    if (!pred) return fail(HC_ERR_ARG, "pred is NULL");
    if (!d_count) return fail(HC_ERR_ARG, "d_count is NULL");
    if ((rc = check_array(d_count, 8, "d_count")) != HC_OK) return rc;
    if (cap < 0) return fail(HC_ERR_ARG, "cap must be >= 0");
    if (pred->kind < HC_PRED_ALL || pred->kind > HC_PRED_SHORT3_BOX)
        return fail(HC_ERR_ARG, "unknown predicate kind %d", pred->kind);
    if (pred->negate != 0 && pred->negate != 1) return fail(HC_ERR_ARG, "negate must be 0 or 1");
    if (pred->kind == HC_PRED_VALUE_RANGE && !is_map(t->kind))
        return fail(HC_ERR_ARG, "HC_PRED_VALUE_RANGE needs a map");
    if ((pred->kind == HC_PRED_BLOCK_BOX || pred->kind == HC_PRED_SHORT3_BOX) && t->kind == HC_SET_U32)
        return fail(HC_ERR_ARG, "a box predicate needs 64-bit keys");
    if (cap > 0 && (rc = check_array(d_keys_out, key_bytes(t->kind), "keys output")) != HC_OK) return rc;
    if (cap > 0 && d_vals_out && is_map(t->kind) &&
        (rc = check_array(d_vals_out, val_bytes(t->kind), "values output")) != HC_OK)
        return rc;
    hc_device_view dv{};
    fill_view(t, &dv);
    hc::SelectPred p{pred->kind, pred->negate, (long long)pred->lo, (long long)pred->hi, {}};
    for (int i = 0; i < 6; ++i) p.box[i] = pred->box[i];
    const cudaError_t e = hc::select_entries(dv, p, d_keys_out, is_map(t->kind) ? d_vals_out : nullptr,
                                             (unsigned long long)cap, reinterpret_cast<unsigned long long *>(d_count),
                                             (unsigned long long)t->phys + 2ull, sm_count_of(t->device),
                                             static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "launching the selection kernel");
    return HC_OK;
}

static void fill_view(const hc_table *t, hc_device_view *out) {
    out->buckets = t->view.buckets;
    out->header = t->view.hdr;
    out->nb = t->view.nb;
    out->seed = t->view.seed;
    out->kind = t->kind;
    out->bucket_bytes = t->bucket_bytes;
    out->hash_mode = t->view.hash_mode;
    out->pad_from = t->view.pad_from;
}

hc_rc hc_pack_short3(const int16_t *d_xyz, int64_t n, int64_t *d_keys, void *stream) {
    if (n < 0) return fail(HC_ERR_ARG, "n must be >= 0 (got %lld)", (long long)n);
    if (n == 0) return HC_OK;
    hc_rc rc;
    if ((rc = check_array(d_xyz, 2, "short3 array")) != HC_OK) return rc;
    if ((rc = check_array(d_keys, 8, "keys")) != HC_OK) return rc;
    int dev = 0;
    HC_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    HC_CUDA(hc::pack_short3(d_xyz, n, reinterpret_cast<long long *>(d_keys), sm_count_of(dev),
                            static_cast<cudaStream_t>(stream)),
            "launching the short3 packing kernel");
    return HC_OK;
}

hc_rc hc_unpack_short3(const int64_t *d_keys, int64_t n, int16_t *d_xyz, void *stream) {
    if (n < 0) return fail(HC_ERR_ARG, "n must be >= 0 (got %lld)", (long long)n);
    if (n == 0) return HC_OK;
    hc_rc rc;
    if ((rc = check_array(d_keys, 8, "keys")) != HC_OK) return rc;
    if ((rc = check_array(d_xyz, 2, "short3 array")) != HC_OK) return rc;
    int dev = 0;
    HC_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    HC_CUDA(hc::unpack_short3(reinterpret_cast<const long long *>(d_keys), n, d_xyz, sm_count_of(dev),
                              static_cast<cudaStream_t>(stream)),
            "launching the short3 unpacking kernel");
    return HC_OK;
}

hc_rc hc_device_view_get(hc_table *t, hc_device_view *out, void *stream) {
    hc_rc rc = check_table(t);
    if (rc != HC_OK) return rc;
    if (!out) return fail(HC_ERR_ARG, "out is NULL");
    fill_view(t, out);
    return HC_OK;
}

hc_rc hc_apply_mixed(hc_table *t, const uint8_t *d_ops, const void *d_keys, const void *d_vals, int64_t n,
                     uint8_t *d_status, void *d_vals_out, void *stream) {
    hc_rc rc = check_table(t);
    if (rc != HC_OK) return rc;
    if (n < 0) return fail(HC_ERR_ARG, "n must be >= 0 (got %lld)", (long long)n);
    if (n == 0) return HC_OK;
    if (!d_ops) return fail(HC_ERR_ARG, "ops array is NULL");
    if ((rc = check_array(d_keys, key_bytes(t->kind), "keys")) != HC_OK) return rc;
    if (is_map(t->kind) && (rc = check_array(d_vals, val_bytes(t->kind), "values")) != HC_OK) return rc;
    if (d_vals_out && is_map(t->kind) && (rc = check_array(d_vals_out, val_bytes(t->kind), "values output")) != HC_OK)
        return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    hc_device_view dv{};
    fill_view(t, &dv);
    const cudaError_t e = hc::mixed_ops(dv, d_ops, d_keys, is_map(t->kind) ? d_vals : nullptr, n, d_status,
                                        is_map(t->kind) ? d_vals_out : nullptr, s);
    if (e != cudaSuccess) return cuda_fail(e, "launching the mixed kernel");
    return HC_OK;
}

}  // extern "C"
