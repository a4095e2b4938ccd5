// hc_serve.cu -- the served form: a continuous-batching request loop over
// resident tables, run natively on the calling host thread (see the hc.h
// section "served form" for the steps).  All device work is the library's
// own range calls and batched launch; this file schedules them.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "hc.h"
#include "hc_internal.h"
#include "hc_table.h"

hc_rc hc_internal_fail(hc_rc rc, const char *msg);

namespace {

constexpr uint32_t kServerMagic = 0x48435356u;   // "HCSV"
constexpr int64_t kPackLimit = 1 << 16;          // requests up to this many keys are packed into one copy

hc_rc sfail(hc_rc rc, const std::string &msg) { return hc_internal_fail(rc, msg.c_str()); }

hc_rc scuda(cudaError_t e, const char *what) {
    return sfail(HC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int64_t round256(int64_t x) { return (x + 255) / 256 * 256; }

int key_bytes(int kind) { return kind == HC_SET_U32 ? 4 : 8; }
int val_bytes(int kind) { return kind == HC_MAP_I64_I32 ? 4 : (kind == HC_MAP_U64_U64 ? 8 : 0); }

// Where one request's arrays sit inside a slot.
struct Placed {
    int64_t req;
    int64_t k_off, v_off;          // device offsets of the inputs (v_off < 0: none)
    int64_t o_off, vo_off;         // device offsets of the outputs (vo_off < 0: none)
    bool packed;                   // inputs copied through the slot's host staging
    bool direct_out;               // outputs copied straight into the request's page-locked arrays
};

bool page_locked(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

struct Slot {
    int lane = 0;
    unsigned char *d_buf = nullptr;    // device staging
    unsigned char *h_in = nullptr;     // pinned host staging of packed inputs
    unsigned char *h_out = nullptr;    // pinned host staging of outputs
    void *desc = nullptr;              // descriptor scratch of hc_batch_run
    int64_t desc_bytes = 0;
    void *h_desc = nullptr;            // pinned staging of the descriptors (copied without waiting)
    cudaEvent_t done = nullptr;
    bool busy = false;
    int64_t out_begin = 0, out_end = 0;
    std::vector<Placed> placed;
    std::vector<hc_batch_item> items;
};

}  // namespace

struct hc_server {
    uint32_t magic;
    std::vector<hc_table *> tables;
    int lanes, depth, merge, max_items;
    int64_t slot_bytes;
    hc_batch_config batch;
    std::vector<cudaStream_t> streams;
    std::vector<Slot> slots;
    std::vector<bool> out_locked;      // per request of the current run: its outputs are page-locked
};

namespace {

void release(hc_server *s) {
    for (Slot &sl : s->slots) {
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.d_buf) cudaFree(sl.d_buf);
        if (sl.desc) cudaFree(sl.desc);
        if (sl.h_in) cudaFreeHost(sl.h_in);
        if (sl.h_out) cudaFreeHost(sl.h_out);
        if (sl.h_desc) cudaFreeHost(sl.h_desc);
    }
    for (cudaStream_t st : s->streams)
        if (st) cudaStreamDestroy(st);
    s->magic = 0;
    delete s;
}

// Device bytes a request takes in a slot: inputs, then outputs.
void need(const hc_server *s, const hc_request &r, int64_t *in, int64_t *out) {
    const int kind = s->tables[r.table]->kind;
    const int kb = key_bytes(kind), vb = val_bytes(kind);
    *in = round256(r.n * kb) + ((r.op == HC_OP_INSERT && vb) ? round256(r.n * vb) : 0);
    *out = round256(r.n) + ((r.op == HC_OP_FIND && vb) ? round256(r.n * vb) : 0);
}

hc_rc launch(hc_server *s, Slot &sl, hc_request *reqs, const std::vector<int64_t> &batch) {
    cudaStream_t st = s->streams[sl.lane];
    sl.placed.clear();
    int64_t off = 0, packed_end = 0;
    for (int64_t ri : batch) {
        const hc_request &r = reqs[ri];
        const int kind = s->tables[r.table]->kind;
        const int kb = key_bytes(kind), vb = val_bytes(kind);
        int64_t in, out;
        need(s, r, &in, &out);
        Placed p{ri, off, (r.op == HC_OP_INSERT && vb) ? off + round256(r.n * kb) : -1, 0, -1, r.n <= kPackLimit,
                 r.n > kPackLimit && s->out_locked[(size_t)ri]};
        if (p.packed) {
            std::memcpy(sl.h_in + p.k_off, r.h_keys, (size_t)(r.n * kb));
            if (p.v_off >= 0) std::memcpy(sl.h_in + p.v_off, r.h_vals, (size_t)(r.n * vb));
            packed_end = off + in;
        }
        sl.placed.push_back(p);
        off += in;
    }
    // outputs: the ones that go through the host staging first (one copy
    // back for all of them), then the ones copied straight into page-locked
    // request arrays
    int64_t o = round256(off);
    sl.out_begin = o;
    for (int pass = 0; pass < 2; ++pass) {
        for (Placed &p : sl.placed) {
            if (p.direct_out != (pass == 1)) continue;
            const hc_request &r = reqs[p.req];
            const int vb = val_bytes(s->tables[r.table]->kind);
            p.o_off = o;
            p.vo_off = (r.op == HC_OP_FIND && vb) ? o + round256(r.n) : -1;
            int64_t in, out;
            need(s, r, &in, &out);
            o += out;
        }
        if (pass == 0) sl.out_end = o;
    }
    cudaError_t e = cudaSuccess;
    if (packed_end > 0) e = cudaMemcpyAsync(sl.d_buf, sl.h_in, (size_t)packed_end, cudaMemcpyHostToDevice, st);
    for (const Placed &p : sl.placed) {
        if (p.packed || e != cudaSuccess) continue;
        const hc_request &r = reqs[p.req];
        const int kind = s->tables[r.table]->kind;
        e = cudaMemcpyAsync(sl.d_buf + p.k_off, r.h_keys, (size_t)(r.n * key_bytes(kind)), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && p.v_off >= 0)
            e = cudaMemcpyAsync(sl.d_buf + p.v_off, r.h_vals, (size_t)(r.n * val_bytes(kind)), cudaMemcpyHostToDevice,
                                st);
    }
    if (e != cudaSuccess) return scuda(e, "copying request inputs to the device");
    sl.items.clear();
    for (const Placed &p : sl.placed) {
        const hc_request &r = reqs[p.req];
        hc_batch_item it{};
        it.table = s->tables[r.table];
        it.op = r.op;
        it.d_keys = sl.d_buf + p.k_off;
        it.d_vals = p.v_off >= 0 ? sl.d_buf + p.v_off : nullptr;
        it.n = r.n;
        it.d_out = sl.d_buf + p.o_off;
        it.d_vals_out = p.vo_off >= 0 ? sl.d_buf + p.vo_off : nullptr;
        sl.items.push_back(it);
    }
    hc_rc rc = HC_OK;
    if (s->merge) {
        rc = hc::batch_run_pinned(sl.items.data(), (int64_t)sl.items.size(), &s->batch, sl.desc, sl.desc_bytes,
                                  sl.h_desc, st);
    } else {
        for (const hc_batch_item &it : sl.items) {
            if (it.op == HC_OP_INSERT) rc = hc_insert(it.table, it.d_keys, it.d_vals, it.n, it.d_out, st);
            else if (it.op == HC_OP_FIND) rc = hc_find(it.table, it.d_keys, it.n, it.d_out, it.d_vals_out, st);
            else rc = hc_erase(it.table, it.d_keys, it.n, it.d_out, st);
            if (rc != HC_OK) break;
        }
    }
    if (rc != HC_OK) return rc;
    if (sl.out_end > sl.out_begin)
        e = cudaMemcpyAsync(sl.h_out + sl.out_begin, sl.d_buf + sl.out_begin, (size_t)(sl.out_end - sl.out_begin),
                            cudaMemcpyDeviceToHost, st);
    for (const Placed &p : sl.placed) {
        if (!p.direct_out || e != cudaSuccess) continue;
        const hc_request &r = reqs[p.req];
        if (r.h_status) e = cudaMemcpyAsync(r.h_status, sl.d_buf + p.o_off, (size_t)r.n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && p.vo_off >= 0 && r.h_vals_out)
            e = cudaMemcpyAsync(r.h_vals_out, sl.d_buf + p.vo_off,
                                (size_t)(r.n * val_bytes(s->tables[r.table]->kind)), cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
    if (e != cudaSuccess) return scuda(e, "copying results to the host");
    sl.busy = true;
    return HC_OK;
}

void complete(hc_server *s, Slot &sl, hc_request *reqs, double t_done) {
    for (const Placed &p : sl.placed) {
        hc_request &r = reqs[p.req];
        const int vb = val_bytes(s->tables[r.table]->kind);
        if (!p.direct_out) {
            if (r.h_status) std::memcpy(r.h_status, sl.h_out + p.o_off, (size_t)r.n);
            if (p.vo_off >= 0 && r.h_vals_out) std::memcpy(r.h_vals_out, sl.h_out + p.vo_off, (size_t)(r.n * vb));
        }
        r.done = t_done;
    }
    sl.busy = false;
    sl.placed.clear();
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (v[hi] - v[lo]) * (pos - (double)lo);   // linear interpolation, as numpy's default
}

}  // namespace

extern "C" {

hc_rc hc_server_create(hc_server **out, hc_table *const *tables, int32_t n_tables, const hc_serve_config *cfg) {
    if (!out) return sfail(HC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_tables < 1 || !tables) return sfail(HC_ERR_ARG, "a server needs at least one table");
    for (int32_t i = 0; i < n_tables; ++i)
        if (!tables[i] || tables[i]->magic != HC_TABLE_MAGIC) return sfail(HC_ERR_ARG, "bad table handle");
    hc_serve_config c{4, 2, 64ll << 20, 1, 256, {0, 1, 256, 0, 0, 0}};
    if (cfg) {
        if (cfg->lanes) c.lanes = cfg->lanes;
        if (cfg->depth) c.depth = cfg->depth;
        if (cfg->slot_bytes) c.slot_bytes = cfg->slot_bytes;
        c.merge = cfg->merge;
        if (cfg->max_items) c.max_items = cfg->max_items;
        c.batch = cfg->batch;
    }
    if (c.lanes < 1 || c.lanes > 64 || c.depth < 1 || c.depth > 16 || c.slot_bytes < 4096 || c.max_items < 1 ||
        c.max_items > 4096 || (c.merge != 0 && c.merge != 1) || c.batch.use_graph)
        return sfail(HC_ERR_ARG, "bad server configuration");
    hc_server *s = new hc_server();
    s->magic = kServerMagic;
    s->tables.assign(tables, tables + n_tables);
    s->lanes = c.lanes;
    s->depth = c.depth;
    s->merge = c.merge;
    s->max_items = c.merge ? c.max_items : 1;
    s->slot_bytes = round256(c.slot_bytes);
    s->batch = c.batch;
    const int64_t desc_bytes = hc_batch_scratch_bytes(s->max_items);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < s->lanes && e == cudaSuccess; ++l) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        s->streams.push_back(st);
    }
    s->slots.resize((size_t)(s->lanes * s->depth));
    for (size_t i = 0; i < s->slots.size() && e == cudaSuccess; ++i) {
        Slot &sl = s->slots[i];
        sl.lane = (int)(i / (size_t)s->depth);
        sl.desc_bytes = desc_bytes;
        e = cudaMalloc(&sl.d_buf, (size_t)s->slot_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&sl.desc, (size_t)desc_bytes);
        if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_in, (size_t)s->slot_bytes, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc(&sl.h_out, (size_t)s->slot_bytes, cudaHostAllocDefault);
        if (e == cudaSuccess)
            e = cudaHostAlloc(&sl.h_desc, hc::batch_desc_bytes(s->max_items) + 256, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        release(s);
        return sfail(HC_ERR_OOM, std::string("allocating the launch slots: ") + cudaGetErrorString(e));
    }
    *out = s;
    return HC_OK;
}

hc_rc hc_server_destroy(hc_server *srv) {
    if (!srv) return HC_OK;
    if (srv->magic != kServerMagic) return sfail(HC_ERR_ARG, "bad server handle");
    for (cudaStream_t st : srv->streams) cudaStreamSynchronize(st);
    release(srv);
    return HC_OK;
}

hc_rc hc_server_run(hc_server *srv, hc_request *reqs, int64_t n_reqs, int32_t realtime, double timeout_s,
                    hc_serve_stats *stats) {
    if (!srv || srv->magic != kServerMagic) return sfail(HC_ERR_ARG, "bad server handle");
    if (n_reqs < 0 || (n_reqs > 0 && !reqs)) return sfail(HC_ERR_ARG, "bad request list");
    const int n_tables = (int)srv->tables.size();
    for (int64_t i = 0; i < n_reqs; ++i) {
        const hc_request &r = reqs[i];
        if (r.table < 0 || r.table >= n_tables || r.op < HC_OP_INSERT || r.op > HC_OP_ERASE || r.n < 0 ||
            (r.n > 0 && !r.h_keys))
            return sfail(HC_ERR_ARG, "bad request " + std::to_string(i));
        if (r.op == HC_OP_INSERT && val_bytes(srv->tables[r.table]->kind) && r.n > 0 && !r.h_vals)
            return sfail(HC_ERR_ARG, "request " + std::to_string(i) + " inserts into a map without values");
        if (i > 0 && realtime && r.arrival < reqs[i - 1].arrival)
            return sfail(HC_ERR_ARG, "requests must be sorted by arrival");
        int64_t in, out;
        need(srv, r, &in, &out);
        if (in + out + 256 > srv->slot_bytes)
            return sfail(HC_ERR_ARG, "request " + std::to_string(i) + " needs more than a launch slot");
    }
    srv->out_locked.assign((size_t)n_reqs, false);
    for (int64_t i = 0; i < n_reqs; ++i) {
        const hc_request &r = reqs[i];
        if (r.n <= kPackLimit) continue;
        const bool vals = r.op == HC_OP_FIND && val_bytes(srv->tables[r.table]->kind) && r.h_vals_out;
        srv->out_locked[(size_t)i] = (!r.h_status || page_locked(r.h_status)) && (!vals || page_locked(r.h_vals_out));
    }
    // work queued before the run (filling the tables, on any stream) comes first
    const cudaError_t e0 = cudaDeviceSynchronize();
    if (e0 != cudaSuccess) return scuda(e0, "synchronising the device before serving");
    std::vector<std::deque<int64_t>> fifo((size_t)n_tables);
    std::vector<std::vector<int>> lane_tables((size_t)srv->lanes);
    for (int t = 0; t < n_tables; ++t) lane_tables[(size_t)(t % srv->lanes)].push_back(t);
    std::vector<size_t> rr((size_t)srv->lanes, 0);
    int64_t next = 0, n_done = 0, launches = 0, queued = 0, queued_max = 0;
    const auto t0 = std::chrono::steady_clock::now();
    auto elapsed = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
    std::vector<int64_t> batch;
    while (n_done < n_reqs) {
        const double now = elapsed();
        if (now > timeout_s) {
            for (cudaStream_t st : srv->streams) cudaStreamSynchronize(st);
            return sfail(HC_ERR_STATE, "served " + std::to_string(n_done) + " of " + std::to_string(n_reqs) +
                                           " requests before the timeout");
        }
        bool progress = false;
        while (next < n_reqs && (!realtime || reqs[next].arrival <= now)) {
            fifo[(size_t)reqs[next].table].push_back(next);
            ++next;
            ++queued;
            progress = true;
        }
        queued_max = std::max(queued_max, queued);
        for (Slot &sl : srv->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) return scuda(q, "a served launch");
            n_done += (int64_t)sl.placed.size();
            complete(srv, sl, reqs, elapsed());
            progress = true;
        }
        for (Slot &sl : srv->slots) {
            if (sl.busy) continue;
            const std::vector<int> &tabs = lane_tables[(size_t)sl.lane];
            if (tabs.empty()) continue;
            batch.clear();
            int64_t used = 256;
            const size_t nt = tabs.size();
            for (size_t j = 0; j < nt && (int)batch.size() < srv->max_items; ++j) {
                const int t = tabs[(rr[(size_t)sl.lane] + j) % nt];
                if (fifo[(size_t)t].empty()) continue;
                int64_t in, out;
                need(srv, reqs[fifo[(size_t)t].front()], &in, &out);
                if (used + in + out > srv->slot_bytes) continue;
                batch.push_back(fifo[(size_t)t].front());
                fifo[(size_t)t].pop_front();
                used += in + out;
            }
            if (batch.empty()) continue;
            rr[(size_t)sl.lane] = (rr[(size_t)sl.lane] + 1) % nt;
            queued -= (int64_t)batch.size();
            const hc_rc rc = launch(srv, sl, reqs, batch);
            if (rc != HC_OK) return rc;
            ++launches;
            progress = true;
        }
        if (!progress) std::this_thread::yield();
    }
    const double wall = elapsed();
    if (stats) {
        std::vector<double> lat;
        lat.reserve((size_t)n_reqs);
        int64_t ops = 0;
        for (int64_t i = 0; i < n_reqs; ++i) {
            lat.push_back((reqs[i].done - (realtime ? reqs[i].arrival : 0.0)) * 1e3);
            ops += reqs[i].n;
        }
        stats->requests = n_reqs;
        stats->ops = ops;
        stats->launches = launches;
        stats->queued_max = queued_max;
        stats->wall_s = wall;
        stats->p50_ms = percentile(lat, 0.5);
        stats->p99_ms = percentile(lat, 0.99);
        stats->p999_ms = percentile(lat, 0.999);
        stats->max_ms = lat.empty() ? 0.0 : *std::max_element(lat.begin(), lat.end());
    }
    return HC_OK;
}

}  // extern "C"
