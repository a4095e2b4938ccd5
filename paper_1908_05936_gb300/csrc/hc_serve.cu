// hc_serve.cu -- the served form: a continuous-batching request loop over
// resident tables, run natively (see the hc.h section "served form" for the
// steps).  All device work is the library's own range calls and batched
// launch; this file schedules them.
//
// Two ways to feed the loop: hc_server_run serves a list of requests with
// arrival times on the calling thread; hc_server_start runs the loop on a
// thread of the server's own, to which any host thread submits requests
// while it runs (hc_server_submit / hc_server_wait / hc_server_stop).
//
// Work units.  A request whose arrays exceed a launch slot is cut into
// chunks that fit; a table's units leave its FIFO in order, so the chunks of
// a request run one after another, before the table's next request, and the
// request is done when its last chunk is.  Each chunk is one concurrent batch
// of the same operation, so the request's results are those of the whole
// batch (per key: one INSERTED / ERASED per distinct key, the rest EXISTS /
// NOT_FOUND).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
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
constexpr int64_t kPackLimit = 1 << 16;          // units up to this many keys are packed into one copy
constexpr int32_t kPending = -1;                 // hc_request.rc while a request is queued or running
constexpr size_t nt_none = ~(size_t)0;

hc_rc sfail(hc_rc rc, const std::string &msg) { return hc_internal_fail(rc, msg.c_str()); }

hc_rc scuda(cudaError_t e, const char *what) {
    return sfail(HC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int64_t round256(int64_t x) { return (x + 255) / 256 * 256; }

int key_bytes(int kind) { return kind == HC_SET_U32 ? 4 : 8; }
int val_bytes(int kind) { return kind == HC_MAP_I64_I32 ? 4 : (kind == HC_MAP_U64_U64 ? 8 : 0); }

// A request, or a chunk [off, off + n) of one.
struct Unit {
    int64_t req;
    int64_t off, n;
};

// Where one unit's arrays sit inside a slot.
struct Placed {
    Unit u;
    int64_t k_off, v_off;          // device offsets of the inputs (v_off < 0: none)
    int64_t o_off, vo_off;         // device offsets of the outputs (vo_off < 0: none)
    bool packed;                   // inputs copied through the slot's host staging
    bool direct_out;               // outputs copied straight into the request's page-locked arrays
    bool in_place;                 // all arrays page-locked: the kernels use them where they are
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

// The device address of a page-locked host array, or nullptr.
unsigned char *mapped_addr(const void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? static_cast<unsigned char *>(a.devicePointer) : nullptr;
}

struct Slot {
    int lane = 0;
    cudaStream_t stream = nullptr;     // each slot has a stream of its own
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

// Book-keeping of one request inside a loop.
struct Track {
    hc_request *r;
    int64_t units_left;            // units not yet completed
    int64_t dispatched;            // units handed to a slot
    bool out_locked;               // outputs page-locked (large units copy into them directly)
    bool in_place = false;         // every array page-locked: no staging, no copies
    unsigned char *dk = nullptr, *dv = nullptr, *ds = nullptr, *dvo = nullptr;   // their device addresses
};

// Whether request r can run where its arrays are: keys, values (map
// inserts), status (when given) and values out (map finds, when given) all
// page-locked.  Fills the device addresses.
bool map_in_place(const hc_server *s, Track &t);

}  // namespace

struct hc_server {
    uint32_t magic;
    int device;
    std::vector<hc_table *> tables;
    int lanes, depth, merge, max_items;
    int64_t slot_bytes;
    hc_batch_config batch;
    std::vector<cudaStream_t> streams;
    std::vector<Slot> slots;
    // live mode
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_submit, cv_done;
    std::vector<hc_request *> pending;     // submitted, not yet seen by the loop
    bool running = false, stopping = false;
    std::chrono::steady_clock::time_point t0;
    hc_rc live_rc = HC_OK;                 // first error of the live loop
    std::string live_err;
    hc_serve_stats live_stats{};
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

// Device bytes n keys of a request take in a slot: inputs, then outputs.
void need(const hc_server *s, const hc_request &r, int64_t n, int64_t *in, int64_t *out) {
    const int kind = s->tables[r.table]->kind;
    const int kb = key_bytes(kind), vb = val_bytes(kind);
    *in = round256(n * kb) + ((r.op == HC_OP_INSERT && vb) ? round256(n * vb) : 0);
    *out = round256(n) + ((r.op == HC_OP_FIND && vb) ? round256(n * vb) : 0);
}

// Largest number of keys of request r that fits one slot (with the 256-byte
// reserve the dispatcher keeps), a multiple of 256.
int64_t chunk_keys(const hc_server *s, const hc_request &r) {
    const int kind = s->tables[r.table]->kind;
    const int kb = key_bytes(kind), vb = val_bytes(kind);
    const int64_t per = kb + 1 + (r.op == HC_OP_INSERT ? vb : 0) + (r.op == HC_OP_FIND ? vb : 0);
    int64_t c = (s->slot_bytes - 256 - 4 * 256) / per;   // room for the round-up of each array
    c = c / 256 * 256;
    return c < 256 ? 256 : c;
}

hc_rc check_request(const hc_server *s, const hc_request &r, const std::string &name) {
    const int n_tables = (int)s->tables.size();
    if (r.table < 0 || r.table >= n_tables || r.op < HC_OP_INSERT || r.op > HC_OP_ERASE || r.n < 0 ||
        (r.n > 0 && !r.h_keys) || r.deadline < 0)
        return sfail(HC_ERR_ARG, "bad " + name);
    if (r.op == HC_OP_INSERT && val_bytes(s->tables[r.table]->kind) && r.n > 0 && !r.h_vals)
        return sfail(HC_ERR_ARG, name + " inserts into a map without values");
    return HC_OK;
}

bool outputs_locked(const hc_server *s, const hc_request &r) {
    const bool vals = r.op == HC_OP_FIND && val_bytes(s->tables[r.table]->kind) && r.h_vals_out;
    return (!r.h_status || page_locked(r.h_status)) && (!vals || page_locked(r.h_vals_out));
}

bool map_in_place(const hc_server *s, Track &t) {
    const hc_request &r = *t.r;
    if (r.n == 0) return false;
    const bool map = val_bytes(s->tables[r.table]->kind) != 0;
    t.dk = mapped_addr(r.h_keys);
    if (!t.dk) return false;
    if (r.op == HC_OP_INSERT && map && !(t.dv = mapped_addr(r.h_vals))) return false;
    if (r.h_status && !(t.ds = mapped_addr(r.h_status))) return false;
    if (r.op == HC_OP_FIND && !t.ds) return false;                 // a find needs its flags array
    if (r.op == HC_OP_FIND && map && r.h_vals_out && !(t.dvo = mapped_addr(r.h_vals_out))) return false;
    return true;
}

hc_rc launch(hc_server *s, Slot &sl, std::vector<Track> &tr, const std::vector<Unit> &batch) {
    cudaStream_t st = sl.stream;
    sl.placed.clear();
    int64_t off = 0, packed_end = 0;
    for (const Unit &u : batch) {
        const hc_request &r = *tr[(size_t)u.req].r;
        const int kind = s->tables[r.table]->kind;
        const int kb = key_bytes(kind), vb = val_bytes(kind);
        if (tr[(size_t)u.req].in_place) {          // no staging: the kernels use the request's arrays
            sl.placed.push_back(Placed{u, -1, -1, -1, -1, false, false, true});
            continue;
        }
        int64_t in, out;
        need(s, r, u.n, &in, &out);
        Placed p{u, off, (r.op == HC_OP_INSERT && vb) ? off + round256(u.n * kb) : -1, 0, -1, u.n <= kPackLimit,
                 u.n > kPackLimit && tr[(size_t)u.req].out_locked, false};
        if (p.packed && u.n > 0) {
            std::memcpy(sl.h_in + p.k_off, static_cast<const unsigned char *>(r.h_keys) + u.off * kb,
                        (size_t)(u.n * kb));
            if (p.v_off >= 0)
                std::memcpy(sl.h_in + p.v_off, static_cast<const unsigned char *>(r.h_vals) + u.off * vb,
                            (size_t)(u.n * vb));
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
            if (p.in_place || p.direct_out != (pass == 1)) continue;
            const hc_request &r = *tr[(size_t)p.u.req].r;
            const int vb = val_bytes(s->tables[r.table]->kind);
            p.o_off = o;
            p.vo_off = (r.op == HC_OP_FIND && vb) ? o + round256(p.u.n) : -1;
            int64_t in, out;
            need(s, r, p.u.n, &in, &out);
            o += out;
        }
        if (pass == 0) sl.out_end = o;
    }
    cudaError_t e = cudaSuccess;
    if (packed_end > 0) e = cudaMemcpyAsync(sl.d_buf, sl.h_in, (size_t)packed_end, cudaMemcpyHostToDevice, st);
    for (const Placed &p : sl.placed) {
        if (p.in_place || p.packed || p.u.n == 0 || e != cudaSuccess) continue;
        const hc_request &r = *tr[(size_t)p.u.req].r;
        const int kind = s->tables[r.table]->kind;
        const int kb = key_bytes(kind), vb = val_bytes(kind);
        e = cudaMemcpyAsync(sl.d_buf + p.k_off, static_cast<const unsigned char *>(r.h_keys) + p.u.off * kb,
                            (size_t)(p.u.n * kb), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && p.v_off >= 0)
            e = cudaMemcpyAsync(sl.d_buf + p.v_off, static_cast<const unsigned char *>(r.h_vals) + p.u.off * vb,
                                (size_t)(p.u.n * vb), cudaMemcpyHostToDevice, st);
    }
    if (e != cudaSuccess) return scuda(e, "copying request inputs to the device");
    sl.items.clear();
    for (const Placed &p : sl.placed) {
        const Track &t = tr[(size_t)p.u.req];
        const hc_request &r = *t.r;
        hc_batch_item it{};
        it.table = s->tables[r.table];
        it.op = r.op;
        it.n = p.u.n;
        if (p.in_place) {
            const int kind = s->tables[r.table]->kind;
            const int kb = key_bytes(kind), vb = val_bytes(kind);
            it.d_keys = t.dk + p.u.off * kb;
            it.d_vals = t.dv ? t.dv + p.u.off * vb : nullptr;
            it.d_out = t.ds ? t.ds + p.u.off : nullptr;
            it.d_vals_out = t.dvo ? t.dvo + p.u.off * vb : nullptr;
        } else {
            it.d_keys = sl.d_buf + p.k_off;
            it.d_vals = p.v_off >= 0 ? sl.d_buf + p.v_off : nullptr;
            it.d_out = sl.d_buf + p.o_off;
            it.d_vals_out = p.vo_off >= 0 ? sl.d_buf + p.vo_off : nullptr;
        }
        sl.items.push_back(it);
    }
    hc_rc rc = HC_OK;
    // a lone unit runs as a plain range call even in merged mode: a batched
    // launch only pays off when it has several requests to share it
    if (s->merge && sl.items.size() > 1) {
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
        if (p.in_place || !p.direct_out || e != cudaSuccess) continue;
        const hc_request &r = *tr[(size_t)p.u.req].r;
        const int vb = val_bytes(s->tables[r.table]->kind);
        if (r.h_status) e = cudaMemcpyAsync(r.h_status + p.u.off, sl.d_buf + p.o_off, (size_t)p.u.n,
                                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && p.vo_off >= 0 && r.h_vals_out)
            e = cudaMemcpyAsync(static_cast<unsigned char *>(r.h_vals_out) + p.u.off * vb, sl.d_buf + p.vo_off,
                                (size_t)(p.u.n * vb), cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, st);
    if (e != cudaSuccess) return scuda(e, "copying results to the host");
    sl.busy = true;
    return HC_OK;
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, v.size() - 1);
    return v[lo] + (v[hi] - v[lo]) * (pos - (double)lo);   // linear interpolation, as numpy's default
}

// Where the loop's requests come from.
struct Source {
    // array mode
    hc_request *reqs = nullptr;
    int64_t n_reqs = 0;
    bool realtime = false;
    // live mode: requests submitted through srv->pending
    bool live = false;
};

// The loop shared by both modes.  Returns after every request it admitted is
// done (array mode: all of them; live mode: once stopping is set and nothing
// is left), or on the first error.
hc_rc serve_loop(hc_server *srv, const Source &src, double timeout_s, hc_serve_stats *stats) {
    const int n_tables = (int)srv->tables.size();
    std::vector<std::deque<Unit>> fifo((size_t)n_tables);
    std::vector<std::vector<int>> lane_tables((size_t)srv->lanes);
    for (int t = 0; t < n_tables; ++t) lane_tables[(size_t)(t % srv->lanes)].push_back(t);
    std::vector<size_t> rr((size_t)srv->lanes, 0);
    std::vector<int> inflight((size_t)n_tables, 0);   // units of each table in a slot (at most one)
    std::vector<Track> tr;
    tr.reserve(src.live ? 1024 : (size_t)src.n_reqs);
    int64_t next = 0, n_admitted = 0, n_done = 0, n_timed_out = 0, launches = 0, queued = 0, queued_max = 0, ops = 0;
    std::vector<double> lat;
    const auto elapsed = [&]() {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - srv->t0).count();
    };
    auto admit = [&](hc_request *r) {
        const int64_t id = (int64_t)tr.size();
        Track t{r, 0, 0, r->n > kPackLimit && outputs_locked(srv, *r)};
        t.in_place = map_in_place(srv, t);
        // a request whose arrays the kernels use in place needs no slot
        // buffer, so it is not cut to a slot's size
        const int64_t c = t.in_place ? r->n : chunk_keys(srv, *r);
        const int64_t units = r->n == 0 ? 1 : (r->n + c - 1) / c;
        t.units_left = units;
        tr.push_back(t);
        r->rc = kPending;
        r->done = -1.0;
        for (int64_t k = 0; k < units; ++k) {
            const int64_t off = k * c;
            fifo[(size_t)r->table].push_back(Unit{id, off, std::min(c, r->n - off)});
        }
        ++n_admitted;
        ++queued;
    };
    auto finish = [&](Track &t, int32_t rc, double when) {
        if (src.live) {
            std::lock_guard<std::mutex> g(srv->mu);
            t.r->done = when;
            t.r->rc = rc;
        } else {
            t.r->done = when;
            t.r->rc = rc;
        }
        ++n_done;
        if (rc == HC_OK) {
            lat.push_back((when - (src.realtime || src.live ? t.r->arrival : 0.0)) * 1e3);
            ops += t.r->n;
        } else {
            ++n_timed_out;
        }
        if (src.live) srv->cv_done.notify_all();
    };
    std::vector<Unit> batch;
    while (true) {
        const double now = elapsed();
        if (!src.live && now > timeout_s) {
            for (cudaStream_t st : srv->streams) cudaStreamSynchronize(st);
            return sfail(HC_ERR_STATE, "served " + std::to_string(n_done) + " of " + std::to_string(src.n_reqs) +
                                           " requests before the timeout");
        }
        bool progress = false;
        // arrivals
        if (src.live) {
            std::vector<hc_request *> got;
            bool stop = false;
            {
                std::unique_lock<std::mutex> lk(srv->mu);
                if (srv->pending.empty() && !srv->stopping && n_done == n_admitted)
                    srv->cv_submit.wait_for(lk, std::chrono::milliseconds(50));
                got.swap(srv->pending);
                stop = srv->stopping;
            }
            for (hc_request *r : got) admit(r);
            progress |= !got.empty();
            if (stop && got.empty() && n_done == n_admitted) break;
        } else {
            while (next < src.n_reqs && (!src.realtime || src.reqs[next].arrival <= now)) {
                admit(&src.reqs[next]);
                ++next;
                progress = true;
            }
            if (n_done == src.n_reqs) break;
        }
        queued_max = std::max(queued_max, queued);
        // completions
        for (Slot &sl : srv->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) return scuda(q, "a served launch");
            const double t_done = elapsed();
            for (const Placed &p : sl.placed) {
                Track &t = tr[(size_t)p.u.req];
                const hc_request &r = *t.r;
                --inflight[(size_t)r.table];
                if (!p.in_place && !p.direct_out && p.u.n > 0) {
                    const int vb = val_bytes(srv->tables[r.table]->kind);
                    if (r.h_status) std::memcpy(r.h_status + p.u.off, sl.h_out + p.o_off, (size_t)p.u.n);
                    if (p.vo_off >= 0 && r.h_vals_out)
                        std::memcpy(static_cast<unsigned char *>(r.h_vals_out) + p.u.off * vb, sl.h_out + p.vo_off,
                                    (size_t)(p.u.n * vb));
                }
                if (--t.units_left == 0) finish(t, HC_OK, t_done);
            }
            sl.busy = false;
            sl.placed.clear();
            progress = true;
        }
        // deadlines: a request none of whose units has been dispatched is
        // dropped once its deadline has passed (the table is not touched)
        for (int t = 0; t < n_tables; ++t) {
            std::deque<Unit> &f = fifo[(size_t)t];
            for (auto it = f.begin(); it != f.end();) {
                Track &k = tr[(size_t)it->req];
                const double arrived = (src.realtime || src.live) ? k.r->arrival : 0.0;
                if (k.r->deadline > 0 && k.dispatched == 0 && now > arrived + k.r->deadline) {
                    const int64_t id = it->req;
                    while (it != f.end() && it->req == id) it = f.erase(it);   // its units are adjacent
                    --queued;
                    finish(k, HC_ERR_TIMEOUT, now);
                    progress = true;
                } else {
                    ++it;
                }
            }
        }
        // dispatch: a free slot takes head units of its lane's tables.  A
        // table has at most one unit in a slot, so its units run in FIFO
        // order although slots run on streams of their own.  In merged mode
        // small units (up to kPackLimit keys) share a launch; a large unit
        // runs alone, so small requests never wait for a large one in the
        // same launch.
        for (Slot &sl : srv->slots) {
            if (sl.busy) continue;
            const std::vector<int> &tabs = lane_tables[(size_t)sl.lane];
            if (tabs.empty()) continue;
            batch.clear();
            int64_t used = 256;
            int mode = 0;                     // 1: small units merged, 2: one large unit
            size_t skipped = nt_none;         // first large head passed over by a merged launch
            const size_t nt = tabs.size();
            // merged mode merges only the units that the lane's free slots
            // cannot take one by one: with w units waiting and f free slots
            // (this one included), this slot takes w - f + 1 of them and each
            // other free slot one, so nothing waits for a batched launch that
            // a slot of its own could have run as its plain call
            int take = srv->max_items;
            if (srv->merge) {
                int free_slots = 0, waiting = 0;
                for (const Slot &o : srv->slots) free_slots += (o.lane == sl.lane && !o.busy) ? 1 : 0;
                for (int t : tabs) waiting += (!fifo[(size_t)t].empty() && !inflight[(size_t)t]) ? 1 : 0;
                take = waiting <= free_slots ? 1 : std::min(srv->max_items, waiting - free_slots + 1);
            }
            for (size_t j = 0; j < nt && (int)batch.size() < take && mode != 2; ++j) {
                const int t = tabs[(rr[(size_t)sl.lane] + j) % nt];
                if (fifo[(size_t)t].empty() || inflight[(size_t)t]) continue;
                const Unit u = fifo[(size_t)t].front();
                const bool large = u.n > kPackLimit;
                if (srv->merge && mode == 1 && large) {
                    if (skipped == nt_none) skipped = j;
                    continue;
                }
                int64_t in = 0, out = 0;
                if (!tr[(size_t)u.req].in_place) need(srv, *tr[(size_t)u.req].r, u.n, &in, &out);
                if (used + in + out > srv->slot_bytes) continue;
                mode = large ? 2 : 1;
                batch.push_back(u);
                fifo[(size_t)t].pop_front();
                ++inflight[(size_t)t];
                Track &k = tr[(size_t)u.req];
                if (k.dispatched++ == 0) --queued;
                used += in + out;
            }
            if (batch.empty()) continue;
            // the lane's next slot starts at a large head this launch passed
            // over, so small requests cannot keep it waiting
            rr[(size_t)sl.lane] = (rr[(size_t)sl.lane] + (skipped != nt_none ? skipped : 1)) % nt;
            const hc_rc rc = launch(srv, sl, tr, batch);
            if (rc != HC_OK) return rc;
            ++launches;
            progress = true;
        }
        if (!progress) std::this_thread::yield();
    }
    if (stats) {
        stats->requests = n_done - n_timed_out;
        stats->ops = ops;
        stats->launches = launches;
        stats->queued_max = queued_max;
        stats->timed_out = n_timed_out;
        stats->wall_s = elapsed();
        stats->p50_ms = percentile(lat, 0.5);
        stats->p99_ms = percentile(lat, 0.99);
        stats->p999_ms = percentile(lat, 0.999);
        stats->max_ms = lat.empty() ? 0.0 : *std::max_element(lat.begin(), lat.end());
    }
    return HC_OK;
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
    if (c.lanes < 1 || c.lanes > 64 || c.depth < 1 || c.depth > 16 || c.slot_bytes < 65536 || c.max_items < 1 ||
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
    cudaError_t e = cudaGetDevice(&s->device);
    s->slots.resize((size_t)(s->lanes * s->depth));
    for (size_t i = 0; i < s->slots.size() && e == cudaSuccess; ++i) {
        cudaStream_t st = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        s->streams.push_back(st);
        Slot &sl = s->slots[i];
        sl.stream = st;
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
    if (srv->running) {
        const hc_rc rc = hc_server_stop(srv, nullptr);
        (void)rc;
    }
    for (cudaStream_t st : srv->streams) cudaStreamSynchronize(st);
    release(srv);
    return HC_OK;
}

hc_rc hc_server_run(hc_server *srv, hc_request *reqs, int64_t n_reqs, int32_t realtime, double timeout_s,
                    hc_serve_stats *stats) {
    if (!srv || srv->magic != kServerMagic) return sfail(HC_ERR_ARG, "bad server handle");
    if (srv->running) return sfail(HC_ERR_ARG, "the server's own loop is running (hc_server_start)");
    if (n_reqs < 0 || (n_reqs > 0 && !reqs)) return sfail(HC_ERR_ARG, "bad request list");
    for (int64_t i = 0; i < n_reqs; ++i) {
        const hc_rc rc = check_request(srv, reqs[i], "request " + std::to_string(i));
        if (rc != HC_OK) return rc;
        if (i > 0 && realtime && reqs[i].arrival < reqs[i - 1].arrival)
            return sfail(HC_ERR_ARG, "requests must be sorted by arrival");
    }
    // work queued before the run (filling the tables, on any stream) comes first
    const cudaError_t e0 = cudaDeviceSynchronize();
    if (e0 != cudaSuccess) return scuda(e0, "synchronising the device before serving");
    Source src;
    src.reqs = reqs;
    src.n_reqs = n_reqs;
    src.realtime = realtime != 0;
    srv->t0 = std::chrono::steady_clock::now();
    return serve_loop(srv, src, timeout_s, stats);
}

hc_rc hc_server_start(hc_server *srv) {
    if (!srv || srv->magic != kServerMagic) return sfail(HC_ERR_ARG, "bad server handle");
    if (srv->running) return sfail(HC_ERR_ARG, "the server's loop is already running");
    const cudaError_t e0 = cudaDeviceSynchronize();
    if (e0 != cudaSuccess) return scuda(e0, "synchronising the device before serving");
    srv->pending.clear();
    srv->stopping = false;
    srv->live_rc = HC_OK;
    srv->live_err.clear();
    srv->live_stats = hc_serve_stats{};
    srv->t0 = std::chrono::steady_clock::now();
    srv->running = true;
    srv->worker = std::thread([srv]() {
        hc_rc rc = HC_OK;
        if (cudaSetDevice(srv->device) != cudaSuccess) rc = sfail(HC_ERR_CUDA, "selecting the server's device");
        Source src;
        src.live = true;
        hc_serve_stats st{};
        if (rc == HC_OK) rc = serve_loop(srv, src, 0.0, &st);
        std::lock_guard<std::mutex> g(srv->mu);
        srv->live_rc = rc;
        if (rc != HC_OK) srv->live_err = hc_last_error();
        srv->live_stats = st;
        srv->running = false;
        srv->cv_done.notify_all();
    });
    return HC_OK;
}

hc_rc hc_server_submit(hc_server *srv, hc_request *req) {
    if (!srv || srv->magic != kServerMagic) return sfail(HC_ERR_ARG, "bad server handle");
    if (!req) return sfail(HC_ERR_ARG, "req is NULL");
    hc_rc rc = check_request(srv, *req, "request");
    if (rc != HC_OK) return rc;
    std::lock_guard<std::mutex> g(srv->mu);
    if (!srv->running || srv->stopping) return sfail(HC_ERR_STATE, "the server's loop is not running");
    req->arrival = std::chrono::duration<double>(std::chrono::steady_clock::now() - srv->t0).count();
    req->done = -1.0;
    req->rc = kPending;
    srv->pending.push_back(req);
    srv->cv_submit.notify_one();
    return HC_OK;
}

hc_rc hc_server_wait(hc_server *srv, hc_request *req, double timeout_s) {
    if (!srv || srv->magic != kServerMagic) return sfail(HC_ERR_ARG, "bad server handle");
    if (!req) return sfail(HC_ERR_ARG, "req is NULL");
    std::unique_lock<std::mutex> lk(srv->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (req->rc == kPending) {
        if (!srv->running) return sfail(HC_ERR_STATE, "the server's loop ended before the request was served");
        if (srv->cv_done.wait_until(lk, until) == std::cv_status::timeout && req->rc == kPending)
            return sfail(HC_ERR_TIMEOUT, "the request was not served within the wait's time limit");
    }
    if (req->rc != HC_OK) return sfail((hc_rc)req->rc, "the request's deadline passed before it was dispatched");
    return HC_OK;
}

hc_rc hc_server_stop(hc_server *srv, hc_serve_stats *stats) {
    if (!srv || srv->magic != kServerMagic) return sfail(HC_ERR_ARG, "bad server handle");
    {
        std::lock_guard<std::mutex> g(srv->mu);
        if (!srv->worker.joinable()) return sfail(HC_ERR_ARG, "the server's loop was not started");
        srv->stopping = true;
        srv->cv_submit.notify_one();
    }
    srv->worker.join();
    if (stats) *stats = srv->live_stats;
    if (srv->live_rc != HC_OK) return sfail(srv->live_rc, srv->live_err);
    return HC_OK;
}

}  // extern "C"
