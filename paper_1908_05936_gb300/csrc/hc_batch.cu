// hc_batch.cu -- the batched form: many range calls on many tables in one
// persistent launch per phase (insert, then find, then erase), optionally
// captured once into a CUDA graph and replayed.
//
// Scheduling.  Every item is cut into chunks of `tile` keys.  A phase kernel
// runs a persistent grid (SMs x blocks per SM); each warp takes the next
// chunk number from a counter in global memory with one atomic add, finds the
// item that chunk belongs to by binary search over the items' chunk offsets,
// and runs the same warp-tile code as the one-launch-per-call kernels over
// the chunk.  Tables of very different sizes are therefore balanced at chunk
// granularity, and no launch is spent per table.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hc.h"
#include "hc_core.cuh"
#include "hc_internal.h"
#include "hc_stream.cuh"
#include "hc_table.h"

namespace hc {

struct BatchItemDev {
    View v;
    const void *keys;
    const void *vals;
    uint8_t *out;
    void *vals_out;
    long long n;
    long long chunk_begin;   // first chunk number of this item within its phase
    int bb;
    int fold;
};

// Work of one phase launch: items [item0, item0 + n_items) of one kind.
struct PhaseDesc {
    int kind;
    int op;
    int bb;        // bucket bytes of every table in the phase
    int item0;
    int n_items;
    long long n_chunks;
    int counter;   // index of this phase's chunk counter
};

template <int KIND, int OP, int BB, int LB, int KPT>
__device__ __forceinline__ void run_chunk(const BatchItemDev &it, long long k0, long long k1) {
    using T = Traits<KIND>;
    constexpr int TILE = Shape<KIND, BB, LB, KPT>::TILE;
    // keys past the chunk end belong to the next chunk: n is clamped to k1
    Counts cnt;
    run_tiles<KIND, BB, LB, KPT, OP>(it.v, (const typename T::Key *)it.keys, (const typename T::Val *)it.vals, nullptr,
                                     it.out, (typename T::Val *)it.vals_out, k1, k0 / TILE, (k1 + TILE - 1) / TILE, 1,
                                     it.fold != 0, cnt);
    if constexpr (OP != OP_FIND) flush_counts(it.v, cnt);
}

// One phase launch covers items of one kind, one op and one bucket size (so
// each launch is a small specialisation).  WIDE: one thread per key reading
// the whole bucket (maps: keys and values) or key region (sets); otherwise
// 32-byte lanes.
template <int KIND, int OP, int BB, int WIDE, int KPT>
__global__ void __launch_bounds__(256)
k_batch_phase(const BatchItemDev *__restrict__ items, int n_items, long long n_chunks, int tile,
              unsigned long long *counter) {
    constexpr int KRB = Slots<KIND, BB>::KRB;
    constexpr int LB = WIDE ? (Traits<KIND>::MAP ? BB : KRB) : (KRB < 32 ? KRB : 32);
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(counter, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        if ((long long)c >= n_chunks) break;
        // last item whose chunk_begin <= c
        int lo = 0, hi = n_items - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].chunk_begin <= (long long)c) lo = mid;
            else hi = mid - 1;
        }
        const BatchItemDev it = items[lo];
        const long long k0 = ((long long)c - it.chunk_begin) * tile;
        const long long k1 = k0 + tile < it.n ? k0 + tile : it.n;
        debug_range(it.v, k0, k1 - k0, it.n);
        run_chunk<KIND, OP, BB, LB, KPT>(it, k0, k1);
    }
}

// The streaming form of a phase (keys_per_group 4 or 8): a block takes the
// next chunk with one atomic add and works through it in pieces of
// blockDim.x * KPT keys with the streaming kernels' chunk functions (keys
// staged in shared memory, S probes in flight per thread).
template <int KIND, int OP, int BB, int KPT, int S>
__global__ void __launch_bounds__(256)
k_batch_stream(const BatchItemDev *__restrict__ items, int n_items, long long n_chunks, int tile,
               unsigned long long *counter) {
    using T = Traits<KIND>;
    __shared__ long long s_chunk;
    const int piece = blockDim.x * KPT;
    while (true) {
        if (threadIdx.x == 0) s_chunk = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long c = s_chunk;
        __syncthreads();                                   // s_chunk is written again only after every thread read it
        if (c >= n_chunks) break;
        int lo = 0, hi = n_items - 1;                      // last item whose chunk_begin <= c
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].chunk_begin <= c) lo = mid;
            else hi = mid - 1;
        }
        const BatchItemDev &it = items[lo];
        const long long k0 = (c - it.chunk_begin) * tile;
        const long long k1 = k0 + tile < it.n ? k0 + tile : it.n;
        const auto *keys = (const typename T::Key *)it.keys;
        for (long long p0 = k0; p0 < k1; p0 += piece) {
            const int m = (int)(k1 - p0 < piece ? k1 - p0 : piece);
            debug_range(it.v, p0, m, it.n);
            if constexpr (OP == OP_INSERT)
                insert_stream_chunk<KIND, BB, KPT, S>(it.v, keys, (const typename T::Val *)it.vals, p0, m, it.out,
                                                      nullptr);
            else if constexpr (OP == OP_FIND)
                find_stream_chunk<KIND, BB, KPT, S>(it.v, keys, p0, m, it.out, (typename T::Val *)it.vals_out);
            else
                erase_stream_chunk<KIND, BB, KPT, S>(it.v, keys, p0, m, it.out, nullptr);
        }
    }
}

__global__ void k_zero_counters(unsigned long long *c, int n) {
    if (threadIdx.x < n) c[threadIdx.x] = 0ull;
}

using PhaseKernel = void (*)(const BatchItemDev *, int, long long, int, unsigned long long *);

template <int KIND, int OP, int BB>
PhaseKernel pick_lb_kpt(int lb, int kpt) {
    if (kpt == 4) return k_batch_stream<KIND, OP, BB, 4, 2>;
    if (kpt == 8) return k_batch_stream<KIND, OP, BB, 8, 4>;
    if (lb == 0) return kpt == 1 ? k_batch_phase<KIND, OP, BB, 1, 1> : k_batch_phase<KIND, OP, BB, 1, 2>;
    return kpt == 1 ? k_batch_phase<KIND, OP, BB, 0, 1> : k_batch_phase<KIND, OP, BB, 0, 2>;
}

// Dynamic shared memory of a phase launch (the streaming form's staging).
size_t phase_smem(int kind, int kpt, int block) {
    if (kpt < 4) return 0;
    const int kb = kind == KIND_SET_U32 ? 4 : 8;
    const int vb = kind == KIND_SET_U32 ? 4 : 8;            // the staging holds a value slot for every kind
    return stream_smem((long long)block * kpt, kb, vb);
}

// A phase kernel with more than the default 48 KB of dynamic shared memory
// must be allowed it before its occupancy is queried or it is launched.
void allow_phase_smem(PhaseKernel k, size_t bytes) {
    if (bytes > 48 * 1024) (void)cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int KIND, int OP>
PhaseKernel pick_bb(int bb, int lb, int kpt) {
    if (bb == 32) return pick_lb_kpt<KIND, OP, 32>(lb, kpt);
    if (bb == 64) return pick_lb_kpt<KIND, OP, 64>(lb, kpt);
    return pick_lb_kpt<KIND, OP, 128>(lb, kpt);
}

template <int KIND>
PhaseKernel pick_op(int op, int bb, int lb, int kpt) {
    if (op == OP_INSERT) return pick_bb<KIND, OP_INSERT>(bb, lb, kpt);
    if (op == OP_FIND) return pick_bb<KIND, OP_FIND>(bb, lb, kpt);
    return pick_bb<KIND, OP_ERASE>(bb, lb, kpt);
}

PhaseKernel pick_kernel(int kind, int op, int bb, int lb, int kpt) {
    switch (kind) {
        case KIND_SET_U32: return pick_op<KIND_SET_U32>(op, bb, lb, kpt);
        case KIND_SET_U64: return pick_op<KIND_SET_U64>(op, bb, lb, kpt);
        case KIND_MAP_I64_I32: return pick_op<KIND_MAP_I64_I32>(op, bb, lb, kpt);
        default: return pick_op<KIND_MAP_U64_U64>(op, bb, lb, kpt);
    }
}

}  // namespace hc

struct hc_batch {
    uint32_t magic;
    int device;
    int block, blocks_per_sm, tile, lane_bytes, kpt;
    bool use_graph;
    void *d_mem = nullptr;   // items then counters
    hc::BatchItemDev *d_items = nullptr;
    unsigned long long *d_counters = nullptr;
    std::vector<hc::PhaseDesc> phases;
    std::vector<int> grid;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// Errors go to the same thread-local message as the rest of the API (owned
// by hc_api.cu).
hc_rc hc_internal_fail(hc_rc rc, const char *msg);

namespace {

constexpr uint32_t kBatchMagic = 0x48434241u;

// tile 0 in the configuration: keys per chunk chosen from the total work so
// that the chunks can occupy every warp slot of the GPU (64 per SM): a power
// of two from 128 to 4096.
int auto_tile(const hc_batch_item *items, int64_t n_items) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || sms <= 0) {
        (void)cudaGetLastError();
        return 4096;
    }
    long long total = 0;
    for (int64_t i = 0; i < n_items; ++i)
        if (items[i].n > 0) total += items[i].n;
    const long long per_slot = total / ((long long)sms * 64);
    int tile = 128;
    while (tile < 1024 && (long long)tile * 2 <= per_slot) tile *= 2;
    return tile;
}

hc_rc bfail(hc_rc rc, const std::string &msg) { return hc_internal_fail(rc, msg.c_str()); }

hc_rc bcuda(cudaError_t e, const char *what) {
    return bfail(HC_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

hc_rc enqueue(hc_batch *b, cudaStream_t s) {
    const int n_ctr = (int)b->phases.size();
    if (n_ctr == 0) return HC_OK;
    hc::k_zero_counters<<<1, 64, 0, s>>>(b->d_counters, n_ctr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bcuda(e, "resetting the batch counters");
    for (size_t p = 0; p < b->phases.size(); ++p) {
        const hc::PhaseDesc &ph = b->phases[p];
        hc::PhaseKernel k = hc::pick_kernel(ph.kind, ph.op, ph.bb, b->lane_bytes, b->kpt);
        const size_t smem = hc::phase_smem(ph.kind, b->kpt, b->block);
        hc::allow_phase_smem(k, smem);
        k<<<b->grid[p], b->block, smem, s>>>(
            b->d_items + ph.item0, ph.n_items, ph.n_chunks, b->tile, b->d_counters + ph.counter);
        e = cudaGetLastError();
        if (e != cudaSuccess) return bcuda(e, "launching a batch phase");
    }
    return HC_OK;
}

}  // namespace

extern "C" {

HC_API hc_rc hc_batch_create(hc_batch **out, const hc_batch_item *items, int64_t n_items, const hc_batch_config *cfg,
                             void *stream) {
    if (!out) return bfail(HC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_items < 0 || (n_items > 0 && !items)) return bfail(HC_ERR_ARG, "bad item list");
    hc_batch_config c{};
    if (cfg) c = *cfg;
    const int lb = c.lane_bytes;
    const int kpt = c.keys_per_group ? c.keys_per_group : 1;
    const int block = c.block ? c.block : 256;
    const int tile = c.tile ? c.tile : auto_tile(items, n_items);
    if (lb != 0 && lb != 32) return bfail(HC_ERR_ARG, "lane_bytes must be 0 (whole bucket) or 32");
    if (kpt != 1 && kpt != 2 && kpt != 4 && kpt != 8)
        return bfail(HC_ERR_ARG, "keys_per_group must be 1 or 2 (lock-step) or 4 or 8 (streaming)");
    if (kpt >= 4 && block > 256) return bfail(HC_ERR_ARG, "streaming phases take at most 256 threads per block");
    if (block < 64 || block > 256 || block % 32) return bfail(HC_ERR_ARG, "block must be a multiple of 32 in [64, 256]");
    if (tile < 128 || tile % 128) return bfail(HC_ERR_ARG, "tile must be a positive multiple of 128");

    // items ordered by (op, kind) so each phase launch sees one contiguous run
    std::vector<hc::BatchItemDev> dev;
    std::vector<hc::PhaseDesc> phases;
    for (int op = 0; op < 3; ++op) {
        for (int kind = 0; kind < 4; ++kind)
        for (int bb = 32; bb <= 128; bb *= 2) {
            hc::PhaseDesc ph{kind, op, bb, (int)dev.size(), 0, 0, (int)phases.size()};
            for (int64_t i = 0; i < n_items; ++i) {
                const hc_batch_item &it = items[i];
                if (!it.table || it.table->magic != HC_TABLE_MAGIC) return bfail(HC_ERR_ARG, "item with a bad table");
                if (it.op < 0 || it.op > 2) return bfail(HC_ERR_ARG, "item with a bad op");
                if (it.n < 0) return bfail(HC_ERR_ARG, "item with n < 0");
                if (it.op != op || it.table->kind != kind || it.table->bucket_bytes != bb || it.n == 0) continue;
                const bool map = kind >= HC_MAP_I64_I32;
                const int kb = kind == HC_SET_U32 ? 4 : 8;
                if (!it.d_keys || reinterpret_cast<uintptr_t>(it.d_keys) % kb)
                    return bfail(HC_ERR_ARG, "item keys NULL or misaligned");
                if (op == HC_OP_INSERT && map && !it.d_vals) return bfail(HC_ERR_ARG, "insert item on a map without values");
                if (op == HC_OP_FIND && !it.d_out) return bfail(HC_ERR_ARG, "find item without a found array");
                hc::BatchItemDev d{};
                d.v = it.table->view;
                d.v.rotate = it.n > (long long)d.v.nb ? 1 : 0;
                d.keys = it.d_keys;
                d.vals = map ? it.d_vals : nullptr;
                d.out = it.d_out;
                d.vals_out = map ? it.d_vals_out : nullptr;
                d.n = it.n;
                d.chunk_begin = ph.n_chunks;
                d.bb = it.table->bucket_bytes;
                d.fold = op == HC_OP_FIND ? 0 : it.table->shape[op].fold;
                ph.n_chunks += (it.n + tile - 1) / tile;
                dev.push_back(d);
                ph.n_items++;
            }
            if (ph.n_items) phases.push_back(ph);
        }
    }

    hc_batch *b = new hc_batch();
    b->magic = kBatchMagic;
    b->block = block;
    b->tile = tile;
    b->lane_bytes = lb;
    b->kpt = kpt;
    b->use_graph = c.use_graph != 0;
    b->phases = phases;
    cudaError_t e = cudaGetDevice(&b->device);
    const size_t items_bytes = (dev.size() * sizeof(hc::BatchItemDev) + 255) / 256 * 256;
    const size_t bytes = items_bytes + 512;   // up to 36 phase counters
    if (e == cudaSuccess) e = cudaMalloc(&b->d_mem, bytes);
    if (e != cudaSuccess) {
        delete b;
        return bcuda(e, "allocating the batch descriptors");
    }
    b->d_items = static_cast<hc::BatchItemDev *>(b->d_mem);
    b->d_counters = reinterpret_cast<unsigned long long *>(static_cast<char *>(b->d_mem) + items_bytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!dev.empty())
        e = cudaMemcpyAsync(b->d_items, dev.data(), dev.size() * sizeof(hc::BatchItemDev), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    for (size_t p = 0; p < phases.size() && e == cudaSuccess; ++p) {
        int per_sm = c.blocks_per_sm;
        if (per_sm <= 0) {
            hc::PhaseKernel k = hc::pick_kernel(phases[p].kind, phases[p].op, phases[p].bb, lb, kpt);
            const size_t smem = hc::phase_smem(phases[p].kind, kpt, block);
            hc::allow_phase_smem(k, smem);
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
            if (per_sm <= 0) per_sm = 1;
        }
        long long g = (long long)sms * per_sm;
        // one warp (lock-step) or one block (streaming) per chunk at most
        const long long need = kpt >= 4 ? phases[p].n_chunks : (phases[p].n_chunks * 32 + block - 1) / block;
        if (g > need) g = need;
        b->grid.push_back((int)(g > 0 ? g : 1));
    }
    if (e == cudaSuccess && b->use_graph) {
        // capture on a private stream so the caller's stream is never in capture mode
        cudaStream_t cs;
        e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) {
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            hc_rc rc = HC_OK;
            if (e == cudaSuccess) rc = enqueue(b, cs);
            cudaError_t e2 = cudaStreamEndCapture(cs, &b->graph);
            if (e == cudaSuccess) e = e2;
            if (rc != HC_OK && e == cudaSuccess) e = cudaErrorUnknown;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
            cudaStreamDestroy(cs);
        }
    }
    if (e != cudaSuccess) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        cudaFree(b->d_mem);
        delete b;
        return bcuda(e, "building the batch");
    }
    *out = b;
    return HC_OK;
}

HC_API hc_rc hc_batch_launch(hc_batch *b, void *stream) {
    if (!b || b->magic != kBatchMagic) return bfail(HC_ERR_ARG, "invalid batch handle");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (b->exec) {
        cudaError_t e = cudaGraphLaunch(b->exec, s);
        if (e != cudaSuccess) return bcuda(e, "launching the batch graph");
        return HC_OK;
    }
    return enqueue(b, s);
}

HC_API hc_rc hc_batch_destroy(hc_batch *b) {
    if (!b) return HC_OK;
    if (b->magic != kBatchMagic) return bfail(HC_ERR_ARG, "invalid batch handle");
    b->magic = 0;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaError_t e = cudaFree(b->d_mem);
    delete b;
    if (e != cudaSuccess) return bcuda(e, "cudaFree");
    return HC_OK;
}

}  // extern "C"

// ---- batched form without any device allocation --------------------------
// hc_batch_create allocates its item descriptors and chunk counters with
// cudaMalloc.  This variant keeps them in one file-scope device array instead,
// for callers that must not allocate device memory themselves.  The array is
// part of the library image: every GPU that loads the library holds it until
// the process exits, and every call shares it.

namespace {

constexpr int kNoAllocMaxItems = 1024;   // items per call (104 KiB of descriptors)
constexpr int kNoAllocMaxPhases = 36;    // 3 operations x 4 container kinds x 3 bucket sizes

struct NoAllocScratch {
    hc::BatchItemDev items[kNoAllocMaxItems];
    unsigned long long counters[64];
};

}  // namespace

// The scratch itself.  Host code must not take its address directly (on the
// host this name is only a stand-in); the device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

namespace {

std::mutex g_noalloc_mu;
NoAllocScratch *g_noalloc_addr[64] = {nullptr};   // device address per device ordinal

// Set-up, once per device, with that device current.
hc_rc noalloc_scratch(int dev, NoAllocScratch **out) {
    if (dev < 0 || dev >= 64) return bfail(HC_ERR_ARG, "device ordinal out of range");
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return bcuda(e, "cudaGetSymbolAddress of the static batch scratch");
        g_noalloc_addr[dev] = static_cast<NoAllocScratch *>(p);
    }
    *out = g_noalloc_addr[dev];
    return HC_OK;
}

// Host-side staging of the descriptors: per host thread, fixed size, so a
// call allocates no memory on the host either.
thread_local hc::BatchItemDev t_noalloc_items[kNoAllocMaxItems];

}  // namespace

extern "C" {

HC_API hc_rc hc_batch_run_noalloc(const hc_batch_item *items, int64_t n_items, const hc_batch_config *cfg,
                                  void *stream) {
    if (n_items < 0 || (n_items > 0 && !items)) return bfail(HC_ERR_ARG, "bad item list");
    if (n_items > kNoAllocMaxItems)
        return bfail(HC_ERR_ARG, "hc_batch_run_noalloc takes at most 1024 items per call (got " +
                                     std::to_string((long long)n_items) + ")");
    hc_batch_config c{};
    if (cfg) c = *cfg;
    const int lb = c.lane_bytes;
    const int kpt = c.keys_per_group ? c.keys_per_group : 1;
    const int block = c.block ? c.block : 256;
    const int tile = c.tile ? c.tile : auto_tile(items, n_items);
    if (lb != 0 && lb != 32) return bfail(HC_ERR_ARG, "lane_bytes must be 0 (whole bucket) or 32");
    if (kpt != 1 && kpt != 2 && kpt != 4 && kpt != 8)
        return bfail(HC_ERR_ARG, "keys_per_group must be 1 or 2 (lock-step) or 4 or 8 (streaming)");
    if (kpt >= 4 && block > 256) return bfail(HC_ERR_ARG, "streaming phases take at most 256 threads per block");
    if (block < 64 || block > 256 || block % 32) return bfail(HC_ERR_ARG, "block must be a multiple of 32 in [64, 256]");
    if (tile < 128 || tile % 128) return bfail(HC_ERR_ARG, "tile must be a positive multiple of 128");
    if (c.use_graph) return bfail(HC_ERR_ARG, "hc_batch_run_noalloc launches directly; use_graph must be 0");

    // descriptors ordered by (op, kind), one phase per non-empty pair
    hc::PhaseDesc phases[kNoAllocMaxPhases];
    int n_phases = 0, n_dev = 0;
    for (int op = 0; op < 3; ++op) {
        for (int kind = 0; kind < 4; ++kind)
        for (int bb = 32; bb <= 128; bb *= 2) {
            hc::PhaseDesc ph{kind, op, bb, n_dev, 0, 0, n_phases};
            for (int64_t i = 0; i < n_items; ++i) {
                const hc_batch_item &it = items[i];
                if (!it.table || it.table->magic != HC_TABLE_MAGIC) return bfail(HC_ERR_ARG, "item with a bad table");
                if (it.op < 0 || it.op > 2) return bfail(HC_ERR_ARG, "item with a bad op");
                if (it.n < 0) return bfail(HC_ERR_ARG, "item with n < 0");
                if (it.op != op || it.table->kind != kind || it.table->bucket_bytes != bb || it.n == 0) continue;
                const bool map = kind >= HC_MAP_I64_I32;
                const int kb = kind == HC_SET_U32 ? 4 : 8;
                if (!it.d_keys || reinterpret_cast<uintptr_t>(it.d_keys) % kb)
                    return bfail(HC_ERR_ARG, "item keys NULL or misaligned");
                if (op == HC_OP_INSERT && map && !it.d_vals) return bfail(HC_ERR_ARG, "insert item on a map without values");
                if (op == HC_OP_FIND && !it.d_out) return bfail(HC_ERR_ARG, "find item without a found array");
                hc::BatchItemDev &d = t_noalloc_items[n_dev++];
                d = hc::BatchItemDev{};
                d.v = it.table->view;
                d.v.rotate = it.n > (long long)d.v.nb ? 1 : 0;
                d.keys = it.d_keys;
                d.vals = map ? it.d_vals : nullptr;
                d.out = it.d_out;
                d.vals_out = map ? it.d_vals_out : nullptr;
                d.n = it.n;
                d.chunk_begin = ph.n_chunks;
                d.bb = it.table->bucket_bytes;
                d.fold = op == HC_OP_FIND ? 0 : it.table->shape[op].fold;
                ph.n_chunks += (it.n + tile - 1) / tile;
                ph.n_items++;
            }
            if (ph.n_items) phases[n_phases++] = ph;
        }
    }
    if (n_phases == 0) return HC_OK;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return bcuda(e, "cudaGetDevice");
    NoAllocScratch *scratch = nullptr;
    hc_rc rc = noalloc_scratch(dev, &scratch);
    if (rc != HC_OK) return rc;
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return bcuda(e, "reading the SM count");

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // pageable source: the call returns once the descriptors are staged, so
    // the per-thread array may be refilled by the next call
    e = cudaMemcpyAsync(scratch->items, t_noalloc_items, (size_t)n_dev * sizeof(hc::BatchItemDev),
                        cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bcuda(e, "copying the batch descriptors");
    // the chunk counters keep the previous call's values: reset them first
    hc::k_zero_counters<<<1, 64, 0, s>>>(scratch->counters, n_phases);
    e = cudaGetLastError();
    if (e != cudaSuccess) return bcuda(e, "resetting the chunk counters");
    for (int p = 0; p < n_phases; ++p) {
        const hc::PhaseDesc &ph = phases[p];
        hc::PhaseKernel k = hc::pick_kernel(ph.kind, ph.op, ph.bb, lb, kpt);
        const size_t smem = hc::phase_smem(ph.kind, kpt, block);
        hc::allow_phase_smem(k, smem);
        int per_sm = c.blocks_per_sm;
        if (per_sm <= 0) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
            if (e != cudaSuccess) return bcuda(e, "querying occupancy");
            if (per_sm <= 0) per_sm = 1;
        }
        long long g = (long long)sms * per_sm;
        const long long need = kpt >= 4 ? ph.n_chunks : (ph.n_chunks * 32 + block - 1) / block;
        if (g > need) g = need;
        k<<<(unsigned)(g > 0 ? g : 1), block, smem, s>>>(
            scratch->items + ph.item0, ph.n_items, ph.n_chunks, tile, scratch->counters + ph.counter);
        e = cudaGetLastError();
        if (e != cudaSuccess) return bcuda(e, "launching a batch phase");
    }
    return HC_OK;
}

}  // extern "C"

// ---- dynamic batched launch with caller scratch ---------------------------
// The served form forms a new batch at every dispatch.  Building a graph or
// allocating descriptors per dispatch would cost more than small requests
// themselves, so the caller hands in a device scratch buffer (one per stream
// it dispatches on) that receives the descriptors and chunk counters.

namespace {

constexpr int kRunMaxItems = 4096;
thread_local hc::BatchItemDev t_run_items[kRunMaxItems];

}  // namespace

extern "C" {

HC_API int64_t hc_batch_scratch_bytes(int64_t n_items) {
    if (n_items < 0 || n_items > kRunMaxItems) return -1;
    return (int64_t)((n_items * sizeof(hc::BatchItemDev) + 255) / 256 * 256 + 512);   // + 36 counters
}

namespace {
hc_rc batch_run(const hc_batch_item *items, int64_t n_items, const hc_batch_config *cfg, void *d_scratch,
                int64_t scratch_bytes, void *h_pinned, void *stream);
}

HC_API hc_rc hc_batch_run(const hc_batch_item *items, int64_t n_items, const hc_batch_config *cfg, void *d_scratch,
                          int64_t scratch_bytes, void *stream) {
    return batch_run(items, n_items, cfg, d_scratch, scratch_bytes, nullptr, stream);
}

namespace {
hc_rc batch_run(const hc_batch_item *items, int64_t n_items, const hc_batch_config *cfg, void *d_scratch,
                int64_t scratch_bytes, void *h_pinned, void *stream) {
    if (n_items < 0 || (n_items > 0 && !items)) return bfail(HC_ERR_ARG, "bad item list");
    if (n_items > kRunMaxItems)
        return bfail(HC_ERR_ARG, "hc_batch_run takes at most 4096 items per call (got " +
                                     std::to_string((long long)n_items) + ")");
    if (n_items == 0) return HC_OK;
    const int64_t need = hc_batch_scratch_bytes(n_items);
    if (!d_scratch || scratch_bytes < need || reinterpret_cast<uintptr_t>(d_scratch) % 256)
        return bfail(HC_ERR_ARG, "scratch must be 256-byte aligned and hold hc_batch_scratch_bytes(n_items) = " +
                                     std::to_string((long long)need) + " bytes");
    hc_batch_config c{};
    if (cfg) c = *cfg;
    const int lb = c.lane_bytes;
    const int kpt = c.keys_per_group ? c.keys_per_group : 1;
    const int block = c.block ? c.block : 256;
    const int tile = c.tile ? c.tile : auto_tile(items, n_items);
    if (lb != 0 && lb != 32) return bfail(HC_ERR_ARG, "lane_bytes must be 0 (whole key region) or 32");
    if (kpt != 1 && kpt != 2 && kpt != 4 && kpt != 8)
        return bfail(HC_ERR_ARG, "keys_per_group must be 1 or 2 (lock-step) or 4 or 8 (streaming)");
    if (kpt >= 4 && block > 256) return bfail(HC_ERR_ARG, "streaming phases take at most 256 threads per block");
    if (block < 64 || block > 256 || block % 32) return bfail(HC_ERR_ARG, "block must be a multiple of 32 in [64, 256]");
    if (tile < 128 || tile % 128) return bfail(HC_ERR_ARG, "tile must be a positive multiple of 128");

    hc::BatchItemDev *desc = h_pinned ? static_cast<hc::BatchItemDev *>(h_pinned) : t_run_items;
    hc::PhaseDesc phases[36];
    int n_phases = 0, n_dev = 0;
    for (int op = 0; op < 3; ++op) {
        for (int kind = 0; kind < 4; ++kind)
        for (int bb = 32; bb <= 128; bb *= 2) {
            hc::PhaseDesc ph{kind, op, bb, n_dev, 0, 0, n_phases};
            for (int64_t i = 0; i < n_items; ++i) {
                const hc_batch_item &it = items[i];
                if (!it.table || it.table->magic != HC_TABLE_MAGIC) return bfail(HC_ERR_ARG, "item with a bad table");
                if (it.op < 0 || it.op > 2) return bfail(HC_ERR_ARG, "item with a bad op");
                if (it.n < 0) return bfail(HC_ERR_ARG, "item with n < 0");
                if (it.op != op || it.table->kind != kind || it.table->bucket_bytes != bb || it.n == 0) continue;
                const bool map = kind >= HC_MAP_I64_I32;
                const int kb = kind == HC_SET_U32 ? 4 : 8;
                if (!it.d_keys || reinterpret_cast<uintptr_t>(it.d_keys) % kb)
                    return bfail(HC_ERR_ARG, "item keys NULL or misaligned");
                if (op == HC_OP_INSERT && map && !it.d_vals) return bfail(HC_ERR_ARG, "insert item on a map without values");
                if (op == HC_OP_FIND && !it.d_out) return bfail(HC_ERR_ARG, "find item without a found array");
                hc::BatchItemDev &d = desc[n_dev++];
                d = hc::BatchItemDev{};
                d.v = it.table->view;
                d.v.rotate = it.n > (long long)d.v.nb ? 1 : 0;
                d.keys = it.d_keys;
                d.vals = map ? it.d_vals : nullptr;
                d.out = it.d_out;
                d.vals_out = map ? it.d_vals_out : nullptr;
                d.n = it.n;
                d.chunk_begin = ph.n_chunks;
                d.bb = it.table->bucket_bytes;
                d.fold = op == HC_OP_FIND ? 0 : it.table->shape[op].fold;
                ph.n_chunks += (it.n + tile - 1) / tile;
                ph.n_items++;
            }
            if (ph.n_items) phases[n_phases++] = ph;
        }
    }
    if (n_phases == 0) return HC_OK;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return bcuda(e, "reading the device");
    auto *d_items = static_cast<hc::BatchItemDev *>(d_scratch);
    auto *d_ctr = reinterpret_cast<unsigned long long *>(static_cast<char *>(d_scratch) + need - 512);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(d_items, desc, (size_t)n_dev * sizeof(hc::BatchItemDev), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bcuda(e, "copying the batch descriptors");
    hc::k_zero_counters<<<1, 64, 0, s>>>(d_ctr, n_phases);
    for (int p = 0; p < n_phases; ++p) {
        const hc::PhaseDesc &ph = phases[p];
        hc::PhaseKernel k = hc::pick_kernel(ph.kind, ph.op, ph.bb, lb, kpt);
        int per_sm = c.blocks_per_sm;
        const size_t smem = hc::phase_smem(ph.kind, kpt, block);
        hc::allow_phase_smem(k, smem);
        if (per_sm <= 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem) != cudaSuccess) per_sm = 1;
        if (per_sm <= 0) per_sm = 1;
        long long g = (long long)sms * per_sm;
        const long long want = kpt >= 4 ? ph.n_chunks : (ph.n_chunks * 32 + block - 1) / block;
        if (g > want) g = want;
        k<<<(unsigned)(g > 0 ? g : 1), block, smem, s>>>(d_items + ph.item0, ph.n_items, ph.n_chunks, tile,
                                                         d_ctr + ph.counter);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return bcuda(e, "launching the batch phases");
    return HC_OK;
}
}  // namespace

}  // extern "C"

namespace hc {
// hc_batch_run for callers that own page-locked staging for the descriptors
// (the served loop: one buffer per launch slot, reused only after the slot's
// launch completed), so that their copy to the device does not wait for the
// stream.
hc_rc batch_run_pinned(const hc_batch_item *items, int64_t n_items, const hc_batch_config *cfg, void *d_scratch,
                       int64_t scratch_bytes, void *h_pinned, void *stream) {
    return batch_run(items, n_items, cfg, d_scratch, scratch_bytes, h_pinned, stream);
}
size_t batch_desc_bytes(int64_t n_items) { return (size_t)n_items * sizeof(BatchItemDev); }
}  // namespace hc
