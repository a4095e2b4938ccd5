/*
 * hc.h -- C ABI of the GB300 concurrent hash-container library (libhc.so).
 *
 * The containers are the hash-based collections of "stdgpu: Efficient
 * STL-like Data Structures on the GPU" (Stotko, 2019), Section 4.1: an
 * unordered_set keeps keys, an unordered_map keeps a key and its mapped
 * value, and each key is held at most once.  Capacity is fixed when the
 * container is created (Section 4, "Capacity"); the range forms of insert,
 * erase, find and contains (Section 4.1) run over whole device arrays with a
 * result per key; inserting beyond the capacity is the only failure
 * (Section 4, "Guarantees").
 *
 * Conventions for every call below:
 *   - Data pointers named d_* are DEVICE pointers on the table's device,
 *     owned by the caller (for example torch tensors); the library never
 *     frees or keeps them after the call's work has run.  Inputs and outputs
 *     must not alias.  Key arrays must be aligned to the key size, value
 *     arrays to the value size.
 *   - Pointers named h_* are HOST pointers (pinned memory gives overlap).
 *   - Counts are signed 64-bit (Section 3.2 chooses a signed index type);
 *     n < 0 is an argument error, n == 0 is a no-op returning HC_OK.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Calls are asynchronous and ordered on `stream` unless their
 *     comment says they synchronise.  Work on one table must be ordered by
 *     the caller (one stream, or events): calls on one table are phases, and
 *     each call is one concurrent batch.
 *   - Argument errors return before anything is launched.  On error the
 *     return code is not HC_OK and hc_last_error() describes it.
 *   - Handles are not safe for concurrent host calls on the same table.
 *
 * Key types: uint32 (HC_SET_U32), uint64 (HC_SET_U64, HC_MAP_U64_U64) and
 * int64 (HC_MAP_I64_I32).  Every bit pattern is a valid key: the paper's
 * containers avoid placeholder values (Section 5.1).  The two largest bit
 * patterns of the key type (all ones, all ones minus one) are held in two side
 * slots of the table header, so they never use one of the `slots`.
 */
#ifndef HC_H
#define HC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HC_ABI_VERSION 2

#if defined(__GNUC__)
#define HC_API __attribute__((visibility("default")))
#else
#define HC_API
#endif

typedef struct hc_table hc_table;
typedef struct hc_batch hc_batch;

/* Container kinds (Section 4.1: set = keys only, map = key -> mapped value). */
typedef enum hc_kind {
    HC_SET_U32 = 0,      /* unordered_set<uint32>                       */
    HC_SET_U64 = 1,      /* unordered_set<uint64>                       */
    HC_MAP_I64_I32 = 2,  /* unordered_map<int64, int32>                 */
    HC_MAP_U64_U64 = 3   /* unordered_map<uint64, uint64>               */
} hc_kind;

/* Return codes. */
typedef enum hc_rc {
    HC_OK = 0,
    HC_ERR_ARG = 1,       /* invalid argument; nothing launched          */
    HC_ERR_OOM = 2,       /* device allocation failed                    */
    HC_ERR_OVERFLOW = 3,  /* an insert found the table full (sticky)     */
    HC_ERR_CUDA = 4,      /* a CUDA runtime call failed                  */
    HC_ERR_STATE = 5,     /* a device-side bound was hit (see hc_stats), or
                             a served run or wait could not complete       */
    HC_ERR_TIMEOUT = 6    /* a served request's deadline passed before it
                             was dispatched; nothing of it ran            */
} hc_rc;

/* Per-key status bytes written by insert and erase. */
enum {
    HC_INSERTED = 0,   /* key was absent and is now stored                */
    HC_EXISTS = 1,     /* key was already stored; its value is unchanged  */
    HC_OVERFLOW = 2,   /* key was absent and the table is full            */
    HC_ERASED = 3,     /* key was stored and is now removed               */
    HC_NOT_FOUND = 4   /* key was not stored                              */
};

/* Operation codes for batches and launch shapes. */
enum { HC_OP_INSERT = 0, HC_OP_FIND = 1, HC_OP_ERASE = 2 };

/* Bucket hash.  HC_HASH_MIX64 is a 64-bit finaliser of (key ^ seed) reduced
 * by a 64x64 high multiply; HC_HASH_TESCHNER is the spatial hash of Section
 * 4.1 (coordinates times 73856093, 19349669, 83492791, combined by xor,
 * reduced modulo the bucket count) applied to keys that pack three signed
 * 21-bit block coordinates as x | y << 21 | z << 42 (HC_MAP_I64_I32 only).
 * HC_HASH_TESCHNER_SHORT3 is the same hash on the paper's own key type, a
 * short3 of signed 16-bit block coordinates, packed into the 8-byte slot as
 * (uint16)x | (uint16)y << 16 | (uint16)z << 32 (hc_pack_short3;
 * HC_MAP_I64_I32 only).  The hash never changes a result, only where keys
 * are stored. */
enum { HC_HASH_MIX64 = 0, HC_HASH_TESCHNER = 1, HC_HASH_TESCHNER_SHORT3 = 2 };

/* Layout chosen at creation.  Zero fields take the defaults.  Keys live in an
 * array of buckets; maps keep their values in a parallel array, so a probe
 * reads keys only and a lookup that found its key reads one value. */
typedef struct hc_config {
    int32_t bucket_bytes;  /* bytes of keys per bucket: 32, 64 or 128
                              (default 32); one probe reads one bucket;
                              buckets are aligned to 32-byte sectors      */
    int32_t hash_mode;     /* HC_HASH_*; default HC_HASH_MIX64             */
    uint64_t seed;         /* hash seed (default 0)                        */
} hc_config;

/* Launch shape of one operation.  A group of bucket_bytes / lane_bytes
 * lanes probes a bucket together (lane_bytes == bucket_bytes: one thread per
 * key); each group handles keys_per_group keys at once so that several
 * bucket reads are in flight per lane.  Zero fields keep the current value.
 * keys_per_group 4 or 8 (any operation, lane_bytes = the key region)
 * selects the streaming form: a block stages its keys in shared memory and
 * each thread keeps 2 or 4 probes in flight, refilling as they finish (no
 * duplicate folding in this form).  Defaults:
 * lane_bytes = the bucket's key region (one thread per key),
 * keys_per_group 4 (streaming), block 64, folding off; until hc_set_launch
 * sets an op's shape, a plain insert of fewer than 8192 keys per
 * multiprocessor and at most one key per bucket, into a table whose buckets
 * exceed the L2 cache, runs one key per thread in lock step.  Results never
 * depend on the shape. */
typedef struct hc_launch {
    int32_t lane_bytes;       /* 32, 64 or 128, at most bucket_bytes     */
    int32_t keys_per_group;   /* 1 or 2; 4 or 8: streaming forms       */
    int32_t block;            /* threads per block: 64..256, multiple of 32  */
    int32_t fold_duplicates;  /* 1: equal keys inside a warp are folded to
                                 one probe (__match_any_sync); 2: off      */
} hc_launch;

/* Counters read back by hc_stats (synchronising). */
typedef struct hc_stats_t {
    int64_t live;            /* stored keys (Section 4.1 size)               */
    int64_t used;            /* slots not EMPTY: stored keys + tombstones,
                                excluding the two side slots                  */
    int64_t capacity;        /* slots, as requested at create / rehash       */
    int64_t slot_bytes;      /* bytes per slot: key plus value                */
    int64_t table_bytes;     /* device bytes held by the table               */
    uint32_t error_bits;     /* 1 = an insert overflowed, 2 = probe bound hit,
                                4 = a bounds check of the debug build failed
                                (a build with -DHC_DEBUG only)                */
    uint32_t reserved;
} hc_stats_t;

/* Library ABI version (HC_ABI_VERSION). */
HC_API int32_t hc_abi_version(void);

/* Message for the last error returned on this host thread ("" if none). */
HC_API const char *hc_last_error(void);

/* Device bytes a table of `slots` slots would hold (for memory budgets).
 * Fixed capacity, Section 4. */
HC_API hc_rc hc_table_bytes(int32_t kind, int64_t slots, const hc_config *cfg, int64_t *bytes);

/* Create a container with a fixed capacity of `slots` slots (Section 4,
 * "Capacity"; Section 3.7, explicit create/destroy of device objects).  The
 * slot array is allocated on the current device with cudaMalloc and
 * initialised to empty on `stream`.  slots >= 1.  *out receives the handle. */
HC_API hc_rc hc_create(hc_table **out, int32_t kind, int64_t slots, const hc_config *cfg, void *stream);

/* Destroy a table and free its device memory.  Synchronises the device
 * first so no queued work still uses it.  NULL is a no-op. */
HC_API hc_rc hc_destroy(hc_table *t);

/* Set the launch shape of one operation (HC_OP_*) on this table. */
HC_API hc_rc hc_set_launch(hc_table *t, int32_t op, const hc_launch *shape);
HC_API hc_rc hc_get_launch(const hc_table *t, int32_t op, hc_launch *shape);

/* Range insert (Section 4.1, insert): for i < n, insert d_keys[i] (and
 * d_vals[i] for maps; NULL for sets).  d_status[i] (nullable) receives
 * HC_INSERTED, HC_EXISTS (present already: stored value unchanged) or
 * HC_OVERFLOW (absent and no free slot: the only failure, Section 4).
 * Equal keys inside one batch: exactly one position gets HC_INSERTED when
 * the key was absent and fits, the others HC_EXISTS; which one is not
 * specified.  An overflow also sets the table's sticky error bit. */
HC_API hc_rc hc_insert(hc_table *t, const void *d_keys, const void *d_vals, int64_t n,
                uint8_t *d_status, void *stream);

/* The insert half of a find-then-insert over a stream of candidate keys
 * (the pattern of the Section 4.1 examples, which add only blocks that are
 * not stored yet): d_found[i] is the flag hc_find wrote for the same
 * d_keys[i], with no call on this table in between.  Keys whose flag is set
 * get HC_EXISTS without a probe; the others are inserted exactly as by
 * hc_insert.  Allocates nothing and needs no host synchronisation. */
HC_API hc_rc hc_insert_if_absent(hc_table *t, const void *d_keys, const void *d_vals, const uint8_t *d_found,
                                 int64_t n, uint8_t *d_status, void *stream);

/* Range find / contains (Section 4.1): d_found[i] = 1 if d_keys[i] is
 * stored, else 0.  For maps, d_vals_out[i] (nullable: contains only)
 * receives the mapped value, or 0 when absent.  Lookups take no lock. */
HC_API hc_rc hc_find(hc_table *t, const void *d_keys, int64_t n, uint8_t *d_found,
              void *d_vals_out, void *stream);

/* Range erase (Section 4.1): d_status[i] (nullable) receives HC_ERASED or
 * HC_NOT_FOUND.  Equal keys in one batch: one HC_ERASED at most.  An erased
 * slot becomes a tombstone that later inserts reuse. */
HC_API hc_rc hc_erase(hc_table *t, const void *d_keys, int64_t n, uint8_t *d_status,
               void *stream);

/* Host-buffer forms of the three range calls: keys, values and results are
 * HOST arrays.  When every array of a call is page-locked (cudaHostAlloc or
 * cudaHostRegister), the kernels read and write them in host memory directly
 * through their mapped addresses (over NVLink-C2C on a Grace-Blackwell
 * node): one launch, no copies.  Otherwise the library copies them in chunks
 * through device staging buffers that the table allocates on first use and
 * keeps, overlapping the copies with the kernels.  Both return after the
 * results are on the host (synchronising `stream`). */
HC_API hc_rc hc_insert_host(hc_table *t, const void *h_keys, const void *h_vals, int64_t n,
                     uint8_t *h_status, void *stream);
HC_API hc_rc hc_find_host(hc_table *t, const void *h_keys, int64_t n, uint8_t *h_found,
                   void *h_vals_out, void *stream);
HC_API hc_rc hc_erase_host(hc_table *t, const void *h_keys, int64_t n, uint8_t *h_status,
                    void *stream);

/* Number of stored keys (Section 4.1).  Synchronises `stream`. */
HC_API hc_rc hc_size(hc_table *t, int64_t *live, void *stream);

/* All counters (synchronises `stream`). */
HC_API hc_rc hc_stats(hc_table *t, hc_stats_t *out, void *stream);

/* HC_ERR_OVERFLOW if an insert overflowed since the last call, HC_ERR_STATE
 * if a device-side bound was hit, else HC_OK; clears the sticky bits.
 * Synchronises `stream`. */
HC_API hc_rc hc_status(hc_table *t, void *stream);

/* Remove every key (the table returns to its state after create). */
HC_API hc_rc hc_clear(hc_table *t, void *stream);

/* Manual resize on the host (Section 4, "Capacity"): move the stored keys
 * into a new slot array of `new_slots` slots (which may equal the current
 * capacity: this purges tombstones).  HC_ERR_ARG if new_slots is below the
 * number of stored keys that use a slot.  Synchronises `stream`; the old
 * array is freed before returning. */
HC_API hc_rc hc_rehash(hc_table *t, int64_t new_slots, void *stream);

/* Copy the stored keys (and values for maps; d_vals_out may be NULL) into
 * device arrays of `cap` entries, in unspecified order (Section 3.6, a range
 * over a container's stored entries).  *n_out receives the number of stored
 * keys; if it exceeds cap only cap entries are written and HC_ERR_ARG is
 * returned.  Synchronises `stream`. */
HC_API hc_rc hc_dump(hc_table *t, void *d_keys_out, void *d_vals_out, int64_t cap,
              int64_t *n_out, void *stream);

/* ---- short3 keys ----------------------------------------------------------
 * Section 4.1's voxel-block map is keyed by short3 (three signed 16-bit
 * block coordinates, 6 bytes).  A map<int64, int32> created with
 * HC_HASH_TESCHNER_SHORT3 keeps such keys packed into its 8-byte slots as
 * (uint16)x | (uint16)y << 16 | (uint16)z << 32 (bits 48-63 zero, so a packed
 * key is never a side-slot pattern) and hashes them with the paper's spatial
 * hash on the three coordinates.  These calls convert device arrays of n
 * short3 (int16 x, y, z consecutive, 2-byte aligned, 6 bytes per key) to and
 * from packed keys (8-byte aligned int64).  Asynchronous on `stream`. */
HC_API hc_rc hc_pack_short3(const int16_t *d_xyz, int64_t n, int64_t *d_keys, void *stream);
HC_API hc_rc hc_unpack_short3(const int64_t *d_keys, int64_t n, int16_t *d_xyz, void *stream);

/* ---- free-running mixed batches --------------------------------------------
 * One launch in which inserts, finds and erases of the same table run at
 * once (Section 4, "Guarantees": concurrency across all defined operations),
 * under the contract of the in-kernel functions of include/hc_device.cuh:
 * for every key the results are those of some serial order of that key's
 * operations, no key is stored twice, map values are seen only with their
 * keys, inserts claim EMPTY slots only (tombstones return with hc_clear /
 * hc_rehash).  No order across keys and no phase order is implied (the
 * batched form's phases are the ordered alternative).  The kernel stages
 * each block's operations in shared memory and keeps several of them in
 * flight per thread, as the range kernels do.
 *   d_ops[i]: 0 insert, 1 find, 2 erase (any other value erases).
 *   d_status[i] (may be NULL): insert / erase status, or 1 / 0 for a find
 *     that found / did not find its key.
 *   d_vals: n map values, used at insert positions;
 *   d_vals_out (maps, may be NULL): the value found at find positions, 0 at
 *     every other position.
 * Allocates nothing; asynchronous on `stream`. */
HC_API hc_rc hc_apply_mixed(hc_table *t, const uint8_t *d_ops, const void *d_keys, const void *d_vals, int64_t n,
                            uint8_t *d_status, void *d_vals_out, void *stream);

/* ---- ordered duplicates: the lowest index wins ---------------------------
 * Section 4 leaves which of several equal keys of one concurrent call
 * succeeds to the scheduler (the plain calls report one INSERTED or ERASED
 * per key, at any of its positions, and a map keeps any one of the equal
 * keys' values).  The ordered calls give every position the result of
 * processing the batch sequentially in index order: the first occurrence of
 * a key probes the container (its value is the one a map stores), every
 * later occurrence reports EXISTS (OVERFLOW if the first overflowed) for an
 * insert and NOT_FOUND for an erase.  Which distinct keys overflow a full
 * table is still unspecified.
 *
 * d_scratch: device memory of hc_ordered_scratch_bytes(n) bytes, 256-byte
 * aligned, owned by the caller, free for reuse once the call's work on
 * `stream` is done (32 to 64 bytes per key, plus 9n bytes).  Asynchronous.
 * HC_ERR_ARG if the scratch is NULL, misaligned or too small. */
HC_API int64_t hc_ordered_scratch_bytes(int64_t n);
HC_API hc_rc hc_insert_ordered(hc_table *t, const void *d_keys, const void *d_vals, int64_t n, uint8_t *d_status,
                               void *d_scratch, int64_t scratch_bytes, void *stream);
HC_API hc_rc hc_erase_ordered(hc_table *t, const void *d_keys, int64_t n, uint8_t *d_status, void *d_scratch,
                              int64_t scratch_bytes, void *stream);

/* ---- selection over the stored entries ----------------------------------
 * Section 3.6 selects, for example, the voxel blocks a camera sees: a range
 * over a container's stored entries, copied with a predicate through a back
 * inserter into a vector.  hc_select does this with the predicates below;
 * kernels of the caller's own can use any predicate with hcd::copy_if of
 * include/hc_device.cuh. */
typedef enum hc_pred_kind {
    HC_PRED_ALL = 0,          /* every stored entry                                  */
    HC_PRED_KEY_RANGE = 1,    /* lo <= key <= hi, compared in the key type: uint32
                                 (HC_SET_U32, lo/hi taken mod 2^32), uint64, or int64
                                 (HC_MAP_I64_I32)                                     */
    HC_PRED_VALUE_RANGE = 2,  /* maps: lo <= value <= hi in the value type, uint64 or
                                 int32 (lo/hi as int64)                               */
    HC_PRED_KEY_MASK = 3,     /* (key & lo) == hi on the key's bits                   */
    HC_PRED_BLOCK_BOX = 4,    /* 64-bit keys packing three signed 21-bit block
                                 coordinates x | y << 21 | z << 42 (Section 4.1's
                                 voxel blocks): box[0] <= x <= box[1],
                                 box[2] <= y <= box[3], box[4] <= z <= box[5]        */
    HC_PRED_SHORT3_BOX = 5    /* the same box on packed short3 keys
                                 (uint16)x | (uint16)y << 16 | (uint16)z << 32       */
} hc_pred_kind;

typedef struct hc_predicate {
    int32_t kind;     /* hc_pred_kind                                          */
    int32_t negate;   /* 0, or 1 to select the entries the predicate rejects   */
    int64_t lo, hi;   /* bounds, or mask and match                             */
    int32_t box[6];   /* HC_PRED_BLOCK_BOX bounds, inclusive                   */
} hc_predicate;

/* Append every stored (key, value) that satisfies *pred to device arrays of
 * `cap` entries, d_keys_out and (maps, may be NULL) d_vals_out, through
 * *d_count: a DEVICE int64 holding the output vector's current size.  Each
 * selected entry goes to the position *d_count had before it and increments
 * it, so several calls append one after another; entries at positions >= cap
 * are counted but not written (the caller sees *d_count > cap).  Order of the
 * appended entries is unspecified.  Asynchronous on `stream`; no insert or
 * erase may run on the table meanwhile.  HC_ERR_ARG for a NULL d_count or
 * pred, an unknown predicate kind, HC_PRED_VALUE_RANGE on a set, or a box
 * predicate on HC_SET_U32. */
HC_API hc_rc hc_select(hc_table *t, const hc_predicate *pred, void *d_keys_out, void *d_vals_out, int64_t cap,
                       int64_t *d_count, void *stream);

/* ---- in-kernel access: the function form inside the caller's kernels ----
 * Section 4.1 lets single threads of a custom kernel call insert, find,
 * contains and erase on a container passed to the kernel by value (a shallow
 * copy, Section 3.7), with insertion as reliable as the range form.  The
 * device functions live in include/hc_device.cuh; a kernel receives the
 * hc_device_view below by value and wraps it in hcd::Table<kind>.
 *
 * Concurrency contract of the device functions (Section 4, "Guarantees":
 * concurrency across all defined operations):
 *   - Any mix of insert / find / contains / erase, from any threads of any
 *     kernels, may run concurrently on one table.  The results for one key
 *     are those of some serial order of that key's operations, and a key is
 *     never stored twice.
 *   - A map insert writes the value before its key becomes visible: it
 *     claims an EMPTY slot by swapping in a marker (the key pattern all ones
 *     minus two), stores the value, then the key, so a find that sees a key
 *     reads the value stored with it.  No lock is taken; an insert that
 *     meets a claim in progress where its own key could be going reads the
 *     bucket again until the claim resolves.  Lookups and erases never wait
 *     (Section 4, "Concurrency": lookups are non-blocking).  A key equal to
 *     the marker is an ordinary key; the table header records where it is
 *     stored.
 *   - In-kernel inserts claim EMPTY slots only, never tombstones: a
 *     tombstone reused concurrently with another insert of the same key could
 *     store the key twice.  Erased slots are reclaimed by hc_clear or
 *     hc_rehash (or by range inserts), and an in-kernel insert returns
 *     OVERFLOW when the key's probe sequence holds no EMPTY slot.
 *   - Kernels that use the device functions and range calls on the same
 *     table must be ordered (one stream, or events), like any two calls.
 *
 * hc_device_view fills *out for table t; it allocates nothing and launches
 * nothing (`stream` is unused).  The view stays valid until the table is
 * rehashed or destroyed. */
typedef struct hc_device_view {
    void *buckets;          /* device: nb buckets of bucket_bytes bytes          */
    void *header;           /* device: the table header (counters, side slots)   */
    uint64_t nb;            /* number of buckets                                 */
    uint64_t seed;          /* hash seed                                         */
    int32_t kind;           /* hc_kind                                           */
    int32_t bucket_bytes;   /* 32, 64 or 128                                     */
    int32_t hash_mode;      /* HC_HASH_*                                         */
    int32_t pad_from;       /* slots of the last bucket at positions >= pad_from are padding */
} hc_device_view;

HC_API hc_rc hc_device_view_get(hc_table *t, hc_device_view *out, void *stream);

/* Device calibration: the time of one launch of n_reads reads of 32 bytes at
 * pseudo-random 32-byte-aligned offsets of d_buf (buf_bytes >= 64, 32-byte
 * aligned; its last 32 bytes may be overwritten), averaged over `reps`
 * launches after one warm-up, in *ms_per_launch.  Every probe of a table is a
 * random read, so n_reads / time is the ceiling of a probe-bound operation on
 * this device.  Synchronises `stream`.  The paper has no counterpart. */
HC_API hc_rc hc_measure_random_reads(const void *d_buf, int64_t buf_bytes, int64_t n_reads, int32_t reps,
                                     float *ms_per_launch, void *stream);

/* ---- batched form: many tables in one persistent launch -----------------
 * Not in the paper (it has one container per call); it schedules many of the
 * Section 4.1 range calls at once.  A batch holds items; each item is one
 * range call (op, table, arrays) exactly as in hc_insert / hc_find /
 * hc_erase.  The batch runs as three phases -- all insert items, then all
 * find items, then all erase items -- each phase one persistent kernel in
 * which warps take fixed-size tiles of any item from a shared counter.  Items
 * on the same table in the same phase form one concurrent batch. */
typedef struct hc_batch_item {
    hc_table *table;
    int32_t op;            /* HC_OP_*                                      */
    int32_t reserved;
    const void *d_keys;
    const void *d_vals;    /* insert into a map: values; else NULL         */
    int64_t n;
    uint8_t *d_out;        /* insert/erase: status (nullable); find: found */
    void *d_vals_out;      /* find on a map: values (nullable)             */
} hc_batch_item;

typedef struct hc_batch_config {
    int32_t lane_bytes;      /* 0: one thread per key (whole bucket); 32: 32-byte lanes */
    int32_t keys_per_group;  /* 1 or 2: lock-step phases (default 1); 4 or 8:
                                streaming phases (keys staged per block, 2 or
                                4 probes in flight per thread; block <= 256) */
    int32_t block;           /* threads per block (0 = 256)                */
    int32_t blocks_per_sm;   /* persistent grid = SMs x this (0 = auto)    */
    int32_t tile;            /* keys per chunk, a multiple of 128 (0 = auto:
                                128..1024 from the total keys, so that the
                                chunks can occupy every warp slot)          */
    int32_t use_graph;       /* 1: capture the three phases in a CUDA graph */
} hc_batch_config;

/* Build a batch over `n_items` items (copied; the arrays they point to must
 * stay valid while the batch is used).  With use_graph the three phase
 * kernels are captured once into a CUDA graph on `stream`. */
HC_API hc_rc hc_batch_create(hc_batch **out, const hc_batch_item *items, int64_t n_items,
                      const hc_batch_config *cfg, void *stream);

/* Run a batch on `stream` (a graph launch when captured). */
HC_API hc_rc hc_batch_launch(hc_batch *b, void *stream);

/* Destroy a batch (synchronises the device first). */
HC_API hc_rc hc_batch_destroy(hc_batch *b);

/* Device scratch bytes hc_batch_run needs for n_items items (-1 if n_items
 * is outside [0, 4096]). */
HC_API int64_t hc_batch_scratch_bytes(int64_t n_items);

/* Run n_items items once as a batch (the same phases and scheduling as a
 * batch from hc_batch_create, without a graph), with the descriptors and
 * chunk counters in the caller's device buffer d_scratch (256-byte aligned,
 * at least hc_batch_scratch_bytes(n_items) bytes).  Nothing is allocated and
 * nothing is kept, so a caller forming a new batch for every dispatch (a
 * request loop) pays no allocation.  Calls on different streams need
 * different scratch buffers; calls ordered on one stream may share one.  At
 * most 4096 items. */
HC_API hc_rc hc_batch_run(const hc_batch_item *items, int64_t n_items, const hc_batch_config *cfg, void *d_scratch,
                          int64_t scratch_bytes, void *stream);

/* The batched form for callers that must not allocate device memory: runs
 * `n_items` items (at most 1024) exactly like a batch built by
 * hc_batch_create and launched once, without a graph (cfg->use_graph must be
 * 0), but allocates nothing.  Some callers cannot call cudaMalloc: a serving
 * process whose device memory is all owned by another allocator's pool, or a
 * latency-bound request loop where an allocation's implicit device-wide
 * synchronisation would stall every other stream.  The descriptors and chunk
 * counters live in one fixed array (about 105 KB) inside the library, which
 * every GPU that loads the library holds until the process exits.
 *   - The first call on a device looks up that array's device address
 *     (cudaGetSymbolAddress) with the device current; make that first call
 *     before any stream capture.  The address is kept for the life of the
 *     process: after cudaDeviceReset (a new primary context) the library
 *     must be loaded again before this call is used.
 *   - Every call shares the array; the counters are reset by each call, the
 *     descriptors are overwritten.  Calls whose work overlaps on the GPU (on
 *     different streams, or several host threads) race on the array and give
 *     wrong results: order them on one stream.
 *   - More than 1024 items is HC_ERR_ARG.
 * The paper has no counterpart to this call. */
HC_API hc_rc hc_batch_run_noalloc(const hc_batch_item *items, int64_t n_items, const hc_batch_config *cfg,
                                  void *stream);

/* ---- served form: a continuous-batching request loop ---------------------
 * Not in the paper (which has one container per call); it serves the range
 * calls of Section 4.1 to a stream of requests over resident tables.  A
 * request is one insert / find / erase of a host key array on one table.
 * The loop:
 *   1. an arrived request joins its table's FIFO; a table belongs to one lane
 *      (table index mod lanes);
 *   2. each lane owns `depth` launch slots; a slot is a CUDA stream of its
 *      own, a device staging buffer of slot_bytes (keys, values, results)
 *      with pinned host staging of the same size, and descriptor scratch --
 *      the slots and the resident tables are the whole HBM budget;
 *   3. a free slot takes the heads of its lane's FIFOs, one per table and only
 *      of tables with nothing in another slot (so a table's requests run in
 *      arrival order), while they fit (at most max_items); with merge = 1 it
 *      takes either small requests (up to 65536 keys), run as one
 *      hc_batch_run (or as the range call of a lone one), or one large
 *      request, run as its range call; with merge = 0 one request.  Merged
 *      mode merges only what the lane's free slots cannot take one by one:
 *      with w heads waiting and f free slots, a slot takes w - f + 1 of them
 *      and each other free slot one.  A request whose arrays are all
 *      page-locked (keys, values of a map insert, status, values out of a
 *      map find) runs where it is: the kernels read and write those arrays
 *      through their mapped addresses (over NVLink-C2C), with no copy and
 *      no room taken in the slot.  For the others the slot copies the inputs
 *      host->device (small requests packed into one copy) and the results
 *      back.  It launches and records an event;
 *   4. a finished slot hands each request its results and completion time.
 * A request larger than a slot that does not run in place is cut into
 * chunks that fit, run one after another before the table's next request;
 * each chunk is one concurrent batch of the request's operation.  Requests
 * wait for a slot; a request is dropped only when its deadline passes before
 * any of it was dispatched.
 *
 * Two ways to feed the loop:
 *   - hc_server_run: a list of requests with arrival times, served on the
 *     calling thread; returns when every request is done;
 *   - hc_server_start: the loop runs on a thread of the server's own;
 *     hc_server_submit hands it requests from any host thread while it runs
 *     (they arrive when submitted), hc_server_wait blocks until one is done,
 *     hc_server_stop serves what was submitted and ends the loop.
 * One server runs one loop at a time. */
typedef struct hc_server hc_server;

typedef struct hc_serve_config {
    int32_t lanes;           /* groups of tables sharing slots (default 4)       */
    int32_t depth;           /* launch slots per lane (default 2)                */
    int64_t slot_bytes;      /* device (and pinned host) bytes per slot (default 64 MiB, at least 64 KiB) */
    int32_t merge;           /* 1: one batched launch per slot; 0: one call per request */
    int32_t max_items;       /* requests per merged launch (default 256, at most 4096) */
    hc_batch_config batch;   /* shape of the merged launches (use_graph must be 0) */
} hc_serve_config;

typedef struct hc_request {
    int32_t table;           /* index into the server's tables                  */
    int32_t op;              /* HC_OP_*                                          */
    const void *h_keys;      /* host keys (pinned memory copies asynchronously)  */
    const void *h_vals;      /* host values of a map insert, else NULL           */
    int64_t n;               /* keys                                            */
    uint8_t *h_status;       /* host output: insert/erase status or found flags  */
    void *h_vals_out;        /* host output: values of a map find, may be NULL   */
    double arrival;          /* seconds after the loop started: given to
                                hc_server_run; written by hc_server_submit       */
    double deadline;         /* seconds after arrival by which the request must
                                be dispatched, else it is dropped (0: none)      */
    double done;             /* written: seconds after the start when the host
                                holds the results (or the request was dropped)  */
    int32_t rc;              /* written: HC_OK when served, HC_ERR_TIMEOUT when
                                dropped; -1 while queued or running              */
    int32_t reserved;
} hc_request;

typedef struct hc_serve_stats {
    int64_t requests, ops, launches, queued_max;
    int64_t timed_out;                        /* requests dropped at their deadline */
    double wall_s;
    double p50_ms, p99_ms, p999_ms, max_ms;   /* latency of the served requests:
                                                 arrival (0 when not realtime) to done */
} hc_serve_stats;

/* tables: n_tables handles on the current device; the server keeps the
 * pointers (the tables must outlive it).  Allocates the slots. */
HC_API hc_rc hc_server_create(hc_server **out, hc_table *const *tables, int32_t n_tables, const hc_serve_config *cfg);
/* Serve `reqs` (sorted by arrival).  realtime = 1 admits a request when its
 * arrival time has passed; 0 treats every request as arrived at the start (a
 * capacity run).  Synchronises the device first (work queued on any stream
 * before the run comes first).  Returns when every request is done or
 * dropped (HC_ERR_STATE after timeout_s seconds).  Fills each request's
 * outputs, `done` and `rc`, and *stats (may be NULL).  HC_ERR_ARG while the
 * server's own loop is running. */
HC_API hc_rc hc_server_run(hc_server *srv, hc_request *reqs, int64_t n_reqs, int32_t realtime, double timeout_s,
                           hc_serve_stats *stats);
/* Start the server's own loop on a new host thread (synchronises the device
 * first).  The loop uses the tables' device and the server's streams. */
HC_API hc_rc hc_server_start(hc_server *srv);
/* Hand *req to the running loop; callable from any host thread, returns at
 * once.  req->arrival is set to now; the request and its arrays must stay
 * valid, and must not be read or written by the caller, until
 * hc_server_wait on it returned (or hc_server_stop did).  HC_ERR_STATE if
 * the loop is not running or is stopping. */
HC_API hc_rc hc_server_submit(hc_server *srv, hc_request *req);
/* Block until *req (submitted to this server) is done: HC_OK with its
 * outputs filled, HC_ERR_TIMEOUT if its deadline passed before it was
 * dispatched, or HC_ERR_TIMEOUT / HC_ERR_STATE if timeout_s passed or the
 * loop ended first. */
HC_API hc_rc hc_server_wait(hc_server *srv, hc_request *req, double timeout_s);
/* Serve every submitted request, end the loop and join its thread; *stats
 * (may be NULL) receives the loop's statistics. */
HC_API hc_rc hc_server_stop(hc_server *srv, hc_serve_stats *stats);
/* Destroy a server (stops its loop first if it runs). */
HC_API hc_rc hc_server_destroy(hc_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* HC_H */
