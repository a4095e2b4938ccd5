/*
 * hc_oracle.c -- plain, slow, single-threaded CPU oracle for the concurrent
 * hash containers (unordered_set / unordered_map over integer keys) of
 * "stdgpu: Efficient STL-like Data Structures on the GPU" (Stotko, 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  It shares no code,
 * header, constant or helper with the GPU library, and the GPU library never
 * calls it.
 *
 * What it computes (Section 4, "Container", and Section 4.1):
 *   - a container is created with a fixed capacity (Section 4, "Capacity");
 *   - each key is held at most once (Section 4.1, uniqueness guarantee);
 *   - a set stores keys only, a map stores a key and its mapped value
 *     (Section 4.1, the map/set distinction);
 *   - insert adds a key (and value) unless the key is already present, in
 *     which case nothing changes and the result is "already there"; erase
 *     removes a key; find returns the mapped value or "not found"; contains
 *     returns presence only (Section 4.1, the insert / erase / find /
 *     contains list);
 *   - inserting beyond the capacity is the only failure (Section 4,
 *     "Guarantees"); the oracle reports it per key and changes nothing.
 *
 * A batch of n operations is defined as the same operations applied one at a
 * time in index order.  Concurrency in the GPU version does not change which
 * keys end up stored (Section 4, "Concurrency": failed internal attempts are
 * retried, lookups are non-blocking), so a sequential hash table is the exact
 * definition.  The table here is textbook separate chaining: an array of
 * chain heads and a pool of {key, value, next} nodes.  Its own hash is
 * Fibonacci (Knuth multiplicative) hashing; it is unrelated to the GPU hash
 * and cannot change any result.
 *
 * Capacity reading.  Section 5.1 says the containers avoid placeholder key
 * values, so every bit pattern is a valid key.  The capacity is the number of
 * storage slots; the two largest bit patterns of the key type (all ones, and
 * all ones minus one) are held outside the slots and never count against the
 * capacity.  An insert of any other absent key fails with OVERFLOW when
 * `capacity` such keys are already stored.
 *
 * Status codes (uint8 per key) follow the library's public meaning:
 *   insert: 0 INSERTED, 1 EXISTS, 2 OVERFLOW
 *   erase:  3 ERASED, 4 NOT_FOUND
 *   find:   found[i] = 1 if present else 0; value 0 when absent.
 *
 * Parity pins for this file: a brute-force sorted-array model and the C++
 * standard library's unordered_map / unordered_set (tests/test_oracle_*.py).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { O_SET_U32 = 0, O_SET_U64 = 1, O_MAP_I64_I32 = 2, O_MAP_U64_U64 = 3 };
enum { O_INSERTED = 0, O_EXISTS = 1, O_OVERFLOW = 2, O_ERASED = 3, O_NOT_FOUND = 4 };

typedef struct otable {
    int kind;
    int64_t capacity;      /* slots for keys other than the two reserved patterns */
    int64_t live;          /* all stored keys */
    int64_t live_regular;  /* stored keys that occupy a slot */
    int64_t nheads;        /* power of two */
    int64_t *heads;        /* node index or -1 */
    uint64_t *nkey, *nval; /* node pool */
    int64_t *nnext;
    int64_t ncap, ntop, freelist;
} otable;

static int is_map(int kind) { return kind == O_MAP_I64_I32 || kind == O_MAP_U64_U64; }

/* Reserved bit patterns of the key type: all ones and all ones minus one. */
static int is_reserved(int kind, uint64_t k)
{
    if (kind == O_SET_U32) return k == 0xFFFFFFFFull || k == 0xFFFFFFFEull;
    return k == ~0ull || k == ~0ull - 1;
}

static uint64_t read_key(int kind, const void *keys, int64_t i)
{
    if (kind == O_SET_U32) return ((const uint32_t *)keys)[i];
    return ((const uint64_t *)keys)[i]; /* int64 keys are kept as their bit pattern */
}

static uint64_t read_val(int kind, const void *vals, int64_t i)
{
    if (kind == O_MAP_I64_I32) return (uint32_t)((const int32_t *)vals)[i];
    if (kind == O_MAP_U64_U64) return ((const uint64_t *)vals)[i];
    return 0;
}

static void write_val(int kind, void *vals, int64_t i, uint64_t v)
{
    if (!vals) return;
    if (kind == O_MAP_I64_I32) ((int32_t *)vals)[i] = (int32_t)(uint32_t)v;
    else if (kind == O_MAP_U64_U64) ((uint64_t *)vals)[i] = v;
}

static void write_key(int kind, void *keys, int64_t i, uint64_t k)
{
    if (kind == O_SET_U32) ((uint32_t *)keys)[i] = (uint32_t)k;
    else ((uint64_t *)keys)[i] = k;
}

static int log2i(int64_t p) { int r = 0; while (((int64_t)1 << r) < p) ++r; return r; }

static int64_t head_of(const otable *t, uint64_t k)
{
    int bits = log2i(t->nheads);
    if (bits == 0) return 0;
    return (int64_t)((k * 0x9E3779B97F4A7C15ull) >> (64 - bits));
}

/* Index of the node holding k, or -1. */
static int64_t lookup(const otable *t, uint64_t k)
{
    for (int64_t n = t->heads[head_of(t, k)]; n >= 0; n = t->nnext[n])
        if (t->nkey[n] == k) return n;
    return -1;
}

static int grow_heads(otable *t)
{
    int64_t nh = t->nheads * 2;
    int64_t *h = (int64_t *)malloc((size_t)nh * sizeof(int64_t));
    if (!h) return -1;
    for (int64_t i = 0; i < nh; ++i) h[i] = -1;
    int64_t old = t->nheads;
    int64_t *oh = t->heads;
    t->heads = h;
    t->nheads = nh;
    for (int64_t b = 0; b < old; ++b) {
        int64_t n = oh[b];
        while (n >= 0) {
            int64_t next = t->nnext[n];
            int64_t hb = head_of(t, t->nkey[n]);
            t->nnext[n] = t->heads[hb];
            t->heads[hb] = n;
            n = next;
        }
    }
    free(oh);
    return 0;
}

static int64_t new_node(otable *t)
{
    if (t->freelist >= 0) {
        int64_t n = t->freelist;
        t->freelist = t->nnext[n];
        return n;
    }
    if (t->ntop == t->ncap) {
        int64_t nc = t->ncap ? t->ncap * 2 : 1024;
        uint64_t *k = (uint64_t *)realloc(t->nkey, (size_t)nc * sizeof(uint64_t));
        if (!k) return -1;
        t->nkey = k;
        uint64_t *v = (uint64_t *)realloc(t->nval, (size_t)nc * sizeof(uint64_t));
        if (!v) return -1;
        t->nval = v;
        int64_t *x = (int64_t *)realloc(t->nnext, (size_t)nc * sizeof(int64_t));
        if (!x) return -1;
        t->nnext = x;
        t->ncap = nc;
    }
    return t->ntop++;
}

otable *o_create(int kind, int64_t capacity)
{
    if (kind < O_SET_U32 || kind > O_MAP_U64_U64 || capacity < 1) return NULL;
    otable *t = (otable *)calloc(1, sizeof(otable));
    if (!t) return NULL;
    t->kind = kind;
    t->capacity = capacity;
    t->nheads = 1024;
    t->heads = (int64_t *)malloc((size_t)t->nheads * sizeof(int64_t));
    if (!t->heads) { free(t); return NULL; }
    for (int64_t i = 0; i < t->nheads; ++i) t->heads[i] = -1;
    t->freelist = -1;
    return t;
}

void o_destroy(otable *t)
{
    if (!t) return;
    free(t->heads);
    free(t->nkey);
    free(t->nval);
    free(t->nnext);
    free(t);
}

/* One insert: the key-uniqueness rule first, then the capacity rule. */
static int insert_one(otable *t, uint64_t k, uint64_t v)
{
    if (lookup(t, k) >= 0) return O_EXISTS;          /* value left unchanged */
    int reserved = is_reserved(t->kind, k);
    if (!reserved && t->live_regular == t->capacity) return O_OVERFLOW;
    if (t->live >= t->nheads && grow_heads(t) != 0) return O_OVERFLOW;
    int64_t n = new_node(t);
    if (n < 0) return O_OVERFLOW;
    int64_t b = head_of(t, k);
    t->nkey[n] = k;
    t->nval[n] = v;
    t->nnext[n] = t->heads[b];
    t->heads[b] = n;
    t->live += 1;
    if (!reserved) t->live_regular += 1;
    return O_INSERTED;
}

static int erase_one(otable *t, uint64_t k)
{
    int64_t b = head_of(t, k);
    int64_t prev = -1;
    for (int64_t n = t->heads[b]; n >= 0; prev = n, n = t->nnext[n]) {
        if (t->nkey[n] != k) continue;
        if (prev < 0) t->heads[b] = t->nnext[n];
        else t->nnext[prev] = t->nnext[n];
        t->nnext[n] = t->freelist;
        t->freelist = n;
        t->live -= 1;
        if (!is_reserved(t->kind, k)) t->live_regular -= 1;
        return O_ERASED;
    }
    return O_NOT_FOUND;
}

void o_insert(otable *t, const void *keys, const void *vals, int64_t n, uint8_t *status)
{
    for (int64_t i = 0; i < n; ++i) {
        uint64_t k = read_key(t->kind, keys, i);
        uint64_t v = (is_map(t->kind) && vals) ? read_val(t->kind, vals, i) : 0;
        int s = insert_one(t, k, v);
        if (status) status[i] = (uint8_t)s;
    }
}

void o_find(otable *t, const void *keys, int64_t n, uint8_t *found, void *vals_out)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t nd = lookup(t, read_key(t->kind, keys, i));
        if (found) found[i] = (uint8_t)(nd >= 0);
        if (vals_out && is_map(t->kind)) write_val(t->kind, vals_out, i, nd >= 0 ? t->nval[nd] : 0);
    }
}

void o_erase(otable *t, const void *keys, int64_t n, uint8_t *status)
{
    for (int64_t i = 0; i < n; ++i) {
        int s = erase_one(t, read_key(t->kind, keys, i));
        if (status) status[i] = (uint8_t)s;
    }
}

int64_t o_size(const otable *t) { return t->live; }
int64_t o_size_regular(const otable *t) { return t->live_regular; }
int64_t o_capacity(const otable *t) { return t->capacity; }

void o_clear(otable *t)
{
    for (int64_t i = 0; i < t->nheads; ++i) t->heads[i] = -1;
    t->ntop = 0;
    t->freelist = -1;
    t->live = 0;
    t->live_regular = 0;
}

/* Manual resize on the host (Section 4, "Capacity"): the contents are kept,
 * only the capacity changes.  Refused (-1) below the stored regular keys. */
int o_rehash(otable *t, int64_t new_capacity)
{
    if (new_capacity < 1 || new_capacity < t->live_regular) return -1;
    t->capacity = new_capacity;
    return 0;
}

/* All stored (key, value) pairs, in chain order; returns the count, writes at
 * most `cap` of them. */
int64_t o_dump(const otable *t, void *keys_out, void *vals_out, int64_t cap)
{
    int64_t c = 0;
    for (int64_t b = 0; b < t->nheads; ++b)
        for (int64_t n = t->heads[b]; n >= 0; n = t->nnext[n]) {
            if (c < cap) {
                if (keys_out) write_key(t->kind, keys_out, c, t->nkey[n]);
                write_val(t->kind, vals_out, c, t->nval[n]);
            }
            ++c;
        }
    return c;
}
