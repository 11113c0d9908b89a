// kc_api.cu -- the C ABI: context, argument validation, region tables,
// scratch management and the launch sequence of every entry point.
//
// Region tables (a 32-byte record per region, page offsets, sorted census
// ranges, comparison pairs) are built and validated on the host the first
// time a call sees a given descriptor list, uploaded once, and kept in a
// per-context cache keyed by the exact descriptor bytes and parameters.  A
// repeated call (the common case: the same snapshot digested, restored and
// compared again and again) does no host-side table work and no upload, so
// the host enqueues kernels faster than the GPU runs them, and the call can
// be captured into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <list>
#include <string>
#include <vector>

#include "kc_internal.cuh"

using namespace kc;

namespace kc {
cudaError_t setup_kernels() {
    cudaError_t e = setup_digest_kernels();
    if (e != cudaSuccess) return e;
    if ((e = setup_dedup_kernels()) != cudaSuccess) return e;
    if ((e = setup_compare_kernels()) != cudaSuccess) return e;
    return setup_batch_kernels();
}

static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace kc

namespace {

constexpr uint32_t CENSUS_UNIT = 64 * 1024;
constexpr size_t TABLE_CACHE = 64;

enum TableKind : uint32_t { TK_PAGES = 1, TK_UNITS = 2, TK_TARGETS = 3, TK_PAIRS = 4, TK_BATCH = 5 };

// Pinned host + device buffer pair holding one table set; recycled through
// the context's free list instead of being freed (a cudaFree would wait for
// the whole device).  `used` is recorded after every call that reads it.
struct TableBuf {
    void *d = nullptr;
    void *h = nullptr;
    size_t cap = 0;
    cudaEvent_t used = nullptr;
};

enum TablePart { TP_REGIONS = 0, TP_PAGEFIRST, TP_RANGES, TP_PAIRS, TP_JOBS, TP_WORK, TP_LEFT, TP_COUNT };

// A device-resident table set for one descriptor list.
struct Tables {
    std::vector<uint8_t> key;
    TableBuf buf;
    const void *part[TP_COUNT] = {};   // device address of each uploaded part
    int n = 0;
    uint64_t units = 0;         // pages, census units or comparison tiles
    uint64_t items = 0;         // batched form: work items
    int nranges = 0;            // batched form: ranges
    bool any_lost = false;
    bool fused = false;         // batched form: has fused (digest + compare) ranges
    bool pinned = false;        // read by a captured graph: never recycled
    std::vector<int> buf_status;
    CensusArgs ca{};
    CmpGroups groups{};         // comparison: pairs grouped by dtype
    const Region *regions() const { return static_cast<const Region *>(part[TP_REGIONS]); }
    const uint64_t *page_first() const { return static_cast<const uint64_t *>(part[TP_PAGEFIRST]); }
    const Range *ranges() const { return static_cast<const Range *>(part[TP_RANGES]); }
    const CmpPair *pairs() const { return static_cast<const CmpPair *>(part[TP_PAIRS]); }
    const BatchJob *jobs() const { return static_cast<const BatchJob *>(part[TP_JOBS]); }
    const BatchRange *work() const { return static_cast<const BatchRange *>(part[TP_WORK]); }
    uint32_t *left() const { return static_cast<uint32_t *>(const_cast<void *>(part[TP_LEFT])); }
};

using HostParts = std::vector<uint8_t>[TP_COUNT];

template <class T>
void put(std::vector<uint8_t> &dst, const std::vector<T> &v) {
    dst.resize(v.size() * sizeof(T));
    if (!v.empty()) memcpy(dst.data(), v.data(), dst.size());
}

}  // namespace

struct kc_ctx {
    int device = 0;
    int sms = 0;
    size_t smem_per_sm = 0;
    std::string err;
    std::vector<int> buf_status;
    uint64_t *d_misc = nullptr;   // [0] status word (u32), [1] task counter (u32)
    void *d_scratch = nullptr;
    size_t scratch_cap = 0;
    std::list<Tables> tables;     // most recently used first
    std::vector<TableBuf> free_bufs;
    DigestShape forced{0, 0, 0, 0, 0};
    cudaEvent_t trace_start = nullptr;   // caller-owned, recorded around main kernels
    cudaEvent_t trace_stop = nullptr;
    uint32_t stall_census_spins = 0;     // test hook: see kc_debug_stall_census
};

namespace {

struct DevGuard {
    int prev = -1;
    bool switched = false;
    explicit DevGuard(int d) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) switched = cudaSetDevice(d) == cudaSuccess;
    }
    ~DevGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

kc_status fail(kc_ctx *c, kc_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

kc_status cuda_fail(kc_ctx *c, cudaError_t e, const char *what) {
    cudaGetLastError();   // clear a sticky launch error from the thread state
    return fail(c, KC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define KC_CHECK(ctx, call, what)                                   \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, (what)); \
    } while (0)

bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

bool pow2_page(uint32_t s) { return s >= 4096 && s <= (2u << 20) && (s & (s - 1)) == 0; }

uint32_t log2u(uint32_t v) {
    uint32_t r = 0;
    while ((1u << r) < v) ++r;
    return r;
}

void key_add(std::vector<uint8_t> &k, const void *p, size_t n) {
    const uint8_t *b = static_cast<const uint8_t *>(p);
    k.insert(k.end(), b, b + n);
}

// Check a region list and fill `regions` (first = unit offsets at `unit`
// bytes; unit 0 = no units).
kc_status check_regions(kc_ctx *c, const kc_buf *b, int n, uint32_t unit, std::vector<Region> &regions,
                        uint64_t *nunits, std::vector<int> &st, bool *any_lost) {
    if (n < 1 || !b) return fail(c, KC_EINVAL, "need at least one region (n=%d)", n);
    regions.resize(n);
    st.assign(n, KC_OK);
    uint64_t total = 0;
    *any_lost = false;
    for (int i = 0; i < n; ++i) {
        if (b[i].bytes == 0) return fail(c, KC_EINVAL, "region %d is empty", i);
        if (b[i].base_va & 15)
            return fail(c, KC_EINVAL, "region %d base 0x%llx is not 16-byte aligned", i, (unsigned long long)b[i].base_va);
        if (b[i].dtype < KC_U8 || b[i].dtype > KC_RAW) return fail(c, KC_EINVAL, "region %d has dtype %d", i, b[i].dtype);
        if (b[i].base_va + b[i].bytes < b[i].base_va) return fail(c, KC_EINVAL, "region %d wraps the address space", i);
        Region &r = regions[i];
        r.base = b[i].base_va;
        r.bytes = b[i].bytes;
        r.first = total;
        r.lost = (b[i].flags & KC_BUF_LOST) ? 1u : 0u;
        r.pad = 0;
        if (r.lost) {
            st[i] = KC_EBUF;
            *any_lost = true;
        }
        if (unit) total += (b[i].bytes + unit - 1) / unit;
    }
    if (nunits) *nunits = total;
    return KC_OK;
}

// Sorted census ranges; KC_EOVERLAP if two regions overlap.
kc_status build_ranges(kc_ctx *c, const kc_buf *b, int n, std::vector<Range> &rg) {
    rg.resize(n);
    for (int i = 0; i < n; ++i) rg[i] = Range{b[i].base_va, b[i].base_va + b[i].bytes, i, 0};
    std::sort(rg.begin(), rg.end(), [](const Range &x, const Range &y) { return x.base < y.base; });
    for (int i = 1; i < n; ++i)
        if (rg[i].base < rg[i - 1].end) return fail(c, KC_EOVERLAP, "regions %d and %d overlap", rg[i - 1].id, rg[i].id);
    return KC_OK;
}

void destroy_buf(TableBuf &b) {
    if (b.d) cudaFree(b.d);
    if (b.h) cudaFreeHost(b.h);
    if (b.used) cudaEventDestroy(b.used);
    b = TableBuf{};
}

// Return an entry's buffer to the free list once the GPU is done with it.
void recycle(kc_ctx *c, Tables &t) {
    if (t.buf.used) cudaEventSynchronize(t.buf.used);
    c->free_bufs.push_back(t.buf);
    t.buf = TableBuf{};
}

kc_status acquire_buf(kc_ctx *c, size_t bytes, TableBuf *out) {
    size_t best = (size_t)-1;
    for (size_t i = 0; i < c->free_bufs.size(); ++i)
        if (c->free_bufs[i].cap >= bytes && (best == (size_t)-1 || c->free_bufs[i].cap < c->free_bufs[best].cap))
            best = i;
    if (best != (size_t)-1) {
        *out = c->free_bufs[best];
        c->free_bufs.erase(c->free_bufs.begin() + best);
        return KC_OK;
    }
    TableBuf b;
    b.cap = 64 * 1024;
    while (b.cap < bytes) b.cap *= 2;
    if (cudaHostAlloc(&b.h, b.cap, cudaHostAllocDefault) != cudaSuccess || cudaMalloc(&b.d, b.cap) != cudaSuccess ||
        cudaEventCreateWithFlags(&b.used, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        destroy_buf(b);
        return fail(c, KC_ENOMEM, "table buffer allocation of %zu bytes failed", bytes);
    }
    *out = b;
    return KC_OK;
}

// Find the tables for `key`, or build them with `fill` (which fills the host
// parts and the derived fields) and upload them on `st`.
template <class Fill>
kc_status tables_for(kc_ctx *c, std::vector<uint8_t> &&key, cudaStream_t st, Fill fill, Tables **out) {
    for (auto it = c->tables.begin(); it != c->tables.end(); ++it) {
        if (it->key == key) {
            c->tables.splice(c->tables.begin(), c->tables, it);
            *out = &c->tables.front();
            c->buf_status = c->tables.front().buf_status;
            return KC_OK;
        }
    }
    Tables t;
    t.key = std::move(key);
    HostParts parts;
    kc_status s = fill(t, parts);
    if (s != KC_OK) return s;
    if (capturing(st))
        return fail(c, KC_ENOMEM, "region tables must be built before a stream capture: make one uncaptured call "
                                  "with the same descriptors first");
    size_t off[TP_COUNT], total = 0;
    for (int i = 0; i < TP_COUNT; ++i) {
        off[i] = total;
        total += (parts[i].size() + 255) & ~size_t(255);
    }
    if (total == 0) total = 256;
    if (c->tables.size() >= TABLE_CACHE) {
        for (auto it = c->tables.rbegin(); it != c->tables.rend(); ++it) {
            if (!it->pinned) {
                recycle(c, *it);
                c->tables.erase(std::next(it).base());
                break;
            }
        }
    }
    if ((s = acquire_buf(c, total, &t.buf)) != KC_OK) return s;
    char *h = static_cast<char *>(t.buf.h), *d = static_cast<char *>(t.buf.d);
    for (int i = 0; i < TP_COUNT; ++i) {
        if (!parts[i].empty()) memcpy(h + off[i], parts[i].data(), parts[i].size());
        t.part[i] = parts[i].empty() ? nullptr : d + off[i];
    }
    t.ca.ranges = t.ranges();
    cudaError_t e = cudaMemcpyAsync(t.buf.d, t.buf.h, total, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        c->free_bufs.push_back(t.buf);
        return cuda_fail(c, e, "table upload");
    }
    c->tables.push_front(std::move(t));
    *out = &c->tables.front();
    c->buf_status = c->tables.front().buf_status;
    return KC_OK;
}

// After the kernels that read `t` are enqueued: remember when it is free.
void touch(kc_ctx *c, Tables *t, cudaStream_t st) {
    if (capturing(st)) t->pinned = true;
    else cudaEventRecord(t->buf.used, st);
    (void)c;
}

std::vector<uint8_t> region_key(TableKind kind, const kc_buf *b, int n, uint64_t a, uint64_t bb, uint64_t cc) {
    std::vector<uint8_t> k;
    k.reserve(40 + (n > 0 ? (size_t)n * sizeof(kc_buf) : 0));
    uint64_t hdr[5] = {kind, (uint64_t)(int64_t)n, a, bb, cc};
    key_add(k, hdr, sizeof hdr);
    if (b && n > 0) key_add(k, b, (size_t)n * sizeof(kc_buf));
    return k;
}

// Page tables: regions with page offsets at `page`, page_first, and (census)
// the sorted ranges and census parameters for the window.
kc_status page_tables(kc_ctx *c, const kc_buf *b, int n, uint32_t page, bool census, uint64_t wlo, uint64_t whi,
                      cudaStream_t st, Tables **out) {
    if (n < 1 || !b) return fail(c, KC_EINVAL, "need at least one region (n=%d)", n);
    auto key = region_key(census ? TK_UNITS : TK_PAGES, b, n, page, census ? wlo : 0, census ? whi : 0);
    return tables_for(c, std::move(key), st,
                      [&](Tables &t, HostParts &parts) -> kc_status {
                          std::vector<Region> regions;
                          kc_status s = check_regions(c, b, n, page, regions, &t.units, t.buf_status, &t.any_lost);
                          if (s != KC_OK) return s;
                          std::vector<uint64_t> pf(n + 1);
                          for (int i = 0; i < n; ++i) pf[i] = regions[i].first;
                          pf[n] = t.units;
                          put(parts[TP_REGIONS], regions);
                          put(parts[TP_PAGEFIRST], pf);
                          if (census) {
                              std::vector<Range> rg;
                              if ((s = build_ranges(c, b, n, rg)) != KC_OK) return s;
                              t.ca = census_args(rg.data(), (int)rg.size(), wlo, whi);
                              put(parts[TP_RANGES], rg);
                          }
                          t.n = n;
                          return KC_OK;
                      },
                      out);
}

// Device scratch of at least `bytes`, grown outside captures only.
kc_status scratch(kc_ctx *c, size_t bytes, cudaStream_t st, void **out) {
    if (bytes > c->scratch_cap) {
        if (capturing(st)) return fail(c, KC_ENOMEM, "scratch must grow inside a stream capture");
        if (c->d_scratch) KC_CHECK(c, cudaFree(c->d_scratch), "scratch release");
        c->d_scratch = nullptr;
        c->scratch_cap = 0;
        size_t cap = std::max<size_t>(bytes + bytes / 4, 1 << 20);
        cudaError_t e = cudaMalloc(&c->d_scratch, cap);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, KC_ENOMEM, "scratch allocation of %zu bytes failed", cap);
        }
        c->scratch_cap = cap;
    }
    *out = c->d_scratch;
    return KC_OK;
}

struct Trace {
    kc_ctx *c;
    cudaStream_t st;
    unsigned flags;
    Trace(kc_ctx *c_, cudaStream_t s) : c(c_), st(s) {
        // inside a capture the records become event nodes of the graph
        flags = capturing(st) ? cudaEventRecordExternal : cudaEventRecordDefault;
        if (c->trace_start) cudaEventRecordWithFlags(c->trace_start, st, flags);
    }
    ~Trace() {
        if (c->trace_stop) cudaEventRecordWithFlags(c->trace_stop, st, flags);
    }
};

uint32_t *status_word(kc_ctx *c) { return reinterpret_cast<uint32_t *>(&c->d_misc[0]); }
uint32_t *task_counter(kc_ctx *c) { return reinterpret_cast<uint32_t *>(&c->d_misc[1]); }

// Shape of the batched kernel (k_batch.cu), whose warps each stream their
// own pages through a per-warp ring.  XXH64 is a serial chain per lane and
// every warp owns 8 pages at a time, so a page started late finishes late:
// keep every item resident at once when that fits (up to 24 warps per SM),
// in CTAs of 2 warps, then give each warp the first ring in the preference
// list that fits its share of the SM's shared memory.
// Shape of the batched kernel: the forced shape, or enough warps per SM for
// the tasks and the first ring that fits.  A launch with fused items (got
// and want chunks in every stage) needs twice the ring; a shape that does
// not fit a CTA's shared memory loses stages, then halves its chunk (down
// to 256 bytes), so every forced shape can be launched.
DigestShape pick_batch_shape(const kc_ctx *c, uint32_t page, uint64_t npages, bool fused) {
    const size_t smem_sm = c->smem_per_sm ? c->smem_per_sm : 228 * 1024;
    const size_t smem_cta = 227 * 1024;
    DigestShape s = c->forced;
    if (s.lanes == 0) s.lanes = 1;
    const uint64_t ppw = 8ull * (uint64_t)s.lanes;
    const uint64_t tasks = (npages + ppw - 1) / ppw;
    if (s.warps == 0) {
        s.warps = 2;
        uint64_t per_sm = (tasks + c->sms - 1) / c->sms;
        if (per_sm < 1) per_sm = 1;
        if (per_sm > 24) per_sm = 24;
        const uint64_t ctas = (per_sm + s.warps - 1) / s.warps;
        const size_t per_cta = smem_sm / ctas - 1024 - 256;
        static const int pref[][2] = {{2048, 4}, {2048, 3}, {1024, 2}, {1024, 4}, {1024, 3}, {512, 4},
                                      {512, 3},  {512, 2},  {256, 4},  {256, 3},  {256, 2}};
        s.chunk = 256;
        s.stages = 2;
        for (auto &pc : pref) {
            if ((uint32_t)pc[0] > page) continue;
            DigestShape t = s;
            t.chunk = pc[0];
            t.stages = pc[1];
            if (batch_smem_bytes(t, fused) <= per_cta) {
                s = t;
                break;
            }
        }
    }
    if ((uint32_t)s.chunk > page) s.chunk = (int)page;
    while (batch_smem_bytes(s, fused) > smem_cta) {
        if (s.stages > 2) --s.stages;
        else if (s.chunk > 256) s.chunk /= 2;
        else break;
    }
    const size_t cta_smem = batch_smem_bytes(s, fused);
    uint64_t ctas_per_sm = smem_sm / (cta_smem + 1024);
    const uint64_t by_threads = 2048 / (32 * s.warps);
    if (ctas_per_sm > by_threads) ctas_per_sm = by_threads;
    if (ctas_per_sm > 32) ctas_per_sm = 32;
    if (ctas_per_sm < 1) ctas_per_sm = 1;
    uint64_t grid = (tasks + s.warps - 1) / s.warps;
    if (grid > ctas_per_sm * c->sms) grid = ctas_per_sm * c->sms;
    s.ctas = (int)(grid ? grid : 1);
    return s;
}

// Shape of the digest kernel (k_digest.cu): hash warps per CTA (`warps`,
// plus as many loader warps), ring stages and chunk bytes per page and
// stage, grid.  Every task (8 pages) runs on one hash warp from start to
// end, and XXH64's chains are serial, so a task started late finishes late:
// give every SM one CTA with enough hash warps for its share of the tasks,
// up to 8 (two per SM
// sub-partition: more only queue behind each other on the same issue
// slots); larger snapshots reuse the warps through the ticket counter.
// Then the first ring in the preference list that fits the SM's shared
// memory.  Measured on the llama-shaped snapshot (6,327 pages of 64 KiB, 6
// hash warps per SM): 2 KiB x 2 stages 91.6 us, 1 KiB x 3 93.2 us, 1 KiB x 4
// 96.4 us, 512 B x 4 115 us; on the 30 GiB MoE pool (2 MiB pages, 8 hash
// warps): 1 KiB x 3 5.09 ms (2 KiB stages do not fit 8 warps).
DigestShape pick_digest_shape(const kc_ctx *c, uint32_t page, uint64_t npages) {
    const size_t smem_sm = c->smem_per_sm ? c->smem_per_sm : 228 * 1024;
    DigestShape s = c->forced;
    s.lanes = 1;
    const uint64_t tasks = (npages + 7) / 8;
    const uint64_t sms = (uint64_t)c->sms;
    if (s.warps == 0) {
        uint64_t per_sm = (tasks + sms - 1) / sms;
        if (per_sm < 1) per_sm = 1;
        if (per_sm > 8) per_sm = 8;
        s.warps = (int)per_sm;
        // few hash warps per SM: each one's chains run fastest, so it needs
        // more bytes in flight; deeper rings first while they fit
        static const int pref[][2] = {{2048, 6}, {2048, 4}, {2048, 3}, {2048, 2}, {1024, 3}, {1024, 4},
                                      {512, 4},  {1024, 2}, {512, 3},  {512, 2},  {256, 4},  {256, 3}, {256, 2}};
        s.chunk = 256;
        s.stages = 2;
        for (auto &pc : pref) {
            if ((uint32_t)pc[0] > page) continue;
            DigestShape t{s.warps, pc[1], pc[0], 1, 1};
            if (digest_smem_bytes(t) + 1024 <= smem_sm) {
                s.chunk = pc[0];
                s.stages = pc[1];
                break;
            }
        }
    }
    if (s.warps > digest_max_hash_warps()) s.warps = digest_max_hash_warps();
    if ((uint32_t)s.chunk > page) s.chunk = (int)page;
    uint64_t per_sm = smem_sm / (digest_smem_bytes(s) + 1024);
    const uint64_t by_threads = 2048 / (64 * s.warps);
    if (per_sm > by_threads) per_sm = by_threads;
    if (per_sm < 1) per_sm = 1;
    uint64_t grid = (tasks + s.warps - 1) / s.warps;
    if (grid < sms && tasks >= sms) grid = sms;   // every SM works, some hash warps idle
    if (grid > per_sm * sms) grid = per_sm * sms;
    s.ctas = (int)(grid ? grid : 1);
    return s;
}

Pages make_pages(const Region *d_regions, int n, uint64_t npages, uint32_t unit) {
    Pages p;
    p.regions = d_regions;
    p.nregions = n;
    p.npages = npages;
    p.page = unit;
    p.log2page = log2u(unit);
    return p;
}

// Census over `units`: ordered write of the counted hits.
kc_status census_tail(kc_ctx *c, const Pages &units, const CensusArgs &ca, uint32_t *unit_hits, uint64_t *unit_off,
                      kc_hit *d_hits, uint64_t cap, cudaStream_t st) {
    if (!d_hits) return KC_OK;
    KC_CHECK(c, launch_scan_u32(unit_hits, unit_off, units.npages, nullptr, st), "census scan");
    KC_CHECK(c, launch_census_write(units, ca, unit_hits, unit_off, d_hits, cap, status_word(c), c->sms, st),
             "census write");
    return KC_OK;
}

kc_status lost_status(kc_ctx *c, const Tables *t) {
    return t->any_lost ? fail(c, KC_EBUF, "one or more regions were marked lost") : KC_OK;
}

}  // namespace

extern "C" {

KC_API int kc_version(void) { return KC_VERSION; }

KC_API uint64_t kc_launch_count(void) { return launches_so_far(); }

KC_API const char *kc_status_name(int s) {
    switch (s) {
    case KC_OK: return "KC_OK";
    case KC_EINVAL: return "KC_EINVAL";
    case KC_EOVERLAP: return "KC_EOVERLAP";
    case KC_ENOMEM: return "KC_ENOMEM";
    case KC_ETRUNC: return "KC_ETRUNC";
    case KC_ECUDA: return "KC_ECUDA";
    case KC_ETIMEOUT: return "KC_ETIMEOUT";
    case KC_EBUF: return "KC_EBUF";
    }
    return "KC_UNKNOWN";
}

KC_API const char *kc_last_error(const kc_ctx *c) { return c ? c->err.c_str() : "null context"; }

KC_API int kc_buf_status(const kc_ctx *c, int i) {
    if (!c || i < 0 || i >= (int)c->buf_status.size()) return -1;
    return c->buf_status[i];
}

KC_API uint64_t kc_page_count(const kc_buf *b, int n, uint32_t page_bytes) {
    if (!b || n < 1 || page_bytes == 0) return 0;
    uint64_t t = 0;
    for (int i = 0; i < n; ++i) t += (b[i].bytes + page_bytes - 1) / page_bytes;
    return t;
}

KC_API kc_status kc_create(kc_ctx **out, int device) {
    if (!out) return KC_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return KC_EINVAL;
    }
    DevGuard g(device);
    kc_ctx *c = new kc_ctx();
    c->device = device;
    int sms = 0, smem = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess ||
        setup_kernels() != cudaSuccess || cudaMalloc(&c->d_misc, 512) != cudaSuccess ||
        cudaMemset(c->d_misc, 0, 512) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return KC_ECUDA;
    }
    c->sms = sms;
    c->smem_per_sm = (size_t)smem;
    *out = c;
    return KC_OK;
}

KC_API void kc_destroy(kc_ctx *c) {
    if (!c) return;
    DevGuard g(c->device);
    cudaDeviceSynchronize();
    for (auto &t : c->tables) destroy_buf(t.buf);
    for (auto &b : c->free_bufs) destroy_buf(b);
    if (c->d_scratch) cudaFree(c->d_scratch);
    if (c->d_misc) cudaFree(c->d_misc);
    delete c;
}

KC_API kc_status kc_sync(kc_ctx *c, void *stream) {
    if (!c) return KC_EINVAL;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    KC_CHECK(c, cudaStreamSynchronize(st), "stream synchronize");
    uint32_t w = 0;
    KC_CHECK(c, cudaMemcpy(&w, c->d_misc, 4, cudaMemcpyDeviceToHost), "status read");
    KC_CHECK(c, cudaMemset(c->d_misc, 0, 4), "status clear");
    if (w & ST_TIMEOUT) return fail(c, KC_ETIMEOUT, "a bounded device wait timed out");
    if (w & ST_INTERNAL) return fail(c, KC_ECUDA, "internal consistency check failed on the device");
    if (w & ST_BADROW) return fail(c, KC_EINVAL, "a page-table row pointed outside its region or the arena");
    if (w & ST_TRUNC) return fail(c, KC_ETRUNC, "an output capacity was exceeded; true counts were written");
    return KC_OK;
}

KC_API kc_status kc_set_digest_shape(kc_ctx *c, int warps, int stages, int chunk, int lanes) {
    if (!c) return KC_EINVAL;
    if (warps == 0 && stages == 0 && chunk == 0 && lanes == 0) {
        c->forced = DigestShape{0, 0, 0, 0, 0};
        return KC_OK;
    }
    if (warps < 1 || warps > 16 || stages < 2 || stages > 8 || chunk < 256 || chunk > 8192 || (chunk % 128) ||
        (lanes != 0 && lanes != 1))
        return fail(c, KC_EINVAL, "digest shape out of range (warps %d, stages %d, chunk %d, lanes %d)", warps, stages,
                    chunk, lanes);
    DigestShape s{warps, stages, chunk, 1, 1};
    if (digest_smem_bytes(s) > 227 * 1024) return fail(c, KC_EINVAL, "digest shape needs too much shared memory");
    c->forced = DigestShape{warps, stages, chunk, 0, 1};
    return KC_OK;
}

KC_API kc_status kc_debug_stall_census(kc_ctx *c, uint32_t spin_limit) {
    if (!c || spin_limit == 0) return KC_EINVAL;
    c->stall_census_spins = spin_limit;
    return KC_OK;
}

KC_API kc_status kc_set_trace_events(kc_ctx *c, void *start, void *stop) {
    if (!c) return KC_EINVAL;
    if ((start == nullptr) != (stop == nullptr)) return fail(c, KC_EINVAL, "give both trace events or neither");
    c->trace_start = static_cast<cudaEvent_t>(start);
    c->trace_stop = static_cast<cudaEvent_t>(stop);
    return KC_OK;
}

KC_API kc_status kc_get_digest_shape(kc_ctx *c, uint32_t page_bytes, uint64_t npages, int *warps, int *stages,
                                     int *chunk, int *ctas, int *lanes) {
    if (!c || !pow2_page(page_bytes)) return KC_EINVAL;
    DigestShape s = pick_digest_shape(c, page_bytes, npages);
    if (warps) *warps = s.warps;
    if (stages) *stages = s.stages;
    if (chunk) *chunk = s.chunk;
    if (ctas) *ctas = s.ctas;
    if (lanes) *lanes = s.lanes;
    return KC_OK;
}

// Shared body of kc_digest and kc_scan.
static kc_status digest_impl(kc_ctx *c, const kc_buf *allocs, int n, uint32_t page_bytes, uint64_t *d_hash,
                             uint8_t *d_zero, uint64_t *d_page_first, bool census, uint64_t win_lo, uint64_t win_hi,
                             kc_hit *d_hits, uint64_t cap, uint64_t *d_counts, void *stream) {
    if (!c) return KC_EINVAL;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!pow2_page(page_bytes)) return fail(c, KC_EINVAL, "page size %u is not a power of two in [4 KiB, 2 MiB]", page_bytes);
    if (!d_hash || !d_zero) return fail(c, KC_EINVAL, "null digest output");
    if (census && !d_counts) return fail(c, KC_EINVAL, "null census counts");
    if (census && cap && !d_hits) return fail(c, KC_EINVAL, "null census hit buffer with cap %llu", (unsigned long long)cap);
    Tables *t = nullptr;
    kc_status s = page_tables(c, allocs, n, page_bytes, census, win_lo, win_hi, st, &t);
    if (s != KC_OK) return s;
    const uint64_t P = t->units;
    const Pages pg = make_pages(t->regions(), n, P, page_bytes);
    const DigestShape shape = pick_digest_shape(c, page_bytes, P);
    uint32_t *page_hits = nullptr;
    unsigned long long *tail = nullptr;
    DigestAux aux;
    uint32_t spin_limit = 0;
    if (census) {
        // page_hits[P] | census tail: ticket + one word per chunk
        const uint64_t nwords = census_tail_words(P, c->sms);
        const uint64_t hb = (P * 4 + 255) & ~255ull, tb = (nwords * 8 + 255) & ~255ull;
        void *scr = nullptr;
        if ((s = scratch(c, hb + tb, st, &scr)) != KC_OK) return s;
        page_hits = static_cast<uint32_t *>(scr);
        tail = reinterpret_cast<unsigned long long *>(static_cast<char *>(scr) + hb);
        aux.zero_words = tail;
        aux.nzero = nwords;
        if (c->stall_census_spins) {   // one-shot test hook: chunk 0 is never taken
            aux.first_ticket = 1;
            spin_limit = c->stall_census_spins;
            c->stall_census_spins = 0;
        }
        aux.counts = d_counts;
    }
    if (d_page_first) {
        aux.pf_src = t->page_first();
        aux.pf_dst = d_page_first;
        aux.npf = (uint64_t)n + 1;
    }
    // The task counter is zero between calls (zeroed with the context; each
    // call that counts tasks on it sets it back to zero behind its kernel):
    // here the census tail does, else a memset after the digest.
    {
        Trace tr(c, st);
        KC_CHECK(c, launch_digest(pg, census ? &t->ca : nullptr, d_hash, d_zero, page_hits, task_counter(c),
                                  status_word(c), shape, aux, st),
                 "digest launch");
    }
    if (census) {
        const cudaError_t e = launch_census_tail(pg, t->ca, page_hits, tail, d_hits, cap, d_counts, status_word(c),
                                                 task_counter(c), c->sms, spin_limit, st);
        if (e != cudaSuccess) {
            cudaMemsetAsync(task_counter(c), 0, 4, st);
            return cuda_fail(c, e, "census tail");
        }
    } else {
        KC_CHECK(c, cudaMemsetAsync(task_counter(c), 0, 4, st), "task counter clear");
    }
    touch(c, t, st);
    return lost_status(c, t);
}

KC_API kc_status kc_digest(kc_ctx *c, const kc_buf *allocs, int n, uint32_t page_bytes, uint64_t *d_hash,
                           uint8_t *d_zero, uint64_t *d_page_first, void *stream) {
    return digest_impl(c, allocs, n, page_bytes, d_hash, d_zero, d_page_first, false, 0, 0, nullptr, 0, nullptr,
                       stream);
}

KC_API kc_status kc_scan(kc_ctx *c, const kc_buf *allocs, int n, uint32_t page_bytes, uint64_t *d_hash,
                         uint8_t *d_zero, uint64_t *d_page_first, uint64_t win_lo, uint64_t win_hi, kc_hit *d_hits,
                         uint64_t cap, uint64_t *d_counts, void *stream) {
    return digest_impl(c, allocs, n, page_bytes, d_hash, d_zero, d_page_first, true, win_lo, win_hi, d_hits, cap,
                       d_counts, stream);
}

KC_API kc_status kc_census(kc_ctx *c, const kc_buf *allocs, int n, uint64_t win_lo, uint64_t win_hi, kc_hit *d_hits,
                           uint64_t cap, uint64_t *d_counts, void *stream) {
    if (!c) return KC_EINVAL;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!d_counts) return fail(c, KC_EINVAL, "null census counts");
    if (cap && !d_hits) return fail(c, KC_EINVAL, "null census hit buffer with cap %llu", (unsigned long long)cap);
    Tables *t = nullptr;
    kc_status s = page_tables(c, allocs, n, CENSUS_UNIT, true, win_lo, win_hi, st, &t);
    if (s != KC_OK) return s;
    const uint64_t U = t->units;
    const Pages units = make_pages(t->regions(), n, U, CENSUS_UNIT);
    void *scr = nullptr;
    if ((s = scratch(c, U * 4 + 256 + U * 8, st, &scr)) != KC_OK) return s;
    uint32_t *unit_hits = static_cast<uint32_t *>(scr);
    uint64_t *unit_off = reinterpret_cast<uint64_t *>(static_cast<char *>(scr) + ((U * 4 + 255) & ~255ull));
    KC_CHECK(c, cudaMemsetAsync(d_counts, 0, 16, st), "census counts clear");
    {
        Trace tr(c, st);
        KC_CHECK(c, launch_census_count(units, t->ca, unit_hits, d_counts, c->sms, st), "census count");
    }
    if ((s = census_tail(c, units, t->ca, unit_hits, unit_off, cap ? d_hits : nullptr, cap, st)) != KC_OK) return s;
    touch(c, t, st);
    return lost_status(c, t);
}

KC_API kc_status kc_dedup(kc_ctx *c, const kc_buf *allocs, int n, uint32_t page_bytes, const uint64_t *d_hash,
                          const uint8_t *d_zero, kc_page *d_table, uint8_t *d_arena, uint64_t arena_cap,
                          uint64_t *d_n_blobs, void *stream) {
    if (!c) return KC_EINVAL;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!pow2_page(page_bytes)) return fail(c, KC_EINVAL, "page size %u is not a power of two in [4 KiB, 2 MiB]", page_bytes);
    if (!d_hash || !d_zero || !d_table) return fail(c, KC_EINVAL, "null dedup input or table");
    if (d_arena && (reinterpret_cast<uintptr_t>(d_arena) & 15)) return fail(c, KC_EINVAL, "arena is not 16-byte aligned");
    Tables *t = nullptr;
    kc_status s = page_tables(c, allocs, n, page_bytes, false, 0, 0, st, &t);
    if (s != KC_OK) return s;
    const uint64_t P = t->units;
    if (P >= 0xFFFFFFF0ull) return fail(c, KC_EINVAL, "too many pages (%llu) for 32-bit page ids", (unsigned long long)P);
    const Pages pg = make_pages(t->regions(), n, P, page_bytes);
    void *scr = nullptr;
    if ((s = scratch(c, dedup_scratch_bytes(P, nullptr), st, &scr)) != KC_OK) return s;
    DedupScratch ds;
    dedup_scratch_carve(scr, P, &ds);
    {
        Trace tr(c, st);
        KC_CHECK(c, run_dedup(pg, d_hash, d_zero, d_table, d_arena, arena_cap, d_n_blobs, ds, status_word(c), c->sms, st),
                 "dedup");
    }
    touch(c, t, st);
    return lost_status(c, t);
}

KC_API kc_status kc_restore(kc_ctx *c, const kc_buf *allocs, int n, uint32_t page_bytes, const kc_page *d_table,
                            uint64_t n_pages, const uint8_t *d_arena, uint64_t arena_bytes, void *stream) {
    if (!c) return KC_EINVAL;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!pow2_page(page_bytes)) return fail(c, KC_EINVAL, "page size %u is not a power of two in [4 KiB, 2 MiB]", page_bytes);
    if (n_pages && !d_table) return fail(c, KC_EINVAL, "null page table");
    if (arena_bytes && !d_arena) return fail(c, KC_EINVAL, "null arena with %llu bytes", (unsigned long long)arena_bytes);
    if (d_arena && (reinterpret_cast<uintptr_t>(d_arena) & 15)) return fail(c, KC_EINVAL, "arena is not 16-byte aligned");
    Tables *t = nullptr;
    kc_status s = page_tables(c, allocs, n, page_bytes, false, 0, 0, st, &t);
    if (s != KC_OK) return s;
    const Pages pg = make_pages(t->regions(), n, n_pages, page_bytes);
    {
        Trace tr(c, st);
        KC_CHECK(c, launch_restore(pg, d_table, n_pages, d_arena, arena_bytes, status_word(c), c->sms, st), "restore");
    }
    touch(c, t, st);
    return lost_status(c, t);
}

KC_API kc_status kc_compare(kc_ctx *c, const kc_buf *got, const kc_buf *want, int npairs, double atol, double rtol,
                            kc_cmp_result *d_out, void *stream) {
    if (!c) return KC_EINVAL;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (npairs < 1 || !got || !want || !d_out) return fail(c, KC_EINVAL, "need at least one pair and an output");
    if (!(atol >= 0.0) || !(rtol >= 0.0)) return fail(c, KC_EINVAL, "tolerances must be >= 0 and not NaN");
    auto key = region_key(TK_PAIRS, got, npairs, 0, 0, 0);
    key_add(key, want, (size_t)npairs * sizeof(kc_buf));
    Tables *t = nullptr;
    kc_status s = tables_for(
        c, std::move(key), st,
        [&](Tables &tb, HostParts &parts) -> kc_status {
            std::vector<CmpPair> pairs(npairs);
            tb.buf_status.assign(npairs, KC_OK);
            uint64_t tiles = 0;
            for (int k = 0; k < npairs; ++k) {
                const int dt = got[k].dtype;
                if (dt < KC_U8 || dt > KC_RAW) return fail(c, KC_EINVAL, "pair %d has dtype %d", k, dt);
                const uint64_t es = (dt == KC_F32 || dt == KC_I32) ? 4 : (dt == KC_F16 || dt == KC_BF16) ? 2 : 1;
                if (got[k].bytes != want[k].bytes) return fail(c, KC_EINVAL, "pair %d: sizes differ", k);
                if (got[k].bytes % es) return fail(c, KC_EINVAL, "pair %d: size is not a multiple of the element size", k);
                if ((got[k].base_va | want[k].base_va) & 15)
                    return fail(c, KC_EINVAL, "pair %d: buffers not 16-byte aligned", k);
                CmpPair &p = pairs[k];
                p.got = got[k].base_va;
                p.want = want[k].base_va;
                p.nelem = got[k].bytes / es;
                p.tile_first = tiles;
                p.dtype = dt == KC_RAW ? KC_U8 : dt;
                p.lost = ((got[k].flags | want[k].flags) & KC_BUF_LOST) ? 1 : 0;
                p.out_index = (uint32_t)k;
                p.pad = 0;
                if (p.lost) {
                    tb.any_lost = true;
                    tb.buf_status[k] = KC_EBUF;
                }
                tiles += (got[k].bytes + CMP_TILE_BYTES - 1) / CMP_TILE_BYTES;
            }
            // group by dtype (stable), vectors numbered within each group
            std::stable_sort(pairs.begin(), pairs.end(),
                             [](const CmpPair &a, const CmpPair &b) { return a.dtype < b.dtype; });
            CmpGroups &gr = tb.groups;
            gr = CmpGroups{};
            int at = 0;
            for (int d = 0; d < 6; ++d) {
                gr.gfirst[d] = at;
                uint64_t v = 0;
                while (at < npairs && pairs[at].dtype == d) {
                    const uint64_t es = (d == KC_F32 || d == KC_I32) ? 4 : (d == KC_F16 || d == KC_BF16) ? 2 : 1;
                    pairs[at].vec_first = v;
                    v += pairs[at].nelem * es / 16;
                    ++at;
                }
                gr.gvec[d] = v;
            }
            gr.gfirst[6] = at;
            tb.units = tiles;
            tb.n = npairs;
            put(parts[TP_PAIRS], pairs);
            return KC_OK;
        },
        &t);
    if (s != KC_OK) return s;
    void *gates = nullptr;
    if ((s = scratch(c, (size_t)npairs * 8, st, &gates)) != KC_OK) return s;
    {
        Trace tr(c, st);
        KC_CHECK(c, launch_compare(t->pairs(), npairs, t->groups, atol, rtol, d_out, static_cast<uint32_t *>(gates),
                                   c->sms, st),
                 "compare");
    }
    touch(c, t, st);
    return t->any_lost ? fail(c, KC_EBUF, "one or more pairs were marked lost") : KC_OK;
}

KC_API int kc_poll_flags(const uint32_t *flags, int n, int32_t *idx_out) {
    if (!flags || !idx_out || n < 0) return -1;
    int k = 0;
    for (int i = 0; i < n; ++i)
        if (__atomic_load_n(flags + i, __ATOMIC_RELAXED)) idx_out[k++] = i;
    std::atomic_thread_fence(std::memory_order_acquire);
    return k;
}

KC_API kc_status kc_batch_run(kc_ctx *c, const kc_job *jobs, int njobs, uint32_t page_bytes, double atol,
                              double rtol, const kc_work *work, int nwork, void *stream) {
    if (!c) return KC_EINVAL;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!pow2_page(page_bytes)) return fail(c, KC_EINVAL, "page size %u is not a power of two in [4 KiB, 2 MiB]", page_bytes);
    if (njobs < 1 || !jobs) return fail(c, KC_EINVAL, "need at least one job");
    if (nwork < 0 || (nwork > 0 && !work)) return fail(c, KC_EINVAL, "bad work list");
    if (!(atol >= 0.0) || !(rtol >= 0.0)) return fail(c, KC_EINVAL, "tolerances must be >= 0 and not NaN");
    auto key = region_key(TK_BATCH, nullptr, njobs, page_bytes, (uint64_t)nwork, 0);
    key_add(key, jobs, (size_t)njobs * sizeof(kc_job));
    if (nwork > 0) key_add(key, work, (size_t)nwork * sizeof(kc_work));
    Tables *t = nullptr;
    kc_status s = tables_for(
        c, std::move(key), st,
        [&](Tables &tb, HostParts &parts) -> kc_status {
            std::vector<BatchJob> bj(njobs);
            std::vector<uint64_t> pages(njobs), items(njobs);
            tb.buf_status.assign(njobs, KC_OK);
            for (int k = 0; k < njobs; ++k) {
                const kc_job &J = jobs[k];
                const bool dg = (J.flags & KC_JOB_DIGEST) != 0, cm = (J.flags & KC_JOB_COMPARE) != 0;
                if (!dg && !cm) return fail(c, KC_EINVAL, "job %d asks for neither digest nor compare", k);
                if (J.bytes == 0 || (J.got_va & 15)) return fail(c, KC_EINVAL, "job %d: empty or misaligned buffer", k);
                if (dg && (!J.d_hash || !J.d_zero)) return fail(c, KC_EINVAL, "job %d: null digest outputs", k);
                const int dt = J.dtype;
                if (dt < KC_U8 || dt > KC_RAW) return fail(c, KC_EINVAL, "job %d has dtype %d", k, dt);
                const uint64_t es = (dt == KC_F32 || dt == KC_I32) ? 4 : (dt == KC_F16 || dt == KC_BF16) ? 2 : 1;
                if (cm && (!J.d_cmp || (J.want_va & 15) || J.bytes % es))
                    return fail(c, KC_EINVAL, "job %d: bad comparison (output, alignment or element size)", k);
                BatchJob &b = bj[k];
                b.got = J.got_va;
                b.want = J.want_va;
                b.bytes = J.bytes;
                b.nelem = J.bytes / es;
                b.hash = J.d_hash;
                b.zero = J.d_zero;
                b.cmp = J.d_cmp;
                b.done = J.d_done;
                b.cmp_copy = J.d_cmp_copy;
                b.items = 0;
                b.pad = 0;
                b.dtype = dt == KC_RAW ? KC_U8 : dt;
                b.flags = (dg ? BJ_DIGEST : 0u) | (cm ? BJ_COMPARE : 0u) | ((J.flags & KC_BUF_LOST) ? BJ_LOST : 0u) |
                          ((work == nullptr || (J.flags & KC_JOB_INIT)) ? BJ_INIT : 0u);
                if (J.flags & KC_BUF_LOST) {
                    tb.any_lost = true;
                    tb.buf_status[k] = KC_EBUF;
                }
                pages[k] = (J.bytes + page_bytes - 1) / page_bytes;
                items[k] = (J.bytes + KC_BATCH_ITEM_BYTES - 1) / KC_BATCH_ITEM_BYTES;
            }
            std::vector<BatchRange> rg;
            auto add = [&](uint32_t job, uint32_t kind, uint64_t first, uint64_t count) {
                if (count == 0) return;
                BatchRange r{first, count, 0, job, kind};
                rg.push_back(r);
            };
            if (nwork == 0) {
                // largest jobs first; a job's digest range, then its comparison range
                std::vector<int> order(njobs);
                for (int k = 0; k < njobs; ++k) order[k] = k;
                std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return jobs[a].bytes > jobs[b].bytes; });
                for (int k : order) {
                    const uint32_t f = bj[k].flags;
                    if ((f & BJ_DIGEST) && (f & BJ_COMPARE)) {
                        add((uint32_t)k, BR_FUSED, 0, pages[k]);
                    } else {
                        if (f & BJ_DIGEST) add((uint32_t)k, BR_DIGEST, 0, pages[k]);
                        if (f & BJ_COMPARE) add((uint32_t)k, BR_COMPARE, 0, items[k]);
                    }
                }
            } else {
                for (int w = 0; w < nwork; ++w) {
                    const kc_work &W = work[w];
                    if (W.job >= (uint32_t)njobs) return fail(c, KC_EINVAL, "work %d: job %u out of range", w, W.job);
                    const BatchJob &b = bj[W.job];
                    if (W.kind == KC_WORK_DIGEST) {
                        if (!(b.flags & BJ_DIGEST) || W.first + W.count > pages[W.job] || W.first + W.count < W.first)
                            return fail(c, KC_EINVAL, "work %d: digest range outside job %u", w, W.job);
                    } else if (W.kind == KC_WORK_COMPARE) {
                        if (!(b.flags & BJ_COMPARE) || W.first + W.count > items[W.job] || W.first + W.count < W.first)
                            return fail(c, KC_EINVAL, "work %d: comparison range outside job %u", w, W.job);
                    } else if (W.kind == KC_WORK_FUSED) {
                        if (!(b.flags & BJ_DIGEST) || !(b.flags & BJ_COMPARE) || W.first + W.count > pages[W.job] ||
                            W.first + W.count < W.first)
                            return fail(c, KC_EINVAL, "work %d: fused range outside job %u (or not both operations)",
                                        w, W.job);
                    } else {
                        return fail(c, KC_EINVAL, "work %d: kind %u", w, W.kind);
                    }
                    add(W.job,
                        W.kind == KC_WORK_DIGEST ? BR_DIGEST : W.kind == KC_WORK_COMPARE ? BR_COMPARE : BR_FUSED,
                        W.first, W.count);
                }
            }
            uint64_t it = 0;
            std::vector<uint64_t> per_job(njobs, 0);
            for (auto &r : rg) {
                r.item_first = it;
                const uint64_t k = r.kind == BR_COMPARE ? r.count : (r.count + 7) / 8;
                it += k;
                per_job[r.job] += k;
                if (r.kind == BR_FUSED) tb.fused = true;
            }
            for (int k = 0; k < njobs; ++k) {
                if (per_job[k] > 0xFFFFFFFFull) return fail(c, KC_EINVAL, "job %d has more than 2^32 - 1 items", k);
                bj[k].items = (uint32_t)per_job[k];
            }
            tb.items = it;
            tb.nranges = (int)rg.size();
            tb.n = njobs;
            put(parts[TP_JOBS], bj);
            put(parts[TP_WORK], rg);
            put(parts[TP_LEFT], std::vector<uint32_t>(njobs, 0u));
            return KC_OK;
        },
        &t);
    if (s != KC_OK) return s;
    // digest shape: the persistent grid fills the GPU; warps take digest
    // items and comparison items alike
    DigestShape shape = pick_batch_shape(c, page_bytes, t->items * 8, t->fused);
    shape.lanes = 1;
    shape.ctas = (int)std::min<uint64_t>((uint64_t)shape.ctas, std::max<uint64_t>(1, t->items));
    {
        Trace tr(c, st);
        KC_CHECK(c, launch_batch(t->jobs(), njobs, t->left(), t->work(), t->nranges, t->items, page_bytes, shape,
                                 t->fused, atol, rtol, task_counter(c), c->sms, st),
                 "batch launch");
    }
    // back to zero for the next call that counts tasks on it
    KC_CHECK(c, cudaMemsetAsync(task_counter(c), 0, 4, st), "task counter clear");
    touch(c, t, st);
    return t->any_lost ? fail(c, KC_EBUF, "one or more jobs were marked lost") : KC_OK;
}

}  // extern "C"
