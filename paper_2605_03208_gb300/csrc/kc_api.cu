// kc_api.cu -- the C ABI: context, argument validation, region tables,
// scratch management and the launch sequence of every entry point.
//
// Region tables (one 32-byte record per region, plus sorted census ranges
// and page offsets) are built on the host, written into a pinned staging
// slot and copied to the device on the caller's stream, so a call never
// blocks the host.  A ring of staging slots, each guarded by an event, lets
// consecutive calls proceed while earlier copies are still queued.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kc_internal.cuh"

using namespace kc;

namespace kc {
static std::atomic<uint64_t> g_launches{0};
void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace kc

namespace {

constexpr int NSLOT = 8;
constexpr uint32_t CENSUS_UNIT = 64 * 1024;

struct Slot {
    void *h = nullptr;
    void *d = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    bool used = false;
};

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
    Slot slots[NSLOT];
    int next = 0;
    DigestShape forced{0, 0, 0, 0};
    cudaEvent_t trace_start = nullptr;   // caller-owned, recorded around main kernels
    cudaEvent_t trace_stop = nullptr;
};

namespace {

struct DevGuard {
    int prev = -1;
    bool switched = false;
    explicit DevGuard(int d) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) {
            switched = cudaSetDevice(d) == cudaSuccess;
        }
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

#define KC_CHECK(ctx, call, what)                                  \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, (what)); \
    } while (0)

bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

bool pow2_page(uint32_t s) { return s >= 4096 && s <= (2u << 20) && (s & (s - 1)) == 0; }

uint32_t log2u(uint32_t v) {
    uint32_t r = 0;
    while ((1u << r) < v) ++r;
    return r;
}

// Check a region list; fill `regions` (first = unit offsets at `unit` bytes,
// 0 = no units) and the context's per-region status.  Returns KC_OK or the error.
kc_status check_regions(kc_ctx *c, const kc_buf *b, int n, uint32_t unit, std::vector<Region> &regions,
                        uint64_t *nunits, bool *any_lost) {
    if (n < 1 || !b) return fail(c, KC_EINVAL, "need at least one region (n=%d)", n);
    regions.resize(n);
    c->buf_status.assign(n, KC_OK);
    uint64_t total = 0;
    *any_lost = false;
    for (int i = 0; i < n; ++i) {
        if (b[i].bytes == 0) return fail(c, KC_EINVAL, "region %d is empty", i);
        if (b[i].base_va & 15) return fail(c, KC_EINVAL, "region %d base 0x%llx is not 16-byte aligned", i,
                                           (unsigned long long)b[i].base_va);
        if (b[i].dtype < KC_U8 || b[i].dtype > KC_RAW) return fail(c, KC_EINVAL, "region %d has dtype %d", i, b[i].dtype);
        if (b[i].base_va + b[i].bytes < b[i].base_va) return fail(c, KC_EINVAL, "region %d wraps the address space", i);
        Region &r = regions[i];
        r.base = b[i].base_va;
        r.bytes = b[i].bytes;
        r.first = total;
        r.lost = (b[i].flags & KC_BUF_LOST) ? 1u : 0u;
        r.pad = 0;
        if (r.lost) {
            c->buf_status[i] = KC_EBUF;
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
        if (rg[i].base < rg[i - 1].end)
            return fail(c, KC_EOVERLAP, "regions %d and %d overlap", rg[i - 1].id, rg[i].id);
    return KC_OK;
}

// Stage `parts` (host pointer, bytes) into the next slot and copy them to the
// device on `st`; device addresses of the parts are returned in `dptr`.
kc_status stage(kc_ctx *c, cudaStream_t st, std::initializer_list<std::pair<const void *, size_t>> parts,
                std::vector<void *> &dptr, Slot **used) {
    size_t total = 0;
    for (auto &p : parts) total += (p.second + 255) & ~size_t(255);
    Slot &s = c->slots[c->next];
    c->next = (c->next + 1) % NSLOT;
    if (s.used) KC_CHECK(c, cudaEventSynchronize(s.ev), "staging slot wait");
    if (total > s.cap) {
        if (capturing(st)) return fail(c, KC_ENOMEM, "region tables must grow inside a stream capture");
        if (s.h) cudaFreeHost(s.h);
        if (s.d) cudaFree(s.d);
        s.h = s.d = nullptr;
        s.cap = 0;
        size_t cap = std::max<size_t>(total, 64 * 1024);
        KC_CHECK(c, cudaHostAlloc(&s.h, cap, cudaHostAllocDefault), "pinned staging allocation");
        KC_CHECK(c, cudaMalloc(&s.d, cap), "device table allocation");
        s.cap = cap;
    }
    size_t off = 0;
    dptr.clear();
    for (auto &p : parts) {
        if (p.second) memcpy(static_cast<char *>(s.h) + off, p.first, p.second);
        dptr.push_back(static_cast<char *>(s.d) + off);
        off += (p.second + 255) & ~size_t(255);
    }
    if (total) KC_CHECK(c, cudaMemcpyAsync(s.d, s.h, total, cudaMemcpyHostToDevice, st), "table upload");
    *used = &s;
    return KC_OK;
}

kc_status release(kc_ctx *c, Slot *s, cudaStream_t st) {
    KC_CHECK(c, cudaEventRecord(s->ev, st), "staging event");
    s->used = true;
    return KC_OK;
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
    Trace(kc_ctx *c_, cudaStream_t s) : c(c_), st(s) {
        if (c->trace_start) cudaEventRecord(c->trace_start, st);
    }
    ~Trace() {
        if (c->trace_stop) cudaEventRecord(c->trace_stop, st);
    }
};

uint32_t *status_word(kc_ctx *c) { return reinterpret_cast<uint32_t *>(&c->d_misc[0]); }
uint32_t *task_counter(kc_ctx *c) { return reinterpret_cast<uint32_t *>(&c->d_misc[1]); }

// Built-in digest shape: enough resident warps for every 8-page task when
// possible (so no page starts late), then the deepest ring that fits.
DigestShape pick_shape(const kc_ctx *c, uint32_t page, uint64_t npages) {
    const uint64_t tasks = (npages + 7) / 8;
    DigestShape s = c->forced;
    const size_t budget = (c->smem_per_sm ? c->smem_per_sm : 228 * 1024) - 8 * 1024;
    if (s.warps == 0) {
        uint64_t per_sm = (tasks + c->sms - 1) / c->sms;
        if (per_sm < 1) per_sm = 1;
        if (per_sm > 16) per_sm = 16;
        const size_t per_warp = budget / per_sm;
        static const int pref[][2] = {{1024, 4}, {1024, 3}, {512, 4}, {512, 3}, {2048, 2},
                                      {1024, 2}, {512, 2},  {256, 4}, {256, 3}, {256, 2}};
        s.chunk = 256;
        s.stages = 2;
        for (auto &pc : pref) {
            if ((uint32_t)pc[0] > page) continue;
            const size_t need = (size_t)pc[1] * 8 * (pc[0] + 32) + pc[1] * 8;
            if (need <= per_warp) {
                s.chunk = pc[0];
                s.stages = pc[1];
                break;
            }
        }
        s.warps = per_sm >= 4 ? 4 : (int)per_sm;
    }
    const size_t cta_smem = digest_smem_bytes(s);
    uint64_t ctas_per_sm = budget / (cta_smem + 1024);
    const uint64_t by_threads = 2048 / (32 * s.warps);
    if (ctas_per_sm > by_threads) ctas_per_sm = by_threads;
    if (ctas_per_sm > 32) ctas_per_sm = 32;
    if (ctas_per_sm < 1) ctas_per_sm = 1;
    uint64_t grid = (tasks + s.warps - 1) / s.warps;
    if (grid > ctas_per_sm * c->sms) grid = ctas_per_sm * c->sms;
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

CensusArgs make_census(const std::vector<Range> &rg, const Range *d_ranges, uint64_t win_lo, uint64_t win_hi) {
    CensusArgs ca;
    ca.ranges = d_ranges;
    ca.nranges = (int)rg.size();
    uint64_t lo = ~0ull, hi = 0;
    for (auto &r : rg) {
        lo = std::min(lo, r.base);
        hi = std::max(hi, r.end);
    }
    ca.span_lo = lo;
    ca.span_len = hi - lo;
    ca.win_lo = win_lo;
    ca.win_len = win_hi > win_lo ? win_hi - win_lo : 0;
    return ca;
}

// Census over `units`: count, scan, ordered write.
kc_status census_tail(kc_ctx *c, const Pages &units, const CensusArgs &ca, uint32_t *unit_hits,
                      uint64_t *unit_off, kc_hit *d_hits, uint64_t cap, cudaStream_t st) {
    if (!d_hits) return KC_OK;
    KC_CHECK(c, launch_scan_u32(unit_hits, unit_off, units.npages, nullptr, st), "census scan");
    KC_CHECK(c, launch_census_write(units, ca, unit_hits, unit_off, d_hits, cap, status_word(c), c->sms, st),
             "census write");
    return KC_OK;
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
        cudaMalloc(&c->d_misc, 512) != cudaSuccess || cudaMemset(c->d_misc, 0, 512) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return KC_ECUDA;
    }
    c->sms = sms;
    c->smem_per_sm = (size_t)smem;
    for (auto &s : c->slots) {
        if (cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return KC_ECUDA;
        }
    }
    *out = c;
    return KC_OK;
}

KC_API void kc_destroy(kc_ctx *c) {
    if (!c) return;
    DevGuard g(c->device);
    for (auto &s : c->slots) {
        if (s.used) cudaEventSynchronize(s.ev);
        if (s.ev) cudaEventDestroy(s.ev);
        if (s.h) cudaFreeHost(s.h);
        if (s.d) cudaFree(s.d);
    }
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

KC_API kc_status kc_set_digest_shape(kc_ctx *c, int warps, int stages, int chunk) {
    if (!c) return KC_EINVAL;
    if (warps == 0 && stages == 0 && chunk == 0) {
        c->forced = DigestShape{0, 0, 0, 0};
        return KC_OK;
    }
    if (warps < 1 || warps > 16 || stages < 2 || stages > 8 || chunk < 256 || chunk > 8192 || (chunk % 128))
        return fail(c, KC_EINVAL, "digest shape out of range (warps %d, stages %d, chunk %d)", warps, stages, chunk);
    DigestShape s{warps, stages, chunk, 1};
    if (digest_smem_bytes(s) > 227 * 1024) return fail(c, KC_EINVAL, "digest shape needs too much shared memory");
    c->forced = DigestShape{warps, stages, chunk, 0};
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
                                     int *chunk, int *ctas) {
    if (!c || !pow2_page(page_bytes)) return KC_EINVAL;
    DigestShape s = pick_shape(c, page_bytes, npages);
    if ((uint32_t)s.chunk > page_bytes) s.chunk = (int)page_bytes;
    if (warps) *warps = s.warps;
    if (stages) *stages = s.stages;
    if (chunk) *chunk = s.chunk;
    if (ctas) *ctas = s.ctas;
    return KC_OK;
}

// Shared body of kc_digest and kc_scan.
static kc_status digest_impl(kc_ctx *c, const kc_buf *allocs, int n, uint32_t page_bytes, uint64_t *d_hash,
                             uint8_t *d_zero, uint64_t *d_page_first, bool census, uint64_t win_lo,
                             uint64_t win_hi, kc_hit *d_hits, uint64_t cap, uint64_t *d_counts, void *stream) {
    if (!c) return KC_EINVAL;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!pow2_page(page_bytes)) return fail(c, KC_EINVAL, "page size %u is not a power of two in [4 KiB, 2 MiB]", page_bytes);
    if (!d_hash || !d_zero) return fail(c, KC_EINVAL, "null digest output");
    if (census && !d_counts) return fail(c, KC_EINVAL, "null census counts");
    if (census && cap && !d_hits) return fail(c, KC_EINVAL, "null census hit buffer with cap %llu", (unsigned long long)cap);
    std::vector<Region> regions;
    uint64_t P = 0;
    bool lost = false;
    kc_status s = check_regions(c, allocs, n, page_bytes, regions, &P, &lost);
    if (s != KC_OK) return s;
    std::vector<Range> rg;
    if (census && (s = build_ranges(c, allocs, n, rg)) != KC_OK) return s;
    std::vector<uint64_t> pf(n + 1);
    for (int i = 0; i < n; ++i) pf[i] = regions[i].first;
    pf[n] = P;
    std::vector<void *> dp;
    Slot *slot = nullptr;
    s = stage(c, st, {{regions.data(), regions.size() * sizeof(Region)}, {pf.data(), pf.size() * 8},
                      {rg.data(), rg.size() * sizeof(Range)}}, dp, &slot);
    if (s != KC_OK) return s;
    const Pages pg = make_pages(static_cast<Region *>(dp[0]), n, P, page_bytes);
    DigestShape shape = pick_shape(c, page_bytes, P);
    if ((uint32_t)shape.chunk > page_bytes) shape.chunk = (int)page_bytes;
    uint32_t *page_hits = nullptr;
    uint64_t *page_off = nullptr;
    CensusArgs ca{};
    if (census) {
        void *scr = nullptr;
        if ((s = scratch(c, P * 4 + 256 + P * 8, st, &scr)) != KC_OK) return s;
        page_hits = static_cast<uint32_t *>(scr);
        page_off = reinterpret_cast<uint64_t *>(static_cast<char *>(scr) + ((P * 4 + 255) & ~255ull));
        ca = make_census(rg, static_cast<Range *>(dp[2]), win_lo, win_hi);
        KC_CHECK(c, cudaMemsetAsync(d_counts, 0, 16, st), "census counts clear");
    }
    KC_CHECK(c, cudaMemsetAsync(task_counter(c), 0, 4, st), "task counter clear");
    {
        Trace tr(c, st);
        KC_CHECK(c, launch_digest(pg, census ? &ca : nullptr, d_hash, d_zero, page_hits, d_counts, task_counter(c),
                                  status_word(c), shape, st),
                 "digest launch");
    }
    if (d_page_first)
        KC_CHECK(c, cudaMemcpyAsync(d_page_first, dp[1], (n + 1) * 8, cudaMemcpyDeviceToDevice, st), "page_first copy");
    if (census && (s = census_tail(c, pg, ca, page_hits, page_off, d_hits, cap, st)) != KC_OK) return s;
    if ((s = release(c, slot, st)) != KC_OK) return s;
    return lost ? fail(c, KC_EBUF, "one or more regions were marked lost") : KC_OK;
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
    std::vector<Region> regions;
    uint64_t U = 0;
    bool lost = false;
    kc_status s = check_regions(c, allocs, n, CENSUS_UNIT, regions, &U, &lost);
    if (s != KC_OK) return s;
    std::vector<Range> rg;
    if ((s = build_ranges(c, allocs, n, rg)) != KC_OK) return s;
    std::vector<void *> dp;
    Slot *slot = nullptr;
    s = stage(c, st, {{regions.data(), regions.size() * sizeof(Region)}, {rg.data(), rg.size() * sizeof(Range)}}, dp,
              &slot);
    if (s != KC_OK) return s;
    const Pages units = make_pages(static_cast<Region *>(dp[0]), n, U, CENSUS_UNIT);
    const CensusArgs ca = make_census(rg, static_cast<Range *>(dp[1]), win_lo, win_hi);
    void *scr = nullptr;
    if ((s = scratch(c, U * 4 + 256 + U * 8, st, &scr)) != KC_OK) return s;
    uint32_t *unit_hits = static_cast<uint32_t *>(scr);
    uint64_t *unit_off = reinterpret_cast<uint64_t *>(static_cast<char *>(scr) + ((U * 4 + 255) & ~255ull));
    KC_CHECK(c, cudaMemsetAsync(d_counts, 0, 16, st), "census counts clear");
    {
        Trace tr(c, st);
        KC_CHECK(c, launch_census_count(units, ca, unit_hits, d_counts, c->sms, st), "census count");
    }
    if ((s = census_tail(c, units, ca, unit_hits, unit_off, cap ? d_hits : nullptr, cap, st)) != KC_OK) return s;
    if ((s = release(c, slot, st)) != KC_OK) return s;
    return lost ? fail(c, KC_EBUF, "one or more regions were marked lost") : KC_OK;
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
    std::vector<Region> regions;
    uint64_t P = 0;
    bool lost = false;
    kc_status s = check_regions(c, allocs, n, page_bytes, regions, &P, &lost);
    if (s != KC_OK) return s;
    if (P >= 0xFFFFFFF0ull) return fail(c, KC_EINVAL, "too many pages (%llu) for 32-bit page ids", (unsigned long long)P);
    std::vector<void *> dp;
    Slot *slot = nullptr;
    s = stage(c, st, {{regions.data(), regions.size() * sizeof(Region)}}, dp, &slot);
    if (s != KC_OK) return s;
    const Pages pg = make_pages(static_cast<Region *>(dp[0]), n, P, page_bytes);
    void *scr = nullptr;
    if ((s = scratch(c, dedup_scratch_bytes(P, nullptr), st, &scr)) != KC_OK) return s;
    DedupScratch ds;
    dedup_scratch_carve(scr, P, &ds);
    {
        Trace tr(c, st);
        KC_CHECK(c, run_dedup(pg, d_hash, d_zero, d_table, d_arena, arena_cap, d_n_blobs, ds, status_word(c), c->sms, st),
                 "dedup");
    }
    if ((s = release(c, slot, st)) != KC_OK) return s;
    return lost ? fail(c, KC_EBUF, "one or more regions were marked lost") : KC_OK;
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
    std::vector<Region> regions;
    bool lost = false;
    kc_status s = check_regions(c, allocs, n, 0, regions, nullptr, &lost);
    if (s != KC_OK) return s;
    std::vector<void *> dp;
    Slot *slot = nullptr;
    s = stage(c, st, {{regions.data(), regions.size() * sizeof(Region)}}, dp, &slot);
    if (s != KC_OK) return s;
    const Pages pg = make_pages(static_cast<Region *>(dp[0]), n, n_pages, page_bytes);
    {
        Trace tr(c, st);
        KC_CHECK(c, launch_restore(pg, d_table, n_pages, d_arena, arena_bytes, status_word(c), c->sms, st), "restore");
    }
    if ((s = release(c, slot, st)) != KC_OK) return s;
    return lost ? fail(c, KC_EBUF, "one or more regions were marked lost") : KC_OK;
}

KC_API kc_status kc_compare(kc_ctx *c, const kc_buf *got, const kc_buf *want, int npairs, double atol, double rtol,
                            kc_cmp_result *d_out, void *stream) {
    if (!c) return KC_EINVAL;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (npairs < 1 || !got || !want || !d_out) return fail(c, KC_EINVAL, "need at least one pair and an output");
    if (!(atol >= 0.0) || !(rtol >= 0.0)) return fail(c, KC_EINVAL, "tolerances must be >= 0 and not NaN");
    std::vector<CmpPair> pairs(npairs);
    c->buf_status.assign(npairs, KC_OK);
    bool lost = false;
    uint64_t tiles = 0;
    for (int k = 0; k < npairs; ++k) {
        const int dt = got[k].dtype;
        if (dt < KC_U8 || dt > KC_RAW) return fail(c, KC_EINVAL, "pair %d has dtype %d", k, dt);
        const uint64_t es = (dt == KC_F32 || dt == KC_I32) ? 4 : (dt == KC_F16 || dt == KC_BF16) ? 2 : 1;
        if (got[k].bytes != want[k].bytes) return fail(c, KC_EINVAL, "pair %d: sizes differ", k);
        if (got[k].bytes % es) return fail(c, KC_EINVAL, "pair %d: size is not a multiple of the element size", k);
        if ((got[k].base_va | want[k].base_va) & 15) return fail(c, KC_EINVAL, "pair %d: buffers not 16-byte aligned", k);
        CmpPair &p = pairs[k];
        p.got = got[k].base_va;
        p.want = want[k].base_va;
        p.nelem = got[k].bytes / es;
        p.tile_first = tiles;
        p.dtype = dt == KC_RAW ? KC_U8 : dt;
        p.lost = ((got[k].flags | want[k].flags) & KC_BUF_LOST) ? 1 : 0;
        if (p.lost) {
            lost = true;
            c->buf_status[k] = KC_EBUF;
        }
        tiles += (got[k].bytes + CMP_TILE_BYTES - 1) / CMP_TILE_BYTES;
    }
    std::vector<void *> dp;
    Slot *slot = nullptr;
    kc_status s = stage(c, st, {{pairs.data(), pairs.size() * sizeof(CmpPair)}}, dp, &slot);
    if (s != KC_OK) return s;
    {
        Trace tr(c, st);
        KC_CHECK(c, launch_compare(static_cast<CmpPair *>(dp[0]), npairs, tiles, atol, rtol, d_out, nullptr, c->sms, st),
                 "compare");
    }
    if ((s = release(c, slot, st)) != KC_OK) return s;
    return lost ? fail(c, KC_EBUF, "one or more pairs were marked lost") : KC_OK;
}

}  // extern "C"
