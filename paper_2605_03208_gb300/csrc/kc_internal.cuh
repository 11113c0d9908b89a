// kc_internal.cuh -- types and launch entry points shared by the library's
// translation units (host planner in kc_api.cu, kernels in k_*.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kc.h"

namespace kc {

// Device-side condition bits, OR-ed into the context's status word.
enum : uint32_t {
    ST_TRUNC = 1u << 0,    // an output capacity was exceeded
    ST_TIMEOUT = 1u << 1,  // a bounded wait gave up
    ST_BADROW = 1u << 2,   // a page-table row pointed outside a region/arena
    ST_INTERNAL = 1u << 3  // an internal consistency check failed
};

// One region as the kernels see it (32 bytes).  `first` is the id of the
// region's first unit (page or census chunk) in the flattened unit space.
struct Region {
    uint64_t base;
    uint64_t bytes;
    uint64_t first;
    uint32_t lost;   // 1: region not readable, skip it
    uint32_t pad;
};

// Census range, sorted by base (24 bytes).
struct Range {
    uint64_t base;
    uint64_t end;
    int32_t id;
    int32_t pad;
};

// Census parameters: a word v is a candidate iff it lies in the captured
// span [span_lo, span_lo + span_len) or the window [win_lo, win_lo + win_len).
// pre_lo / pre_span: a cheap conservative pre-filter on the high 32 bits of
// a word -- every candidate satisfies (hi32(v) - pre_lo) <= pre_span
// (unsigned); pre_span = 0xFFFFFFFF disables it.
struct CensusArgs {
    const Range *ranges;
    int nranges;
    uint64_t span_lo, span_len;
    uint64_t win_lo, win_len;
    uint32_t pre_lo, pre_span;
};

// Census parameters for the ranges rg[0..n) (sorted by base, disjoint) and
// the window [win_lo, win_hi): the captured span, the window, and the
// high-32-bit pre-filter over the hull of the non-empty intervals (every
// value inside either interval passes it; pre_span 0 with pre_lo all-ones
// when nothing can be a hit).  Used by both the context-based census and
// the static one, so the two classify identically.
inline CensusArgs census_args(const Range *rg, int n, uint64_t win_lo, uint64_t win_hi) {
    CensusArgs ca{};
    ca.nranges = n;
    uint64_t lo = ~0ull, hi = 0;
    for (int i = 0; i < n; ++i) {
        lo = rg[i].base < lo ? rg[i].base : lo;
        hi = rg[i].end > hi ? rg[i].end : hi;
    }
    ca.span_lo = lo;
    ca.span_len = n > 0 ? hi - lo : 0;
    ca.win_lo = win_lo;
    ca.win_len = win_hi > win_lo ? win_hi - win_lo : 0;
    uint64_t plo = ~0ull, phi = 0;   // inclusive bounds
    if (ca.span_len) {
        plo = ca.span_lo < plo ? ca.span_lo : plo;
        phi = ca.span_lo + ca.span_len - 1 > phi ? ca.span_lo + ca.span_len - 1 : phi;
    }
    if (ca.win_len) {
        plo = ca.win_lo < plo ? ca.win_lo : plo;
        phi = ca.win_lo + ca.win_len - 1 > phi ? ca.win_lo + ca.win_len - 1 : phi;
    }
    if (plo > phi) {
        ca.pre_lo = 0xFFFFFFFFu;
        ca.pre_span = 0;
    } else {
        ca.pre_lo = (uint32_t)(plo >> 32);
        ca.pre_span = (uint32_t)(phi >> 32) - ca.pre_lo;
    }
    return ca;
}

// Work description shared by the page-granular kernels.
struct Pages {
    const Region *regions;
    int nregions;
    uint64_t npages;   // P
    uint32_t page;     // bytes per page (power of two)
    uint32_t log2page;
};

// Digest kernel shape (chosen by the host planner or the autotuner).
struct DigestShape {
    int warps;        // hash warps per CTA (digest kernel: plus as many loader warps)
    int stages;       // ring depth per hash warp
    int chunk;        // bytes per page per stage (multiple of 128, <= page)
    int ctas;         // grid size
    int lanes;        // XXH64 lanes per thread: always 1 (8 pages per warp)
};

// Dynamic shared memory of a CTA of the digest kernel (warps = hash warps)
// and of the batched kernel (warps = warps of the CTA; fused: its stages
// also hold the compared buffer's chunks).
size_t digest_smem_bytes(const DigestShape &s);
size_t batch_smem_bytes(const DigestShape &s, bool fused);
int digest_max_hash_warps();

// Process-wide count of kernels launched by this library (every launcher
// adds its launches); read by kc_launch_count().
void count_launches(uint64_t n);
uint64_t launches_so_far();

// One-time per-process kernel attributes (maximum dynamic shared memory).
cudaError_t setup_kernels();
cudaError_t setup_digest_kernels();
cudaError_t setup_dedup_kernels();

// Launchers (each returns the cudaError_t of its launch).
// Set-up work done by the digest kernel's threads before hashing.
struct DigestAux {
    unsigned long long *zero_words = nullptr;   // zeroed (census tail ticket + chunk words)
    uint64_t nzero = 0;
    unsigned long long first_ticket = 0;        // zero_words[0] gets this instead (a test hook)
    uint64_t *counts = nullptr;                 // caller's census counts, zeroed
    const uint64_t *pf_src = nullptr;           // page offsets copied to the caller
    uint64_t *pf_dst = nullptr;
    uint64_t npf = 0;
};
// `census` NULL: digest only.  Otherwise page_hits[P] receives 0 for pages
// that cannot hold a census hit and a pending mark for the others, which
// launch_census_tail then resolves.
cudaError_t launch_digest(const Pages &pg, const CensusArgs *census, uint64_t *hash, uint8_t *zero,
                          uint32_t *page_hits, uint32_t *task_ctr, uint32_t *status, const DigestShape &shape,
                          const DigestAux &aux, cudaStream_t st);
// Census of the fused scan, launched right after the digest kernel on the
// same stream (programmatic dependent launch: it waits for the digest inside
// the kernel).  tail: census_tail_words(P, sms) words zeroed by the digest
// kernel; task_ctr: the digest's task counter, reset to zero for the next
// call (also when P = 0).
uint64_t census_tail_words(uint64_t npages, int sms);
// spin_limit: polls each look-back wait makes before it gives up (0 = the
// built-in limit of a few seconds).
cudaError_t launch_census_tail(const Pages &pg, const CensusArgs &ca, uint32_t *page_hits, unsigned long long *tail,
                               kc_hit *hits, uint64_t cap, uint64_t *counts, uint32_t *status, uint32_t *task_ctr,
                               int sms, uint32_t spin_limit, cudaStream_t st);
cudaError_t launch_census_count(const Pages &units, const CensusArgs &ca, uint32_t *unit_hits,
                                uint64_t *counts, int sms, cudaStream_t st);
cudaError_t launch_census_write(const Pages &units, const CensusArgs &ca,
                                const uint32_t *unit_hits, const uint64_t *unit_off,
                                kc_hit *hits, uint64_t cap, uint32_t *status, int sms,
                                cudaStream_t st);

// Load the standalone census kernels (count, scan, write) on the current
// device now -- each launched once with no work on `st` -- so that a later
// call launches code that is already resident.
cudaError_t preload_census_kernels(cudaStream_t st);

// Single-CTA exclusive scan of n u32 values into u64 offsets; total -> *total.
cudaError_t launch_scan_u32(const uint32_t *in, uint64_t *out, uint64_t n, uint64_t *total,
                            cudaStream_t st);

// Dedup pipeline (k_dedup.cu).
struct DedupScratch {
    uint64_t *keys[2];
    uint32_t *vals[2];
    uint32_t *flags;      // per page
    uint64_t *pos;        // per page scan output
    uint64_t *misc;       // small counters: [0] m (non-zero pages), [1] n_blobs, [2] ndup
    uint32_t *hist;       // radix histograms (256 * ntiles)
    uint64_t *hist_off;   // scanned histograms
    uint32_t *seg;        // per sorted element: segment start index
    uint32_t *neq;        // per sorted element: 1 if bytes differ from predecessor
    uint32_t *bad;        // per sorted element: segment needs the slow path
    uint32_t *canon;      // per page: canonical page id
    uint32_t *blob_page;  // per blob: canonical page id
    uint32_t *dups;       // compacted positions with an equal-hash predecessor
    uint32_t *reps;       // slow path representatives
    uint64_t capacity_pages;
    uint64_t capacity_tiles;
};
size_t dedup_scratch_bytes(uint64_t P, uint64_t *tiles_out);
void dedup_scratch_carve(void *base, uint64_t P, DedupScratch *s);
cudaError_t run_dedup(const Pages &pg, const uint64_t *hash, const uint8_t *zero, kc_page *table,
                      uint8_t *arena, uint64_t arena_cap, uint64_t *n_blobs, DedupScratch &s,
                      uint32_t *status, int sms, cudaStream_t st);

// Restore (k_restore.cu).
cudaError_t launch_restore(const Pages &pg, const kc_page *table, uint64_t nrows,
                           const uint8_t *arena, uint64_t arena_bytes, uint32_t *status, int sms,
                           cudaStream_t st);

// Compare (k_compare.cu).
struct CmpPair {
    uint64_t got;
    uint64_t want;
    uint64_t nelem;
    uint64_t tile_first;   // first global tile id of this pair
    int32_t dtype;
    int32_t lost;
    uint64_t vec_first;    // first of this pair's whole 16-byte vectors among its dtype group's
    uint32_t out_index;    // index of the pair's record in the caller's output
    uint32_t pad;
};
// Pairs sorted by dtype: group d (dtype d) is pairs [gfirst[d], gfirst[d+1])
// with gvec[d] whole 16-byte vectors in all (vec_first counts within the
// group); each record goes to out[pair.out_index].
struct CmpGroups {
    int gfirst[7];
    uint64_t gvec[6];
};
// gates: 2 x npairs words of device scratch (the pairs' proxy maxima).
cudaError_t launch_compare(const CmpPair *pairs, int npairs, const CmpGroups &groups, double atol, double rtol,
                           kc_cmp_result *out, uint32_t *gates, int sms, cudaStream_t st);
cudaError_t setup_compare_kernels();
constexpr uint32_t CMP_TILE_BYTES = 16 * 1024;

// Batched form (k_batch.cu).  A job is one buffer to digest and/or compare,
// with its own outputs; a range is a run of a job's units (pages or
// comparison items) scheduled in one launch.
enum : uint32_t { BJ_DIGEST = 1, BJ_COMPARE = 2, BJ_LOST = 4, BJ_INIT = 8 };
struct BatchJob {          // 88 bytes
    uint64_t got, want, bytes, nelem;
    uint64_t *hash;
    uint8_t *zero;
    kc_cmp_result *cmp;
    int32_t dtype;         // comparison dtype (KC_RAW folded into KC_U8)
    uint32_t flags;        // BJ_*
    uint32_t *done;        // completion flag, or null
    kc_cmp_result *cmp_copy;
    uint32_t items;        // work items of this job in the launch
    uint32_t pad;
};
struct BatchRange {        // 32 bytes
    uint64_t first;        // first unit
    uint64_t count;        // units
    uint64_t item_first;   // first work item of the range in the launch
    uint32_t job;
    uint32_t kind;         // BR_DIGEST / BR_COMPARE / BR_FUSED
};
// Range kinds: pages to digest (8 per item); comparison items (64 KiB of
// each buffer per item); pages to digest and compare in one pass (8 per
// item: got is read once).
enum : uint32_t { BR_DIGEST = 0, BR_COMPARE = 1, BR_FUSED = 2 };
constexpr uint32_t BATCH_CMP_ITEM_BYTES = 4 * CMP_TILE_BYTES;   // 64 KiB per comparison item
static_assert(BATCH_CMP_ITEM_BYTES == KC_BATCH_ITEM_BYTES, "comparison item size");
cudaError_t launch_batch(const BatchJob *jobs, int njobs, uint32_t *left, const BatchRange *ranges, int nranges,
                         uint64_t nitems, uint32_t page, const DigestShape &shape, bool fused, double atol,
                         double rtol, uint32_t *ctr, int sms, cudaStream_t st);
cudaError_t setup_batch_kernels();

}  // namespace kc
