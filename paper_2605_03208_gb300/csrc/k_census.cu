// k_census.cu -- the pointer census kernels: the tail of the fused scan
// (count, decoupled look-back, ordered write in one launch), the standalone
// count pass, the ordered write pass, and a single-CTA scan (Section
// "Address-Space Closure": embedded device pointers inside or outside the
// captured ranges; the classification of a word is census_classify in
// kc_device.cuh).
#include <cuda_runtime.h>

#include "kc_device.cuh"
#include "kc_internal.cuh"

namespace kc {

// ---- census: classification of flagged units ------------------------------------
//
// A unit (a page, or a 64 KiB census chunk) is split between the 8 warps of
// a CTA, each taking a contiguous run of its words; a warp walks its run 256
// words per step (8 loads in flight per lane), each lane classifying its
// words against the ranges held in shared memory.  Counting needs no order;
// writing places each hit at the unit's offset plus the hits of the warps
// before it (a scan of the warps' counts) plus the hits before it in the
// warp (ballot ranks), i.e. in word order.

constexpr int CENSUS_THREADS = 256;
constexpr int CENSUS_WARPS = CENSUS_THREADS / 32;

// Hits among words [wb, we) of a unit; with `hits`, they are written from
// index `out` on (indices >= cap are dropped).
__device__ __forceinline__ void warp_census_range(const CensusArgs &ca, const Range *rg, const uint8_t *base,
                                                  uint64_t wb, uint64_t we, uint64_t unit_off, uint32_t region,
                                                  kc_hit *hits, uint64_t out, uint64_t cap, uint32_t &nin,
                                                  uint32_t &nout) {
    const uint32_t lane = lane_id();
    const uint32_t lt = lanemask_lt();
    nin = 0;
    nout = 0;
    for (uint64_t w0 = wb; w0 < we; w0 += 256) {
        uint64_t v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint64_t w = w0 + 32 * j + lane;
            v[j] = w < we ? ldg_u64(base + 8 * w) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint64_t w = w0 + 32 * j + lane;
            int cl = 0;
            int32_t tg = -1;
            if (w < we && census_pre(ca, v[j]) <= ca.pre_span) cl = census_classify(ca, rg, v[j], &tg);
            const uint32_t bin = __ballot_sync(0xffffffffu, cl == 1);
            const uint32_t bout = __ballot_sync(0xffffffffu, cl == 2);
            if (hits && cl) {
                const uint64_t idx = out + nin + nout + __popc((bin | bout) & lt);
                if (idx < cap) {
                    kc_hit h;
                    h.src_offset = unit_off + 8 * w;
                    h.value = v[j];
                    h.src_alloc = region;
                    h.target = tg;
                    hits[idx] = h;
                }
            }
            nin += __popc(bin);
            nout += __popc(bout);
        }
    }
}

struct UnitSpan {
    const uint8_t *base;
    uint64_t off, nwords;
    int region;
};

__device__ __forceinline__ UnitSpan unit_span(const Pages &u, uint64_t unit) {
    UnitSpan s;
    s.region = region_of(u.regions, u.nregions, unit);
    const Region r = u.regions[s.region];
    s.off = (unit - r.first) << u.log2page;
    const uint64_t len = r.bytes - s.off < u.page ? r.bytes - s.off : u.page;
    s.base = reinterpret_cast<const uint8_t *>(r.base + s.off);
    s.nwords = len >> 3;
    return s;
}

// ---- census tail of the fused scan: one kernel, decoupled look-back ---------------
//
// After the digest kernel, page_hits[p] is the region index + 1 for pages
// holding a word that passed the pre-filter and 0 otherwise.  The kernel is
// launched right behind the digest as a programmatic dependent: its CTAs
// stage the range table while the digest finishes and wait for it before
// reading anything it wrote.  CTAs take chunks in ticket order -- up to
// TAIL_CHUNK flagged pages each (list mode), or runs of consecutive pages
// above TAIL_LIST_MAX pages (page mode).  For each chunk: (A) the
// words of its flagged pages, taken as one sequence in page order, are split
// evenly between the CTA's warps; each warp classifies its run, counts its
// hits and keeps the first TAIL_STASH of them, in word order, in shared
// memory; (B) warp 0 scans the warps' counts, publishes the chunk's total,
// walks back over earlier chunks' published words until one carries an
// inclusive prefix (decoupled look-back) and publishes this chunk's
// inclusive prefix; (C) each warp stores its hits at prefix + the hits of
// earlier warps: from its stash, or, if it found more than TAIL_STASH, by
// classifying its run again and writing as it goes (mostly from L2).  A
// chunk waits only on chunks whose tickets were taken before its own, by
// CTAs that are running and publish their totals without waiting, so the
// walk always ends; each wait is also bounded and reports ST_TIMEOUT if it
// gives up.

constexpr int TAIL_THREADS = 512;
constexpr int TAIL_WARPS = TAIL_THREADS / 32;
constexpr int TAIL_CHUNK = 32;     // most pages per chunk (one warp lane each when listing them)
constexpr int TAIL_STASH = 128;    // hits a warp keeps in shared memory (48 KB per CTA)
constexpr uint64_t TAIL_LIST_MAX = 128ull * TAIL_THREADS;   // list mode up to here (128 page marks per thread)
constexpr unsigned long long LB_AGG = 1ull << 62;      // chunk word: total of the chunk
constexpr unsigned long long LB_PREFIX = 2ull << 62;   // chunk word: inclusive prefix
constexpr unsigned long long LB_VALUE = (1ull << 62) - 1;
constexpr uint32_t LB_SPIN_LIMIT = 1u << 22;   // polls of ~1 us each: a few seconds at most

// Span of page p of region ri.
__device__ __forceinline__ UnitSpan page_span(const Pages &u, uint64_t p, int ri) {
    UnitSpan sp;
    sp.region = ri;
    const Region r = u.regions[ri];
    sp.off = (p - r.first) << u.log2page;
    const uint64_t len = r.bytes - sp.off < u.page ? r.bytes - sp.off : u.page;
    sp.base = reinterpret_cast<const uint8_t *>(r.base + sp.off);
    sp.nwords = len >> 3;
    return sp;
}

// Exclusive prefix of chunk c: warp 0 reads the words of 256 earlier chunks
// at a time -- load k of lane l is the chunk at distance 32k + l + 1, so each
// load instruction covers 32 consecutive words (two cache lines: many chunks
// poll the same few lines) -- waits (bounded) until each is published, and
// stops at the nearest inclusive prefix, adding the totals of the chunks
// between it and c.
__device__ __forceinline__ unsigned long long lookback(volatile unsigned long long *word, uint64_t c,
                                                       uint32_t *status, uint32_t spin_limit) {
    const uint32_t lane = lane_id();
    unsigned long long prefix = 0;
    int64_t base = (int64_t)c - 1;
    while (base >= 0) {
        unsigned long long w[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = 0;
        uint32_t spins = 0;
        bool missing = true;
        while (true) {
            missing = false;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if ((w[k] & ~LB_VALUE) == 0) {   // not seen published yet
                    const int64_t j = base - (32 * k + (int64_t)lane);
                    unsigned long long x = LB_PREFIX;   // before the first chunk: prefix 0
                    if (j >= 0) x = word[j];
                    w[k] = x;
                    missing |= (w[k] & ~LB_VALUE) == 0;
                }
            }
            if (!__any_sync(0xffffffffu, missing) || ++spins >= spin_limit) break;
        }
        if (__any_sync(0xffffffffu, missing)) {
            if (lane == 0) set_status(status, ST_TIMEOUT);
            break;   // give up: the prefix is wrong, the status says so
        }
        // nearest inclusive prefix: the smallest distance 32k + l holding one
        uint32_t dmin = 0xffffffffu;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if ((w[k] & LB_PREFIX) && dmin == 0xffffffffu) dmin = 32 * k + lane;
        dmin = __reduce_min_sync(0xffffffffu, dmin);
        unsigned long long part = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if ((uint32_t)(32 * k) + lane <= dmin) part += w[k] & LB_VALUE;
#pragma unroll
        for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        prefix += part;
        if (dmin != 0xffffffffu) break;
        base -= 256;
    }
    return prefix;
}

// One warp's run [a, b) of the chunk's flagged-page word sequence: classify
// (hits to `out`, up to `cap` of them, in word order) and count.  fpid /
// freg: the flagged pages' ids and region index + 1, fstart their word
// offsets in the sequence.
__device__ __forceinline__ void tail_run(const Pages &u, const CensusArgs &ca, const Range *rg,
                                         const uint64_t *fpid, const uint32_t *freg, const uint64_t *fstart,
                                         int nflag, uint64_t a, uint64_t b, kc_hit *out, uint64_t cap,
                                         uint32_t &nin, uint32_t &nout) {
    nin = 0;
    nout = 0;
    for (int i = 0; i < nflag && a < b; ++i) {
        const uint64_t s0 = fstart[i], s1 = fstart[i + 1];
        if (s1 <= a) continue;
        if (s0 >= b) break;
        const uint64_t wb = (a > s0 ? a : s0) - s0, we = (b < s1 ? b : s1) - s0;
        const UnitSpan sp = page_span(u, fpid[i], (int)freg[i] - 1);
        uint32_t ni = 0, no = 0;
        const uint64_t done = nin + nout;
        warp_census_range(ca, rg, sp.base, wb, we, sp.off, (uint32_t)sp.region, out, done, cap, ni, no);
        nin += ni;
        nout += no;
    }
}

// List mode (snapshots up to TAIL_LIST_MAX pages): every CTA reads the
// digest's page marks itself -- thread i a run of G consecutive pages, G the
// pages per thread rounded up to 4 (at most 128), kept as bits -- and a
// block-wide scan of the bit counts numbers the flagged pages (mark != 0) in
// page order.  Chunk c holds flagged pages [c * cpages, ...), so a chunk's
// work is bounded by cpages pages however the flagged pages cluster, and
// each CTA finds its chunk's pages from the scan, with no list kernel.
__global__ void __launch_bounds__(TAIL_THREADS, 2) census_tail_kernel(Pages u, CensusArgs ca,
                                                                    const uint32_t *__restrict__ page_hits,
                                                                    unsigned long long *__restrict__ tail,
                                                                    uint64_t nchunks, uint32_t cpages,
                                                                    bool list,
                                                                    kc_hit *__restrict__ hits, uint64_t cap,
                                                                    uint64_t *__restrict__ counts,
                                                                    uint32_t *__restrict__ status,
                                                                    uint32_t *__restrict__ task_ctr,
                                                                    uint32_t spin_limit) {
    __shared__ Range srg[SMEM_RANGES];
    __shared__ kc_hit stash[TAIL_WARPS][TAIL_STASH];
    __shared__ uint32_t freg[TAIL_CHUNK];
    __shared__ uint64_t fpid[TAIL_CHUNK];
    __shared__ uint64_t fstart[TAIL_CHUNK + 1];
    __shared__ uint32_t wn[TAIL_WARPS], win_s[TAIL_WARPS], wout_s[TAIL_WARPS];
    __shared__ int s_nflag;
    __shared__ unsigned long long s_chunk, s_prefix;
    __shared__ uint32_t s_fpage[TAIL_CHUNK];   // list mode: the chunk's flagged pages
    __shared__ uint32_t s_mred[TAIL_WARPS];
    const int warp = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    unsigned long long *ticket = tail;
    volatile unsigned long long *word = tail + 1;
    // The ranges are inputs of the call, ready before the digest kernel
    // started: stage them while it finishes.  Everything after the wait reads
    // what the digest wrote (page marks, zeroed ticket, chunk words and
    // counts); the digest's task counter is then free and is reset here for
    // the next call.
    const Range *rg = stage_ranges(ca, srg);
    grid_dep_wait();
    if (threadIdx.x == 0) s_chunk = atomicAdd(ticket, 1ull);
    if (blockIdx.x == 0 && threadIdx.x == 0) *task_ctr = 0u;
    const uint32_t G = list ? (uint32_t)((u.npages + 4 * TAIL_THREADS - 1) / (4 * TAIL_THREADS)) * 4 : 0u;
    uint32_t mw[4] = {0u, 0u, 0u, 0u};   // list mode: bit 32 k + b = page G i + 32 k + b flagged
    if (list) {
        const uint64_t p0 = (uint64_t)threadIdx.x * G;
#pragma unroll
        for (uint32_t k = 0; k < 128; k += 4) {
            const uint64_t p = p0 + k;
            if (k < G && p < u.npages) {
                uint32_t m;
                if (p + 4 <= u.npages) {   // 16-byte aligned: page_hits is, and p is a multiple of 4
                    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(page_hits + p));
                    m = (v.x != 0u) | (v.y != 0u) << 1 | (v.z != 0u) << 2 | (v.w != 0u) << 3;
                } else {
                    m = 0;
                    for (uint32_t d = 0; p + d < u.npages; ++d) m |= (uint32_t)(page_hits[p + d] != 0u) << d;
                }
                mw[k >> 5] |= m << (k & 31);
            }
        }
    }
    __syncthreads();   // the first ticket
    uint64_t nentries = u.npages;
    uint32_t mpre = 0, mcnt = 0;   // list mode: flagged pages before this thread's, and its own
    if (list) {
        mcnt = __popc(mw[0]) + __popc(mw[1]) + __popc(mw[2]) + __popc(mw[3]);
        uint32_t inc = mcnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= (uint32_t)o) inc += y;
        }
        if (lane == 31) s_mred[warp] = inc;
        __syncthreads();
        uint32_t before = 0, all = 0;
        for (int w = 0; w < TAIL_WARPS; ++w) {
            if (w < warp) before += s_mred[w];
            all += s_mred[w];
        }
        mpre = before + inc - mcnt;
        nentries = all;
    }
    if (list) {   // spread the flagged pages over the grid: at most TAIL_CHUNK per chunk
        uint64_t cp = (nentries + gridDim.x - 1) / gridDim.x;
        cpages = (uint32_t)(cp < 1 ? 1 : cp > (uint64_t)TAIL_CHUNK ? TAIL_CHUNK : cp);
        nchunks = (nentries + cpages - 1) / cpages;
    }
    // with no more chunks than CTAs, every CTA takes exactly one ticket, so the
    // tickets 0 .. gridDim.x - 1 cover every chunk and none takes a second
    const bool one_round = nchunks <= gridDim.x;
    for (bool first = true;; first = false) {
        if (!first) {
            if (one_round) break;
            if (threadIdx.x == 0) s_chunk = atomicAdd(ticket, 1ull);
            __syncthreads();
        }
        const uint64_t c = s_chunk;
        if (c >= nchunks) break;
        const uint64_t e0 = c * cpages;
        const uint64_t e1 = e0 + cpages < nentries ? e0 + cpages : nentries;
        if (list) {   // the chunk's flagged pages, from the threads whose bits hold them
            if (mcnt && mpre < e1 && mpre + mcnt > e0) {
                uint32_t r = mpre;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    uint32_t x = mw[k];
                    while (x) {
                        const uint32_t b = __ffs(x) - 1;
                        x &= x - 1;
                        if (r >= e0 && r < e1) s_fpage[r - e0] = G * threadIdx.x + 32u * k + b;
                        ++r;
                    }
                }
            }
            __syncthreads();
        }
        if (warp == 0) {   // the flagged pages and their word offsets in the chunk's sequence
            const uint64_t e = e0 + lane;
            const uint64_t p = e < e1 ? (list ? (uint64_t)s_fpage[lane] : e) : 0;
            const uint32_t r = e < e1 ? page_hits[p] : 0u;
            const uint64_t nw = r ? page_span(u, p, (int)r - 1).nwords : 0;
            const uint32_t fm = __ballot_sync(0xffffffffu, r != 0);
            uint64_t inc = nw;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= (uint32_t)o) inc += y;
            }
            if (r) {
                const int slot = __popc(fm & lanemask_lt());
                fpid[slot] = p;
                freg[slot] = r;
                fstart[slot] = inc - nw;
            }
            if (lane == 31) {
                fstart[__popc(fm)] = inc;
                s_nflag = __popc(fm);
            }
        }
        __syncthreads();
        const int nflag = s_nflag;
        uint64_t total = 0;
        if (nflag) {
            // (A) count, keeping the first hits of each warp
            const uint64_t T = fstart[nflag];
            const uint64_t a = T * warp / TAIL_WARPS, b = T * (warp + 1) / TAIL_WARPS;
            uint32_t nin, nout;
            tail_run(u, ca, rg, fpid, freg, fstart, nflag, a, b, stash[warp], TAIL_STASH, nin, nout);
            if (lane == 0) {
                wn[warp] = nin + nout;
                win_s[warp] = nin;
                wout_s[warp] = nout;
            }
            __syncthreads();
            for (int w = 0; w < TAIL_WARPS; ++w) total += wn[w];
        }
        // (B) publish the total, look back, publish the inclusive prefix; a
        // chunk without hits needs no prefix: it publishes its zero total
        // and later chunks walk past it
        if (warp == 0) {
            unsigned long long prefix = 0;
            if (c == 0) {
                if (lane == 0) word[0] = LB_PREFIX | total;
            } else if (total == 0) {
                if (lane == 0) word[c] = LB_AGG;
            } else {
                if (lane == 0) word[c] = LB_AGG | total;
                prefix = lookback(word, c, status, spin_limit);
                if (lane == 0) word[c] = LB_PREFIX | (prefix + total);
            }
            if (lane == 0) {
                s_prefix = prefix;
                if (hits && prefix + total > cap) set_status(status, ST_TRUNC);
                if (nflag) {
                    uint32_t si = 0, so = 0;
                    for (int w = 0; w < TAIL_WARPS; ++w) {
                        si += win_s[w];
                        so += wout_s[w];
                    }
                    if (si) atomicAdd(reinterpret_cast<unsigned long long *>(&counts[0]), (unsigned long long)si);
                    if (so) atomicAdd(reinterpret_cast<unsigned long long *>(&counts[1]), (unsigned long long)so);
                }
            }
        }
        __syncthreads();
        // (C) ordered write
        if (hits && total) {
            uint64_t before = s_prefix;
            for (int w = 0; w < warp; ++w) before += wn[w];
            const uint32_t n = wn[warp];
            if (n <= (uint32_t)TAIL_STASH) {
                for (uint32_t i = lane; i < n; i += 32)
                    if (before + i < cap) hits[before + i] = stash[warp][i];
            } else {
                const uint64_t T = fstart[nflag];
                const uint64_t a = T * warp / TAIL_WARPS, b = T * (warp + 1) / TAIL_WARPS;
                uint32_t nin, nout;
                tail_run(u, ca, rg, fpid, freg, fstart, nflag, a, b, hits + before, cap > before ? cap - before : 0,
                         nin, nout);
            }
        }
        __syncthreads();
    }
}

// Pages per chunk (page mode): enough chunks for every resident CTA to take
// one, as few as 8 pages and at most TAIL_CHUNK.
static uint32_t tail_chunk_pages(uint64_t npages, int sms) {
    const uint64_t ctas = (uint64_t)sms * 2;   // resident CTAs (2 per SM by registers)
    uint64_t cp = (npages + ctas - 1) / ctas;
    if (cp < 8) cp = 8;
    if (cp > (uint64_t)TAIL_CHUNK) cp = TAIL_CHUNK;
    return (uint32_t)cp;
}

uint64_t census_tail_words(uint64_t npages, int sms) {
    if (npages <= TAIL_LIST_MAX) return 1 + npages;
    const uint32_t cp = tail_chunk_pages(npages, sms);
    return 1 + (npages + cp - 1) / cp;
}

cudaError_t launch_census_tail(const Pages &pg, const CensusArgs &ca, uint32_t *page_hits, unsigned long long *tail,
                               kc_hit *hits, uint64_t cap, uint64_t *counts, uint32_t *status, uint32_t *task_ctr,
                               int sms, uint32_t spin_limit, cudaStream_t st) {
    if (spin_limit == 0) spin_limit = LB_SPIN_LIMIT;
    const uint64_t maxb = (uint64_t)sms * 2;
    const bool list = pg.npages <= TAIL_LIST_MAX;
    uint64_t nchunks = pg.npages, blocks = maxb;
    uint32_t cp = 1;
    if (!list) {
        cp = tail_chunk_pages(pg.npages, sms);
        nchunks = (pg.npages + cp - 1) / cp;
        blocks = nchunks < maxb ? nchunks : maxb;
    }
    if (blocks == 0) blocks = 1;   // no pages: one CTA still resets the task counter
    // programmatic dependent launch after the digest kernel (which triggers it early)
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(TAIL_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, census_tail_kernel, pg, ca, (const uint32_t *)page_hits, tail, nchunks,
                                       cp, list, cap ? hits : nullptr, cap, counts, status, task_ctr, spin_limit);
    count_launches(1);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// ---- census: standalone count pass ---------------------------------------------------
//
// Units are 64 KiB chunks of the regions.  One CTA counts one unit with
// 16-byte streaming loads; candidates (rare unless the data holds pointers)
// are classified against the ranges in shared memory.

__device__ __forceinline__ void census_word(const CensusArgs &ca, const Range *rg, uint64_t v, uint32_t &hin,
                                            uint32_t &hout) {
    if (census_pre(ca, v) > ca.pre_span) return;
    int32_t tg;
    const int cl = census_classify(ca, rg, v, &tg);
    hin += cl == 1;
    hout += cl == 2;
}

__global__ void __launch_bounds__(CENSUS_THREADS) census_count_kernel(Pages u, CensusArgs ca,
                                                                      uint32_t *__restrict__ unit_hits,
                                                                      uint64_t *__restrict__ counts) {
    __shared__ Range srg[SMEM_RANGES];
    __shared__ uint32_t red_in[CENSUS_THREADS / 32], red_out[CENSUS_THREADS / 32];
    const Range *rg = stage_ranges(ca, srg);
    for (uint64_t unit = blockIdx.x; unit < u.npages; unit += gridDim.x) {
        const int a = region_of(u.regions, u.nregions, unit);
        const Region r = u.regions[a];
        uint32_t hin = 0, hout = 0;
        if (!r.lost) {
            const uint64_t off = (unit - r.first) << u.log2page;
            const uint64_t len = r.bytes - off < u.page ? r.bytes - off : u.page;
            const uint8_t *base = reinterpret_cast<const uint8_t *>(r.base + off);
            const uint64_t nwords = len >> 3;
            const uint64_t nvec = nwords >> 1;
            uint64_t i = threadIdx.x;
            for (; i + 3 * CENSUS_THREADS < nvec; i += 4 * CENSUS_THREADS) {
                uint4 v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) v[j] = ldg_stream(base + 16 * (i + j * CENSUS_THREADS));
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    census_word(ca, rg, ((uint64_t)v[j].y << 32) | v[j].x, hin, hout);
                    census_word(ca, rg, ((uint64_t)v[j].w << 32) | v[j].z, hin, hout);
                }
            }
            for (; i < nvec; i += CENSUS_THREADS) {
                const uint4 v = ldg_stream(base + 16 * i);
                census_word(ca, rg, ((uint64_t)v.y << 32) | v.x, hin, hout);
                census_word(ca, rg, ((uint64_t)v.w << 32) | v.z, hin, hout);
            }
            if ((nwords & 1) && threadIdx.x == 0) census_word(ca, rg, ldg_u64(base + 8 * (nwords - 1)), hin, hout);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            hin += __shfl_xor_sync(0xffffffffu, hin, o);
            hout += __shfl_xor_sync(0xffffffffu, hout, o);
        }
        if (lane_id() == 0) {
            red_in[threadIdx.x >> 5] = hin;
            red_out[threadIdx.x >> 5] = hout;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t si = 0, so = 0;
            for (int w = 0; w < CENSUS_THREADS / 32; ++w) {
                si += red_in[w];
                so += red_out[w];
            }
            unit_hits[unit] = si + so;
            if (si) atomicAdd(reinterpret_cast<unsigned long long *>(&counts[0]), (unsigned long long)si);
            if (so) atomicAdd(reinterpret_cast<unsigned long long *>(&counts[1]), (unsigned long long)so);
        }
        __syncthreads();
    }
}

cudaError_t launch_census_count(const Pages &units, const CensusArgs &ca, uint32_t *unit_hits, uint64_t *counts,
                                int sms, cudaStream_t st) {
    uint64_t blocks = units.npages;
    const uint64_t maxb = (uint64_t)sms * 8;
    if (blocks > maxb) blocks = maxb;
    if (blocks == 0) return cudaSuccess;
    census_count_kernel<<<(unsigned)blocks, CENSUS_THREADS, 0, st>>>(units, ca, unit_hits, counts);
    count_launches(1);
    return cudaGetLastError();
}

// ---- census: ordered write pass ---------------------------------------------------
//
// One CTA per unit that holds hits: a counting pass per warp, a scan of the
// warps' counts, then the writing pass.  Only units with hits are read
// again (the second walk mostly hits L2).

__global__ void __launch_bounds__(CENSUS_THREADS) census_write_kernel(Pages u, CensusArgs ca,
                                                                      const uint32_t *__restrict__ unit_hits,
                                                                      const uint64_t *__restrict__ unit_off,
                                                                      kc_hit *__restrict__ hits, uint64_t cap,
                                                                      uint32_t *__restrict__ status) {
    __shared__ Range srg[SMEM_RANGES];
    __shared__ uint32_t wcount[CENSUS_WARPS];
    const Range *rg = stage_ranges(ca, srg);
    const int warp = threadIdx.x >> 5;
    for (uint64_t unit = blockIdx.x; unit < u.npages; unit += gridDim.x) {
        const uint32_t cnt = unit_hits[unit];
        if (cnt == 0) continue;   // uniform across the CTA
        const UnitSpan sp = unit_span(u, unit);
        const uint64_t per = (sp.nwords + CENSUS_WARPS - 1) / CENSUS_WARPS;
        const uint64_t wb = per * warp, we = wb + per < sp.nwords ? wb + per : sp.nwords;
        uint32_t nin = 0, nout = 0;
        if (wb < we) warp_census_range(ca, rg, sp.base, wb, we, sp.off, (uint32_t)sp.region, nullptr, 0, 0, nin, nout);
        if (lane_id() == 0) wcount[warp] = nin + nout;
        __syncthreads();
        uint64_t before = 0, total = 0;
        for (int w = 0; w < CENSUS_WARPS; ++w) {
            if (w < warp) before += wcount[w];
            total += wcount[w];
        }
        const uint64_t out = unit_off[unit];
        if (wb < we)
            warp_census_range(ca, rg, sp.base, wb, we, sp.off, (uint32_t)sp.region, hits, out + before, cap, nin,
                              nout);
        if (threadIdx.x == 0) {
            if (total != cnt) set_status(status, ST_INTERNAL);
            if (out + cnt > cap) set_status(status, ST_TRUNC);
        }
        __syncthreads();
    }
}

cudaError_t launch_census_write(const Pages &units, const CensusArgs &ca, const uint32_t *unit_hits,
                                const uint64_t *unit_off, kc_hit *hits, uint64_t cap, uint32_t *status, int sms,
                                cudaStream_t st) {
    uint64_t blocks = units.npages;
    const uint64_t maxb = (uint64_t)sms * 8;
    if (blocks > maxb) blocks = maxb;
    if (blocks == 0) return cudaSuccess;
    census_write_kernel<<<(unsigned)blocks, CENSUS_THREADS, 0, st>>>(units, ca, unit_hits, unit_off, hits, cap,
                                                                     status);
    count_launches(1);
    return cudaGetLastError();
}

// ---- single-CTA exclusive scan ------------------------------------------------

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 8;

__global__ void __launch_bounds__(SCAN_THREADS) scan_u32_kernel(const uint32_t *__restrict__ in,
                                                                uint64_t *__restrict__ out, uint64_t n,
                                                                uint64_t *__restrict__ total) {
    __shared__ uint64_t warp_sum[SCAN_THREADS / 32];
    __shared__ uint64_t carry_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (uint64_t base = 0; base < n; base += (uint64_t)SCAN_THREADS * SCAN_ITEMS) {
        uint32_t v[SCAN_ITEMS];
        uint64_t local = 0;
        const uint64_t i0 = base + (uint64_t)tid * SCAN_ITEMS;
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) {
            v[j] = (i0 + j < n) ? in[i0 + j] : 0u;
            local += v[j];
        }
        uint64_t incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint64_t ws = warp_sum[lane];
            uint64_t wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            warp_sum[lane] = wi - ws;   // exclusive prefix of warps
        }
        __syncthreads();
        uint64_t run = carry_s + warp_sum[warp] + (incl - local);
#pragma unroll
        for (int j = 0; j < SCAN_ITEMS; ++j) {
            if (i0 + j < n) out[i0 + j] = run;
            run += v[j];
        }
        __syncthreads();
        if (tid == SCAN_THREADS - 1) carry_s = run;
        __syncthreads();
    }
    if (tid == 0 && total) *total = carry_s;
}

cudaError_t launch_scan_u32(const uint32_t *in, uint64_t *out, uint64_t n, uint64_t *total, cudaStream_t st) {
    scan_u32_kernel<<<1, SCAN_THREADS, 0, st>>>(in, out, n, total);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t preload_census_kernels(cudaStream_t st) {
    cudaFuncAttributes fa;
    cudaError_t e;
    if ((e = cudaFuncGetAttributes(&fa, census_count_kernel)) != cudaSuccess ||
        (e = cudaFuncGetAttributes(&fa, census_write_kernel)) != cudaSuccess ||
        (e = cudaFuncGetAttributes(&fa, scan_u32_kernel)) != cudaSuccess)
        return e;
    Pages none{};
    CensusArgs ca{};
    census_count_kernel<<<1, CENSUS_THREADS, 0, st>>>(none, ca, nullptr, nullptr);
    census_write_kernel<<<1, CENSUS_THREADS, 0, st>>>(none, ca, nullptr, nullptr, nullptr, 0, nullptr);
    scan_u32_kernel<<<1, SCAN_THREADS, 0, st>>>(nullptr, nullptr, 0, nullptr);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace kc
