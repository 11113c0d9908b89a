// k_dedup.cu -- byte-verified page dedup and blob packing.
//
// Pipeline (every count the host cannot know without a sync -- the number of
// non-zero pages m, of equal-hash neighbours, of bad segments, of blobs --
// stays in device memory and is read by the kernels themselves):
//   1. compact the non-zero pages into (hash, page id) pairs, page order;
//   2. stable LSD radix sort on the low SORT_BITS = 32 bits of the hash,
//      8-bit digits, 4 passes: equal hashes end up adjacent, in increasing
//      page id (two different hashes that share their low 32 bits may
//      interleave; their segment then fails verification and takes the
//      slow path below, which decides by bytes alone, so the result is the
//      same as a sort on all 64 bits);
//   3. segments = runs of equal sort key; every element that has an equal-key
//      predecessor is byte-compared with it (16 KiB pieces, one warp each);
//   4. a segment whose elements all equal their predecessors is one class,
//      canonical = its first (smallest) page id; any other segment (a hash
//      collision, or equal hashes of different lengths) takes the slow path:
//      one CTA visits its pages in order and compares each with the
//      representatives found so far, exactly the class definition;
//   5. blob ids = exclusive scan of "page is canonical" in page order; the
//      page table is written VA-faithfully (region index, offset);
//   6. pack copies every canonical page into its arena slot, zero-filled.
// Snapshots of at most DD_SMALL pages replace steps 1-5 by hash tables in
// shared memory, the keys split over DD_PARTS CTAs (no sort; see "small
// snapshots" below).
#include <cuda_runtime.h>

#include "kc_device.cuh"
#include "kc_internal.cuh"

namespace kc {

constexpr int RS_TILE_THREADS = 256;
constexpr int RS_TILE_ITEMS = 16;
constexpr int RS_TILE = RS_TILE_THREADS * RS_TILE_ITEMS;      // 4096 keys per tile
constexpr uint32_t DD_PIECE = 16 * 1024;
constexpr int SORT_BITS = 32;   // bits of the hash the radix sort orders by

__device__ __forceinline__ uint32_t sort_key(uint64_t k) { return (uint32_t)k; }

static inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

size_t dedup_scratch_bytes(uint64_t P, uint64_t *tiles_out) {
    const uint64_t tiles = ceil_div(P ? P : 1, RS_TILE);
    if (tiles_out) *tiles_out = tiles;
    const uint64_t n = P ? P : 1;
    size_t b = 0;
    b += 2 * n * 8;          // keys[2]
    b += 2 * n * 4;          // vals[2]
    b += n * 4;              // flags
    b += n * 8;              // pos
    b += 64;                 // misc
    b += 256 * tiles * 4;    // hist
    b += 256 * tiles * 8;    // hist_off
    b += 6 * n * 4;          // seg, neq, bad, canon, blob_page, dups
    b += n * 4;              // reps
    return b + 16 * 256;     // alignment slack
}

void dedup_scratch_carve(void *base, uint64_t P, DedupScratch *s) {
    uint64_t tiles;
    dedup_scratch_bytes(P, &tiles);
    const uint64_t n = P ? P : 1;
    uintptr_t p = reinterpret_cast<uintptr_t>(base);
    auto take = [&](size_t bytes) {
        p = (p + 255) & ~(uintptr_t)255;
        void *r = reinterpret_cast<void *>(p);
        p += bytes;
        return r;
    };
    s->keys[0] = (uint64_t *)take(n * 8);
    s->keys[1] = (uint64_t *)take(n * 8);
    s->vals[0] = (uint32_t *)take(n * 4);
    s->vals[1] = (uint32_t *)take(n * 4);
    s->flags = (uint32_t *)take(n * 4);
    s->pos = (uint64_t *)take(n * 8);
    s->misc = (uint64_t *)take(64);
    s->hist = (uint32_t *)take(256 * tiles * 4);
    s->hist_off = (uint64_t *)take(256 * tiles * 8);
    s->seg = (uint32_t *)take(n * 4);
    s->neq = (uint32_t *)take(n * 4);
    s->bad = (uint32_t *)take(n * 4);
    s->canon = (uint32_t *)take(n * 4);
    s->blob_page = (uint32_t *)take(n * 4);
    s->dups = (uint32_t *)take(n * 4);
    s->reps = (uint32_t *)take(n * 4);
    s->capacity_pages = n;
    s->capacity_tiles = tiles;
}

// ---- page location ---------------------------------------------------------------

struct PageLoc {
    const uint8_t *ptr;
    uint64_t len;
    uint64_t off;
    int region;
};

__device__ __forceinline__ PageLoc locate(const Pages &pg, uint64_t p) {
    PageLoc l;
    l.region = region_of(pg.regions, pg.nregions, p);
    const Region r = pg.regions[l.region];
    l.off = (p - r.first) << pg.log2page;
    l.len = r.bytes - l.off < pg.page ? r.bytes - l.off : pg.page;
    l.ptr = reinterpret_cast<const uint8_t *>(r.base + l.off);
    return l;
}

// ---- 1. compaction ----------------------------------------------------------------

__global__ void dd_flag_kernel(const uint8_t *__restrict__ zero, uint64_t P, uint32_t *__restrict__ flags) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (uint64_t)gridDim.x * blockDim.x)
        flags[p] = zero[p] == KC_PAGE_DATA ? 1u : 0u;
}

__global__ void dd_compact_kernel(const uint64_t *__restrict__ hash, const uint32_t *__restrict__ flags,
                                  const uint64_t *__restrict__ pos, uint64_t P, uint64_t *__restrict__ keys,
                                  uint32_t *__restrict__ vals) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (uint64_t)gridDim.x * blockDim.x) {
        if (flags[p]) {
            keys[pos[p]] = hash[p];
            vals[pos[p]] = (uint32_t)p;
        }
    }
}

// ---- 2. radix sort ----------------------------------------------------------------
//
// Stable ranking inside a group of warps: warp w owns a contiguous run of the
// input and walks it 32 elements at a time in order; __match_any_sync finds
// the lanes with the same digit, so an element's rank inside its warp and
// digit is the warp's running count for that digit plus the number of
// earlier lanes with that digit.  Warp counts are then scanned digit-major
// (digit, then warp), which keeps the order of equal digits.

__device__ __forceinline__ uint32_t digit_of(uint64_t k, int shift) { return (uint32_t)(k >> shift) & 0xffu; }

// Rank ITEMS striped elements of this warp; wcnt = this warp's 256 counters.
// The lanes sharing a lane's 8-bit digit are found with eight ballots, one
// per digit bit (a lane's peers agree with it on every bit).
template <int ITEMS>
__device__ __forceinline__ void warp_rank(const uint64_t (&key)[ITEMS], int shift, uint32_t *wcnt,
                                          uint16_t (&local)[ITEMS]) {
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
        const uint32_t d = digit_of(key[r], shift);
        uint32_t peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const uint32_t bit = (d >> b) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bal : ~bal;
        }
        const uint32_t before = __popc(peers & lt);
        const uint32_t base = wcnt[d];
        local[r] = (uint16_t)(base + before);
        __syncwarp();
        if (before == 0) wcnt[d] = base + __popc(peers);
        __syncwarp();
    }
}

// Block-wide exclusive sum of one u32 per thread; *total gets the sum.
// `ws` is 32 words of shared scratch.  Every thread must call it.
__device__ __forceinline__ uint32_t block_excl_sum(uint32_t v, uint32_t *ws, uint32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = lane < nw ? ws[lane] : 0u;
        uint32_t xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        ws[lane] = xi - x;
        if (lane == 31) ws[32] = xi;
    }
    __syncthreads();
    const uint32_t r = ws[warp] + inc - v;
    if (total) *total = ws[32];
    __syncthreads();
    return r;
}

// Block-wide inclusive max of one u32 per thread.  `ws`: 33 words of scratch.
__device__ __forceinline__ uint32_t block_incl_max(uint32_t v, uint32_t *ws) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = y > inc ? y : inc;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const uint32_t x = lane < nw ? ws[lane] : 0u;
        uint32_t xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi = y > xi ? y : xi;
        }
        uint32_t ex = __shfl_up_sync(0xffffffffu, xi, 1);
        ws[lane] = lane ? ex : 0u;
    }
    __syncthreads();
    const uint32_t r = ws[warp] > inc ? ws[warp] : inc;
    __syncthreads();
    return r;
}

// Block-wide exclusive max of one u32 per thread (0 for thread 0).
__device__ __forceinline__ uint32_t block_excl_max(uint32_t v, uint32_t *ws) {
    const uint32_t inc = block_incl_max(v, ws);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t prev = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (lane == 0) prev = warp ? ws[warp - 1] : 0u;
    __syncthreads();
    return prev;
}

// Tiled pass, part 1: per-tile digit histogram, stored digit-major.
__global__ void __launch_bounds__(RS_TILE_THREADS) rs_hist_kernel(const uint64_t *__restrict__ keys,
                                                                  const uint64_t *__restrict__ m_ptr, int shift,
                                                                  uint32_t *__restrict__ hist, uint32_t ntiles) {
    __shared__ uint32_t h[256];
    const uint64_t m = *m_ptr;
    const uint32_t tile = blockIdx.x;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint64_t t0 = (uint64_t)tile * RS_TILE;
    for (int j = threadIdx.x; j < RS_TILE; j += blockDim.x) {
        const uint64_t i = t0 + j;
        if (i < m) atomicAdd(&h[digit_of(keys[i], shift)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(uint64_t)d * ntiles + tile] = h[d];
}

// Tiled pass, part 3: stable scatter of one tile at its scanned offsets.
__global__ void __launch_bounds__(RS_TILE_THREADS) rs_scatter_kernel(const uint64_t *__restrict__ kin,
                                                                     const uint32_t *__restrict__ vin,
                                                                     const uint64_t *__restrict__ m_ptr, int shift,
                                                                     const uint64_t *__restrict__ hist_off,
                                                                     uint32_t ntiles, uint64_t *__restrict__ kout,
                                                                     uint32_t *__restrict__ vout) {
    constexpr int NW = RS_TILE_THREADS / 32;
    constexpr int PER_WARP = 32 * RS_TILE_ITEMS;
    __shared__ uint32_t cnt[NW * 256];
    __shared__ uint64_t base[256];
    const uint64_t m = *m_ptr;
    const uint32_t tile = blockIdx.x;
    const uint64_t t0 = (uint64_t)tile * RS_TILE;
    if (t0 >= m) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < NW * 256; i += blockDim.x) cnt[i] = 0;
    for (int d = threadIdx.x; d < 256; d += blockDim.x) base[d] = hist_off[(uint64_t)d * ntiles + tile];
    uint64_t key[RS_TILE_ITEMS];
    uint32_t val[RS_TILE_ITEMS];
    uint16_t loc[RS_TILE_ITEMS];
    bool ok[RS_TILE_ITEMS];
#pragma unroll
    for (int r = 0; r < RS_TILE_ITEMS; ++r) {
        const uint64_t i = t0 + warp * PER_WARP + r * 32 + lane;
        ok[r] = i < m;
        key[r] = ok[r] ? kin[i] : ~0ull;   // padding sorts last and is never written
        val[r] = ok[r] ? vin[i] : 0u;
    }
    __syncthreads();
    warp_rank<RS_TILE_ITEMS>(key, shift, cnt + warp * 256, loc);
    __syncthreads();
    if (threadIdx.x < 256) {
        const int d = threadIdx.x;
        uint32_t run = 0;
        for (int w = 0; w < NW; ++w) {
            const uint32_t t = cnt[w * 256 + d];
            cnt[w * 256 + d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_TILE_ITEMS; ++r) {
        if (!ok[r]) continue;
        const uint32_t d = digit_of(key[r], shift);
        const uint64_t o = base[d] + cnt[warp * 256 + d] + loc[r];
        kout[o] = key[r];
        vout[o] = val[r];
    }
}

// ---- 3. segments, neighbours, byte verification ----------------------------------
//
// One CTA scans the sorted keys: seg[i] = index of the first element of i's
// equal-hash run (an inclusive max-scan of "i if head else 0"), and the
// positions with an equal-hash predecessor are compacted into dups[].

constexpr int SEG_THREADS = 1024;

__global__ void __launch_bounds__(SEG_THREADS) dd_segments_kernel(const uint64_t *__restrict__ keys,
                                                                  uint64_t *__restrict__ misc,
                                                                  uint32_t *__restrict__ seg,
                                                                  uint32_t *__restrict__ dups) {
    __shared__ uint32_t wmax[32], wsum[32];
    __shared__ uint32_t carry_max, carry_sum;
    const uint64_t m = misc[0];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        carry_max = 0;
        carry_sum = 0;
    }
    __syncthreads();
    for (uint64_t b = 0; b < m; b += SEG_THREADS) {
        const uint64_t i = b + tid;
        uint32_t head_idx = 0, dup = 0;
        if (i < m) {
            const bool head = (i == 0) || sort_key(keys[i]) != sort_key(keys[i - 1]);
            head_idx = head ? (uint32_t)i : 0u;
            dup = head ? 0u : 1u;
        }
        uint32_t mx = head_idx, sm = dup;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, mx, o);
            uint32_t z = __shfl_up_sync(0xffffffffu, sm, o);
            if (lane >= o) {
                mx = y > mx ? y : mx;
                sm += z;
            }
        }
        if (lane == 31) {
            wmax[warp] = mx;
            wsum[warp] = sm;
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t a = wmax[lane], s = wsum[lane];
            uint32_t ai = a, si = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, ai, o);
                uint32_t z = __shfl_up_sync(0xffffffffu, si, o);
                if (lane >= o) {
                    ai = y > ai ? y : ai;
                    si += z;
                }
            }
            // exclusive over warps, combined with the carry of earlier chunks
            uint32_t ea = __shfl_up_sync(0xffffffffu, ai, 1);
            uint32_t es = si - s;
            if (lane == 0) ea = 0;
            wmax[lane] = ea > carry_max ? ea : carry_max;
            wsum[lane] = carry_sum + es;
        }
        __syncthreads();
        const uint32_t segv = mx > wmax[warp] ? mx : wmax[warp];
        const uint32_t dpos = wsum[warp] + sm - dup;
        if (i < m) {
            seg[i] = segv;
            if (dup) dups[dpos] = (uint32_t)i;
        }
        __syncthreads();
        if (tid == SEG_THREADS - 1) {
            carry_max = segv;
            carry_sum = dpos + dup;
        }
        __syncthreads();
    }
    if (tid == 0) misc[2] = carry_sum;
}

// Byte comparison of one 16 KiB piece of pages pa and pb by one warp; true
// if they differ there (or differ in length).
__device__ __forceinline__ bool warp_piece_differs(const Pages &pg, uint32_t pa, uint32_t pb, uint32_t piece) {
    const uint32_t lane = lane_id();
    const PageLoc a = locate(pg, pa);
    const PageLoc b = locate(pg, pb);
    if (a.len != b.len) return true;
    const uint64_t p0 = (uint64_t)piece * DD_PIECE;
    if (p0 >= a.len) return false;
    const uint64_t plen = a.len - p0 < DD_PIECE ? a.len - p0 : DD_PIECE;
    const uint8_t *x = a.ptr + p0, *y = b.ptr + p0;
    const uint64_t nvec = plen >> 4;
    bool diff = false;
    uint64_t v = lane;
    for (; v + 96 < nvec; v += 128) {
        uint4 a0 = ldg_stream(x + 16 * v), a1 = ldg_stream(x + 16 * (v + 32));
        uint4 a2 = ldg_stream(x + 16 * (v + 64)), a3 = ldg_stream(x + 16 * (v + 96));
        uint4 b0 = ldg_stream(y + 16 * v), b1 = ldg_stream(y + 16 * (v + 32));
        uint4 b2 = ldg_stream(y + 16 * (v + 64)), b3 = ldg_stream(y + 16 * (v + 96));
        diff |= (a0.x ^ b0.x) | (a0.y ^ b0.y) | (a0.z ^ b0.z) | (a0.w ^ b0.w);
        diff |= (a1.x ^ b1.x) | (a1.y ^ b1.y) | (a1.z ^ b1.z) | (a1.w ^ b1.w);
        diff |= (a2.x ^ b2.x) | (a2.y ^ b2.y) | (a2.z ^ b2.z) | (a2.w ^ b2.w);
        diff |= (a3.x ^ b3.x) | (a3.y ^ b3.y) | (a3.z ^ b3.z) | (a3.w ^ b3.w);
    }
    for (; v < nvec; v += 32) {
        uint4 a0 = ldg_stream(x + 16 * v), b0 = ldg_stream(y + 16 * v);
        diff |= (a0.x ^ b0.x) | (a0.y ^ b0.y) | (a0.z ^ b0.z) | (a0.w ^ b0.w);
    }
    for (uint64_t t = (nvec << 4) + lane; t < plen; t += 32) diff |= x[t] != y[t];
    return __any_sync(0xffffffffu, diff) != 0;
}

// Byte-compare sorted element i with element i-1, one 16 KiB piece per warp.
__global__ void __launch_bounds__(256) dd_verify_kernel(Pages pg, const uint32_t *__restrict__ vals,
                                                        const uint32_t *__restrict__ dups,
                                                        const uint64_t *__restrict__ misc,
                                                        uint32_t *__restrict__ neq) {
    const uint64_t ndup = misc[2];
    const uint32_t pieces = (pg.page + DD_PIECE - 1) / DD_PIECE;
    const uint64_t items = ndup * pieces;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t it = gw; it < items; it += nw) {
        const uint32_t i = dups[it / pieces];
        const uint32_t piece = (uint32_t)(it % pieces);
        if (warp_piece_differs(pg, vals[i], vals[i - 1], piece) && lane_id() == 0) neq[i] = 1;
    }
}

// Small path: byte-compare page dups[j] with its group's representative
// rep[dups[j]], one 16 KiB piece per warp; neq[j] = 1 where they differ.
__global__ void __launch_bounds__(256) dd_verify_rep_kernel(Pages pg, const uint32_t *__restrict__ dups,
                                                            const uint32_t *__restrict__ rep,
                                                            const uint64_t *__restrict__ misc,
                                                            uint32_t *__restrict__ neq) {
    const uint64_t ndup = misc[2];
    const uint32_t pieces = (pg.page + DD_PIECE - 1) / DD_PIECE;
    const uint64_t items = ndup * pieces;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t it = gw; it < items; it += nw) {
        const uint64_t j = it / pieces;
        const uint32_t p = dups[j];
        if (warp_piece_differs(pg, p, rep[p], (uint32_t)(it % pieces)) && lane_id() == 0) neq[j] = 1;
    }
}

// ---- 4. classes ------------------------------------------------------------------

// Mark segments holding an element that differs from its predecessor and
// list each such segment once.
__global__ void dd_bad_kernel(const uint32_t *__restrict__ dups, const uint32_t *__restrict__ neq,
                              const uint32_t *__restrict__ seg, uint64_t *__restrict__ misc,
                              uint32_t *__restrict__ bad, uint32_t *__restrict__ badlist) {
    const uint64_t ndup = misc[2];
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ndup; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = dups[j];
        if (neq[i]) {
            const uint32_t s = seg[i];
            if (atomicExch(&bad[s], 1u) == 0u) {
                const unsigned long long slot = atomicAdd(reinterpret_cast<unsigned long long *>(&misc[3]), 1ull);
                badlist[slot] = s;
            }
        }
    }
}

__global__ void dd_canon_kernel(const uint32_t *__restrict__ vals, const uint32_t *__restrict__ seg,
                                const uint32_t *__restrict__ bad, const uint64_t *__restrict__ misc,
                                uint32_t *__restrict__ canon) {
    const uint64_t m = misc[0];
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = seg[i];
        if (!bad[s]) canon[vals[i]] = vals[s];
    }
}

__device__ bool cta_pages_equal(const Pages &pg, uint32_t p, uint32_t q) {
    const PageLoc a = locate(pg, p), b = locate(pg, q);
    if (a.len != b.len) return false;
    bool diff = false;
    const uint64_t nvec = a.len >> 4;
    for (uint64_t v = threadIdx.x; v < nvec; v += blockDim.x) {
        const uint4 x = ldg_stream(a.ptr + 16 * v), y = ldg_stream(b.ptr + 16 * v);
        diff |= (x.x != y.x) | (x.y != y.y) | (x.z != y.z) | (x.w != y.w);
    }
    for (uint64_t t = (nvec << 4) + threadIdx.x; t < a.len; t += blockDim.x) diff |= a.ptr[t] != b.ptr[t];
    return __syncthreads_or(diff) == 0;
}

// Slow path: one CTA per listed segment assigns classes by direct comparison
// with the representatives found so far (pages visited in increasing id).
__global__ void __launch_bounds__(256) dd_slow_kernel(Pages pg, const uint32_t *__restrict__ vals,
                                                      const uint32_t *__restrict__ seg,
                                                      const uint32_t *__restrict__ badlist,
                                                      const uint64_t *__restrict__ misc,
                                                      uint32_t *__restrict__ reps, uint32_t *__restrict__ canon) {
    const uint64_t nbad = misc[3];
    const uint64_t m = misc[0];
    for (uint64_t b = blockIdx.x; b < nbad; b += gridDim.x) {
        const uint32_t s = badlist[b];
        uint32_t nrep = 0;
        for (uint64_t j = s; j < m && seg[j] == s; ++j) {
            const uint32_t pj = vals[j];
            uint32_t found = 0xffffffffu;
            for (uint32_t r = 0; r < nrep; ++r) {
                if (cta_pages_equal(pg, pj, reps[s + r])) {
                    found = reps[s + r];
                    break;
                }
            }
            if (threadIdx.x == 0) {
                if (found != 0xffffffffu) canon[pj] = found;
                else {
                    reps[s + nrep] = pj;
                    canon[pj] = pj;
                }
            }
            if (found == 0xffffffffu) ++nrep;
            __syncthreads();
        }
    }
}

// ---- 5. blobs and the page table ---------------------------------------------------

__global__ void dd_canonflag_kernel(const uint8_t *__restrict__ zero, const uint32_t *__restrict__ canon,
                                    uint64_t P, uint32_t *__restrict__ flags) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (uint64_t)gridDim.x * blockDim.x)
        flags[p] = (zero[p] == KC_PAGE_DATA && canon[p] == (uint32_t)p) ? 1u : 0u;
}

__global__ void dd_table_kernel(Pages pg, const uint8_t *__restrict__ zero, const uint32_t *__restrict__ canon,
                                const uint32_t *__restrict__ flags, const uint64_t *__restrict__ pos,
                                kc_page *__restrict__ table, uint32_t *__restrict__ blob_page) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < pg.npages;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const int a = region_of(pg.regions, pg.nregions, p);
        const uint64_t first = pg.regions[a].first;
        kc_page row;
        row.va_offset = (p - first) << pg.log2page;
        row.alloc_id = (uint32_t)a;
        const uint8_t z = zero[p];
        if (z == KC_PAGE_ZERO) row.blob = KC_BLOB_ZERO;
        else if (z == KC_PAGE_LOST) row.blob = KC_BLOB_LOST;
        else row.blob = (uint32_t)pos[canon[p]];
        table[p] = row;
        if (z == KC_PAGE_DATA && flags[p]) blob_page[pos[p]] = (uint32_t)p;
    }
}

// ---- small snapshots (P <= DD_SMALL pages) -------------------------------------
//
// The candidates for a page's class are the pages whose hashes share their
// low 32 bits (as in the sort of the large path).  The key space is split
// over DD_PARTS CTAs by its top bits; each CTA inserts its share of the data
// pages into an open-addressing table in shared memory keyed by those 32 bits
// (32-bit atomics), keeping the smallest page id of each key (the group's
// representative), so no sort is needed and the atomics of one SM handle a
// DD_PARTS-th of the pages.  Pages whose full hashes differ fail the byte
// comparison like any collision.  A page that is not its group's
// representative is listed for a byte comparison with it
// (dd_verify_rep_kernel); the list's order does not matter.  Each CTA also
// writes a slice of the page table as if every data page were canonical
// (blob ids = data pages numbered in page order, which every CTA can count
// from the zero flags alone); that is the table when no two data pages share
// a key.  Otherwise dd_small_finish_kernel rewrites it after the
// verification: a group whose members all equal the representative is one
// class, and a group with a failed comparison (a hash collision, or equal
// hashes of pages of different lengths) is split by direct comparison exactly
// as the class definition reads (members in increasing page id, each
// compared with the classes found so far).

constexpr int DD_SMALL = 8192;                              // pages
constexpr int DD_SMALL_THREADS = 1024;
constexpr int DD_SMALL_PER = DD_SMALL / DD_SMALL_THREADS;   // pages per thread, blocked
constexpr int DD_TABLE = 2 * DD_SMALL;                      // hash-table slots
constexpr uint32_t DD_EMPTY = 0xffffffffu;
constexpr int DD_PARTS = 8;                                 // CTAs of the grouping kernel
constexpr size_t DD_SMALL_SMEM = (size_t)DD_TABLE * 4 + (size_t)DD_TABLE * 4 + (size_t)DD_SMALL * 2;
constexpr size_t DD_FINISH_SMEM = (size_t)DD_SMALL * 4 * 4 + (size_t)DD_SMALL * 2 + (size_t)DD_SMALL;

// Region of each page of thread tid's blocked range, from a mark at each
// region's first page and a block-wide running max.  `mark` holds DD_SMALL
// u16 entries; ws 33 words.  Every thread calls it.
__device__ void small_regions(const Pages &pg, uint16_t *mark, uint32_t *ws, uint32_t (&reg)[DD_SMALL_PER]) {
    const int tid = threadIdx.x;
    for (int i = tid; i < DD_SMALL; i += blockDim.x) mark[i] = 0;
    __syncthreads();
    for (int a = tid; a < pg.nregions; a += blockDim.x) {
        const uint64_t f = pg.regions[a].first;
        if (f < (uint64_t)DD_SMALL) mark[f] = (uint16_t)a;   // every region holds at least one page
    }
    __syncthreads();
    uint32_t run = 0;
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) {
        const uint32_t m = mark[tid * DD_SMALL_PER + j];
        run = m > run ? m : run;
        reg[j] = run;
    }
    const uint32_t before = block_excl_max(run, ws);
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) reg[j] = reg[j] > before ? reg[j] : before;
}

// Blob ids (canonical data pages numbered in page order), the page table and
// blob_page.  canon_of(j) gives the canonical page of the thread's j-th
// (blocked) page.  Shared memory: bid (DD_SMALL u32) receives each
// canonical page's blob id, cano (DD_SMALL u32) each page's canonical page,
// regs (DD_SMALL u16) each page's region.  The ids are assigned over the
// blocked pages; the table rows are then written warp-striped, so that a
// warp's 16-byte stores are contiguous.
template <class CanonOf>
__device__ void small_table(const Pages &pg, const uint8_t *__restrict__ zero, const uint32_t (&reg)[DD_SMALL_PER],
                            CanonOf canon_of, uint32_t *bid, uint32_t *cano, uint16_t *regs, uint32_t *ws,
                            kc_page *__restrict__ table, uint32_t *__restrict__ blob_page,
                            uint64_t *__restrict__ misc, uint64_t *__restrict__ n_blobs_out) {
    const int tid = threadIdx.x;
    const uint32_t P = (uint32_t)pg.npages;
    uint32_t flags = 0, nloc = 0;
    // the thread's 8 zero flags in one load when the array is 8-byte aligned
    const bool whole = P >= (uint32_t)(tid + 1) * DD_SMALL_PER && (reinterpret_cast<uintptr_t>(zero) & 7) == 0;
    const uint64_t z8 = whole ? __ldg(reinterpret_cast<const unsigned long long *>(zero) + tid) : 0ull;
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) {
        const uint32_t p = tid * DD_SMALL_PER + j;
        const uint8_t z = whole ? (uint8_t)(z8 >> (8 * j)) : (p < P ? zero[p] : (uint8_t)KC_PAGE_ZERO);
        const uint32_t c = canon_of(j);
        if (p < P) {
            cano[p] = c;
            regs[p] = (uint16_t)reg[j];
        }
        const bool f = p < P && z == KC_PAGE_DATA && c == p;
        flags |= (uint32_t)f << j;
        nloc += f;
    }
    uint32_t nb = 0;
    uint32_t o = block_excl_sum(nloc, ws, &nb);
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) {
        if ((flags >> j) & 1) {
            const uint32_t p = tid * DD_SMALL_PER + j;
            bid[p] = o;
            blob_page[o] = p;
            ++o;
        }
    }
    __syncthreads();
    for (uint32_t p = tid; p < P; p += blockDim.x) {
        const uint8_t z = zero[p];
        const uint32_t r = regs[p];
        kc_page row;
        row.va_offset = (p - __ldg(&pg.regions[r].first)) << pg.log2page;
        row.alloc_id = r;
        row.blob = z == KC_PAGE_ZERO ? KC_BLOB_ZERO : z == KC_PAGE_LOST ? KC_BLOB_LOST : bid[cano[p]];
        table[p] = row;
    }
    if (tid == 0) {
        misc[1] = nb;
        if (n_blobs_out) *n_blobs_out = nb;
    }
}

__device__ __forceinline__ uint32_t dd_slot(uint32_t k) {
    return (k ^ (k >> 14) ^ (k >> 28)) & (DD_TABLE - 1);
}

// The CTA that owns a 32-bit key (its top bits).
__device__ __forceinline__ uint32_t dd_part(uint32_t k, uint32_t nparts) {
    return (uint32_t)(((uint64_t)k * nparts) >> 32);
}

// misc[2] (the count of listed pages) must be 0 at launch.
__global__ void __launch_bounds__(DD_SMALL_THREADS) dd_small_kernel(
    Pages pg, const uint64_t *__restrict__ hash, const uint8_t *__restrict__ zero, uint64_t *__restrict__ misc,
    uint32_t *__restrict__ rep_out, uint32_t *__restrict__ dups, uint32_t *__restrict__ neq,
    kc_page *__restrict__ table, uint32_t *__restrict__ blob_page, uint64_t *__restrict__ n_blobs_out) {
    extern __shared__ __align__(16) uint8_t sm[];
    uint32_t *tkey = reinterpret_cast<uint32_t *>(sm);                       // [DD_TABLE] low 32 hash bits
    uint32_t *tval = tkey + DD_TABLE;                                        // [DD_TABLE]
    __shared__ uint32_t ws[33];
    __shared__ uint32_t empty_min;   // smallest data page whose key equals the empty-slot marker
    __shared__ uint32_t dup_base;
    const int tid = threadIdx.x;
    const uint32_t P = (uint32_t)pg.npages;
    const uint32_t part = blockIdx.x, nparts = gridDim.x;

    for (int i = tid; i < DD_TABLE; i += blockDim.x) {
        tkey[i] = DD_EMPTY;
        tval[i] = 0xffffffffu;
    }
    if (tid == 0) empty_min = 0xffffffffu;

    // the thread's DD_SMALL_PER consecutive pages: keys and zero flags
    uint32_t h[DD_SMALL_PER];
    uint8_t zf[DD_SMALL_PER];
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) {   // all loads first: one memory round trip
        const uint32_t p = tid * DD_SMALL_PER + j;
        zf[j] = p < P ? __ldg(zero + p) : (uint8_t)KC_PAGE_ZERO;
        h[j] = p < P ? (uint32_t)__ldg(hash + p) : 0u;
    }
    uint32_t isdata = 0, mine = 0;
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) {
        const bool d = zf[j] == KC_PAGE_DATA;
        isdata |= (uint32_t)d << j;
        mine |= (uint32_t)(d && dd_part(h[j], nparts) == part) << j;
    }
    __syncthreads();   // table initialised

    // insert this CTA's keys: value = smallest page id with the key.  The
    // first insertion attempt of every page is issued at once; a taken slot
    // (another key) continues along the probe chain
    uint32_t prev[DD_SMALL_PER];
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) {
        prev[j] = DD_EMPTY;
        if (((mine >> j) & 1) && h[j] != DD_EMPTY) prev[j] = atomicCAS(&tkey[dd_slot(h[j])], DD_EMPTY, h[j]);
    }
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) {
        if (!((mine >> j) & 1)) continue;
        const uint32_t p = tid * DD_SMALL_PER + j;
        if (h[j] == DD_EMPTY) {
            atomicMin(&empty_min, p);
            continue;
        }
        uint32_t s = dd_slot(h[j]);
        if (prev[j] != DD_EMPTY && prev[j] != h[j]) {
            // at most DD_SMALL keys in DD_TABLE slots: a free or matching slot is always found
            for (uint32_t k = 1; k < DD_TABLE; ++k) {
                s = (s + 1) & (DD_TABLE - 1);
                const uint32_t q = atomicCAS(&tkey[s], DD_EMPTY, h[j]);
                if (q == DD_EMPTY || q == h[j]) break;
            }
        }
        atomicMin(&tval[s], p);
    }
    __syncthreads();
    // look up each of this CTA's pages' representative: the first probe of
    // every page is issued at once, the rest of a probe chain only on a miss
    uint32_t rep[DD_SMALL_PER], slot[DD_SMALL_PER], k0[DD_SMALL_PER];
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) {
        slot[j] = dd_slot(h[j]);
        k0[j] = ((mine >> j) & 1) ? tkey[slot[j]] : 0u;
    }
    uint32_t nd = 0;
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) {
        const uint32_t p = tid * DD_SMALL_PER + j;
        rep[j] = p;
        if (!((mine >> j) & 1)) continue;
        if (h[j] == DD_EMPTY) {
            rep[j] = empty_min;
        } else if (k0[j] == h[j]) {
            rep[j] = tval[slot[j]];
        } else {
            for (uint32_t s = (slot[j] + 1) & (DD_TABLE - 1), k = 1; k < DD_TABLE; s = (s + 1) & (DD_TABLE - 1), ++k) {
                if (tkey[s] == h[j]) {
                    rep[j] = tval[s];
                    break;
                }
            }
        }
        nd += rep[j] != p;
    }
    // pages to verify (appended at a CTA-wide offset) and each of this CTA's
    // data pages' representative
    uint32_t ndc = 0;
    uint32_t o = block_excl_sum(nd, ws, &ndc);   // (its barriers end the table's use)
    if (tid == 0)
        dup_base = ndc ? (uint32_t)atomicAdd(reinterpret_cast<unsigned long long *>(&misc[2]), (unsigned long long)ndc)
                       : 0u;
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) {
        if (!((mine >> j) & 1)) continue;
        const uint32_t p = tid * DD_SMALL_PER + j;
        rep_out[p] = rep[j];
    }

    // the table as if every data page were canonical: blob id = data pages
    // before it; this CTA writes the rows of its slice of pages.  The
    // regions' first pages go to the table's memory (every region holds a
    // page, so there are at most P <= DD_SMALL of them) for the page ->
    // region search.
    uint64_t *sfirst = reinterpret_cast<uint64_t *>(tval);
    for (int a = tid; a < pg.nregions; a += blockDim.x) sfirst[a] = __ldg(&pg.regions[a].first);
    uint32_t nb = 0;
    uint32_t r0 = block_excl_sum((uint32_t)__popc(isdata), ws, &nb);   // (its barriers publish dup_base, sfirst)
    o += dup_base;
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) {
        if (((mine >> j) & 1) && rep[j] != tid * DD_SMALL_PER + j) {
            dups[o] = tid * DD_SMALL_PER + j;
            neq[o] = 0;
            ++o;
        }
    }
    const uint32_t span = (P + nparts - 1) / nparts;
    const uint32_t lo = part * span < P ? part * span : P;
    const uint32_t hi = lo + span < P ? lo + span : P;
    uint32_t *bid = tkey;   // [DD_SMALL] blob id of each data page of the slice
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) {
        const uint32_t p = tid * DD_SMALL_PER + j;
        if (p >= lo && p < hi && ((isdata >> j) & 1)) {
            bid[p] = r0;
            blob_page[r0] = p;
        }
        r0 += (isdata >> j) & 1;
    }
    __syncthreads();
    for (uint32_t p = lo + tid; p < hi; p += blockDim.x) {
        const uint8_t z = zero[p];
        int rl = 0, rh = pg.nregions - 1;   // last region whose first page <= p
        while (rl < rh) {
            const int mid = (rl + rh + 1) >> 1;
            if (sfirst[mid] <= p) rl = mid;
            else rh = mid - 1;
        }
        kc_page row;
        row.va_offset = (p - sfirst[rl]) << pg.log2page;
        row.alloc_id = (uint32_t)rl;
        row.blob = z == KC_PAGE_ZERO ? KC_BLOB_ZERO : z == KC_PAGE_LOST ? KC_BLOB_LOST : bid[p];
        table[p] = row;
    }
    if (part == 0 && tid == 0) {
        misc[0] = P;
        misc[1] = nb;
        if (n_blobs_out) *n_blobs_out = nb;
    }
}

// After dd_verify_rep_kernel, when some data pages share a hash.  `classes`
// (P entries of scratch) holds, per failed group, the classes found so far.
__global__ void __launch_bounds__(DD_SMALL_THREADS) dd_small_finish_kernel(
    Pages pg, const uint8_t *__restrict__ zero, const uint32_t *__restrict__ rep, const uint32_t *__restrict__ dups,
    const uint32_t *__restrict__ neq, uint64_t *__restrict__ misc, uint32_t *__restrict__ classes,
    kc_page *__restrict__ table, uint32_t *__restrict__ blob_page, uint64_t *__restrict__ n_blobs_out) {
    const uint32_t ndup = (uint32_t)misc[2];
    if (ndup == 0) return;   // dd_small_kernel wrote everything
    extern __shared__ __align__(16) uint8_t sm[];
    uint32_t *canon = reinterpret_cast<uint32_t *>(sm);   // [DD_SMALL] per page
    uint32_t *order = canon + DD_SMALL;                   // [DD_SMALL] pages of failed groups; later blob ids
    uint32_t *seg = order + DD_SMALL;                     // [DD_SMALL] per group: member count, then first slot
    uint32_t *ncls = seg + DD_SMALL;                      // [DD_SMALL] per group: classes found so far
    uint16_t *mark = reinterpret_cast<uint16_t *>(ncls + DD_SMALL);   // [DD_SMALL]
    uint8_t *bad = reinterpret_cast<uint8_t *>(mark + DD_SMALL);      // [DD_SMALL] per representative
    __shared__ uint32_t ws[33];
    const int tid = threadIdx.x;
    const uint32_t P = (uint32_t)pg.npages;
    uint32_t reg[DD_SMALL_PER];
    for (uint32_t i = tid; i < DD_SMALL; i += blockDim.x) {
        bad[i] = 0;
        seg[i] = 0;
        ncls[i] = 0;
    }
    small_regions(pg, mark, ws, reg);   // (its barriers order the initialisation above)
    for (uint32_t j = tid; j < ndup; j += blockDim.x)
        if (neq[j]) bad[rep[dups[j]]] = 1;
    __syncthreads();
    // a page of a verified group: canonical = the representative
    uint32_t c[DD_SMALL_PER];
    uint32_t nslow = 0, slow = 0;
#pragma unroll
    for (int j = 0; j < DD_SMALL_PER; ++j) {
        const uint32_t p = tid * DD_SMALL_PER + j;
        c[j] = p;
        if (p < P && zero[p] == KC_PAGE_DATA) {
            c[j] = rep[p];
            if (bad[c[j]]) {
                slow |= 1u << j;
                ++nslow;
                atomicAdd(&seg[c[j]], 1u);
            }
        }
        if (p < P) canon[p] = c[j];
    }
    uint32_t total = 0;
    uint32_t o = block_excl_sum(nslow, ws, &total);   // (its barriers order the counts above)
    if (total) {
        // pages of failed groups in increasing id, and each group's slots in
        // `classes` (an exclusive scan of the member counts)
        uint32_t cnt[DD_SMALL_PER], sum = 0;
#pragma unroll
        for (int j = 0; j < DD_SMALL_PER; ++j) {
            if ((slow >> j) & 1) order[o++] = tid * DD_SMALL_PER + j;
            cnt[j] = seg[tid * DD_SMALL_PER + j];
            sum += cnt[j];
        }
        uint32_t at = block_excl_sum(sum, ws, nullptr);
#pragma unroll
        for (int j = 0; j < DD_SMALL_PER; ++j) {
            seg[tid * DD_SMALL_PER + j] = at;
            at += cnt[j];
        }
        __syncthreads();
        for (uint32_t k = 0; k < total; ++k) {   // rare: hash collisions only
            const uint32_t pj = order[k];
            const uint32_t g = rep[pj];
            const uint32_t base = seg[g], n = ncls[g];
            uint32_t found = 0xffffffffu;
            for (uint32_t r = 0; r < n; ++r) {
                const uint32_t q = classes[base + r];
                if (cta_pages_equal(pg, pj, q)) {
                    found = q;
                    break;
                }
            }
            if (tid == 0) {
                if (found != 0xffffffffu) {
                    canon[pj] = found;
                } else {
                    classes[base + n] = pj;
                    ncls[g] = n + 1;
                    canon[pj] = pj;
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int j = 0; j < DD_SMALL_PER; ++j) {
            const uint32_t p = tid * DD_SMALL_PER + j;
            if (p < P) c[j] = canon[p];
        }
        __syncthreads();
    }
    small_table(pg, zero, reg, [&](int j) { return c[j]; }, order, seg, mark, ws, table, blob_page, misc,
                n_blobs_out);
}

// ---- 6. pack ----------------------------------------------------------------------

__global__ void __launch_bounds__(256) dd_pack_kernel(Pages pg, const uint32_t *__restrict__ blob_page,
                                                      const uint64_t *__restrict__ misc, uint8_t *__restrict__ arena,
                                                      uint64_t arena_cap, uint32_t *__restrict__ status) {
    const uint64_t nb = misc[1];
    if ((uint64_t)pg.page * nb > arena_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(status, ST_TRUNC);
        return;
    }
    const uint32_t pieces = (pg.page + DD_PIECE - 1) / DD_PIECE;
    const uint64_t items = nb * pieces;
    const uint32_t lane = lane_id();
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t it = gw; it < items; it += nw) {
        const uint64_t b = it / pieces;
        const uint32_t piece = (uint32_t)(it - b * pieces);
        const PageLoc l = locate(pg, blob_page[b]);
        const uint64_t p0 = (uint64_t)piece * DD_PIECE;
        const uint64_t plen = pg.page - p0 < DD_PIECE ? pg.page - p0 : DD_PIECE;   // slot piece
        uint8_t *dst = arena + b * pg.page + p0;
        const uint64_t have = l.len > p0 ? (l.len - p0 < plen ? l.len - p0 : plen) : 0;   // source bytes
        const uint8_t *src = l.ptr + p0;
        const uint64_t nvec = have >> 4;
        uint64_t v = lane;
        for (; v + 96 < nvec; v += 128) {
            uint4 x0 = ldg_stream(src + 16 * v), x1 = ldg_stream(src + 16 * (v + 32));
            uint4 x2 = ldg_stream(src + 16 * (v + 64)), x3 = ldg_stream(src + 16 * (v + 96));
            *reinterpret_cast<uint4 *>(dst + 16 * v) = x0;
            *reinterpret_cast<uint4 *>(dst + 16 * (v + 32)) = x1;
            *reinterpret_cast<uint4 *>(dst + 16 * (v + 64)) = x2;
            *reinterpret_cast<uint4 *>(dst + 16 * (v + 96)) = x3;
        }
        for (; v < nvec; v += 32) *reinterpret_cast<uint4 *>(dst + 16 * v) = ldg_stream(src + 16 * v);
        // bytes [16*nvec, have) copied one by one, [have, plen) zero-filled
        const uint64_t z0 = (have + 15) & ~15ull;
        for (uint64_t t = (nvec << 4) + lane; t < z0 && t < plen; t += 32) dst[t] = t < have ? src[t] : 0;
        const uint4 zz = make_uint4(0, 0, 0, 0);
        for (uint64_t t = z0 + 16 * lane; t + 16 <= plen; t += 512) *reinterpret_cast<uint4 *>(dst + t) = zz;
    }
}

// ---- driver ------------------------------------------------------------------------

cudaError_t setup_dedup_kernels() {
    cudaError_t e = cudaFuncSetAttribute(dd_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)DD_SMALL_SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(dd_small_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)DD_FINISH_SMEM);
}

static inline unsigned grid_for(uint64_t n, int threads, int sms, int per_sm) {
    uint64_t b = (n + threads - 1) / threads;
    const uint64_t cap = (uint64_t)sms * per_sm;
    if (b > cap) b = cap;
    return (unsigned)(b ? b : 1);
}

#define KC_TRY(x)                                   \
    do {                                            \
        cudaError_t e_ = (x);                       \
        if (e_ != cudaSuccess) return e_;           \
    } while (0)

cudaError_t run_dedup(const Pages &pg, const uint64_t *hash, const uint8_t *zero, kc_page *table,
                      uint8_t *arena, uint64_t arena_cap, uint64_t *n_blobs, DedupScratch &s,
                      uint32_t *status, int sms, cudaStream_t st) {
    const uint64_t P = pg.npages;
    const unsigned g = grid_for(P, 256, sms, 8);
    const uint32_t pieces = (pg.page + DD_PIECE - 1) / DD_PIECE;
    if (P <= (uint64_t)DD_SMALL) {
        // small: grouping by shared-memory hash tables (the keys split over
        // DD_PARTS CTAs), the wide verification of pages sharing a key, and
        // (only when there were such pages) the classes and table in one CTA
        KC_TRY(cudaMemsetAsync(s.misc + 2, 0, 8, st));
        dd_small_kernel<<<DD_PARTS, DD_SMALL_THREADS, DD_SMALL_SMEM, st>>>(pg, hash, zero, s.misc, s.canon, s.dups,
                                                                           s.neq, table, s.blob_page, n_blobs);
        count_launches(1);
        KC_TRY(cudaGetLastError());
        dd_verify_rep_kernel<<<grid_for(P * pieces * 32, 256, sms, 8), 256, 0, st>>>(pg, s.dups, s.canon, s.misc,
                                                                                     s.neq);
        count_launches(1);
        KC_TRY(cudaGetLastError());
        dd_small_finish_kernel<<<1, DD_SMALL_THREADS, DD_FINISH_SMEM, st>>>(pg, zero, s.canon, s.dups, s.neq, s.misc,
                                                                            s.reps, table, s.blob_page, n_blobs);
        count_launches(1);
        KC_TRY(cudaGetLastError());
    } else {
    KC_TRY(cudaMemsetAsync(s.misc, 0, 64, st));
    KC_TRY(cudaMemsetAsync(s.neq, 0, P * 4, st));
    KC_TRY(cudaMemsetAsync(s.bad, 0, P * 4, st));
    // 1. compaction
    dd_flag_kernel<<<g, 256, 0, st>>>(zero, P, s.flags);
    count_launches(1);
    KC_TRY(cudaGetLastError());
    KC_TRY(launch_scan_u32(s.flags, s.pos, P, &s.misc[0], st));
    dd_compact_kernel<<<g, 256, 0, st>>>(hash, s.flags, s.pos, P, s.keys[0], s.vals[0]);
    count_launches(1);
    KC_TRY(cudaGetLastError());
    // 2. sort: tiled passes
    {
        const uint32_t ntiles = (uint32_t)ceil_div(P, RS_TILE);
        int src = 0;
        for (int shift = 0; shift < SORT_BITS; shift += 8) {
            rs_hist_kernel<<<ntiles, RS_TILE_THREADS, 0, st>>>(s.keys[src], &s.misc[0], shift, s.hist, ntiles);
            count_launches(1);
            KC_TRY(cudaGetLastError());
            KC_TRY(launch_scan_u32(s.hist, s.hist_off, 256ull * ntiles, nullptr, st));
            rs_scatter_kernel<<<ntiles, RS_TILE_THREADS, 0, st>>>(s.keys[src], s.vals[src], &s.misc[0], shift,
                                                                  s.hist_off, ntiles, s.keys[src ^ 1],
                                                                  s.vals[src ^ 1]);
            count_launches(1);
            KC_TRY(cudaGetLastError());
            src ^= 1;
        }
        // an even number of passes: the result is back in buffer 0
    }
    // 3. segments, neighbours, verification
    dd_segments_kernel<<<1, SEG_THREADS, 0, st>>>(s.keys[0], s.misc, s.seg, s.dups);
    count_launches(1);
    KC_TRY(cudaGetLastError());
    dd_verify_kernel<<<grid_for(P * pieces * 32, 256, sms, 8), 256, 0, st>>>(pg, s.vals[0], s.dups, s.misc, s.neq);
    count_launches(1);
    KC_TRY(cudaGetLastError());
    // 4. classes
    dd_bad_kernel<<<g, 256, 0, st>>>(s.dups, s.neq, s.seg, s.misc, s.bad, s.flags);
    count_launches(1);
    KC_TRY(cudaGetLastError());
    dd_canon_kernel<<<g, 256, 0, st>>>(s.vals[0], s.seg, s.bad, s.misc, s.canon);
    count_launches(1);
    KC_TRY(cudaGetLastError());
    dd_slow_kernel<<<(unsigned)sms, 256, 0, st>>>(pg, s.vals[0], s.seg, s.flags, s.misc, s.reps, s.canon);
    count_launches(1);
    KC_TRY(cudaGetLastError());
    // 5. blobs and table
    dd_canonflag_kernel<<<g, 256, 0, st>>>(zero, s.canon, P, s.flags);
    count_launches(1);
    KC_TRY(cudaGetLastError());
    KC_TRY(launch_scan_u32(s.flags, s.pos, P, &s.misc[1], st));
    dd_table_kernel<<<g, 256, 0, st>>>(pg, zero, s.canon, s.flags, s.pos, table, s.blob_page);
    count_launches(1);
    KC_TRY(cudaGetLastError());
    if (n_blobs) KC_TRY(cudaMemcpyAsync(n_blobs, &s.misc[1], 8, cudaMemcpyDeviceToDevice, st));
    }
    // 6. pack
    if (arena) {
        dd_pack_kernel<<<grid_for(P * pieces * 32, 256, sms, 8), 256, 0, st>>>(pg, s.blob_page, s.misc, arena,
                                                                               arena_cap, status);
        count_launches(1);
        KC_TRY(cudaGetLastError());
    }
    return cudaSuccess;
}

}  // namespace kc
