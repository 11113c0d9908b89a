// k_digest.cu -- page digest (XXH64 seed 0 + zero flag), optionally fused
// with the pointer-census pre-filter, and the census count / write / scan
// kernels.
//
// Digest mapping.  XXH64 keeps four serial accumulators, one per 8-byte lane
// of every 32-byte stripe, so one page is hashed by a quad of four threads
// (thread k owns accumulator k).  A warp hashes eight pages at once (one per
// quad) and takes its next eight pages from a global ticket counter, so
// warps that finish early steal the remaining work.  Each warp owns a ring of
// `stages` shared-memory stages; a stage holds one `chunk` of each of its
// pages.  The threads of a page copy its chunk with per-thread 16-byte
// asynchronous copies (cp.async), one commit group per stage, and wait for
// the group before hashing it.  (One bulk TMA copy per page per stage moves
// the same bytes, but issuing eight of them per chunk stalled the issuing
// warp for ~900 cycles -- time it could not spend hashing -- while the
// per-thread copies never block.)  Page slots are padded by 32 bytes so the
// eight pages' shared loads spread over all 32 banks.  The < 32-byte tail of
// a page is read from global memory by the page leader while it finishes the
// hash.
//
// The serial chain per accumulator is the critical path: each step is an
// add, a rotate and a multiply by PRIME1 (xx_step); the lane products
// (lane * PRIME2) and the next stripes' shared loads are issued ahead of it.
//
// Census when fused: the hashing loop only keeps, per page, the minimum of
// (high 32 bits of a word - pre_lo), a branch-free conservative test of
// whether any word can be a hit.  Pages that pass are classified afterwards
// by census_flagged_kernel, one word per lane, so a pointer-dense page never
// holds up the hashing warps.
#include <cuda_runtime.h>

#include "kc_device.cuh"
#include "kc_internal.cuh"

namespace kc {

// page_hits value of a page whose words must still be classified
constexpr uint32_t HITS_PENDING = 0xFFFFFFFFu;

size_t digest_smem_bytes(const DigestShape &s) {
    const size_t ppw = 8 * (size_t)(s.lanes == 2 ? 2 : 1);
    return (size_t)s.warps * s.stages * ppw * (size_t)(s.chunk + 32);
}

// CHUNK = the chunk size as a compile-time constant (0: runtime only); full
// chunks of that size take a fully unrolled path.
// LPT = XXH64 lanes per thread.  LPT = 1: four threads per page (8 pages per
// warp), the most parallel layout, for few pages.  LPT = 2: two threads per
// page, each owning two adjacent lanes (one 16-byte shared load per stripe
// feeds two independent chains), 16 pages per warp: half the instructions
// per byte and twice the instruction-level parallelism, for many pages.
template <bool CENSUS, int LPT, int CHUNK>
__global__ void __launch_bounds__(512) digest_kernel(Pages pg, CensusArgs ca, uint64_t *__restrict__ hash,
                                                     uint8_t *__restrict__ zero,
                                                     uint32_t *__restrict__ page_hits,
                                                     uint32_t *__restrict__ task_ctr,
                                                     uint32_t *__restrict__ status, int stages, int chunk) {
    constexpr int TPP = 4 / LPT;    // threads per page
    constexpr int PPW = 32 / TPP;   // pages per warp task
    extern __shared__ __align__(128) uint8_t smem[];
    (void)status;                   // no waits here can time out: cp.async groups always complete
    const int warp = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    const int q = lane / TPP;       // page slot of this thread
    const int j = lane % TPP;       // this thread owns lanes j*LPT .. j*LPT+LPT-1
    const uint32_t FULL = 0xffffffffu;

    const size_t slot_stride = (size_t)chunk + 32;
    const size_t stage_stride = PPW * slot_stride;
    uint8_t *ring = smem + (size_t)warp * stages * stage_stride;

    while (true) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(task_ctr, 1u);
        t = __shfl_sync(FULL, t, 0);
        const uint64_t p0 = (uint64_t)t * PPW;
        if (p0 >= pg.npages) break;
        const uint64_t p = p0 + q;
        const bool valid = p < pg.npages;

        const uint8_t *src = nullptr;
        uint64_t len = 0;
        bool lost = false;
        if (valid) {
            const int region = region_of(pg.regions, pg.nregions, p);
            const Region r = pg.regions[region];
            const uint64_t off = (p - r.first) << pg.log2page;
            len = r.bytes - off < pg.page ? r.bytes - off : pg.page;
            src = reinterpret_cast<const uint8_t *>(r.base + off);
            lost = r.lost != 0;
        }
        const uint32_t sbytes = lost ? 0u : (uint32_t)(len & ~31ull);   // bytes in full stripes
        const uint32_t nch = (sbytes + chunk - 1) / chunk;
        const uint32_t maxch = __reduce_max_sync(FULL, nch);

        // Copy chunk c of this thread's page into stage c % stages: the
        // page's threads split its 16-byte pieces.  Every thread commits one
        // group per call (empty past the page's end), so group counts agree.
        auto issue = [&](uint32_t c) {
            if (c < nch) {
                const uint32_t rest = sbytes - c * chunk;
                const uint32_t b = rest < (uint32_t)chunk ? rest : (uint32_t)chunk;
                uint8_t *dst = ring + (c % stages) * stage_stride + q * slot_stride;
                const uint8_t *from = src + (size_t)c * chunk;
                for (uint32_t o = 16 * j; o < b; o += 16 * TPP) cp_async16(dst + o, from + o);
            }
            cp_async_commit();
        };
        for (int c = 0; c < stages - 1; ++c) issue((uint32_t)c);

        uint64_t acc[LPT];
#pragma unroll
        for (int i = 0; i < LPT; ++i) acc[i] = xx_init(j * LPT + i);
        uint32_t zlo = 0, zhi = 0;
        uint32_t cmin = 0xFFFFFFFFu;   // census pre-filter, minimum over the page
        for (uint32_t c = 0; c < maxch; ++c) {
            issue(c + stages - 1);        // refills the stage consumed in the previous iteration
            cp_async_wait(stages - 1);    // this thread's pieces of chunk c have landed
            __syncwarp();                 // ... and so have those of the page's other threads
            const int st = (int)(c % stages);
            uint32_t b = 0;
            if (c < nch) {
                const uint32_t rest = sbytes - c * chunk;
                b = rest < (uint32_t)chunk ? rest : (uint32_t)chunk;
            }
            const uint8_t *slot = ring + st * stage_stride + q * slot_stride + 8 * LPT * j;
            // one load per stripe: LPT consecutive 8-byte lanes
            auto ld = [&](uint32_t off, uint64_t (&w)[LPT]) {
                if (LPT == 1) {
                    w[0] = *reinterpret_cast<const uint64_t *>(slot + off);
                } else {
                    const uint4 v = *reinterpret_cast<const uint4 *>(slot + off);
                    w[0] = ((uint64_t)v.y << 32) | v.x;
                    w[LPT - 1] = ((uint64_t)v.w << 32) | v.z;
                }
            };
            auto eat = [&](const uint64_t (&w)[LPT]) {
#pragma unroll
                for (int i = 0; i < LPT; ++i) {
                    zlo |= (uint32_t)w[i];
                    zhi |= (uint32_t)(w[i] >> 32);
                    if (CENSUS) cmin = min(cmin, census_pre(ca, w[i]));
                }
            };
            uint32_t s = 0;
            if (CHUNK && b == (uint32_t)CHUNK) {
                // a full chunk of compile-time size: fully unrolled, the
                // loads of all its stripes issued ahead of the chains
                uint64_t w[4][LPT];
#pragma unroll
                for (int u = 0; u < 4; ++u) ld(32 * u, w[u]);
#pragma unroll
                for (int g = 0; g < CHUNK / 128; ++g) {
                    uint64_t nw[4][LPT];
                    if (g + 1 < CHUNK / 128) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) ld(128 * (g + 1) + 32 * u, nw[u]);
                    }
                    uint64_t m[4][LPT];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int i = 0; i < LPT; ++i) m[u][i] = w[u][i] * XXP2;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int i = 0; i < LPT; ++i) acc[i] = xx_step(acc[i], m[u][i]);
#pragma unroll
                    for (int u = 0; u < 4; ++u) eat(w[u]);
                    if (g + 1 < CHUNK / 128) {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
#pragma unroll
                            for (int i = 0; i < LPT; ++i) w[u][i] = nw[u][i];
                    }
                }
                s = b;
            } else if (b >= 128) {
                // register double buffer: the next four stripes are loaded
                // while the current four run through the chains
                uint64_t w[4][LPT];
#pragma unroll
                for (int u = 0; u < 4; ++u) ld(32 * u, w[u]);
                for (; s + 128 <= b; s += 128) {
                    const uint32_t ns = (s + 256 <= b) ? s + 128 : s;   // last group reloads itself
                    uint64_t nw[4][LPT];
#pragma unroll
                    for (int u = 0; u < 4; ++u) ld(ns + 32 * u, nw[u]);
                    uint64_t m[4][LPT];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int i = 0; i < LPT; ++i) m[u][i] = w[u][i] * XXP2;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int i = 0; i < LPT; ++i) acc[i] = xx_step(acc[i], m[u][i]);
#pragma unroll
                    for (int u = 0; u < 4; ++u) eat(w[u]);
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int i = 0; i < LPT; ++i) w[u][i] = nw[u][i];
                }
            }
            for (; s < b; s += 32) {
                uint64_t w[LPT];
                ld(s, w);
#pragma unroll
                for (int i = 0; i < LPT; ++i) acc[i] = xx_step(acc[i], w[i] * XXP2);
                eat(w);
            }
            __syncwarp();                 // the stage is free for the next refill
        }
        cp_async_wait(0);                 // trailing (empty) groups

        // Page reduction: accumulators to the page leader, OR of bytes, census flag.
        const int lead = lane - j;
        uint64_t a[4];
        if (LPT == 1) {
            a[0] = acc[0];
#pragma unroll
            for (int i = 1; i < 4; ++i) a[i] = __shfl_sync(FULL, acc[0], lead + i);
        } else {
            a[0] = acc[0];
            a[1] = acc[LPT - 1];
            a[2] = __shfl_sync(FULL, acc[0], lead + 1);
            a[3] = __shfl_sync(FULL, acc[LPT - 1], lead + 1);
        }
        uint64_t zor = ((uint64_t)zhi << 32) | zlo;
#pragma unroll
        for (int o = 1; o < TPP; o <<= 1) {
            zor |= __shfl_xor_sync(FULL, zor, o);
            if (CENSUS) cmin = min(cmin, __shfl_xor_sync(FULL, cmin, o));
        }
        if (j == 0 && valid) {
            if (lost) {
                hash[p] = 0;
                zero[p] = KC_PAGE_LOST;
                if (CENSUS) page_hits[p] = 0;
            } else {
                uint64_t h;
                if (len >= 32) {
                    h = rotl(a[0], 1) + rotl(a[1], 7) + rotl(a[2], 12) + rotl(a[3], 18);
#pragma unroll
                    for (int i = 0; i < 4; ++i) h = (h ^ xx_round(0, a[i])) * XXP1 + XXP4;
                } else {
                    h = XXP5;
                }
                h += len;
                const uint8_t *tp = src + sbytes;
                uint32_t rem = (uint32_t)(len - sbytes);
                while (rem >= 8) {
                    const uint64_t w = ldg_u64(tp);
                    h ^= xx_round(0, w);
                    h = rotl(h, 27) * XXP1 + XXP4;
                    zor |= w;
                    if (CENSUS) cmin = min(cmin, census_pre(ca, w));
                    tp += 8;
                    rem -= 8;
                }
                if (rem >= 4) {
                    const uint32_t w = __ldg(reinterpret_cast<const unsigned int *>(tp));
                    h ^= (uint64_t)w * XXP1;
                    h = rotl(h, 23) * XXP2 + XXP3;
                    zor |= w;
                    tp += 4;
                    rem -= 4;
                }
                while (rem) {
                    const uint32_t bb = __ldg(tp);
                    h ^= (uint64_t)bb * XXP5;
                    h = rotl(h, 11) * XXP1;
                    zor |= bb;
                    ++tp;
                    --rem;
                }
                h ^= h >> 33;
                h *= XXP2;
                h ^= h >> 29;
                h *= XXP3;
                h ^= h >> 32;
                hash[p] = h;
                zero[p] = zor == 0 ? KC_PAGE_ZERO : KC_PAGE_DATA;
                if (CENSUS) page_hits[p] = (cmin <= ca.pre_span && len >= 8) ? HITS_PENDING : 0u;
            }
        }
    }
}

template <bool CENSUS, int LPT, int CHUNK>
static cudaError_t setup_one() {
    return cudaFuncSetAttribute(digest_kernel<CENSUS, LPT, CHUNK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                227 * 1024);
}

template <bool CENSUS, int LPT>
static cudaError_t setup_lanes() {
    cudaError_t e;
    if ((e = setup_one<CENSUS, LPT, 0>())) return e;
    if ((e = setup_one<CENSUS, LPT, 512>())) return e;
    return setup_one<CENSUS, LPT, 1024>();
}

cudaError_t setup_digest_kernels() {
    cudaError_t e;
    if ((e = setup_lanes<true, 1>())) return e;
    if ((e = setup_lanes<true, 2>())) return e;
    if ((e = setup_lanes<false, 1>())) return e;
    return setup_lanes<false, 2>();
}

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

// Count the hits of every unit whose page_hits entry is HITS_PENDING.
__global__ void __launch_bounds__(CENSUS_THREADS) census_flagged_kernel(Pages u, CensusArgs ca,
                                                                         uint32_t *__restrict__ unit_hits,
                                                                         uint64_t *__restrict__ counts) {
    __shared__ Range srg[SMEM_RANGES];
    __shared__ uint32_t red_in[CENSUS_WARPS], red_out[CENSUS_WARPS];
    const Range *rg = stage_ranges(ca, srg);
    const int warp = threadIdx.x >> 5;
    for (uint64_t unit = blockIdx.x; unit < u.npages; unit += gridDim.x) {
        if (unit_hits[unit] != HITS_PENDING) continue;   // uniform across the CTA
        const UnitSpan sp = unit_span(u, unit);
        const uint64_t per = (sp.nwords + CENSUS_WARPS - 1) / CENSUS_WARPS;
        const uint64_t wb = per * warp, we = wb + per < sp.nwords ? wb + per : sp.nwords;
        uint32_t nin = 0, nout = 0;
        if (wb < we) warp_census_range(ca, rg, sp.base, wb, we, sp.off, (uint32_t)sp.region, nullptr, 0, 0, nin, nout);
        if (lane_id() == 0) {
            red_in[warp] = nin;
            red_out[warp] = nout;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t si = 0, so = 0;
            for (int w = 0; w < CENSUS_WARPS; ++w) {
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

cudaError_t launch_census_flagged(const Pages &units, const CensusArgs &ca, uint32_t *unit_hits, uint64_t *counts,
                                  int sms, cudaStream_t st) {
    uint64_t blocks = units.npages;
    const uint64_t maxb = (uint64_t)sms * 8;
    if (blocks > maxb) blocks = maxb;
    if (blocks == 0) return cudaSuccess;
    census_flagged_kernel<<<(unsigned)blocks, CENSUS_THREADS, 0, st>>>(units, ca, unit_hits, counts);
    count_launches(1);
    return cudaGetLastError();
}

template <bool CENSUS, int LPT>
static void launch_lanes(dim3 grid, dim3 block, size_t smem, cudaStream_t st, const Pages &pg, const CensusArgs &ca,
                         uint64_t *hash, uint8_t *zero, uint32_t *page_hits, uint32_t *task_ctr, uint32_t *status,
                         const DigestShape &shape) {
    switch (shape.chunk) {
    case 512:
        digest_kernel<CENSUS, LPT, 512><<<grid, block, smem, st>>>(pg, ca, hash, zero, page_hits, task_ctr, status,
                                                                   shape.stages, shape.chunk);
        break;
    case 1024:
        digest_kernel<CENSUS, LPT, 1024><<<grid, block, smem, st>>>(pg, ca, hash, zero, page_hits, task_ctr, status,
                                                                    shape.stages, shape.chunk);
        break;
    default:
        digest_kernel<CENSUS, LPT, 0><<<grid, block, smem, st>>>(pg, ca, hash, zero, page_hits, task_ctr, status,
                                                                 shape.stages, shape.chunk);
    }
}

cudaError_t launch_digest(const Pages &pg, const CensusArgs *census, uint64_t *hash, uint8_t *zero,
                          uint32_t *page_hits, uint64_t *counts, uint32_t *task_ctr, uint32_t *status,
                          const DigestShape &shape, cudaStream_t st) {
    (void)counts;
    const size_t smem = digest_smem_bytes(shape);
    const dim3 block(32 * shape.warps), grid(shape.ctas);
    CensusArgs none{};
    if (census && shape.lanes == 2)
        launch_lanes<true, 2>(grid, block, smem, st, pg, *census, hash, zero, page_hits, task_ctr, status, shape);
    else if (census)
        launch_lanes<true, 1>(grid, block, smem, st, pg, *census, hash, zero, page_hits, task_ctr, status, shape);
    else if (shape.lanes == 2)
        launch_lanes<false, 2>(grid, block, smem, st, pg, none, hash, zero, nullptr, task_ctr, status, shape);
    else
        launch_lanes<false, 1>(grid, block, smem, st, pg, none, hash, zero, nullptr, task_ctr, status, shape);
    count_launches(1);
    return cudaGetLastError();
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

}  // namespace kc
