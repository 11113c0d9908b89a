// k_digest.cu -- the page digest kernel (XXH64 seed 0 + zero flag, optionally
// with the census pre-filter flag per page; hashing in digest_task.cuh) and
// the census kernels: classification of flagged pages, the standalone count
// pass, the ordered write pass, and a single-CTA scan.
#include <cuda_runtime.h>

#include "digest_task.cuh"
#include "kc_device.cuh"
#include "kc_internal.cuh"

namespace kc {

// page_hits value of a page whose words must still be classified
constexpr uint32_t HITS_PENDING = 0xFFFFFFFFu;

size_t digest_smem_bytes(const DigestShape &s) {
    const size_t ppw = 8 * (size_t)(s.lanes == 2 ? 2 : 1);
    return (size_t)s.warps * s.stages * ppw * (size_t)(s.chunk + 32);
}

// One warp per task of PPW consecutive pages (8 with one XXH64 lane per
// thread, 16 with two), tasks taken from a global ticket counter so warps
// that finish early steal the rest; see digest_task.cuh for the hashing.
template <bool CENSUS, int LPT, int CHUNK>
__global__ void __launch_bounds__(512) digest_kernel(Pages pg, CensusArgs ca, uint64_t *__restrict__ hash,
                                                     uint8_t *__restrict__ zero,
                                                     uint32_t *__restrict__ page_hits,
                                                     uint32_t *__restrict__ task_ctr,
                                                     uint32_t *__restrict__ status, int stages, int chunk) {
    constexpr int TPP = 4 / LPT;
    constexpr int PPW = 32 / TPP;
    extern __shared__ __align__(128) uint8_t smem[];
    (void)status;   // no waits here can time out: cp.async groups always complete
    const int warp = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    uint8_t *ring = smem + (size_t)warp * stages * PPW * ((size_t)chunk + 32);
    while (true) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(task_ctr, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        const uint64_t p0 = (uint64_t)t * PPW;
        if (p0 >= pg.npages) break;
        const uint64_t p = p0 + lane / TPP;
        const bool valid = p < pg.npages;
        const uint8_t *src = nullptr;
        uint64_t len = 0;
        bool lost = false;
        if (valid) {
            const Region r = pg.regions[region_of(pg.regions, pg.nregions, p)];
            const uint64_t off = (p - r.first) << pg.log2page;
            len = r.bytes - off < pg.page ? r.bytes - off : pg.page;
            src = reinterpret_cast<const uint8_t *>(r.base + off);
            lost = r.lost != 0;
        }
        const PageDigest d = digest_pages<CENSUS, LPT, CHUNK>(ring, stages, chunk, src, len, lost, ca);
        if (lane % TPP == 0 && valid) {
            if (lost) {
                hash[p] = 0;
                zero[p] = KC_PAGE_LOST;
                if (CENSUS) page_hits[p] = 0;
            } else {
                hash[p] = d.hash;
                zero[p] = d.zero ? KC_PAGE_ZERO : KC_PAGE_DATA;
                if (CENSUS) page_hits[p] = d.cand ? HITS_PENDING : 0u;
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
