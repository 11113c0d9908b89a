// k_batch.cu -- the batched form: one persistent, work-stealing launch over
// many jobs of uneven sizes, replacing one launch per buffer per operation.
//
// The work of a launch is a list of ranges (a job's pages to digest, its
// comparison items, or its pages to digest and compare in one pass),
// flattened into one item space: a digest or fused item is one 8-page task,
// a comparison item is 64 KiB of a (got, want) pair.  Every warp
// takes its next item from a global ticket counter (work stealing) and runs
// the same device code as the single-operation kernels (digest_task.cuh,
// compare_tile.cuh), so results are identical to them.  A digest item
// writes the job's per-page outputs; a comparison item merges into the job's
// record with order-independent atomics, so a job split over many items --
// or over many launches, as a serving loop does -- gives the same result.
// The host orders the ranges (largest jobs first) and the launch needs no
// host work once its tables are cached, so it can be captured in a CUDA
// graph.
#include <cuda_runtime.h>

#include "compare_tile.cuh"
#include "digest_task.cuh"
#include "kc_internal.cuh"

namespace kc {

constexpr int BATCH_PPW = 8;   // pages per digest item (one XXH64 lane per thread)
constexpr uint32_t BATCH_QCAP = 64;                   // fused items: queued differing elements per warp
constexpr size_t BATCH_QBYTES = 16 + BATCH_QCAP * 16; // count, then SlowItems

// Per launch: comparison records of jobs that start here, the per-job
// count of unfinished items, and the completion flag of jobs with no item.
__global__ void batch_init_kernel(const BatchJob *__restrict__ jobs, int njobs, uint32_t *__restrict__ left) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= njobs) return;
    const BatchJob J = jobs[i];
    if ((J.flags & BJ_COMPARE) && (J.flags & BJ_INIT)) cmp_record_init(J.cmp, (J.flags & BJ_LOST) ? KC_EBUF : KC_OK);
    left[i] = J.items;
    if (J.done && J.items == 0) {
        if (J.cmp_copy && (J.flags & BJ_COMPARE)) *J.cmp_copy = *J.cmp;
        __threadfence_system();
        *reinterpret_cast<volatile uint32_t *>(J.done) = 1u;
    }
}

// Called by every lane of a warp after it finished one item of job J.  The
// warp's outputs are fenced at system scope before the job's count drops;
// the warp that takes it to zero copies the record (if asked) and sets the
// flag, so a host that sees the flag sees every output of the job.
__device__ __forceinline__ void batch_item_done(const BatchJob &J, uint32_t *left) {
    __threadfence_system();
    __syncwarp();
    if (lane_id() != 0) return;
    if (atomicSub(left, 1u) != 1u) return;
    __threadfence_system();
    if (J.cmp_copy && (J.flags & BJ_COMPARE)) {
        const volatile unsigned long long *from = reinterpret_cast<const volatile unsigned long long *>(J.cmp);
        volatile unsigned long long *to = reinterpret_cast<volatile unsigned long long *>(J.cmp_copy);
#pragma unroll
        for (int k = 0; k < (int)(sizeof(kc_cmp_result) / 8); ++k) to[k] = from[k];
    }
    __threadfence_system();
    *reinterpret_cast<volatile uint32_t *>(J.done) = 1u;
}

// ---- fused item: digest and compare of the same 8 pages, got read once -------
//
// The warp's ring stages hold, per page, one chunk of got (hashed, as in
// digest_pages) and the same chunk of want; after hashing a stage the warp
// compares it from shared memory, 16 bytes per lane, so got crosses HBM
// once for both operations.  A page's < 32-byte end (only the job's last
// page has one) is compared from global memory.  Differing elements go to
// the warp's queue (evaluated at the end of the item with every lane busy)
// or, when it is full, are evaluated where they are.

// Stage st's chunk c of the 8 pages: page r's got bytes at gslot(r), want
// bytes one half-stage later; br = that page's bytes in this chunk.
// With a compile-time chunk of at most 512 bytes every lane takes at most one
// vector of each page: no loop.
template <int DT, int CHUNK>
__device__ __forceinline__ void fused_cmp_stage(const uint8_t *stage, size_t slot_stride, uint32_t b, uint64_t off0,
                                                uint32_t log2page, uint32_t chunk_off, double atol, double rtol,
                                                CmpAcc &acc, const SlowQ &q) {
    constexpr uint64_t ES = esize<DT>();
    const uint32_t lane = lane_id();
#pragma unroll 1
    for (int r = 0; r < BATCH_PPW; ++r) {
        const uint32_t br = __shfl_sync(0xffffffffu, b, 4 * r);   // from the page's leader
        const uint8_t *gs = stage + (size_t)r * slot_stride;
        const uint8_t *ws = gs + BATCH_PPW * slot_stride;
        const uint64_t byte0 = off0 + ((uint64_t)r << log2page) + chunk_off;
        if (CHUNK > 0 && CHUNK <= 512) {
            if (lane < br / 16)
                cmp_vec<DT>(*reinterpret_cast<const uint4 *>(gs + 16 * lane),
                            *reinterpret_cast<const uint4 *>(ws + 16 * lane), (byte0 + 16 * lane) / ES, atol, rtol,
                            acc, q);
        } else {
            for (uint32_t i = lane; i < br / 16; i += 32)
                cmp_vec<DT>(*reinterpret_cast<const uint4 *>(gs + 16 * i),
                            *reinterpret_cast<const uint4 *>(ws + 16 * i), (byte0 + 16 * i) / ES, atol, rtol, acc, q);
        }
    }
}

template <int DT>
__device__ __forceinline__ void fused_cmp_tails(const BatchJob &J, uint64_t len, uint64_t off0, uint32_t log2page,
                                                double atol, double rtol, CmpAcc &acc, const SlowQ &q) {
    constexpr uint32_t ES = esize<DT>();
    const uint32_t lane = lane_id();
    const uint32_t tl = (uint32_t)(len & 31);
#pragma unroll 1
    for (int r = 0; r < BATCH_PPW; ++r) {
        const uint32_t t = __shfl_sync(0xffffffffu, tl, 4 * r);
        if (t == 0) continue;
        const uint64_t lr = ((uint64_t)__shfl_sync(0xffffffffu, (uint32_t)(len >> 32), 4 * r) << 32) |
                            __shfl_sync(0xffffffffu, (uint32_t)len, 4 * r);
        const uint64_t b = off0 + ((uint64_t)r << log2page) + (lr & ~31ull) + (uint64_t)lane * ES;
        if (lane * ES >= t) continue;
        const uint8_t *g = reinterpret_cast<const uint8_t *>(J.got) + b;
        const uint8_t *w = reinterpret_cast<const uint8_t *>(J.want) + b;
        uint32_t gb = 0, wb = 0;
        for (uint32_t k = 0; k < ES; ++k) {
            gb |= (uint32_t)g[k] << (8 * k);
            wb |= (uint32_t)w[k] << (8 * k);
        }
        if (gb == wb) {
            const uint32_t n = bits_nan<DT>(gb);
            acc.nan_g += n;
            acc.nan_w += n;
        } else {
            cmp_defer<DT>(q, gb, wb, b / ES, atol, rtol, acc);
        }
    }
}

// All 32 lanes call this, each with its page (src / wsrc / len, len 0 for a
// slot without a page); off0: byte offset in the job of the item's first
// page.  The digest result is valid in the page leader; the comparison is
// accumulated into acc (every lane).
template <int CHUNK>
__device__ __forceinline__ PageDigest fused_pages(uint8_t *ring, int stages, int chunk, const uint8_t *src,
                                                  const uint8_t *wsrc, uint64_t len, const BatchJob &J, uint64_t off0,
                                                  uint32_t log2page, double atol, double rtol, CmpAcc &acc,
                                                  const SlowQ &q) {
    const uint32_t FULL = 0xffffffffu;
    const uint32_t lane = lane_id();
    const int qs = lane / 4;        // page slot
    const int j = lane % 4;         // XXH64 lane of this thread
    const size_t slot_stride = (size_t)chunk + 32;
    const size_t stage_stride = 2 * BATCH_PPW * slot_stride;
    const uint32_t sbytes = (uint32_t)(len & ~31ull);
    const uint32_t nch = (sbytes + chunk - 1) / chunk;
    const uint32_t maxch = __reduce_max_sync(FULL, nch);
    const CensusArgs none{};
    auto issue = [&](uint32_t c) {
        if (c < nch) {
            const uint32_t rest = sbytes - c * chunk;
            const uint32_t b = rest < (uint32_t)chunk ? rest : (uint32_t)chunk;
            uint8_t *dst = ring + (c % stages) * stage_stride + qs * slot_stride;
            const uint8_t *from = src + (size_t)c * chunk;
            const uint8_t *wfrom = wsrc + (size_t)c * chunk;
            if (CHUNK && b == (uint32_t)CHUNK) {   // a full chunk of compile-time size: unrolled
#pragma unroll
                for (int o = 16 * j; o < (CHUNK ? CHUNK : 64); o += 64) {
                    cp_async16(dst + o, from + o);
                    cp_async16(dst + BATCH_PPW * slot_stride + o, wfrom + o);
                }
            } else {
                for (uint32_t o = 16 * j; o < b; o += 64) {
                    cp_async16(dst + o, from + o);
                    cp_async16(dst + BATCH_PPW * slot_stride + o, wfrom + o);
                }
            }
        }
        cp_async_commit();
    };
    for (int c = 0; c < stages - 1; ++c) issue((uint32_t)c);
    PageLanes<1> L;
    lanes_init(L, j);
    for (uint32_t c = 0; c < maxch; ++c) {
        issue(c + stages - 1);
        cp_async_wait(stages - 1);
        __syncwarp();
        const uint8_t *stage = ring + (c % stages) * stage_stride;
        uint32_t b = 0;
        if (c < nch) {
            const uint32_t rest = sbytes - c * chunk;
            b = rest < (uint32_t)chunk ? rest : (uint32_t)chunk;
        }
        hash_chunk<false, 1, CHUNK>(L, stage + qs * slot_stride + 8 * j, b, none);
        switch (J.dtype) {
        case KC_F32: fused_cmp_stage<KC_F32, CHUNK>(stage, slot_stride, b, off0, log2page, c * chunk, atol, rtol, acc, q); break;
        case KC_F16: fused_cmp_stage<KC_F16, CHUNK>(stage, slot_stride, b, off0, log2page, c * chunk, atol, rtol, acc, q); break;
        case KC_BF16: fused_cmp_stage<KC_BF16, CHUNK>(stage, slot_stride, b, off0, log2page, c * chunk, atol, rtol, acc, q); break;
        case KC_I32: fused_cmp_stage<KC_I32, CHUNK>(stage, slot_stride, b, off0, log2page, c * chunk, atol, rtol, acc, q); break;
        default: fused_cmp_stage<KC_U8, CHUNK>(stage, slot_stride, b, off0, log2page, c * chunk, atol, rtol, acc, q); break;
        }
        __syncwarp();   // the stage is free for the next refill
    }
    cp_async_wait(0);
    switch (J.dtype) {
    case KC_F32: fused_cmp_tails<KC_F32>(J, len, off0, log2page, atol, rtol, acc, q); break;
    case KC_F16: fused_cmp_tails<KC_F16>(J, len, off0, log2page, atol, rtol, acc, q); break;
    case KC_BF16: fused_cmp_tails<KC_BF16>(J, len, off0, log2page, atol, rtol, acc, q); break;
    case KC_I32: fused_cmp_tails<KC_I32>(J, len, off0, log2page, atol, rtol, acc, q); break;
    default: fused_cmp_tails<KC_U8>(J, len, off0, log2page, atol, rtol, acc, q); break;
    }
    return finish_page<false, 1>(L, src, len, false, none);
}

template <int CHUNK>
__global__ void __launch_bounds__(512) batch_kernel(const BatchJob *__restrict__ jobs,
                                                    uint32_t *__restrict__ left,
                                                    const BatchRange *__restrict__ ranges, int nranges,
                                                    uint64_t nitems, uint32_t page, uint32_t log2page, int stages,
                                                    int chunk, int slots, double atol, double rtol,
                                                    uint32_t *__restrict__ ctr) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int warp = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    const size_t ring_bytes = (size_t)stages * slots * ((size_t)chunk + 32);
    uint8_t *ring = smem + (size_t)warp * ring_bytes;
    // fused items' queue: a count, then BATCH_QCAP items, after all rings
    uint8_t *qarea = smem + (size_t)(blockDim.x >> 5) * ring_bytes + (size_t)warp * BATCH_QBYTES;
    const CensusArgs none{};
    while (true) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(ctr, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= nitems) break;
        // range holding item t: the last range whose first item <= t
        int lo = 0, hi = nranges - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ranges[mid].item_first <= t) lo = mid;
            else hi = mid - 1;
        }
        const BatchRange R = ranges[lo];
        const BatchJob J = jobs[R.job];
        const uint64_t k = t - R.item_first;
        const bool lost = (J.flags & BJ_LOST) != 0;
        if (R.kind == BR_FUSED && !lost) {
            const uint64_t u = BATCH_PPW * k + lane / 4;
            const bool valid = u < R.count;
            const uint64_t p0 = R.first + BATCH_PPW * k;     // the item's first page
            const uint64_t p = R.first + u;
            const uint64_t off = p << log2page;
            const uint64_t len = valid ? (J.bytes - off < page ? J.bytes - off : page) : 0;
            const uint8_t *src = reinterpret_cast<const uint8_t *>(J.got) + (valid ? off : 0);
            const uint8_t *wsrc = reinterpret_cast<const uint8_t *>(J.want) + (valid ? off : 0);
            const SlowQ q{reinterpret_cast<SlowItem *>(qarea + 16), reinterpret_cast<uint32_t *>(qarea), BATCH_QCAP};
            if (lane == 0) *q.count = 0;
            __syncwarp();
            CmpAcc acc{0ull, ~0ull, 0ull, 0ull, 0ull, 0.0, 0.0};
            const PageDigest d = fused_pages<CHUNK>(ring, stages, chunk, src, wsrc, len, J, p0 << log2page, log2page,
                                                    atol, rtol, acc, q);
            if ((lane & 3) == 0 && valid) {
                J.hash[p] = d.hash;
                J.zero[p] = d.zero ? KC_PAGE_ZERO : KC_PAGE_DATA;
            }
            cmp_drain_any(J.dtype, q, 1, atol, rtol, acc, lane, 32, WarpSync{});
            cmp_warp_flush(acc, J.cmp);
        } else if (R.kind == BR_DIGEST || R.kind == BR_FUSED) {   // (a lost fused job: digest outputs only)
            const uint64_t u = BATCH_PPW * k + lane / 4;   // unit within the range
            const bool valid = u < R.count;
            const uint64_t p = R.first + u;                 // page within the job
            const uint64_t off = p << log2page;
            const uint64_t len = valid ? (J.bytes - off < page ? J.bytes - off : page) : 0;
            const uint8_t *src = reinterpret_cast<const uint8_t *>(J.got) + (valid ? off : 0);
            const PageDigest d = digest_pages<false, 1, CHUNK>(ring, stages, chunk, src, len, lost, none);
            if ((lane & 3) == 0 && valid) {
                J.hash[p] = lost ? 0 : d.hash;
                J.zero[p] = lost ? KC_PAGE_LOST : (d.zero ? KC_PAGE_ZERO : KC_PAGE_DATA);
            }
        } else if (!lost) {
            CmpPair pr;
            pr.got = J.got;
            pr.want = J.want;
            pr.nelem = J.nelem;
            pr.tile_first = 0;
            pr.dtype = J.dtype;
            pr.lost = 0;
            pr.vec_first = 0;
            CmpAcc acc{0ull, ~0ull, 0ull, 0ull, 0ull, 0.0, 0.0};
            const uint64_t tiles = (J.bytes + CMP_TILE_BYTES - 1) / CMP_TILE_BYTES;
            const uint64_t t0 = (R.first + k) * (BATCH_CMP_ITEM_BYTES / CMP_TILE_BYTES);
            // the warp's digest ring is idle during a comparison item: it
            // holds the queue of differing elements (count, then items)
            const SlowQ q{reinterpret_cast<SlowItem *>(ring + 16), reinterpret_cast<uint32_t *>(ring),
                          (uint32_t)((ring_bytes - 16) / sizeof(SlowItem))};
            if (lane == 0) *q.count = 0;
            __syncwarp();
            for (uint64_t tile = t0; tile < t0 + BATCH_CMP_ITEM_BYTES / CMP_TILE_BYTES && tile < tiles; ++tile)
                cmp_tile_any<6>(pr, tile, atol, rtol, acc, lane, 32, q, WarpSync{});
            cmp_drain_any(pr.dtype, q, 1, atol, rtol, acc, lane, 32, WarpSync{});
            cmp_warp_flush(acc, J.cmp);
        }
        if (J.done) batch_item_done(J, left + R.job);
    }
}

template <int CHUNK>
static cudaError_t setup_batch_one() {
    return cudaFuncSetAttribute(batch_kernel<CHUNK>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

cudaError_t setup_batch_kernels() {
    cudaError_t e;
    if ((e = setup_batch_one<0>())) return e;
    if ((e = setup_batch_one<512>())) return e;
    return setup_batch_one<1024>();
}

size_t batch_smem_bytes(const DigestShape &s, bool fused) {
    return (size_t)s.warps * ((size_t)s.stages * (fused ? 2 : 1) * BATCH_PPW * ((size_t)s.chunk + 32) + BATCH_QBYTES);
}

cudaError_t launch_batch(const BatchJob *jobs, int njobs, uint32_t *left, const BatchRange *ranges, int nranges,
                         uint64_t nitems, uint32_t page, const DigestShape &shape, bool fused, double atol,
                         double rtol, uint32_t *ctr, int sms, cudaStream_t st) {
    batch_init_kernel<<<(njobs + 255) / 256, 256, 0, st>>>(jobs, njobs, left);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nitems == 0) return e;
    uint32_t log2page = 0;
    while ((1u << log2page) < page) ++log2page;
    const size_t smem = batch_smem_bytes(shape, fused);
    const int slots = fused ? 2 * BATCH_PPW : BATCH_PPW;
    const dim3 grid(shape.ctas), block(32 * shape.warps);
    switch (shape.chunk) {
    case 512:
        batch_kernel<512><<<grid, block, smem, st>>>(jobs, left, ranges, nranges, nitems, page, log2page,
                                                     shape.stages, shape.chunk, slots, atol, rtol, ctr);
        break;
    case 1024:
        batch_kernel<1024><<<grid, block, smem, st>>>(jobs, left, ranges, nranges, nitems, page, log2page,
                                                      shape.stages, shape.chunk, slots, atol, rtol, ctr);
        break;
    default:
        batch_kernel<0><<<grid, block, smem, st>>>(jobs, left, ranges, nranges, nitems, page, log2page,
                                                   shape.stages, shape.chunk, slots, atol, rtol, ctr);
    }
    count_launches(1);
    (void)sms;
    return cudaGetLastError();
}

}  // namespace kc
