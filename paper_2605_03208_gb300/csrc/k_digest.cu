// k_digest.cu -- the page digest kernel: XXH64 (seed 0) of every page, its
// zero flag and, in the fused scan, its census pre-filter flag (the hashing
// itself is in digest_task.cuh; the census kernels that finish the fused
// scan are in k_census.cu).
//
// XXH64 is four serial chains per page, so the digest of a snapshot of P
// pages has only 4P independent chains: on 64 KiB pages about one hashing
// warp per SM sub-partition.  Such a warp is bound by its own instruction
// latency, and every instruction it spends on copies or waits for data
// lengthens its chains' time, so each CTA pairs H hash warps with H loader
// warps:
//
//   loader warp H + w takes tasks of 8 consecutive pages from a global
//   ticket counter and streams the pages' full 32-byte stripes, one `chunk`
//   of each page per stage, into hash warp w's ring of shared-memory stages:
//   16-byte cp.async copies, all 32 lanes on one page at a time so that each
//   warp instruction moves 512 contiguous bytes, tracked by the stage's
//   "full" mbarrier (cp.async.mbarrier.arrive);
//
//   hash warp w runs the 8 pages with one XXH64 lane per thread: it waits
//   for a stage to be full, hashes it from shared memory, releases it (its
//   "empty" mbarrier), and after the last stage of a task finishes the pages
//   (tails < 32 bytes from global memory) and writes the outputs.
//
// Measured on this part before this design: one producer warp serving all
// hash warps of a CTA could not keep up (its serial cost per stage was
// ~0.7-1.2 us), and one bulk copy (cp.async.bulk) per page and stage cost the
// copy engine ~190 cycles per request whatever its size, too much for 1-2
// KiB pieces.
//
// The first stage of a task carries the task number in a header word; a
// header of all-ones ends the hash warp.  Every wait is bounded: a wait
// that gives up sets ST_TIMEOUT and an abort flag that makes the other
// warps of the CTA give up too, and each loader lane waits for the copies it
// issued before the CTA exits.
#include <cuda_runtime.h>

#include "digest_task.cuh"
#include "kc_device.cuh"
#include "kc_internal.cuh"

namespace kc {

constexpr int DG_PPW = 8;                   // pages per task
constexpr uint32_t DG_END = 0xFFFFFFFFu;    // stage header: no more tasks
constexpr uint32_t DG_WAIT_LIMIT = 1u << 15;   // suspended polls: ~2 s at most
constexpr int DG_MAX_HASH_WARPS = 8;

struct DgLayout {
    size_t hdr, ring, total;
};

// Shared memory of one CTA: full and empty barriers (hw x stages each), the
// stage headers and the abort word, the rings.
__host__ __device__ inline DgLayout dg_layout(int hw, int stages, int chunk) {
    DgLayout L;
    size_t o = (size_t)2 * hw * stages * 8;
    o = (o + 127) & ~(size_t)127;
    L.hdr = o;
    o += (size_t)hw * stages * 4 + 4;
    o = (o + 127) & ~(size_t)127;
    L.ring = o;
    o += (size_t)hw * stages * DG_PPW * ((size_t)chunk + 32);
    L.total = o;
    return L;
}

size_t digest_smem_bytes(const DigestShape &s) { return dg_layout(s.warps, s.stages, s.chunk).total; }
int digest_max_hash_warps() { return DG_MAX_HASH_WARPS; }

// Bytes of chunk c of a page holding `sb` bytes in full stripes.
__device__ __forceinline__ uint32_t chunk_bytes(uint32_t sb, uint32_t c, uint32_t chunk) {
    const uint32_t at = c * chunk;
    const uint32_t rest = sb > at ? sb - at : 0u;
    return rest < chunk ? rest : chunk;
}

// The fused digest leaves page_hits[p] = 0 for a page that cannot hold a
// census hit and region index + 1 for a page whose words must still be
// classified.  Small set-up work of the call rides along at the start (no
// extra launches): zeroing the census tail's ticket and chunk words and the
// caller's census counts, and copying the page offsets to the caller.
template <bool CENSUS, int CHUNK>
__global__ void __launch_bounds__(64 * DG_MAX_HASH_WARPS)
    digest_kernel(Pages pg, CensusArgs ca, uint64_t *__restrict__ hash, uint8_t *__restrict__ zero,
                  uint32_t *__restrict__ page_hits, uint32_t *__restrict__ task_ctr, uint32_t *__restrict__ status,
                  int stages, int chunk_, DigestAux aux) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t FULL = 0xffffffffu;
    const uint32_t chunk = (uint32_t)chunk_;
    const int hw = (int)(blockDim.x >> 6);
    const DgLayout lay = dg_layout(hw, stages, chunk_);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + hw * stages;
    uint32_t *hdr = reinterpret_cast<uint32_t *>(smem + lay.hdr);
    volatile uint32_t *abort = hdr + hw * stages;
    uint8_t *ring = smem + lay.ring;
    const size_t slot_stride = (size_t)chunk + 32;
    const size_t stage_stride = DG_PPW * slot_stride;
    const size_t ring_stride = (size_t)stages * stage_stride;
    {
        const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t i = gt; i < aux.nzero; i += nt) aux.zero_words[i] = i == 0 ? aux.first_ticket : 0ull;
        if (aux.counts && gt < 2) aux.counts[gt] = 0ull;
        for (uint64_t i = gt; i < aux.npf; i += nt) aux.pf_dst[i] = aux.pf_src[i];
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < hw * stages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        *abort = 0;
        mbar_fence_init();
    }
    __syncthreads();
    // the census tail (next on the stream) may be scheduled now: its CTAs
    // take the SMs this grid leaves and wait for its completion themselves
    grid_dep_launch();
    const int warp = threadIdx.x >> 5;
    const uint32_t lane = lane_id();

    if (warp >= hw) {
        // ---- loader of hash warp w ------------------------------------------
        const int w = warp - hw;
        uint8_t *ring_w = ring + w * ring_stride;
        uint32_t k = 0;
        bool end = false;
        while (!end) {
            uint32_t t = 0;
            if (lane == 0) t = atomicAdd(task_ctr, 1u);
            t = __shfl_sync(FULL, t, 0);
            end = (uint64_t)t * DG_PPW >= pg.npages;
            // lane q < 8: page q of the task (source, bytes in full stripes)
            uint64_t src = 0;
            uint32_t sb = 0;
            if (!end && lane < DG_PPW) {
                const uint64_t p = (uint64_t)t * DG_PPW + lane;
                if (p < pg.npages) {
                    const Region r = pg.regions[region_of(pg.regions, pg.nregions, p)];
                    const uint64_t off = (p - r.first) << pg.log2page;
                    const uint64_t len = r.bytes - off < pg.page ? r.bytes - off : pg.page;
                    if (!r.lost) {
                        src = r.base + off;
                        sb = (uint32_t)(len & ~31ull);
                    }
                }
            }
            uint32_t nch = __reduce_max_sync(FULL, (sb + chunk - 1) / chunk);
            if (nch == 0) nch = 1;
            // every lane keeps all 8 pages' sources and sizes in registers, so
            // the copy loop below has no shuffle in its dependency chains
            uint64_t psrc[DG_PPW];
            uint32_t psb[DG_PPW];
#pragma unroll
            for (int pq = 0; pq < DG_PPW; ++pq) {
                psrc[pq] = __shfl_sync(FULL, (unsigned long long)src, pq);
                psb[pq] = __shfl_sync(FULL, sb, pq);
            }
            for (uint32_t c = 0; c < nch; ++c, ++k) {
                const uint32_t s = k % (uint32_t)stages;
                bool ok = true;
                if (k >= (uint32_t)stages)
                    ok = mbar_wait(&empty[w * stages + s], ((k / stages) - 1) & 1u, DG_WAIT_LIMIT, abort);
                if (!__all_sync(FULL, ok)) {
                    if (lane == 0) {
                        set_status(status, ST_TIMEOUT);
                        *abort = 1;
                    }
                    end = true;
                    break;
                }
                uint64_t *fb = &full[w * stages + s];
                if (!end) {
                    uint8_t *stage = ring_w + s * stage_stride + 16 * lane;
                    const uint32_t at = c * chunk;
#pragma unroll
                    for (int pq = 0; pq < DG_PPW; ++pq) {
                        const uint32_t nb = psb[pq];
                        if (nb <= at) continue;   // uniform across the warp
                        uint8_t *to = stage + pq * slot_stride;
                        const uint8_t *from = reinterpret_cast<const uint8_t *>(psrc[pq]) + at + 16 * lane;
                        if (CHUNK && nb - at >= (uint32_t)CHUNK) {
#pragma unroll
                            for (int o = 0; o < (CHUNK ? CHUNK : 512); o += 512) cp_async16(to + o, from + o);
                        } else {
                            const uint32_t b = nb - at < chunk ? nb - at : chunk;
                            for (uint32_t o = 16 * lane; o < b; o += 512) cp_async16(to + o - 16 * lane, from + o - 16 * lane);
                        }
                    }
                    mbar_track_cp_async(fb);
                }
                __syncwarp();   // every lane's copies are tracked before the phase can complete
                if (lane == 0) {
                    if (end) hdr[w * stages + s] = DG_END;
                    else if (c == 0) hdr[w * stages + s] = t;
                    mbar_arrive(fb);
                }
            }
        }
        // The CTA must not exit while copies into its shared memory are in
        // flight: each lane waits for the copies it issued.
        cp_async_wait_all();
        return;
    }

    // ---- hash warp w ------------------------------------------------------
    const int w = warp;
    const int q = lane >> 2;   // page slot
    const int j = lane & 3;    // XXH64 lane
    const uint8_t *ring_w = ring + w * ring_stride;
    uint32_t k = 0;
    while (true) {
        uint32_t s = k % (uint32_t)stages;
        bool ok = mbar_wait(&full[w * stages + s], (k / stages) & 1u, DG_WAIT_LIMIT, abort);
        if (!__all_sync(FULL, ok)) {
            if (lane == 0) {
                set_status(status, ST_TIMEOUT);
                *abort = 1;
            }
            return;
        }
        const uint32_t t = hdr[w * stages + s];
        if (t == DG_END) return;
        const uint64_t p = (uint64_t)t * DG_PPW + q;
        const bool valid = p < pg.npages;
        const uint8_t *src = nullptr;
        uint64_t len = 0;
        bool lost = false;
        int ri = 0;
        if (valid) {
            ri = region_of(pg.regions, pg.nregions, p);
            const Region r = pg.regions[ri];
            const uint64_t off = (p - r.first) << pg.log2page;
            len = r.bytes - off < pg.page ? r.bytes - off : pg.page;
            src = reinterpret_cast<const uint8_t *>(r.base + off);
            lost = r.lost != 0;
        }
        const uint32_t sb = lost ? 0u : (uint32_t)(len & ~31ull);
        uint32_t nch = __reduce_max_sync(FULL, (sb + chunk - 1) / chunk);
        if (nch == 0) nch = 1;
        PageLanes<1> L;
        lanes_init(L, j);
        for (uint32_t c = 0; c < nch; ++c) {
            if (c > 0) {
                s = k % (uint32_t)stages;
                ok = mbar_wait(&full[w * stages + s], (k / stages) & 1u, DG_WAIT_LIMIT, abort);
                if (!__all_sync(FULL, ok)) {
                    if (lane == 0) {
                        set_status(status, ST_TIMEOUT);
                        *abort = 1;
                    }
                    return;
                }
            }
            hash_chunk<CENSUS, 1, CHUNK>(L, ring_w + s * stage_stride + q * slot_stride + 8 * j,
                                         chunk_bytes(sb, c, chunk), ca);
            __syncwarp();   // every lane is done reading the stage
            if (lane == 0) mbar_arrive(&empty[w * stages + s]);
            ++k;
        }
        const PageDigest d = finish_page<CENSUS, 1>(L, src, len, lost, ca);
        if (j == 0 && valid) {
            if (lost) {
                hash[p] = 0;
                zero[p] = KC_PAGE_LOST;
                if (CENSUS) page_hits[p] = 0;
            } else {
                hash[p] = d.hash;
                zero[p] = d.zero ? KC_PAGE_ZERO : KC_PAGE_DATA;
                if (CENSUS) page_hits[p] = d.cand ? (uint32_t)ri + 1u : 0u;   // region + 1: still to classify
            }
        }
    }
}

template <bool CENSUS, int CHUNK>
static cudaError_t setup_one() {
    return cudaFuncSetAttribute(digest_kernel<CENSUS, CHUNK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                227 * 1024);
}

template <bool CENSUS>
static cudaError_t setup_census() {
    cudaError_t e;
    if ((e = setup_one<CENSUS, 0>())) return e;
    if ((e = setup_one<CENSUS, 512>())) return e;
    return setup_one<CENSUS, 1024>();
}

cudaError_t setup_digest_kernels() {
    cudaError_t e;
    if ((e = setup_census<true>())) return e;
    return setup_census<false>();
}

template <bool CENSUS>
static void launch_chunk(dim3 grid, dim3 block, size_t smem, cudaStream_t st, const Pages &pg, const CensusArgs &ca,
                         uint64_t *hash, uint8_t *zero, uint32_t *page_hits, uint32_t *task_ctr, uint32_t *status,
                         const DigestShape &shape, const DigestAux &aux) {
    switch (shape.chunk) {
    case 512:
        digest_kernel<CENSUS, 512><<<grid, block, smem, st>>>(pg, ca, hash, zero, page_hits, task_ctr, status,
                                                              shape.stages, shape.chunk, aux);
        break;
    case 1024:
        digest_kernel<CENSUS, 1024><<<grid, block, smem, st>>>(pg, ca, hash, zero, page_hits, task_ctr, status,
                                                               shape.stages, shape.chunk, aux);
        break;
    default:
        digest_kernel<CENSUS, 0><<<grid, block, smem, st>>>(pg, ca, hash, zero, page_hits, task_ctr, status,
                                                            shape.stages, shape.chunk, aux);
    }
}

cudaError_t launch_digest(const Pages &pg, const CensusArgs *census, uint64_t *hash, uint8_t *zero,
                          uint32_t *page_hits, uint32_t *task_ctr, uint32_t *status, const DigestShape &shape,
                          const DigestAux &aux, cudaStream_t st) {
    if (shape.warps < 1 || shape.warps > DG_MAX_HASH_WARPS || shape.stages < 2 || shape.chunk < 128 ||
        (shape.chunk % 128))
        return cudaErrorInvalidValue;
    const size_t smem = digest_smem_bytes(shape);
    const dim3 block(64 * shape.warps), grid(shape.ctas);
    if (census)
        launch_chunk<true>(grid, block, smem, st, pg, *census, hash, zero, page_hits, task_ctr, status, shape, aux);
    else
        launch_chunk<false>(grid, block, smem, st, pg, CensusArgs{}, hash, zero, nullptr, task_ctr, status, shape,
                            aux);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace kc
