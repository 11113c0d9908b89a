// k_digest.cu -- the page digest kernel (XXH64 seed 0 + zero flag, optionally
// with the census pre-filter flag per page; hashing in digest_task.cuh).
// The census kernels that finish the fused scan are in k_census.cu.
#include <cuda_runtime.h>

#include "digest_task.cuh"
#include "kc_device.cuh"
#include "kc_internal.cuh"

namespace kc {

// The fused digest leaves page_hits[p] = 0 for a page that cannot hold a
// census hit and region index + 1 for a page whose words must still be
// classified.

size_t digest_smem_bytes(const DigestShape &s) {
    const size_t ppw = 8 * (size_t)(s.lanes == 2 ? 2 : 1);
    return (size_t)s.warps * s.stages * ppw * (size_t)(s.chunk + 32);
}

// One warp per task of PPW consecutive pages (8 with one XXH64 lane per
// thread, 16 with two), tasks taken from a global ticket counter so warps
// that finish early steal the rest; see digest_task.cuh for the hashing.
//
// Small set-up work of the call rides along at the start (no extra
// launches): zeroing the census tail's ticket and chunk words and the
// caller's census counts, and copying the page offsets to the caller.
template <bool CENSUS, int LPT, int CHUNK>
__global__ void __launch_bounds__(512) digest_kernel(Pages pg, CensusArgs ca, uint64_t *__restrict__ hash,
                                                     uint8_t *__restrict__ zero,
                                                     uint32_t *__restrict__ page_hits,
                                                     uint32_t *__restrict__ task_ctr,
                                                     uint32_t *__restrict__ status, int stages, int chunk,
                                                     DigestAux aux) {
    constexpr int TPP = 4 / LPT;
    constexpr int PPW = 32 / TPP;
    extern __shared__ __align__(128) uint8_t smem[];
    (void)status;   // no waits here can time out: cp.async groups always complete
    {
        const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t i = gt; i < aux.nzero; i += nt) aux.zero_words[i] = i == 0 ? aux.first_ticket : 0ull;
        if (aux.counts && gt < 2) aux.counts[gt] = 0ull;
        for (uint64_t i = gt; i < aux.npf; i += nt) aux.pf_dst[i] = aux.pf_src[i];
    }
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
        int ri = 0;
        if (valid) {
            ri = region_of(pg.regions, pg.nregions, p);
            const Region r = pg.regions[ri];
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
                if (CENSUS) page_hits[p] = d.cand ? (uint32_t)ri + 1u : 0u;   // region + 1: still to classify
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

template <bool CENSUS, int LPT>
static void launch_lanes(dim3 grid, dim3 block, size_t smem, cudaStream_t st, const Pages &pg, const CensusArgs &ca,
                         uint64_t *hash, uint8_t *zero, uint32_t *page_hits, uint32_t *task_ctr, uint32_t *status,
                         const DigestShape &shape, const DigestAux &aux) {
    switch (shape.chunk) {
    case 512:
        digest_kernel<CENSUS, LPT, 512><<<grid, block, smem, st>>>(pg, ca, hash, zero, page_hits, task_ctr, status,
                                                                   shape.stages, shape.chunk, aux);
        break;
    case 1024:
        digest_kernel<CENSUS, LPT, 1024><<<grid, block, smem, st>>>(pg, ca, hash, zero, page_hits, task_ctr, status,
                                                                    shape.stages, shape.chunk, aux);
        break;
    default:
        digest_kernel<CENSUS, LPT, 0><<<grid, block, smem, st>>>(pg, ca, hash, zero, page_hits, task_ctr, status,
                                                                 shape.stages, shape.chunk, aux);
    }
}

cudaError_t launch_digest(const Pages &pg, const CensusArgs *census, uint64_t *hash, uint8_t *zero,
                          uint32_t *page_hits, uint32_t *task_ctr, uint32_t *status, const DigestShape &shape,
                          const DigestAux &aux, cudaStream_t st) {
    const size_t smem = digest_smem_bytes(shape);
    const dim3 block(32 * shape.warps), grid(shape.ctas);
    CensusArgs none{};
    if (census && shape.lanes == 2)
        launch_lanes<true, 2>(grid, block, smem, st, pg, *census, hash, zero, page_hits, task_ctr, status, shape, aux);
    else if (census)
        launch_lanes<true, 1>(grid, block, smem, st, pg, *census, hash, zero, page_hits, task_ctr, status, shape, aux);
    else if (shape.lanes == 2)
        launch_lanes<false, 2>(grid, block, smem, st, pg, none, hash, zero, nullptr, task_ctr, status, shape, aux);
    else
        launch_lanes<false, 1>(grid, block, smem, st, pg, none, hash, zero, nullptr, task_ctr, status, shape, aux);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace kc
