// k_batch.cu -- the batched form: one persistent, work-stealing launch over
// many jobs of uneven sizes, replacing one launch per buffer per operation.
//
// The work of a launch is a list of ranges (a job's pages to digest, or its
// comparison items), flattened into one item space: a digest item is one
// 8-page task, a comparison item is 64 KiB of a (got, want) pair.  Every warp
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

template <int CHUNK>
__global__ void __launch_bounds__(512) batch_kernel(const BatchJob *__restrict__ jobs,
                                                    uint32_t *__restrict__ left,
                                                    const BatchRange *__restrict__ ranges, int nranges,
                                                    uint64_t nitems, uint32_t page, uint32_t log2page, int stages,
                                                    int chunk, double atol, double rtol, uint32_t *__restrict__ ctr) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int warp = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    uint8_t *ring = smem + (size_t)warp * stages * BATCH_PPW * ((size_t)chunk + 32);
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
        if (R.kind == 0) {
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
            const size_t ring_bytes = (size_t)stages * BATCH_PPW * ((size_t)chunk + 32);
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

size_t batch_smem_bytes(const DigestShape &s) {
    return (size_t)s.warps * s.stages * BATCH_PPW * ((size_t)s.chunk + 32);
}

cudaError_t launch_batch(const BatchJob *jobs, int njobs, uint32_t *left, const BatchRange *ranges, int nranges,
                         uint64_t nitems, uint32_t page, const DigestShape &shape, double atol, double rtol,
                         uint32_t *ctr, int sms, cudaStream_t st) {
    batch_init_kernel<<<(njobs + 255) / 256, 256, 0, st>>>(jobs, njobs, left);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nitems == 0) return e;
    uint32_t log2page = 0;
    while ((1u << log2page) < page) ++log2page;
    const size_t smem = batch_smem_bytes(shape);
    const dim3 grid(shape.ctas), block(32 * shape.warps);
    switch (shape.chunk) {
    case 512:
        batch_kernel<512><<<grid, block, smem, st>>>(jobs, left, ranges, nranges, nitems, page, log2page,
                                                     shape.stages, shape.chunk, atol, rtol, ctr);
        break;
    case 1024:
        batch_kernel<1024><<<grid, block, smem, st>>>(jobs, left, ranges, nranges, nitems, page, log2page,
                                                      shape.stages, shape.chunk, atol, rtol, ctr);
        break;
    default:
        batch_kernel<0><<<grid, block, smem, st>>>(jobs, left, ranges, nranges, nitems, page, log2page,
                                                   shape.stages, shape.chunk, atol, rtol, ctr);
    }
    count_launches(1);
    (void)sms;
    return cudaGetLastError();
}

}  // namespace kc
