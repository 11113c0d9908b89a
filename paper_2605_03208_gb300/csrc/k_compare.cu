// k_compare.cu -- per-dtype comparison of replayed outputs against captured
// ones (Section "Replay Validation": byte-exact and numpy.allclose-style
// tolerance comparison, NaNs reported explicitly); the element logic is in
// compare_tile.cuh.
//
// The pairs are grouped by dtype; each group's whole 16-byte vectors are
// laid end to end and split evenly over every warp of its kernel's grid
// (the warp-streaming body is in compare_tile.cuh).  Partial results are
// merged with order-independent atomics -- sums of counts, min of the first
// index (u64, initial all-ones = -1 as i64) and max of the non-negative
// FP64 maxima as u64 bit patterns (their order is the numeric order; NaN is
// never stored) -- into each pair's record, once per warp and pair.
#include <cuda_runtime.h>

#include "compare_tile.cuh"
#include "kc_internal.cuh"

namespace kc {

// One kernel per dtype (a kernel holding every dtype's loops missed the
// instruction cache: "no instruction" was its top stall), over the pairs of
// that dtype.  Every warp of the grid takes an equal, contiguous share of
// the group's 16-byte vectors (its pairs laid end to end) and streams it
// with CW_U loads of each buffer in flight per lane and no block barriers;
// where its share crosses into a new pair it evaluates its queue and merges
// its accumulators into the finished pair's record (one merge per warp and
// pair touched).  (Handing out blocks of vectors grid-stride instead, so
// that the grid sweeps one window of each buffer, measured slower: 29.8
// against 25.8 us on a 117 MB bf16 pair.)  The < 16-byte end of pair k is
// taken by warp k (mod the warp count) after its share.
constexpr int CW_WARPS = 8;
constexpr int CW_THREADS = 32 * CW_WARPS;
constexpr int CW_U = 8;
constexpr uint32_t CW_QCAP = 128;   // queued vectors per warp (40 B each)

template <int DT>
__device__ __forceinline__ void cw_pair(const CmpPair &pr, uint64_t va, uint64_t vb, bool tail, double atol,
                                        double rtol, kc_cmp_result *o, WarpQ &q) {
    CmpAcc acc = cmp_acc_zero();
    if (va < vb) warp_compare_range<DT, CW_U>(pr, va, vb, atol, rtol, acc, q);
    if (tail) warp_compare_tail<DT>(pr, atol, rtol, acc, q);
    wq_drain<DT>(q, atol, rtol, acc);
    cmp_warp_flush(acc, o);
}

template <int DT>
__global__ void __launch_bounds__(CW_THREADS, 2) cmp_kernel(const CmpPair *__restrict__ pairs, int npairs, uint64_t nvec,
                                                            double atol, double rtol,
                                                            kc_cmp_result *__restrict__ out) {
    extern __shared__ __align__(16) uint8_t cw_smem[];
    constexpr uint64_t ES = esize<DT>();
    const int warp = threadIdx.x >> 5;
    WarpQ q{reinterpret_cast<VecItem *>(cw_smem) + warp * CW_QCAP, CW_QCAP, 0u, 0.0f, 0.0f};
    const uint64_t nw = (uint64_t)gridDim.x * CW_WARPS;
    const uint64_t wid = (uint64_t)blockIdx.x * CW_WARPS + warp;
    uint64_t va = nvec * wid / nw;
    const uint64_t vb = nvec * (wid + 1) / nw;
    if (va < vb) {
        // the pair holding vector va: the last whose first vector is <= va
        int lo = 0, hi = npairs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pairs[mid].vec_first <= va) lo = mid;
            else hi = mid - 1;
        }
        for (int k = lo; k < npairs && va < vb; ++k) {
            const CmpPair pr = pairs[k];
            const uint64_t pend = pr.vec_first + ((pr.nelem * ES) >> 4);
            const uint64_t end = pend < vb ? pend : vb;
            if (end > va && !pr.lost)
                cw_pair<DT>(pr, va - pr.vec_first, end - pr.vec_first, false, atol, rtol, &out[pr.out_index], q);
            if (end > va) va = end;
        }
    }
    for (uint64_t k = wid; k < (uint64_t)npairs; k += nw) {
        const CmpPair pr = pairs[k];
        if (!pr.lost && ((pr.nelem * ES) & 15))
            cw_pair<DT>(pr, 0, 0, true, atol, rtol, &out[pr.out_index], q);
    }
}

__global__ void cmp_init_kernel(const CmpPair *__restrict__ pairs, int npairs, kc_cmp_result *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npairs) return;
    cmp_record_init(&out[pairs[i].out_index], pairs[i].lost ? KC_EBUF : KC_OK);
}

constexpr size_t CW_SMEM = (size_t)CW_WARPS * CW_QCAP * sizeof(VecItem);

cudaError_t setup_compare_kernels() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(cmp_kernel<KC_U8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CW_SMEM))) return e;
    if ((e = cudaFuncSetAttribute(cmp_kernel<KC_I32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CW_SMEM)))
        return e;
    if ((e = cudaFuncSetAttribute(cmp_kernel<KC_F16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CW_SMEM)))
        return e;
    if ((e = cudaFuncSetAttribute(cmp_kernel<KC_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CW_SMEM)))
        return e;
    return cudaFuncSetAttribute(cmp_kernel<KC_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CW_SMEM);
}

cudaError_t launch_compare(const CmpPair *pairs, int npairs, const CmpGroups &gr, double atol, double rtol,
                           kc_cmp_result *out, int sms, cudaStream_t st) {
    cmp_init_kernel<<<(npairs + 127) / 128, 128, 0, st>>>(pairs, npairs, out);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    for (int d = 0; d < 6 && e == cudaSuccess; ++d) {
        const int n = gr.gfirst[d + 1] - gr.gfirst[d];
        if (n == 0) continue;
        // two CTAs of 8 warps per SM; small groups use fewer, at least 2048
        // vectors per warp, and at least one warp per pair
        const uint64_t nvec = gr.gvec[d];
        uint64_t blocks = (uint64_t)sms * 2;
        const uint64_t want = (nvec + 2048ull * CW_WARPS - 1) / (2048ull * CW_WARPS);
        const uint64_t least = ((uint64_t)n + CW_WARPS - 1) / CW_WARPS;
        if (want < blocks) blocks = want > least ? want : least;
        if (blocks > (uint64_t)sms * 2) blocks = (uint64_t)sms * 2;
        if (blocks == 0) blocks = 1;
        const CmpPair *gp = pairs + gr.gfirst[d];
        const dim3 g((unsigned)blocks), b(CW_THREADS);
        switch (d) {
        case KC_F32: cmp_kernel<KC_F32><<<g, b, CW_SMEM, st>>>(gp, n, nvec, atol, rtol, out); break;
        case KC_F16: cmp_kernel<KC_F16><<<g, b, CW_SMEM, st>>>(gp, n, nvec, atol, rtol, out); break;
        case KC_BF16: cmp_kernel<KC_BF16><<<g, b, CW_SMEM, st>>>(gp, n, nvec, atol, rtol, out); break;
        case KC_I32: cmp_kernel<KC_I32><<<g, b, CW_SMEM, st>>>(gp, n, nvec, atol, rtol, out); break;
        default: cmp_kernel<KC_U8><<<g, b, CW_SMEM, st>>>(gp, n, nvec, atol, rtol, out); break;
        }
        count_launches(1);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace kc
