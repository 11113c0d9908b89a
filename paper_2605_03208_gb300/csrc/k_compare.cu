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
// that dtype, whose whole 16-byte vectors are laid end to end.  The warps of
// the grid sweep that vector space together, grid-stride, in blocks of
// 32 x CW_U vectors: each lane keeps CW_U loads of each buffer in flight,
// and at any moment the whole GPU reads one window of the space (measured
// on a 117 MB bf16 pair: 42.5 us, against 52.6 us for one contiguous share
// per warp).  A warp's blocks go up through the space, so it meets each pair
// once, in order; it evaluates its queue and merges its accumulators into a
// pair's record when it moves past the pair.  The < 16-byte end of pair k
// is taken by warp k (mod the warp count) at the end.
constexpr int CW_WARPS = 8;
constexpr int CW_THREADS = 32 * CW_WARPS;
constexpr int CW_U = 4;
constexpr uint32_t CW_QCAP = 128;   // queued vectors per warp (48 B each; both tolerance modes)

template <int DT, bool ZT>
__global__ void __launch_bounds__(CW_THREADS, 2) cmp_kernel(const CmpPair *__restrict__ pairs, int npairs, uint64_t nvec,
                                                            double atol, double rtol,
                                                            kc_cmp_result *__restrict__ out,
                                                            uint32_t *__restrict__ gates) {
    extern __shared__ __align__(16) uint8_t cw_smem[];
    constexpr uint64_t ES = esize<DT>();
    constexpr uint64_t BV = 32 * CW_U;
    const int warp = threadIdx.x >> 5;
    WarpQ q{reinterpret_cast<VecItem *>(cw_smem) + warp * CW_QCAP, CW_QCAP, 0u, 0.0f, 0.0f, nullptr};
    const uint64_t nw = (uint64_t)gridDim.x * CW_WARPS;
    const uint64_t wid = (uint64_t)blockIdx.x * CW_WARPS + warp;
    int k = -1;          // the pair whose accumulators acc holds
    CmpPair pr{};
    uint64_t pend = 0;   // end of pair k's vectors
    CmpAcc acc = cmp_acc_zero();
    for (uint64_t b0 = wid * BV; b0 < nvec; b0 += nw * BV) {
        const uint64_t b1 = b0 + BV < nvec ? b0 + BV : nvec;
        uint64_t v = b0;
        while (v < b1) {
            if (k < 0 || v >= pend) {
                if (k >= 0) {
                    wq_drain<DT, ZT>(q, atol, rtol, acc);
                    cmp_warp_flush(acc, &out[pr.out_index]);
                    acc = cmp_acc_zero();
                }
                // the pair holding v: the last whose first vector is <= v
                int lo = k < 0 ? 0 : k, hi = npairs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (pairs[mid].vec_first <= v) lo = mid;
                    else hi = mid - 1;
                }
                k = lo;
                pr = pairs[k];
                pend = pr.vec_first + ((pr.nelem * ES) >> 4);
                q.gate = gates + 2 * (uint64_t)pr.out_index;
                q.run_abs = 0.0f;
                q.run_rel = 0.0f;
            }
            const uint64_t e = pend < b1 ? pend : b1;
            if (!pr.lost)
                warp_compare_range<DT, CW_U, ZT>(pr, v - pr.vec_first, e - pr.vec_first, atol, rtol, acc, q);
            v = e;
        }
    }
    if (k >= 0) {
        wq_drain<DT, ZT>(q, atol, rtol, acc);
        cmp_warp_flush(acc, &out[pr.out_index]);
    }
    for (uint64_t t = wid; t < (uint64_t)npairs; t += nw) {
        const CmpPair tp = pairs[t];
        if (tp.lost || !((tp.nelem * ES) & 15)) continue;
        CmpAcc ta = cmp_acc_zero();
        warp_compare_tail<DT>(tp, atol, rtol, ta, q);
        cmp_warp_flush(ta, &out[tp.out_index]);
    }
}

// Every pair's record starts empty (status KC_EBUF for a lost pair) and its
// proxy gate at zero.
__global__ void cmp_init_kernel(const CmpPair *__restrict__ pairs, int npairs, kc_cmp_result *__restrict__ out,
                                uint32_t *__restrict__ gates) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npairs) return;
    const uint32_t o = pairs[i].out_index;
    cmp_record_init(&out[o], pairs[i].lost ? KC_EBUF : KC_OK);
    gates[2 * (uint64_t)o] = 0u;
    gates[2 * (uint64_t)o + 1] = 0u;
}

constexpr size_t CW_SMEM = (size_t)CW_WARPS * CW_QCAP * sizeof(VecItem);   // the warps' queues

template <int DT>
cudaError_t setup_cmp_dtype() {
    const cudaError_t e =
        cudaFuncSetAttribute(cmp_kernel<DT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CW_SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(cmp_kernel<DT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CW_SMEM);
}

cudaError_t setup_compare_kernels() {
    cudaError_t e;
    if ((e = setup_cmp_dtype<KC_U8>())) return e;
    if ((e = setup_cmp_dtype<KC_I32>())) return e;
    if ((e = setup_cmp_dtype<KC_F16>())) return e;
    if ((e = setup_cmp_dtype<KC_BF16>())) return e;
    return setup_cmp_dtype<KC_F32>();
}

template <int DT>
void launch_cmp_dtype(dim3 g, const CmpPair *gp, int n, uint64_t nvec, double atol, double rtol, kc_cmp_result *out,
                      uint32_t *gates, cudaStream_t st) {
    const dim3 b(CW_THREADS);
    if (atol == 0.0 && rtol == 0.0) cmp_kernel<DT, true><<<g, b, CW_SMEM, st>>>(gp, n, nvec, atol, rtol, out, gates);
    else cmp_kernel<DT, false><<<g, b, CW_SMEM, st>>>(gp, n, nvec, atol, rtol, out, gates);
}

cudaError_t launch_compare(const CmpPair *pairs, int npairs, const CmpGroups &gr, double atol, double rtol,
                           kc_cmp_result *out, uint32_t *gates, int sms, cudaStream_t st) {
    cmp_init_kernel<<<(npairs + 127) / 128, 128, 0, st>>>(pairs, npairs, out, gates);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    for (int d = 0; d < 6 && e == cudaSuccess; ++d) {
        const int n = gr.gfirst[d + 1] - gr.gfirst[d];
        if (n == 0) continue;
        // two CTAs of 8 warps per SM; a small group uses fewer, one block of
        // 32 x CW_U vectors per warp (its time is then about one memory
        // latency), and at least one warp per pair
        const uint64_t nvec = gr.gvec[d];
        uint64_t blocks = (uint64_t)sms * 2;
        const uint64_t want = (nvec + 32ull * CW_U * CW_WARPS - 1) / (32ull * CW_U * CW_WARPS);
        const uint64_t least = ((uint64_t)n + CW_WARPS - 1) / CW_WARPS;
        if (want < blocks) blocks = want > least ? want : least;
        if (blocks > (uint64_t)sms * 2) blocks = (uint64_t)sms * 2;
        if (blocks == 0) blocks = 1;
        const CmpPair *gp = pairs + gr.gfirst[d];
        const dim3 g((unsigned)blocks);
        switch (d) {
        case KC_F32: launch_cmp_dtype<KC_F32>(g, gp, n, nvec, atol, rtol, out, gates, st); break;
        case KC_F16: launch_cmp_dtype<KC_F16>(g, gp, n, nvec, atol, rtol, out, gates, st); break;
        case KC_BF16: launch_cmp_dtype<KC_BF16>(g, gp, n, nvec, atol, rtol, out, gates, st); break;
        case KC_I32: launch_cmp_dtype<KC_I32>(g, gp, n, nvec, atol, rtol, out, gates, st); break;
        default: launch_cmp_dtype<KC_U8>(g, gp, n, nvec, atol, rtol, out, gates, st); break;
        }
        count_launches(1);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace kc
