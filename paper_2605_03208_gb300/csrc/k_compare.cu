// k_compare.cu -- per-dtype comparison of replayed outputs against captured
// ones (Section "Replay Validation": byte-exact and numpy.allclose-style
// tolerance comparison, NaNs reported explicitly); the element logic is in
// compare_tile.cuh.
//
// All pairs are cut into 16 KiB tiles of `got` bytes, flattened into one
// tile space; each CTA takes a contiguous range of tiles.  Per-tile partial
// results are merged with order-independent atomics: sums of counts, min of
// the first index (u64, initial all-ones = -1 as i64) and max of the
// non-negative FP64 maxima as u64 bit patterns (their order is the numeric
// order; NaN is never stored).
#include <cuda_runtime.h>

#include "compare_tile.cuh"
#include "kc_internal.cuh"

namespace kc {

constexpr int CMP_THREADS = 256;
constexpr uint32_t CMP_QCAP = 1024;   // queued differing elements per CTA (16 KB)

__global__ void cmp_init_kernel(const CmpPair *__restrict__ pairs, int npairs, kc_cmp_result *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npairs) return;
    cmp_record_init(&out[i], pairs[i].lost ? KC_EBUF : KC_OK);
}

// Merge one CTA's accumulators into the pair's record (all threads call it).
__device__ void cmp_flush(CmpAcc &acc, kc_cmp_result *o, unsigned long long (*red)[CMP_THREADS / 32]) {
    unsigned long long v[7] = {acc.mism, acc.first, acc.nan_g, acc.nan_w, acc.nan_m,
                               dbits(acc.max_abs), dbits(acc.max_rel)};
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        v[0] += __shfl_xor_sync(0xffffffffu, v[0], off);
        const unsigned long long f = __shfl_xor_sync(0xffffffffu, v[1], off);
        v[1] = f < v[1] ? f : v[1];
        v[2] += __shfl_xor_sync(0xffffffffu, v[2], off);
        v[3] += __shfl_xor_sync(0xffffffffu, v[3], off);
        v[4] += __shfl_xor_sync(0xffffffffu, v[4], off);
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, v[5], off);
        v[5] = a > v[5] ? a : v[5];
        const unsigned long long r = __shfl_xor_sync(0xffffffffu, v[6], off);
        v[6] = r > v[6] ? r : v[6];
    }
    if (lane_id() == 0) {
#pragma unroll
        for (int j = 0; j < 7; ++j) red[j][threadIdx.x >> 5] = v[j];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long sm[7] = {0ull, ~0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
        for (int wi = 0; wi < CMP_THREADS / 32; ++wi) {
            sm[0] += red[0][wi];
            sm[1] = red[1][wi] < sm[1] ? red[1][wi] : sm[1];
            sm[2] += red[2][wi];
            sm[3] += red[3][wi];
            sm[4] += red[4][wi];
            sm[5] = red[5][wi] > sm[5] ? red[5][wi] : sm[5];
            sm[6] = red[6][wi] > sm[6] ? red[6][wi] : sm[6];
        }
        if (sm[0]) atomicAdd(reinterpret_cast<unsigned long long *>(&o->mismatches), sm[0]);
        if (sm[1] != ~0ull) atomicMin(reinterpret_cast<unsigned long long *>(&o->first), sm[1]);
        if (sm[2]) atomicAdd(reinterpret_cast<unsigned long long *>(&o->nan_got), sm[2]);
        if (sm[3]) atomicAdd(reinterpret_cast<unsigned long long *>(&o->nan_want), sm[3]);
        if (sm[4]) atomicAdd(reinterpret_cast<unsigned long long *>(&o->nan_mismatch), sm[4]);
        if (sm[5]) atomicMax(reinterpret_cast<unsigned long long *>(&o->max_abs), sm[5]);
        if (sm[6]) atomicMax(reinterpret_cast<unsigned long long *>(&o->max_rel), sm[6]);
    }
    __syncthreads();
    acc = CmpAcc{0ull, ~0ull, 0ull, 0ull, 0ull, 0.0, 0.0};
}

// Each CTA takes a contiguous range of tiles, so consecutive tiles mostly
// belong to the same pair and a CTA merges into a pair's record once per
// pair it touches, not once per tile.
__global__ void __launch_bounds__(CMP_THREADS, 3) cmp_kernel(const CmpPair *__restrict__ pairs, int npairs,
                                                          uint64_t ntiles, double atol, double rtol,
                                                          kc_cmp_result *__restrict__ out) {
    __shared__ unsigned long long red[7][CMP_THREADS / 32];
    __shared__ SlowItem qitems[CMP_QCAP];
    __shared__ uint32_t qcount;
    const uint64_t t0 = ntiles * blockIdx.x / gridDim.x;
    const uint64_t t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    if (t0 >= t1) return;
    if (threadIdx.x == 0) qcount = 0;
    __syncthreads();
    const SlowQ q{qitems, &qcount, CMP_QCAP};
    // pair owning t0: last pair whose first tile <= t0
    int lo = 0, hi = npairs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (pairs[mid].tile_first <= t0) lo = mid;
        else hi = mid - 1;
    }
    int k = lo;
    CmpPair pr = pairs[k];
    CmpAcc acc{0ull, ~0ull, 0ull, 0ull, 0ull, 0.0, 0.0};
    for (uint64_t tile = t0; tile < t1; ++tile) {
        bool moved = false;
        while (k + 1 < npairs && pairs[k + 1].tile_first <= tile) {
            if (!moved) {
                cmp_drain_any(pr.dtype, q, 1, atol, rtol, acc, threadIdx.x, CMP_THREADS, CtaSync{});
                cmp_flush(acc, &out[k], red);
            }
            moved = true;
            ++k;
        }
        if (moved) pr = pairs[k];
        if (pr.lost) continue;
        cmp_tile_any<4>(pr, tile - pr.tile_first, atol, rtol, acc, threadIdx.x, CMP_THREADS, q, CtaSync{});
        cmp_drain_any(pr.dtype, q, CMP_QCAP / 2, atol, rtol, acc, threadIdx.x, CMP_THREADS, CtaSync{});
    }
    cmp_drain_any(pr.dtype, q, 1, atol, rtol, acc, threadIdx.x, CMP_THREADS, CtaSync{});
    cmp_flush(acc, &out[k], red);
}

cudaError_t launch_compare(const CmpPair *pairs, int npairs, uint64_t ntiles, double atol, double rtol,
                           kc_cmp_result *out, const int32_t *, int sms, cudaStream_t st) {
    cmp_init_kernel<<<(npairs + 127) / 128, 128, 0, st>>>(pairs, npairs, out);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || ntiles == 0) return e;
    uint64_t blocks = ntiles;
    const uint64_t maxb = (uint64_t)sms * 6;   // 2 waves of 3 resident CTAs per SM: measured best of 3..8
    if (blocks > maxb) blocks = maxb;
    cmp_kernel<<<(unsigned)blocks, CMP_THREADS, 0, st>>>(pairs, npairs, ntiles, atol, rtol, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace kc
