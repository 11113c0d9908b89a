// compare_tile.cuh -- per-element comparison of a tile of a (got, want)
// pair, shared by the comparison kernel and the batched kernel (Section
// "Replay Validation": numpy.allclose-style tolerance comparison with NaNs
// reported explicitly).
//
// Each thread streams 16-byte vectors of both buffers.  A vector whose 16
// bytes are bitwise equal in got and want only needs its NaNs counted (equal
// bits are equal values, NaN == NaN), so the FP64 unit -- slow on this part
// -- is used only for elements whose bits differ: those are widened exactly
// to double, and the error values are one IEEE operation each (__dsub_rn,
// __ddiv_rn, __dmul_rn, __dadd_rn: no FMA contraction), hence identical to
// any other correctly rounded evaluation.
//
// Two bodies use this.  The batched kernel compares tiles with a CTA: its
// differing elements are queued (index and both bit patterns, in shared
// memory) and evaluated at the end of the tile with every lane busy, since
// on this part a warp's FP64 instruction costs the same whatever its active
// lanes; an element that finds the queue full is evaluated where it is.
// The comparison kernel streams with warps (warp_compare_range): with
// tolerances it queues differing vectors per warp the same way; with zero
// tolerances it classifies them where they are found and uses FP64 only for
// the few elements that can hold the maxima (below).  What is accumulated
// -- counts, the smallest index, maxima -- does not depend on the order, so
// the results are unchanged.
#pragma once

#include <cuda_fp16.h>
#include <math_constants.h>

#include "kc_device.cuh"

namespace kc {

struct CmpAcc {
    unsigned long long mism, first, nan_g, nan_w, nan_m;
    double max_abs, max_rel;
};

template <int DT>
__device__ __forceinline__ double widen(uint32_t bits) {
    if (DT == KC_F32) return (double)__uint_as_float(bits);
    if (DT == KC_BF16) return (double)__uint_as_float(bits << 16);
    if (DT == KC_F16) return (double)__half2float(__ushort_as_half((unsigned short)bits));
    if (DT == KC_I32) return (double)(int32_t)bits;
    return (double)bits;   // KC_U8 / KC_RAW
}

// NaN test on the raw bits of one element.
template <int DT>
__device__ __forceinline__ bool bits_nan(uint32_t bits) {
    if (DT == KC_F32) return (bits & 0x7fffffffu) > 0x7f800000u;
    if (DT == KC_BF16) return (bits & 0x7fffu) > 0x7f80u;
    if (DT == KC_F16) return (bits & 0x7fffu) > 0x7c00u;
    return false;
}

template <int DT>
__device__ __forceinline__ void cmp_slow(uint32_t gb, uint32_t wb, unsigned long long idx, double atol,
                                         double rtol, CmpAcc &acc) {
    const double a = widen<DT>(gb), b = widen<DT>(wb);
    const bool na = isnan(a), nb = isnan(b);
    acc.nan_g += na;
    acc.nan_w += nb;
    if (na && nb) return;
    if (na != nb) {
        acc.mism += 1;
        acc.nan_m += 1;
        acc.first = idx < acc.first ? idx : acc.first;
        return;
    }
    if (a == b) return;
    const double d = fabs(__dsub_rn(a, b));
    const double r = (b == 0.0 || isinf(d)) ? CUDART_INF : __ddiv_rn(d, fabs(b));
    acc.max_abs = d > acc.max_abs ? d : acc.max_abs;
    acc.max_rel = r > acc.max_rel ? r : acc.max_rel;
    const bool mis = isinf(a) || isinf(b) || d > __dadd_rn(atol, __dmul_rn(rtol, fabs(b)));
    if (mis) {
        acc.mism += 1;
        acc.first = idx < acc.first ? idx : acc.first;
    }
}

// Synchronisation of the threads sharing a tile.
struct CtaSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct WarpSync {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};

// Queue of elements whose bits differ (shared memory).
struct SlowItem {
    unsigned long long idx;
    uint32_t g, w;
};
struct SlowQ {
    SlowItem *items;   // null: no queue, evaluate in place
    uint32_t *count;
    uint32_t cap;
};

template <int DT>
__device__ __forceinline__ void cmp_defer(const SlowQ &q, uint32_t gb, uint32_t wb, unsigned long long idx,
                                          double atol, double rtol, CmpAcc &acc) {
    if (q.items) {
        const uint32_t pos = atomicAdd(q.count, 1u);
        if (pos < q.cap) {
            q.items[pos] = SlowItem{idx, gb, wb};
            return;
        }
    }
    cmp_slow<DT>(gb, wb, idx, atol, rtol, acc);
}

// Evaluate the queued elements with all nthr threads; the caller
// synchronises its threads before (the queue is complete) and after (the
// queue may be reset).
template <int DT>
__device__ __forceinline__ void cmp_drain(const SlowQ &q, double atol, double rtol, CmpAcc &acc, uint32_t tid,
                                          uint32_t nthr) {
    if (!q.items) return;
    const uint32_t n = *q.count < q.cap ? *q.count : q.cap;
    for (uint32_t i = tid; i < n; i += nthr) {
        const SlowItem it = q.items[i];
        cmp_slow<DT>(it.g, it.w, it.idx, atol, rtol, acc);
    }
}

template <int DT>
__host__ __device__ constexpr int esize() {
    return DT == KC_F32 || DT == KC_I32 ? 4 : DT == KC_F16 || DT == KC_BF16 ? 2 : 1;
}

// Element j (0-based) of a 32-bit word.
template <int DT>
__device__ __forceinline__ uint32_t elem_of(uint32_t w, int j) {
    if (esize<DT>() == 4) return w;
    if (esize<DT>() == 2) return (w >> (16 * j)) & 0xffffu;
    return (w >> (8 * j)) & 0xffu;
}

// NaN elements of a word: the high bit of each element's slot set by one
// carry per element ((x & mag) + (mag - inf)) -- an element is NaN iff its
// magnitude exceeds the infinity pattern -- then counted.
template <int DT>
__device__ __forceinline__ uint32_t nan_bits(uint32_t w) {
    if (DT == KC_F32) return ((w & 0x7fffffffu) + 0x007fffffu) & 0x80000000u;
    if (DT == KC_BF16) return ((w & 0x7fff7fffu) + 0x007f007fu) & 0x80008000u;
    if (DT == KC_F16) return ((w & 0x7fff7fffu) + 0x03ff03ffu) & 0x80008000u;
    return 0u;
}

template <int DT>
__device__ __forceinline__ uint32_t vec_nans(const uint4 &v) {
    if (!(DT == KC_F32 || DT == KC_F16 || DT == KC_BF16)) return 0u;
    const uint32_t a = nan_bits<DT>(v.x), b = nan_bits<DT>(v.y), c = nan_bits<DT>(v.z), d = nan_bits<DT>(v.w);
    if ((a | b | c | d) == 0u) return 0u;
    return __popc(a) + __popc(b) + __popc(c) + __popc(d);
}

// NaNs in a word whose got and want bits are identical.
template <int DT>
__device__ __forceinline__ uint32_t word_nans(uint32_t w) {
    return __popc(nan_bits<DT>(w));
}

template <int DT>
__device__ __forceinline__ void cmp_word(uint32_t g, uint32_t w, unsigned long long first_elem,
                                         double atol, double rtol, CmpAcc &acc, const SlowQ &q) {
    constexpr int per = 4 / esize<DT>();
    if (g == w) {
        const uint32_t n = word_nans<DT>(g);
        acc.nan_g += n;
        acc.nan_w += n;
        return;
    }
#pragma unroll
    for (int j = 0; j < per; ++j) {
        const uint32_t ge = elem_of<DT>(g, j), we = elem_of<DT>(w, j);
        if (ge == we) {
            const uint32_t n = bits_nan<DT>(ge);
            acc.nan_g += n;
            acc.nan_w += n;
        } else {
            cmp_defer<DT>(q, ge, we, first_elem + j, atol, rtol, acc);
        }
    }
}

template <int DT>
__device__ __forceinline__ void cmp_vec(uint4 g, uint4 w, unsigned long long first_elem, double atol,
                                        double rtol, CmpAcc &acc, const SlowQ &q) {
    constexpr int per = 4 / esize<DT>();
    if (g.x == w.x && g.y == w.y && g.z == w.z && g.w == w.w) {
        const uint32_t n = vec_nans<DT>(g);
        acc.nan_g += n;
        acc.nan_w += n;
        return;
    }
    cmp_word<DT>(g.x, w.x, first_elem, atol, rtol, acc, q);
    cmp_word<DT>(g.y, w.y, first_elem + per, atol, rtol, acc, q);
    cmp_word<DT>(g.z, w.z, first_elem + 2 * per, atol, rtol, acc, q);
    cmp_word<DT>(g.w, w.w, first_elem + 3 * per, atol, rtol, acc, q);
}

// One tile of one pair, shared by `nthr` threads (tid = 0 .. nthr-1); each
// thread keeps U 16-byte loads of each buffer in flight (a CTA-wide tile
// needs few, a warp alone on a tile needs more to cover the DRAM latency).
// sync() synchronises the nthr threads; the tile ends by draining the queue.
template <int DT, int U, class Sync>
__device__ void cmp_tile(const CmpPair &pr, uint64_t tile_in_pair, double atol, double rtol, CmpAcc &acc,
                         uint32_t tid, uint32_t nthr, const SlowQ &q, Sync sync) {
    constexpr int ES = esize<DT>();
    const uint64_t nbytes = pr.nelem * ES;
    const uint64_t t0 = tile_in_pair * CMP_TILE_BYTES;
    const uint64_t tlen = nbytes - t0 < CMP_TILE_BYTES ? nbytes - t0 : CMP_TILE_BYTES;
    const uint8_t *g = reinterpret_cast<const uint8_t *>(pr.got) + t0;
    const uint8_t *w = reinterpret_cast<const uint8_t *>(pr.want) + t0;
    const uint64_t nvec = tlen >> 4;
    uint64_t v = tid;
    for (; v + (U - 1) * nthr < nvec; v += U * nthr) {
        uint4 gv[U], wv[U];
#pragma unroll
        for (int j = 0; j < U; ++j) {
            gv[j] = ldg_stream(g + 16 * (v + j * nthr));
            wv[j] = ldg_stream(w + 16 * (v + j * nthr));
        }
#pragma unroll
        for (int j = 0; j < U; ++j)
            cmp_vec<DT>(gv[j], wv[j], (t0 + 16 * (v + j * nthr)) / ES, atol, rtol, acc, q);
    }
    for (; v < nvec; v += nthr) {
        uint4 gv = ldg_stream(g + 16 * v), wv = ldg_stream(w + 16 * v);
        cmp_vec<DT>(gv, wv, (t0 + 16 * v) / ES, atol, rtol, acc, q);
    }
    // ragged end of the pair: fewer than 16 bytes, element by element
    const uint64_t tail0 = nvec << 4;
    for (uint64_t b = tail0 + (uint64_t)tid * ES; b < tlen; b += (uint64_t)nthr * ES) {
        uint32_t gb = 0, wb = 0;
        for (int j = 0; j < ES; ++j) {
            gb |= (uint32_t)g[b + j] << (8 * j);
            wb |= (uint32_t)w[b + j] << (8 * j);
        }
        if (gb == wb) {
            const uint32_t n = bits_nan<DT>(gb);
            acc.nan_g += n;
            acc.nan_w += n;
        } else {
            cmp_defer<DT>(q, gb, wb, (t0 + b) / ES, atol, rtol, acc);
        }
    }
    (void)sync;
}

// Drain the queue (elements of the pair of dtype dt) if it holds at least
// `min_items`: all nthr threads call it; returns with the queue empty or
// below that mark.  A queue is drained at the latest when the pair changes
// and when the caller's work ends (min_items = 1).
template <class Sync>
__device__ __forceinline__ void cmp_drain_any(int dt, const SlowQ &q, uint32_t min_items, double atol, double rtol,
                                              CmpAcc &acc, uint32_t tid, uint32_t nthr, Sync sync) {
    if (!q.items) return;
    sync();
    const uint32_t n = *q.count;
    sync();                      // every thread has read the count before any adds to it again
    if (n < min_items) return;   // uniform: every thread read the same count
    switch (dt) {
    case KC_F32: cmp_drain<KC_F32>(q, atol, rtol, acc, tid, nthr); break;
    case KC_F16: cmp_drain<KC_F16>(q, atol, rtol, acc, tid, nthr); break;
    case KC_BF16: cmp_drain<KC_BF16>(q, atol, rtol, acc, tid, nthr); break;
    case KC_I32: cmp_drain<KC_I32>(q, atol, rtol, acc, tid, nthr); break;
    default: cmp_drain<KC_U8>(q, atol, rtol, acc, tid, nthr); break;
    }
    sync();
    if (tid == 0) *q.count = 0;
    sync();
}

// ---- warp-streaming comparison -------------------------------------------------
//
// A warp streams blocks of 16-byte vectors of a pair (no block barriers;
// the kernel decides which blocks, k_compare.cu).  Equal vectors only have
// their NaNs counted (two bit tricks per word).  A vector whose bits differ
// is rare: it goes to the warp's queue in shared memory (one ballot per
// load, its slot from a popcount), and the warp evaluates queued vectors 32
// at a time, one per lane, with every lane busy, when the queue would
// overflow and when it leaves the pair.  With tolerances every differing
// element is evaluated in FP64; with zero tolerances FP64 runs only for the
// few elements that can hold the maxima (below).

__device__ __forceinline__ CmpAcc cmp_acc_zero() { return CmpAcc{0ull, ~0ull, 0ull, 0ull, 0ull, 0.0, 0.0}; }

struct VecItem {        // a queued vector: its index in the pair and both sides' bits
    unsigned long long v;
    uint4 g, w;
};

struct WarpQ {
    VecItem *items;     // this warp's slots in shared memory
    uint32_t cap;       // >= 32
    uint32_t n;         // queued vectors (the same in every lane)
    float run_abs;      // running maxima of the warp's proxies (the same in every lane)
    float run_rel;
    uint32_t *gate;     // the pair's proxy maxima over every warp (2 x fp32 bits, global), or null
};

// ---- zero tolerances: FP64 only where it can matter -------------------------
//
// An element whose bits differ is classified from its bits alone: both NaN
// (equal), one NaN (a mismatch, nan_mismatch), +0 against -0 (equal), or two
// unequal numbers.  With zero tolerances an unequal pair is always a
// mismatch (its FP64 difference is never zero: the difference of two
// distinct values of these types is at least 2^-149), so only the two
// maxima need FP64 -- and only for elements that can hold them.  Each
// element gets fp32 proxies of |a - b| and |a - b| / |b| (relative error
// below 2^-20, a subnormal reciprocal of |b| > 2^126 included; the integer
// types' difference is formed exactly first).  The warp keeps running
// maxima of its proxies and shares them through the pair's gate (a global
// maximum every warp of the grid reads and raises), and an element is
// evaluated in FP64 only if a proxy reaches the larger of the two times
// (1 - 2^-18), or is infinite or NaN.  An element below that threshold is
// smaller, exactly, than an element some warp has seen, so it cannot hold
// the exact FP64 maximum; by induction the element with the largest proxy
// is always evaluated, and the results are bit for bit those of evaluating
// every element.  (On this part a warp's FP64 instruction holds the FP64
// pipe for about sixteen cycles, so this matters: evaluating every
// differing element cost 0.4-0.7 ns of whole-GPU time each.)

constexpr float PROXY_KEEP = 1.0f - 1.0f / 262144.0f;   // 1 - 2^-18

template <int DT>
__device__ __forceinline__ float elem_float(uint32_t bits) {
    if (DT == KC_F32) return __uint_as_float(bits);
    if (DT == KC_BF16) return __uint_as_float(bits << 16);
    if (DT == KC_F16) return __half2float(__ushort_as_half((unsigned short)bits));
    if (DT == KC_I32) return (float)(int32_t)bits;
    return (float)bits;
}

// 0: equal (no contribution but NaN counts), 1: one side NaN, 2: unequal numbers.
template <int DT>
__device__ __forceinline__ int elem_class(uint32_t gb, uint32_t wb) {
    const bool na = bits_nan<DT>(gb), nb = bits_nan<DT>(wb);
    if (na && nb) return 0;
    if (na != nb) return 1;
    if (DT == KC_F32) return ((gb | wb) & 0x7fffffffu) == 0u ? 0 : 2;
    if (DT == KC_BF16 || DT == KC_F16) return ((gb | wb) & 0x7fffu) == 0u ? 0 : 2;
    return 2;
}

// Proxies of |a - b| and |a - b| / |b| for unequal numbers; +inf stands for
// an infinite or undefined one.
template <int DT>
__device__ __forceinline__ void elem_proxies(uint32_t gb, uint32_t wb, float &pa, float &pr) {
    float d;
    if (DT == KC_I32) d = (float)llabs((long long)(int32_t)gb - (long long)(int32_t)wb);
    else if (DT == KC_U8 || DT == KC_RAW) d = (float)(gb > wb ? gb - wb : wb - gb);
    else d = fabsf(elem_float<DT>(gb) - elem_float<DT>(wb));
    const float r = d * __frcp_rn(fabsf(elem_float<DT>(wb)));
    pa = d == d ? d : CUDART_INF_F;
    pr = r == r ? r : CUDART_INF_F;
}

// FP64 maxima of one pair of unequal numbers (one IEEE operation each).
template <int DT>
__device__ __forceinline__ void elem_maxima(uint32_t gb, uint32_t wb, CmpAcc &acc) {
    const double a = widen<DT>(gb), b = widen<DT>(wb);
    const double d = fabs(__dsub_rn(a, b));
    const double r = (b == 0.0 || isinf(d)) ? CUDART_INF : __ddiv_rn(d, fabs(b));
    acc.max_abs = d > acc.max_abs ? d : acc.max_abs;
    acc.max_rel = r > acc.max_rel ? r : acc.max_rel;
}

// ---- with tolerances: differing vectors queued, evaluated in FP64 ----------
//
// The mismatch test d > atol + rtol |b| needs every unequal element's FP64
// values, so differing vectors are queued per warp and evaluated 32 at a
// time with every lane busy (one FP64 sequence per element, none idle).

// One lane's queued vector.
template <int DT>
__device__ __forceinline__ void vec_eval(const VecItem &it, double atol, double rtol, CmpAcc &acc) {
    constexpr int per = 4 / esize<DT>();
    constexpr int PER = 16 / esize<DT>();
    const uint32_t gw[4] = {it.g.x, it.g.y, it.g.z, it.g.w}, ww[4] = {it.w.x, it.w.y, it.w.z, it.w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int j = 0; j < per; ++j) {
            const uint32_t ge = elem_of<DT>(gw[k], j), we = elem_of<DT>(ww[k], j);
            if (ge == we) {
                const uint32_t n = bits_nan<DT>(ge);
                acc.nan_g += n;
                acc.nan_w += n;
                continue;
            }
            cmp_slow<DT>(ge, we, it.v * PER + k * per + j, atol, rtol, acc);
        }
    }
}

// n queued vectors, 32 at a time; returns this lane's share of the accumulators.
template <int DT>
__device__ __noinline__ CmpAcc wq_eval(const VecItem *items, uint32_t n, double atol, double rtol) {
    CmpAcc a = cmp_acc_zero();
    __syncwarp();
    for (uint32_t i = lane_id(); i < n; i += 32) vec_eval<DT>(items[i], atol, rtol, a);
    __syncwarp();
    return a;
}

__device__ __forceinline__ void cmp_acc_merge(CmpAcc &a, const CmpAcc &b) {
    a.mism += b.mism;
    a.first = b.first < a.first ? b.first : a.first;
    a.nan_g += b.nan_g;
    a.nan_w += b.nan_w;
    a.nan_m += b.nan_m;
    a.max_abs = b.max_abs > a.max_abs ? b.max_abs : a.max_abs;
    a.max_rel = b.max_rel > a.max_rel ? b.max_rel : a.max_rel;
}


// ---- zero tolerances: queued differing vectors, classified in batches -------
//
// With atol == rtol == 0 an unequal element is a mismatch from its bits
// alone.  Differing vectors are queued per warp (as with tolerances) and
// evaluated 32 at a time, one per lane: each lane classifies its vector's
// elements (counts, first index, NaN rules) and takes the largest proxies;
// only when some lane's proxy reaches the warp's running threshold (the
// warp's and the pair's gate maxima times 1 - 2^-18) does the warp reduce
// the proxies, publish them to the gate, refresh the threshold and evaluate
// the elements still above it in FP64.  Such records are few (a running
// maximum over the pair).  (Classifying each differing vector where it was
// found instead cost its warp that latency in the middle of the stream:
// flipped MoE pair 33.3 against 29.4 us, 300k flips 85 against 48 us.)

// Lane-local pass over one differing vector: everything but the FP64
// maxima; ma / mr receive the largest proxies of its unequal numbers.
template <int DT>
__device__ __forceinline__ void vec_classify(const uint4 &g, const uint4 &w, unsigned long long v, CmpAcc &acc,
                                             float &ma, float &mr) {
    constexpr int per = 4 / esize<DT>();
    constexpr int PER = 16 / esize<DT>();
    const uint32_t gw[4] = {g.x, g.y, g.z, g.w}, ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (gw[k] == ww[k]) {
            const uint32_t n = __popc(nan_bits<DT>(gw[k]));
            acc.nan_g += n;
            acc.nan_w += n;
            continue;
        }
#pragma unroll
        for (int j = 0; j < per; ++j) {
            const uint32_t ge = elem_of<DT>(gw[k], j), we = elem_of<DT>(ww[k], j);
            const uint32_t ng = bits_nan<DT>(ge), nw = bits_nan<DT>(we);
            acc.nan_g += ng;
            acc.nan_w += nw;
            if (ge == we) continue;
            const int cls = elem_class<DT>(ge, we);
            if (cls == 0) continue;
            const unsigned long long idx = v * PER + k * per + j;
            acc.mism += 1;
            acc.first = idx < acc.first ? idx : acc.first;
            if (cls == 1) {
                acc.nan_m += 1;
                continue;
            }
            float pa, pr;
            elem_proxies<DT>(ge, we, pa, pr);
            ma = fmaxf(ma, pa);
            mr = fmaxf(mr, pr);
        }
    }
}

// FP64 maxima of the unequal numbers of one vector whose proxies reach the thresholds.
template <int DT>
__device__ __forceinline__ void vec_exact_max(const uint4 &g, const uint4 &w, float ta, float tr, CmpAcc &acc) {
    constexpr int per = 4 / esize<DT>();
    const uint32_t gw[4] = {g.x, g.y, g.z, g.w}, ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (gw[k] == ww[k]) continue;
#pragma unroll
        for (int j = 0; j < per; ++j) {
            const uint32_t ge = elem_of<DT>(gw[k], j), we = elem_of<DT>(ww[k], j);
            if (ge == we || elem_class<DT>(ge, we) != 2) continue;
            float pa, pr;
            elem_proxies<DT>(ge, we, pa, pr);
            if (!(pa < ta) || !(pr < tr)) elem_maxima<DT>(ge, we, acc);
        }
    }
}

// Zero tolerances: n queued vectors, 32 at a time with every lane busy --
// classified (vec_classify), then, only where a lane's proxy reaches the
// threshold, the warp maxima, the pair's gate and FP64.
// run: the warp's running proxy maxima, updated.
template <int DT>
__device__ __noinline__ CmpAcc wq_eval_zt(const VecItem *items, uint32_t n, float *run, uint32_t *gate) {
    const uint32_t FULL = 0xffffffffu;
    CmpAcc a = cmp_acc_zero();
    float ra = run[0], rr = run[1];
    __syncwarp();
    for (uint32_t b0 = 0; b0 < n; b0 += 32) {
        const uint32_t i = b0 + lane_id();
        const bool have = i < n;
        VecItem it{0ull, make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
        float ma = 0.0f, mr = 0.0f;
        if (have) {
            it = items[i];
            vec_classify<DT>(it.g, it.w, it.v, a, ma, mr);
        }
        const bool beat = ma > 0.0f && (!(ma < ra * PROXY_KEEP) || !(mr < rr * PROXY_KEEP));
        if (!__any_sync(FULL, beat)) continue;
        ra = fmaxf(ra, __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(ma))));
        rr = fmaxf(rr, __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(mr))));
        if (gate) {
            uint32_t ga = 0u, gr = 0u;
            if (lane_id() == 0) {
                ga = *reinterpret_cast<volatile uint32_t *>(gate);
                gr = *reinterpret_cast<volatile uint32_t *>(gate + 1);
                if (__float_as_uint(ra) > ga) atomicMax(gate, __float_as_uint(ra));
                if (__float_as_uint(rr) > gr) atomicMax(gate + 1, __float_as_uint(rr));
            }
            ra = fmaxf(ra, __uint_as_float(__shfl_sync(FULL, ga, 0)));
            rr = fmaxf(rr, __uint_as_float(__shfl_sync(FULL, gr, 0)));
        }
        if (have) vec_exact_max<DT>(it.g, it.w, ra * PROXY_KEEP, rr * PROXY_KEEP, a);
    }
    __syncwarp();
    run[0] = ra;
    run[1] = rr;
    return a;
}

template <int DT, bool ZT>
__device__ __forceinline__ void wq_drain(WarpQ &q, double atol, double rtol, CmpAcc &acc) {
    if (q.n == 0) return;
    if (ZT) {
        float run[2] = {q.run_abs, q.run_rel};
        cmp_acc_merge(acc, wq_eval_zt<DT>(q.items, q.n, run, q.gate));
        q.run_abs = run[0];
        q.run_rel = run[1];
    } else {
        cmp_acc_merge(acc, wq_eval<DT>(q.items, q.n, atol, rtol));
    }
    q.n = 0;
}

// One vector per lane (vector index v, `differs` when its bits differ):
// NaNs of equal vectors are counted; differing ones are queued (evaluated
// by wq_eval_zt with zero tolerances, ZT, else by wq_eval).  All lanes call it.
template <int DT, bool ZT>
__device__ __forceinline__ void vec_step(WarpQ &q, const uint4 &g, const uint4 &w, unsigned long long v,
                                         bool valid, double atol, double rtol, CmpAcc &acc) {
    const bool differs = valid && (g.x != w.x || g.y != w.y || g.z != w.z || g.w != w.w);
    if (valid && !differs) {
        const uint32_t n = vec_nans<DT>(g);
        acc.nan_g += n;
        acc.nan_w += n;
    }
    const uint32_t b = __ballot_sync(0xffffffffu, differs);
    if (b == 0u) return;
    if (q.n + 32 > q.cap) wq_drain<DT, ZT>(q, atol, rtol, acc);
    if (differs) q.items[q.n + __popc(b & lanemask_lt())] = VecItem{v, g, w};
    q.n += __popc(b);
}

// Vectors [va, vb) of a pair (16-byte units from its start), U loads of
// each buffer in flight per lane; all 32 lanes call it.
template <int DT, int U, bool ZT>
__device__ __forceinline__ void warp_compare_range(const CmpPair &pr, uint64_t va, uint64_t vb, double atol,
                                                   double rtol, CmpAcc &acc, WarpQ &q) {
    const uint8_t *g = reinterpret_cast<const uint8_t *>(pr.got);
    const uint8_t *w = reinterpret_cast<const uint8_t *>(pr.want);
    const uint64_t lane = lane_id();
    uint64_t v = va;
    for (; v + 32 * U <= vb; v += 32 * U) {
        uint4 gv[U], wv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            gv[u] = ldg_stream(g + 16 * (v + 32 * u + lane));
            wv[u] = ldg_stream(w + 16 * (v + 32 * u + lane));
        }
        if (ZT) {
            // one vote per block; the rare handling appears once in the code
            uint32_t dm = 0u;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool d = gv[u].x != wv[u].x || gv[u].y != wv[u].y || gv[u].z != wv[u].z || gv[u].w != wv[u].w;
                if (!d) {
                    const uint32_t n = vec_nans<DT>(gv[u]);
                    acc.nan_g += n;
                    acc.nan_w += n;
                }
                dm |= (uint32_t)d << u;
            }
            if (__any_sync(0xffffffffu, dm != 0u)) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool d = (dm >> u) & 1u;
                    const uint32_t b = __ballot_sync(0xffffffffu, d);
                    if (b == 0u) continue;
                    if (q.n + 32 > q.cap) wq_drain<DT, true>(q, atol, rtol, acc);
                    if (d) q.items[q.n + __popc(b & lanemask_lt())] = VecItem{v + 32 * u + lane, gv[u], wv[u]};
                    q.n += __popc(b);
                }
            }
        } else {
#pragma unroll
            for (int u = 0; u < U; ++u) vec_step<DT, ZT>(q, gv[u], wv[u], v + 32 * u + lane, true, atol, rtol, acc);
        }
    }
    for (; v < vb; v += 32) {
        const bool ok = v + lane < vb;
        uint4 gv = make_uint4(0, 0, 0, 0), wv = gv;
        if (ok) {
            gv = ldg_stream(g + 16 * (v + lane));
            wv = ldg_stream(w + 16 * (v + lane));
        }
        vec_step<DT, ZT>(q, gv, wv, v + lane, ok, atol, rtol, acc);
    }
}

// The < 16-byte end of a pair, element by element (lane e takes element e).
template <int DT>
__device__ __forceinline__ void warp_compare_tail(const CmpPair &pr, double atol, double rtol, CmpAcc &acc,
                                                  WarpQ &) {
    constexpr int ES = esize<DT>();
    const uint64_t nbytes = pr.nelem * ES;
    const uint64_t b = (nbytes & ~15ull) + (uint64_t)lane_id() * ES;
    if (b >= nbytes) return;
    const uint8_t *g = reinterpret_cast<const uint8_t *>(pr.got) + b;
    const uint8_t *w = reinterpret_cast<const uint8_t *>(pr.want) + b;
    uint32_t gb = 0, wb = 0;
    for (int j = 0; j < ES; ++j) {
        gb |= (uint32_t)g[j] << (8 * j);
        wb |= (uint32_t)w[j] << (8 * j);
    }
    if (gb == wb) {
        const uint32_t n = bits_nan<DT>(gb);
        acc.nan_g += n;
        acc.nan_w += n;
    } else {
        cmp_slow<DT>(gb, wb, b / ES, atol, rtol, acc);
    }
}

__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

// Reduce a warp's accumulators and merge them into the pair's record with
// order-independent atomics (lane 0).
__device__ __forceinline__ void cmp_warp_flush(const CmpAcc &acc, kc_cmp_result *o) {
    unsigned long long v[7] = {acc.mism, acc.first, acc.nan_g, acc.nan_w, acc.nan_m, dbits(acc.max_abs),
                               dbits(acc.max_rel)};
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
        if (v[0]) atomicAdd(reinterpret_cast<unsigned long long *>(&o->mismatches), v[0]);
        if (v[1] != ~0ull) atomicMin(reinterpret_cast<unsigned long long *>(&o->first), v[1]);
        if (v[2]) atomicAdd(reinterpret_cast<unsigned long long *>(&o->nan_got), v[2]);
        if (v[3]) atomicAdd(reinterpret_cast<unsigned long long *>(&o->nan_want), v[3]);
        if (v[4]) atomicAdd(reinterpret_cast<unsigned long long *>(&o->nan_mismatch), v[4]);
        if (v[5]) atomicMax(reinterpret_cast<unsigned long long *>(&o->max_abs), v[5]);
        if (v[6]) atomicMax(reinterpret_cast<unsigned long long *>(&o->max_rel), v[6]);
    }
}

// Comparison of one tile by `nthr` threads, dispatched on the pair's dtype.
template <int U, class Sync>
__device__ __forceinline__ void cmp_tile_any(const CmpPair &pr, uint64_t tile, double atol, double rtol, CmpAcc &acc,
                                             uint32_t tid, uint32_t nthr, const SlowQ &q, Sync sync) {
    switch (pr.dtype) {
    case KC_F32: cmp_tile<KC_F32, U>(pr, tile, atol, rtol, acc, tid, nthr, q, sync); break;
    case KC_F16: cmp_tile<KC_F16, U>(pr, tile, atol, rtol, acc, tid, nthr, q, sync); break;
    case KC_BF16: cmp_tile<KC_BF16, U>(pr, tile, atol, rtol, acc, tid, nthr, q, sync); break;
    case KC_I32: cmp_tile<KC_I32, U>(pr, tile, atol, rtol, acc, tid, nthr, q, sync); break;
    default: cmp_tile<KC_U8, U>(pr, tile, atol, rtol, acc, tid, nthr, q, sync); break;
    }
}

__device__ __forceinline__ void cmp_record_init(kc_cmp_result *o, int32_t status) {
    kc_cmp_result r;
    r.mismatches = 0;
    r.first = -1;
    r.max_abs = 0.0;
    r.max_rel = 0.0;
    r.nan_got = 0;
    r.nan_want = 0;
    r.nan_mismatch = 0;
    r.status = status;
    r.reserved = 0;
    *o = r;
}

}  // namespace kc
