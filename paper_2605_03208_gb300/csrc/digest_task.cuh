// digest_task.cuh -- XXH64 (seed 0) of pages held in shared memory, their
// zero flags and (optionally) their census pre-filter flags: the hashing
// body shared by the digest kernel (stages filled by a producer warp with
// bulk copies, k_digest.cu) and the batched kernel (each warp filling its
// own ring with per-thread asynchronous copies, digest_pages below).
//
// XXH64 keeps four serial accumulators, one per 8-byte lane of every 32-byte
// stripe.  With LPT lanes per thread, a page is hashed by TPP = 4 / LPT
// threads and a warp holds PPW = 32 / TPP pages.  Page slots in a stage are
// padded by 32 bytes so the pages' shared loads spread over all 32 banks.
// The < 32-byte tail of a page is read from global memory by the page
// leader while it finishes.
//
// The serial chain per accumulator is the critical path; it is carried in
// pre-rotate form (xx_t_step: two funnel shifts, a 32 x 32 -> 64
// multiply-add, two 32-bit multiplies and an add), and the lane products
// (lane * PRIME2) and the next stripes' shared loads are issued ahead of it.
// CHUNK (compile-time, 0 = none) gives full chunks of that size a fully
// unrolled path.
//
// Zero flag: one 32-bit OR of both halves of every word.  Census
// pre-filter: the minimum over words of (high 32 bits - pre_lo), taken
// pairwise, a branch-free conservative test of whether any word can be a
// census hit.
#pragma once

#include "kc_device.cuh"

namespace kc {

struct PageDigest {
    uint64_t hash;
    bool zero;   // every byte is 0
    bool cand;   // some word passed the census pre-filter
};

// One thread's share of a page being hashed: its XXH64 lanes (pre-rotate
// form), the OR of its words' halves and its census pre-filter minimum.
template <int LPT>
struct PageLanes {
    uint64_t acc[LPT];
    uint32_t zor32;
    uint32_t cmin;
};

// j: this thread's position among the page's threads (lanes j*LPT ..).
template <int LPT>
__device__ __forceinline__ void lanes_init(PageLanes<LPT> &L, int j) {
#pragma unroll
    for (int i = 0; i < LPT; ++i) L.acc[i] = xx_t_init(j * LPT + i);
    L.zor32 = 0;
    L.cmin = 0xFFFFFFFFu;
}

// Hash b bytes (a multiple of 32) of one page held in shared memory.
// `slot` is where those bytes start, plus this thread's lane offset
// (8 * LPT * j).
template <bool CENSUS, int LPT, int CHUNK>
__device__ __forceinline__ void hash_chunk(PageLanes<LPT> &L, const uint8_t *slot, uint32_t b,
                                           const CensusArgs &ca) {
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
            L.zor32 |= (uint32_t)w[i] | (uint32_t)(w[i] >> 32);
            if (CENSUS) L.cmin = min(L.cmin, census_pre(ca, w[i]));
        }
    };
    auto group = [&](const uint64_t (&w)[4][LPT]) {
        uint64_t m[4][LPT];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < LPT; ++i) m[u][i] = w[u][i] * XXP2;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int i = 0; i < LPT; ++i) L.acc[i] = xx_t_step(L.acc[i], m[u][i]);
#pragma unroll
        for (int i = 0; i < LPT; ++i) {
#pragma unroll
            for (int u = 0; u < 4; ++u) L.zor32 |= (uint32_t)w[u][i] | (uint32_t)(w[u][i] >> 32);
            if (CENSUS)
                L.cmin = min(L.cmin, min(min(census_pre(ca, w[0][i]), census_pre(ca, w[1][i])),
                                         min(census_pre(ca, w[2][i]), census_pre(ca, w[3][i]))));
        }
    };
    uint32_t s = 0;
    if (CHUNK && b == (uint32_t)CHUNK) {
        // a full chunk of compile-time size: fully unrolled, the loads of
        // the next four stripes issued ahead of the chains
        uint64_t w[4][LPT];
#pragma unroll
        for (int u = 0; u < 4; ++u) ld(32 * u, w[u]);
#pragma unroll
        for (int g = 0; g < (CHUNK ? CHUNK : 128) / 128; ++g) {
            uint64_t nw[4][LPT];
            if (g + 1 < CHUNK / 128) {
#pragma unroll
                for (int u = 0; u < 4; ++u) ld(128 * (g + 1) + 32 * u, nw[u]);
            }
            group(w);
            if (g + 1 < CHUNK / 128) {
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int i = 0; i < LPT; ++i) w[u][i] = nw[u][i];
            }
        }
        s = b;
    } else if (b >= 128) {
        // register double buffer: the next four stripes are loaded while
        // the current four run through the chains
        uint64_t w[4][LPT];
#pragma unroll
        for (int u = 0; u < 4; ++u) ld(32 * u, w[u]);
        for (; s + 128 <= b; s += 128) {
            const uint32_t ns = (s + 256 <= b) ? s + 128 : s;   // last group reloads itself
            uint64_t nw[4][LPT];
#pragma unroll
            for (int u = 0; u < 4; ++u) ld(ns + 32 * u, nw[u]);
            group(w);
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
        for (int i = 0; i < LPT; ++i) L.acc[i] = xx_t_step(L.acc[i], w[i] * XXP2);
        eat(w);
    }
}

// All 32 lanes of the warp call this together, each with its page (src,
// len, lost; len 0 for a slot without a page) after hashing the page's
// full stripes: the page's accumulators are gathered in its leader (the
// thread whose lane % TPP == 0), which hashes the < 32-byte tail from
// global memory and finishes.  The result is valid in the leader.
template <bool CENSUS, int LPT>
__device__ __forceinline__ PageDigest finish_page(PageLanes<LPT> &L, const uint8_t *src, uint64_t len, bool lost,
                                                  const CensusArgs &ca) {
    constexpr int TPP = 4 / LPT;
    const uint32_t FULL = 0xffffffffu;
    const uint32_t lane = lane_id();
    const int j = lane % TPP;
    uint64_t acc[LPT];
#pragma unroll
    for (int i = 0; i < LPT; ++i) acc[i] = xx_t_final(L.acc[i]);
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
    uint64_t zor = L.zor32;
    uint32_t cmin = L.cmin;
#pragma unroll
    for (int o = 1; o < TPP; o <<= 1) {
        zor |= __shfl_xor_sync(FULL, zor, o);
        if (CENSUS) cmin = min(cmin, __shfl_xor_sync(FULL, cmin, o));
    }
    PageDigest r{0, false, false};
    if (j != 0 || lost) return r;
    const uint32_t sbytes = (uint32_t)(len & ~31ull);
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
    r.hash = h;
    r.zero = zor == 0;
    r.cand = CENSUS && cmin <= ca.pre_span && len >= 8;
    return r;
}

// A warp hashes its pages streaming them through its own ring of `stages`
// shared-memory stages (a stage holds one `chunk` of each page): the
// threads of a page copy its chunk with per-thread 16-byte asynchronous
// copies (cp.async), one commit group per stage, and wait for the group
// (and the warp) before hashing it.  All 32 lanes call this together, each
// passing its page: src/len (len 0 for a slot without a page) and lost (not
// readable: no bytes are touched).  The result is valid in the page leader.
template <bool CENSUS, int LPT, int CHUNK>
__device__ __forceinline__ PageDigest digest_pages(uint8_t *ring, int stages, int chunk, const uint8_t *src,
                                                   uint64_t len, bool lost, const CensusArgs &ca) {
    constexpr int TPP = 4 / LPT;    // threads per page
    constexpr int PPW = 32 / TPP;   // pages per warp
    const uint32_t FULL = 0xffffffffu;
    const uint32_t lane = lane_id();
    const int q = lane / TPP;       // page slot of this thread
    const int j = lane % TPP;       // this thread owns lanes j*LPT .. j*LPT+LPT-1
    const size_t slot_stride = (size_t)chunk + 32;
    const size_t stage_stride = PPW * slot_stride;

    const uint32_t sbytes = lost ? 0u : (uint32_t)(len & ~31ull);   // bytes in full stripes
    const uint32_t nch = (sbytes + chunk - 1) / chunk;
    const uint32_t maxch = __reduce_max_sync(FULL, nch);

    // Copy chunk c of this thread's page into stage c % stages: the page's
    // threads split its 16-byte pieces (a copy pattern that keeps the
    // warp's instruction stream short: taking each page with all 32 lanes
    // instead, for 512 contiguous bytes per instruction, measured slower
    // here, from the extra registers and instructions per page).  Every
    // thread commits one group per call (empty past the page's end), so
    // group counts agree.
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

    PageLanes<LPT> L;
    lanes_init(L, j);
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
        hash_chunk<CENSUS, LPT, CHUNK>(L, ring + st * stage_stride + q * slot_stride + 8 * LPT * j, b, ca);
        __syncwarp();                 // the stage is free for the next refill
    }
    cp_async_wait(0);                 // trailing (empty) groups
    return finish_page<CENSUS, LPT>(L, src, len, lost, ca);
}

}  // namespace kc
