// kc_device.cuh -- device helpers: warp utilities, asynchronous copies into
// shared memory, XXH64 pieces, census classification.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kc_internal.cuh"

namespace kc {

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the kernel before it in the stream is still
// running; grid_dep_wait() returns once that kernel has completed and its
// writes are visible (at once when there is no such kernel), and
// grid_dep_launch() lets the next such kernel be scheduled before this one
// ends.  Both are no-ops for launches without the attribute.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Per-thread asynchronous 16-byte copy global -> shared (both 16-byte
// aligned), and its commit / wait groups.
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src_gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst_smem)), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// Wait until at most `n` (0..7) of this thread's committed groups are pending.
__device__ __forceinline__ void cp_async_wait(int n) {
    switch (n) {
    case 0: asm volatile("cp.async.wait_group 0;" ::: "memory"); break;
    case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
    case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
    case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
    case 4: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
    case 5: asm volatile("cp.async.wait_group 5;" ::: "memory"); break;
    case 6: asm volatile("cp.async.wait_group 6;" ::: "memory"); break;
    default: asm volatile("cp.async.wait_group 7;" ::: "memory"); break;
    }
}

// ---- mbarriers and bulk copies (shared memory of this CTA) --------------------
//
// A stage of a ring is guarded by two mbarriers with one arrival each:
// "full" (the producer arrives with the stage's byte count; the bulk copies
// complete the transaction) and "empty" (the consumer arrives when it has
// read the stage).  Waits poll try_wait with a phase parity and give up
// after `limit` polls or when *abort is set, so no wait can hang a kernel.

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
// Makes initialised barriers visible to the asynchronous (bulk copy) proxy.
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// As mbar_test, but a thread whose phase has not completed is suspended by
// the hardware until it completes or about `hint_ns` nanoseconds pass, so a
// waiting warp takes no issue slots from the warps doing the work.
__device__ __forceinline__ bool mbar_test_sleep(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
// Wait until the phase of parity `parity` has completed; false if the wait
// gave up (after `limit` suspended polls of up to ~64 us each, or when
// *abort was set by another warp).
constexpr uint32_t MBAR_SLEEP_NS = 1u << 16;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit,
                                          const volatile uint32_t *abort) {
    for (uint32_t i = 0; i < limit; ++i) {
        if (mbar_test_sleep(bar, parity, MBAR_SLEEP_NS)) return true;
        if (*abort) return false;
    }
    return false;
}
// The barrier's current phase also waits for every cp.async this thread has
// issued so far: its pending count rises by one now and falls by one when
// those copies have landed.
__device__ __forceinline__ void mbar_track_cp_async(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One bulk copy global -> this CTA's shared memory, completing `bytes` of
// the barrier's transaction.  dst and src 16-byte aligned, bytes a multiple
// of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void set_status(uint32_t *status, uint32_t bits) {
    if (status) atomicOr(status, bits);
}

// ---- loads ------------------------------------------------------------------

__device__ __forceinline__ uint4 ldg_stream(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint64_t ldg_u64(const void *p) {
    return __ldg(reinterpret_cast<const unsigned long long *>(p));
}

// ---- region lookup ----------------------------------------------------------

// Region holding flattened unit `u`: the last region whose first unit <= u.
__device__ __forceinline__ int region_of(const Region *r, int n, uint64_t u) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(reinterpret_cast<const unsigned long long *>(&r[mid].first)) <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---- census classification ---------------------------------------------------

// Classify word v against the sorted ranges `rg` (shared or global memory):
// 0 = not a hit, 1 = inside (target in *tgt), 2 = outside.
__device__ __forceinline__ int census_classify(const CensusArgs &ca, const Range *rg, uint64_t v, int32_t *tgt) {
    const bool in_span = (v - ca.span_lo) < ca.span_len;
    const bool in_win = (v - ca.win_lo) < ca.win_len;
    if (!(in_span || in_win)) return 0;
    if (in_span) {
        // first range with base > v, then check the one before it
        int lo = 0, hi = ca.nranges;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (rg[mid].base <= v) lo = mid + 1;
            else hi = mid;
        }
        if (lo > 0 && v < rg[lo - 1].end) {
            *tgt = rg[lo - 1].id;
            return 1;
        }
    }
    if (in_win) {
        *tgt = -1;
        return 2;
    }
    return 0;
}

// Ranges held in shared memory by the census kernels when they fit.
constexpr int SMEM_RANGES = 1024;

// Copy the ranges into `buf` (SMEM_RANGES entries) if they fit; every thread
// of the CTA must call it.  Returns the array to search.
__device__ __forceinline__ const Range *stage_ranges(const CensusArgs &ca, Range *buf) {
    if (ca.nranges > SMEM_RANGES) return ca.ranges;
    for (int i = threadIdx.x; i < ca.nranges; i += blockDim.x) buf[i] = ca.ranges[i];
    __syncthreads();
    return buf;
}

// Conservative pre-filter: can v be a census hit at all?
__device__ __forceinline__ uint32_t census_pre(const CensusArgs &ca, uint64_t v) {
    return (uint32_t)(v >> 32) - ca.pre_lo;   // candidate iff result <= ca.pre_span
}

// ---- XXH64 (public xxHash specification) -------------------------------------

constexpr uint64_t XXP1 = 0x9E3779B185EBCA87ULL;
constexpr uint64_t XXP2 = 0xC2B2AE3D27D4EB4FULL;
constexpr uint64_t XXP3 = 0x165667B19E3779F9ULL;
constexpr uint64_t XXP4 = 0x85EBCA77C2B2AE63ULL;
constexpr uint64_t XXP5 = 0x27D4EB2F165667C5ULL;

__device__ __forceinline__ uint64_t rotl(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

// Accumulator step for one 8-byte lane of a stripe.
__device__ __forceinline__ uint64_t xx_round(uint64_t acc, uint64_t lane) {
    return rotl(acc + lane * XXP2, 31) * XXP1;
}

// ---- the lane chain in "pre-rotate" form ---------------------------------------
//
// One XXH64 round is acc' = rotl(acc + m, 31) * PRIME1 with m = lane *
// PRIME2.  Carrying t = acc + m instead of acc gives t' = rotl(t, 31) *
// PRIME1 + m', and the low product with m' added is a single 32 x 32 -> 64
// multiply-add, so a round is two funnel shifts, three multiplies and an
// add, four dependent steps (same value mod 2^64 as the round above).  The
// chain starts from the t whose step yields the specification's initial
// accumulator, t0 = rotr(acc0 * PRIME1^-1, 31) (PRIME1 is odd, so it is
// invertible mod 2^64), and ends with acc = rotl(t, 31) * PRIME1.

constexpr uint64_t inv_odd(uint64_t a) {   // a^-1 mod 2^64 by Newton's iteration, a odd
    uint64_t x = a;                          // correct to 3 bits: a * a == 1 mod 8
    for (int i = 0; i < 6; ++i) x *= 2 - a * x;
    return x;
}
constexpr uint64_t XXP1_INV = inv_odd(XXP1);
static_assert(XXP1 * XXP1_INV == 1, "PRIME1 inverse");
constexpr uint64_t rotr_c(uint64_t x, int r) { return (x >> r) | (x << (64 - r)); }
constexpr uint64_t xx_t0(uint64_t acc0) { return rotr_c(acc0 * XXP1_INV, 31); }

__device__ __forceinline__ uint64_t xx_t_init(int k) {
    return k == 0 ? xx_t0(XXP1 + XXP2) : k == 1 ? xx_t0(XXP2) : k == 2 ? xx_t0(0ULL) : xx_t0(0ULL - XXP1);
}

// t' = rotl(t, 31) * PRIME1 + m  (mod 2^64)
__device__ __forceinline__ uint64_t xx_t_step(uint64_t t, uint64_t m) {
    uint32_t olo, ohi;
    asm("{\n\t.reg .u32 rl, rh, x;\n\t.reg .u64 w, mm;\n\t"
        "shf.l.wrap.b32 rh, %2, %3, 31;\n\t"
        "shf.l.wrap.b32 rl, %3, %2, 31;\n\t"
        "mov.b64 mm, {%4, %5};\n\t"
        "mad.wide.u32 w, rl, 0x85EBCA87, mm;\n\t"
        "mul.lo.u32 x, rl, 0x9E3779B1;\n\t"
        "mad.lo.u32 x, rh, 0x85EBCA87, x;\n\t"
        "mov.b64 {%0, %1}, w;\n\t"
        "add.u32 %1, %1, x;\n\t}"
        : "=r"(olo), "=r"(ohi)
        : "r"((uint32_t)t), "r"((uint32_t)(t >> 32)), "r"((uint32_t)m), "r"((uint32_t)(m >> 32)));
    return ((uint64_t)ohi << 32) | olo;
}

__device__ __forceinline__ uint64_t xx_t_final(uint64_t t) { return rotl(t, 31) * XXP1; }

}  // namespace kc
