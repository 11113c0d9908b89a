// kc_noalloc.cu -- kc_census_static: the pointer census for callers that
// cannot allocate device memory.
//
// Some callers of a snapshot library must not call cudaMalloc (or anything
// that allocates): a hook that runs inside the application's own allocator
// or memory-tracking callback, where allocating re-enters the code being
// observed; a handler that snapshots device memory after a failure, when a
// new allocation may itself fail or disturb the state being captured; or a
// process whose device memory is entirely reserved by another runtime.  The
// regular kc_census keeps its region tables and per-chunk counters in
// context-owned device memory, so it cannot serve them.
//
// kc_census_static runs the same census kernels, but all of its scratch --
// the region table, the sorted ranges, the per-chunk hit counts and their
// offsets, a status word -- lives in one file-scope static device array that
// is part of this file's module: a device holds it (about 0.8 MiB) from the
// moment the module is loaded there until the process exits, and no call
// allocates anything.  Host code cannot pass the array's name to a kernel
// (in host code it is a host-side stand-in, not a device address), so the
// set-up of each device looks up its device address with
// cudaGetSymbolAddress while that device is current, and every later call
// on that device reuses it.
//
// Module loading is lazy by default in CUDA: a module's code and static
// data are put on the device when first used, which itself takes device
// memory.  The set-up therefore also loads every kernel a census call
// launches (one launch each with no work), so that calls made after it load
// nothing.  The set-up runs on the first call on a device, or explicitly
// with kc_census_static(NULL, 0, ...), which does only the set-up.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "kc_internal.cuh"

using namespace kc;

namespace {

constexpr int NA_MAX_REGIONS = 1024;          // regions per call
constexpr uint64_t NA_MAX_UNITS = 65536;      // 64 KiB census chunks per call
constexpr uint32_t NA_UNIT = 64 * 1024;
constexpr int NA_MAX_DEVICES = 64;

// Layout of the static scratch array.
constexpr size_t NA_OFF_REGIONS = 0;
constexpr size_t NA_OFF_RANGES = NA_OFF_REGIONS + NA_MAX_REGIONS * sizeof(Region);
constexpr size_t NA_OFF_HITS = NA_OFF_RANGES + NA_MAX_REGIONS * sizeof(Range);
constexpr size_t NA_OFF_OFFS = NA_OFF_HITS + NA_MAX_UNITS * sizeof(uint32_t);
constexpr size_t NA_OFF_STATUS = NA_OFF_OFFS + NA_MAX_UNITS * sizeof(uint64_t);
constexpr size_t NA_BYTES = NA_OFF_STATUS + 256;

}  // namespace

// The scratch itself: one copy per device on which this module is loaded.
static __device__ __align__(256) unsigned char g_census_scratch[NA_BYTES];

namespace {

// Last kernel of a call: if the write pass found a chunk whose recount
// differs from its first count -- which happens when another call
// overwrote the shared scratch in between -- both counts become all-ones,
// a value no census can produce, so the caller sees that the call's hits
// are not to be trusted.
__global__ void census_static_finish_kernel(const uint32_t *__restrict__ status, uint64_t *__restrict__ counts) {
    if (status && counts && (*status & ST_INTERNAL)) {
        counts[0] = ~0ull;
        counts[1] = ~0ull;
    }
}

struct DeviceScratch {
    std::once_flag once;
    cudaError_t err = cudaSuccess;
    unsigned char *ptr = nullptr;   // device address of g_census_scratch on this device
    int sms = 0;
};

DeviceScratch g_dev[NA_MAX_DEVICES];

// One-time set-up on the current device: the array's device address, the
// SM count, and every kernel of the call loaded (empty launches on `st`).
// None of it allocates once the module is loaded; loading it is the one
// moment device memory is taken.
DeviceScratch *scratch_for(int device, cudaStream_t st) {
    DeviceScratch &d = g_dev[device];
    std::call_once(d.once, [&d, device, st]() {
        void *p = nullptr;
        cudaFuncAttributes fa;
        d.err = cudaGetSymbolAddress(&p, g_census_scratch);
        if (d.err == cudaSuccess) d.err = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, device);
        if (d.err == cudaSuccess) d.err = cudaFuncGetAttributes(&fa, census_static_finish_kernel);
        if (d.err == cudaSuccess) {
            census_static_finish_kernel<<<1, 1, 0, st>>>(nullptr, nullptr);
            count_launches(1);
            d.err = cudaGetLastError();
        }
        if (d.err == cudaSuccess) d.err = preload_census_kernels(st);
        if (d.err == cudaSuccess) d.ptr = static_cast<unsigned char *>(p);
        else cudaGetLastError();
    });
    return d.err == cudaSuccess ? &d : nullptr;
}

uint32_t log2u32(uint32_t v) {
    uint32_t r = 0;
    while ((1u << r) < v) ++r;
    return r;
}

// Host-side tables, file-scope so a call allocates no host memory either;
// g_host_lock serialises their use by concurrent host threads.
std::mutex g_host_lock;
Region g_h_regions[NA_MAX_REGIONS];
Range g_h_ranges[NA_MAX_REGIONS];

}  // namespace

extern "C" {

KC_API kc_status kc_census_static(const kc_buf *allocs, int n, uint64_t win_lo, uint64_t win_hi, kc_hit *d_hits,
                                  uint64_t cap, uint64_t *d_counts, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool setup_only = allocs == nullptr && n == 0;
    if (!setup_only && (!allocs || n < 1 || n > NA_MAX_REGIONS || !d_counts || (cap && !d_hits))) return KC_EINVAL;
    std::lock_guard<std::mutex> hold(g_host_lock);
    Region *regions = g_h_regions;
    Range *ranges = g_h_ranges;
    uint64_t units = 0;
    bool any_lost = false;
    for (int i = 0; i < n; ++i) {
        const kc_buf &b = allocs[i];
        if (b.bytes == 0 || (b.base_va & 15) || b.dtype < KC_U8 || b.dtype > KC_RAW ||
            b.base_va + b.bytes < b.base_va)
            return KC_EINVAL;
        regions[i] = Region{b.base_va, b.bytes, units, (b.flags & KC_BUF_LOST) ? 1u : 0u, 0u};
        any_lost |= (b.flags & KC_BUF_LOST) != 0;
        ranges[i] = Range{b.base_va, b.base_va + b.bytes, i, 0};
        units += (b.bytes + NA_UNIT - 1) / NA_UNIT;
    }
    if (units > NA_MAX_UNITS) return KC_EINVAL;   // more than the static counters hold
    std::sort(ranges, ranges + n, [](const Range &x, const Range &y) { return x.base < y.base; });
    for (int i = 1; i < n; ++i)
        if (ranges[i].base < ranges[i - 1].end) return KC_EOVERLAP;

    // The host tables above are shared by every call and copied with plain
    // asynchronous copies: a captured copy would read them again at every
    // replay, after later calls have rewritten them, so capture is refused.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return KC_ECUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) return KC_EINVAL;

    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= NA_MAX_DEVICES) {
        cudaGetLastError();
        return KC_ECUDA;
    }
    DeviceScratch *ds = scratch_for(device, st);
    if (!ds) return KC_ECUDA;
    if (setup_only) return KC_OK;
    Region *d_regions = reinterpret_cast<Region *>(ds->ptr + NA_OFF_REGIONS);
    Range *d_ranges = reinterpret_cast<Range *>(ds->ptr + NA_OFF_RANGES);
    uint32_t *unit_hits = reinterpret_cast<uint32_t *>(ds->ptr + NA_OFF_HITS);
    uint64_t *unit_off = reinterpret_cast<uint64_t *>(ds->ptr + NA_OFF_OFFS);
    uint32_t *status = reinterpret_cast<uint32_t *>(ds->ptr + NA_OFF_STATUS);

    // The tables are copied from host memory into the static array (the
    // runtime stages pageable memory itself; nothing is allocated here).
    // Every count the kernels accumulate starts at zero: the caller's two
    // counters and the status word; unit_hits is written whole by the count
    // kernel and unit_off by the scan.
    CensusArgs ca = census_args(ranges, n, win_lo, win_hi);
    ca.ranges = d_ranges;
    Pages u;
    u.regions = d_regions;
    u.nregions = n;
    u.npages = units;
    u.page = NA_UNIT;
    u.log2page = log2u32(NA_UNIT);
    if (cudaMemcpyAsync(d_regions, regions, n * sizeof(Region), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_ranges, ranges, n * sizeof(Range), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(status, 0, sizeof(uint32_t), st) != cudaSuccess ||
        cudaMemsetAsync(d_counts, 0, 2 * sizeof(uint64_t), st) != cudaSuccess ||
        launch_census_count(u, ca, unit_hits, d_counts, ds->sms, st) != cudaSuccess) {
        cudaGetLastError();
        return KC_ECUDA;
    }
    if (cap) {
        if (launch_scan_u32(unit_hits, unit_off, units, nullptr, st) != cudaSuccess ||
            launch_census_write(u, ca, unit_hits, unit_off, d_hits, cap, status, ds->sms, st) != cudaSuccess) {
            cudaGetLastError();
            return KC_ECUDA;
        }
        census_static_finish_kernel<<<1, 1, 0, st>>>(status, d_counts);
        count_launches(1);
        if (cudaGetLastError() != cudaSuccess) return KC_ECUDA;
    }
    return any_lost ? KC_EBUF : KC_OK;
}

}  // extern "C"
