// kc_vmm.cu -- exact-VA reservation: map device memory at the virtual
// addresses a snapshot was captured at, in a process that did not capture
// it, so that kc_restore writes every page back to its original VA and the
// snapshot's embedded device pointers hold again (Section "VA-Faithful HSA
// Replay": replay reserves each captured region's address before copying
// its data back; Section "Memory Capture", paragraph "Handling embedded
// device pointers via address-space closure").
//
// CUDA's virtual memory management does the three steps the paper's replay
// does with its runtime's interposed allocator: reserve a VA range
// (cuMemAddressReserve), back it with physical device memory (cuMemCreate +
// cuMemMap) and grant the device read/write access (cuMemSetAccess).
//
// Placement.  The driver takes the requested address as a hint only and,
// measured on this platform, does not honour it; but it places a large
// reservation at the lowest free address of the VA zone it keeps for large
// reservations, which is also where VMM-based allocators (PyTorch's
// expandable segments) place their memory, so in a fresh process that zone
// starts where the capturing process's zone started.  kc_va_reserve
// therefore makes one covering reservation -- at least 4 GiB of VA, no
// memory -- and accepts it only if it spans every captured range; if the
// driver put it below the captured ranges, it retries once from there with
// a size reaching the last range.  Physical memory is then mapped at
// exactly the captured ranges (each region rounded out to the allocation
// granularity, overlapping or touching ranges merged); the rest of the
// covering reservation stays unmapped.  Any other placement is undone and
// reported as KC_EOVERLAP: a snapshot is never silently relocated.  The
// driver entry points are looked up at run time through the CUDA runtime,
// so the library does not link the driver.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "kc_internal.cuh"

namespace {

struct Driver {
    decltype(&cuMemAddressReserve) reserve = nullptr;
    decltype(&cuMemAddressFree) free = nullptr;
    decltype(&cuMemCreate) create = nullptr;
    decltype(&cuMemRelease) release = nullptr;
    decltype(&cuMemMap) map = nullptr;
    decltype(&cuMemUnmap) unmap = nullptr;
    decltype(&cuMemSetAccess) access = nullptr;
    decltype(&cuMemGetAllocationGranularity) granularity = nullptr;
    bool ok = false;
};

template <class F>
bool entry(const char *name, F *fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
        cudaGetLastError();
        return false;
    }
    *fn = reinterpret_cast<F>(p);
    return true;
}

const Driver *driver() {
    static Driver d;
    static std::once_flag once;
    std::call_once(once, [] {
        d.ok = entry("cuMemAddressReserve", &d.reserve) && entry("cuMemAddressFree", &d.free) &&
               entry("cuMemCreate", &d.create) && entry("cuMemRelease", &d.release) &&
               entry("cuMemMap", &d.map) && entry("cuMemUnmap", &d.unmap) &&
               entry("cuMemSetAccess", &d.access) && entry("cuMemGetAllocationGranularity", &d.granularity);
    });
    return d.ok ? &d : nullptr;
}

struct Span {
    CUdeviceptr base = 0;
    size_t size = 0;
    CUmemGenericAllocationHandle handle = 0;
    bool created = false, mapped = false;
};

struct Reservation {
    CUdeviceptr base = 0;
    size_t size = 0;
};

void undo(const Driver *d, std::vector<Span> &spans, Reservation &res) {
    for (auto it = spans.rbegin(); it != spans.rend(); ++it) {
        if (it->mapped) d->unmap(it->base, it->size);
        if (it->created) d->release(it->handle);
    }
    spans.clear();
    if (res.size) d->free(res.base, res.size);
    res = Reservation{};
}

constexpr uint64_t VA_COVER_MIN = 4ull << 30;   // a reservation this large goes to the large-reservation zone

// One reservation covering [lo, hi), or false.
bool reserve_covering(const Driver *d, uint64_t lo, uint64_t hi, size_t g, Reservation *out) {
    uint64_t size = hi - lo < VA_COVER_MIN ? VA_COVER_MIN : hi - lo;
    CUdeviceptr got = 0;
    if (d->reserve(&got, size, g, (CUdeviceptr)lo, 0) != CUDA_SUCCESS) return false;
    if ((uint64_t)got <= lo && (uint64_t)got + size >= hi) {
        *out = Reservation{got, (size_t)size};
        return true;
    }
    d->free(got, size);
    if ((uint64_t)got > lo) return false;       // the zone starts above the captured ranges: taken
    const uint64_t from = (uint64_t)got;        // below them: reach up to the last range from there
    size = hi - from < VA_COVER_MIN ? VA_COVER_MIN : hi - from;
    got = 0;
    if (d->reserve(&got, size, g, (CUdeviceptr)from, 0) != CUDA_SUCCESS) return false;
    if ((uint64_t)got <= lo && (uint64_t)got + size >= hi) {
        *out = Reservation{got, (size_t)size};
        return true;
    }
    d->free(got, size);
    return false;
}

}  // namespace

struct kc_va_lease {
    int device = 0;
    Reservation res;
    std::vector<Span> spans;
};

extern "C" {

KC_API kc_status kc_va_reserve(int device, const kc_buf *regions, int n, kc_va_lease **out) {
    if (!out) return KC_EINVAL;
    *out = nullptr;
    if (!regions || n < 1) return KC_EINVAL;
    for (int i = 0; i < n; ++i)
        if (regions[i].bytes == 0 || regions[i].base_va == 0 ||
            regions[i].base_va + regions[i].bytes < regions[i].base_va)
            return KC_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return KC_EINVAL;
    }
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (cudaSetDevice(device) != cudaSuccess || cudaFree(nullptr) != cudaSuccess) {   // primary context
        cudaGetLastError();
        return KC_ECUDA;
    }
    const Driver *d = driver();
    kc_status st = KC_OK;
    std::vector<Span> spans;
    Reservation res;
    CUmemAllocationProp prop{};
    prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
    prop.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
    prop.location.id = device;
    size_t g = 0;
    if (!d || d->granularity(&g, &prop, CU_MEM_ALLOC_GRANULARITY_MINIMUM) != CUDA_SUCCESS || g == 0) {
        st = KC_ECUDA;
    } else {
        // granule ranges of the regions, sorted and merged
        std::vector<std::pair<uint64_t, uint64_t>> iv(n);
        for (int i = 0; i < n; ++i) {
            const uint64_t lo = regions[i].base_va / g * g;
            const uint64_t hi = (regions[i].base_va + regions[i].bytes + g - 1) / g * g;
            iv[i] = {lo, hi};
        }
        std::sort(iv.begin(), iv.end());
        std::vector<std::pair<uint64_t, uint64_t>> merged;
        for (auto &r : iv) {
            if (!merged.empty() && r.first <= merged.back().second)
                merged.back().second = std::max(merged.back().second, r.second);
            else
                merged.push_back(r);
        }
        if (!reserve_covering(d, merged.front().first, merged.back().second, g, &res)) st = KC_EOVERLAP;
        CUmemAccessDesc acc{};
        acc.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
        acc.location.id = device;
        acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
        for (size_t k = 0; st == KC_OK && k < merged.size(); ++k) {
            spans.push_back(Span{});
            Span &b = spans.back();
            b.base = (CUdeviceptr)merged[k].first;
            b.size = (size_t)(merged[k].second - merged[k].first);
            if (d->create(&b.handle, b.size, &prop, 0) != CUDA_SUCCESS) {
                st = KC_ENOMEM;
                break;
            }
            b.created = true;
            if (d->map(b.base, b.size, 0, b.handle, 0) != CUDA_SUCCESS) {
                st = KC_ECUDA;
                break;
            }
            b.mapped = true;
            if (d->access(b.base, b.size, &acc, 1) != CUDA_SUCCESS) {
                st = KC_ECUDA;
                break;
            }
        }
    }
    if (st == KC_OK) {
        kc_va_lease *l = new (std::nothrow) kc_va_lease();
        if (!l) {
            st = KC_ENOMEM;
        } else {
            l->device = device;
            l->res = res;
            l->spans = std::move(spans);
            *out = l;
        }
    }
    if (st != KC_OK && d) undo(d, spans, res);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return st;
}

KC_API uint64_t kc_va_lease_bytes(const kc_va_lease *lease) {
    if (!lease) return 0;
    uint64_t t = 0;
    for (auto &s : lease->spans) t += s.size;
    return t;
}

KC_API void kc_va_release(kc_va_lease *lease) {
    if (!lease) return;
    const Driver *d = driver();
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (cudaSetDevice(lease->device) == cudaSuccess) cudaDeviceSynchronize();   // no work may still use the ranges
    cudaGetLastError();
    if (d) undo(d, lease->spans, lease->res);
    if (prev >= 0 && prev != lease->device) cudaSetDevice(prev);
    delete lease;
}

}  // extern "C"
