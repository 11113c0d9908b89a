// k_restore.cu -- write every page of a page table back to its region at the
// same VA offset (Section "VA-Faithful HSA Replay", stage 5: copy captured
// data into each restored region).
//
// Work items are (row, 16 KiB piece of the page); one warp moves one item
// with 16-byte loads and stores, four loads in flight per lane.  Rows are
// untrusted input: a row whose region index, offset or arena slot falls
// outside its bounds is skipped and reported (ST_BADROW) instead of touching
// memory it does not own.
#include <cuda_runtime.h>

#include "kc_device.cuh"
#include "kc_internal.cuh"

namespace kc {

constexpr uint32_t RESTORE_PIECE = 16 * 1024;

__global__ void __launch_bounds__(256) restore_kernel(Pages pg, const kc_page *__restrict__ table, uint64_t nrows,
                                                      const uint8_t *__restrict__ arena, uint64_t arena_bytes,
                                                      uint32_t *__restrict__ status) {
    const uint32_t lane = lane_id();
    const uint32_t pieces = (pg.page + RESTORE_PIECE - 1) / RESTORE_PIECE;
    const uint64_t items = nrows * pieces;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t it = gw; it < items; it += nw) {
        const uint64_t row = it / pieces;
        const uint32_t piece = (uint32_t)(it - row * pieces);
        const kc_page r = table[row];
        if (r.blob == KC_BLOB_LOST) continue;
        if (r.alloc_id >= (uint32_t)pg.nregions) {
            if (lane == 0 && piece == 0) set_status(status, ST_BADROW);
            continue;
        }
        const Region reg = pg.regions[r.alloc_id];
        if (reg.lost) continue;
        if (r.va_offset >= reg.bytes || (r.va_offset & 15)) {
            if (lane == 0 && piece == 0) set_status(status, ST_BADROW);
            continue;
        }
        const uint64_t len = reg.bytes - r.va_offset < pg.page ? reg.bytes - r.va_offset : pg.page;
        const uint64_t p0 = (uint64_t)piece * RESTORE_PIECE;
        if (p0 >= len) continue;
        const uint64_t plen = len - p0 < RESTORE_PIECE ? len - p0 : RESTORE_PIECE;
        uint8_t *dst = reinterpret_cast<uint8_t *>(reg.base + r.va_offset + p0);
        const uint64_t nvec = plen >> 4;
        if (r.blob == KC_BLOB_ZERO) {
            const uint4 z = make_uint4(0, 0, 0, 0);
            for (uint64_t v = lane; v < nvec; v += 32) *reinterpret_cast<uint4 *>(dst + 16 * v) = z;
            for (uint64_t b = (nvec << 4) + lane; b < plen; b += 32) dst[b] = 0;
            continue;
        }
        // arena slot bounds: blob < 2^32 and page <= 2^21, so the product cannot overflow
        if ((uint64_t)r.blob * pg.page + len > arena_bytes) {
            if (lane == 0 && piece == 0) set_status(status, ST_BADROW);
            continue;
        }
        const uint8_t *src = arena + (uint64_t)r.blob * pg.page + p0;
        uint64_t v = lane;
        for (; v + 96 < nvec; v += 128) {
            uint4 x0 = ldg_stream(src + 16 * v), x1 = ldg_stream(src + 16 * (v + 32));
            uint4 x2 = ldg_stream(src + 16 * (v + 64)), x3 = ldg_stream(src + 16 * (v + 96));
            *reinterpret_cast<uint4 *>(dst + 16 * v) = x0;
            *reinterpret_cast<uint4 *>(dst + 16 * (v + 32)) = x1;
            *reinterpret_cast<uint4 *>(dst + 16 * (v + 64)) = x2;
            *reinterpret_cast<uint4 *>(dst + 16 * (v + 96)) = x3;
        }
        for (; v < nvec; v += 32) *reinterpret_cast<uint4 *>(dst + 16 * v) = ldg_stream(src + 16 * v);
        for (uint64_t b = (nvec << 4) + lane; b < plen; b += 32) dst[b] = src[b];
    }
}

cudaError_t launch_restore(const Pages &pg, const kc_page *table, uint64_t nrows, const uint8_t *arena,
                           uint64_t arena_bytes, uint32_t *status, int sms, cudaStream_t st) {
    const uint64_t pieces = (pg.page + RESTORE_PIECE - 1) / RESTORE_PIECE;
    const uint64_t warps = nrows * pieces;
    if (warps == 0) return cudaSuccess;
    uint64_t blocks = (warps + 7) / 8;
    const uint64_t maxb = (uint64_t)sms * 8;
    if (blocks > maxb) blocks = maxb;
    restore_kernel<<<(unsigned)blocks, 256, 0, st>>>(pg, table, nrows, arena, arena_bytes, status);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace kc
