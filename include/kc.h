/*
 * kc.h -- C ABI of the GB300 snapshot library: page digest, page dedup,
 * embedded-pointer census, VA-faithful restore and per-dtype comparison of
 * captured device memory.
 *
 * The operations follow the data path of address-space-closure capture and
 * replay validation (Kerncap):
 *   - a snapshot covers every tracked device region, streamed in fixed-size
 *     chunks (Section "Memory Capture", HIP path: VA-faithful device memory
 *     snapshot);
 *   - capturing every region at its original VA captures embedded pointers,
 *     and pointers escaping the captured set break the closure (same
 *     section, paragraphs "Handling embedded device pointers via
 *     address-space closure" and "Bounds of the closure");
 *   - replay copies the captured data back into each region at the same VA
 *     (Section "VA-Faithful HSA Replay", stage 5);
 *   - validation compares replayed outputs byte-exactly or with
 *     numpy.allclose-style tolerances and reports NaNs explicitly (Section
 *     "Replay Validation");
 *   - a region freed before its copy is a per-region failure that must not
 *     corrupt the other regions' results (Section "Memory Capture",
 *     paragraph "Ordering and crash safety"; Section "Limitations", memory
 *     snapshot fragility).
 * The paper copies regions verbatim; hashing pages with XXH64 (seed 0,
 * public xxHash specification), deduplicating them and classifying pointers
 * word by word are this library's GPU formulation of that snapshot.
 *
 * Conventions for every call:
 *   - `d_` pointers are device pointers owned by the caller; plain pointers
 *     are host pointers read during the call only.  kc_buf.base_va names a
 *     device VA of the context's device.
 *   - Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *     default stream) and return after enqueueing; the host-side return
 *     value reports argument errors and launch failures.  Conditions only
 *     the GPU can see (truncation, a wait that timed out, a malformed page
 *     table row) are accumulated in the context and returned by kc_sync().
 *   - A context serves one stream at a time: two calls on one context that
 *     may overlap on the GPU (different streams without ordering) race on
 *     the context's scratch.  Use one context per stream.
 *   - Region bases must be 16-byte aligned; sizes must be > 0.  No call
 *     aborts the process or traps on the device.
 *   - Page sizes are powers of two in [4 KiB, 2 MiB].
 */
#ifndef KC_H
#define KC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KC_VERSION 1

#if defined(__GNUC__)
#define KC_API __attribute__((visibility("default")))
#else
#define KC_API
#endif

/* Element type of a buffer; only kc_compare interprets it. */
typedef enum {
    KC_U8 = 0,   /* uint8: also the byte-exact diff of the validation section */
    KC_I32 = 1,  /* int32 */
    KC_F16 = 2,  /* IEEE binary16 */
    KC_BF16 = 3, /* bfloat16 */
    KC_F32 = 4,  /* IEEE binary32 */
    KC_RAW = 5   /* opaque bytes; compared as uint8 */
} kc_dtype;

typedef enum {
    KC_OK = 0,
    KC_EINVAL = 1,   /* bad argument (size, alignment, dtype, page size, table row) */
    KC_EOVERLAP = 2, /* two regions' VA ranges overlap */
    KC_ENOMEM = 3,   /* scratch allocation failed, or would be needed inside a
                        stream capture */
    KC_ETRUNC = 4,   /* an output was too small; true counts were still written */
    KC_ECUDA = 5,    /* a CUDA runtime call failed; see kc_last_error */
    KC_ETIMEOUT = 6, /* a bounded device wait gave up; the affected outputs are stale */
    KC_EBUF = 7      /* one or more regions could not be read (see kc_buf_status);
                        the other regions' results are complete */
} kc_status;

/* kc_buf.flags */
#define KC_BUF_LOST 0x1 /* the region could not be captured (e.g. freed before
                           its copy): skip it, mark its outputs, report KC_EBUF */

/* One captured region: [base_va, base_va + bytes) on the context's device. */
typedef struct {
    uint64_t base_va;
    uint64_t bytes;
    int32_t dtype; /* kc_dtype */
    int32_t flags; /* KC_BUF_* */
} kc_buf;

/* zero[] values written by kc_digest */
#define KC_PAGE_DATA 0 /* page holds a non-zero byte */
#define KC_PAGE_ZERO 1 /* every byte of the page is 0 */
#define KC_PAGE_LOST 2 /* region was not readable; hash is 0 */

/* One row of the VA-faithful page table (16 bytes). */
typedef struct {
    uint64_t va_offset; /* byte offset of the page inside its region (j * page_bytes) */
    uint32_t alloc_id;  /* index of the region in the caller's kc_buf list */
    uint32_t blob;      /* arena slot, or KC_BLOB_ZERO / KC_BLOB_LOST */
} kc_page;

#define KC_BLOB_ZERO 0xFFFFFFFFu /* all-zero page: restore writes zeros */
#define KC_BLOB_LOST 0xFFFFFFFEu /* page of a lost region: restore skips it */

/* One embedded pointer found by the census (24 bytes). */
typedef struct {
    uint64_t src_offset; /* byte offset of the word inside its source region (multiple of 8) */
    uint64_t value;      /* the word, little-endian u64 */
    uint32_t src_alloc;  /* source region's index in the caller's list */
    int32_t target;      /* index of the region holding `value`, or -1 (outside) */
} kc_hit;

/* Result of one comparison pair (64 bytes). */
typedef struct {
    uint64_t mismatches;   /* elements that are not close (NaN==NaN is close) */
    int64_t first;         /* smallest mismatching element index, -1 if none */
    double max_abs;        /* max |got - want| over non-NaN unequal elements (FP64) */
    double max_rel;        /* max |got - want| / |want| over the same set (+inf if want == 0) */
    uint64_t nan_got;      /* NaN elements in got */
    uint64_t nan_want;     /* NaN elements in want */
    uint64_t nan_mismatch; /* elements where exactly one side is NaN */
    int32_t status;        /* KC_OK, or KC_EBUF if either buffer was lost */
    uint32_t reserved;
} kc_cmp_result;

typedef struct kc_ctx kc_ctx;

/* ---- context --------------------------------------------------------------
 * kc_create: make a context on CUDA device `device`.  The context owns
 * device scratch (sort buffers, counters, region tables) that grows on
 * demand; growth is refused inside a stream capture (KC_ENOMEM), so make one
 * uncaptured call of each shape first.  Calls on one context share that
 * scratch (and the task counter of the digest), so they must be ordered on
 * the device: one stream per context, or streams the caller orders with
 * events; for work that should overlap, use one context per stream.
 * Returns KC_OK, KC_EINVAL (null out, bad device) or KC_ECUDA.
 * kc_destroy: release everything (waits for the context's work to finish).
 * kc_last_error: human-readable reason of the last failing call (owned by
 * the context, valid until the next call).
 */
KC_API kc_status kc_create(kc_ctx **out, int device);
KC_API void kc_destroy(kc_ctx *ctx);
KC_API const char *kc_last_error(const kc_ctx *ctx);
KC_API const char *kc_status_name(int status);
KC_API int kc_version(void);
/* kc_launch_count: number of CUDA kernels this library has launched in this
 * process so far (all contexts). */
KC_API uint64_t kc_launch_count(void);

/* kc_sync: wait for `stream`, then return (and clear) the worst device-side
 * condition raised by the context's kernels since the previous kc_sync:
 * KC_ETIMEOUT > KC_EINVAL (malformed page-table row) > KC_ETRUNC > KC_OK. */
KC_API kc_status kc_sync(kc_ctx *ctx, void *stream);

/* kc_buf_status: status of region `i` in the context's last call that took
 * a region list (KC_OK, or KC_EBUF when it was lost).  -1 if out of range. */
KC_API int kc_buf_status(const kc_ctx *ctx, int i);

/* kc_set_digest_shape: pin the digest's launch shape for this context.
 * The digest kernel (kc_digest, kc_scan) runs CTAs of one producer warp,
 * which streams pages into shared memory with bulk copies, and `warps` hash
 * warps (1..16) of 8 pages each (one XXH64 accumulator per thread); each
 * hash warp owns a ring of `stages` (2..8) stages of `chunk` bytes per page
 * (multiple of 128, 256..8192).  The batched kernel (kc_batch_run) reads
 * the same three numbers as its warps per CTA, per-warp ring stages and
 * chunk.  `lanes` must be 0 or 1 (one accumulator per thread).  All four 0
 * restores the built-in choice.  The shape changes speed only, never
 * results.  KC_EINVAL if out of range or if the rings do not fit a CTA's
 * shared memory.
 * kc_get_digest_shape: the shape a digest of `npages` pages of
 * `page_bytes` would use now (`warps` = hash warps), and its grid size
 * (`ctas`). */
KC_API kc_status kc_set_digest_shape(kc_ctx *ctx, int warps, int stages, int chunk, int lanes);
KC_API kc_status kc_get_digest_shape(kc_ctx *ctx, uint32_t page_bytes, uint64_t npages, int *warps,
                                     int *stages, int *chunk, int *ctas, int *lanes);

/* kc_debug_stall_census: test hook for the bounded waits of kc_scan's
 * census.  The census orders its hits with a decoupled look-back: each
 * chunk of pages publishes its hit total and waits (bounded) for earlier
 * chunks' totals, following the paper's rule that a failure is reported,
 * never silently lost (Section "Memory Capture", paragraph "Ordering and
 * crash safety").  After this call, the context's next kc_scan starts the
 * chunk tickets at 1, so chunk 0 is never taken and never published, and
 * bounds every look-back wait at `spin_limit` polls: a later chunk with
 * hits gives up after the limit, the kernel finishes, and kc_sync reports
 * KC_ETIMEOUT (that call's census outputs are incomplete; its digest is
 * exact).  One-shot: the call after it runs normally.  KC_EINVAL if ctx
 * is NULL or spin_limit is 0. */
KC_API kc_status kc_debug_stall_census(kc_ctx *ctx, uint32_t spin_limit);

/* kc_set_trace_events: `start` and `stop` (cudaEvent_t, or NULL to turn
 * tracing off) are recorded on the call's stream around the main kernel of
 * every following call: the digest kernel of kc_digest / kc_scan, the count
 * kernel of kc_census, the whole pipeline of kc_dedup, the restore kernel,
 * the compare kernels.  Timing them with cudaEventElapsedTime measures that
 * kernel alone.  The events stay owned by the caller. */
KC_API kc_status kc_set_trace_events(kc_ctx *ctx, void *start, void *stop);

/* kc_page_count: number of pages of `n` regions at `page_bytes` per page
 * (the last page of each region is partial).  Host only. */
KC_API uint64_t kc_page_count(const kc_buf *bufs, int n, uint32_t page_bytes);

/* ---- digest ---------------------------------------------------------------
 * Defined by: Section "Memory Capture" (HIP path), which snapshots every
 * tracked region verbatim at its VA; the per-page XXH64 digest is this
 * library's reduction of that snapshot on the device (the paper hashes only
 * code objects), so that equal pages can be found and stored once.
 * For region i (list order) and page j = 0 .. ceil(bytes_i / S) - 1:
 *   d_hash[p] = XXH64(seed 0) of bytes [jS, min((j+1)S, bytes_i)), unpadded;
 *   d_zero[p] = KC_PAGE_ZERO if every one of those bytes is 0, else
 *               KC_PAGE_DATA (KC_PAGE_LOST, hash 0, for a lost region),
 * with p = d_page_first[i] + j; d_page_first has n + 1 entries, the last
 * being the page count P.  d_hash: P u64; d_zero: P u8.
 * Errors: KC_EINVAL (n < 1, null output, page size, alignment, empty
 * region), KC_ECUDA, KC_EBUF (other regions complete).
 */
KC_API kc_status kc_digest(kc_ctx *ctx, const kc_buf *allocs, int n, uint32_t page_bytes,
                    uint64_t *d_hash, uint8_t *d_zero, uint64_t *d_page_first, void *stream);

/* ---- census ---------------------------------------------------------------
 * Defined by: Section "Memory Capture", paragraphs "Handling embedded device
 * pointers via address-space closure" and its bounds -- the snapshot stays
 * valid only if the pointers it embeds point into captured regions; the
 * census counts and lists the words that do (inside) and the words that
 * point elsewhere in the device VA window (outside).
 * For every region i (list order) and every offset o = 0, 8, ... with
 * o + 8 <= bytes_i, the little-endian u64 word v at base_i + o is
 *   INSIDE  (target k) if base_k <= v < base_k + bytes_k for some region k,
 *   OUTSIDE (target -1) otherwise, if win_lo <= v < win_hi,
 *   not a hit otherwise.
 * Regions are half-open VA ranges and must not overlap (KC_EOVERLAP).  Hits
 * are written to d_hits in (region, offset) order, at most `cap` of them;
 * d_counts (device, 2 x u64) receives {n_inside, n_outside}, the true
 * counts even when they exceed cap (kc_sync then reports KC_ETRUNC).
 * d_hits may be NULL with cap 0 to count only.  A lost region is not
 * scanned but stays a target.
 */
KC_API kc_status kc_census(kc_ctx *ctx, const kc_buf *allocs, int n, uint64_t win_lo, uint64_t win_hi,
                    kc_hit *d_hits, uint64_t cap, uint64_t *d_counts, void *stream);

/* kc_census_static: kc_census for callers that must not allocate memory.
 * The paper has no counterpart; this entry point exists because some
 * callers cannot call cudaMalloc (or any allocating routine): a hook running
 * inside the application's allocator or memory-tracking callback, a handler
 * snapshotting device memory after a failure, or a process whose device
 * memory is fully reserved.  It computes exactly what kc_census computes on
 * the caller's current device, with no context, and allocates nothing: its
 * scratch (region table, sorted ranges, per-64-KiB-chunk hit counts and
 * offsets, a status word) is one static device array of about 0.8 MiB in
 * the library's image.
 * Set-up: CUDA loads a module's code and static data onto a device lazily,
 * when first used, and that load takes device memory.  The first call on a
 * device therefore does a one-time set-up -- it loads the array and every
 * kernel a call launches (one empty launch each on `stream`) and looks up
 * the array's device address -- after which the device holds the array
 * until the process exits and calls load nothing.  kc_census_static(NULL,
 * 0, 0, 0, NULL, 0, NULL, stream) does only that set-up and returns KC_OK;
 * make it (or a first call) while device memory is still available.
 * Limits: n <= 1024 regions and at most 65536 chunks of 64 KiB
 * (ceil(bytes / 64 KiB) summed over the regions, i.e. about 4 GiB); larger
 * requests return KC_EINVAL before any work.
 * Not capturable: the call copies its tables from shared host memory, so
 * inside a stream capture it returns KC_EINVAL and enqueues nothing.
 * Every call on a device shares the array and overwrites the previous
 * call's contents: calls that may overlap on the GPU (different streams, or
 * different host threads with unordered streams) race, so serialise them.
 * A race that the write pass detects (a chunk whose recount differs from
 * its count) sets both counts to all-ones (UINT64_MAX), a value no census
 * produces; not every race is detected.  Truncation is not reported
 * separately: the true counts are written to d_counts, so n_inside +
 * n_outside > cap means the list was cut.  Returns KC_OK, KC_EINVAL,
 * KC_EOVERLAP, KC_ECUDA or KC_EBUF. */
KC_API kc_status kc_census_static(const kc_buf *allocs, int n, uint64_t win_lo, uint64_t win_hi,
                                  kc_hit *d_hits, uint64_t cap, uint64_t *d_counts, void *stream);

/* kc_scan (Sections "Memory Capture" and its address-space closure
 * paragraphs, as kc_digest and kc_census): kc_digest and kc_census fused
 * into one read of the snapshot
 * (while pages are hashed, a conservative test on the high 32 bits of every
 * word flags the pages that may hold hits; only those are read a second
 * time, classified and written in order).  Outputs and errors
 * are exactly those of the two calls. */
KC_API kc_status kc_scan(kc_ctx *ctx, const kc_buf *allocs, int n, uint32_t page_bytes,
                  uint64_t *d_hash, uint8_t *d_zero, uint64_t *d_page_first,
                  uint64_t win_lo, uint64_t win_hi, kc_hit *d_hits, uint64_t cap,
                  uint64_t *d_counts, void *stream);

/* ---- dedup ----------------------------------------------------------------
 * Defined by: Section "Memory Capture" (the verbatim snapshot the paper
 * writes per region); storing each distinct page once, with a table that
 * rebuilds every region, is this library's device-side reduction of it and
 * loses no byte (byte equality decides, below).
 * Input: the digest of the same regions at the same page size (d_hash,
 * d_zero).  Non-zero pages are grouped by their hashes (a device radix sort;
 * up to 8192 pages, shared-memory hash tables) and byte-verified; the
 * grouping never decides a result: two pages are duplicates iff they have the same
 * length and the same bytes.  canonical(p) = the smallest page id of p's
 * class; blobs are numbered 0, 1, ... in increasing canonical page id.
 * d_table[p] = {j * S, i, blob(canonical(p))}, KC_BLOB_ZERO for zero pages,
 * KC_BLOB_LOST for lost pages (P rows).  *d_n_blobs (device u64) = number
 * of blobs.  If d_arena is not NULL and arena_cap >= n_blobs * S, every
 * canonical page is packed into d_arena[blob * S ...], zero-filled to S;
 * if it is too small nothing is packed and kc_sync reports KC_ETRUNC
 * (d_arena NULL = table only).
 */
KC_API kc_status kc_dedup(kc_ctx *ctx, const kc_buf *allocs, int n, uint32_t page_bytes,
                   const uint64_t *d_hash, const uint8_t *d_zero, kc_page *d_table,
                   uint8_t *d_arena, uint64_t arena_cap, uint64_t *d_n_blobs, void *stream);

/* ---- restore --------------------------------------------------------------
 * Defined by: Section "VA-Faithful HSA Replay", stage 5 (the captured data
 * is copied back at the VAs it was captured at, so embedded pointers hold).
 * For each of the n_pages rows r of d_table: len = min(S, bytes_a - off)
 * with a = r.alloc_id, off = r.va_offset; write len bytes at base_a + off:
 * zeros for KC_BLOB_ZERO, nothing for KC_BLOB_LOST, else the bytes
 * d_arena[r.blob * S ...].  Rows that point outside a region or outside
 * the arena (arena_bytes) are skipped and reported as KC_EINVAL by kc_sync.
 * `allocs` gives the restore targets: the captured VAs for a VA-faithful
 * restore, or explicit new bases (a relocation the caller asks for).
 * d_arena may also be pinned host memory the device can address (e.g. a
 * snapshot image loaded from disk): the kernel then reads it over the host
 * link, with no staging copy.  A table whose row p has blob = p restores a
 * page-slotted image (page p in bytes [p*S, (p+1)*S)).
 */
KC_API kc_status kc_restore(kc_ctx *ctx, const kc_buf *allocs, int n, uint32_t page_bytes,
                     const kc_page *d_table, uint64_t n_pages, const uint8_t *d_arena,
                     uint64_t arena_bytes, void *stream);

/* ---- compare --------------------------------------------------------------
 * Defined by: Section "Replay Validation" (replayed outputs are checked
 * against the captured ones byte for byte, or with numpy.allclose-style
 * tolerances, NaNs reported explicitly).
 * For pair k, got[k] and want[k] hold the same number of bytes, a multiple
 * of the element size of got[k].dtype (want[k].dtype is ignored).  Every
 * element is widened exactly to FP64 (a = got, b = want):
 *   both NaN -> equal;  one NaN -> mismatch, nan_mismatch++;
 *   a == b (so +0 == -0) -> equal;
 *   otherwise d = |a - b|, r = d / |b| (+inf if b == 0 or d is infinite),
 *   max_abs = max d, max_rel = max r over these elements, and the element
 *   mismatches if a or b is infinite or d > atol + rtol * |b|.
 * d_out[k] receives the kc_cmp_result; all FP64 operations are single IEEE
 * round-to-nearest steps, so results do not depend on the order of work.
 * Errors: KC_EINVAL (sizes, dtype, alignment to 16 bytes, negative or NaN
 * tolerance), KC_EBUF (a lost buffer: that pair's status is KC_EBUF).
 */
KC_API kc_status kc_compare(kc_ctx *ctx, const kc_buf *got, const kc_buf *want, int npairs,
                     double atol, double rtol, kc_cmp_result *d_out, void *stream);

/* ---- exact-VA reservation (replay in a fresh process) ---------------------
 * A snapshot's embedded device pointers are valid only at the VAs it was
 * captured at, so the paper's replay reserves every captured region's
 * address before copying the data back (Section "VA-Faithful HSA Replay",
 * stages 4-5; Section "Memory Capture", paragraph "Handling embedded device
 * pointers via address-space closure").  kc_va_reserve does that for a
 * process that did not capture the snapshot: every region of `regions`
 * (base_va, bytes; dtype and flags ignored) on CUDA device `device` gets
 * physical device memory mapped at exactly [base_va, base_va + bytes)
 * rounded out to the device's allocation granularity (regions sharing a
 * granule share the mapping), readable and writable by the device.
 * kc_restore with the same descriptors then writes every page at its
 * captured VA.  The CUDA driver treats a requested address as a hint it may
 * not honour; it places a large reservation at the lowest free address of
 * its large-reservation zone, where VMM-based allocators (PyTorch with
 * expandable segments) also place their memory.  So the call makes one
 * covering VA reservation (at least 4 GiB, no memory) and keeps it only if
 * it spans every captured range -- which holds when the snapshot was
 * allocated that way and the calling process has not yet used that zone --
 * and maps memory at the captured ranges inside it.  Call it before the
 * process allocates device memory.  *out receives a lease that owns the
 * mappings until kc_va_release.  Returns KC_OK; KC_EINVAL (null out or
 * regions, n < 1, an empty, null or wrapping region, bad device);
 * KC_EOVERLAP when the captured ranges cannot be had at their VAs in this
 * process (in use, or the driver placed the reservation elsewhere; nothing
 * is relocated, everything made so far is undone and *out stays NULL);
 * KC_ENOMEM when physical memory could not be allocated; KC_ECUDA for other
 * driver failures.  The memory is not initialised.
 * kc_va_lease_bytes: bytes reserved by a lease (granule-rounded), 0 for NULL.
 * kc_va_release: wait for the device, unmap, free and delete the lease. */
typedef struct kc_va_lease kc_va_lease;
KC_API kc_status kc_va_reserve(int device, const kc_buf *regions, int n, kc_va_lease **out);
KC_API uint64_t kc_va_lease_bytes(const kc_va_lease *lease);
KC_API void kc_va_release(kc_va_lease *lease);

/* ---- batched form --------------------------------------------------------
 * The operations above launch a few kernels per call; validating thousands
 * of replayed buffers (one tuning campaign re-runs a kernel many times and
 * compares every output region) that way spends most of its time in
 * launches.  kc_batch_run digests and/or compares many buffers in one
 * persistent, work-stealing launch.  (The paper has no batched form; its
 * validator compares regions one after another on the host -- Section
 * "Replay Validation".)
 *
 * A job is one buffer: with KC_JOB_DIGEST its pages are hashed exactly as
 * kc_digest would (into its own d_hash / d_zero, ceil(bytes / page_bytes)
 * entries each); with KC_JOB_COMPARE it is compared with want_va exactly as
 * kc_compare would (into d_cmp).  KC_BUF_LOST marks a buffer that could not
 * be read (outputs marked as by the single-operation calls).
 *
 * work / nwork: which units this launch processes, as ranges of a job's
 * pages (KC_WORK_DIGEST), of its comparison items (KC_WORK_COMPARE,
 * KC_BATCH_ITEM_BYTES of each buffer per item) or of its pages to digest
 * and compare in one pass (KC_WORK_FUSED: a job with both operations; the
 * comparison of those pages' bytes rides on the digest's read of got, so
 * got crosses HBM once).  NULL = every unit of every job, largest jobs
 * first, a job with both operations as one fused range.  A job may be spread over several launches (a
 * serving loop does this); its comparison record is initialised by the
 * launch whose job carries KC_JOB_INIT and accumulates over later launches
 * with order-independent merges, so the result does not depend on how the
 * work was split.  Without `work`, every compare job is initialised.
 *
 * Completion signal (optional, per job): with d_done set, the launch
 * stores 1 to *d_done once every unit of the job in this launch has
 * finished and its outputs are visible to the host (system-scope fence);
 * a job with no unit in the launch is flagged when the launch starts.  With
 * d_cmp_copy also set, the job's comparison record (accumulated over every
 * launch so far) is copied there just before the flag.  Both may point to
 * pinned host memory the device can address, so that a host loop sees a
 * job finish while the rest of the launch is still running.  The caller
 * clears *d_done before the launch; the launch only sets it.
 *
 * Repeated calls with the same jobs and work hit the context's table cache
 * and can be captured in a CUDA graph.  The digest kernel shape
 * (kc_set_digest_shape) also applies here.
 * Errors: KC_EINVAL (alignment, sizes, dtype, null outputs, a work range
 * outside its job), KC_EBUF (a lost buffer; the others are complete). */
#define KC_JOB_DIGEST 0x10
#define KC_JOB_COMPARE 0x20
#define KC_JOB_INIT 0x40
#define KC_WORK_DIGEST 0
#define KC_WORK_COMPARE 1
#define KC_WORK_FUSED 2
#define KC_BATCH_ITEM_BYTES 65536

typedef struct {
    uint64_t got_va;       /* buffer to digest and/or compare (16-byte aligned) */
    uint64_t want_va;      /* comparison reference (KC_JOB_COMPARE), same size */
    uint64_t bytes;        /* size of the buffer(s) */
    int32_t dtype;         /* element type for the comparison */
    int32_t flags;         /* KC_JOB_* | KC_BUF_LOST */
    uint64_t *d_hash;      /* KC_JOB_DIGEST: page hashes */
    uint8_t *d_zero;       /* KC_JOB_DIGEST: page zero flags */
    kc_cmp_result *d_cmp;  /* KC_JOB_COMPARE: the comparison record */
    uint32_t *d_done;      /* optional completion flag (see above), or NULL */
    kc_cmp_result *d_cmp_copy; /* optional copy of the finished record, or NULL */
} kc_job;                  /* 72 bytes */

typedef struct {
    uint32_t job;          /* index in the job list */
    uint32_t kind;         /* KC_WORK_DIGEST, KC_WORK_COMPARE or KC_WORK_FUSED */
    uint64_t first;        /* first unit (page, or comparison item) */
    uint64_t count;        /* number of units */
} kc_work;

KC_API kc_status kc_batch_run(kc_ctx *ctx, const kc_job *jobs, int njobs, uint32_t page_bytes, double atol,
                              double rtol, const kc_work *work, int nwork, void *stream);

/* Host helper for the completion flags above (no device work): reads the
 * n flags at `flags` (host memory the device writes, e.g. pinned), writes
 * the indices of those that are non-zero to idx_out (room for n) and
 * returns their number.  The reads are followed by an acquire fence, so
 * the caller's later reads of a flagged job's outputs see what the device
 * wrote before setting the flag, also on weakly ordered hosts.  Returns -1
 * if flags or idx_out is NULL or n < 0. */
KC_API int kc_poll_flags(const uint32_t *flags, int n, int32_t *idx_out);

#ifdef __cplusplus
}
#endif

#endif /* KC_H */
