/*
 * kc_oracle.c -- plain, slow, single-threaded CPU oracle for the snapshot
 * digest / dedup / census / restore / compare path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this file's library.  The
 * product path (the CUDA library under paper_2605_03208_gb300/csrc) shares no
 * code, header, table or helper with it, and never calls it.
 *
 * What it computes (every function names the passage it follows):
 *   - The snapshot covers every tracked device region, copied verbatim
 *     (Section "Memory Capture", HIP path: VA-faithful device memory snapshot).
 *     Here a region is split into fixed-size pages of S bytes; the last page
 *     of a region is partial and is never padded.
 *   - kco_xxh64: the XXH64 hash as defined in the public xxHash specification
 *     (XXH64 algorithm description: four accumulators over 32-byte stripes,
 *     convergence, length add, 8/4/1-byte tail, avalanche).  Input words are
 *     little-endian.  The snapshot method itself never hashes pages (it hashes
 *     only code objects, with SHA-256); per-page XXH64 with seed 0 is the
 *     digest this library defines on top of the verbatim snapshot.
 *   - kco_dedup / kco_pack: byte-equal pages form one class; the canonical
 *     page of a class is its smallest global page id; blob ids follow the
 *     canonical pages in page order; all-zero pages get no blob.  The result
 *     is VA-faithful: every page keeps (alloc id, VA offset).
 *   - kco_census: every 8-byte word of every region, read as a little-endian
 *     u64, is looked up in the sorted half-open VA ranges of the captured set
 *     (Section "Memory Capture", paragraphs on address-space closure and on
 *     the bounds of the closure: pointers that escape the captured set).
 *   - kco_restore: copy each page's blob back to base + VA offset (Section
 *     "VA-Faithful HSA Replay", stage 5: copy captured data into each restored
 *     region).
 *   - kco_compare: numpy.allclose-style tolerance comparison with explicit
 *     NaN reporting (Section "Replay Validation", tolerance-based comparison),
 *     every value widened exactly to FP64.  With atol = rtol = 0 it is the
 *     byte/element-exact comparison of the same section.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC.  No FMA
 * contraction, so every FP64 operation is one IEEE round-to-nearest-even step.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* XXH64 (public xxHash specification, "XXH64 algorithm description").      */
/* ------------------------------------------------------------------------ */

static const uint64_t XP1 = 0x9E3779B185EBCA87ULL;
static const uint64_t XP2 = 0xC2B2AE3D27D4EB4FULL;
static const uint64_t XP3 = 0x165667B19E3779F9ULL;
static const uint64_t XP4 = 0x85EBCA77C2B2AE63ULL;
static const uint64_t XP5 = 0x27D4EB2F165667C5ULL;

static uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

/* Little-endian loads written out byte by byte, independent of host order. */
static uint64_t le64(const uint8_t *p) {
    uint64_t v = 0;
    for (int i = 7; i >= 0; --i) v = (v << 8) | (uint64_t)p[i];
    return v;
}
static uint32_t le32(const uint8_t *p) {
    uint32_t v = 0;
    for (int i = 3; i >= 0; --i) v = (v << 8) | (uint32_t)p[i];
    return v;
}

/* One accumulator round: acc + lane * PRIME2, rotate left 31, times PRIME1. */
static uint64_t xround(uint64_t acc, uint64_t lane) {
    acc = acc + lane * XP2;
    acc = rotl64(acc, 31);
    return acc * XP1;
}

/* Merge of one accumulator into the converged value. */
static uint64_t xmerge(uint64_t acc, uint64_t accn) {
    acc = acc ^ xround(0, accn);
    return acc * XP1 + XP4;
}

uint64_t kco_xxh64(const void *data, uint64_t len, uint64_t seed) {
    const uint8_t *p = (const uint8_t *)data;
    uint64_t remaining = len;
    uint64_t acc;
    if (len >= 32) {
        /* Step 1: initialise the four accumulators. */
        uint64_t a1 = seed + XP1 + XP2;
        uint64_t a2 = seed + XP2;
        uint64_t a3 = seed;
        uint64_t a4 = seed - XP1;
        /* Step 2: every full 32-byte stripe feeds one 8-byte lane to each. */
        while (remaining >= 32) {
            a1 = xround(a1, le64(p + 0));
            a2 = xround(a2, le64(p + 8));
            a3 = xround(a3, le64(p + 16));
            a4 = xround(a4, le64(p + 24));
            p += 32;
            remaining -= 32;
        }
        /* Step 3: convergence. */
        acc = rotl64(a1, 1) + rotl64(a2, 7) + rotl64(a3, 12) + rotl64(a4, 18);
        acc = xmerge(acc, a1);
        acc = xmerge(acc, a2);
        acc = xmerge(acc, a3);
        acc = xmerge(acc, a4);
    } else {
        /* Short input: no stripes. */
        acc = seed + XP5;
    }
    /* Step 4: add the total input length. */
    acc = acc + len;
    /* Step 5: consume the remaining (< 32) bytes: 8-byte, 4-byte, 1-byte. */
    while (remaining >= 8) {
        acc = acc ^ xround(0, le64(p));
        acc = rotl64(acc, 27) * XP1 + XP4;
        p += 8;
        remaining -= 8;
    }
    if (remaining >= 4) {
        acc = acc ^ ((uint64_t)le32(p) * XP1);
        acc = rotl64(acc, 23) * XP2 + XP3;
        p += 4;
        remaining -= 4;
    }
    while (remaining >= 1) {
        acc = acc ^ ((uint64_t)(*p) * XP5);
        acc = rotl64(acc, 11) * XP1;
        p += 1;
        remaining -= 1;
    }
    /* Step 6: final avalanche. */
    acc = acc ^ (acc >> 33);
    acc = acc * XP2;
    acc = acc ^ (acc >> 29);
    acc = acc * XP3;
    acc = acc ^ (acc >> 32);
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Pages.                                                                    */
/* ------------------------------------------------------------------------ */

/* Number of S-byte pages of a region of `bytes` bytes (last one partial). */
static uint64_t npages(uint64_t bytes, uint64_t S) { return (bytes + S - 1) / S; }

/* page_first[i] = global id of region i's first page; page_first[n] = P. */
uint64_t kco_page_first(int n, const uint64_t *bytes, uint32_t S, uint64_t *page_first) {
    uint64_t total = 0;
    for (int i = 0; i < n; ++i) {
        if (page_first) page_first[i] = total;
        total += npages(bytes[i], S);
    }
    if (page_first) page_first[n] = total;
    return total;
}

/*
 * Digest: for region i (list order) and page j (VA order) the hash is XXH64
 * with seed 0 over exactly that page's bytes, and zero = 1 iff all of them
 * are 0.  Pages are numbered region-major: page id = page_first[i] + j.
 */
void kco_digest(int n, const uint8_t *const *img, const uint64_t *bytes, uint32_t S,
                uint64_t *hash, uint8_t *zero, uint64_t *page_first) {
    uint64_t pid = 0;
    for (int i = 0; i < n; ++i) {
        if (page_first) page_first[i] = pid;
        for (uint64_t off = 0; off < bytes[i]; off += S) {
            uint64_t len = bytes[i] - off < S ? bytes[i] - off : S;
            const uint8_t *pg = img[i] + off;
            hash[pid] = kco_xxh64(pg, len, 0);
            uint8_t all0 = 1;
            for (uint64_t b = 0; b < len; ++b)
                if (pg[b] != 0) { all0 = 0; break; }
            zero[pid] = all0;
            ++pid;
        }
    }
    if (page_first) page_first[n] = pid;
}

/* ------------------------------------------------------------------------ */
/* Dedup.                                                                    */
/* ------------------------------------------------------------------------ */

#define KCO_BLOB_ZERO 0xFFFFFFFFu

typedef struct {
    uint64_t hash;
    uint64_t page;
} kco_hp;

static int cmp_hp(const void *a, const void *b) {
    const kco_hp *x = (const kco_hp *)a, *y = (const kco_hp *)b;
    if (x->hash != y->hash) return x->hash < y->hash ? -1 : 1;
    if (x->page != y->page) return x->page < y->page ? -1 : 1;
    return 0;
}

/* Locate page `pid`: its region, its offset inside the region and its length. */
static void page_loc(int n, const uint64_t *bytes, const uint64_t *page_first, uint32_t S,
                     uint64_t pid, int *alloc, uint64_t *off, uint64_t *len) {
    int lo = 0, hi = n - 1;
    while (lo < hi) { /* last region whose first page id is <= pid */
        int mid = (lo + hi + 1) / 2;
        if (page_first[mid] <= pid) lo = mid; else hi = mid - 1;
    }
    *alloc = lo;
    *off = (pid - page_first[lo]) * (uint64_t)S;
    uint64_t rest = bytes[lo] - *off;
    *len = rest < S ? rest : S;
}

static int pages_equal(int n, const uint8_t *const *img, const uint64_t *bytes,
                       const uint64_t *page_first, uint32_t S, uint64_t p, uint64_t q) {
    int ap, aq;
    uint64_t op, oq, lp, lq;
    page_loc(n, bytes, page_first, S, p, &ap, &op, &lp);
    page_loc(n, bytes, page_first, S, q, &aq, &oq, &lq);
    if (lp != lq) return 0;
    return memcmp(img[ap] + op, img[aq] + oq, (size_t)lp) == 0;
}

/*
 * Dedup of the non-zero pages.  `hash` is only an accelerator: equal bytes
 * imply equal hashes, so classes are searched inside groups of equal hash
 * (a library sort forms the groups) and decided by memcmp of equal-length
 * pages.  Inside a group the pages are visited in increasing page id; each is
 * compared with the representatives found so far, in order, and joins the
 * first equal one, else it becomes a new representative.  A representative is
 * thus the smallest page id of its class, i.e. the canonical page.
 * Outputs (all of length P): canon[p] (p itself for zero pages),
 * tbl_off/tbl_alloc/tbl_blob, and *n_blobs.  Returns 0, or -1 if out of
 * memory.
 */
int kco_dedup(int n, const uint8_t *const *img, const uint64_t *bytes, uint32_t S,
              const uint64_t *hash, const uint8_t *zero,
              uint64_t *tbl_off, uint32_t *tbl_alloc, uint32_t *tbl_blob,
              uint64_t *canon, uint64_t *n_blobs) {
    uint64_t *pf = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n + 1));
    if (!pf) return -1;
    uint64_t P = kco_page_first(n, bytes, S, pf);
    kco_hp *rec = (kco_hp *)malloc(sizeof(kco_hp) * (size_t)(P ? P : 1));
    uint64_t *reps = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(P ? P : 1));
    uint32_t *blob_of = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(P ? P : 1));
    if (!rec || !reps || !blob_of) { free(pf); free(rec); free(reps); free(blob_of); return -1; }

    uint64_t m = 0;
    for (uint64_t p = 0; p < P; ++p) {
        canon[p] = p;
        if (!zero[p]) { rec[m].hash = hash[p]; rec[m].page = p; ++m; }
    }
    qsort(rec, (size_t)m, sizeof(kco_hp), cmp_hp);

    for (uint64_t g = 0; g < m;) {
        uint64_t e = g;
        while (e < m && rec[e].hash == rec[g].hash) ++e;
        uint64_t nrep = 0;
        for (uint64_t k = g; k < e; ++k) {
            uint64_t p = rec[k].page;
            uint64_t r;
            for (r = 0; r < nrep; ++r)
                if (pages_equal(n, img, bytes, pf, S, p, reps[r])) break;
            if (r < nrep) canon[p] = reps[r];
            else { reps[nrep++] = p; canon[p] = p; }
        }
        g = e;
    }

    /* Blob ids: canonical non-zero pages numbered in increasing page id. */
    uint32_t next = 0;
    for (uint64_t p = 0; p < P; ++p) {
        if (!zero[p] && canon[p] == p) blob_of[p] = next++;
    }
    for (int i = 0; i < n; ++i) {
        for (uint64_t j = 0; pf[i] + j < pf[i + 1]; ++j) {
            uint64_t p = pf[i] + j;
            tbl_off[p] = j * (uint64_t)S;
            tbl_alloc[p] = (uint32_t)i;
            tbl_blob[p] = zero[p] ? KCO_BLOB_ZERO : blob_of[canon[p]];
        }
    }
    *n_blobs = next;
    free(pf); free(rec); free(reps); free(blob_of);
    return 0;
}

/*
 * Pack: blob b's S-byte arena slot holds the bytes of its canonical page; a
 * partial page is followed by zeros up to S.
 */
void kco_pack(int n, const uint8_t *const *img, const uint64_t *bytes, uint32_t S,
              const uint64_t *tbl_off, const uint32_t *tbl_alloc, const uint32_t *tbl_blob,
              const uint64_t *canon, uint8_t *arena) {
    uint64_t P = kco_page_first(n, bytes, S, NULL);
    for (uint64_t p = 0; p < P; ++p) {
        if (tbl_blob[p] == KCO_BLOB_ZERO || canon[p] != p) continue;
        uint32_t a = tbl_alloc[p];
        uint64_t off = tbl_off[p];
        uint64_t len = bytes[a] - off < S ? bytes[a] - off : S;
        uint8_t *slot = arena + (uint64_t)tbl_blob[p] * S;
        memcpy(slot, img[a] + off, (size_t)len);
        memset(slot + len, 0, (size_t)(S - len));
    }
}

/*
 * Restore: every page row writes its region at base + VA offset; a zero page
 * writes zeros, any other page copies `len` bytes of its blob's arena slot.
 * `img[i]` is region i's restore target (the caller may pre-fill it with a
 * sentinel to prove that every byte gets written).
 */
void kco_restore(int n, uint8_t *const *img, const uint64_t *bytes, uint32_t S,
                 uint64_t P, const uint64_t *tbl_off, const uint32_t *tbl_alloc,
                 const uint32_t *tbl_blob, const uint8_t *arena) {
    (void)n;
    for (uint64_t p = 0; p < P; ++p) {
        uint32_t a = tbl_alloc[p];
        uint64_t off = tbl_off[p];
        uint64_t len = bytes[a] - off < S ? bytes[a] - off : S;
        if (tbl_blob[p] == KCO_BLOB_ZERO) memset(img[a] + off, 0, (size_t)len);
        else memcpy(img[a] + off, arena + (uint64_t)tbl_blob[p] * S, (size_t)len);
    }
}

/* ------------------------------------------------------------------------ */
/* Census.                                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t src_offset;
    uint64_t value;
    uint32_t src_alloc;
    int32_t target;
} kco_hit;

typedef struct {
    uint64_t base;
    uint64_t end;
    int32_t id;
} kco_range;

static int cmp_range(const void *a, const void *b) {
    const kco_range *x = (const kco_range *)a, *y = (const kco_range *)b;
    if (x->base != y->base) return x->base < y->base ? -1 : 1;
    return 0;
}

/*
 * Census of embedded device pointers.  Regions are the half-open ranges
 * [base_k, base_k + bytes_k); they must not overlap.  For region i in list
 * order and every offset o = 0, 8, 16, ... with o + 8 <= scan_i, the word v
 * (little-endian u64) is INSIDE when some range holds it (target = that
 * region's list index), else OUTSIDE when win_lo <= v < win_hi (target -1),
 * else not a hit.  scan_i = bytes_i unless `scan` is given: a region with a
 * shorter scan length is still a whole target range but only its first
 * scan_i bytes (the image provided) are read; scan_i = 0 makes it a target
 * only, like a region that could not be read.  Hits are listed in (region,
 * offset) order; at most `cap` are stored, the counts are always the true
 * ones.  Returns 0; 2 if the ranges overlap; 4 if hits were truncated; -1 on
 * OOM.
 */
int kco_census(int n, const uint8_t *const *img, const uint64_t *base, const uint64_t *bytes,
               const uint64_t *scan, uint64_t win_lo, uint64_t win_hi, kco_hit *hits,
               uint64_t cap, uint64_t *n_inside, uint64_t *n_outside) {
    kco_range *rg = (kco_range *)malloc(sizeof(kco_range) * (size_t)(n ? n : 1));
    if (!rg) return -1;
    for (int k = 0; k < n; ++k) { rg[k].base = base[k]; rg[k].end = base[k] + bytes[k]; rg[k].id = k; }
    qsort(rg, (size_t)n, sizeof(kco_range), cmp_range);
    for (int k = 1; k < n; ++k) {
        if (rg[k].base < rg[k - 1].end) { free(rg); return 2; }
    }
    uint64_t cnt = 0, nin = 0, nout = 0;
    for (int i = 0; i < n; ++i) {
        uint64_t lim = scan ? scan[i] : bytes[i];
        for (uint64_t o = 0; o + 8 <= lim; o += 8) {
            uint64_t v = le64(img[i] + o);
            /* upper bound: first range whose base is > v */
            int lo = 0, hi = n;
            while (lo < hi) {
                int mid = lo + (hi - lo) / 2;
                if (rg[mid].base <= v) lo = mid + 1; else hi = mid;
            }
            int32_t target;
            if (lo > 0 && v < rg[lo - 1].end) { target = rg[lo - 1].id; ++nin; }
            else if (win_lo <= v && v < win_hi) { target = -1; ++nout; }
            else continue;
            if (cnt < cap && hits) {
                hits[cnt].src_offset = o;
                hits[cnt].value = v;
                hits[cnt].src_alloc = (uint32_t)i;
                hits[cnt].target = target;
            }
            ++cnt;
        }
    }
    *n_inside = nin;
    *n_outside = nout;
    free(rg);
    return cnt > cap ? 4 : 0;
}

/* ------------------------------------------------------------------------ */
/* Compare.                                                                  */
/* ------------------------------------------------------------------------ */

enum { KCO_U8 = 0, KCO_I32 = 1, KCO_F16 = 2, KCO_BF16 = 3, KCO_F32 = 4, KCO_RAW = 5 };

typedef struct {
    uint64_t mismatches;
    int64_t first;
    double max_abs;
    double max_rel;
    uint64_t nan_got;
    uint64_t nan_want;
    uint64_t nan_mismatch;
    int32_t status;
    uint32_t reserved;
} kco_cmp;

/* IEEE binary16 -> double from the bit fields (sign, 5-bit exponent, 10-bit
 * fraction): subnormals are frac * 2^-24, exponent 31 is inf or NaN. */
static double f16_to_f64(uint16_t h) {
    int sign = (h >> 15) & 1;
    int ex = (h >> 10) & 0x1F;
    int fr = h & 0x3FF;
    double v;
    if (ex == 0) v = ldexp((double)fr, -24);
    else if (ex == 31) v = fr ? NAN : INFINITY;
    else v = ldexp((double)(fr | 0x400), ex - 25);
    return sign ? -v : v;
}

/* bfloat16 is the top half of an IEEE binary32: widen the bits, then cast. */
static double bf16_to_f64(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double elem_f64(const uint8_t *p, int dtype, uint64_t i) {
    switch (dtype) {
    case KCO_U8:
    case KCO_RAW: return (double)p[i];
    case KCO_I32: { int32_t v; memcpy(&v, p + 4 * i, 4); return (double)v; }
    case KCO_F16: { uint16_t v; memcpy(&v, p + 2 * i, 2); return f16_to_f64(v); }
    case KCO_BF16: { uint16_t v; memcpy(&v, p + 2 * i, 2); return bf16_to_f64(v); }
    case KCO_F32: { float v; memcpy(&v, p + 4 * i, 4); return (double)v; }
    }
    return NAN;
}

/*
 * Element-wise comparison of `got` against `want`, n elements of `dtype`,
 * both widened exactly to double (a, b):
 *   - a, b both NaN: equal (any NaN equals any NaN).
 *   - exactly one NaN: a mismatch, counted in nan_mismatch, no error value.
 *   - a == b (so +0 == -0 and equal infinities): equal.
 *   - otherwise d = |a - b| and r = d / |b| (r = +inf when b == 0 or d is
 *     infinite); max_abs / max_rel are the maxima of d / r over all such
 *     unequal pairs, starting at +0.  The pair is a mismatch when either
 *     value is infinite, or when d > atol + rtol * |b| (numpy.isclose's
 *     closeness test, negated).
 * first = smallest mismatching element index, -1 if none.
 */
void kco_compare(const void *got, const void *want, int dtype, uint64_t n,
                 double atol, double rtol, kco_cmp *out) {
    const uint8_t *g = (const uint8_t *)got, *w = (const uint8_t *)want;
    kco_cmp r;
    memset(&r, 0, sizeof(r));
    r.first = -1;
    r.max_abs = 0.0;
    r.max_rel = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        double a = elem_f64(g, dtype, i);
        double b = elem_f64(w, dtype, i);
        int na = isnan(a) != 0, nb = isnan(b) != 0;
        r.nan_got += (uint64_t)na;
        r.nan_want += (uint64_t)nb;
        if (na && nb) continue;
        if (na != nb) {
            r.mismatches += 1;
            r.nan_mismatch += 1;
            if (r.first < 0) r.first = (int64_t)i;
            continue;
        }
        if (a == b) continue;
        double d = fabs(a - b);
        double rel = (b == 0.0 || isinf(d)) ? INFINITY : d / fabs(b);
        if (d > r.max_abs) r.max_abs = d;
        if (rel > r.max_rel) r.max_rel = rel;
        int mis;
        if (isinf(a) || isinf(b)) mis = 1;
        else mis = d > atol + rtol * fabs(b);
        if (mis) {
            r.mismatches += 1;
            if (r.first < 0) r.first = (int64_t)i;
        }
    }
    *out = r;
}
