/*
 * CPU oracle for the CRUM capture/restore path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  The product path
 * (the CUDA library under paper_1808_00117_b300/) never calls it, and this
 * file shares no code, header or constant table with that path.
 *
 * Plain, slow and obviously correct: every function is one loop over the
 * definition it implements, in the order the definition states it, with no
 * blocking, fusion or reordering.  All arithmetic is on uint64_t, which C
 * defines modulo 2^64.
 *
 * What is defined where (CRUM, Garg, Mohan, Sullivan, Cooperman, 2018):
 *   - Dirty pages.  Algorithm 1 and Section 3.2 track, per page of a managed
 *     region, whether it was written since the last synchronisation; a new
 *     region starts with every page dirty, and the dirty set is cleared once
 *     the pages have been flushed.  Device stores raise no fault that a user
 *     can trap, so here a page is dirty when the 64-bit hash of its contents
 *     differs from the hash taken at the previous checkpoint (or the
 *     checkpoint is full, or it is the first one since the region was
 *     registered).
 *   - The page hash is the sum modulo 2^64 of splitmix64's output function
 *     (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 *     OOPSLA 2014; Vigna's public-domain splitmix64) applied to each 8-byte
 *     little-endian word XOR its page-local index times the golden-ratio
 *     constant.  A sum is order-free, so any split of a page gives the same
 *     value.
 *   - Capture.  Section 3.4: at a checkpoint every region's data is read
 *     from the device to the host and saved; Section 3.3: the device is
 *     drained first, and storage proceeds while the application resumes.
 *     Here only dirty pages are copied, into an image, in ascending
 *     (registration order, page index) order.
 *   - Restore.  Section 3.4: a new process replays the allocations and the
 *     saved data is copied back into them; Section 5 relies on the regions
 *     coming back at the same places.  Here the registration table of the
 *     image must match the target's (count and sizes, in order) and each
 *     image of a chain is applied from the full base to the end, later pages
 *     winning.
 *   - Verify mode.  Section 3.2.1 asks for a slower verified mode that checks
 *     the assumption dirty tracking rests on.  Here it is an exact byte
 *     compare of every hash-clean page against the previous contents: a
 *     mismatch is a hash collision, which is counted and makes the page dirty.
 *
 * Image layout (all integers little-endian):
 *   header, 64 bytes:
 *     [0,8)   magic "CRUMIMG1"
 *     [8,12)  u32 version (1)
 *     [12,16) u32 flags (bit 0: full image)
 *     [16,24) u64 seq
 *     [24,32) u64 parent seq (all ones for a full image)
 *     [32,36) u32 page size (65536)
 *     [36,40) u32 number of allocations A
 *     [40,48) u64 number of dirty pages n
 *     [48,56) u64 payload offset (64 + 16 A + 16 n)
 *     [56,64) u64 image size in bytes, trailer included
 *   allocation table, A x 16 bytes: u32 id, u32 zero, u64 bytes
 *   page table, n x 8 bytes: u32 allocation index, u32 page index
 *   page hashes, n x u64
 *   payload, n x 65536 bytes: the page's valid bytes, then zeros
 *   trailer: u64 checksum = the hash above applied to every preceding byte
 *            of the image, with word indices counted from the image start.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#define OR_PAGE  65536ull
#define OR_PHI   0x9E3779B97F4A7C15ull
#define OR_HDR   64ull
#define OR_NONE  0xFFFFFFFFFFFFFFFFull

enum { OR_OK = 0, OR_CORRUPT = -1, OR_MISMATCH = -2, OR_SPACE = -3 };

/* splitmix64's output function ("mix"), from its published definition. */
uint64_t oracle_mix(uint64_t z)
{
    z = z ^ (z >> 30);
    z = z * 0xBF58476D1CE4E5B9ull;
    z = z ^ (z >> 27);
    z = z * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return z;
}

/* Word i of an n-byte string: little-endian, bytes at or past n read as 0. */
static uint64_t word_at(const uint8_t *p, uint64_t n, uint64_t i)
{
    uint64_t w = 0;
    for (uint64_t b = 0; b < 8; ++b) {
        uint64_t k = 8 * i + b;
        if (k < n)
            w = w | ((uint64_t)p[k] << (8 * b));
    }
    return w;
}

/* sum over i < ceil(n/8) of mix(w_i XOR (first + i) * phi), modulo 2^64. */
uint64_t oracle_hash_bytes(const uint8_t *p, uint64_t n, uint64_t first)
{
    uint64_t nw = (n + 7) / 8;
    uint64_t h = 0;
    for (uint64_t i = 0; i < nw; ++i)
        h = h + oracle_mix(word_at(p, n, i) ^ ((first + i) * OR_PHI));
    return h;
}

/* Page hash: page-local indices from 0 over the page's valid bytes. */
uint64_t oracle_page_hash(const uint8_t *page, uint64_t valid)
{
    return oracle_hash_bytes(page, valid, 0);
}

uint64_t oracle_pages_of(uint64_t bytes)
{
    return (bytes + OR_PAGE - 1) / OR_PAGE;
}

/* Valid bytes of page p of an allocation of `bytes` bytes. */
uint64_t oracle_valid_bytes(uint64_t bytes, uint64_t p)
{
    uint64_t start = p * OR_PAGE;
    uint64_t left = bytes - start;
    return left < OR_PAGE ? left : OR_PAGE;
}

uint64_t oracle_total_pages(const uint64_t *bytes, uint32_t n_allocs)
{
    uint64_t t = 0;
    for (uint32_t a = 0; a < n_allocs; ++a)
        t += oracle_pages_of(bytes[a]);
    return t;
}

/* out[g] for every global page g = (registration order, page index). */
void oracle_hash_all(const uint8_t *const *data, const uint64_t *bytes,
                     uint32_t n_allocs, uint64_t *out)
{
    uint64_t g = 0;
    for (uint32_t a = 0; a < n_allocs; ++a)
        for (uint64_t p = 0; p < oracle_pages_of(bytes[a]); ++p) {
            out[g] = oracle_page_hash(data[a] + p * OR_PAGE,
                                      oracle_valid_bytes(bytes[a], p));
            g = g + 1;
        }
}

/*
 * dirty[g] = full OR force[g] OR h[g] != h_prev[g].  force marks pages of
 * allocations with no checkpoint since registration (Algorithm 1: a new
 * region starts all dirty); NULL means none.  Returns the dirty count.
 */
uint64_t oracle_dirty(const uint64_t *h, const uint64_t *h_prev,
                      const uint8_t *force, int full, uint64_t n_pages,
                      uint8_t *dirty)
{
    uint64_t n = 0;
    for (uint64_t g = 0; g < n_pages; ++g) {
        int d = full || (force && force[g]) || h[g] != h_prev[g];
        dirty[g] = (uint8_t)d;
        n += (uint64_t)d;
    }
    return n;
}

/*
 * Verify mode: every page the hash calls clean (dirty[g] == 0) is compared
 * byte for byte with its previous contents; a difference is a collision,
 * which is counted and turns the page dirty.  Returns the collision count.
 */
uint64_t oracle_verify(const uint8_t *const *data, const uint8_t *const *prev,
                       const uint64_t *bytes, uint32_t n_allocs, uint8_t *dirty)
{
    uint64_t g = 0, collisions = 0;
    for (uint32_t a = 0; a < n_allocs; ++a)
        for (uint64_t p = 0; p < oracle_pages_of(bytes[a]); ++p) {
            if (!dirty[g]) {
                uint64_t v = oracle_valid_bytes(bytes[a], p);
                if (memcmp(data[a] + p * OR_PAGE, prev[a] + p * OR_PAGE, v) != 0) {
                    dirty[g] = 1;
                    collisions = collisions + 1;
                }
            }
            g = g + 1;
        }
    return collisions;
}

uint64_t oracle_image_size(uint32_t n_allocs, uint64_t n_dirty)
{
    return OR_HDR + 16ull * n_allocs + 16ull * n_dirty + OR_PAGE * n_dirty + 8;
}

static void put32(uint8_t *p, uint32_t v)
{
    for (int b = 0; b < 4; ++b)
        p[b] = (uint8_t)(v >> (8 * b));
}

static void put64(uint8_t *p, uint64_t v)
{
    for (int b = 0; b < 8; ++b)
        p[b] = (uint8_t)(v >> (8 * b));
}

static uint32_t get32(const uint8_t *p)
{
    uint32_t v = 0;
    for (int b = 0; b < 4; ++b)
        v |= (uint32_t)p[b] << (8 * b);
    return v;
}

static uint64_t get64(const uint8_t *p)
{
    uint64_t v = 0;
    for (int b = 0; b < 8; ++b)
        v |= (uint64_t)p[b] << (8 * b);
    return v;
}

/*
 * Write the image of the pages with dirty[g] set, in ascending g, into out
 * (out_size bytes, which must be oracle_image_size(n_allocs, n_dirty)).
 * Returns the image size, or 0 if out_size is wrong.
 */
uint64_t oracle_build_image(const uint8_t *const *data, const uint64_t *bytes,
                            const uint32_t *ids, uint32_t n_allocs,
                            const uint64_t *h, const uint8_t *dirty,
                            int full, uint64_t seq, uint64_t parent_seq,
                            uint8_t *out, uint64_t out_size)
{
    uint64_t n_pages = oracle_total_pages(bytes, n_allocs);
    uint64_t n = 0;
    for (uint64_t g = 0; g < n_pages; ++g)
        n += dirty[g] ? 1 : 0;
    uint64_t size = oracle_image_size(n_allocs, n);
    if (out_size != size)
        return 0;
    memset(out, 0, size);

    uint64_t payload_off = OR_HDR + 16ull * n_allocs + 16ull * n;
    memcpy(out, "CRUMIMG1", 8);
    put32(out + 8, 1);
    put32(out + 12, full ? 1u : 0u);
    put64(out + 16, seq);
    put64(out + 24, full ? OR_NONE : parent_seq);
    put32(out + 32, (uint32_t)OR_PAGE);
    put32(out + 36, n_allocs);
    put64(out + 40, n);
    put64(out + 48, payload_off);
    put64(out + 56, size);

    uint8_t *atab = out + OR_HDR;
    for (uint32_t a = 0; a < n_allocs; ++a) {
        put32(atab + 16ull * a, ids[a]);
        put32(atab + 16ull * a + 4, 0);
        put64(atab + 16ull * a + 8, bytes[a]);
    }

    uint8_t *ptab = atab + 16ull * n_allocs;
    uint8_t *htab = ptab + 8ull * n;
    uint8_t *payload = out + payload_off;
    uint64_t g = 0, s = 0;
    for (uint32_t a = 0; a < n_allocs; ++a)
        for (uint64_t p = 0; p < oracle_pages_of(bytes[a]); ++p) {
            if (dirty[g]) {
                put32(ptab + 8 * s, a);
                put32(ptab + 8 * s + 4, (uint32_t)p);
                put64(htab + 8 * s, h[g]);
                memcpy(payload + OR_PAGE * s, data[a] + p * OR_PAGE,
                       oracle_valid_bytes(bytes[a], p));
                s = s + 1;
            }
            g = g + 1;
        }

    put64(out + size - 8, oracle_hash_bytes(out, size - 8, 0));
    return size;
}

/*
 * Check an image: magic, version, page size, self-described size equal to
 * `size`, table bounds, and the trailer checksum.  OR_OK or OR_CORRUPT.
 */
int oracle_check_image(const uint8_t *img, uint64_t size)
{
    if (size < OR_HDR + 8 || memcmp(img, "CRUMIMG1", 8) != 0)
        return OR_CORRUPT;
    if (get32(img + 8) != 1 || get32(img + 32) != (uint32_t)OR_PAGE)
        return OR_CORRUPT;
    uint32_t A = get32(img + 36);
    uint64_t n = get64(img + 40);
    if (n > size / OR_PAGE)
        return OR_CORRUPT;
    if (get64(img + 56) != size || oracle_image_size(A, n) != size)
        return OR_CORRUPT;
    if (get64(img + 48) != OR_HDR + 16ull * A + 16ull * n)
        return OR_CORRUPT;
    if (oracle_hash_bytes(img, size - 8, 0) != get64(img + size - 8))
        return OR_CORRUPT;
    return OR_OK;
}

/*
 * Apply one image to the registered allocations (data[a] writable, bytes[a]
 * their sizes): the image's allocation table must list the same sizes in
 * the same order (else OR_MISMATCH); each payload slot's valid bytes go to
 * its page and the image's hash for that page goes to h_prev (global page
 * numbering).  The image is checked first and nothing is written if it
 * fails.
 */
int oracle_apply_image(const uint8_t *img, uint64_t size,
                       uint8_t *const *data, const uint64_t *bytes,
                       uint32_t n_allocs, uint64_t *h_prev)
{
    int st = oracle_check_image(img, size);
    if (st != OR_OK)
        return st;
    uint32_t A = get32(img + 36);
    uint64_t n = get64(img + 40);
    if (A != n_allocs)
        return OR_MISMATCH;
    const uint8_t *atab = img + OR_HDR;
    for (uint32_t a = 0; a < A; ++a)
        if (get64(atab + 16ull * a + 8) != bytes[a])
            return OR_MISMATCH;

    const uint8_t *ptab = atab + 16ull * A;
    const uint8_t *htab = ptab + 8ull * n;
    const uint8_t *payload = img + get64(img + 48);
    for (uint64_t s = 0; s < n; ++s) {
        uint32_t a = get32(ptab + 8 * s);
        uint32_t p = get32(ptab + 8 * s + 4);
        if (a >= A || (uint64_t)p >= oracle_pages_of(bytes[a]))
            return OR_CORRUPT;
    }
    for (uint64_t s = 0; s < n; ++s) {
        uint32_t a = get32(ptab + 8 * s);
        uint32_t p = get32(ptab + 8 * s + 4);
        uint64_t first = 0;
        for (uint32_t b = 0; b < a; ++b)
            first += oracle_pages_of(bytes[b]);
        memcpy(data[a] + (uint64_t)p * OR_PAGE, payload + OR_PAGE * s,
               oracle_valid_bytes(bytes[a], p));
        if (h_prev)
            h_prev[first + p] = get64(htab + 8 * s);
    }
    return OR_OK;
}
