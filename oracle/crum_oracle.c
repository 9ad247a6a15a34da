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
 *
 * Compressed form (version 2, flags bit 1 set): the same header fields,
 * then the allocation table, page table and page hashes as above, then a
 * slot-offset table, n x u64 (offset of each encoded slot from the payload
 * start, ascending from 0), zeros up to the payload offset
 * 64 + 16 A + 24 n rounded up to a multiple of 16, the encoded slots back to
 * back, and the trailer.  A slot is the 65,536-byte payload slot above
 * (valid bytes, then zeros), encoded by oracle_bpd_encode; an encoded length
 * of 65,536 means the slot is stored as is.
 *
 * Byte-plane dictionary code of one slot (the compression of the drained
 * bytes stated in include/crum.h; the paper compresses whole images with
 * gzip or LZ4 on the host, Section 4.4): plane j (j = 0..7) is the 8,192 bytes at offsets
 * 8i + j.  For each plane let D be its distinct byte values in ascending
 * order, k = |D| and b = ceil(log2 k) (b = 0 when k = 1).  A plane with
 * b = 8 is stored as its 8,192 bytes; otherwise as D (k bytes, zero-padded
 * to a multiple of 16) followed by 1,024 b bytes holding, for i = 0..8191,
 * the position of plane byte i in D as b bits at bit offset i b (bit t of
 * the stream is bit t mod 8 of byte t / 8).  The encoded slot is a 16-byte
 * head (b of each plane, then k - 1 of each plane, 255 for a stored plane)
 * and the eight plane sections in order; if that would not be shorter than
 * 65,536 bytes the slot is stored as is.
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

/* ------------------------------------------------------ compressed form --- */

#define OR_PLANE 8192ull

static uint64_t round16(uint64_t x)
{
    return (x + 15) / 16 * 16;
}

/* Encode one 65,536-byte slot into out (room for 65,536 bytes); returns the
 * encoded length, 65,536 meaning stored as is. */
uint64_t oracle_bpd_encode(const uint8_t *slot, uint8_t *out)
{
    uint8_t dict[8][256];
    int k[8], b[8];
    uint64_t len = 16;
    for (int j = 0; j < 8; ++j) {
        uint8_t present[256];
        memset(present, 0, sizeof present);
        for (uint64_t i = 0; i < OR_PLANE; ++i)
            present[slot[8 * i + j]] = 1;
        k[j] = 0;
        for (int v = 0; v < 256; ++v)
            if (present[v])
                dict[j][k[j]++] = (uint8_t)v;
        b[j] = 0;
        while ((1 << b[j]) < k[j])
            b[j] = b[j] + 1;
        if (b[j] == 8)
            len += OR_PLANE;
        else
            len += round16((uint64_t)k[j]) + 1024ull * (uint64_t)b[j];
    }
    if (len >= OR_PAGE) {
        memcpy(out, slot, OR_PAGE);
        return OR_PAGE;
    }
    memset(out, 0, len);
    for (int j = 0; j < 8; ++j) {
        out[j] = (uint8_t)b[j];
        out[8 + j] = b[j] == 8 ? 255 : (uint8_t)(k[j] - 1);
    }
    uint64_t pos = 16;
    for (int j = 0; j < 8; ++j) {
        if (b[j] == 8) {
            for (uint64_t i = 0; i < OR_PLANE; ++i)
                out[pos + i] = slot[8 * i + j];
            pos += OR_PLANE;
            continue;
        }
        memcpy(out + pos, dict[j], (size_t)k[j]);
        pos += round16((uint64_t)k[j]);
        for (uint64_t i = 0; i < OR_PLANE; ++i) {
            int rank = 0;
            while (dict[j][rank] != slot[8 * i + j])
                rank = rank + 1;
            for (int t = 0; t < b[j]; ++t) {
                uint64_t bit = i * (uint64_t)b[j] + (uint64_t)t;
                out[pos + bit / 8] |= (uint8_t)(((rank >> t) & 1) << (bit % 8));
            }
        }
        pos += 1024ull * (uint64_t)b[j];
    }
    return len;
}

/* Decode `len` encoded bytes into a 65,536-byte slot.  OR_OK, or
 * OR_CORRUPT for anything the encoder cannot have written. */
int oracle_bpd_decode(const uint8_t *in, uint64_t len, uint8_t *slot)
{
    if (len == OR_PAGE) {
        memcpy(slot, in, OR_PAGE);
        return OR_OK;
    }
    if (len < 16 || len > OR_PAGE || len % 16 != 0)
        return OR_CORRUPT;
    uint64_t pos = 16;
    for (int j = 0; j < 8; ++j) {
        int b = in[j];
        if (b == 8) {
            if (in[8 + j] != 255 || pos + OR_PLANE > len)
                return OR_CORRUPT;
            for (uint64_t i = 0; i < OR_PLANE; ++i)
                slot[8 * i + j] = in[pos + i];
            pos += OR_PLANE;
            continue;
        }
        if (b > 7)
            return OR_CORRUPT;
        int k = in[8 + j] + 1;
        int canon = 0;
        while ((1 << canon) < k)
            canon = canon + 1;
        if (canon != b)
            return OR_CORRUPT;
        const uint8_t *dict = in + pos;
        if (pos + round16((uint64_t)k) + 1024ull * (uint64_t)b > len)
            return OR_CORRUPT;
        for (int v = 1; v < k; ++v)
            if (dict[v] <= dict[v - 1])
                return OR_CORRUPT;
        pos += round16((uint64_t)k);
        for (uint64_t i = 0; i < OR_PLANE; ++i) {
            int rank = 0;
            for (int t = 0; t < b; ++t) {
                uint64_t bit = i * (uint64_t)b + (uint64_t)t;
                rank |= ((in[pos + bit / 8] >> (bit % 8)) & 1) << t;
            }
            if (rank >= k)
                return OR_CORRUPT;
            slot[8 * i + j] = dict[rank];
        }
        pos += 1024ull * (uint64_t)b;
    }
    return pos == len ? OR_OK : OR_CORRUPT;
}

static uint64_t cimage_payload_off(uint32_t A, uint64_t n)
{
    return round16(OR_HDR + 16ull * A + 24ull * n);
}

/*
 * Compressed image (version 2) of the pages with dirty[g] set into out;
 * `scratch` holds n x 65,536 bytes (the encoded slots are made there
 * first).  Returns the image size, 0 if out_size is too small.  With out
 * NULL it only returns the size.
 */
uint64_t oracle_build_cimage(const uint8_t *const *data, const uint64_t *bytes,
                             const uint32_t *ids, uint32_t n_allocs,
                             const uint64_t *h, const uint8_t *dirty,
                             int full, uint64_t seq, uint64_t parent_seq,
                             uint8_t *scratch, uint64_t *lens,
                             uint8_t *out, uint64_t out_size)
{
    uint64_t n_pages = oracle_total_pages(bytes, n_allocs);
    uint64_t n = 0;
    for (uint64_t g = 0; g < n_pages; ++g)
        n += dirty[g] ? 1 : 0;
    /* encode every dirty slot (valid bytes, then zeros) */
    uint8_t slot[65536];
    uint64_t g = 0, s = 0, total = 0;
    for (uint32_t a = 0; a < n_allocs; ++a)
        for (uint64_t p = 0; p < oracle_pages_of(bytes[a]); ++p) {
            if (dirty[g]) {
                memset(slot, 0, sizeof slot);
                memcpy(slot, data[a] + p * OR_PAGE, oracle_valid_bytes(bytes[a], p));
                lens[s] = oracle_bpd_encode(slot, scratch + OR_PAGE * s);
                total += lens[s];
                s = s + 1;
            }
            g = g + 1;
        }
    uint64_t payload_off = cimage_payload_off(n_allocs, n);
    uint64_t size = payload_off + total + 8;
    if (out == NULL)
        return size;
    if (out_size < size)
        return 0;
    memset(out, 0, size);
    memcpy(out, "CRUMIMG1", 8);
    put32(out + 8, 2);
    put32(out + 12, (full ? 1u : 0u) | 2u);
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
        put64(atab + 16ull * a + 8, bytes[a]);
    }
    uint8_t *ptab = atab + 16ull * n_allocs;
    uint8_t *htab = ptab + 8ull * n;
    uint8_t *otab = htab + 8ull * n;
    g = 0;
    s = 0;
    uint64_t off = 0;
    for (uint32_t a = 0; a < n_allocs; ++a)
        for (uint64_t p = 0; p < oracle_pages_of(bytes[a]); ++p) {
            if (dirty[g]) {
                put32(ptab + 8 * s, a);
                put32(ptab + 8 * s + 4, (uint32_t)p);
                put64(htab + 8 * s, h[g]);
                put64(otab + 8 * s, off);
                memcpy(out + payload_off + off, scratch + OR_PAGE * s, lens[s]);
                off += lens[s];
                s = s + 1;
            }
            g = g + 1;
        }
    put64(out + size - 8, oracle_hash_bytes(out, size - 8, 0));
    return size;
}

/* Check a compressed image like oracle_check_image, plus its offset table
 * (ascending from 0, each length a multiple of 16 in [16, 65536]). */
int oracle_check_cimage(const uint8_t *img, uint64_t size)
{
    if (size < OR_HDR + 8 || memcmp(img, "CRUMIMG1", 8) != 0)
        return OR_CORRUPT;
    if (get32(img + 8) != 2 || (get32(img + 12) & 2u) == 0 || get32(img + 32) != (uint32_t)OR_PAGE)
        return OR_CORRUPT;
    uint32_t A = get32(img + 36);
    uint64_t n = get64(img + 40);
    if (n > size / 16)
        return OR_CORRUPT;
    uint64_t payload_off = get64(img + 48);
    if (payload_off != cimage_payload_off(A, n) || get64(img + 56) != size || payload_off + 8 > size)
        return OR_CORRUPT;
    const uint8_t *otab = img + OR_HDR + 16ull * A + 16ull * n;
    uint64_t total = size - 8 - payload_off;
    for (uint64_t s = 0; s < n; ++s) {
        uint64_t lo = get64(otab + 8 * s);
        uint64_t hi = s + 1 < n ? get64(otab + 8 * (s + 1)) : total;
        if ((s == 0 && lo != 0) || hi < lo || hi - lo < 16 || hi - lo > OR_PAGE || (hi - lo) % 16 != 0)
            return OR_CORRUPT;
    }
    if (n == 0 && total != 0)
        return OR_CORRUPT;
    if (oracle_hash_bytes(img, size - 8, 0) != get64(img + size - 8))
        return OR_CORRUPT;
    return OR_OK;
}

/* Apply one compressed image, as oracle_apply_image does an uncompressed
 * one (every slot is decoded first; nothing is written if any fails). */
int oracle_apply_cimage(const uint8_t *img, uint64_t size,
                        uint8_t *const *data, const uint64_t *bytes,
                        uint32_t n_allocs, uint64_t *h_prev, uint8_t *scratch)
{
    int st = oracle_check_cimage(img, size);
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
    const uint8_t *otab = htab + 8ull * n;
    uint64_t payload_off = get64(img + 48);
    uint64_t total = size - 8 - payload_off;
    for (uint64_t s = 0; s < n; ++s) {
        uint32_t a = get32(ptab + 8 * s);
        uint32_t p = get32(ptab + 8 * s + 4);
        if (a >= A || (uint64_t)p >= oracle_pages_of(bytes[a]))
            return OR_CORRUPT;
        uint64_t lo = get64(otab + 8 * s);
        uint64_t hi = s + 1 < n ? get64(otab + 8 * (s + 1)) : total;
        if (oracle_bpd_decode(img + payload_off + lo, hi - lo, scratch + OR_PAGE * s) != OR_OK)
            return OR_CORRUPT;
    }
    for (uint64_t s = 0; s < n; ++s) {
        uint32_t a = get32(ptab + 8 * s);
        uint32_t p = get32(ptab + 8 * s + 4);
        uint64_t first = 0;
        for (uint32_t b = 0; b < a; ++b)
            first += oracle_pages_of(bytes[b]);
        memcpy(data[a] + (uint64_t)p * OR_PAGE, scratch + OR_PAGE * s,
               oracle_valid_bytes(bytes[a], p));
        if (h_prev)
            h_prev[first + p] = get64(htab + 8 * s);
    }
    return OR_OK;
}
