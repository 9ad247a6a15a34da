/*
 * crum.h -- C ABI of the B300 capture/restore library for device-resident
 * managed allocations (CRUM: Checkpoint-Restart Support for CUDA's Unified
 * Memory, Garg, Mohan, Sullivan, Cooperman, 2018).
 *
 * Conventions for every entry point:
 *   - Returns a crum_status; CRUM_OK is 0.  No C++ exception crosses this
 *     boundary.  crum_last_error() gives a message for the calling thread's
 *     last failure.
 *   - "device pointer" means a pointer the current CUDA device can read
 *     and write (cudaMalloc, cudaMallocManaged with the device as preferred
 *     location, or a PyTorch CUDA tensor's data pointer).  "host pointer" is
 *     ordinary process memory.
 *   - crum_stream_t is a cudaStream_t passed as an opaque pointer (0 means
 *     the legacy default stream).
 *   - Work is stream ordered: a call that takes a stream sees every earlier
 *     operation on that stream and nothing later.
 *   - Page size is fixed at CRUM_PAGE_SIZE bytes.  Page p of an allocation
 *     of B bytes covers bytes [p*P, min((p+1)*P, B)); the last page may be
 *     partial ("tail page").
 *   - The library owns sets, images, staging buffers, pinned host memory and
 *     hash tables.  The caller owns the registered allocations; the library
 *     never frees, moves or resizes them.
 *
 * Page hash used for dirty detection (stands in for the write-fault dirty
 * tracking of Algorithm 1 / Section 3.2, since device stores cannot be
 * trapped): for a page with v valid bytes, read as ceil(v/8) little-endian
 * 64-bit words w_i (a final partial word zero-padded),
 *     h = sum_i mix(w_i XOR (i * 0x9E3779B97F4A7C15))   (mod 2^64)
 * where mix is splitmix64's output function (Steele, Lea, Flood, 2014).
 *
 * Image byte layout (little-endian), produced by crum_checkpoint and read by
 * crum_image_load / crum_restore:
 *   header (64 B): "CRUMIMG1", u32 version=1, u32 flags (bit0 full),
 *     u64 seq, u64 parent seq (all ones for a full image), u32 page size,
 *     u32 allocation count A, u64 dirty page count n, u64 payload offset
 *     (64+16A+16n), u64 image size including the trailer;
 *   allocation table A x {u32 id, u32 0, u64 bytes};
 *   page table n x {u32 allocation index, u32 page index}, ascending;
 *   page hashes n x u64;
 *   payload n x CRUM_PAGE_SIZE bytes (valid bytes, then zeros);
 *   trailer u64 = the hash formula above over every preceding image byte,
 *     word indices counted from the start of the image.
 *
 * Compressed form (crum_config.compress; version 2, flags bit 1): header,
 * allocation table, page table and hashes as above, then n x u64 slot
 * offsets (from the payload start, ascending from 0), zeros up to the
 * payload offset round_up(64 + 16A + 24n, 16), the encoded slots back to
 * back (slot s ends where slot s + 1 starts, the last at the trailer), the
 * trailer.  A slot (64 KiB: valid bytes, then zeros) is split into 8 byte
 * planes of 8,192 bytes (plane j = bytes 8i + j).  For a plane with k
 * distinct values and b = ceil(log2 k) < 8 the code holds the values in
 * ascending order (zero-padded to a multiple of 16 bytes) and 1,024 b bytes
 * with the position of each plane byte among them, b bits each at bit
 * offset i b, LSB first; a plane with b = 8 is stored as is.  An encoded
 * slot is a 16-byte head (b of each plane, then k - 1, 255 for a stored
 * plane) and the 8 plane sections in order, or, when that would not be
 * shorter, the 65,536 slot bytes as they are (length 65,536).
 */
#ifndef CRUM_H
#define CRUM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CRUM_PAGE_SIZE 65536u
#define CRUM_NO_PARENT 0xFFFFFFFFFFFFFFFFull

typedef enum crum_status {
    CRUM_OK = 0,
    CRUM_EINVAL = 1,      /* bad argument (null, misaligned, overlapping, out of range) */
    CRUM_ENOMEM = 2,      /* device or pinned host allocation failed */
    CRUM_EBUSY = 3,       /* the set has work in flight that forbids the call */
    CRUM_ECUDA = 4,       /* a CUDA runtime call failed; crum_last_error has its text */
    CRUM_EIO = 5,         /* the image sink or a file read/write failed */
    CRUM_EMISMATCH = 6,   /* image allocation table differs from the set's registrations */
    CRUM_ECOLLISION = 7,  /* verify mode found pages whose hash matched but bytes differ */
    CRUM_ETIMEOUT = 8,    /* a bounded wait ran out (host wait or a device-side spin) */
    CRUM_ECORRUPT = 9     /* image failed its structural or checksum checks */
} crum_status;

typedef void *crum_stream_t; /* a cudaStream_t */
typedef struct crum_set crum_set;
typedef struct crum_image crum_image;

/* Where a checkpoint image goes once it has reached host memory. */
typedef enum crum_sink {
    CRUM_SINK_MEMORY = 0, /* keep the image in library-owned pinned host memory */
    CRUM_SINK_FILE = 1,   /* also write it to <sink_dir>/crum_<set>_<seq>.img */
    CRUM_SINK_NULL = 2    /* drain to host, then drop the payload (link benchmark) */
} crum_sink;

typedef struct crum_config {
    int device;                /* CUDA device ordinal the set lives on */
    uint64_t staging_bytes;    /* device staging budget, split into two halves that
                                  alternate between consecutive checkpoints; 0: 1 GiB */
    uint64_t chunk_bytes;      /* largest single device->host copy of a drain: a
                                  payload drains as copies of at most this many
                                  bytes (rounded up to 16, at least 4 KiB), and a
                                  payload that is not kept (null sink,
                                  CRUM_NO_PAYLOAD) lands in a pinned bounce region
                                  of this size; 0: 64 MiB */
    uint64_t host_pool_bytes;  /* initial pinned host pool for images; 0: grow on demand.
                                  Size it for the most image bytes held at once (a
                                  chain kept in memory plus the next full image while
                                  the old chain is still referenced): growing it
                                  pins host memory, which took about 0.3 s for
                                  half a GB here, and the driver holds other
                                  threads' CUDA calls meanwhile */
    int sink;                  /* crum_sink */
    const char *sink_dir;      /* directory for CRUM_SINK_FILE (copied at create) */
    int verify;                /* 1: keep a device copy of the last checkpointed
                                  contents so CRUM_VERIFY checkpoints can byte-compare */
    int fsync;                 /* 1: fsync image files before reporting PERSISTED */
    int hash_mapping;          /* thread mapping of the hash kernel,
                                  0..CRUM_NUM_HASH_MAPPINGS-1; -1 default.
                                  0-5: register mappings (one warp or one CTA of
                                  256 per page), 6-8: shared-memory bulk-copy
                                  mappings, 9-11: register mappings capped at 32
                                  registers, 12-14: one CTA of 64 or 128 threads
                                  per page */
    int gather_mapping;        /* thread mapping of the gather kernel, 0..5; -1 default */
    int external_staging;      /* 1: allocate no staging; a crum_server lends staging
                                  to the set for each request it admits */
    int use_graph;             /* 1: launch each capture (memsets, hash, scan, gather
                                  and their events; with compress, the encoding
                                  stage too) as one instantiated CUDA graph per
                                  staging half, rebuilt when registrations or
                                  mappings change; verify-mode and chunked captures
                                  use plain launches */
    int max_chain;             /* > 0: after this many incremental images the next
                                  checkpoint is full, so restore replays at most
                                  max_chain + 1 images and older chains can be freed;
                                  0: chains grow without limit */
    int restore_mode;          /* crum_restore of a chain (crum_restore_mode):
                                  0 auto (merged when the chain's incrementals hold
                                  more than 8 % of the base's pages, else replay),
                                  1 replay every image in order, 2 merged: every
                                  page once, from the newest image holding it,
                                  3 delta: merged, but a page whose current
                                  contents already hash to the chain's value is
                                  not copied (a rollback moves only what changed;
                                  a changed page with an equal hash, probability
                                  2^-64, is left as it is, as a checkpoint would) */
    int max_pending;           /* > 0: crum_checkpoint waits until fewer than this
                                  many of the set's images are not yet PERSISTED,
                                  so a sink slower than the checkpoints bounds the
                                  pinned host memory they hold; 0: no bound */
    int compress;              /* 1: images take the compressed form (version 2,
                                  flags bit 1): each payload slot is encoded with
                                  the byte-plane dictionary code below on the
                                  device before it drains, so fewer bytes cross
                                  the link; needs owned (not external) staging.
                                  With staging smaller than the set, the dirty
                                  pages are encoded and drained one staging half
                                  at a time, each chunk's code placed after the
                                  previous chunk's */
    int managed_in_place;      /* 1: managed allocations whose pages the application
                                  placed in host memory (preferred location the
                                  host, or last prefetched there) are read where
                                  they are, over the host link, instead of being
                                  migrated to the device by the capture's page
                                  faults (the oversubscribed case of Section 4.4's
                                  synthetic benchmark, where the device cannot
                                  hold them).  At each checkpoint and restore the
                                  set looks up every managed allocation's
                                  placement (cudaMemRangeGetAttribute) and keeps
                                  its device mapped to the host-placed ones
                                  (cudaMemAdviseSetAccessedBy), withdrawing that
                                  advice when the range moves back, is
                                  unregistered or the set is destroyed; advice the
                                  application set itself is left alone.  While the
                                  advice stands, the application's own kernels
                                  also read those pages in place.  0: pages are
                                  read wherever the driver's policy puts them */
} crum_config;

typedef enum crum_restore_mode {
    CRUM_RESTORE_AUTO = 0,
    CRUM_RESTORE_REPLAY = 1,
    CRUM_RESTORE_MERGED = 2,
    CRUM_RESTORE_DELTA = 3
} crum_restore_mode;

/* Fill *cfg with defaults (device 0, 1 GiB staging, 64 MiB chunks, memory sink). */
void crum_config_default(crum_config *cfg);

/* Thread-local text of the calling thread's last error ("" if none).  The
   pointer stays valid until that thread's next crum_* call. */
const char *crum_last_error(void);

/* Library version string, e.g. "crum-b300 1.0 sm_103a". */
const char *crum_version(void);

/* ---- registration set (Section 3.2: regions tracked per allocation;
        Algorithm 1 "create region": a new region starts with every page
        dirty) ---- */

/* Create a set on cfg->device (NULL: defaults).  Allocates the staging
   halves, hash table capacity grows with registrations.
   Errors: EINVAL (bad config), ENOMEM, ECUDA. */
crum_status crum_set_create(const crum_config *cfg, crum_set **out);

/* Wait for all in-flight checkpoints of the set to persist, stop its writer
   thread and free its device/host memory.  Images the caller still holds
   stay valid (they keep their own host memory).  NULL is a no-op. */
crum_status crum_set_destroy(crum_set *set);

/* Register the allocation [ptr, ptr+bytes) (device pointer, caller owned).
   ptr must be 16-byte aligned and bytes > 0, and the range must not overlap
   a registered one; otherwise EINVAL.  Its pages are dirty at the next
   checkpoint (Algorithm 1: a new region starts all dirty).  *alloc_id gets
   a set-unique id.  Registration order fixes the page order of images.
   Errors: EINVAL, EBUSY (a checkpoint is being captured), ENOMEM. */
crum_status crum_register(crum_set *set, void *ptr, size_t bytes, uint32_t *alloc_id);

/* Remove a registration.  Errors: EINVAL (unknown id), EBUSY. */
crum_status crum_unregister(crum_set *set, uint32_t alloc_id);

/* Number of registrations and total pages of the set. */
crum_status crum_set_info(const crum_set *set, uint32_t *n_allocs, uint64_t *n_pages);

#define CRUM_NUM_HASH_MAPPINGS 15
#define CRUM_NUM_GATHER_MAPPINGS 6

/* Autotuner: time every hash mapping and every gather mapping
   on the set's current registrations and keep the fastest of each for its
   later checkpoints.  Every candidate's page hashes must be bit-identical
   (else ECORRUPT and nothing changes).  Waits for in-flight checkpoints;
   leaves committed hashes and images untouched (it hashes into scratch and
   gathers a synthetic 1-in-8 page set into idle staging).  *hash_mapping and
   *gather_mapping (either may be NULL) receive the choice; *hash_ms and
   *gather_ms (may be NULL) arrays of CRUM_NUM_HASH_MAPPINGS and
   CRUM_NUM_GATHER_MAPPINGS doubles receive the mean
   device time of each candidate.  Errors: EINVAL (no registrations), ECUDA. */
crum_status crum_autotune(crum_set *set, int *hash_mapping, int *gather_mapping,
                          double *hash_ms, double *gather_ms);

/* ---- checkpoint (Section 3.4: read every region from the device and save
        it; Section 3.3: drain the device, then let storage proceed while the
        application runs) ---- */

#define CRUM_INCR   0  /* pages whose hash changed, plus never-checkpointed pages */
#define CRUM_FULL   1  /* every page */
#define CRUM_VERIFY 2  /* also byte-compare hash-clean pages (needs cfg.verify) */
#define CRUM_NO_PAYLOAD 4  /* drain this image's payload across the link but keep only
                              its metadata on the host (as the null sink does): for a
                              base image larger than host memory that only has to set
                              the hashes; a chain through it cannot be restored (EIO) */

/* Take a checkpoint of every registered allocation as of this point in
   app_stream's order.  The capture runs on the set's own streams after the
   work already queued on app_stream; app_stream is made to wait (on the
   device) only until the dirty pages are copied into device staging
   ("captured"); draining to host and persisting continue in the background.
   *out receives a new image handle (refcount 1) whose parent is the
   previous checkpoint's image.  The first checkpoint of a set, and any
   checkpoint after a failed one, is full.
   Returns without waiting for the device when the staging half can hold
   every page of the set; otherwise it waits on the host until the dirty
   count is known (the hash pass), then proceeds in staging-sized chunks,
   and app_stream waits until the last chunk is captured.
   Errors: EINVAL (no registrations, CRUM_VERIFY without cfg.verify),
   ENOMEM, ECUDA, ETIMEOUT. */
crum_status crum_checkpoint(crum_set *set, crum_stream_t app_stream, int flags,
                            crum_image **out);

#define CRUM_WAIT_CAPTURED  1  /* dirty pages copied to device staging */
#define CRUM_WAIT_DRAINED   2  /* image bytes are in host memory */
#define CRUM_WAIT_PERSISTED 3  /* the sink has accepted the image */

/* Block until the image reaches stage `what` or timeout_ns passes (<0: no
   limit).  Returns the image's final status once it is PERSISTED or failed:
   EIO (sink failure; the set's next checkpoint is then full), ECOLLISION
   (verify mode found collisions; the image is still complete and correct,
   the colliding pages were captured), ECUDA, ETIMEOUT. */
crum_status crum_image_wait(crum_image *img, int what, int64_t timeout_ns);

typedef struct crum_image_info {
    uint64_t seq;            /* checkpoint sequence number within the set */
    uint64_t parent_seq;     /* CRUM_NO_PARENT for a full image */
    uint64_t n_dirty;        /* pages in the image */
    uint64_t n_pages;        /* pages of the set when it was taken */
    uint64_t image_bytes;    /* serialized size, trailer included */
    uint64_t checksum;       /* trailer value */
    uint64_t collisions;     /* verify mode: hash-clean pages whose bytes differed */
    uint32_t n_allocs;
    uint32_t full;           /* 1 if this image holds every page */
    int stage;               /* highest CRUM_WAIT_* reached (0: submitted) */
    int status;              /* crum_status of the image so far */
    double t_captured_ms;    /* device time submit->captured (CUDA events) */
    double t_drained_ms;     /* device time submit->drained */
    double t_persisted_ms;   /* host time submit->persisted */
    double t_hash_ms;        /* device time of the page-hash kernel */
    double t_compact_ms;     /* device time of scan + gather into staging, from the
                                moment the staging half was free */
    double t_drain_ms;       /* device time of the device->host copies */
    uint64_t host_pages;     /* pages of host-placed managed allocations the
                                capture read in place (cfg.managed_in_place) */
    double t_encode_ms;      /* compressed images: device time of the encoding
                                stage, from captured until the code and the
                                trailer are written (0 otherwise) */
} crum_image_info;

/* Fill *info.  Fields past `stage` are zero until the image gets there. */
crum_status crum_image_info_get(const crum_image *img, crum_image_info *info);

/* Copy the serialized image (image_bytes bytes) into host memory dst, which
   must hold dst_bytes >= image_bytes.  Waits for DRAINED.
   Errors: EINVAL (dst too small), EIO. */
crum_status crum_image_copy(crum_image *img, void *dst, uint64_t dst_bytes);

/* Write the serialized image to a file.  Waits for DRAINED.  Errors: EIO. */
crum_status crum_image_save(crum_image *img, const char *path);

/* Read an image from a file or a host buffer and check it on the set's
   device: structure, sizes and the trailer checksum (ECORRUPT on any
   failure, ENOENT-like failures are EIO).  parent must be the image with
   seq equal to the file's parent seq (NULL for a full image), else
   EMISMATCH.  The new handle holds a reference to parent. */
crum_status crum_image_load(crum_set *set, const char *path, crum_image *parent,
                            crum_image **out);
crum_status crum_image_from_bytes(crum_set *set, const void *bytes, uint64_t n,
                                  crum_image *parent, crum_image **out);

/* Drop a reference.  The image's memory is freed, and its parent released,
   when the last reference goes. */
crum_status crum_image_release(crum_image *img);

/* ---- restore (Section 3.4: replay allocations, copy the saved data back;
        Section 5: regions must come back at matching places) ---- */

/* Restore the set's registered allocations to the state captured by
   chain_end: the chain's full base image first, then each incremental in
   order, later pages winning.  Only each page's valid bytes are written.
   Two forms with the same result (crum_config.restore_mode): replay copies
   each image's payload to the device in turn (sum of the chain's payloads
   over the link, by DMA); merged finds the newest image of every page on
   the device and copies each page once, read by the kernels straight from
   the images' pinned host memory (one footprint over the link at the
   link's read rate, about 7 % below DMA).
   The set's hash table becomes the chain's hashes, so the next incremental
   checkpoint is relative to chain_end (its parent).  Stream ordered on
   `stream`; returns once the work is queued, and the caller's host image
   memory stays owned by the images.
   Errors: EMISMATCH (allocation count or sizes differ, in registration
   order), ECORRUPT (broken chain), EBUSY (checkpoint being captured),
   ECUDA. */
crum_status crum_restore(crum_set *set, const crum_image *chain_end, crum_stream_t stream);

/* Pages the set's last crum_restore copied across the host link (replay:
   every slot of every chain image; merged: every page; delta: the pages
   whose contents differed).  Waits for that restore to finish.  0 before
   any restore.  Errors: EINVAL, ETIMEOUT, ECUDA. */
crum_status crum_restore_pages(crum_set *set, uint64_t *pages);

/* ---- single-step entry points (each a single step of the path, for tests
        and for callers that manage their own memory) ---- */

/* Page hashes of one allocation: out[p] for every page p of [ptr, ptr+bytes).
   ptr 16-byte aligned device pointer; out a device array of
   ceil(bytes/65536) u64.  Errors: EINVAL, ECUDA. */
crum_status crum_hash_pages(const void *ptr, uint64_t bytes, uint64_t *out,
                            crum_stream_t stream);

/* The same hash over an arbitrary byte string with word indices starting at
   first_index (the image checksum uses first_index 0 over the whole image):
   *out (device u64) = sum of mix(w_i XOR (first_index+i)*phi).  ptr 16-byte
   aligned device pointer.  Errors: EINVAL, ECUDA. */
crum_status crum_hash_bytes(const void *ptr, uint64_t bytes, uint64_t first_index,
                            uint64_t *out, crum_stream_t stream);

/* Copy the set's committed page-hash table (n_pages u64, global page order:
   registration order, then page index) to host memory.  Synchronous. */
crum_status crum_get_hashes(crum_set *set, uint64_t *host_out, uint64_t n);

/* Overwrite one committed page hash (test hook for collision injection:
   verify mode must then report the page).  Synchronous. */
crum_status crum_poke_hash(crum_set *set, uint64_t global_page, uint64_t value);

/* Kernel launches the library has issued since load (for launch accounting). */
uint64_t crum_kernel_launches(void);

/* Self-test of the bounded device waits: hashes [ptr, ptr+bytes) (device
   pointer, 16-byte aligned, at least one full page) with a shared-memory
   bulk-copy mapping whose producer deliberately never issues one chunk, so
   the consumers' wait for it runs out after limit_ns (clamped to 1 ms..10 s).
   *timed_out receives 1 if the kernel reported the timeout and finished.
   The device stays usable afterwards.  Synchronous.  Errors: EINVAL, ECUDA. */
crum_status crum_selftest_wait_timeout(const void *ptr, uint64_t bytes, uint64_t limit_ns,
                                       int *timed_out, crum_stream_t stream);

/* ---- serving: checkpoint/restore requests from many clients ----
   The paper checkpoints each MPI rank's process (Sections 3.3-3.4); here a
   server takes checkpoint and restore requests from many clients as they
   arrive and keeps several on the device at once ("continuous batching"):
   a request is admitted when a slot is free and the staging it needs fits
   the remaining staging budget, so requests that arrive while others run
   join as soon as memory frees up.  Each client is a crum_set created with
   external_staging = 1 (its hash table and page tables stay resident on the
   device between requests) plus the stream its application runs on.  One
   request per client is on the device at a time; a client's requests run
   in arrival order.  A client must not enqueue further work that writes
   its registered memory on its stream until its checkpoint request has
   reached CRUM_WAIT_CAPTURED (the consistency point is the capture). */

typedef struct crum_server crum_server;

typedef struct crum_server_config {
    int device;
    uint64_t staging_budget;  /* device bytes lent to admitted requests; 0: 16 GiB */
    int max_inflight;         /* requests on the device at once; 0: 8 */
    int max_checkpoints;      /* of those, checkpoint requests at once; 0: 2 with
                                 serialized drains, else 1; negative: no separate limit */
    int max_restores;         /* of those, restore requests at once (host->device link);
                                 0: 1; negative: no separate limit.  One of each, in
                                 arrival order, keeps large requests from being slowed by
                                 later arrivals while the two link directions and the
                                 device overlap */
    int serialize_drains;     /* 0 (default) or 1: the clients' checkpoint drains cross
                                 the link one at a time, in admission order, while their
                                 captures overlap, so max_checkpoints > 1 keeps the link
                                 busy without sharing it; negative: each drain starts as
                                 soon as its capture is done */
    int order;                /* admission order among admissible requests: 0 (default)
                                 arrival order; 1 the request whose client footprint
                                 would cross the link fastest, less the time it has
                                 waited, first (a client's own requests stay in
                                 arrival order) */
    int keep_images;          /* 1: a completed checkpoint request keeps a reference
                                 to its image until crum_server_take_image hands it
                                 out (or the server is destroyed or its statistics
                                 reset), so a caller can read every request's image;
                                 0 (default): the server drops it at completion */
} crum_server_config;

#define CRUM_REQ_CHECKPOINT 0      /* incremental checkpoint of the client's set */
#define CRUM_REQ_CHECKPOINT_FULL 1 /* full checkpoint (starts a new chain) */
#define CRUM_REQ_RESTORE 2         /* restore the client's newest persisted image chain */

typedef struct crum_request_info {
    uint64_t id;
    uint32_t client;
    int kind;
    int status;               /* crum_status; CRUM_ETIMEOUT while still running */
    int done;                 /* 1 once complete */
    uint64_t n_dirty;         /* checkpoint: pages in the image; restore: pages written */
    uint64_t bytes;           /* image bytes drained (checkpoint) or restored payload */
    uint64_t image_seq;       /* checkpoint: seq of the new image; restore: chain end seq */
    uint64_t checksum;        /* checkpoint: the new image's trailer checksum */
    double t_queue_ms;        /* submit -> admitted */
    double t_total_ms;        /* submit -> complete (checkpoint: persisted) */
} crum_request_info;

typedef struct crum_server_stats {
    uint64_t submitted, completed, failed;
    uint64_t bytes_checkpointed;  /* footprint bytes of completed checkpoint requests */
    uint64_t bytes_restored;
    double p50_ms, p99_ms;        /* submit -> complete over completed requests */
    double p50_ckpt_ms, p99_ckpt_ms, p50_restore_ms, p99_restore_ms;
    double wall_ms;               /* first submit -> last completion */
    uint32_t peak_inflight;
    uint64_t peak_staging;        /* most staging bytes lent at once */
} crum_server_stats;

/* Create a server (allocates the staging budget on the device and starts its
   admission thread).  Errors: EINVAL, ENOMEM, ECUDA. */
crum_status crum_server_create(const crum_server_config *cfg, crum_server **out);

/* Wait for every submitted request, stop the thread, free the staging. */
crum_status crum_server_destroy(crum_server *srv);

/* Add a client: a set made with external_staging = 1 and registered
   allocations, and the stream its application uses.  The server does not
   own the set.  Errors: EINVAL (set without external staging, or larger
   than the whole budget). */
crum_status crum_server_add_client(crum_server *srv, crum_set *set, crum_stream_t app_stream,
                                   uint32_t *client_id);

/* Queue a request (CRUM_REQ_*); returns at once with its id. */
crum_status crum_server_submit(crum_server *srv, uint32_t client, int kind, uint64_t *request_id);

/* Wait until a request completes (timeout_ns < 0: no limit) and fill *info.
   CRUM_WAIT_CAPTURED-like early return: stage = 1 waits only until a
   checkpoint request's pages are captured.  Returns the request's status,
   or ETIMEOUT. */
crum_status crum_server_wait(crum_server *srv, uint64_t request_id, int stage, int64_t timeout_ns,
                             crum_request_info *info);

/* The image of a completed checkpoint request of a server created with
   keep_images = 1: *out receives the server's reference to it (the caller
   releases it with crum_image_release); a second call for the same request
   is EINVAL.  Errors: EINVAL (unknown, unfinished, failed or restore
   request, image already taken, or keep_images off). */
crum_status crum_server_take_image(crum_server *srv, uint64_t request_id, crum_image **out);

/* Wait for every submitted request, then fill *stats (latencies over all
   completed requests since create or the last reset). */
crum_status crum_server_drain(crum_server *srv, crum_server_stats *stats);

/* Forget completed requests and their latencies (for a fresh measurement). */
crum_status crum_server_reset_stats(crum_server *srv);

/* ---- allocation-free dirty-page detection (the paper has no counterpart;
        this exists for callers that cannot allocate device memory) ---- */

#define CRUM_STATIC_MAX_PAGES 4194304u /* 256 GiB of 64 KiB pages */

/* Which pages of one allocation changed, without allocating any memory.
   For callers that cannot call cudaMalloc when they need the answer: an
   out-of-memory handler that wants a last checkpoint before freeing
   anything (where cudaMalloc is what fails), or an allocator hook or
   CUDA-call interposer in which a nested cudaMalloc would re-enter the
   allocator being served.
   ptr/bytes: the allocation (16-byte aligned device pointer, bytes > 0,
   at most CRUM_STATIC_MAX_PAGES pages, else EINVAL).  hashes: device array
   of ceil(bytes/65536) u64 holding the previous page hashes; overwritten
   with the current ones.  full != 0 lists every page.  pages_out: device
   array with room for ceil(bytes/65536) u32; receives the changed page
   indices in ascending order.  count_out: device u64, receives their number.
   Stream ordered on `stream`; returns once the work is queued.
   Scratch: a 512 KiB dirty bitmap in a fixed device array inside the
   library, which every GPU that loads the library keeps until exit.  The
   first call on a device looks up that array's address with the device
   current; make that first call before any stream capture and before
   memory runs short.  All calls on a device share the bitmap, so calls
   that overlap on the GPU (unordered streams) race; each call clears what
   it uses first.  Errors: EINVAL, ECUDA. */
crum_status crum_dirty_pages_static(const void *ptr, uint64_t bytes, uint64_t *hashes, int full,
                                    uint32_t *pages_out, uint64_t *count_out,
                                    crum_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* CRUM_H */
