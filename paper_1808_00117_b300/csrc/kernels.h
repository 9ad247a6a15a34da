// Launch interface of the capture/restore kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "device.cuh"

namespace crum {

extern std::atomic<uint64_t> g_kernel_launches;

// Thread mapping of the page kernels.  Register mappings: G threads per page
// (32: one warp per page, several pages per CTA; 256: one CTA per page) and
// U 16-byte loads in flight per thread.  Bulk-copy mappings (hash only):
// one producer thread streams 16 KiB quarter-pages into a ring of `stages`
// shared-memory buffers with cp.async.bulk, `group` consumer threads hash
// them.  Chosen per set by the autotuner.
struct Mapping {
  int group;
  int unroll;
  int stages;  // 0: register mapping
};
extern const Mapping kMappings[];
extern const int kNumMappings;

struct HashArgs {
  const DevAlloc* allocs;      // device table, or nullptr to use `one`
  const uint64_t* first_page;  // device, n_allocs entries (first page of each)
  DevAlloc one;                // single allocation (allocs == nullptr)
  uint32_t n_allocs;
  uint64_t n_pages;
  uint64_t* h_table;      // committed hashes: read as previous, overwritten with new
  uint64_t* h_out;        // if set: write hashes here and skip the dirty logic
  uint32_t* dirty_mask;   // bit g%32 of word g/32 set for dirty page g (pre-zeroed)
  int full;               // every page dirty
  const uint8_t* shadow;  // verify mode: last checkpointed bytes, page g at g*64 KiB
  unsigned long long* collisions;
  unsigned int* error;    // bulk-copy mappings: set to 1 if a bounded wait ran out (optional)
  uint64_t wait_limit_ns;     // bulk-copy mappings: bound of each wait (0: 2 s)
  uint32_t test_skip_chunk;   // self-test only: CTA 0 never issues chunk n-1 (0: off)
};

struct ScanArgs {
  const uint32_t* mask;
  uint64_t n_words;          // ceil(n_pages / 32)
  uint32_t* word_offset;     // n_words + 1: dirty pages before each word; last = total
  uint64_t* n_dirty_out;     // device
  volatile uint64_t* mailbox;  // mapped pinned host: [0] dirty count, [1] collisions,
                               // [2] hash timeout flag (optional)
  const unsigned long long* collisions;  // verify-mode collision counter (optional)
  const unsigned int* error;             // hash-kernel wait-timeout flag (optional)
  const DevAlloc* allocs;
  uint32_t n_allocs;
  uint8_t* meta;             // header + allocation table + page table + hashes
  uint64_t* trailer;         // set to the checksum of header + allocation table
  uint64_t seq, parent_seq;
  uint32_t flags;
};

struct GatherArgs {
  const DevAlloc* allocs;
  const uint64_t* first_page;
  uint32_t n_allocs;
  const uint32_t* mask;
  const uint32_t* word_offset;
  uint64_t n_words;
  uint64_t n_pages;
  const uint64_t* n_dirty;   // device
  const uint64_t* h_table;
  uint8_t* meta;
  uint8_t* payload;          // slot s goes to payload + (s - s_begin) * 64 KiB
  uint64_t* trailer;         // checksum accumulator
  uint64_t s_begin, s_end;   // slot range of this launch (clipped to n_dirty)
  uint8_t* shadow;           // verify mode: copy of each gathered page
};

struct RestoreArgs {
  const DevAlloc* allocs;
  uint32_t n_allocs;
  const uint32_t* ptab;      // 2 u32 per slot: allocation index, page index
  const uint64_t* hashes;    // per slot
  const uint8_t* payload;    // slot s at payload + s * 64 KiB
  uint64_t n_slots;
  uint64_t* h_table;
};

// One image of a restore chain as the device sees it: pointers into the
// image's pinned host buffer (mapped, read by the kernels across the link).
struct ChainImage {
  const uint8_t* ptab;     // 2 u32 per slot: allocation index, page index
  const uint8_t* hashes;   // u64 per slot
  const uint8_t* payload;  // slot s at payload + s * 64 KiB (or encoded, see offs)
  uint64_t slot0;          // slots of the images before this one
  const uint64_t* offs;    // compressed image: slot offsets in the payload, else nullptr
  uint64_t payload_bytes;  // compressed image: encoded payload bytes
  uint64_t n_slots;
};

// owner[g] = (image + 1) << 40 | slot of the newest chain image holding
// page g; 0 if no image holds it (pre-zeroed).
struct OwnerArgs {
  const DevAlloc* allocs;
  uint32_t n_allocs;
  const ChainImage* images;  // device, base first
  uint32_t n_images;
  uint64_t total_slots;
  uint64_t* owner;
};

struct MergedRestoreArgs {
  const DevAlloc* allocs;
  const uint64_t* first_page;
  uint32_t n_allocs;
  uint64_t n_pages;
  const ChainImage* images;
  const uint64_t* owner;
  uint64_t* h_table;
  const uint64_t* current;          // delta mode: current hash of every page, else nullptr
  unsigned long long* copied;       // pages copied across the link (optional)
  unsigned int* error;              // set when a compressed slot does not decode (optional)
};

// Compressed images (byte-plane dictionary code of each payload slot; the
// format is stated with crum_config.compress in crum.h).
struct BpdSizeArgs {
  const uint8_t* payload;    // raw slots, slot s at payload + s * 64 KiB
  const uint64_t* n_dirty;   // device
  uint32_t* enc_len;         // out: encoded length of every slot
};

// Offsets of `n` encoded slots (base + exclusive prefix of their lengths)
// into offs[0, n).  With offs null the slots are a whole image's (base 0):
// the table is the image's own (64 + 16 A + 16 n into meta), and the header
// words of the compressed form and the padding after the tables are
// written too.
struct BpdScanArgs {
  const uint32_t* enc_len;
  const uint64_t* n;         // device: slots
  uint64_t* offs;            // or null, see above
  uint64_t base;
  uint64_t* total_out;       // device: encoded bytes of these slots
  volatile uint64_t* mailbox;  // [3] = the same (optional)
  uint8_t* meta;
  uint32_t n_allocs;
};

// Encodes slot s of `payload` to out + offs[s] - base, s < n, and adds
// the code's terms of the image checksum to *trailer (offs null: the whole
// image, with the image's own table in meta as for BpdScanArgs, the payload
// offset found from n, and the header and tables' terms added too).
struct BpdEncodeArgs {
  const uint8_t* payload;    // raw slots
  const uint64_t* n;         // device: slots
  const uint64_t* offs;
  uint64_t base;
  uint8_t* out;              // encoded bytes
  const uint8_t* meta;
  uint32_t n_allocs;
  uint64_t poff;             // image byte offset of the encoded payload (offs non-null)
  unsigned long long* trailer;  // zeroed before the image's first launch
};

// Replay restore of a compressed image's slots [0, n_slots): slot s is
// encoded at enc + offs[s] - offs[0] with length offs[s + 1] - offs[s]
// (the last one ends at enc_end).
struct BpdRestoreArgs {
  const DevAlloc* allocs;
  uint32_t n_allocs;
  const uint32_t* ptab;
  const uint64_t* hashes;
  const uint64_t* offs;
  const uint8_t* enc;
  uint64_t enc_end;          // offset, in the image's payload, where the last slot ends
  uint64_t n_slots;
  uint64_t* h_table;
  unsigned int* error;       // set when a slot does not decode (skipped)
};

// Launch shape of one kernel: launched directly (launch_spec) or added to a
// CUDA graph as a kernel node whose single parameter is the args struct.
struct KernelSpec {
  const void* func;
  unsigned grid;
  unsigned block;
  size_t smem;
};
cudaError_t hash_spec(uint64_t n_pages, int mapping, bool verify, KernelSpec* out);
cudaError_t scan_spec(KernelSpec* out);
cudaError_t gather_spec(uint64_t max_slots, int mapping, bool verify, KernelSpec* out);
cudaError_t launch_spec(const KernelSpec& s, void* arg, cudaStream_t st);

cudaError_t launch_hash_dirty(const HashArgs& a, int mapping, bool verify, cudaStream_t st);
cudaError_t launch_scan(const ScanArgs& a, cudaStream_t st);
cudaError_t launch_gather(const GatherArgs& a, uint64_t max_slots, int mapping, bool verify,
                          cudaStream_t st);
cudaError_t launch_restore(const RestoreArgs& a, cudaStream_t st);
cudaError_t launch_chain_owner(const OwnerArgs& a, cudaStream_t st);
cudaError_t launch_bpd_size(const BpdSizeArgs& a, uint64_t max_slots, cudaStream_t st);
cudaError_t launch_bpd_scan(const BpdScanArgs& a, cudaStream_t st);
cudaError_t launch_bpd_encode(const BpdEncodeArgs& a, uint64_t max_slots, cudaStream_t st);
cudaError_t launch_bpd_restore(const BpdRestoreArgs& a, cudaStream_t st);
cudaError_t launch_restore_merged(const MergedRestoreArgs& a, bool compressed, cudaStream_t st);
cudaError_t launch_hash_bytes(const uint8_t* p, uint64_t n, uint64_t first_index, uint64_t* out,
                              cudaStream_t st);

}  // namespace crum
