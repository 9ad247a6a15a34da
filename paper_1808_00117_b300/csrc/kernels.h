// Launch interface of the capture kernels (internal to the library); the
// restore and compression kernels' is in restore_codec.h.
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
cudaError_t launch_hash_bytes(const uint8_t* p, uint64_t n, uint64_t first_index, uint64_t* out,
                              cudaStream_t st);

}  // namespace crum
