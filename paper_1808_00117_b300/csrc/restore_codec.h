// Launch interface of the restore kernels (restore.cu) and of the
// compression kernels (codec.cu), internal to the library.  The capture
// kernels' interface, and KernelSpec, are in kernels.h.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "device.cuh"
#include "kernels.h"

namespace crum {

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
  uint8_t* alph;             // out: every slot's alphabets (kBpdAlphBytes a slot)
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
  const uint8_t* alph;       // the size kernel's alphabets of these slots
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

cudaError_t launch_restore(const RestoreArgs& a, cudaStream_t st);
cudaError_t launch_chain_owner(const OwnerArgs& a, cudaStream_t st);
cudaError_t launch_bpd_size(const BpdSizeArgs& a, uint64_t max_slots, cudaStream_t st);
cudaError_t launch_bpd_scan(const BpdScanArgs& a, cudaStream_t st);
cudaError_t launch_bpd_encode(const BpdEncodeArgs& a, uint64_t max_slots, cudaStream_t st);
cudaError_t launch_bpd_restore(const BpdRestoreArgs& a, cudaStream_t st);
cudaError_t launch_restore_merged(const MergedRestoreArgs& a, bool compressed, cudaStream_t st);

}  // namespace crum
