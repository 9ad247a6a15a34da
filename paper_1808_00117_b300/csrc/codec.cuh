// Byte-plane dictionary code: shared-memory layout, launch shape and the
// decoder, used by the encoding kernels and by the restore kernels
// (internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "device.cuh"
#include "launch.cuh"

namespace crum {

// ------------------------------------------- byte-plane dictionary code ---
//
// Optional compression of the drained payload.  A slot (64 KiB: the page's
// valid bytes, then zeros) is split into 8 byte planes of 8,192 bytes
// (plane j = bytes 8i + j).  A plane with k distinct values and
// b = ceil(log2 k) < 8 is stored as its values in ascending order (padded
// to 16 bytes) and 1,024 b bytes holding each byte's position among them, b
// bits each, LSB first; a plane with b = 8 is stored as is.  A 16-byte head
// (b of each plane, then k - 1, 255 for a stored plane) leads; a slot whose
// code would not be shorter than 64 KiB is stored as is.  One CTA of 256
// threads handles one slot; group q of 32 consecutive plane bytes belongs
// to thread q, so its b bits x 32 are exactly b words of the packed stream.

constexpr uint32_t kPlaneBytes = kPage / 8;
constexpr int kBpdThreads = 256;

struct BpdSmem {
  uint8_t present[8][256];
  uint8_t rank[8][256];
  uint32_t k[8];
  uint32_t b[8];
  uint32_t sec[9];  // section offsets in the encoded slot; sec[8] = code length
  uint32_t len;     // encoded length (kPage: stored as is)
  int skip;
  uint32_t open;    // planes whose sample alphabet left b < 8 possible (bit j)
};

// A plane holding 129 or more distinct byte values has b = 8 and is stored
// as is, whatever its other bytes are: an alphabet only grows as bytes are
// added.  The capture kernels therefore mark a sample of every plane first
// (1,024 of its 8,192 bytes), and only the planes whose sample alphabet is
// still at most 128 values are marked in full and ranked.
constexpr uint32_t kBpdRawAlphabet = 129;

// The alphabets the size kernel found, handed to the encoder: bit v % 8 of
// byte 32 j + v / 8 is plane j's presence of value v (256 bytes a slot).
constexpr uint32_t kBpdAlphBytes = 8 * 256 / 8;

// Where value x sits in a plane's 256-byte presence and rank tables: bit 4
// is flipped for x >= 128, so x and x + 128 (the same bank otherwise) fall
// into banks 4 apart.  Float sign-and-exponent planes hold exactly such
// pairs (the same exponent with either sign).
__device__ __forceinline__ uint32_t tslot(uint32_t x) { return x ^ ((x >> 7) << 4); }
// tslot of each byte of a word, four at a time.
__device__ __forceinline__ uint32_t tslot4(uint32_t w) { return w ^ (((w >> 7) & 0x01010101u) << 4); }

__device__ __forceinline__ uint32_t ceil_log2(uint32_t k) {
  uint32_t b = 0;
  while ((1u << b) < k) ++b;
  return b;
}


// Decodes the `len` encoded bytes at `enc` (device or mapped host memory)
// into `page` (shared, 64 KiB) using `plane` (shared, 8 KiB) and `dict`
// (shared, 8 x 128).  Returns false, CTA-uniformly, for a code the encoder
// cannot have written (the slot is then skipped).
__device__ inline bool bpd_decode(const uint8_t* enc, uint32_t len, uint8_t* page, uint8_t* plane,
                           uint8_t (*dict)[128], BpdSmem& m) {
  const int tid = threadIdx.x;
  if (len == kPage) {
    for (uint32_t v = tid; v < kPageVecs; v += blockDim.x)
      reinterpret_cast<uint4*>(page)[v] = reinterpret_cast<const uint4*>(enc)[v];
    __syncthreads();
    return true;
  }
  if (tid == 0) {
    int ok = len >= 16 && len % 16 == 0 && len < kPage;
    uint32_t pos = 16;
    for (int j = 0; ok && j < 8; ++j) {
      const uint32_t b = enc[j], km1 = enc[8 + j];
      m.b[j] = b;
      m.k[j] = km1 + 1;
      m.sec[j] = pos;
      if (b == 8) {
        ok = km1 == 255;
        pos += kPlaneBytes;
      } else {
        ok = b < 8 && km1 < 128 && ceil_log2(km1 + 1) == b;
        pos += ((km1 + 1 + 15) & ~15u) + 1024u * b;
      }
    }
    m.skip = !(ok && pos == len);
  }
  __syncthreads();
  if (m.skip) return false;
  for (int j = 0; j < 8; ++j) {
    const uint32_t b = m.b[j];
    const uint8_t* sec = enc + m.sec[j];
    if (b == 8) {
      for (uint32_t v = tid; v < kPlaneBytes / 16; v += blockDim.x)
        reinterpret_cast<uint4*>(plane)[v] = reinterpret_cast<const uint4*>(sec)[v];
    } else {
      const uint32_t k = m.k[j], dpad = (k + 15u) & ~15u;
      if (tid < 128) dict[j][tid] = tid < k ? sec[tid] : 0;
      __syncthreads();
      uint32_t outw[8];
      if (b == 0) {
        const uint32_t x = dict[j][0] * 0x01010101u;
#pragma unroll
        for (int q = 0; q < 8; ++q) outw[q] = x;
      } else {
        const uint32_t* words = reinterpret_cast<const uint32_t*>(sec + dpad) + tid * b;
        uint64_t acc = 0;
        uint32_t nb = 0, e = 0;
        const uint32_t mask = (1u << b) - 1u;
#pragma unroll
        for (int q = 0; q < 8; ++q) outw[q] = 0;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          if (nb < b) {
            acc |= static_cast<uint64_t>(words[e++]) << nb;
            nb += 32;
          }
          const uint32_t r = static_cast<uint32_t>(acc) & mask;
          acc >>= b;
          nb -= b;
          outw[q >> 2] |= static_cast<uint32_t>(dict[j][r & 127u]) << (8 * (q & 3));
        }
      }
      reinterpret_cast<uint4*>(plane)[2 * tid] = make_uint4(outw[0], outw[1], outw[2], outw[3]);
      reinterpret_cast<uint4*>(plane)[2 * tid + 1] = make_uint4(outw[4], outw[5], outw[6], outw[7]);
    }
    __syncthreads();
    for (uint32_t i = tid; i < kPlaneBytes; i += blockDim.x) page[8 * i + j] = plane[i];
    __syncthreads();
  }
  return true;
}

// Valid bytes of the decoded page to the allocation (CTA-wide).
__device__ __forceinline__ void bpd_store(const uint8_t* page, uint8_t* dst, uint32_t valid) {
  const uint32_t nvec = valid >> 4;
  for (uint32_t v = threadIdx.x; v < nvec; v += blockDim.x)
    reinterpret_cast<uint4*>(dst)[v] = reinterpret_cast<const uint4*>(page)[v];
  const uint32_t rem = valid & 15u;
  if (rem != 0 && threadIdx.x == 0)
    for (uint32_t b = 0; b < rem; ++b) dst[16ull * nvec + b] = page[16ull * nvec + b];
}

constexpr size_t kBpdDynSmem = kPage + kPlaneBytes;  // the slot + one plane

// Kernels that use more than 48 KiB of dynamic shared memory must say so
// once per device.
template <typename K>
cudaError_t allow_big_smem(K kern, size_t bytes = kBpdDynSmem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, bool> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_pair(reinterpret_cast<const void*>(kern), dev);
  if (done.count(key)) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e == cudaSuccess) done[key] = true;
  return e;
}

// The encoder stages its slot in shared memory: 4,096 chunks of 16 bytes,
// chunk c of 256-byte group g stored at position 16 g + (c ^ (g & 7)).  A
// warp's coalesced loads (two groups per instruction) and a thread's reads
// of its own group (one chunk per instruction, 32 groups) then each touch
// every bank group of shared memory exactly four times: no conflicts.
constexpr size_t kEncDynSmem = kPage;
__device__ __forceinline__ uint32_t enc_chunk_pos(uint32_t g, uint32_t c) { return 16u * g + (c ^ (g & 7u)); }

template <typename K>
unsigned bpd_grid(K kern, uint64_t units) {
  const uint64_t cap =
      static_cast<uint64_t>(resident_per_sm(reinterpret_cast<const void*>(kern), kBpdThreads, kBpdDynSmem)) *
      num_sms();
  return static_cast<unsigned>(std::max<uint64_t>(1, std::min(units, cap)));
}

// Launch shapes of the compression kernels (the launchers in kernels.h use
// them; the capture graph adds them as nodes).
KernelSpec bpd_size_spec(uint64_t max_slots);
KernelSpec bpd_scan_spec();
cudaError_t bpd_encode_spec(uint64_t max_slots, KernelSpec* out);

}  // namespace crum
