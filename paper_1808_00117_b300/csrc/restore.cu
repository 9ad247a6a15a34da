// Restore kernels and their launchers (Section 3.4's restart: image slots
// back onto the registered allocations, committed hashes reinstalled).
//
//   k_restore         inverse scatter of one image's slots (replay)
//   k_bpd_restore     the same for a compressed image: each slot decoded in
//                     shared memory first
//   k_chain_owner     newest (image, slot) of every page over a restore chain
//   k_restore_merged  every page once from that image, read from the
//                     image's pinned host memory (optionally only pages whose
//                     current hash differs: delta restore)
//   k_restore_merged_bpd  the merged restore of chains with compressed images
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "codec.cuh"
#include "device.cuh"
#include "kernels.h"
#include "restore_codec.h"
#include "launch.cuh"

namespace crum {
namespace {

using dev::ld_stream;

// --------------------------------------------------------------- restore ---

template <int G>
__global__ void __launch_bounds__(256) k_restore(RestoreArgs a) {
  constexpr int kGroupsPerCta = (G == 32) ? 256 / 32 : 1;
  const int t = threadIdx.x % G;
  const uint64_t group = static_cast<uint64_t>(blockIdx.x) * kGroupsPerCta + threadIdx.x / G;
  const uint64_t n_groups = static_cast<uint64_t>(gridDim.x) * kGroupsPerCta;
  for (uint64_t s = group; s < a.n_slots; s += n_groups) {
    const uint32_t k = a.ptab[2 * s];
    const uint64_t p = a.ptab[2 * s + 1];
    if (k >= a.n_allocs || p >= a.allocs[k].n_pages) continue;  // rejected on the host already
    uint8_t* dst = a.allocs[k].base + p * kPage;
    const uint32_t valid = dev::valid_bytes(a.allocs[k].bytes, p);
    const uint8_t* src = a.payload + s * kPage;
    const uint32_t nvec = valid >> 4;
    for (uint32_t v = t; v < nvec; v += G)
      *reinterpret_cast<uint4*>(dst + 16ull * v) = ld_stream(src + 16ull * v);
    const uint32_t rem = valid & 15u;
    if (rem != 0 && t == 0)
      for (uint32_t b = 0; b < rem; ++b) dst[16ull * nvec + b] = src[16ull * nvec + b];
    if (t == 0) a.h_table[a.allocs[k].first_page + p] = a.hashes[s];
  }
}

__global__ void __launch_bounds__(kBpdThreads) k_bpd_restore(BpdRestoreArgs a) {
  extern __shared__ __align__(16) uint8_t dyn[];
  uint8_t* page = dyn;
  uint8_t* plane = dyn + kPage;
  __shared__ uint8_t dict[8][128];
  __shared__ BpdSmem m;
  for (uint64_t s = blockIdx.x; s < a.n_slots; s += gridDim.x) {
    const uint32_t k = a.ptab[2 * s];
    const uint64_t p = a.ptab[2 * s + 1];
    if (k >= a.n_allocs || p >= a.allocs[k].n_pages) continue;  // rejected on the host already
    const uint64_t lo = a.offs[s], hi = s + 1 < a.n_slots ? a.offs[s + 1] : a.enc_end;
    if (!bpd_decode(a.enc + (lo - a.offs[0]), static_cast<uint32_t>(hi - lo), page, plane, dict, m)) {
      if (threadIdx.x == 0 && a.error) atomicExch(a.error, 1u);
      __syncthreads();
      continue;
    }
    bpd_store(page, a.allocs[k].base + p * kPage, dev::valid_bytes(a.allocs[k].bytes, p));
    if (threadIdx.x == 0) a.h_table[a.allocs[k].first_page + p] = a.hashes[s];
    __syncthreads();
  }
}

// ----------------------------------------------- merged (last-writer) restore ---
//
// A chain base..end restored page by page from the newest image that holds
// each page, so every page crosses the link once however long the chain.
// The images stay in pinned host memory; both kernels read them there.

constexpr uint64_t kSlotMask = (1ull << 40) - 1;

__global__ void __launch_bounds__(256) k_chain_owner(OwnerArgs a) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  for (uint64_t j = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
       j < a.total_slots; j += stride) {
    uint32_t lo = 0, hi = a.n_images;  // image holding global slot j, in [lo, hi)
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (a.images[mid].slot0 <= j)
        lo = mid;
      else
        hi = mid;
    }
    const uint64_t s = j - a.images[lo].slot0;
    const uint2 e = *reinterpret_cast<const uint2*>(a.images[lo].ptab + 8 * s);
    if (e.x >= a.n_allocs || e.y >= a.allocs[e.x].n_pages) continue;  // rejected on the host already
    const uint64_t g = a.allocs[e.x].first_page + e.y;
    // later images carry larger tags, so the maximum is the last writer
    atomicMax(reinterpret_cast<unsigned long long*>(a.owner + g),
              static_cast<unsigned long long>((static_cast<uint64_t>(lo) + 1) << 40 | s));
  }
}

// An image's payload starts 64 + 16A + 16n bytes into it: 16-byte aligned,
// rarely 128-byte aligned.  Read across the link, a warp's 512 contiguous
// bytes would then span five 128-byte lines instead of four; so each CTA
// reads whole aligned lines of a 16 KiB stretch into shared memory and
// writes the page from there, shifted by the misalignment (a whole number
// of 16-byte vectors).
constexpr uint32_t kMergeChunkVecs = 1024;  // 16 KiB per step

// One page from an image payload slot in host memory to the allocation,
// whole 128-byte lines at a time through `buf` (kMergeChunkVecs + 8 vectors).
__device__ __forceinline__ void merged_copy_page(const uint8_t* src, uint8_t* dst, uint32_t valid,
                                                 uint4* buf) {
  const uint32_t nvec = valid >> 4;
  const uintptr_t sa = reinterpret_cast<uintptr_t>(src);
  const uint4* line = reinterpret_cast<const uint4*>(sa & ~uintptr_t(127));
  const uint32_t m = static_cast<uint32_t>(sa & 127u) >> 4;
  for (uint32_t c = 0; c < nvec; c += kMergeChunkVecs) {
    const uint32_t cnt = min(kMergeChunkVecs, nvec - c);
    // vectors line[c .. c+cnt+m) end at the last whole vector of the page
    for (uint32_t i = threadIdx.x; i < cnt + m; i += blockDim.x) buf[i] = line[c + i];
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x)
      reinterpret_cast<uint4*>(dst)[c + i] = buf[i + m];
    __syncthreads();
  }
  const uint32_t rem = valid & 15u;
  if (rem != 0 && threadIdx.x == 0)
    for (uint32_t b = 0; b < rem; ++b) dst[16ull * nvec + b] = src[16ull * nvec + b];
}

// Installs the chain's hash of page g and decides, CTA-uniformly, whether
// the page is copied (delta mode leaves a page whose current contents
// already hash to the chain's value).
__device__ __forceinline__ bool merged_take_page(const MergedRestoreArgs& a, const ChainImage& im,
                                                 uint64_t g, uint64_t s, int* flag) {
  if (threadIdx.x == 0) {
    const uint64_t hc = reinterpret_cast<const uint64_t*>(im.hashes)[s];
    a.h_table[g] = hc;
    const bool skip = a.current != nullptr && a.current[g] == hc;
    if (!skip && a.copied != nullptr) atomicAdd(a.copied, 1ull);
    *flag = skip;
  }
  __syncthreads();
  const bool skip = *flag;
  __syncthreads();  // every thread has read the flag before it is rewritten
  return !skip;
}

__global__ void __launch_bounds__(256) k_restore_merged(MergedRestoreArgs a) {
  __shared__ uint4 buf[kMergeChunkVecs + 8];
  __shared__ int skip_sh;
  for (uint64_t g = blockIdx.x; g < a.n_pages; g += gridDim.x) {
    const uint64_t o = a.owner[g];
    if (o == 0) continue;  // no image of the chain holds this page
    const ChainImage& im = a.images[(o >> 40) - 1];
    const uint64_t s = o & kSlotMask;
    if (!merged_take_page(a, im, g, s, &skip_sh)) continue;
    const uint32_t k = dev::find_alloc(a.first_page, a.n_allocs, g);
    const uint64_t p = g - a.allocs[k].first_page;
    merged_copy_page(im.payload + s * kPage, a.allocs[k].base + p * kPage,
                     dev::valid_bytes(a.allocs[k].bytes, p), buf);
  }
}

// The merged restore of a chain holding compressed images: a compressed
// slot is decoded from host memory in shared memory, then stored.
__global__ void __launch_bounds__(kBpdThreads) k_restore_merged_bpd(MergedRestoreArgs a) {
  extern __shared__ __align__(16) uint8_t dyn[];
  uint8_t* page = dyn;
  uint8_t* plane = dyn + kPage;
  __shared__ uint8_t dict[8][128];
  __shared__ BpdSmem m;
  __shared__ int skip_sh;
  for (uint64_t g = blockIdx.x; g < a.n_pages; g += gridDim.x) {
    const uint64_t o = a.owner[g];
    if (o == 0) continue;
    const ChainImage& im = a.images[(o >> 40) - 1];
    const uint64_t s = o & kSlotMask;
    if (!merged_take_page(a, im, g, s, &skip_sh)) continue;
    const uint32_t k = dev::find_alloc(a.first_page, a.n_allocs, g);
    const uint64_t p = g - a.allocs[k].first_page;
    uint8_t* dst = a.allocs[k].base + p * kPage;
    const uint32_t valid = dev::valid_bytes(a.allocs[k].bytes, p);
    if (im.offs == nullptr) {
      merged_copy_page(im.payload + s * kPage, dst, valid, reinterpret_cast<uint4*>(page));
      continue;
    }
    const uint64_t lo = im.offs[s], hi = s + 1 < im.n_slots ? im.offs[s + 1] : im.payload_bytes;
    if (!bpd_decode(im.payload + lo, static_cast<uint32_t>(hi - lo), page, plane, dict, m)) {
      if (threadIdx.x == 0 && a.error) atomicExch(a.error, 1u);
      __syncthreads();
      continue;
    }
    bpd_store(page, dst, valid);
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_restore(const RestoreArgs& a, cudaStream_t st) {
  if (a.n_slots == 0) return cudaSuccess;
  // one CTA per image slot: restores carry few slots per launch, and a
  // warp per slot left most of the device idle
  auto kern = k_restore<256>;
  const unsigned grid = grid_for(kern, a.n_slots, 1);
  kern<<<grid, 256, 0, st>>>(a);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_chain_owner(const OwnerArgs& a, cudaStream_t st) {
  if (a.total_slots == 0 || a.n_images == 0) return cudaSuccess;
  const uint64_t cap = static_cast<uint64_t>(resident_ctas(k_chain_owner, 256));
  const unsigned grid =
      static_cast<unsigned>(std::max<uint64_t>(1, std::min((a.total_slots + 255) / 256, cap)));
  k_chain_owner<<<grid, 256, 0, st>>>(a);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_restore_merged(const MergedRestoreArgs& a, bool compressed, cudaStream_t st) {
  if (a.n_pages == 0) return cudaSuccess;
  if (compressed) {
    cudaError_t e = allow_big_smem(k_restore_merged_bpd);
    if (e != cudaSuccess) return e;
    k_restore_merged_bpd<<<bpd_grid(k_restore_merged_bpd, a.n_pages), kBpdThreads, kBpdDynSmem, st>>>(a);
    g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
  }
  // one CTA per page; any shape that keeps a few MB of reads in flight
  // saturates the link
  const unsigned grid = grid_for(k_restore_merged, a.n_pages, 1);
  k_restore_merged<<<grid, 256, 0, st>>>(a);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

cudaError_t launch_bpd_restore(const BpdRestoreArgs& a, cudaStream_t st) {
  if (a.n_slots == 0) return cudaSuccess;
  cudaError_t e = allow_big_smem(k_bpd_restore);
  if (e != cudaSuccess) return e;
  k_bpd_restore<<<bpd_grid(k_bpd_restore, a.n_slots), kBpdThreads, kBpdDynSmem, st>>>(a);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace crum
