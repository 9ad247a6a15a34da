// Capture kernels and their host-side launchers.
//
//   k_hash_dirty  hash every page of the flattened work-list, compare with
//                 the committed hash, commit the new one, set dirty bits
//                 (the dirty test standing in for Algorithm 1's write faults)
//   k_scan        one CTA: prefix sum of the dirty bitmap (ballot-free, since
//                 the bitmap already packs 32 pages a word) -> slot of every
//                 dirty page, dirty count, image header and allocation table
//   k_gather      one group per dirty slot: page table entry, hash entry and
//                 the page's bytes into staging ("drain the device", Sections
//                 3.3-3.4), plus the image checksum of everything it writes
//   k_hash_bytes  the hash over an arbitrary byte string (image checksum)
//   k_hash_dirty_bulk  k_hash_dirty with pages staged into shared memory by
//                 cp.async.bulk (warp-specialised; bounded mbarrier waits)
// The compression kernels are in codec.cu, the restore kernels in restore.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>

#include "crum.h"
#include "device.cuh"
#include "kernels.h"
#include "launch.cuh"

namespace crum {

std::atomic<uint64_t> g_kernel_launches{0};

namespace {

using dev::hash_vec;
using dev::ld_stream;
using dev::mix;

// ---------------------------------------------------------------- groups ---
// A "group" of G threads owns one page at a time.  G == 32: a warp, several
// groups per CTA.  G > 32: the whole CTA (blockDim.x == G).

template <int G>
struct GroupShared {
  uint64_t red[G > 32 ? G / 32 : 1];
  int flag;
};

template <int G>
__device__ __forceinline__ uint64_t group_sum(uint64_t v, GroupShared<G>& sh) {
  v = dev::warp_sum(v);
  if constexpr (G == 32) {
    return v;
  } else {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();  // previous readers of sh.red are done
    if (lane == 0) sh.red[warp] = v;
    __syncthreads();
    return dev::warp_sum(lane < G / 32 ? sh.red[lane] : 0ull);
  }
}

// Value of thread 0 of the group, in every thread of the group.
template <int G>
__device__ __forceinline__ int group_bcast0(int v, GroupShared<G>& sh) {
  if constexpr (G == 32) {
    return __shfl_sync(0xffffffffu, v, 0);
  } else {
    __syncthreads();
    if (threadIdx.x == 0) sh.flag = v;
    __syncthreads();
    return sh.flag;
  }
}

template <int G>
__device__ __forceinline__ bool group_any(bool v, GroupShared<G>& sh) {
  if constexpr (G == 32) {
    return __any_sync(0xffffffffu, v);
  } else {
    return __syncthreads_or(v) != 0;
  }
}

// ------------------------------------------------------------- page hash ---

// Full 64 KiB page; thread t of G hashes vectors t, t+G, ...  U loads are
// issued before their arithmetic so each thread keeps U*16 bytes in flight.
template <int G, int U>
__device__ __forceinline__ uint64_t hash_full_page(const uint8_t* src, int t) {
  constexpr int kPer = kPageVecs / G;
  static_assert(kPer % U == 0, "unroll must divide the per-thread vector count");
  constexpr uint64_t kStep = static_cast<uint64_t>(2 * G) * kPhi;
  const uint4* v4 = reinterpret_cast<const uint4*>(src) + t;
  uint64_t c = static_cast<uint64_t>(2 * t) * kPhi;
  uint64_t h = 0;
  // evict-normal, stated explicitly: with an evict-first policy (or no
  // hint) an 8 GiB pass after the application's 5 % page update took 1.39-
  // 1.40 ms against 1.34 ms, and 1.43-1.46 against 1.39 ms with a
  // device-to-host copy running beside it
  const uint64_t pol = dev::l2_evict_normal_policy();
#pragma unroll 1
  for (int k = 0; k < kPer; k += U) {
    uint4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = dev::ld_stream_hint(v4 + (k + u) * G, pol);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      h += hash_vec(v[u], c);
      c += kStep;
    }
  }
  return h;
}

// Verify mode, full page: the hash of `src` as above, and whether any of
// its bytes differs from `shadow`, in one pass over both.
template <int G, int U>
__device__ __forceinline__ uint64_t hash_full_page_cmp(const uint8_t* src, const uint8_t* shadow,
                                                       int t, bool& differs) {
  constexpr int kPer = kPageVecs / G;
  static_assert(kPer % U == 0, "unroll must divide the per-thread vector count");
  constexpr uint64_t kStep = static_cast<uint64_t>(2 * G) * kPhi;
  const uint4* v4 = reinterpret_cast<const uint4*>(src) + t;
  const uint4* w4 = reinterpret_cast<const uint4*>(shadow) + t;
  uint64_t c = static_cast<uint64_t>(2 * t) * kPhi;
  uint64_t h = 0;
  uint32_t x = 0;
  const uint64_t pol = dev::l2_evict_normal_policy();
#pragma unroll 1
  for (int k = 0; k < kPer; k += U) {
    uint4 v[U], w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      v[u] = dev::ld_stream_hint(v4 + (k + u) * G, pol);
      w[u] = dev::ld_stream_hint(w4 + (k + u) * G, pol);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      h += hash_vec(v[u], c);
      c += kStep;
      x |= (v[u].x ^ w[u].x) | (v[u].y ^ w[u].y) | (v[u].z ^ w[u].z) | (v[u].w ^ w[u].w);
    }
  }
  differs = x != 0;
  return h;
}

// Page with valid < 64 KiB bytes: whole vectors, then the partial vector.
template <int G>
__device__ __forceinline__ uint64_t hash_tail_page(const uint8_t* src, uint32_t valid, int t) {
  const uint32_t nvec = valid >> 4;
  uint64_t h = 0;
  for (uint32_t v = t; v < nvec; v += G)
    h += hash_vec(ld_stream(src + 16ull * v), static_cast<uint64_t>(2 * v) * kPhi);
  const uint32_t rem = valid & 15u;
  if (rem != 0 && static_cast<uint32_t>(t) == nvec % G)
    h += dev::hash_partial(dev::ld_partial(src + 16ull * nvec, rem), rem, 2ull * nvec);
  return h;
}

// Verify mode: does any valid byte differ from the shadow copy?
template <int G>
__device__ __forceinline__ bool page_differs(const uint8_t* src, const uint8_t* shadow,
                                             uint32_t valid, int t, GroupShared<G>& sh) {
  const uint32_t nvec = valid >> 4;
  bool diff = false;
  for (uint32_t v = t; v < nvec; v += G) {
    const uint4 x = ld_stream(src + 16ull * v);
    const uint4 y = ld_stream(shadow + 16ull * v);
    diff |= (x.x != y.x) | (x.y != y.y) | (x.z != y.z) | (x.w != y.w);
  }
  const uint32_t rem = valid & 15u;
  if (rem != 0 && t == 0)
    for (uint32_t b = 0; b < rem; ++b) diff |= src[16ull * nvec + b] != shadow[16ull * nvec + b];
  return group_any<G>(diff, sh);
}

// MINB > 1 caps registers so MINB CTAs fit on an SM (more warps, hence more
// loads in flight, at the cost of registers for the unrolled loads).
template <int G, int U, bool VERIFY, int MINB = 1>
__global__ void __launch_bounds__(256, (MINB > 1 ? MINB : 0)) k_hash_dirty(HashArgs a) {
  __shared__ GroupShared<G> sh;
  constexpr int kGroupsPerCta = (G == 32) ? 256 / 32 : 1;
  const int t = threadIdx.x % G;
  const uint64_t group = static_cast<uint64_t>(blockIdx.x) * kGroupsPerCta + threadIdx.x / G;
  const uint64_t n_groups = static_cast<uint64_t>(gridDim.x) * kGroupsPerCta;
  for (uint64_t g = group; g < a.n_pages; g += n_groups) {
    uint8_t* base;
    uint64_t bytes, first;
    if (a.allocs != nullptr) {
      const uint32_t k = dev::find_alloc(a.first_page, a.n_allocs, g);
      base = a.allocs[k].base;
      bytes = a.allocs[k].bytes;
      first = a.allocs[k].first_page;
    } else {
      base = a.one.base;
      bytes = a.one.bytes;
      first = 0;
    }
    const uint64_t p = g - first;
    const uint8_t* src = base + p * kPage;
    const uint32_t valid = dev::valid_bytes(bytes, p);
    // the committed hash is loaded before the page so that its latency hides
    // under the page's loads instead of following them
    uint64_t prev = 0;
    if (a.h_out == nullptr && t == 0 && !a.full) prev = a.h_table[g];
    // verify mode reads a full page's shadow in the same pass (two page
    // reads instead of three for an unchanged page)
    bool fused = false, differs = false;
    uint64_t h;
    if constexpr (VERIFY) fused = !a.full && valid == kPage;
    if (fused)
      h = hash_full_page_cmp<G, U>(src, a.shadow + g * kPage, t, differs);
    else
      h = (valid == kPage) ? hash_full_page<G, U>(src, t) : hash_tail_page<G>(src, valid, t);
    h = group_sum<G>(h, sh);
    if (a.h_out != nullptr) {
      if (t == 0) a.h_out[g] = h;
      continue;
    }
    int d = 0;
    if (t == 0) d = a.full || h != prev;
    if constexpr (VERIFY) {
      d = group_bcast0<G>(d, sh);
      const bool any = fused ? group_any<G>(differs, sh)
                             : (!d && page_differs<G>(src, a.shadow + g * kPage, valid, t, sh));
      if (!d && any) {
        d = 1;
        if (t == 0) atomicAdd(a.collisions, 1ull);
      }
    }
    if (t == 0) {
      a.h_table[g] = h;
      if (d) atomicOr(a.dirty_mask + (g >> 5), 1u << (g & 31));
    }
  }
}

// ------------------------------------------------------------------ scan ---

constexpr int kScanThreads = 1024;
constexpr uint64_t kMagic = 0x31474D494D555243ull;  // "CRUMIMG1" little-endian

__global__ void __launch_bounds__(kScanThreads) k_scan(ScanArgs a) {
  __shared__ uint32_t wsum[32];
  __shared__ uint64_t red[32];
  __shared__ uint32_t total_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // Each warp owns a contiguous segment of bitmap words and walks it 32
  // words at a time, lane l reading word base + l, so every load of the
  // warp is one contiguous 128-byte line (a thread-contiguous split made
  // each warp load touch 32 lines).
  constexpr int kWarps = kScanThreads / 32;
  const uint64_t seg = (a.n_words + kWarps - 1) / kWarps;
  const uint64_t s0 = min(static_cast<uint64_t>(warp) * seg, a.n_words);
  const uint64_t s1 = min(s0 + seg, a.n_words);
  // kB lines per batch are loaded before any is used: one CTA has to keep
  // enough loads in flight on its own
  constexpr int kB = 16;
  uint32_t cnt = 0;
  for (uint64_t base = s0; base < s1; base += 32 * kB) {
    uint32_t m[kB];
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      const uint64_t w = base + 32 * j + lane;
      m[j] = w < s1 ? __ldg(a.mask + w) : 0u;
    }
#pragma unroll
    for (int j = 0; j < kB; ++j) cnt += __popc(m[j]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) wsum[warp] = cnt;
  __syncthreads();
  if (warp == 0) {
    const uint32_t x = wsum[lane];
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    wsum[lane] = incl - x;  // exclusive prefix of the segments' totals
    if (lane == 31) total_sh = incl;
  }
  __syncthreads();
  uint32_t carry = wsum[warp];
  for (uint64_t base = s0; base < s1; base += 32 * kB) {
    uint32_t c[kB];
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      const uint64_t w = base + 32 * j + lane;
      c[j] = w < s1 ? __popc(__ldg(a.mask + w)) : 0u;
    }
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      const uint64_t w = base + 32 * j + lane;
      uint32_t incl = c[j];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (w < s1) a.word_offset[w] = carry + incl - c[j];
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  const uint32_t run = total_sh;
  if (tid == kScanThreads - 1) {
    a.word_offset[a.n_words] = run;
    *a.n_dirty_out = run;
    if (a.mailbox != nullptr) {
      a.mailbox[0] = run;
      a.mailbox[1] = a.collisions != nullptr ? *a.collisions : 0ull;
      a.mailbox[2] = a.error != nullptr ? *a.error : 0u;
      __threadfence_system();
    }
  }
  __syncthreads();
  const uint64_t n = total_sh;
  const uint64_t A = a.n_allocs;
  const uint64_t payload_off = kHeaderBytes + 16 * A + 16 * n;
  const uint64_t image_bytes = payload_off + n * kPage + 8;
  // header words 0..7, then allocation-table words 8 .. 8+2A-1
  uint64_t* meta = reinterpret_cast<uint64_t*>(a.meta);
  uint64_t cks = 0;
  for (uint64_t k = tid; k < 8 + 2 * A; k += kScanThreads) {
    uint64_t w;
    if (k < 8) {
      switch (k) {
        case 0: w = kMagic; break;
        case 1: w = 1ull | (static_cast<uint64_t>(a.flags) << 32); break;
        case 2: w = a.seq; break;
        case 3: w = a.parent_seq; break;
        case 4: w = static_cast<uint64_t>(kPage) | (A << 32); break;
        case 5: w = n; break;
        case 6: w = payload_off; break;
        default: w = image_bytes; break;
      }
    } else {
      const uint64_t e = (k - 8) >> 1;
      w = ((k - 8) & 1) ? __ldg(&a.allocs[e].bytes) : static_cast<uint64_t>(__ldg(&a.allocs[e].id));
    }
    meta[k] = w;
    cks += mix(w ^ (k * kPhi));
  }
  cks = dev::warp_sum(cks);
  if (lane == 0) red[warp] = cks;
  __syncthreads();
  if (warp == 0) {
    cks = dev::warp_sum(red[lane]);
    if (lane == 0) *a.trailer = cks;
  }
}

// ---------------------------------------------------------------- gather ---

// Global page of dirty slot s: the word w holding it, then the r-th set bit.
__device__ __forceinline__ uint64_t slot_to_page(const uint32_t* mask, const uint32_t* word_offset,
                                                 uint64_t n_words, uint64_t s) {
  uint64_t lo = 0, hi = n_words;  // last w with word_offset[w] <= s
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (word_offset[mid] <= s)
      lo = mid;
    else
      hi = mid;
  }
  uint32_t m = mask[lo];
  for (uint32_t r = static_cast<uint32_t>(s - word_offset[lo]); r > 0 && m != 0; --r) m &= m - 1;
  if (m == 0) return ~0ull;  // inconsistent bitmap: the caller skips the slot
  return lo * 32 + static_cast<uint64_t>(__ffs(m) - 1);
}

template <int G, int U, bool VERIFY>
__global__ void __launch_bounds__(256) k_gather(GatherArgs a) {
  __shared__ GroupShared<G> sh;
  constexpr int kGroupsPerCta = (G == 32) ? 256 / 32 : 1;
  const int t = threadIdx.x % G;
  const uint64_t group = static_cast<uint64_t>(blockIdx.x) * kGroupsPerCta + threadIdx.x / G;
  const uint64_t n_groups = static_cast<uint64_t>(gridDim.x) * kGroupsPerCta;
  const uint64_t n = *a.n_dirty;
  const uint64_t end = min(a.s_end, n);
  const uint64_t A = a.n_allocs;
  const uint64_t pt_w0 = (kHeaderBytes + 16 * A) / 8;           // first page-table word
  const uint64_t pay_w0 = (kHeaderBytes + 16 * A + 16 * n) / 8;  // first payload word
  uint64_t* meta = reinterpret_cast<uint64_t*>(a.meta);
  for (uint64_t s = a.s_begin + group; s < end; s += n_groups) {
    const uint64_t g = slot_to_page(a.mask, a.word_offset, a.n_words, s);
    if (g >= a.n_pages) continue;  // never taken when the scan is consistent
    const uint32_t k = dev::find_alloc(a.first_page, a.n_allocs, g);
    const uint64_t p = g - a.allocs[k].first_page;
    const uint8_t* src = a.allocs[k].base + p * kPage;
    const uint32_t valid = dev::valid_bytes(a.allocs[k].bytes, p);
    uint8_t* dst = a.payload + (s - a.s_begin) * kPage;
    uint64_t cks = 0;
    if (t == 0) {
      const uint64_t pte = static_cast<uint64_t>(k) | (p << 32);
      const uint64_t hv = a.h_table[g];
      meta[pt_w0 + s] = pte;
      meta[pt_w0 + n + s] = hv;
      cks = mix(pte ^ ((pt_w0 + s) * kPhi)) + mix(hv ^ ((pt_w0 + n + s) * kPhi));
    }
    uint64_t c = (pay_w0 + s * (kPage / 8) + 2ull * t) * kPhi;
    constexpr uint64_t kStep = static_cast<uint64_t>(2 * G) * kPhi;
    if (valid == kPage) {
      constexpr int kPer = kPageVecs / G;
#pragma unroll 1
      for (int j = 0; j < kPer; j += U) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = ld_stream(src + 16ull * (t + (j + u) * G));
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const uint64_t off = 16ull * (t + (j + u) * G);
          dev::st_stream(dst + off, v[u]);
          if constexpr (VERIFY) dev::st_stream(a.shadow + g * kPage + off, v[u]);
          cks += hash_vec(v[u], c);
          c += kStep;
        }
      }
    } else {
      for (uint32_t v = t; v < kPageVecs; v += G) {
        const uint32_t lo = 16u * v;
        uint4 x = make_uint4(0u, 0u, 0u, 0u);
        if (lo + 16 <= valid)
          x = ld_stream(src + lo);
        else if (lo < valid)
          x = dev::ld_partial(src + lo, valid - lo);
        dev::st_stream(dst + lo, x);
        if constexpr (VERIFY) dev::st_stream(a.shadow + g * kPage + lo, x);
        cks += hash_vec(x, c);
        c += kStep;
      }
    }
    cks = group_sum<G>(cks, sh);
    if (t == 0) atomicAdd(reinterpret_cast<unsigned long long*>(a.trailer),
                          static_cast<unsigned long long>(cks));
  }
}

// ------------------------------------------------------------ hash bytes ---

__global__ void __launch_bounds__(256) k_hash_bytes(const uint8_t* p, uint64_t n,
                                                    uint64_t first_index,
                                                    unsigned long long* out) {
  const uint64_t nvec = n >> 4;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  uint64_t h = 0;
  for (uint64_t v = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < nvec;
       v += stride)
    h += hash_vec(ld_stream(p + 16 * v), (first_index + 2 * v) * kPhi);
  const uint32_t rem = static_cast<uint32_t>(n & 15u);
  if (rem != 0 && blockIdx.x == 0 && threadIdx.x == 0)
    h += dev::hash_partial(dev::ld_partial(p + 16 * nvec, rem), rem, first_index + 2 * nvec);
  h = dev::warp_sum(h);
  if ((threadIdx.x & 31) == 0 && h != 0) atomicAdd(out, static_cast<unsigned long long>(h));
}

// ------------------------------------------------- bulk-copy page hashing ---
//
// Warp-specialised variant of k_hash_dirty for sm_90+ bulk copies: lane 0 of
// warp 0 streams every full page of the CTA's share, as four 16 KiB
// quarters, into a ring of STAGES shared-memory buffers with
// cp.async.bulk (completion counted on a "full" mbarrier per buffer); CW
// consumer warps hash each buffer from shared memory and release it on an
// "empty" mbarrier.  Bytes in flight per CTA = STAGES * 16 KiB, independent
// of register allocation.  Tail pages (valid < 64 KiB) are hashed by the
// consumers straight from global memory.  Every wait is bounded; a wait that
// runs out sets *error and `stop`: the producer stops issuing and waits
// (bounded) for its copies in flight, consumers stop waiting and hashing but
// keep meeting at their per-page barrier, so every thread still exits.

constexpr uint32_t kQuarter = kPage / 4;
constexpr uint32_t kWaitLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// true once the barrier's phase with this parity has completed; false if the
// bounded number of polls ran out or *stop became nonzero.
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for at most `limit_ns` (globaltimer) and kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity,
                                          const volatile int* stop, uint64_t limit_ns) {
  const uint32_t addr = smem_u32(bar);
  const uint64_t deadline = global_ns() + limit_ns;
  for (uint32_t i = 0; i < kWaitLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 255u) == 255u) {
      if (stop != nullptr && *stop) return false;
      if (global_ns() > deadline) return false;
    }
  }
  return false;
}

__device__ __forceinline__ void bulk_load(void* dst_smem, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst_smem)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void consumer_sync(int threads) {
  asm volatile("bar.sync 1, %0;" ::"r"(threads) : "memory");
}

template <int STAGES, int CW>
__global__ void __launch_bounds__(32 * (CW + 1)) k_hash_dirty_bulk(HashArgs a) {
  extern __shared__ __align__(128) uint8_t ring[];
  __shared__ __align__(8) uint64_t full_bar[STAGES];
  __shared__ __align__(8) uint64_t empty_bar[STAGES];
  __shared__ uint64_t red[CW];
  __shared__ int stop;
  constexpr int kConsumers = 32 * CW;
  const uint64_t limit_ns = a.wait_limit_ns != 0 ? a.wait_limit_ns : 2000000000ull;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], CW);
    }
    stop = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == 0) {
    // ---- producer ----
    if (lane != 0) return;
    uint32_t chunk = 0;
    int last_issued[STAGES];  // newest chunk issued into each stage, -1: none
#pragma unroll
    for (int s = 0; s < STAGES; ++s) last_issued[s] = -1;
    bool ok = true;
    for (uint64_t g = blockIdx.x; ok && g < a.n_pages; g += gridDim.x) {
      const uint8_t* base;
      uint64_t bytes, first;
      if (a.allocs != nullptr) {
        const uint32_t k = dev::find_alloc(a.first_page, a.n_allocs, g);
        base = a.allocs[k].base;
        bytes = a.allocs[k].bytes;
        first = a.allocs[k].first_page;
      } else {
        base = a.one.base;
        bytes = a.one.bytes;
        first = 0;
      }
      const uint64_t p = g - first;
      if (dev::valid_bytes(bytes, p) != kPage) continue;
      const uint8_t* src = base + p * kPage;
      for (uint32_t q = 0; q < 4; ++q, ++chunk) {
        const uint32_t s = chunk % STAGES, k = chunk / STAGES;
        if (k > 0 && !mbar_wait(&empty_bar[s], (k - 1) & 1, &stop, limit_ns)) {
          ok = false;
          break;
        }
        // self-test hook: one chunk is never issued, so its consumers' wait
        // runs out (a flag nothing sets)
        if (a.test_skip_chunk != 0 && blockIdx.x == 0 && chunk + 1 == a.test_skip_chunk) continue;
        mbar_arrive_expect_tx(&full_bar[s], kQuarter);
        bulk_load(ring + s * kQuarter, src + q * kQuarter, kQuarter, &full_bar[s]);
        last_issued[s] = static_cast<int>(chunk);
      }
    }
    if (!ok) {
      if (a.error) atomicExch(a.error, 1u);
      stop = 1;
    }
    // The CTA must not retire with a copy into its shared memory in flight,
    // also when the consumers gave up on it: wait for the newest copy of
    // every stage (bounded as well).
    for (uint32_t s = 0; s < STAGES; ++s)
      if (last_issued[s] >= 0)
        mbar_wait(&full_bar[s], (static_cast<uint32_t>(last_issued[s]) / STAGES) & 1, nullptr,
                  limit_ns);
    return;
  }

  // ---- consumers ----
  const int ct = threadIdx.x - 32, cw = warp - 1;
  uint32_t chunk = 0;
  bool bad = false;
  const uint64_t c_base = static_cast<uint64_t>(2 * ct) * kPhi;
  constexpr uint64_t kStepU = static_cast<uint64_t>(2 * kConsumers) * kPhi;
  constexpr uint64_t kStepQ = static_cast<uint64_t>(2 * (kQuarter / 16)) * kPhi;
  for (uint64_t g = blockIdx.x; g < a.n_pages; g += gridDim.x) {
    const uint8_t* base;
    uint64_t bytes, first;
    if (a.allocs != nullptr) {
      const uint32_t k = dev::find_alloc(a.first_page, a.n_allocs, g);
      base = a.allocs[k].base;
      bytes = a.allocs[k].bytes;
      first = a.allocs[k].first_page;
    } else {
      base = a.one.base;
      bytes = a.one.bytes;
      first = 0;
    }
    const uint64_t p = g - first;
    const uint32_t valid = dev::valid_bytes(bytes, p);
    uint64_t prev = 0;  // committed hash, loaded early (see k_hash_dirty)
    if (a.h_out == nullptr && ct == 0 && !a.full) prev = a.h_table[g];
    uint64_t h = 0;
    if (valid == kPage) {
      for (uint32_t q = 0; q < 4; ++q, ++chunk) {
        const uint32_t s = chunk % STAGES, k = chunk / STAGES;
        bool got = false;
        if (!bad) got = mbar_wait(&full_bar[s], k & 1, &stop, limit_ns);
        // warp-uniform, so the warp's later collectives see all 32 lanes
        if (!__all_sync(0xffffffffu, got)) {
          bad = true;
          stop = 1;  // the producer stops issuing at its next poll
          continue;
        }
        const uint4* buf = reinterpret_cast<const uint4*>(ring + s * kQuarter);
        uint64_t c = c_base + q * kStepQ;
#pragma unroll
        for (int u = 0; u < static_cast<int>(kQuarter / 16) / kConsumers; ++u) {
          h += hash_vec(buf[ct + u * kConsumers], c);
          c += kStepU;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_bar[s]);
      }
    } else if (!bad) {
      h = hash_tail_page<kConsumers>(base + p * kPage, valid, ct);
    }
    h = dev::warp_sum(h);
    consumer_sync(kConsumers);
    if (lane == 0) red[cw] = h;
    consumer_sync(kConsumers);
    // `stop` is set before the barrier by any warp that gave up on this page
    if (ct == 0 && !*static_cast<volatile int*>(&stop)) {
      uint64_t total = 0;
#pragma unroll
      for (int w = 0; w < CW; ++w) total += red[w];
      if (a.h_out != nullptr) {
        a.h_out[g] = total;
      } else {
        const bool d = a.full || total != prev;
        a.h_table[g] = total;
        if (d) atomicOr(a.dirty_mask + (g >> 5), 1u << (g & 31));
      }
    }
  }
  if (bad) {
    stop = 1;
    if (a.error) atomicExch(a.error, 1u);
  }
}

// G == 32: eight one-warp groups in a 256-thread CTA; G > 32: one group
// per CTA of G threads.
template <int G, int U, bool V, int MINB = 1>
KernelSpec hash_spec_t(uint64_t n_pages) {
  auto kern = k_hash_dirty<G, U, V, MINB>;
  constexpr int kThreads = G == 32 ? 256 : G;
  return KernelSpec{reinterpret_cast<const void*>(kern),
                    grid_for(kern, n_pages, G == 32 ? 8 : 1, kThreads), kThreads, 0};
}

template <int STAGES, int CW>
cudaError_t hash_bulk_spec_t(uint64_t n_pages, KernelSpec* out) {
  auto kern = k_hash_dirty_bulk<STAGES, CW>;
  constexpr int kThreads = 32 * (CW + 1);
  constexpr int kSmem = STAGES * static_cast<int>(kQuarter);
  const cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess) return e;
  const int per_sm = resident_per_sm(reinterpret_cast<const void*>(kern), kThreads, kSmem);
  const uint64_t cap = static_cast<uint64_t>(per_sm) * num_sms();
  *out = KernelSpec{reinterpret_cast<const void*>(kern),
                    static_cast<unsigned>(std::max<uint64_t>(1, std::min(n_pages, cap))), kThreads,
                    kSmem};
  return cudaSuccess;
}

template <int G, int U, bool V>
KernelSpec gather_spec_t(uint64_t max_slots) {
  auto kern = k_gather<G, U, V>;
  return KernelSpec{reinterpret_cast<const void*>(kern), grid_for(kern, max_slots, G == 32 ? 8 : 1),
                    256, 0};
}

}  // namespace

static int g_num_sms = 0;

int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

int resident_per_sm(const void* func, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(func, threads, smem, dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  per_sm = std::max(1, per_sm);
  cache.emplace(key, per_sm);
  return per_sm;
}

// Hash mappings 0-5 are register mappings, 6-8 bulk-copy mappings; gather
// and restore use the register mappings 0-5 only.
// 9-11: register mappings capped at 32 registers (8 CTAs of 256 per SM).
const Mapping kMappings[] = {
    {32, 4, 0},  {32, 8, 0},  {32, 16, 0},  {256, 2, 0}, {256, 4, 0}, {256, 8, 0},
    {256, 0, 4}, {256, 0, 6}, {512, 0, 4},  {32, 4, 0},  {32, 8, 0},  {256, 4, 0},
    {64, 8, 0},  {128, 4, 0}, {128, 8, 0},
};
static_assert(sizeof(kMappings) / sizeof(kMappings[0]) == CRUM_NUM_HASH_MAPPINGS,
              "the header's mapping count");
const int kNumMappings = sizeof(kMappings) / sizeof(kMappings[0]);

cudaError_t hash_spec(uint64_t n_pages, int mapping, bool verify, KernelSpec* out) {
  // verify mode compares pages against the shadow copy, which only the
  // register mappings do; bulk-copy mappings fall back to mapping 1 there
  if (verify && mapping >= 6 && mapping <= 11) mapping = 1;
#define CRUM_HASH_CASE(i, G, U)                                                       \
  case i:                                                                             \
    *out = verify ? hash_spec_t<G, U, true>(n_pages) : hash_spec_t<G, U, false>(n_pages); \
    return cudaSuccess;
  switch (mapping) {
    CRUM_HASH_CASE(0, 32, 4)
    CRUM_HASH_CASE(1, 32, 8)
    CRUM_HASH_CASE(2, 32, 16)
    CRUM_HASH_CASE(3, 256, 2)
    CRUM_HASH_CASE(4, 256, 4)
    CRUM_HASH_CASE(5, 256, 8)
    case 6:
      return hash_bulk_spec_t<4, 8>(n_pages, out);
    case 7:
      return hash_bulk_spec_t<6, 8>(n_pages, out);
    case 8:
      return hash_bulk_spec_t<4, 16>(n_pages, out);
    case 9:
      *out = hash_spec_t<32, 4, false, 8>(n_pages);
      return cudaSuccess;
    case 10:
      *out = hash_spec_t<32, 8, false, 8>(n_pages);
      return cudaSuccess;
    case 11:
      *out = hash_spec_t<256, 4, false, 8>(n_pages);
      return cudaSuccess;
    CRUM_HASH_CASE(12, 64, 8)
    CRUM_HASH_CASE(13, 128, 4)
    CRUM_HASH_CASE(14, 128, 8)
    default:
      return cudaErrorInvalidValue;
  }
#undef CRUM_HASH_CASE
}

cudaError_t scan_spec(KernelSpec* out) {
  *out = KernelSpec{reinterpret_cast<const void*>(k_scan), 1, kScanThreads, 0};
  return cudaSuccess;
}

cudaError_t gather_spec(uint64_t max_slots, int mapping, bool verify, KernelSpec* out) {
#define CRUM_GATHER_CASE(i, G, U)                                                              \
  case i:                                                                                      \
    *out = verify ? gather_spec_t<G, U, true>(max_slots) : gather_spec_t<G, U, false>(max_slots); \
    return cudaSuccess;
  switch (mapping) {
    CRUM_GATHER_CASE(0, 32, 4)
    CRUM_GATHER_CASE(1, 32, 8)
    CRUM_GATHER_CASE(2, 32, 16)
    CRUM_GATHER_CASE(3, 256, 2)
    CRUM_GATHER_CASE(4, 256, 4)
    CRUM_GATHER_CASE(5, 256, 8)
    default:
      return cudaErrorInvalidValue;
  }
#undef CRUM_GATHER_CASE
}

cudaError_t launch_spec(const KernelSpec& s, void* arg, cudaStream_t st) {
  void* args[] = {arg};
  const cudaError_t e = cudaLaunchKernel(s.func, dim3(s.grid), dim3(s.block), args, s.smem, st);
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return e;
}

cudaError_t launch_hash_dirty(const HashArgs& a, int mapping, bool verify, cudaStream_t st) {
  if (a.n_pages == 0) return cudaSuccess;
  KernelSpec s;
  const cudaError_t e = hash_spec(a.n_pages, mapping, verify, &s);
  if (e != cudaSuccess) return e;
  HashArgs copy = a;
  return launch_spec(s, &copy, st);
}

cudaError_t launch_scan(const ScanArgs& a, cudaStream_t st) {
  KernelSpec s;
  scan_spec(&s);
  ScanArgs copy = a;
  return launch_spec(s, &copy, st);
}

cudaError_t launch_gather(const GatherArgs& a, uint64_t max_slots, int mapping, bool verify,
                          cudaStream_t st) {
  if (max_slots == 0) return cudaSuccess;
  KernelSpec s;
  const cudaError_t e = gather_spec(max_slots, mapping, verify, &s);
  if (e != cudaSuccess) return e;
  GatherArgs copy = a;
  return launch_spec(s, &copy, st);
}

cudaError_t launch_hash_bytes(const uint8_t* p, uint64_t n, uint64_t first_index, uint64_t* out,
                              cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const uint64_t nvec = (n + 15) / 16;
  const uint64_t cap = static_cast<uint64_t>(resident_ctas(k_hash_bytes, 256));
  const unsigned grid =
      static_cast<unsigned>(std::max<uint64_t>(1, std::min((nvec + 255) / 256, cap)));
  k_hash_bytes<<<grid, 256, 0, st>>>(p, n, first_index, reinterpret_cast<unsigned long long*>(out));
  g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace crum
