// Device-side building blocks of the capture/restore path (sm_103a).
//
// Page hash (the dirty test that replaces the write-fault tracking of
// Algorithm 1 / Section 3.2, since device stores cannot be trapped):
//   h(page) = sum_i mix(w_i ^ (i * PHI))  mod 2^64
// over the page's little-endian 64-bit words, i page-local, a final partial
// word zero-padded.  mix is splitmix64's output function (Steele, Lea,
// Flood, OOPSLA 2014).  The sum is order-free, so threads hash disjoint
// slices and any reduction tree gives the same bits.
#pragma once
#include <cstdint>

namespace crum {

constexpr uint32_t kPage = 65536;
constexpr uint32_t kPageVecs = kPage / 16;  // 16-byte vectors per page
constexpr uint32_t kHeaderBytes = 64;
constexpr uint64_t kPhi = 0x9E3779B97F4A7C15ull;

// One registered allocation as the kernels see it.
struct DevAlloc {
  uint8_t* base;        // 16-byte aligned device pointer
  uint64_t bytes;       // registered size
  uint64_t first_page;  // global index of its page 0
  uint32_t id;          // registration id (written to the image)
  uint32_t n_pages;
};

namespace dev {

__device__ __forceinline__ uint64_t mix(uint64_t z) {
  z ^= z >> 30;
  z *= 0xBF58476D1CE4E5B9ull;
  z ^= z >> 27;
  z *= 0x94D049BB133111EBull;
  z ^= z >> 31;
  return z;
}

// Streaming 16-byte load: read once, keep out of L1.
__device__ __forceinline__ uint4 ld_stream(const void* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p));
  return v;
}

// Explicit evict-normal L2 policy for a stream read once.  A load with no
// cache hint does not behave the same on this path: after an application
// kernel has left lines dirty in L2, an 8 GiB pass with no hint (or with an
// evict-first policy) ran 0.05-0.08 ms longer than with this policy.
__device__ __forceinline__ uint64_t l2_evict_normal_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// ld_stream with an explicit L2 cache policy.
__device__ __forceinline__ uint4 ld_stream_hint(const void* p, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
      : "l"(p), "l"(pol));
  return v;
}

// Coherent 16-byte load (data written earlier in the same stream).
__device__ __forceinline__ uint4 ld_plain(const void* p) {
  return *reinterpret_cast<const uint4*>(p);
}

// Streaming 16-byte store (staging is read next by the copy engine).
__device__ __forceinline__ void st_stream(void* p, uint4 v) {
  asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}

// Contribution of one 16-byte vector whose first word has index i0:
// words i0 and i0+1, with c0 = i0 * PHI.
__device__ __forceinline__ uint64_t hash_vec(uint4 v, uint64_t c0) {
  const uint64_t w0 = (static_cast<uint64_t>(v.y) << 32) | v.x;
  const uint64_t w1 = (static_cast<uint64_t>(v.w) << 32) | v.z;
  return mix(w0 ^ c0) + mix(w1 ^ (c0 + kPhi));
}

// Bytes [0, n) of a 16-byte vector at p (n < 16), the rest zero.
__device__ __forceinline__ uint4 ld_partial(const uint8_t* p, uint32_t n) {
  uint64_t lo = 0, hi = 0;
  for (uint32_t b = 0; b < n; ++b) {
    const uint64_t byte = p[b];
    if (b < 8)
      lo |= byte << (8 * b);
    else
      hi |= byte << (8 * (b - 8));
  }
  return make_uint4(static_cast<uint32_t>(lo), static_cast<uint32_t>(lo >> 32),
                    static_cast<uint32_t>(hi), static_cast<uint32_t>(hi >> 32));
}

// Hash of the partial last vector of a byte string: bytes [0, n) of the
// vector whose first word has index i0.  Includes word i0+1 only if n > 8,
// since words wholly past the end are not part of the string.
__device__ __forceinline__ uint64_t hash_partial(uint4 v, uint32_t n, uint64_t i0) {
  const uint64_t w0 = (static_cast<uint64_t>(v.y) << 32) | v.x;
  const uint64_t w1 = (static_cast<uint64_t>(v.w) << 32) | v.z;
  uint64_t h = mix(w0 ^ (i0 * kPhi));
  if (n > 8) h += mix(w1 ^ ((i0 + 1) * kPhi));
  return h;
}

__device__ __forceinline__ uint64_t warp_sum(uint64_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Allocation holding global page g: the last a with first_page <= g.
__device__ __forceinline__ uint32_t find_alloc(const uint64_t* first_page, uint32_t n_allocs,
                                               uint64_t g) {
  uint32_t lo = 0, hi = n_allocs;  // answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(first_page + mid) <= g)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t valid_bytes(uint64_t bytes, uint64_t p) {
  const uint64_t left = bytes - p * kPage;
  return left < kPage ? static_cast<uint32_t>(left) : kPage;
}

}  // namespace dev
}  // namespace crum
