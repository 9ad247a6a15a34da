// Kernels of the byte-plane dictionary code on the capture side and their
// launchers (the code itself is stated in codec.cuh and include/crum.h).
//
//   k_bpd_size      one CTA per staged slot: alphabet of each byte plane and
//                   the slot's encoded length
//   k_bpd_scan      one CTA: slot offsets (exclusive prefix of the lengths),
//                   encoded payload size, compressed-form header words
//   k_bpd_encode    one CTA per slot: the slot's code at its offset, and
//                   the compressed image's checksum
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

using dev::hash_vec;
using dev::ld_stream;

// present[plane][value] for every byte of one 16-byte vector of the slot
// that falls in a plane of `planes` (bit j: plane j); several threads may
// store the same 1, no atomics needed.
__device__ __forceinline__ void bpd_mark(const uint4& x, BpdSmem& m, uint32_t planes) {
  const uint32_t w[4] = {tslot4(x.x), tslot4(x.y), tslot4(x.z), tslot4(x.w)};
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (planes & (1u << ((q & 1) * 4 + t))) m.present[(q & 1) * 4 + t][(w[q] >> (8 * t)) & 255u] = 1;
}

// 4 x 4 byte transpose: o_c gets byte c of a0, a1, a2, a3 (in that order).
__device__ __forceinline__ void transpose4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                           uint32_t& o0, uint32_t& o1, uint32_t& o2, uint32_t& o3) {
  const uint32_t t0 = __byte_perm(a0, a1, 0x5140), t1 = __byte_perm(a0, a1, 0x7362);
  const uint32_t t2 = __byte_perm(a2, a3, 0x5140), t3 = __byte_perm(a2, a3, 0x7362);
  o0 = __byte_perm(t0, t2, 0x5410);
  o1 = __byte_perm(t0, t2, 0x7632);
  o2 = __byte_perm(t1, t3, 0x5410);
  o3 = __byte_perm(t1, t3, 0x7632);
}

// Starts the asynchronous copy of one 64 KiB slot into the encoder's
// swizzled shared-memory layout (enc_chunk_pos): each thread copies 16
// chunks of 16 bytes, a warp's copies covering 512 contiguous bytes each.
// The caller waits for it with cp.async.wait_all and a barrier.
__device__ __forceinline__ void enc_prefetch(const uint8_t* slot, uint4* slot_sm, int tid) {
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const uint32_t v = tid + 256u * i;
    const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(slot_sm + enc_chunk_pos(v >> 4, v & 15u)));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(slot + 16ull * v) : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// One 64-bit word's term of the image checksum: word w at index i.
__device__ __forceinline__ uint64_t hash_word(uint64_t w, uint64_t i) { return dev::mix(w ^ (i * kPhi)); }

__device__ __forceinline__ uint64_t pair64(uint32_t lo, uint32_t hi) {
  return (static_cast<uint64_t>(hi) << 32) | lo;
}

// This thread's 32 bytes of a plane (pw) as B-bit ranks, LSB first: exactly
// B words at `words`.  B is a template argument, so every rank's bit
// position is known at compile time.  Returns the image-checksum terms of
// the 64-bit words this thread completes: 64-bit word i of the packed
// section (image index u0 + i) is its 32-bit words 2i and 2i + 1.  For odd
// B a run starts (odd threads) or ends (even threads) in the middle of one;
// the even thread takes that word, its high half from the next lane.  Every
// lane of the warp calls it (B is uniform across the CTA).
template <int B>
__device__ __forceinline__ uint64_t pack_ranks(const uint32_t (&pw)[8], const uint8_t* rank, uint32_t* words,
                                               uint64_t u0) {
  uint32_t out[B];
#pragma unroll
  for (int e = 0; e < B; ++e) out[e] = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t t = tslot4(pw[k]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t r = rank[(t >> (8 * i)) & 255u];
      const int bit = (4 * k + i) * B;  // a constant once unrolled
      out[bit >> 5] |= r << (bit & 31);
      if ((bit & 31) + B > 32) out[(bit >> 5) + 1] |= r >> (32 - (bit & 31));
    }
  }
#pragma unroll
  for (int e = 0; e < B; ++e) words[e] = out[e];
  const uint64_t t = threadIdx.x;
  uint64_t h = 0;
  if constexpr (B % 2 == 0) {
    const uint64_t c = (u0 + t * (B / 2)) * kPhi;  // index terms: c + i kPhi
#pragma unroll
    for (int i = 0; i < B / 2; ++i) h += dev::mix(pair64(out[2 * i], out[2 * i + 1]) ^ (c + i * kPhi));
  } else {
    // one instruction stream for both parities (a divergent branch would
    // run both): odd threads start one 32-bit word later
    const uint32_t next = __shfl_down_sync(0xffffffffu, out[0], 1);
    const bool odd = t & 1;
    const uint64_t c = (u0 + (t * B + odd) / 2) * kPhi;
#pragma unroll
    for (int i = 0; i < B / 2; ++i)
      h += dev::mix(pair64(odd ? out[2 * i + 1] : out[2 * i], odd ? out[2 * i + 2] : out[2 * i + 1]) ^
                    (c + i * kPhi));
    if (!odd) h += dev::mix(pair64(out[B - 1], next) ^ (c + (B / 2) * kPhi));
  }
  return h;
}

__device__ __forceinline__ void plane_words(const uint32_t (&p)[8], uint32_t (&pw)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) pw[k] = p[k];
}

// After the sample marks: the planes that may still have b < 8 (sample
// alphabet below kBpdRawAlphabet), into m.open (CTA-wide; leaves the CTA
// synchronised).  Warp j counts plane j.
__device__ __forceinline__ void bpd_open_planes(BpdSmem& m) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) m.open = 0;
  __syncthreads();
  if (warp < 8) {
    const uint2 p = reinterpret_cast<const uint2*>(m.present[warp])[lane];
    // each byte is 0 or 1: the byte sum of a word is its popcount
    uint32_t c = __popc(p.x) + __popc(p.y);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0 && c < kBpdRawAlphabet) atomicOr(&m.open, 1u << warp);
  }
  __syncthreads();
}

// Alphabet size, width, ranks and section layout of every plane (CTA-wide,
// after the presence marks; leaves the CTA synchronised).
__device__ void bpd_plan(BpdSmem& m) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < 8) {
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) c += m.present[warp][tslot(lane * 8 + j)];
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    uint32_t r = incl - c;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      m.rank[warp][tslot(lane * 8 + j)] = static_cast<uint8_t>(r);
      r += m.present[warp][tslot(lane * 8 + j)];
    }
    if (lane == 31) {
      m.k[warp] = incl;
      m.b[warp] = ceil_log2(incl);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t pos = 16;
    for (int j = 0; j < 8; ++j) {
      m.sec[j] = pos;
      pos += m.b[j] == 8 ? kPlaneBytes : ((m.k[j] + 15u) & ~15u) + 1024u * m.b[j];
    }
    m.sec[8] = pos;
    m.len = pos >= kPage ? static_cast<uint32_t>(kPage) : pos;
  }
  __syncthreads();
}

static_assert(kBpdAlphBytes == kBpdThreads, "one alphabet byte per thread");

__global__ void __launch_bounds__(kBpdThreads) k_bpd_size(BpdSizeArgs a) {
  __shared__ BpdSmem m;
  const uint64_t n = *a.n_dirty;
  for (uint64_t s = blockIdx.x; s < n; s += gridDim.x) {
    for (uint32_t i = threadIdx.x; i < 8 * 256 / 4; i += blockDim.x)
      reinterpret_cast<uint32_t*>(m.present)[i] = 0;
    __syncthreads();
    const uint8_t* slot = a.payload + s * kPage;
    // the sample: the first 8 KiB of the slot (1,024 bytes of every plane),
    // two vectors per thread, both loads in flight before the marks
    static_assert(kPlaneBytes / 16 == 2 * kBpdThreads, "sample = two vectors per thread");
    {
      const uint4 x0 = ld_stream(slot + 16ull * threadIdx.x);
      const uint4 x1 = ld_stream(slot + 16ull * (threadIdx.x + kBpdThreads));
      bpd_mark(x0, m, 0xffu);
      bpd_mark(x1, m, 0xffu);
    }
    __syncthreads();
    bpd_open_planes(m);
    const uint32_t open = m.open;
    // the rest only when some plane may still have b < 8 (random words:
    // never, so only an eighth of such a slot is read), seven loads in
    // flight per thread
    if (open != 0) {
#pragma unroll 1
      for (uint32_t v0 = 2 * kBpdThreads; v0 < kPageVecs; v0 += 7 * kBpdThreads) {
        uint4 x[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) x[i] = ld_stream(slot + 16ull * (v0 + threadIdx.x + i * kBpdThreads));
#pragma unroll
        for (int i = 0; i < 7; ++i) bpd_mark(x[i], m, open);
      }
    }
    __syncthreads();
    bpd_plan(m);
    if (threadIdx.x == 0) a.enc_len[s] = m.len;
    {
      // the alphabets for the encoder: thread t packs plane t / 32's
      // presence of values 8 (t % 32) .. 8 (t % 32) + 7
      const uint32_t j = threadIdx.x >> 5, v0 = 8u * (threadIdx.x & 31);
      uint32_t bits = 0;
#pragma unroll
      for (uint32_t i = 0; i < 8; ++i) bits |= static_cast<uint32_t>(m.present[j][tslot(v0 + i)]) << i;
      a.alph[s * kBpdAlphBytes + threadIdx.x] = static_cast<uint8_t>(bits);
    }
    __syncthreads();
  }
}

// Slot offsets (exclusive prefix of the encoded lengths) into the image's
// offset table, the encoded payload size, and the header words that differ
// in the compressed form.  One CTA; warp w owns a contiguous segment.
__global__ void __launch_bounds__(1024) k_bpd_scan(BpdScanArgs a) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long total_sh;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t n = *a.n;
  const uint64_t A = a.n_allocs;
  const uint64_t seg = (n + 31) / 32;
  const uint64_t s0 = min(static_cast<uint64_t>(warp) * seg, n), s1 = min(s0 + seg, n);
  unsigned long long cnt = 0;
  for (uint64_t s = s0 + lane; s < s1; s += 32) cnt += a.enc_len[s];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) wsum[warp] = cnt;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long x = wsum[lane];
    unsigned long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    wsum[lane] = incl - x;
    if (lane == 31) total_sh = incl;
  }
  __syncthreads();
  unsigned long long carry = wsum[warp] + a.base;
  uint64_t* off = a.offs != nullptr ? a.offs
                                    : reinterpret_cast<uint64_t*>(a.meta + kHeaderBytes + 16 * A + 16 * n);
  for (uint64_t base = s0; base < s1; base += 32) {
    const uint64_t s = base + lane;
    const unsigned long long len = s < s1 ? a.enc_len[s] : 0ull;
    unsigned long long incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (s < s1) off[s] = carry + incl - len;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (tid == 0) {
    const uint64_t total = total_sh;
    if (a.offs == nullptr) {
      const uint64_t tab_end = kHeaderBytes + 16 * A + 24 * n;
      const uint64_t poff = (tab_end + 15) & ~15ull;
      for (uint64_t b = tab_end; b < poff; ++b) a.meta[b] = 0;
      uint64_t* h = reinterpret_cast<uint64_t*>(a.meta);
      const uint64_t flags = (h[1] >> 32) | 2ull;
      h[1] = 2ull | (flags << 32);
      h[6] = poff;
      h[7] = poff + total + 8;
    }
    *a.total_out = total;
    if (a.mailbox != nullptr) {
      a.mailbox[3] = total;
      __threadfence_system();
    }
  }
}

// Encodes slot s into out + offset[s].  Thread t owns bytes [256 t, 256 t +
// 256) of the slot: 32 little-endian 64-bit words, byte j of word q being
// byte 32 t + q of plane j.  It holds them in registers transposed into its
// 32 bytes of every plane, so it packs exactly b words of each plane's rank
// stream and, once the alphabets are known, needs no shared memory but the
// rank tables and no further barrier.  The slot arrives by coalesced 16-byte loads into
// a swizzled shared-memory copy (enc_chunk_pos), from which each thread
// reads its own 256 bytes without bank conflicts.
//
// The image checksum is summed as the code is written: each thread adds the
// terms of the 64-bit words it stores (a slot stored as is, the header,
// planes stored as is, packed ranks, and after the slot's last barrier one
// word of the dictionaries, which the CTA builds in shared memory); for the
// whole image (offs null) the grid also adds the header and tables, which
// are final before this launch.
__global__ void __launch_bounds__(kBpdThreads, 2) k_bpd_encode(BpdEncodeArgs a) {
  __shared__ BpdSmem m;
  __shared__ uint64_t dict_sm[8][16];  // each plane's dictionary, stored and hashed after the slot
  extern __shared__ uint4 slot_sm[];
  const int tid = threadIdx.x;
  const uint64_t n = *a.n;
  const bool whole = a.offs == nullptr;
  const uint64_t* off =
      whole ? reinterpret_cast<const uint64_t*>(a.meta + kHeaderBytes + 16ull * a.n_allocs + 16 * n) : a.offs;
  const uint64_t poff = whole ? (kHeaderBytes + 16ull * a.n_allocs + 24 * n + 15) & ~15ull : a.poff;
  uint64_t h = 0;  // this thread's terms of the image checksum
  if (whole)
    for (uint64_t v = static_cast<uint64_t>(blockIdx.x) * blockDim.x + tid; v < poff / 16;
         v += static_cast<uint64_t>(gridDim.x) * blockDim.x)
      h += hash_vec(ld_stream(a.meta + 16 * v), (2 * v) * kPhi);
  if (blockIdx.x < n) enc_prefetch(a.payload + blockIdx.x * kPage, slot_sm, tid);
  for (uint64_t s = blockIdx.x; s < n; s += gridDim.x) {
    // loaded now, used after the transposition
    const uint64_t off_s = off[s];
    const uint32_t alph = a.alph[s * kBpdAlphBytes + tid];
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
    // this thread's 32 bytes of each plane: P[j][k] holds plane-j bytes
    // 4k .. 4k+3, taken from words 4k .. 4k+3 by a 4 x 4 byte transpose of
    // their low halves (planes 0-3) and of their high halves (planes 4-7)
    uint32_t P[8][8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const uint4 c0 = slot_sm[enc_chunk_pos(tid, 2 * k)];
      const uint4 c1 = slot_sm[enc_chunk_pos(tid, 2 * k + 1)];
      transpose4(c0.x, c0.z, c1.x, c1.z, P[0][k], P[1][k], P[2][k], P[3][k]);
      transpose4(c0.y, c0.w, c1.y, c1.w, P[4][k], P[5][k], P[6][k], P[7][k]);
    }
    __syncthreads();  // every thread has its bytes: the buffer takes the next slot
    if (s + gridDim.x < n) enc_prefetch(a.payload + (s + gridDim.x) * kPage, slot_sm, tid);
    // the slot's alphabets as the size kernel found them (so both plan the
    // same layout): thread t expands plane t / 32's presence of values
    // 8 (t % 32) .. 8 (t % 32) + 7
    {
      const uint32_t j = tid >> 5, v0 = 8u * (tid & 31);
#pragma unroll
      for (uint32_t i = 0; i < 8; ++i) m.present[j][tslot(v0 + i)] = static_cast<uint8_t>((alph >> i) & 1u);
    }
    __syncthreads();
    bpd_plan(m);
    uint8_t* out = a.out + (off_s - a.base);
    const uint64_t u0 = (poff + off_s) / 8;  // image index of the slot's first 64-bit word
    if (m.len == kPage) {
      // stored as is: this thread's 256 bytes, transposed back (the byte
      // transpose is its own inverse; the staging buffer already holds the
      // next slot)
      uint4* dst = reinterpret_cast<uint4*>(out + 256ull * tid);
      const uint64_t craw = (u0 + 32ull * tid) * kPhi;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        uint4 c0, c1;
        transpose4(P[0][k], P[1][k], P[2][k], P[3][k], c0.x, c0.z, c1.x, c1.z);
        transpose4(P[4][k], P[5][k], P[6][k], P[7][k], c0.y, c0.w, c1.y, c1.w);
        dst[2 * k] = c0;
        dst[2 * k + 1] = c1;
        const uint64_t c = craw + (4 * k) * kPhi;  // index terms of words u0 + 32 tid + 4k + i
        h += dev::mix(pair64(c0.x, c0.y) ^ c) + dev::mix(pair64(c0.z, c0.w) ^ (c + kPhi)) +
             dev::mix(pair64(c1.x, c1.y) ^ (c + 2 * kPhi)) + dev::mix(pair64(c1.z, c1.w) ^ (c + 3 * kPhi));
      }
    } else {
      if (tid < 16)
        out[tid] = tid < 8 ? static_cast<uint8_t>(m.b[tid])
                           : static_cast<uint8_t>(m.b[tid - 8] == 8 ? 255u : m.k[tid - 8] - 1u);
      if (tid == 0) {
        uint64_t w0 = 0, w1 = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          w0 |= static_cast<uint64_t>(m.b[j] & 255u) << (8 * j);
          w1 |= static_cast<uint64_t>((m.b[j] == 8 ? 255u : m.k[j] - 1u) & 255u) << (8 * j);
        }
        h += hash_word(w0, u0) + hash_word(w1, u0 + 1);
      }
#pragma unroll 1
      for (int j = 0; j < 8; ++j) {
        const uint32_t b = m.b[j];
        uint8_t* sec = out + m.sec[j];
        uint32_t pw[8];  // this plane's words (a switch keeps P's indices static)
        switch (j) {
          case 0: plane_words(P[0], pw); break;
          case 1: plane_words(P[1], pw); break;
          case 2: plane_words(P[2], pw); break;
          case 3: plane_words(P[3], pw); break;
          case 4: plane_words(P[4], pw); break;
          case 5: plane_words(P[5], pw); break;
          case 6: plane_words(P[6], pw); break;
          default: plane_words(P[7], pw); break;
        }
        if (b == 8) {
          // the plane as is: this thread's 32 bytes of it
          uint4* dst = reinterpret_cast<uint4*>(sec + 32 * tid);
          dst[0] = make_uint4(pw[0], pw[1], pw[2], pw[3]);
          dst[1] = make_uint4(pw[4], pw[5], pw[6], pw[7]);
          const uint64_t c = (u0 + m.sec[j] / 8 + 4ull * tid) * kPhi;
          h += dev::mix(pair64(pw[0], pw[1]) ^ c) + dev::mix(pair64(pw[2], pw[3]) ^ (c + kPhi)) +
               dev::mix(pair64(pw[4], pw[5]) ^ (c + 2 * kPhi)) + dev::mix(pair64(pw[6], pw[7]) ^ (c + 3 * kPhi));
          continue;
        }
        const uint32_t k = m.k[j], dpad = (k + 15u) & ~15u;
        uint8_t* dict = reinterpret_cast<uint8_t*>(dict_sm[j]);
        if (m.present[j][tslot(tid)]) dict[m.rank[j][tslot(tid)]] = static_cast<uint8_t>(tid);
        for (uint32_t i = k + tid; i < dpad; i += blockDim.x) dict[i] = 0;
        if (b == 0) continue;
        uint32_t* words = reinterpret_cast<uint32_t*>(sec + dpad) + tid * b;
        const uint64_t uw = u0 + (m.sec[j] + dpad) / 8;
        switch (b) {
          case 1: h += pack_ranks<1>(pw, m.rank[j], words, uw); break;
          case 2: h += pack_ranks<2>(pw, m.rank[j], words, uw); break;
          case 3: h += pack_ranks<3>(pw, m.rank[j], words, uw); break;
          case 4: h += pack_ranks<4>(pw, m.rank[j], words, uw); break;
          case 5: h += pack_ranks<5>(pw, m.rank[j], words, uw); break;
          case 6: h += pack_ranks<6>(pw, m.rank[j], words, uw); break;
          default: h += pack_ranks<7>(pw, m.rank[j], words, uw); break;
        }
      }
    }
    __syncthreads();  // the tables are read until here; the dictionaries are complete
    if (m.len != kPage && tid < 128) {
      // the dictionaries (at most 128 bytes a plane): one 64-bit word a thread
      const int j = tid >> 4, q = tid & 15;
      if (m.b[j] != 8 && 8u * q < ((m.k[j] + 15u) & ~15u)) {
        const uint64_t w = dict_sm[j][q];
        *reinterpret_cast<uint64_t*>(out + m.sec[j] + 8 * q) = w;
        h += hash_word(w, u0 + m.sec[j] / 8 + q);
      }
    }
  }
  h = dev::warp_sum(h);
  if ((tid & 31) == 0 && h != 0) atomicAdd(a.trailer, static_cast<unsigned long long>(h));
}

}  // namespace

KernelSpec bpd_size_spec(uint64_t max_slots) {
  return KernelSpec{reinterpret_cast<const void*>(k_bpd_size),
                    grid_for(k_bpd_size, std::max<uint64_t>(max_slots, 1), 1, kBpdThreads), kBpdThreads, 0};
}

KernelSpec bpd_scan_spec() { return KernelSpec{reinterpret_cast<const void*>(k_bpd_scan), 1, 1024, 0}; }

cudaError_t bpd_encode_spec(uint64_t max_slots, KernelSpec* out) {
  const cudaError_t e = allow_big_smem(k_bpd_encode, kEncDynSmem);
  if (e != cudaSuccess) return e;
  const uint64_t cap = static_cast<uint64_t>(resident_per_sm(reinterpret_cast<const void*>(k_bpd_encode),
                                                             kBpdThreads, kEncDynSmem)) * num_sms();
  const unsigned grid = static_cast<unsigned>(std::max<uint64_t>(1, std::min(std::max<uint64_t>(max_slots, 1), cap)));
  *out = KernelSpec{reinterpret_cast<const void*>(k_bpd_encode), grid, kBpdThreads, kEncDynSmem};
  return cudaSuccess;
}

cudaError_t launch_bpd_size(const BpdSizeArgs& a, uint64_t max_slots, cudaStream_t st) {
  if (max_slots == 0) return cudaSuccess;
  BpdSizeArgs copy = a;
  return launch_spec(bpd_size_spec(max_slots), &copy, st);
}

cudaError_t launch_bpd_scan(const BpdScanArgs& a, cudaStream_t st) {
  BpdScanArgs copy = a;
  return launch_spec(bpd_scan_spec(), &copy, st);
}

cudaError_t launch_bpd_encode(const BpdEncodeArgs& a, uint64_t max_slots, cudaStream_t st) {
  if (max_slots == 0) return cudaSuccess;
  KernelSpec sp;
  const cudaError_t e = bpd_encode_spec(max_slots, &sp);
  if (e != cudaSuccess) return e;
  BpdEncodeArgs copy = a;
  return launch_spec(sp, &copy, st);
}

}  // namespace crum
