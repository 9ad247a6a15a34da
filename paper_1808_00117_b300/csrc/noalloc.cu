// crum_dirty_pages_static: dirty-page detection for one allocation that
// allocates no memory at all.
//
// Who needs it: callers that cannot call cudaMalloc at the moment they want
// to know which pages changed.  Typical cases are an out-of-memory handler
// that wants a last checkpoint before it frees anything (cudaMalloc is
// exactly what fails there), and allocator hooks or CUDA-call interposers
// (the kind of layer CRUM itself is built from) where a nested cudaMalloc
// would re-enter the allocator that is being served.  Everything else in
// this library draws its scratch from a registration set it allocated
// earlier; this entry point instead keeps its scratch, the dirty bitmap, in
// a fixed file-scope device array.
//
// The bitmap holds one bit per page for at most kStaticMaxPages pages
// (4,194,304 pages = 256 GiB of 64 KiB pages), i.e. 512 KiB of device
// memory that every GPU which loads this library keeps until the process
// exits.  All calls on a device share it: calls that overlap on the GPU
// (different streams, no ordering between them) race on it and give wrong
// answers; calls ordered on one stream are fine.  Each call clears the part
// it uses before using it, so nothing depends on what the previous call left.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "crum.h"
#include "device.cuh"
#include "kernels.h"

namespace crum {
void set_last_error(const char* msg);
namespace {

constexpr uint64_t kStaticMaxPages = 1ull << 22;
constexpr uint64_t kStaticWords = kStaticMaxPages / 32;

// The scratch.  In host code this name is only a stand-in for the device
// array; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) uint32_t g_static_dirty_bits[kStaticWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_bits_addr[kMaxDevices] = {};

// Ascending list of the set bits of the bitmap (one CTA): thread t owns a
// contiguous run of words; an exclusive scan of the per-thread popcounts
// gives each thread its first output slot.
constexpr int kEmitThreads = 1024;

__global__ void __launch_bounds__(kEmitThreads)
k_emit_dirty_pages(const uint32_t* bits, uint64_t n_words, uint32_t* pages_out,
                   uint64_t* count_out) {
  __shared__ uint32_t wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t per = (n_words + kEmitThreads - 1) / kEmitThreads;
  const uint64_t w0 = min(static_cast<uint64_t>(tid) * per, n_words);
  const uint64_t w1 = min(w0 + per, n_words);
  uint32_t cnt = 0;
  for (uint64_t w = w0; w < w1; ++w) cnt += __popc(bits[w]);
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t x = wsum[lane];
    uint32_t s = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    wsum[lane] = s - x;
  }
  __syncthreads();
  uint32_t slot = wsum[warp] + incl - cnt;
  for (uint64_t w = w0; w < w1; ++w) {
    uint32_t m = bits[w];
    while (m != 0) {
      const int b = __ffs(m) - 1;
      pages_out[slot++] = static_cast<uint32_t>(w * 32 + b);
      m &= m - 1;
    }
  }
  if (tid == kEmitThreads - 1) *count_out = slot;
}

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
cudaError_t static_bits(int device, uint32_t** out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_bits_addr[device] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_dirty_bits);
    if (e != cudaSuccess) return e;
    g_bits_addr[device] = static_cast<uint32_t*>(p);
  }
  *out = g_bits_addr[device];
  return cudaSuccess;
}

}  // namespace
}  // namespace crum

extern "C" crum_status crum_dirty_pages_static(const void* ptr, uint64_t bytes, uint64_t* hashes,
                                               int full, uint32_t* pages_out, uint64_t* count_out,
                                               crum_stream_t stream) {
  crum::set_last_error("");
  if (ptr == nullptr || hashes == nullptr || pages_out == nullptr || count_out == nullptr ||
      bytes == 0) {
    crum::set_last_error("crum_dirty_pages_static: null pointer or zero size");
    return CRUM_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0) {
    crum::set_last_error("crum_dirty_pages_static: pointer not 16-byte aligned");
    return CRUM_EINVAL;
  }
  // compared in bytes before any rounding: near 2^64 the page count of
  // `bytes` would wrap to a small number
  if (bytes > crum::kStaticMaxPages * crum::kPage) {
    crum::set_last_error(
        "crum_dirty_pages_static: more pages than the static scratch holds "
        "(CRUM_STATIC_MAX_PAGES = 4194304, 256 GiB)");
    return CRUM_EINVAL;
  }
  const uint64_t n_pages = (bytes + crum::kPage - 1) / crum::kPage;
  int device = -1;
  uint32_t* bits = nullptr;
  if (cudaGetDevice(&device) != cudaSuccess || crum::static_bits(device, &bits) != cudaSuccess) {
    crum::set_last_error("crum_dirty_pages_static: cannot locate the static scratch on this device");
    return CRUM_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t n_words = (n_pages + 31) / 32;
  if (cudaMemsetAsync(bits, 0, n_words * sizeof(uint32_t), st) != cudaSuccess) {
    crum::set_last_error("crum_dirty_pages_static: clearing the scratch failed");
    return CRUM_ECUDA;
  }
  crum::HashArgs ha{};
  ha.allocs = nullptr;
  ha.one = crum::DevAlloc{static_cast<uint8_t*>(const_cast<void*>(ptr)), bytes, 0, 0,
                          static_cast<uint32_t>(n_pages)};
  ha.n_allocs = 1;
  ha.n_pages = n_pages;
  ha.h_table = hashes;
  ha.dirty_mask = bits;
  ha.full = full != 0;
  if (crum::launch_hash_dirty(ha, 1, false, st) != cudaSuccess) {
    crum::set_last_error("crum_dirty_pages_static: hash launch failed");
    return CRUM_ECUDA;
  }
  // launched through cudaLaunchKernel so that its own return value is the
  // launch's status (cudaGetLastError would also report, and clear, an
  // earlier unrelated error of the caller's)
  const uint32_t* bits_arg = bits;
  void* args[] = {&bits_arg, const_cast<uint64_t*>(&n_words), &pages_out, &count_out};
  if (cudaLaunchKernel(reinterpret_cast<const void*>(crum::k_emit_dirty_pages), dim3(1),
                       dim3(crum::kEmitThreads), args, 0, st) != cudaSuccess) {
    crum::set_last_error("crum_dirty_pages_static: list launch failed");
    return CRUM_ECUDA;
  }
  crum::g_kernel_launches.fetch_add(1, std::memory_order_relaxed);
  return CRUM_OK;
}
