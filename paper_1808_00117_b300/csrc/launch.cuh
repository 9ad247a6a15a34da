// Grid sizing shared by the kernel files (internal).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "kernels.h"

namespace crum {

// SMs of the current device (cached).
int num_sms();
// CTAs of `func` resident per SM at once (cached per device and shape).
int resident_per_sm(const void* func, int threads, size_t smem);

template <typename K>
int resident_ctas(K kernel, int threads) {
  return resident_per_sm(reinterpret_cast<const void*>(kernel), threads, 0) * num_sms();
}

// Grid for `units` groups of a kernel with `groups_per_cta` groups per CTA:
// enough CTAs for every unit, at most what is resident at once.
template <typename K>
unsigned grid_for(K kernel, uint64_t units, int groups_per_cta, int threads = 256) {
  const uint64_t need = (units + groups_per_cta - 1) / groups_per_cta;
  const uint64_t cap = static_cast<uint64_t>(resident_ctas(kernel, threads));
  return static_cast<unsigned>(std::max<uint64_t>(1, std::min(need, cap)));
}

}  // namespace crum
