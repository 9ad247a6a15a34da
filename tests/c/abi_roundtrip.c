/* The C ABI used from C alone (no Python): register two device buffers,
 * take a full and an incremental checkpoint, check the incremental image's
 * version and page table against the pages this program changed, scribble,
 * restore the chain, and compare every byte; once with plain and once with
 * compressed images.  Prints "ok" and exits 0 on success.  Built and run by
 * tests/test_c_abi.py. */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "crum.h"

#define CHECK(x)                                                               \
  do {                                                                         \
    crum_status st_ = (x);                                                     \
    if (st_ != CRUM_OK) {                                                      \
      fprintf(stderr, "%s: %d %s\n", #x, (int)st_, crum_last_error());        \
      return 1;                                                                \
    }                                                                          \
  } while (0)
#define CUDA(x)                                                                \
  do {                                                                         \
    cudaError_t e_ = (x);                                                      \
    if (e_ != cudaSuccess) {                                                   \
      fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));                 \
      return 1;                                                                \
    }                                                                          \
  } while (0)

static const size_t kSizes[2] = {5 * CRUM_PAGE_SIZE + 40, 3 * CRUM_PAGE_SIZE};

static int round_trip(int compress) {
  uint8_t *dev[2], *host[2], *back[2];
  for (int i = 0; i < 2; ++i) {
    CUDA(cudaMalloc((void **)&dev[i], kSizes[i]));
    host[i] = (uint8_t *)malloc(kSizes[i]);
    back[i] = (uint8_t *)malloc(kSizes[i]);
    for (size_t b = 0; b < kSizes[i]; ++b) host[i][b] = (uint8_t)(b * 131u + i * 7u + (b >> 9));
    CUDA(cudaMemcpy(dev[i], host[i], kSizes[i], cudaMemcpyHostToDevice));
  }
  crum_config cfg;
  crum_config_default(&cfg);
  cfg.compress = compress;
  crum_set *set = NULL;
  CHECK(crum_set_create(&cfg, &set));
  uint32_t ids[2];
  for (int i = 0; i < 2; ++i) CHECK(crum_register(set, dev[i], kSizes[i], &ids[i]));
  cudaStream_t stream;
  CUDA(cudaStreamCreate(&stream));

  crum_image *full = NULL, *incr = NULL;
  CHECK(crum_checkpoint(set, stream, CRUM_FULL, &full));
  CHECK(crum_image_wait(full, CRUM_WAIT_PERSISTED, -1));

  /* change page 1 of buffer 0 and the tail page of buffer 0 */
  host[0][1 * CRUM_PAGE_SIZE + 3] ^= 0x5a;
  host[0][5 * CRUM_PAGE_SIZE + 39] ^= 0x01;
  for (int i = 0; i < 2; ++i) CUDA(cudaMemcpy(dev[i], host[i], kSizes[i], cudaMemcpyHostToDevice));
  CHECK(crum_checkpoint(set, stream, CRUM_INCR, &incr));
  CHECK(crum_image_wait(incr, CRUM_WAIT_PERSISTED, -1));
  crum_image_info info;
  CHECK(crum_image_info_get(incr, &info));
  if (info.n_dirty != 2 || info.full != 0 || info.parent_seq != 0) {
    fprintf(stderr, "unexpected incremental: n_dirty %llu full %u parent %llu\n",
            (unsigned long long)info.n_dirty, info.full, (unsigned long long)info.parent_seq);
    return 1;
  }
  uint8_t *img = (uint8_t *)malloc(info.image_bytes);
  CHECK(crum_image_copy(incr, img, info.image_bytes));
  uint32_t version;
  memcpy(&version, img + 8, 4);
  if (version != (compress ? 2u : 1u)) {
    fprintf(stderr, "image version %u with compress=%d\n", version, compress);
    return 1;
  }
  const uint32_t *ptab = (const uint32_t *)(img + 64 + 16 * 2);
  if (ptab[0] != 0 || ptab[1] != 1 || ptab[2] != 0 || ptab[3] != 5) {
    fprintf(stderr, "unexpected page table %u:%u %u:%u\n", ptab[0], ptab[1], ptab[2], ptab[3]);
    return 1;
  }

  for (int i = 0; i < 2; ++i) CUDA(cudaMemset(dev[i], 0xee, kSizes[i]));
  CHECK(crum_restore(set, incr, stream));
  CUDA(cudaStreamSynchronize(stream));
  for (int i = 0; i < 2; ++i) {
    CUDA(cudaMemcpy(back[i], dev[i], kSizes[i], cudaMemcpyDeviceToHost));
    if (memcmp(back[i], host[i], kSizes[i]) != 0) {
      fprintf(stderr, "buffer %d differs after restore\n", i);
      return 1;
    }
  }
  CHECK(crum_image_release(incr));
  CHECK(crum_image_release(full));
  CHECK(crum_set_destroy(set));
  for (int i = 0; i < 2; ++i) {
    cudaFree(dev[i]);
    free(host[i]);
    free(back[i]);
  }
  free(img);
  CUDA(cudaStreamDestroy(stream));
  return 0;
}

int main(void) {
  for (int compress = 0; compress < 2; ++compress)
    if (round_trip(compress) != 0) return 1;
  printf("ok\n");
  return 0;
}
