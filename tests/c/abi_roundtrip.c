/* The C ABI used from C alone (no Python): register two device buffers,
 * take a full and an incremental checkpoint, check the incremental image's
 * version and page table against the pages this program changed, scribble,
 * restore the chain, and compare every byte; once with plain and once with
 * compressed images; then the same through the request server.  Prints "ok"
 * and exits 0 on success.  Built and run by tests/test_c_abi.py. */
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

/* The request server from C: one client (a set with external staging) on a
 * server that keeps request images and admits size-first; a full and an
 * incremental checkpoint request, the incremental's image taken from the
 * server and its page table checked, then a restore request onto scribbled
 * memory compared byte for byte. */
static int server_round_trip(void) {
  const size_t n = 4 * CRUM_PAGE_SIZE + 4096;
  uint8_t *dev, *host = (uint8_t *)malloc(n), *back = (uint8_t *)malloc(n);
  for (size_t b = 0; b < n; ++b) host[b] = (uint8_t)(b * 29u + (b >> 11));
  CUDA(cudaMalloc((void **)&dev, n));
  CUDA(cudaMemcpy(dev, host, n, cudaMemcpyHostToDevice));
  crum_config cfg;
  crum_config_default(&cfg);
  cfg.external_staging = 1;
  crum_set *set = NULL;
  CHECK(crum_set_create(&cfg, &set));
  uint32_t id;
  CHECK(crum_register(set, dev, n, &id));
  cudaStream_t stream;
  CUDA(cudaStreamCreate(&stream));
  crum_server_config sc;
  memset(&sc, 0, sizeof sc);
  sc.staging_budget = 64ull << 20;
  sc.max_inflight = 2;
  sc.order = 1;
  sc.keep_images = 1;
  crum_server *srv = NULL;
  CHECK(crum_server_create(&sc, &srv));
  uint32_t client;
  CHECK(crum_server_add_client(srv, set, stream, &client));
  uint64_t r0, r1, r2;
  crum_request_info ri;
  CHECK(crum_server_submit(srv, client, CRUM_REQ_CHECKPOINT_FULL, &r0));
  CHECK(crum_server_wait(srv, r0, CRUM_WAIT_PERSISTED, -1, &ri));
  host[2 * CRUM_PAGE_SIZE + 5] ^= 0x33; /* page 2 changes */
  CUDA(cudaMemcpy(dev, host, n, cudaMemcpyHostToDevice));
  CHECK(crum_server_submit(srv, client, CRUM_REQ_CHECKPOINT, &r1));
  CHECK(crum_server_wait(srv, r1, CRUM_WAIT_PERSISTED, -1, &ri));
  if (ri.n_dirty != 1 || !ri.done) {
    fprintf(stderr, "server checkpoint: n_dirty %llu done %d\n", (unsigned long long)ri.n_dirty, ri.done);
    return 1;
  }
  crum_image *img = NULL;
  CHECK(crum_server_take_image(srv, r1, &img));
  crum_image_info info;
  CHECK(crum_image_info_get(img, &info));
  uint8_t *bytes = (uint8_t *)malloc(info.image_bytes);
  CHECK(crum_image_copy(img, bytes, info.image_bytes));
  const uint32_t *ptab = (const uint32_t *)(bytes + 64 + 16);
  if (info.n_dirty != 1 || ptab[0] != 0 || ptab[1] != 2 || info.checksum != ri.checksum) {
    fprintf(stderr, "server image: n_dirty %llu page %u:%u\n", (unsigned long long)info.n_dirty,
            ptab[0], ptab[1]);
    return 1;
  }
  if (crum_server_take_image(srv, r1, &img) != CRUM_EINVAL) {
    fprintf(stderr, "a second take of the same image was not refused\n");
    return 1;
  }
  CUDA(cudaMemset(dev, 0x11, n));
  CUDA(cudaDeviceSynchronize());
  CHECK(crum_server_submit(srv, client, CRUM_REQ_RESTORE, &r2));
  CHECK(crum_server_wait(srv, r2, CRUM_WAIT_PERSISTED, -1, &ri));
  CUDA(cudaStreamSynchronize(stream));
  CUDA(cudaMemcpy(back, dev, n, cudaMemcpyDeviceToHost));
  if (memcmp(back, host, n) != 0) {
    fprintf(stderr, "server restore differs\n");
    return 1;
  }
  crum_server_stats stats;
  CHECK(crum_server_drain(srv, &stats));
  if (stats.completed != 3 || stats.failed != 0) {
    fprintf(stderr, "server stats: completed %llu failed %llu\n", (unsigned long long)stats.completed,
            (unsigned long long)stats.failed);
    return 1;
  }
  CHECK(crum_image_release(img));
  CHECK(crum_server_destroy(srv));
  CHECK(crum_set_destroy(set));
  CUDA(cudaStreamDestroy(stream));
  cudaFree(dev);
  free(host);
  free(back);
  free(bytes);
  return 0;
}

int main(void) {
  for (int compress = 0; compress < 2; ++compress)
    if (round_trip(compress) != 0) return 1;
  if (server_round_trip() != 0) return 1;
  printf("ok\n");
  return 0;
}
