// Registration sets, checkpoint orchestration, images, drain/writer threads
// and the extern "C" entry points declared in include/crum.h.
#include <fcntl.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <cerrno>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>

#include "engine.h"
#include "codec.cuh"
#include "kernels.h"

using crum::Alloc;
using crum::DevAlloc;
using crum::Half;
using crum::kHeaderBytes;
using crum::kPage;

namespace {

thread_local std::string t_err;

crum_status fail(crum_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return st;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(CRUM_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                \
  } while (0)

// Makes `dev` current for the scope, restoring the caller's device after.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

constexpr uint64_t kDefaultStaging = 1ull << 30;
constexpr uint64_t kDefaultChunk = 64ull << 20;
constexpr int64_t kBackgroundLimitNs = 600ll * 1000 * 1000 * 1000;  // 10 min

uint64_t pages_of(uint64_t bytes) { return (bytes + kPage - 1) / kPage; }
uint64_t meta_bytes(uint64_t A, uint64_t n) { return kHeaderBytes + 16 * A + 16 * n; }
uint64_t image_size(uint64_t A, uint64_t n) { return meta_bytes(A, n) + n * kPage + 8; }
// compressed form: tables with the slot offsets, padded to 16 bytes
uint64_t cmeta_bytes(uint64_t A, uint64_t n) { return (kHeaderBytes + 16 * A + 24 * n + 15) & ~15ull; }
uint64_t payload_offset(const crum_image* img) {
  return img->compressed ? img->payload_off : meta_bytes(img->n_allocs, img->n_dirty);
}

std::atomic<uint32_t> g_set_ids{0};

// Poll an event until it completes or `limit_ns` passes.
crum_status wait_event(cudaEvent_t ev, int64_t limit_ns) {
  const auto t0 = std::chrono::steady_clock::now();
  int spins = 0;
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return CRUM_OK;
    if (e != cudaErrorNotReady)
      return fail(CRUM_ECUDA, "event wait failed: %s", cudaGetErrorString(e));
    if (limit_ns >= 0 &&
        std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now() - t0)
                .count() > limit_ns)
      return fail(CRUM_ETIMEOUT, "timed out waiting for the device");
    if (++spins > 64) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

void image_set_stage(crum_image* img, int stage, crum_status st, const std::string& err) {
  std::lock_guard<std::mutex> lk(img->mu);
  if (st != CRUM_OK && (img->status == CRUM_OK || img->status == CRUM_ECOLLISION)) {
    img->status = st;
    img->err = err;
  }
  if (stage > img->stage) img->stage = stage;
  img->cv.notify_all();
}

void image_unref(crum_image* img) {
  while (img != nullptr) {
    if (img->refs.fetch_sub(1) != 1) return;
    crum_image* parent = img->parent;
    if (img->host != nullptr && img->pool) img->pool->free(img->host, img->host_len);
    if (img->ev_submit) cudaEventDestroy(img->ev_submit);
    if (img->ev_captured) cudaEventDestroy(img->ev_captured);
    if (img->ev_drained) cudaEventDestroy(img->ev_drained);
    for (cudaEvent_t ev : {img->ev_k0, img->ev_k1, img->ev_k2, img->ev_d0, img->ev_e1})
      if (ev) cudaEventDestroy(ev);
    delete img;
    img = parent;
  }
}

void image_ref(crum_image* img) {
  if (img) img->refs.fetch_add(1);
}

// Quiesce: every queued drain is enqueued and the set's streams are idle.
// Caller holds s->mu via lk.
crum_status quiesce(crum_set* s, std::unique_lock<std::mutex>& lk) {
  const bool ok = s->cv.wait_for(lk, std::chrono::seconds(600), [&] {
    return s->half[0].drain_enqueued && s->half[1].drain_enqueued;
  });
  if (!ok) return fail(CRUM_ETIMEOUT, "timed out waiting for pending drains");
  CK(cudaStreamSynchronize(s->cap_stream));
  CK(cudaStreamSynchronize(s->drain_stream));
  return CRUM_OK;
}

template <typename T>
crum_status grow_device(T** p, size_t* cap, size_t need, bool keep) {
  if (need <= *cap) return CRUM_OK;
  size_t n = std::max(need, *cap + *cap / 2);
  T* q = nullptr;
  CK(cudaMalloc(&q, n * sizeof(T)));
  if (keep && *p != nullptr && *cap > 0) CK(cudaMemcpy(q, *p, *cap * sizeof(T), cudaMemcpyDeviceToDevice));
  if (*p != nullptr) CK(cudaFree(*p));
  *p = q;
  *cap = n;
  return CRUM_OK;
}

// Device buffers sized for the current registrations.  Caller holds the
// lock and has made sure nothing in flight uses the buffers it may move.
crum_status ensure_capacity(crum_set* s, std::unique_lock<std::mutex>& lk) {
  const size_t A = s->allocs.size();
  const uint64_t words = (s->n_pages + 31) / 32;
  // room for the compressed form's tables, and for a replayed chunk of a
  // compressed image (page table, hashes and offsets of a half's slots)
  const size_t meta_need = cmeta_bytes(A, std::max<uint64_t>(s->n_pages, s->half_slots));
  const bool grow = A > s->alloc_cap || s->n_pages > s->h_cap || words + 1 > s->words_cap ||
                    meta_need > s->half[0].meta_cap || meta_need > s->half[1].meta_cap ||
                    (s->cfg.verify && s->n_pages > s->shadow_cap);
  if (!grow) return CRUM_OK;
  crum_status st = quiesce(s, lk);
  if (st != CRUM_OK) return st;
  size_t cap_a = s->alloc_cap;
  st = grow_device(&s->d_allocs, &cap_a, std::max<size_t>(A, 16), false);
  if (st != CRUM_OK) return st;
  size_t cap_f = s->alloc_cap;
  st = grow_device(&s->d_first_page, &cap_f, std::max<size_t>(A, 16), false);
  if (st != CRUM_OK) return st;
  s->alloc_cap = std::min(cap_a, cap_f);
  st = grow_device(&s->d_h, &s->h_cap, s->n_pages, true);
  if (st != CRUM_OK) return st;
  size_t wc = s->words_cap;
  st = grow_device(&s->d_mask, &wc, words + 1, false);
  if (st != CRUM_OK) return st;
  wc = s->words_cap;
  st = grow_device(&s->d_word_offset, &wc, words + 1, false);
  if (st != CRUM_OK) return st;
  s->words_cap = wc;
  for (Half& H : s->half) {
    st = grow_device(&H.meta, &H.meta_cap, meta_need, false);
    if (st != CRUM_OK) return st;
  }
  if (s->cfg.verify && s->n_pages > s->shadow_cap) {
    if (s->d_shadow) CK(cudaFree(s->d_shadow));
    s->d_shadow = nullptr;
    CK(cudaMalloc(&s->d_shadow, s->n_pages * kPage));
    s->shadow_cap = s->n_pages;
    s->needs_full = true;  // the shadow starts empty
  }
  s->table_dirty = true;
  s->graph_epoch++;
  return CRUM_OK;
}

crum_status upload_table(crum_set* s) {
  if (!s->table_dirty) return CRUM_OK;
  std::vector<DevAlloc> t(s->allocs.size());
  std::vector<uint64_t> f(s->allocs.size());
  for (size_t i = 0; i < s->allocs.size(); ++i) {
    const Alloc& a = s->allocs[i];
    t[i] = DevAlloc{a.ptr, a.bytes, a.first_page, a.id, static_cast<uint32_t>(a.n_pages)};
    f[i] = a.first_page;
  }
  // pageable source: the runtime stages it before returning, so the vectors
  // may go out of scope; the copy stays ordered on the capture stream
  CK(cudaMemcpyAsync(s->d_allocs, t.data(), t.size() * sizeof(DevAlloc), cudaMemcpyHostToDevice,
                     s->cap_stream));
  CK(cudaMemcpyAsync(s->d_first_page, f.data(), f.size() * sizeof(uint64_t),
                     cudaMemcpyHostToDevice, s->cap_stream));
  s->table_dirty = false;
  return CRUM_OK;
}

// Queues the device->host copy of `bytes` of payload on the drain stream, as
// copies of at most cfg.chunk_bytes each: into the image's own buffer at
// host_off, or, when the image keeps no payload, each into the set's bounce
// region (cfg.chunk_bytes of pinned memory), so that a footprint larger than
// host memory can still be drained and timed.
crum_status drain_payload(crum_set* s, crum_image* img, uint64_t host_off, const uint8_t* src,
                          uint64_t bytes) {
  const uint64_t chunk = s->cfg.chunk_bytes;
  if (!img->drop_payload) {
    for (uint64_t off = 0; off < bytes; off += chunk)
      CK(cudaMemcpyAsync(img->host + host_off + off, src + off, std::min(chunk, bytes - off),
                         cudaMemcpyDeviceToHost, s->drain_stream));
    return CRUM_OK;
  }
  {
    std::lock_guard<std::mutex> lk(s->bounce_mu);
    if (s->bounce == nullptr) s->bounce = s->pool->alloc(chunk);
    if (s->bounce == nullptr) return fail(CRUM_ENOMEM, "pinned host pool exhausted (bounce region)");
  }
  for (uint64_t off = 0; off < bytes; off += chunk)
    CK(cudaMemcpyAsync(s->bounce, src + off, std::min(chunk, bytes - off), cudaMemcpyDeviceToHost,
                       s->drain_stream));
  return CRUM_OK;
}

uint8_t* trailer_dst(crum_image* img) { return img->host + img->host_len - 8; }

// Queue the device->host copies of a captured image from half H into its
// pinned host buffer, on the drain stream.
crum_status enqueue_drain(crum_set* s, crum_image* img, Half& H) {
  const uint64_t n = img->n_dirty;
  CK(cudaStreamWaitEvent(s->drain_stream, img->compressed ? H.ev_encoded : img->ev_captured, 0));
  if (img->ticket >= 0 && s->sequencer) {
    crum::DrainSequencer* q = s->sequencer.get();
    std::lock_guard<std::mutex> lk(q->mu);
    if (q->tail_recorded) CK(cudaStreamWaitEvent(s->drain_stream, q->tail, 0));
  }
  CK(cudaEventRecord(img->ev_d0, s->drain_stream));
  CK(cudaMemcpyAsync(img->host, H.meta, payload_offset(img), cudaMemcpyDeviceToHost, s->drain_stream));
  // the null sink drains too (the bytes cross the link); the writer drops them
  const uint64_t payload = img->compressed ? img->payload_bytes : n * kPage;
  if (payload > 0) {
    const crum_status st =
        drain_payload(s, img, payload_offset(img), img->compressed ? H.cpay : H.payload, payload);
    if (st != CRUM_OK) return st;
  }
  CK(cudaMemcpyAsync(trailer_dst(img), H.scalars + 1, 8, cudaMemcpyDeviceToHost, s->drain_stream));
  CK(cudaEventRecord(img->ev_drained, s->drain_stream));
  CK(cudaEventRecord(H.ev_drained, s->drain_stream));
  return CRUM_OK;
}

crum_status alloc_image_host(crum_set* s, crum_image* img) {
  img->image_bytes = img->compressed ? img->payload_off + img->payload_bytes + 8
                                     : image_size(img->n_allocs, img->n_dirty);
  img->host_len = img->image_bytes;
  if (img->drop_payload) img->host_len = payload_offset(img) + 8;
  img->host = s->pool->alloc(img->host_len);
  if (img->host == nullptr) return fail(CRUM_ENOMEM, "pinned host pool exhausted (%zu bytes)", img->host_len);
  return CRUM_OK;
}

// Waits (host) until it is this image's turn to queue its drain.
crum_status sequencer_turn(crum::DrainSequencer* q, crum_image* img) {
  std::unique_lock<std::mutex> lk(q->mu);
  const bool ok = q->cv.wait_for(lk, std::chrono::seconds(600), [&] {
    return q->next == static_cast<uint64_t>(img->ticket);
  });
  return ok ? CRUM_OK : fail(CRUM_ETIMEOUT, "timed out waiting for the drain order");
}

// Marks the image's drain queued (or skipped): later drains wait for it.
void sequencer_done(crum::DrainSequencer* q, crum_image* img, cudaStream_t drain, bool queued) {
  std::lock_guard<std::mutex> lk(q->mu);
  (void)img;
  if (queued) {
    if (q->tail == nullptr) cudaEventCreateWithFlags(&q->tail, cudaEventDisableTiming);
    if (q->tail != nullptr && cudaEventRecord(q->tail, drain) == cudaSuccess) q->tail_recorded = true;
  }
  q->next++;
  q->cv.notify_all();
}

void planner_main(crum_set* s) {
  DeviceGuard dg(s->device);
  crum::trace_name_thread("crum planner");
  for (;;) {
    crum_image* img;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->plan_cv.wait(lk, [&] { return s->stop || !s->plan_q.empty(); });
      if (s->plan_q.empty()) return;
      img = s->plan_q.front();
      s->plan_q.pop_front();
    }
    crum::TraceRange tr("crum plan drain");
    Half& H = s->half[img->half];
    crum_status st = wait_event(img->compressed ? H.ev_sized : H.ev_scanned, kBackgroundLimitNs);
    std::string err = st == CRUM_OK ? "" : t_err;
    crum::DrainSequencer* q = img->ticket >= 0 ? s->sequencer.get() : nullptr;
    bool my_turn = false;  // a failed capture still takes (and passes) its turn
    if (q != nullptr) {
      const crum_status t = sequencer_turn(q, img);
      my_turn = t == CRUM_OK;
      if (st == CRUM_OK && !my_turn) {
        st = t;
        err = t_err;
      }
    }
    if (st == CRUM_OK) {
      img->n_dirty = reinterpret_cast<volatile uint64_t*>(H.mailbox)[0];
      img->collisions = reinterpret_cast<volatile uint64_t*>(H.mailbox)[1];
      if (img->compressed) {
        img->payload_bytes = reinterpret_cast<volatile uint64_t*>(H.mailbox)[3];
        img->payload_off = cmeta_bytes(img->n_allocs, img->n_dirty);
      }
      if (reinterpret_cast<volatile uint64_t*>(H.mailbox)[2] != 0)
        st = fail(CRUM_ETIMEOUT, "hash kernel: a bounded device wait ran out");
      if (st == CRUM_OK) st = alloc_image_host(s, img);
      if (st == CRUM_OK) st = enqueue_drain(s, img, H);
      if (st != CRUM_OK) err = t_err;
    }
    if (my_turn) sequencer_done(q, img, s->drain_stream, st == CRUM_OK);
    if (st != CRUM_OK) {
      // keep later users of this half ordered after the capture
      cudaEventRecord(H.ev_drained, s->cap_stream);
      image_set_stage(img, CRUM_WAIT_PERSISTED, st, err);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      H.drain_enqueued = true;
      if (st != CRUM_OK) {
        s->needs_full = true;
        --s->inflight;
      } else {
        s->done_q.push_back(img);
        s->done_cv.notify_one();
      }
      s->cv.notify_all();
    }
    if (st != CRUM_OK) image_unref(img);
  }
}

crum_status write_file(const uint8_t* data, uint64_t n, const char* path, bool do_fsync) {
  const int fd = ::open(path, O_WRONLY | O_CREAT | O_TRUNC, 0644);
  if (fd < 0) return fail(CRUM_EIO, "open %s: %s", path, strerror(errno));
  uint64_t off = 0;
  while (off < n) {
    const size_t want = static_cast<size_t>(std::min<uint64_t>(n - off, 1ull << 30));
    const ssize_t w = ::write(fd, data + off, want);
    if (w <= 0) {
      const int e = errno;
      ::close(fd);
      return fail(CRUM_EIO, "write %s: %s", path, w == 0 ? "short write" : strerror(e));
    }
    off += static_cast<uint64_t>(w);
  }
  if (do_fsync && ::fsync(fd) != 0) {
    const int e = errno;
    ::close(fd);
    return fail(CRUM_EIO, "fsync %s: %s", path, strerror(e));
  }
  if (::close(fd) != 0) return fail(CRUM_EIO, "close %s: %s", path, strerror(errno));
  return CRUM_OK;
}

// Last step of every image: PERSISTED (or the error), and its in-flight
// reference dropped.
void finish_image(crum_set* s, crum_image* img, crum_status st, const std::string& err) {
  img->t_persisted_ms = std::chrono::duration<double, std::milli>(
                            std::chrono::steady_clock::now() - img->t_submit)
                            .count();
  image_set_stage(img, CRUM_WAIT_PERSISTED, st, err);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (st != CRUM_OK) s->needs_full = true;
    --s->inflight;
    s->cv.notify_all();
  }
  image_unref(img);
}

// Drain watcher: marks each image DRAINED as soon as its device->host copies
// are done (in drain order), whatever its sink, then hands images with a
// file to write to the writer and finishes the others.
void drainer_main(crum_set* s) {
  DeviceGuard dg(s->device);
  crum::trace_name_thread("crum drainer");
  for (;;) {
    crum_image* img;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->done_cv.wait(lk, [&] { return s->stop || !s->done_q.empty(); });
      if (s->done_q.empty()) return;
      img = s->done_q.front();
      s->done_q.pop_front();
    }
    crum::TraceRange tr("crum await drain");
    crum_status st = wait_event(img->ev_drained, kBackgroundLimitNs);
    if (st != CRUM_OK) {
      finish_image(s, img, st, t_err);
      continue;
    }
    float ms = 0;
    if (cudaEventElapsedTime(&ms, img->ev_submit, img->ev_captured) == cudaSuccess)
      img->t_captured_ms = ms;
    if (cudaEventElapsedTime(&ms, img->ev_submit, img->ev_drained) == cudaSuccess)
      img->t_drained_ms = ms;
    if (cudaEventElapsedTime(&ms, img->ev_k0, img->ev_k1) == cudaSuccess) img->t_hash_ms = ms;
    if (img->compressed && cudaEventElapsedTime(&ms, img->ev_captured, img->ev_e1) == cudaSuccess)
      img->t_encode_ms = ms;
    if (cudaEventElapsedTime(&ms, img->ev_k2, img->ev_captured) == cudaSuccess)
      img->t_compact_ms = ms;
    if (cudaEventElapsedTime(&ms, img->ev_d0, img->ev_drained) == cudaSuccess)
      img->t_drain_ms = ms;
    std::memcpy(&img->checksum, trailer_dst(img), 8);
    image_set_stage(img, CRUM_WAIT_DRAINED, img->collisions ? CRUM_ECOLLISION : CRUM_OK, "");
    if (img->drop_payload) {
      std::lock_guard<std::mutex> lk(img->mu);
      img->pool->free(img->host, img->host_len);
      img->host = nullptr;
      img->host_len = 0;
    } else if (!img->sink_path.empty()) {
      std::lock_guard<std::mutex> lk(s->mu);
      s->write_q.push_back(img);
      s->write_cv.notify_one();
      continue;
    }
    finish_image(s, img, CRUM_OK, "");
  }
}

// Writer: persists drained images to their files, one at a time, while
// later images keep draining (the forked child's role, Section 3.3).
void writer_main(crum_set* s) {
  crum::trace_name_thread("crum writer");
  for (;;) {
    crum_image* img;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->write_cv.wait(lk, [&] { return s->stop || !s->write_q.empty(); });
      if (s->write_q.empty()) return;
      img = s->write_q.front();
      s->write_q.pop_front();
    }
    crum::TraceRange tr("crum persist");
    const crum_status st = write_file(img->host, img->image_bytes, img->sink_path.c_str(), img->do_fsync);
    finish_image(s, img, st, st == CRUM_OK ? "" : t_err);
  }
}

crum_status new_image_events(crum_image* img) {
  for (cudaEvent_t* ev : {&img->ev_submit, &img->ev_captured, &img->ev_drained, &img->ev_k0,
                          &img->ev_k1, &img->ev_k2, &img->ev_d0, &img->ev_e1})
    CK(cudaEventCreate(ev));
  return CRUM_OK;
}

// Restore of a whole chain in two launches (see k_chain_owner and
// k_restore_merged): every page once, from the newest image holding it.
crum_status restore_merged(crum_set* s, const std::vector<crum::ChainImage>& ci,
                           uint64_t total_slots, bool delta, bool compressed) {
  if (s->owner_cap < s->n_pages) {
    cudaFree(s->d_owner);
    s->d_owner = nullptr;
    s->owner_cap = 0;
    CK(cudaMalloc(&s->d_owner, s->n_pages * sizeof(uint64_t)));
    s->owner_cap = s->n_pages;
  }
  if (s->chain_cap < ci.size()) {
    cudaFree(s->d_chain);
    s->d_chain = nullptr;
    s->chain_cap = 0;
    CK(cudaMalloc(&s->d_chain, ci.size() * sizeof(crum::ChainImage)));
    s->chain_cap = ci.size();
  }
  if (delta && s->cur_cap < s->n_pages) {
    cudaFree(s->d_cur);
    s->d_cur = nullptr;
    s->cur_cap = 0;
    CK(cudaMalloc(&s->d_cur, s->n_pages * sizeof(uint64_t)));
    s->cur_cap = s->n_pages;
  }
  // pageable source: staged by the runtime before the call returns
  CK(cudaMemcpyAsync(s->d_chain, ci.data(), ci.size() * sizeof(crum::ChainImage),
                     cudaMemcpyHostToDevice, s->cap_stream));
  if (delta) {
    // the current contents' page hashes, to leave pages that already match
    crum::HashArgs ha{};
    ha.allocs = s->d_allocs;
    ha.first_page = s->d_first_page;
    ha.n_allocs = static_cast<uint32_t>(s->allocs.size());
    ha.n_pages = s->n_pages;
    ha.h_out = s->d_cur;
    CK(crum::launch_hash_dirty(ha, s->map_hash, false, s->cap_stream));
  }
  CK(cudaMemsetAsync(s->d_owner, 0, s->n_pages * sizeof(uint64_t), s->cap_stream));
  crum::OwnerArgs oa{};
  oa.allocs = s->d_allocs;
  oa.n_allocs = static_cast<uint32_t>(s->allocs.size());
  oa.images = s->d_chain;
  oa.n_images = static_cast<uint32_t>(ci.size());
  oa.total_slots = total_slots;
  oa.owner = s->d_owner;
  CK(crum::launch_chain_owner(oa, s->cap_stream));
  crum::MergedRestoreArgs ma{};
  ma.allocs = s->d_allocs;
  ma.first_page = s->d_first_page;
  ma.n_allocs = oa.n_allocs;
  ma.n_pages = s->n_pages;
  ma.images = s->d_chain;
  ma.owner = s->d_owner;
  ma.h_table = s->d_h;
  ma.current = delta ? s->d_cur : nullptr;
  ma.copied = s->d_copied;
  ma.error = reinterpret_cast<unsigned int*>(s->d_copied + 1);
  CK(crum::launch_restore_merged(ma, compressed, s->cap_stream));
  return CRUM_OK;
}

// Captures in staging-sized chunks when the set has more pages than one
// staging half holds.  The dirty count is read on the host first; each
// chunk is gathered (and, for compressed images, encoded) into one half
// while the other half drains.
crum_status checkpoint_chunked(crum_set* s, crum_image* img, cudaStream_t app,
                               std::unique_lock<std::mutex>& lk, const crum::GatherArgs& base) {
  crum::TraceRange tr("crum chunked capture");
  Half& H0 = s->half[img->half];
  crum_status st = wait_event(H0.ev_scanned, kBackgroundLimitNs);
  if (st != CRUM_OK) return st;
  img->n_dirty = reinterpret_cast<volatile uint64_t*>(H0.mailbox)[0];
  img->collisions = reinterpret_cast<volatile uint64_t*>(H0.mailbox)[1];
  if (reinterpret_cast<volatile uint64_t*>(H0.mailbox)[2] != 0)
    return fail(CRUM_ETIMEOUT, "hash kernel: a bounded device wait ran out");
  const uint64_t n = img->n_dirty, A = img->n_allocs, hs = s->half_slots;
  const bool comp = img->compressed;
  const uint64_t poff = cmeta_bytes(A, n);
  if (comp) {
    // sized for the plain payload until the chunks are encoded, then trimmed
    img->payload_off = poff;
    img->payload_bytes = n * kPage;
    // the compressed checksum is summed afresh (the scan left the plain
    // form's header in it)
    CK(cudaMemsetAsync(H0.scalars + 1, 0, sizeof(uint64_t), s->cap_stream));
  }
  st = alloc_image_host(s, img);
  if (st != CRUM_OK) return st;
  uint64_t* const offs = reinterpret_cast<uint64_t*>(H0.meta + kHeaderBytes + 16 * A + 16 * n);
  uint64_t enc_base = 0;  // encoded bytes of the chunks before this one
  int h = img->half;
  for (uint64_t s0 = 0; s0 < n || s0 == 0; s0 += hs) {
    const uint64_t s1 = std::min(n, s0 + hs);
    Half& H = s->half[h];
    if (&H != &H0) {
      const bool ok = s->cv.wait_for(lk, std::chrono::seconds(600), [&] { return H.drain_enqueued; });
      if (!ok) return fail(CRUM_ETIMEOUT, "timed out waiting for a staging half");
    }
    CK(cudaStreamWaitEvent(s->cap_stream, H.ev_drained, 0));
    crum::GatherArgs g = base;
    g.payload = H.payload;
    g.s_begin = s0;
    g.s_end = s1;
    if (comp) g.trailer = H0.cn + 1;  // the plain form's checksum is not wanted
    CK(crum::launch_gather(g, s1 - s0, s->map_gather, g.shadow != nullptr, s->cap_stream));
    if (s1 == n) {
      // every dirty page is in staging: the application continues while the
      // last chunk is encoded and the image's tables are finished
      CK(cudaEventRecord(img->ev_captured, s->cap_stream));
      CK(cudaStreamWaitEvent(app, img->ev_captured, 0));
    }
    if (n == 0) break;
    const uint8_t* src = H.payload;
    uint64_t bytes = (s1 - s0) * kPage, host_off = poff + s0 * kPage;
    if (comp) {
      // this chunk's slots: sizes, offsets after enc_base, code, checksum
      const uint64_t m = s1 - s0;
      CK(cudaMemcpyAsync(H.cn, &m, sizeof m, cudaMemcpyHostToDevice, s->cap_stream));
      crum::BpdSizeArgs za{H.payload, H.cn, H.enc_len, H.alph};
      CK(crum::launch_bpd_size(za, m, s->cap_stream));
      crum::BpdScanArgs qa{H.enc_len, H.cn, offs + s0, enc_base, H.ctotal, H.mailbox_dev, H0.meta,
                           static_cast<uint32_t>(A)};
      CK(crum::launch_bpd_scan(qa, s->cap_stream));
      CK(cudaEventRecord(H.ev_sized, s->cap_stream));
      if ((st = wait_event(H.ev_sized, kBackgroundLimitNs)) != CRUM_OK) return st;
      bytes = reinterpret_cast<volatile uint64_t*>(H.mailbox)[3];
      crum::BpdEncodeArgs ea{H.payload, H.cn, offs + s0, enc_base, H.cpay, H0.meta, static_cast<uint32_t>(A),
                             poff, reinterpret_cast<unsigned long long*>(H0.scalars + 1), H.alph};
      CK(crum::launch_bpd_encode(ea, m, s->cap_stream));
      src = H.cpay;
      host_off = poff + enc_base;
      enc_base += bytes;
    } else {
      host_off = meta_bytes(A, n) + s0 * kPage;
    }
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, s->cap_stream));
    CK(cudaStreamWaitEvent(s->drain_stream, ev, 0));
    CK(cudaEventDestroy(ev));  // released once the recorded work completes
    if (s0 == 0) CK(cudaEventRecord(img->ev_d0, s->drain_stream));  // drain starts here
    if ((st = drain_payload(s, img, host_off, src, bytes)) != CRUM_OK) return st;
    CK(cudaEventRecord(H.ev_drained, s->drain_stream));
    h ^= 1;
  }
  if (comp) {
    // the compressed header words, the padding after the tables, and the
    // tables' share of the checksum; then the image buffer shrinks to fit
    const uint64_t final_len = poff + enc_base + 8;
    const uint64_t tab_end = kHeaderBytes + 16 * A + 24 * n;
    const uint64_t w1 = 2ull | ((static_cast<uint64_t>(img->full ? 1u : 0u) | 2ull) << 32);
    if (poff > tab_end) CK(cudaMemsetAsync(H0.meta + tab_end, 0, poff - tab_end, s->cap_stream));
    CK(cudaMemcpyAsync(H0.meta + 8, &w1, 8, cudaMemcpyHostToDevice, s->cap_stream));
    CK(cudaMemcpyAsync(H0.meta + 48, &poff, 8, cudaMemcpyHostToDevice, s->cap_stream));
    CK(cudaMemcpyAsync(H0.meta + 56, &final_len, 8, cudaMemcpyHostToDevice, s->cap_stream));
    CK(crum::launch_hash_bytes(H0.meta, poff, 0, H0.scalars + 1, s->cap_stream));
    CK(cudaEventRecord(img->ev_e1, s->cap_stream));
    img->payload_bytes = enc_base;
    img->image_bytes = final_len;
    if (!img->drop_payload) {
      const size_t have = (img->host_len + 4095) & ~size_t(4095), need = (final_len + 4095) & ~size_t(4095);
      if (have > need) img->pool->free(img->host + need, have - need);
      img->host_len = final_len;
    }
  }
  {
    cudaEvent_t ev;  // the tables and the trailer are final
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, s->cap_stream));
    CK(cudaStreamWaitEvent(s->drain_stream, ev, 0));
    CK(cudaEventDestroy(ev));
  }
  if (n == 0) CK(cudaEventRecord(img->ev_d0, s->drain_stream));  // no payload chunk was copied
  CK(cudaMemcpyAsync(img->host, H0.meta, payload_offset(img), cudaMemcpyDeviceToHost, s->drain_stream));
  CK(cudaMemcpyAsync(trailer_dst(img), H0.scalars + 1, 8, cudaMemcpyDeviceToHost, s->drain_stream));
  CK(cudaEventRecord(img->ev_drained, s->drain_stream));
  CK(cudaEventRecord(s->half[0].ev_drained, s->drain_stream));
  CK(cudaEventRecord(s->half[1].ev_drained, s->drain_stream));
  s->next_half = h;
  return CRUM_OK;
}

// Builds the capture graph of staging half h for the current registrations
// (see crum::CaptureGraph); the node arguments are placeholders that
// graph_launch replaces before every launch.
crum_status graph_build(crum_set* s, int h, crum_image* img, const crum::HashArgs& ha,
                        const crum::ScanArgs& sa, const crum::GatherArgs& ga) {
  crum::CaptureGraph& G = s->graph[h];
  Half& H = s->half[h];
  if (G.exec) {
    cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
  }
  if (G.graph) {
    cudaGraphDestroy(G.graph);
    G.graph = nullptr;
  }
  G.encoded = nullptr;
  for (cudaEvent_t& ev : G.placeholder)
    if (ev == nullptr) CK(cudaEventCreate(&ev));
  (void)img;
  CK(crum::hash_spec(s->n_pages, s->map_hash, false, &G.hs));
  CK(crum::scan_spec(&G.ss));
  CK(crum::gather_spec(s->n_pages, s->map_gather, ga.shadow != nullptr, &G.gs));
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphNode_t prev = nullptr, n = nullptr;
  auto after = [&](cudaGraphNode_t node) { prev = node; };
  cudaError_t e = cudaSuccess;
  cudaMemsetParams mp{};
  mp.dst = s->d_mask;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = (s->n_pages + 31) / 32;
  mp.height = 1;
  if (e == cudaSuccess) e = cudaGraphAddMemsetNode(&n, g, nullptr, 0, &mp);
  after(n);
  mp.dst = s->d_collisions;
  mp.width = 4;  // two u64 counters as four u32
  if (e == cudaSuccess) e = cudaGraphAddMemsetNode(&n, g, &prev, 1, &mp);
  after(n);
  if (e == cudaSuccess) e = cudaGraphAddEventRecordNode(&G.k0, g, &prev, 1, G.placeholder[0]);
  after(G.k0);
  auto kparams = [](const crum::KernelSpec& sp, void** args) {
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(sp.func);
    kp.gridDim = dim3(sp.grid);
    kp.blockDim = dim3(sp.block);
    kp.sharedMemBytes = static_cast<unsigned>(sp.smem);
    kp.kernelParams = args;
    return kp;
  };
  crum::HashArgs ha_c = ha;
  crum::ScanArgs sa_c = sa;
  crum::GatherArgs ga_c = ga;
  void* a_h[] = {&ha_c};
  void* a_s[] = {&sa_c};
  void* a_g[] = {&ga_c};
  cudaKernelNodeParams kp = kparams(G.hs, a_h);
  if (e == cudaSuccess) e = cudaGraphAddKernelNode(&G.hash, g, &prev, 1, &kp);
  after(G.hash);
  if (e == cudaSuccess) e = cudaGraphAddEventRecordNode(&G.k1, g, &prev, 1, G.placeholder[1]);
  after(G.k1);
  if (e == cudaSuccess) e = cudaGraphAddEventWaitNode(&n, g, &prev, 1, H.ev_drained);
  after(n);
  if (e == cudaSuccess) e = cudaGraphAddEventRecordNode(&G.k2, g, &prev, 1, G.placeholder[2]);
  after(G.k2);
  kp = kparams(G.ss, a_s);
  if (e == cudaSuccess) e = cudaGraphAddKernelNode(&G.scan, g, &prev, 1, &kp);
  after(G.scan);
  if (e == cudaSuccess) e = cudaGraphAddEventRecordNode(&n, g, &prev, 1, H.ev_scanned);
  after(n);
  kp = kparams(G.gs, a_g);
  if (e == cudaSuccess) e = cudaGraphAddKernelNode(&G.gather, g, &prev, 1, &kp);
  after(G.gather);
  if (e == cudaSuccess) e = cudaGraphAddEventRecordNode(&G.captured, g, &prev, 1, G.placeholder[3]);
  after(G.captured);
  if (s->cfg.compress) {
    // the encoding stage behind the capture: its arguments are this half's
    // buffers, fixed for the graph's life, so the nodes are never updated
    const uint32_t A = static_cast<uint32_t>(s->allocs.size());
    crum::BpdSizeArgs za{H.payload, H.scalars, H.enc_len, H.alph};
    crum::BpdScanArgs qa{H.enc_len, H.scalars, nullptr, 0, H.ctotal, H.mailbox_dev, H.meta, A};
    crum::BpdEncodeArgs ea{H.payload, H.scalars, nullptr, 0, H.cpay, H.meta, A, 0,
                           reinterpret_cast<unsigned long long*>(H.scalars + 1), H.alph};
    void* a_z[] = {&za};
    void* a_q[] = {&qa};
    void* a_e[] = {&ea};
    crum::KernelSpec es{};
    if (e == cudaSuccess) e = crum::bpd_encode_spec(s->n_pages, &es);
    kp = kparams(crum::bpd_size_spec(s->n_pages), a_z);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n, g, &prev, 1, &kp);
    after(n);
    kp = kparams(crum::bpd_scan_spec(), a_q);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n, g, &prev, 1, &kp);
    after(n);
    if (e == cudaSuccess) e = cudaGraphAddEventRecordNode(&n, g, &prev, 1, H.ev_sized);
    after(n);
    cudaMemsetParams zp{};  // the trailer receives the compressed image's checksum
    zp.dst = H.scalars + 1;
    zp.value = 0;
    zp.elementSize = 4;
    zp.width = 2;
    zp.height = 1;
    if (e == cudaSuccess) e = cudaGraphAddMemsetNode(&n, g, &prev, 1, &zp);
    after(n);
    kp = kparams(es, a_e);
    if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n, g, &prev, 1, &kp);
    after(n);
    if (e == cudaSuccess) e = cudaGraphAddEventRecordNode(&n, g, &prev, 1, H.ev_encoded);
    after(n);
    if (e == cudaSuccess) e = cudaGraphAddEventRecordNode(&G.encoded, g, &prev, 1, G.placeholder[4]);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&G.exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    G.exec = nullptr;
    return fail(CRUM_ECUDA, "capture graph: %s", cudaGetErrorString(e));
  }
  G.graph = g;
  G.epoch = s->graph_epoch;
  return CRUM_OK;
}

crum_status graph_launch(crum_set* s, int h, crum_image* img, const crum::HashArgs& ha,
                         const crum::ScanArgs& sa, const crum::GatherArgs& ga) {
  crum::CaptureGraph& G = s->graph[h];
  if (G.exec == nullptr || G.epoch != s->graph_epoch) {
    crum_status st = graph_build(s, h, img, ha, sa, ga);
    if (st != CRUM_OK) return st;
  }
  auto set_kernel = [&](cudaGraphNode_t node, const crum::KernelSpec& sp, void* arg) {
    void* args[] = {arg};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void*>(sp.func);
    kp.gridDim = dim3(sp.grid);
    kp.blockDim = dim3(sp.block);
    kp.sharedMemBytes = static_cast<unsigned>(sp.smem);
    kp.kernelParams = args;
    return cudaGraphExecKernelNodeSetParams(G.exec, node, &kp);
  };
  crum::HashArgs ha_c = ha;
  crum::ScanArgs sa_c = sa;
  crum::GatherArgs ga_c = ga;
  cudaError_t e = set_kernel(G.hash, G.hs, &ha_c);
  if (e == cudaSuccess) e = set_kernel(G.scan, G.ss, &sa_c);
  if (e == cudaSuccess) e = set_kernel(G.gather, G.gs, &ga_c);
  if (e == cudaSuccess) e = cudaGraphExecEventRecordNodeSetEvent(G.exec, G.k0, img->ev_k0);
  if (e == cudaSuccess) e = cudaGraphExecEventRecordNodeSetEvent(G.exec, G.k1, img->ev_k1);
  if (e == cudaSuccess) e = cudaGraphExecEventRecordNodeSetEvent(G.exec, G.k2, img->ev_k2);
  if (e == cudaSuccess)
    e = cudaGraphExecEventRecordNodeSetEvent(G.exec, G.captured, img->ev_captured);
  if (e == cudaSuccess && G.encoded != nullptr)
    e = cudaGraphExecEventRecordNodeSetEvent(G.exec, G.encoded, img->ev_e1);
  if (e == cudaSuccess) e = cudaGraphLaunch(G.exec, s->cap_stream);
  // back to the placeholders: the launch just queued keeps the image's
  // events, and the executable graph never refers to an event that may die
  const cudaGraphNode_t nodes[5] = {G.k0, G.k1, G.k2, G.captured, G.encoded};
  for (int i = 0; i < 5; ++i) {
    if (nodes[i] == nullptr) continue;
    const cudaError_t r = cudaGraphExecEventRecordNodeSetEvent(G.exec, nodes[i], G.placeholder[i]);
    if (e == cudaSuccess) e = r;
  }
  if (e != cudaSuccess) return fail(CRUM_ECUDA, "capture graph launch: %s", cudaGetErrorString(e));
  crum::g_kernel_launches.fetch_add(s->cfg.compress ? 7 : 3, std::memory_order_relaxed);
  return CRUM_OK;
}

// Placement of managed allocations (cfg.managed_in_place).  A range is
// host-placed when its preferred location is the host, or it has none and
// was last prefetched to the host; those are the pages a fault would
// migrate to the device.  The device keeps a mapping to them
// (cudaMemAdviseSetAccessedBy: no migration, reads cross the link), added
// by the set only where the application has not set it for this device.
void withdraw_advice(crum_set* s, Alloc& a) {
  if (!a.advised) return;
  cudaMemLocation loc{};
  loc.type = cudaMemLocationTypeDevice;
  loc.id = s->device;
  // the application may have freed the range after the set's last use
  if (cudaMemAdvise(a.ptr, a.bytes, cudaMemAdviseUnsetAccessedBy, loc) != cudaSuccess) cudaGetLastError();
  a.advised = false;
}

bool accessed_by_device(const Alloc& a, int device) {
  int devs[64];
  for (int& d : devs) d = cudaInvalidDeviceId;
  if (cudaMemRangeGetAttribute(devs, sizeof devs, cudaMemRangeAttributeAccessedBy, a.ptr, a.bytes) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  for (int d : devs)
    if (d == device) return true;
  return false;
}

// Looks up each managed allocation's placement and sets or withdraws the
// set's advice; returns the pages of host-placed allocations.
crum_status refresh_placement(crum_set* s, uint64_t* host_pages) {
  *host_pages = 0;
  if (!s->cfg.managed_in_place) return CRUM_OK;
  for (Alloc& a : s->allocs) {
    if (!a.managed) continue;
    int pref = cudaInvalidDeviceId, last = cudaInvalidDeviceId;
    if (cudaMemRangeGetAttribute(&pref, sizeof pref, cudaMemRangeAttributePreferredLocation, a.ptr, a.bytes) !=
            cudaSuccess ||
        cudaMemRangeGetAttribute(&last, sizeof last, cudaMemRangeAttributeLastPrefetchLocation, a.ptr,
                                 a.bytes) != cudaSuccess)
      return fail(CRUM_ECUDA, "placement of allocation %u: %s", a.id, cudaGetErrorString(cudaGetLastError()));
    const bool host = pref == cudaCpuDeviceId || (pref == cudaInvalidDeviceId && last == cudaCpuDeviceId);
    if (host) {
      *host_pages += a.n_pages;
      if (!a.advised && !accessed_by_device(a, s->device)) {
        cudaMemLocation loc{};
        loc.type = cudaMemLocationTypeDevice;
        loc.id = s->device;
        if (cudaMemAdvise(a.ptr, a.bytes, cudaMemAdviseSetAccessedBy, loc) != cudaSuccess)
          return fail(CRUM_ECUDA, "advice for allocation %u: %s", a.id, cudaGetErrorString(cudaGetLastError()));
        a.advised = true;
      }
    } else {
      withdraw_advice(s, a);
    }
  }
  return CRUM_OK;
}

}  // namespace

// ------------------------------------------------------------ PinnedPool ---

namespace crum {

PinnedPool::PinnedPool(size_t initial) : initial_(initial) {}

PinnedPool::~PinnedPool() {
  for (Arena& a : arenas_) cudaFreeHost(a.base);
}

uint8_t* PinnedPool::alloc(size_t n) {
  n = (n + 4095) & ~size_t(4095);
  std::lock_guard<std::mutex> lk(mu_);
  for (Arena& a : arenas_)
    for (auto it = a.free_list.begin(); it != a.free_list.end(); ++it)
      if (it->second >= n) {
        const size_t off = it->first, len = it->second;
        a.free_list.erase(it);
        if (len > n) a.free_list.emplace(off + n, len - n);
        return a.base + off;
      }
  // grow geometrically (at least 4 MiB, at most 256 MiB beyond the request)
  // so small sets pin little and large ones pin rarely
  size_t size = std::max(n, arenas_.empty() ? initial_ : size_t(0));
  size = std::max(size, std::min(std::max(reserved_, size_t(4) << 20), size_t(256) << 20));
  size = (size + (size_t(2) << 20) - 1) & ~((size_t(2) << 20) - 1);
  uint8_t* p = nullptr;
  if (cudaHostAlloc(reinterpret_cast<void**>(&p), size, cudaHostAllocPortable | cudaHostAllocMapped) !=
      cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  Arena a{p, size, {}};
  if (size > n) a.free_list.emplace(n, size - n);
  arenas_.push_back(std::move(a));
  reserved_ += size;
  return p;
}

void PinnedPool::free(uint8_t* p, size_t n) {
  if (p == nullptr) return;
  n = (n + 4095) & ~size_t(4095);
  std::lock_guard<std::mutex> lk(mu_);
  for (Arena& a : arenas_) {
    if (p < a.base || p >= a.base + a.size) continue;
    size_t off = static_cast<size_t>(p - a.base), len = n;
    auto next = a.free_list.lower_bound(off);
    if (next != a.free_list.end() && next->first == off + len) {
      len += next->second;
      next = a.free_list.erase(next);
    }
    if (next != a.free_list.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        off = prev->first;
        len += prev->second;
        a.free_list.erase(prev);
      }
    }
    a.free_list.emplace(off, len);
    return;
  }
}

}  // namespace crum

// ------------------------------------------------------------------ C ABI ---

extern "C" {

void crum_config_default(crum_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof *cfg);
  cfg->device = 0;
  cfg->staging_bytes = kDefaultStaging;
  cfg->chunk_bytes = kDefaultChunk;
  cfg->sink = CRUM_SINK_MEMORY;
  cfg->hash_mapping = -1;
  cfg->gather_mapping = -1;
}

const char* crum_last_error(void) { return t_err.c_str(); }

const char* crum_version(void) { return "crum-b300 1.0 sm_103a"; }

uint64_t crum_kernel_launches(void) { return crum::g_kernel_launches.load(); }

crum_status crum_set_create(const crum_config* cfg_in, crum_set** out) {
  t_err.clear();
  if (out == nullptr) return fail(CRUM_EINVAL, "out is null");
  *out = nullptr;
  crum_config cfg;
  crum_config_default(&cfg);
  if (cfg_in) cfg = *cfg_in;
  if (cfg.staging_bytes == 0) cfg.staging_bytes = kDefaultStaging;
  if (cfg.chunk_bytes == 0) cfg.chunk_bytes = kDefaultChunk;
  // copies stay 16-byte aligned, and none is so small that issuing it costs
  // more than moving it
  cfg.chunk_bytes = std::max<uint64_t>((cfg.chunk_bytes + 15) & ~15ull, 4096);
  if (cfg.staging_bytes < 2ull * kPage)
    return fail(CRUM_EINVAL, "staging_bytes must hold at least one page per half");
  if (cfg.sink < CRUM_SINK_MEMORY || cfg.sink > CRUM_SINK_NULL) return fail(CRUM_EINVAL, "bad sink");
  if (cfg.sink == CRUM_SINK_FILE && (cfg.sink_dir == nullptr || cfg.sink_dir[0] == 0))
    return fail(CRUM_EINVAL, "file sink needs sink_dir");
  if (cfg.hash_mapping < -1 || cfg.hash_mapping >= crum::kNumMappings ||
      cfg.gather_mapping < -1 || cfg.gather_mapping > 5)
    return fail(CRUM_EINVAL, "mapping out of range");
  if (cfg.restore_mode < 0 || cfg.restore_mode > 3) return fail(CRUM_EINVAL, "bad restore_mode");
  if (cfg.max_pending < 0) return fail(CRUM_EINVAL, "bad max_pending");
  if (cfg.compress && cfg.external_staging) return fail(CRUM_EINVAL, "compression needs the set's own staging");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg.device < 0 || cfg.device >= ndev) {
    cudaGetLastError();
    return fail(CRUM_EINVAL, "no CUDA device %d", cfg.device);
  }
  DeviceGuard dg(cfg.device);
  auto s = std::make_unique<crum_set>();
  s->cfg = cfg;
  if (cfg.sink_dir) s->sink_dir = cfg.sink_dir;
  s->cfg.sink_dir = nullptr;
  s->device = cfg.device;
  s->set_id = g_set_ids.fetch_add(1);
  s->half_slots = cfg.external_staging ? 0 : cfg.staging_bytes / 2 / kPage;
  if (cfg.hash_mapping >= 0) s->map_hash = cfg.hash_mapping;
  if (cfg.gather_mapping >= 0) s->map_gather = cfg.gather_mapping;
  s->pool = std::make_shared<crum::PinnedPool>(cfg.host_pool_bytes);
  if (cfg.host_pool_bytes) {
    uint8_t* p = s->pool->alloc(cfg.host_pool_bytes);
    if (!p) return fail(CRUM_ENOMEM, "cannot pin %llu host bytes", (unsigned long long)cfg.host_pool_bytes);
    s->pool->free(p, cfg.host_pool_bytes);
  }
  CK(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&s->drain_stream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&s->ev_app, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&s->ev_done, cudaEventDisableTiming));
  CK(cudaMalloc(&s->d_collisions, 2 * sizeof(unsigned long long)));  // [0] collisions, [1] error
  for (Half& H : s->half) {
    if (!cfg.external_staging && cudaMalloc(&H.payload, s->half_slots * kPage) != cudaSuccess) {
      cudaGetLastError();
      return fail(CRUM_ENOMEM, "cannot allocate %llu bytes of staging",
                  (unsigned long long)(s->half_slots * kPage));
    }
    CK(cudaMalloc(&H.scalars, 2 * sizeof(uint64_t)));
    if (cfg.compress) {
      if (cudaMalloc(&H.cpay, s->half_slots * kPage) != cudaSuccess) {
        cudaGetLastError();
        return fail(CRUM_ENOMEM, "cannot allocate %llu bytes of compressed staging",
                    (unsigned long long)(s->half_slots * kPage));
      }
      CK(cudaMalloc(&H.enc_len, std::max<uint64_t>(s->half_slots, 1) * sizeof(uint32_t)));
      CK(cudaMalloc(&H.alph, std::max<uint64_t>(s->half_slots, 1) * crum::kBpdAlphBytes));
      CK(cudaMalloc(&H.ctotal, sizeof(uint64_t)));
      CK(cudaMalloc(&H.cn, 2 * sizeof(uint64_t)));
      CK(cudaEventCreateWithFlags(&H.ev_sized, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&H.ev_encoded, cudaEventDisableTiming));
    }
    CK(cudaHostAlloc(reinterpret_cast<void**>(&H.mailbox), 4 * sizeof(uint64_t), cudaHostAllocMapped));
    CK(cudaHostGetDevicePointer(reinterpret_cast<void**>(&H.mailbox_dev), H.mailbox, 0));
    CK(cudaEventCreateWithFlags(&H.ev_scanned, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&H.ev_drained, cudaEventDisableTiming));
    CK(cudaEventRecord(H.ev_drained, s->drain_stream));
  }
  crum_set* raw = s.release();
  raw->planner = std::thread(planner_main, raw);
  raw->drainer = std::thread(drainer_main, raw);
  raw->writer = std::thread(writer_main, raw);
  *out = raw;
  return CRUM_OK;
}

crum_status crum_set_destroy(crum_set* s) {
  t_err.clear();
  if (s == nullptr) return CRUM_OK;
  DeviceGuard dg(s->device);
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv.wait_for(lk, std::chrono::seconds(600), [&] { return s->inflight == 0; });
    s->stop = true;
    s->plan_cv.notify_all();
    s->done_cv.notify_all();
    s->write_cv.notify_all();
  }
  if (s->planner.joinable()) s->planner.join();
  if (s->drainer.joinable()) s->drainer.join();
  if (s->writer.joinable()) s->writer.join();
  cudaStreamSynchronize(s->cap_stream);
  cudaStreamSynchronize(s->drain_stream);
  if (s->bounce != nullptr) s->pool->free(s->bounce, s->cfg.chunk_bytes);
  for (Alloc& a : s->allocs) withdraw_advice(s, a);
  image_unref(s->last);
  for (crum::CaptureGraph& G : s->graph) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    if (G.graph) cudaGraphDestroy(G.graph);
    for (cudaEvent_t ev : G.placeholder)
      if (ev) cudaEventDestroy(ev);
  }
  for (Half& H : s->half) {
    cudaFree(H.meta);
    if (!s->cfg.external_staging) cudaFree(H.payload);
    cudaFree(H.scalars);
    cudaFreeHost(H.mailbox);
    cudaEventDestroy(H.ev_scanned);
    cudaEventDestroy(H.ev_drained);
    cudaFree(H.cpay);
    cudaFree(H.enc_len);
    cudaFree(H.alph);
    cudaFree(H.ctotal);
    cudaFree(H.cn);
    if (H.ev_sized) cudaEventDestroy(H.ev_sized);
    if (H.ev_encoded) cudaEventDestroy(H.ev_encoded);
  }
  cudaFree(s->d_allocs);
  cudaFree(s->d_first_page);
  cudaFree(s->d_h);
  cudaFree(s->d_mask);
  cudaFree(s->d_word_offset);
  cudaFree(s->d_collisions);
  cudaFree(s->d_shadow);
  cudaFree(s->d_owner);
  cudaFree(s->d_chain);
  cudaFree(s->d_cur);
  cudaFree(s->d_copied);
  cudaEventDestroy(s->ev_app);
  cudaEventDestroy(s->ev_done);
  cudaStreamDestroy(s->cap_stream);
  cudaStreamDestroy(s->drain_stream);
  delete s;
  return CRUM_OK;
}

crum_status crum_register(crum_set* s, void* ptr, size_t bytes, uint32_t* alloc_id) {
  t_err.clear();
  if (s == nullptr || ptr == nullptr) return fail(CRUM_EINVAL, "null set or pointer");
  if (bytes == 0) return fail(CRUM_EINVAL, "zero-byte registration");
  if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0) return fail(CRUM_EINVAL, "pointer not 16-byte aligned");
  if (pages_of(bytes) > 0xFFFFFFFFull) return fail(CRUM_EINVAL, "allocation too large");
  // both ends must be device memory of the set's device or managed memory
  // (read by the kernels wherever its pages are), so no kernel is ever
  // handed an address it cannot read
  bool managed = true;
  for (const uint8_t* q : {static_cast<const uint8_t*>(ptr), static_cast<const uint8_t*>(ptr) + bytes - 1}) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, q) != cudaSuccess) {
      cudaGetLastError();
      return fail(CRUM_EINVAL, "not a CUDA allocation");
    }
    if (pa.type != cudaMemoryTypeManaged && (pa.type != cudaMemoryTypeDevice || pa.device != s->device)) {
      return fail(CRUM_EINVAL, "range is neither device memory of device %d nor managed memory",
                  s->device);
    }
    managed = managed && pa.type == cudaMemoryTypeManaged;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  const uintptr_t lo = reinterpret_cast<uintptr_t>(ptr), hi = lo + bytes;
  for (const Alloc& a : s->allocs) {
    const uintptr_t alo = reinterpret_cast<uintptr_t>(a.ptr), ahi = alo + a.bytes;
    if (lo < ahi && alo < hi) return fail(CRUM_EINVAL, "range overlaps registration %u", a.id);
  }
  Alloc a{s->next_id++, static_cast<uint8_t*>(ptr), bytes, pages_of(bytes), s->n_pages};
  a.managed = managed;
  s->allocs.push_back(a);
  s->n_pages += a.n_pages;
  s->table_dirty = s->reg_changed = true;
  s->graph_epoch++;
  if (alloc_id) *alloc_id = a.id;
  return CRUM_OK;
}

crum_status crum_unregister(crum_set* s, uint32_t id) {
  t_err.clear();
  if (s == nullptr) return fail(CRUM_EINVAL, "null set");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = std::find_if(s->allocs.begin(), s->allocs.end(), [&](const Alloc& a) { return a.id == id; });
  if (it == s->allocs.end()) return fail(CRUM_EINVAL, "unknown allocation id %u", id);
  {
    DeviceGuard dg(s->device);
    withdraw_advice(s, *it);
  }
  s->allocs.erase(it);
  uint64_t first = 0;
  for (Alloc& a : s->allocs) {
    a.first_page = first;
    first += a.n_pages;
  }
  s->n_pages = first;
  s->table_dirty = s->reg_changed = true;
  s->graph_epoch++;
  return CRUM_OK;
}

crum_status crum_set_info(const crum_set* s, uint32_t* n_allocs, uint64_t* n_pages) {
  if (s == nullptr) return fail(CRUM_EINVAL, "null set");
  std::lock_guard<std::mutex> lk(const_cast<crum_set*>(s)->mu);
  if (n_allocs) *n_allocs = static_cast<uint32_t>(s->allocs.size());
  if (n_pages) *n_pages = s->n_pages;
  return CRUM_OK;
}

crum_status crum_autotune(crum_set* s, int* hash_mapping, int* gather_mapping, double* hash_ms,
                          double* gather_ms) {
  crum::TraceRange tr("crum_autotune");
  t_err.clear();
  if (s == nullptr) return fail(CRUM_EINVAL, "null set");
  DeviceGuard dg(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->allocs.empty()) return fail(CRUM_EINVAL, "no registered allocations");
  crum_status st = ensure_capacity(s, lk);
  if (st == CRUM_OK) st = quiesce(s, lk);
  if (st != CRUM_OK) return st;
  if ((st = upload_table(s)) != CRUM_OK) return st;
  const uint64_t n = s->n_pages;
  const uint64_t words = (n + 31) / 32;
  constexpr int kReps = 3;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  uint64_t* d_out = nullptr;
  CK(cudaMalloc(&d_out, n * sizeof(uint64_t)));
  std::vector<uint64_t> ref(n), got(n);
  double best = 1e30;
  int best_h = s->map_hash;
  crum::HashArgs ha{};
  ha.allocs = s->d_allocs;
  ha.first_page = s->d_first_page;
  ha.n_allocs = static_cast<uint32_t>(s->allocs.size());
  ha.n_pages = n;
  ha.h_out = d_out;
  auto cleanup = [&]() {
    cudaFree(d_out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  };
  for (int m = 0; m < crum::kNumMappings && st == CRUM_OK; ++m) {
    cudaError_t ce = crum::launch_hash_dirty(ha, m, false, s->cap_stream);  // warm-up
    if (ce == cudaSuccess) ce = cudaEventRecord(e0, s->cap_stream);
    for (int r = 0; r < kReps && ce == cudaSuccess; ++r)
      ce = crum::launch_hash_dirty(ha, m, false, s->cap_stream);
    if (ce == cudaSuccess) ce = cudaEventRecord(e1, s->cap_stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->cap_stream);
    float ms = 0;
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (ce == cudaSuccess)
      ce = cudaMemcpy(m == 0 ? ref.data() : got.data(), d_out, n * 8, cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) {
      st = fail(CRUM_ECUDA, "autotune hash mapping %d: %s", m, cudaGetErrorString(ce));
      break;
    }
    if (m > 0 && got != ref) {
      st = fail(CRUM_ECORRUPT, "hash mapping %d disagrees with mapping 0", m);
      break;
    }
    const double mean = ms / kReps;
    if (hash_ms) hash_ms[m] = mean;
    if (mean < best) {
      best = mean;
      best_h = m;
    }
  }
  // gather: a synthetic dirty set (bit 0 of every bitmap byte, 1 page in 8)
  // scanned into staging half 0, then each mapping gathers its first slots
  // (as many as one staging half holds)
  int best_g = s->map_gather;
  Half& H = s->half[0];
  const uint64_t slots = std::min<uint64_t>((n + 7) / 8, s->half_slots);
  if (st == CRUM_OK && slots > 0) {
    cudaError_t ce = cudaMemsetAsync(s->d_mask, 0x01, words * sizeof(uint32_t), s->cap_stream);
    crum::ScanArgs sa{};
    sa.mask = s->d_mask;
    sa.n_words = words;
    sa.word_offset = s->d_word_offset;
    sa.n_dirty_out = H.scalars;
    sa.allocs = s->d_allocs;
    sa.n_allocs = ha.n_allocs;
    sa.meta = H.meta;
    sa.trailer = H.scalars + 1;
    sa.parent_seq = CRUM_NO_PARENT;
    // bits past the last page may be set by the pattern: clear that word's tail
    if (ce == cudaSuccess && (n & 31) != 0) {
      const uint32_t last = 0x01010101u & ((1u << (n & 31)) - 1u);
      ce = cudaMemcpyAsync(s->d_mask + words - 1, &last, 4, cudaMemcpyHostToDevice, s->cap_stream);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->cap_stream);
    }
    if (ce == cudaSuccess) ce = crum::launch_scan(sa, s->cap_stream);
    crum::GatherArgs ga{};
    ga.allocs = s->d_allocs;
    ga.first_page = s->d_first_page;
    ga.n_allocs = ha.n_allocs;
    ga.mask = s->d_mask;
    ga.word_offset = s->d_word_offset;
    ga.n_words = words;
    ga.n_pages = n;
    ga.n_dirty = H.scalars;
    ga.h_table = s->d_h;
    ga.meta = H.meta;
    ga.payload = H.payload;
    ga.trailer = H.scalars + 1;
    ga.s_begin = 0;
    ga.s_end = slots;
    best = 1e30;
    for (int m = 0; m <= 5 && ce == cudaSuccess; ++m) {
      ce = crum::launch_gather(ga, slots, m, false, s->cap_stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(e0, s->cap_stream);
      for (int r = 0; r < kReps && ce == cudaSuccess; ++r)
        ce = crum::launch_gather(ga, slots, m, false, s->cap_stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, s->cap_stream);
      if (ce == cudaSuccess) ce = cudaStreamSynchronize(s->cap_stream);
      float ms = 0;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce != cudaSuccess) break;
      const double mean = ms / kReps;
      if (gather_ms) gather_ms[m] = mean;
      if (mean < best) {
        best = mean;
        best_g = m;
      }
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(H.ev_drained, s->cap_stream);
    if (ce != cudaSuccess) st = fail(CRUM_ECUDA, "autotune gather: %s", cudaGetErrorString(ce));
  }
  cleanup();
  if (st != CRUM_OK) return st;
  s->map_hash = best_h;
  s->map_gather = best_g;
  s->graph_epoch++;
  if (hash_mapping) *hash_mapping = best_h;
  if (gather_mapping) *gather_mapping = best_g;
  return CRUM_OK;
}

crum_status crum_checkpoint(crum_set* s, crum_stream_t app_stream, int flags, crum_image** out) {
  crum::TraceRange tr("crum_checkpoint");
  t_err.clear();
  if (s == nullptr || out == nullptr) return fail(CRUM_EINVAL, "null set or out");
  *out = nullptr;
  const bool verify = (flags & CRUM_VERIFY) != 0;
  if (verify && !s->cfg.verify) return fail(CRUM_EINVAL, "CRUM_VERIFY needs a set created with verify=1");
  cudaStream_t app = static_cast<cudaStream_t>(app_stream);
  DeviceGuard dg(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->allocs.empty()) return fail(CRUM_EINVAL, "no registered allocations");
  if (s->half_slots == 0) return fail(CRUM_EINVAL, "no staging bound to this set");
  crum_status st = ensure_capacity(s, lk);
  if (st != CRUM_OK) return st;
  if (s->cfg.max_pending > 0 &&
      !s->cv.wait_for(lk, std::chrono::seconds(600), [&] { return s->inflight < s->cfg.max_pending; }))
    return fail(CRUM_ETIMEOUT, "timed out waiting for earlier images to be persisted");
  const int h = s->next_half;
  Half& H = s->half[h];
  if (!s->cv.wait_for(lk, std::chrono::seconds(600), [&] { return H.drain_enqueued; }))
    return fail(CRUM_ETIMEOUT, "timed out waiting for a staging half");

  const bool full = (flags & CRUM_FULL) || s->needs_full || s->reg_changed ||
                    (s->cfg.max_chain > 0 && s->chain_len >= static_cast<uint64_t>(s->cfg.max_chain));
  auto* img = new crum_image();
  img->pool = s->pool;
  img->device = s->device;
  img->seq = s->seq;
  img->full = full;
  img->parent = full ? nullptr : s->last;
  img->parent_seq = full ? CRUM_NO_PARENT : s->last->seq;
  image_ref(img->parent);
  img->n_allocs = static_cast<uint32_t>(s->allocs.size());
  img->n_pages = s->n_pages;
  for (const Alloc& a : s->allocs) img->table.emplace_back(a.id, a.bytes);
  img->half = h;
  img->t_submit = std::chrono::steady_clock::now();
  img->drop_payload = s->cfg.sink == CRUM_SINK_NULL || (flags & CRUM_NO_PAYLOAD) != 0;
  img->do_fsync = s->cfg.fsync != 0;
  if (s->cfg.sink == CRUM_SINK_FILE) {
    char name[96];
    snprintf(name, sizeof name, "/crum_%u_%llu.img", s->set_id, (unsigned long long)img->seq);
    img->sink_path = s->sink_dir + name;
  }
  st = new_image_events(img);
  if (st != CRUM_OK) {
    image_unref(img);
    return st;
  }

  auto bail = [&](crum_status e) {
    // leave the set consistent: the next checkpoint starts a new full chain
    s->needs_full = true;
    image_unref(img);
    return e;
  };
  if (cudaEventRecord(s->ev_app, app) != cudaSuccess ||
      cudaStreamWaitEvent(s->cap_stream, s->ev_app, 0) != cudaSuccess ||
      cudaEventRecord(img->ev_submit, s->cap_stream) != cudaSuccess)
    return bail(fail(CRUM_ECUDA, "cannot order capture after the application stream: %s",
                     cudaGetErrorString(cudaGetLastError())));
  if ((st = refresh_placement(s, &img->host_pages)) != CRUM_OK) return bail(st);
  if ((st = upload_table(s)) != CRUM_OK) return bail(st);
  const uint64_t words = (s->n_pages + 31) / 32;

  crum::HashArgs ha{};
  ha.allocs = s->d_allocs;
  ha.first_page = s->d_first_page;
  ha.n_allocs = img->n_allocs;
  ha.n_pages = s->n_pages;
  ha.h_table = s->d_h;
  ha.dirty_mask = s->d_mask;
  ha.full = full;
  ha.shadow = s->d_shadow;
  ha.collisions = s->d_collisions;
  ha.error = reinterpret_cast<unsigned int*>(s->d_collisions + 1);
  crum::ScanArgs sa{};
  sa.mask = s->d_mask;
  sa.n_words = words;
  sa.word_offset = s->d_word_offset;
  sa.n_dirty_out = H.scalars;
  sa.mailbox = H.mailbox_dev;
  sa.collisions = verify ? s->d_collisions : nullptr;
  sa.error = reinterpret_cast<const unsigned int*>(s->d_collisions + 1);
  sa.allocs = s->d_allocs;
  sa.n_allocs = img->n_allocs;
  sa.meta = H.meta;
  sa.trailer = H.scalars + 1;
  sa.seq = img->seq;
  sa.parent_seq = img->parent_seq;
  sa.flags = full ? 1u : 0u;
  crum::GatherArgs ga{};
  ga.allocs = s->d_allocs;
  ga.first_page = s->d_first_page;
  ga.n_allocs = img->n_allocs;
  ga.mask = s->d_mask;
  ga.word_offset = s->d_word_offset;
  ga.n_words = words;
  ga.n_pages = s->n_pages;
  ga.n_dirty = H.scalars;
  ga.h_table = s->d_h;
  ga.meta = H.meta;
  ga.trailer = H.scalars + 1;
  // with verify enabled the shadow follows every capture, so a later
  // CRUM_VERIFY checkpoint compares against the last checkpointed bytes
  ga.shadow = s->cfg.verify ? s->d_shadow : nullptr;
  const bool gather_shadow = ga.shadow != nullptr;
  const bool fast = s->n_pages <= s->half_slots;
  img->compressed = s->cfg.compress != 0;
  if (fast) {
    ga.payload = H.payload;
    ga.s_begin = 0;
    ga.s_end = s->n_pages;
  }

  image_ref(img);  // in-flight reference, dropped when the image is finished
  s->inflight++;
  H.drain_enqueued = false;
  auto unwind = [&](crum_status e) {
    cudaEventRecord(H.ev_drained, s->cap_stream);
    H.drain_enqueued = true;
    s->cv.notify_all();
    s->inflight--;
    image_unref(img);
    return bail(e);
  };
  cudaError_t ce = cudaSuccess;
  if (fast && s->cfg.use_graph && !verify && !s->cfg.external_staging) {
    // one graph launch for the whole capture sequence
    st = graph_launch(s, h, img, ha, sa, ga);
    if (st != CRUM_OK) return unwind(st);
  } else {
    ce = cudaMemsetAsync(s->d_mask, 0, words * sizeof(uint32_t), s->cap_stream);
    if (ce == cudaSuccess)
      ce = cudaMemsetAsync(s->d_collisions, 0, 2 * sizeof(unsigned long long), s->cap_stream);
    if (ce == cudaSuccess) ce = cudaEventRecord(img->ev_k0, s->cap_stream);
    if (ce == cudaSuccess) ce = crum::launch_hash_dirty(ha, s->map_hash, verify, s->cap_stream);
    if (ce == cudaSuccess) ce = cudaEventRecord(img->ev_k1, s->cap_stream);
    // this half's previous drain must be done before its metadata is rewritten
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(s->cap_stream, H.ev_drained, 0);
    if (ce == cudaSuccess) ce = cudaEventRecord(img->ev_k2, s->cap_stream);
    if (ce == cudaSuccess) ce = crum::launch_scan(sa, s->cap_stream);
    if (ce == cudaSuccess) ce = cudaEventRecord(H.ev_scanned, s->cap_stream);
    if (ce == cudaSuccess && fast)
      ce = crum::launch_gather(ga, s->n_pages, s->map_gather, gather_shadow, s->cap_stream);
    if (ce == cudaSuccess && fast) ce = cudaEventRecord(img->ev_captured, s->cap_stream);
    if (ce == cudaSuccess && fast && img->compressed) {
      // the application has its memory back; the staged slots are encoded
      // behind it: sizes, offsets and header, then the code and checksum
      crum::BpdSizeArgs za{H.payload, H.scalars, H.enc_len, H.alph};
      ce = crum::launch_bpd_size(za, s->n_pages, s->cap_stream);
      // the whole image: the kernels place the offset table after the
      // hashes once n is known on the device
      crum::BpdScanArgs qa{H.enc_len, H.scalars, nullptr, 0, H.ctotal, H.mailbox_dev, H.meta, img->n_allocs};
      if (ce == cudaSuccess) ce = crum::launch_bpd_scan(qa, s->cap_stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(H.ev_sized, s->cap_stream);
      crum::BpdEncodeArgs ea{H.payload, H.scalars, nullptr, 0, H.cpay, H.meta, img->n_allocs, 0,
                             reinterpret_cast<unsigned long long*>(H.scalars + 1), H.alph};
      if (ce == cudaSuccess) ce = cudaMemsetAsync(H.scalars + 1, 0, sizeof(uint64_t), s->cap_stream);
      if (ce == cudaSuccess) ce = crum::launch_bpd_encode(ea, s->n_pages, s->cap_stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(H.ev_encoded, s->cap_stream);
      if (ce == cudaSuccess) ce = cudaEventRecord(img->ev_e1, s->cap_stream);
    }
    if (ce != cudaSuccess)
      return unwind(fail(CRUM_ECUDA, "capture launch: %s", cudaGetErrorString(ce)));
  }
  if (fast) {
    ce = cudaStreamWaitEvent(app, img->ev_captured, 0);
    if (ce != cudaSuccess) return unwind(fail(CRUM_ECUDA, "app wait: %s", cudaGetErrorString(ce)));
    s->next_half = h ^ 1;
    if (s->sequencer) {
      std::lock_guard<std::mutex> qlk(s->sequencer->mu);
      img->ticket = static_cast<int64_t>(s->sequencer->issued++);
    }
    s->plan_q.push_back(img);
    s->plan_cv.notify_one();
  } else {
    st = checkpoint_chunked(s, img, app, lk, ga);
    H.drain_enqueued = true;
    s->cv.notify_all();
    if (st != CRUM_OK) {
      s->inflight--;
      image_unref(img);
      return bail(st);
    }
    s->done_q.push_back(img);
    s->done_cv.notify_one();
  }
  image_ref(img);  // the set's reference as the newest chain link
  image_unref(s->last);
  s->last = img;
  s->seq++;
  s->chain_len = full ? 0 : s->chain_len + 1;
  s->needs_full = false;
  s->reg_changed = false;
  *out = img;
  return CRUM_OK;
}

crum_status crum_image_wait(crum_image* img, int what, int64_t timeout_ns) {
  t_err.clear();
  if (img == nullptr || what < CRUM_WAIT_CAPTURED || what > CRUM_WAIT_PERSISTED)
    return fail(CRUM_EINVAL, "bad image or stage");
  if (what == CRUM_WAIT_CAPTURED && img->ev_captured != nullptr) {
    {
      std::lock_guard<std::mutex> lk(img->mu);
      if (img->stage >= CRUM_WAIT_CAPTURED) return img->status == CRUM_ECOLLISION ? CRUM_OK : img->status;
    }
    DeviceGuard dg(img->device);
    crum_status st = wait_event(img->ev_captured, timeout_ns);
    if (st == CRUM_OK) image_set_stage(img, CRUM_WAIT_CAPTURED, CRUM_OK, "");
    return st;
  }
  std::unique_lock<std::mutex> lk(img->mu);
  auto done = [&] { return img->stage >= what || (img->status != CRUM_OK && img->status != CRUM_ECOLLISION); };
  if (timeout_ns < 0) {
    img->cv.wait(lk, done);
  } else if (!img->cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns), done)) {
    return fail(CRUM_ETIMEOUT, "image %llu did not reach stage %d in time", (unsigned long long)img->seq, what);
  }
  if (img->status != CRUM_OK) {
    if (!img->err.empty()) t_err = img->err;
    else if (img->status == CRUM_ECOLLISION) t_err = "verify mode found hash collisions";
  }
  return img->status;
}

// OK once the image's bytes are in host memory, even if its sink failed
// afterwards (those bytes stay usable for copies, saves and restores).
static crum_status wait_drained(crum_image* img) {
  const crum_status st = crum_image_wait(img, CRUM_WAIT_DRAINED, -1);
  if (st == CRUM_OK || st == CRUM_ECOLLISION) return CRUM_OK;
  std::lock_guard<std::mutex> lk(img->mu);
  return img->stage >= CRUM_WAIT_DRAINED ? CRUM_OK : st;
}

crum_status crum_image_info_get(const crum_image* cimg, crum_image_info* info) {
  if (cimg == nullptr || info == nullptr) return fail(CRUM_EINVAL, "null image or info");
  crum_image* img = const_cast<crum_image*>(cimg);
  std::lock_guard<std::mutex> lk(img->mu);
  std::memset(info, 0, sizeof *info);
  info->seq = img->seq;
  info->parent_seq = img->parent_seq;
  info->n_pages = img->n_pages;
  info->n_allocs = img->n_allocs;
  info->full = img->full ? 1 : 0;
  info->stage = img->stage;
  info->status = img->status;
  if (img->stage >= CRUM_WAIT_DRAINED) {
    info->n_dirty = img->n_dirty;
    info->image_bytes = img->image_bytes;
    info->checksum = img->checksum;
    info->collisions = img->collisions;
    info->t_captured_ms = img->t_captured_ms;
    info->t_drained_ms = img->t_drained_ms;
    info->t_hash_ms = img->t_hash_ms;
    info->t_compact_ms = img->t_compact_ms;
    info->t_drain_ms = img->t_drain_ms;
  }
  info->host_pages = img->host_pages;
  if (img->stage >= CRUM_WAIT_DRAINED) info->t_encode_ms = img->t_encode_ms;
  if (img->stage >= CRUM_WAIT_PERSISTED) info->t_persisted_ms = img->t_persisted_ms;
  return CRUM_OK;
}

crum_status crum_image_copy(crum_image* img, void* dst, uint64_t dst_bytes) {
  t_err.clear();
  if (img == nullptr || dst == nullptr) return fail(CRUM_EINVAL, "null image or destination");
  crum_status st = wait_drained(img);
  if (st != CRUM_OK) return st;
  std::lock_guard<std::mutex> lk(img->mu);
  if (img->host == nullptr) return fail(CRUM_EIO, "image payload was dropped (null sink)");
  if (dst_bytes < img->image_bytes) return fail(CRUM_EINVAL, "destination holds %llu of %llu bytes",
                                                (unsigned long long)dst_bytes, (unsigned long long)img->image_bytes);
  std::memcpy(dst, img->host, img->image_bytes);
  return CRUM_OK;
}

crum_status crum_image_save(crum_image* img, const char* path) {
  t_err.clear();
  if (img == nullptr || path == nullptr) return fail(CRUM_EINVAL, "null image or path");
  crum_status st = wait_drained(img);
  if (st != CRUM_OK) return st;
  if (img->host == nullptr) return fail(CRUM_EIO, "image payload was dropped (null sink)");
  return write_file(img->host, img->image_bytes, path, false);
}

crum_status crum_image_release(crum_image* img) {
  if (img == nullptr) return CRUM_OK;
  DeviceGuard dg(img->device);
  image_unref(img);
  return CRUM_OK;
}

}  // extern "C"

// ------------------------------------------------------- image loading ---

namespace {

uint32_t rd32(const uint8_t* p) {
  uint32_t v;
  std::memcpy(&v, p, 4);
  return v;
}
uint64_t rd64(const uint8_t* p) {
  uint64_t v;
  std::memcpy(&v, p, 8);
  return v;
}

// Structural check of a serialized image held in host memory.
crum_status parse_image(const uint8_t* b, uint64_t n, crum_image* img) {
  if (n < kHeaderBytes + 8 || std::memcmp(b, "CRUMIMG1", 8) != 0) return fail(CRUM_ECORRUPT, "bad magic");
  const uint32_t version = rd32(b + 8);
  if ((version != 1 && version != 2) || rd32(b + 32) != kPage)
    return fail(CRUM_ECORRUPT, "bad version or page size");
  const uint64_t A = rd32(b + 36), nd = rd64(b + 40);
  if (version == 1) {
    if (nd > n / kPage || A > n / 16) return fail(CRUM_ECORRUPT, "counts exceed the image size");
    if (rd64(b + 56) != n || image_size(A, nd) != n || rd64(b + 48) != meta_bytes(A, nd))
      return fail(CRUM_ECORRUPT, "size fields disagree with the image length");
    img->compressed = false;
  } else {
    if (nd > n / 16 || A > n / 16 || (rd32(b + 12) & 2u) == 0)
      return fail(CRUM_ECORRUPT, "counts exceed the image size");
    const uint64_t poff = rd64(b + 48);
    if (rd64(b + 56) != n || poff != cmeta_bytes(A, nd) || poff + 8 > n)
      return fail(CRUM_ECORRUPT, "size fields disagree with the image length");
    const uint64_t total = n - 8 - poff;
    const uint8_t* ot = b + kHeaderBytes + 16 * A + 16 * nd;
    for (uint64_t s = 0; s < nd; ++s) {
      const uint64_t lo = rd64(ot + 8 * s), hi = s + 1 < nd ? rd64(ot + 8 * (s + 1)) : total;
      if ((s == 0 && lo != 0) || hi < lo + 16 || hi - lo > kPage || (hi - lo) % 16 != 0)
        return fail(CRUM_ECORRUPT, "slot offsets out of order or out of range");
    }
    if (nd == 0 && total != 0) return fail(CRUM_ECORRUPT, "payload without slots");
    img->compressed = true;
    img->payload_off = poff;
    img->payload_bytes = total;
  }
  img->full = (rd32(b + 12) & 1u) != 0;
  img->seq = rd64(b + 16);
  img->parent_seq = rd64(b + 24);
  img->n_allocs = static_cast<uint32_t>(A);
  img->n_dirty = nd;
  img->image_bytes = n;
  img->table.clear();
  uint64_t pages = 0;
  for (uint64_t a = 0; a < A; ++a) {
    const uint64_t bytes = rd64(b + kHeaderBytes + 16 * a + 8);
    if (bytes == 0) return fail(CRUM_ECORRUPT, "zero-sized allocation in table");
    img->table.emplace_back(rd32(b + kHeaderBytes + 16 * a), bytes);
    pages += pages_of(bytes);
  }
  img->n_pages = pages;
  const uint8_t* pt = b + kHeaderBytes + 16 * A;
  uint64_t prev = 0;
  for (uint64_t s = 0; s < nd; ++s) {
    const uint32_t a = rd32(pt + 8 * s), p = rd32(pt + 8 * s + 4);
    if (a >= A || p >= pages_of(img->table[a].second)) return fail(CRUM_ECORRUPT, "page table entry out of range");
    const uint64_t key = (static_cast<uint64_t>(a) << 32) | p;
    if (s > 0 && key <= prev) return fail(CRUM_ECORRUPT, "page table not ascending");
    prev = key;
  }
  img->checksum = rd64(b + n - 8);
  return CRUM_OK;
}

// Checksum of a host image computed on the device through staging half 0.
crum_status device_checksum(crum_set* s, const uint8_t* host, uint64_t n, uint64_t* out) {
  Half& H = s->half[0];
  const uint64_t chunk = s->half_slots * kPage;
  CK(cudaMemsetAsync(H.scalars + 1, 0, 8, s->cap_stream));
  for (uint64_t off = 0; off < n; off += chunk) {
    const uint64_t len = std::min(chunk, n - off);
    CK(cudaMemcpyAsync(H.payload, host + off, len, cudaMemcpyHostToDevice, s->cap_stream));
    CK(crum::launch_hash_bytes(H.payload, len, off / 8, H.scalars + 1, s->cap_stream));
  }
  CK(cudaMemcpyAsync(out, H.scalars + 1, 8, cudaMemcpyDeviceToHost, s->cap_stream));
  CK(cudaStreamSynchronize(s->cap_stream));
  return CRUM_OK;
}

crum_status load_common(crum_set* s, crum_image* parent, crum_image** out,
                        const std::function<crum_status(uint8_t*, uint64_t)>& fill, uint64_t n) {
  if ((n & 7) != 0 || n < kHeaderBytes + 8) return fail(CRUM_ECORRUPT, "image length %llu is not a valid size", (unsigned long long)n);
  DeviceGuard dg(s->device);
  auto* img = new crum_image();
  img->pool = s->pool;
  img->device = s->device;
  img->host_len = n;
  img->host = s->pool->alloc(n);
  if (img->host == nullptr) {
    image_unref(img);
    return fail(CRUM_ENOMEM, "pinned host pool exhausted");
  }
  crum_status st = fill(img->host, n);
  if (st == CRUM_OK) st = parse_image(img->host, n, img);
  if (st == CRUM_OK) {
    std::unique_lock<std::mutex> lk(s->mu);
    st = quiesce(s, lk);
    uint64_t cks = 0;
    if (st == CRUM_OK) st = device_checksum(s, img->host, n - 8, &cks);
    if (st == CRUM_OK && cks != img->checksum) st = fail(CRUM_ECORRUPT, "checksum mismatch");
    if (st == CRUM_OK) {
      // staging half 0 was overwritten: keep the two-halves protocol intact
      cudaEventRecord(s->half[0].ev_drained, s->cap_stream);
    }
  }
  if (st == CRUM_OK) {
    if (img->full) {
      img->parent_seq = CRUM_NO_PARENT;
    } else if (parent == nullptr || parent->seq != img->parent_seq) {
      st = fail(CRUM_EMISMATCH, "incremental image %llu needs parent %llu", (unsigned long long)img->seq,
                (unsigned long long)img->parent_seq);
    } else {
      img->parent = parent;
      image_ref(parent);
    }
  }
  if (st != CRUM_OK) {
    image_unref(img);
    return st;
  }
  img->stage = CRUM_WAIT_PERSISTED;
  *out = img;
  return CRUM_OK;
}

}  // namespace

extern "C" {

crum_status crum_image_load(crum_set* s, const char* path, crum_image* parent, crum_image** out) {
  t_err.clear();
  if (s == nullptr || path == nullptr || out == nullptr) return fail(CRUM_EINVAL, "null argument");
  *out = nullptr;
  const int fd = ::open(path, O_RDONLY);
  if (fd < 0) return fail(CRUM_EIO, "open %s: %s", path, strerror(errno));
  struct stat stt;
  if (fstat(fd, &stt) != 0) {
    ::close(fd);
    return fail(CRUM_EIO, "stat %s: %s", path, strerror(errno));
  }
  const uint64_t n = static_cast<uint64_t>(stt.st_size);
  crum_status st = load_common(
      s, parent, out,
      [&](uint8_t* dst, uint64_t len) -> crum_status {
        uint64_t off = 0;
        while (off < len) {
          const ssize_t r = ::read(fd, dst + off, static_cast<size_t>(std::min<uint64_t>(len - off, 1ull << 30)));
          if (r <= 0) return fail(CRUM_EIO, "read %s: %s", path, r == 0 ? "short file" : strerror(errno));
          off += static_cast<uint64_t>(r);
        }
        return CRUM_OK;
      },
      n);
  ::close(fd);
  return st;
}

crum_status crum_image_from_bytes(crum_set* s, const void* bytes, uint64_t n, crum_image* parent,
                                  crum_image** out) {
  t_err.clear();
  if (s == nullptr || bytes == nullptr || out == nullptr) return fail(CRUM_EINVAL, "null argument");
  *out = nullptr;
  return load_common(
      s, parent, out,
      [&](uint8_t* dst, uint64_t len) -> crum_status {
        std::memcpy(dst, bytes, len);
        return CRUM_OK;
      },
      n);
}

crum_status crum_restore(crum_set* s, const crum_image* chain_end, crum_stream_t stream) {
  crum::TraceRange tr("crum_restore");
  t_err.clear();
  if (s == nullptr || chain_end == nullptr) return fail(CRUM_EINVAL, "null set or image");
  cudaStream_t us = static_cast<cudaStream_t>(stream);
  std::vector<crum_image*> chain;
  for (crum_image* p = const_cast<crum_image*>(chain_end); p != nullptr; p = p->parent) {
    chain.push_back(p);
    if (p->full) break;
  }
  std::reverse(chain.begin(), chain.end());
  if (!chain.front()->full) return fail(CRUM_ECORRUPT, "chain has no full base image");
  for (crum_image* img : chain) {
    const crum_status st = wait_drained(img);
    if (st != CRUM_OK) return st;
    if (img->host == nullptr) return fail(CRUM_EIO, "image %llu has no payload (null sink)", (unsigned long long)img->seq);
  }
  DeviceGuard dg(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (crum_image* img : chain) {
    if (img->table.size() != s->allocs.size()) return fail(CRUM_EMISMATCH, "image has %zu allocations, set has %zu", img->table.size(), s->allocs.size());
    for (size_t a = 0; a < s->allocs.size(); ++a)
      if (img->table[a].second != s->allocs[a].bytes)
        return fail(CRUM_EMISMATCH, "allocation %zu: image %llu bytes, set %llu bytes", a,
                    (unsigned long long)img->table[a].second, (unsigned long long)s->allocs[a].bytes);
  }
  const uint64_t A = s->allocs.size();
  {
    // restored pages of host-placed managed allocations are written in place
    uint64_t host_pages = 0;
    const crum_status pst = refresh_placement(s, &host_pages);
    if (pst != CRUM_OK) return pst;
  }
  // auto: merged when the incrementals would carry more than 8 % of the
  // base's pages a second time (kernel reads of host memory run ~7 % below
  // DMA); delta is merged restricted to pages whose contents differ
  uint64_t incr_pages = 0;
  for (size_t i = 1; i < chain.size(); ++i) incr_pages += chain[i]->n_dirty;
  const bool delta = s->cfg.restore_mode == 3;
  bool merged = s->cfg.restore_mode == 2 || delta ||
                (s->cfg.restore_mode == 0 && incr_pages * 100 > 8 * chain.front()->n_dirty);
  std::vector<crum::ChainImage> ci;
  uint64_t total_slots = 0;
  bool any_compressed = false;
  for (size_t i = 0; merged && i < chain.size(); ++i) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, chain[i]->host) != cudaSuccess || pa.devicePointer == nullptr) {
      cudaGetLastError();
      if (s->cfg.restore_mode >= 2)
        return fail(CRUM_EINVAL, "image %llu is not in device-mapped host memory",
                    (unsigned long long)chain[i]->seq);
      merged = false;
      break;
    }
    const uint8_t* d = static_cast<const uint8_t*>(pa.devicePointer);
    const crum_image* im = chain[i];
    const uint64_t n = im->n_dirty;
    ci.push_back(crum::ChainImage{
        d + kHeaderBytes + 16 * A, d + kHeaderBytes + 16 * A + 8 * n, d + payload_offset(im), total_slots,
        im->compressed ? reinterpret_cast<const uint64_t*>(d + kHeaderBytes + 16 * A + 16 * n) : nullptr,
        im->payload_bytes, n});
    any_compressed = any_compressed || im->compressed;
    total_slots += n;
  }
  if (!merged && s->half_slots == 0) return fail(CRUM_EINVAL, "no staging bound to this set");
  crum_status st = ensure_capacity(s, lk);
  if (st != CRUM_OK) return st;
  CK(cudaEventRecord(s->ev_app, us));
  CK(cudaStreamWaitEvent(s->cap_stream, s->ev_app, 0));
  if ((st = upload_table(s)) != CRUM_OK) return st;
  if (s->d_copied == nullptr) CK(cudaMalloc(&s->d_copied, 2 * sizeof(unsigned long long)));
  CK(cudaMemsetAsync(s->d_copied, 0, 2 * sizeof(unsigned long long), s->cap_stream));
  if (merged && (st = restore_merged(s, ci, total_slots, delta, any_compressed)) != CRUM_OK) return st;
  s->restore_counted_on_device = merged;
  s->restore_pages = merged ? 0 : incr_pages + chain.front()->n_dirty;
  int h = s->next_half;
  for (crum_image* img : (merged ? std::vector<crum_image*>{} : chain)) {
    const uint64_t n = img->n_dirty;
    const uint8_t* ptab = img->host + kHeaderBytes + 16 * A;
    const uint8_t* hashes = ptab + 8 * n;
    const uint8_t* payload = img->host + payload_offset(img);
    const uint64_t* offs = reinterpret_cast<const uint64_t*>(hashes + 8 * n);
    for (uint64_t s0 = 0; s0 < n; s0 += s->half_slots) {
      const uint64_t s1 = std::min(n, s0 + s->half_slots);
      Half& H = s->half[h];
      if (!s->cv.wait_for(lk, std::chrono::seconds(600), [&] { return H.drain_enqueued; }))
        return fail(CRUM_ETIMEOUT, "timed out waiting for a staging half");
      CK(cudaStreamWaitEvent(s->cap_stream, H.ev_drained, 0));
      const uint64_t m = s1 - s0;
      CK(cudaMemcpyAsync(H.meta, ptab + 8 * s0, 8 * m, cudaMemcpyHostToDevice, s->cap_stream));
      CK(cudaMemcpyAsync(H.meta + 8 * m, hashes + 8 * s0, 8 * m, cudaMemcpyHostToDevice, s->cap_stream));
      if (img->compressed) {
        // encoded slots [s0, s1): their offsets, then their bytes
        const uint64_t lo = offs[s0], hi = s1 < n ? offs[s1] : img->payload_bytes;
        CK(cudaMemcpyAsync(H.meta + 16 * m, offs + s0, 8 * m, cudaMemcpyHostToDevice, s->cap_stream));
        CK(cudaMemcpyAsync(H.payload, payload + lo, hi - lo, cudaMemcpyHostToDevice, s->cap_stream));
        crum::BpdRestoreArgs ba{};
        ba.allocs = s->d_allocs;
        ba.n_allocs = static_cast<uint32_t>(A);
        ba.ptab = reinterpret_cast<const uint32_t*>(H.meta);
        ba.hashes = reinterpret_cast<const uint64_t*>(H.meta + 8 * m);
        ba.offs = reinterpret_cast<const uint64_t*>(H.meta + 16 * m);
        ba.enc = H.payload;
        ba.enc_end = hi;
        ba.n_slots = m;
        ba.h_table = s->d_h;
        ba.error = reinterpret_cast<unsigned int*>(s->d_copied + 1);
        CK(crum::launch_bpd_restore(ba, s->cap_stream));
        CK(cudaEventRecord(H.ev_drained, s->cap_stream));
        h ^= 1;
        continue;
      }
      CK(cudaMemcpyAsync(H.payload, payload + kPage * s0, kPage * m, cudaMemcpyHostToDevice, s->cap_stream));
      crum::RestoreArgs ra{};
      ra.allocs = s->d_allocs;
      ra.n_allocs = static_cast<uint32_t>(A);
      ra.ptab = reinterpret_cast<const uint32_t*>(H.meta);
      ra.hashes = reinterpret_cast<const uint64_t*>(H.meta + 8 * m);
      ra.payload = H.payload;
      ra.n_slots = m;
      ra.h_table = s->d_h;
      CK(crum::launch_restore(ra, s->cap_stream));
      CK(cudaEventRecord(H.ev_drained, s->cap_stream));
      h ^= 1;
    }
  }
  s->next_half = h;
  CK(cudaEventRecord(s->ev_done, s->cap_stream));
  CK(cudaStreamWaitEvent(us, s->ev_done, 0));
  crum_image* end = const_cast<crum_image*>(chain_end);
  image_ref(end);
  image_unref(s->last);
  s->last = end;
  s->seq = end->seq + 1;
  s->chain_len = chain.size() - 1;
  s->needs_full = s->cfg.verify != 0;  // the verify shadow does not hold the restored bytes
  s->reg_changed = false;
  return CRUM_OK;
}

crum_status crum_restore_pages(crum_set* s, uint64_t* pages) {
  t_err.clear();
  if (s == nullptr || pages == nullptr) return fail(CRUM_EINVAL, "null argument");
  DeviceGuard dg(s->device);
  bool on_device;
  uint64_t host_count;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    on_device = s->restore_counted_on_device;
    host_count = s->restore_pages;
  }
  crum_status st = wait_event(s->ev_done, kBackgroundLimitNs);
  if (st != CRUM_OK) return st;
  unsigned long long n[2] = {0, 0};  // pages copied by the kernels, decode failures
  if (s->d_copied != nullptr) CK(cudaMemcpy(n, s->d_copied, sizeof n, cudaMemcpyDeviceToHost));
  *pages = on_device ? n[0] : host_count;
  if (n[1] != 0) return fail(CRUM_ECORRUPT, "a compressed slot did not decode (it was skipped)");
  return CRUM_OK;
}

crum_status crum_hash_pages(const void* ptr, uint64_t bytes, uint64_t* out, crum_stream_t stream) {
  t_err.clear();
  if (ptr == nullptr || out == nullptr || bytes == 0) return fail(CRUM_EINVAL, "null pointer or zero size");
  if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0) return fail(CRUM_EINVAL, "pointer not 16-byte aligned");
  crum::HashArgs ha{};
  ha.allocs = nullptr;
  ha.one = DevAlloc{static_cast<uint8_t*>(const_cast<void*>(ptr)), bytes, 0, 0,
                    static_cast<uint32_t>(pages_of(bytes))};
  ha.n_allocs = 1;
  ha.n_pages = pages_of(bytes);
  ha.h_out = out;
  CK(crum::launch_hash_dirty(ha, 1, false, static_cast<cudaStream_t>(stream)));
  return CRUM_OK;
}

crum_status crum_hash_bytes(const void* ptr, uint64_t bytes, uint64_t first_index, uint64_t* out,
                            crum_stream_t stream) {
  t_err.clear();
  if (out == nullptr || (bytes > 0 && ptr == nullptr)) return fail(CRUM_EINVAL, "null pointer");
  if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0) return fail(CRUM_EINVAL, "pointer not 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(out, 0, 8, st));
  CK(crum::launch_hash_bytes(static_cast<const uint8_t*>(ptr), bytes, first_index, out, st));
  return CRUM_OK;
}

crum_status crum_get_hashes(crum_set* s, uint64_t* host_out, uint64_t n) {
  t_err.clear();
  if (s == nullptr || host_out == nullptr) return fail(CRUM_EINVAL, "null argument");
  DeviceGuard dg(s->device);
  std::lock_guard<std::mutex> lk(s->mu);
  if (n > s->n_pages || n > s->h_cap) return fail(CRUM_EINVAL, "asked for %llu hashes, table holds %llu", (unsigned long long)n, (unsigned long long)std::min<uint64_t>(s->n_pages, s->h_cap));
  CK(cudaStreamSynchronize(s->cap_stream));
  if (n) CK(cudaMemcpy(host_out, s->d_h, n * 8, cudaMemcpyDeviceToHost));
  return CRUM_OK;
}

crum_status crum_poke_hash(crum_set* s, uint64_t g, uint64_t value) {
  t_err.clear();
  if (s == nullptr) return fail(CRUM_EINVAL, "null set");
  DeviceGuard dg(s->device);
  std::lock_guard<std::mutex> lk(s->mu);
  if (g >= s->n_pages || g >= s->h_cap) return fail(CRUM_EINVAL, "page %llu out of range", (unsigned long long)g);
  CK(cudaStreamSynchronize(s->cap_stream));
  CK(cudaMemcpy(s->d_h + g, &value, 8, cudaMemcpyHostToDevice));
  return CRUM_OK;
}

}  // extern "C"

namespace crum {
// Lets other translation units of the library report a message through
// crum_last_error().
void set_last_error(const char* msg) { t_err = msg; }
}  // namespace crum

namespace crum {
// Point both staging halves of an external-staging set at `payload`
// (`slots` pages), or detach them (payload == nullptr).  The caller (the
// server) guarantees the set has nothing in flight.
// A server's clients share one drain order (see DrainSequencer); nullptr
// detaches the set.
crum_status set_drain_sequencer(crum_set* s, std::shared_ptr<DrainSequencer> q) {
  std::unique_lock<std::mutex> lk(s->mu);
  crum_status st = quiesce(s, lk);
  if (st != CRUM_OK) return st;
  s->sequencer = std::move(q);
  return CRUM_OK;
}

crum_status bind_staging(crum_set* s, uint8_t* payload, uint64_t slots) {
  std::unique_lock<std::mutex> lk(s->mu);
  if (!s->cfg.external_staging) return fail(CRUM_EINVAL, "set owns its staging");
  if (!(s->half[0].drain_enqueued && s->half[1].drain_enqueued))
    return fail(CRUM_EBUSY, "set has a capture in flight");
  for (Half& H : s->half) H.payload = payload;
  s->half_slots = payload != nullptr ? slots : 0;
  return CRUM_OK;
}
}  // namespace crum

extern "C" crum_status crum_selftest_wait_timeout(const void* ptr, uint64_t bytes, uint64_t limit_ns,
                                                  int* timed_out, crum_stream_t stream) {
  t_err.clear();
  if (ptr == nullptr || timed_out == nullptr || bytes < kPage)
    return fail(CRUM_EINVAL, "needs a device pointer to at least one full page");
  if (reinterpret_cast<uintptr_t>(ptr) % 16 != 0) return fail(CRUM_EINVAL, "pointer not 16-byte aligned");
  limit_ns = std::min<uint64_t>(std::max<uint64_t>(limit_ns, 1000000ull), 10000000000ull);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const uint64_t n = pages_of(bytes);
  uint64_t* out = nullptr;
  unsigned int* flag = nullptr;
  CK(cudaMalloc(&out, n * sizeof(uint64_t)));
  if (cudaMalloc(&flag, sizeof(unsigned int)) != cudaSuccess) {
    cudaFree(out);
    return fail(CRUM_ENOMEM, "cannot allocate the self-test flag");
  }
  crum::HashArgs ha{};
  ha.one = DevAlloc{static_cast<uint8_t*>(const_cast<void*>(ptr)), bytes, 0, 0, static_cast<uint32_t>(n)};
  ha.n_allocs = 1;
  ha.n_pages = n;
  ha.h_out = out;
  ha.error = flag;
  ha.wait_limit_ns = limit_ns;
  ha.test_skip_chunk = 1;  // CTA 0 never issues its first quarter page
  unsigned int host_flag = 0;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) e = crum::launch_hash_dirty(ha, 6, false, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host_flag, flag, sizeof host_flag, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(out);
  cudaFree(flag);
  if (e != cudaSuccess) return fail(CRUM_ECUDA, "self-test: %s", cudaGetErrorString(e));
  *timed_out = host_flag != 0 ? 1 : 0;
  return CRUM_OK;
}
