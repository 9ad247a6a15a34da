// crum_server: checkpoint and restore requests from many clients, admitted
// as slots and staging memory free up, several on the device at once.
//
// The paper checkpoints one process per MPI rank (Sections 3.3-3.4); a
// serving deployment instead sees requests from many independent clients
// arriving at random.  Each client is a registration set whose hash table
// and page tables stay resident on the device; the server owns one staging
// pool (the budget) and lends each admitted request a region large enough
// for a full capture of its client (pages x 64 KiB).  Requests of different
// clients overlap on the device (each set has its own streams); a client's
// own requests run one at a time, in arrival order.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "crum.h"
#include "engine.h"

namespace crum {
crum_status bind_staging(crum_set* s, uint8_t* payload, uint64_t slots);
crum_status set_drain_sequencer(crum_set* s, std::shared_ptr<DrainSequencer> q);
void set_last_error(const char* msg);
}  // namespace crum

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  uint64_t id = 0;
  uint32_t client = 0;
  int kind = 0;
  int state = 0;  // 0 queued, 1 running, 2 done
  bool captured = false;
  crum_status status = CRUM_OK;
  Clock::time_point t_submit, t_admit, t_done;
  crum_image* img = nullptr;  // running checkpoint's image (released at completion,
                              // or kept for crum_server_take_image with keep_images)
  cudaEvent_t ev_done = nullptr;  // running restore's completion
  uint64_t region_off = 0, region_len = 0;
  uint64_t n_dirty = 0, bytes = 0, image_seq = 0, checksum = 0;
};

struct Client {
  crum_set* set = nullptr;
  cudaStream_t stream = nullptr;
  uint64_t pages = 0;
  crum_image* newest = nullptr;  // newest checkpoint image (reference held)
  bool busy = false;
};

}  // namespace

struct crum_server {
  crum_server_config cfg{};
  uint8_t* pool = nullptr;
  std::map<uint64_t, uint64_t> free_list;  // offset -> length, within pool
  uint64_t lent = 0, peak_lent = 0;
  std::mutex mu;
  std::condition_variable wake, done_cv;
  std::vector<Client> clients;
  std::unordered_map<uint64_t, Request> reqs;
  std::deque<uint64_t> pending;
  std::vector<uint64_t> running;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread th;
  // statistics since create / reset
  uint64_t submitted = 0, completed = 0, failed = 0, bytes_ckpt = 0, bytes_restored = 0;
  std::vector<double> lat_all, lat_ckpt, lat_restore;
  Clock::time_point t_first{}, t_last{};
  bool have_first = false;
  uint32_t peak_inflight = 0;
  std::shared_ptr<crum::DrainSequencer> sequencer;  // cfg.serialize_drains
};

namespace {

crum_status srv_fail(crum_status st, const char* msg) {
  crum::set_last_error(msg);
  return st;
}

// First-fit over the pool; 256-byte aligned regions.
bool region_alloc(crum_server* S, uint64_t len, uint64_t* off) {
  len = (len + 255) & ~uint64_t(255);
  for (auto it = S->free_list.begin(); it != S->free_list.end(); ++it) {
    if (it->second >= len) {
      *off = it->first;
      const uint64_t rest = it->second - len, at = it->first + len;
      S->free_list.erase(it);
      if (rest) S->free_list.emplace(at, rest);
      S->lent += len;
      S->peak_lent = std::max(S->peak_lent, S->lent);
      return true;
    }
  }
  return false;
}

void region_free(crum_server* S, uint64_t off, uint64_t len) {
  len = (len + 255) & ~uint64_t(255);
  S->lent -= len;
  auto next = S->free_list.lower_bound(off);
  if (next != S->free_list.end() && next->first == off + len) {
    len += next->second;
    next = S->free_list.erase(next);
  }
  if (next != S->free_list.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == off) {
      off = prev->first;
      len += prev->second;
      S->free_list.erase(prev);
    }
  }
  S->free_list.emplace(off, len);
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q / 100.0 * (v.size() - 1);
  const size_t lo = static_cast<size_t>(pos);
  const size_t hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (v[hi] - v[lo]) * (pos - lo);
}

void finish(crum_server* S, Request& r, crum_status st) {
  r.state = 2;
  r.status = st;
  r.t_done = Clock::now();
  Client& c = S->clients[r.client];
  c.busy = false;
  crum::bind_staging(c.set, nullptr, 0);
  region_free(S, r.region_off, r.region_len);
  if (r.ev_done) {
    cudaEventDestroy(r.ev_done);
    r.ev_done = nullptr;
  }
  const double ms = ms_between(r.t_submit, r.t_done);
  if (st == CRUM_OK || st == CRUM_ECOLLISION) {
    S->completed++;
    S->lat_all.push_back(ms);
    if (r.kind == CRUM_REQ_RESTORE) {
      S->lat_restore.push_back(ms);
      S->bytes_restored += r.bytes;
    } else {
      S->lat_ckpt.push_back(ms);
      S->bytes_ckpt += c.pages * crum::kPage;
    }
  } else {
    S->failed++;
  }
  S->t_last = r.t_done;
}

bool done_failed(crum_status st) { return st != CRUM_OK && st != CRUM_ECOLLISION; }

// Drops the images completed requests still hold (server lock held).
void drop_kept_images(crum_server* S) {
  for (auto& kv : S->reqs) {
    Request& r = kv.second;
    if (r.state == 2 && r.img != nullptr) {
      crum_image_release(r.img);
      r.img = nullptr;
    }
  }
}

// Polls running requests for completion (server lock held).
void poll_running(crum_server* S) {
  for (size_t i = 0; i < S->running.size();) {
    Request& r = S->reqs[S->running[i]];
    bool done = false;
    crum_status st = CRUM_OK;
    if (r.kind == CRUM_REQ_RESTORE) {
      const cudaError_t e = cudaEventQuery(r.ev_done);
      if (e == cudaSuccess) {
        done = true;
        r.captured = true;
      } else if (e != cudaErrorNotReady) {
        done = true;
        st = CRUM_ECUDA;
      }
    } else {
      if (!r.captured && cudaEventQuery(r.img->ev_captured) == cudaSuccess) r.captured = true;
      crum_image_info info;
      crum_image_info_get(r.img, &info);
      if (info.stage >= CRUM_WAIT_PERSISTED ||
          (info.status != CRUM_OK && info.status != CRUM_ECOLLISION)) {
        done = true;
        st = static_cast<crum_status>(info.status);
        r.captured = true;
        r.n_dirty = info.n_dirty;
        r.bytes = info.image_bytes;
        r.image_seq = info.seq;
        r.checksum = info.checksum;
        if (!S->cfg.keep_images || done_failed(st)) {
          crum_image_release(r.img);
          r.img = nullptr;
        }
      }
    }
    if (done) {
      finish(S, r, st);
      S->running[i] = S->running.back();
      S->running.pop_back();
      S->done_cv.notify_all();
    } else {
      ++i;
    }
  }
}

// Starts one admitted request (server lock held; engine calls only enqueue).
crum_status start(crum_server* S, Request& r) {
  Client& c = S->clients[r.client];
  crum_status st = crum::bind_staging(c.set, S->pool + r.region_off, c.pages);
  if (st != CRUM_OK) return st;
  if (r.kind == CRUM_REQ_RESTORE) {
    if (c.newest == nullptr) return srv_fail(CRUM_EINVAL, "restore request before any checkpoint");
    st = crum_restore(c.set, c.newest, c.stream);
    if (st != CRUM_OK) return st;
    if (cudaEventCreateWithFlags(&r.ev_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(r.ev_done, c.stream) != cudaSuccess)
      return srv_fail(CRUM_ECUDA, "cannot record restore completion");
    crum_image_info info;
    crum_image_info_get(c.newest, &info);
    r.image_seq = info.seq;
    for (crum_image* p = c.newest; p != nullptr; p = p->parent) {
      r.n_dirty += p->n_dirty;
      if (p->full) break;
    }
    r.bytes = r.n_dirty * crum::kPage;
    return CRUM_OK;
  }
  crum_image* img = nullptr;
  st = crum_checkpoint(c.set, c.stream, r.kind == CRUM_REQ_CHECKPOINT_FULL ? CRUM_FULL : CRUM_INCR,
                       &img);
  if (st != CRUM_OK) return st;
  r.img = img;
  // the client's newest image: a second reference, dropped when replaced
  img->refs.fetch_add(1);
  if (c.newest) crum_image_release(c.newest);
  c.newest = img;
  return CRUM_OK;
}

// Admits request r (server lock held): lends its staging region, starts it.
void launch(crum_server* S, Request& r, int* n_ckpt, int* n_rest) {
  crum::TraceRange tr(r.kind == CRUM_REQ_RESTORE ? "crum server restore" : "crum server checkpoint");
  Client& c = S->clients[r.client];
  r.state = 1;
  r.t_admit = Clock::now();
  c.busy = true;
  const crum_status st = start(S, r);
  if (st != CRUM_OK) {
    finish(S, r, st);
    S->done_cv.notify_all();
  } else {
    S->running.push_back(r.id);
    (r.kind == CRUM_REQ_RESTORE ? *n_rest : *n_ckpt)++;
    S->peak_inflight = std::max<uint32_t>(S->peak_inflight, S->running.size());
  }
}

// Admission by expected transfer (crum_server_config.order = 1): among the
// oldest pending request of every idle client, within the lanes, the one
// whose client footprint would take least time across the link, less the
// time it has waited (so a large request is not passed over for ever: once
// it has waited longer than its transfer would take, it also keeps smaller
// requests from taking the staging memory it waits for).  A burst of small
// requests then no longer queues behind a few long drains.
void admit_by_size(crum_server* S) {
  int n_ckpt = 0, n_rest = 0;
  for (uint64_t id : S->running) (S->reqs[id].kind == CRUM_REQ_RESTORE ? n_rest : n_ckpt)++;
  constexpr double kBytesPerMs = 50e6;  // the host link's order of magnitude
  const auto now = Clock::now();
  while (S->running.size() < static_cast<size_t>(S->cfg.max_inflight)) {
    std::vector<bool> seen(S->clients.size(), false);
    std::vector<std::pair<double, std::deque<uint64_t>::iterator>> cand;
    for (auto it = S->pending.begin(); it != S->pending.end(); ++it) {
      Request& r = S->reqs[*it];
      if (seen[r.client]) continue;  // a client's requests run in arrival order
      seen[r.client] = true;
      const Client& c = S->clients[r.client];
      if (c.busy) continue;
      const int k = r.kind == CRUM_REQ_RESTORE ? 1 : 0;
      const int lim = k ? S->cfg.max_restores : S->cfg.max_checkpoints;
      if (lim > 0 && (k ? n_rest : n_ckpt) >= lim) continue;
      const double key = c.pages * crum::kPage / kBytesPerMs - ms_between(r.t_submit, now);
      cand.emplace_back(key, it);
    }
    if (cand.empty()) return;
    std::sort(cand.begin(), cand.end(),
              [](const auto& a, const auto& b) { return a.first < b.first; });
    bool admitted = false;
    for (auto& kv : cand) {
      Request& r = S->reqs[*kv.second];
      r.region_len = S->clients[r.client].pages * crum::kPage;
      if (!region_alloc(S, r.region_len, &r.region_off)) {
        // a request that has waited longer than its own transfer would take
        // holds the budget's next free memory: nothing smaller passes it
        if (kv.first <= 0) return;
        continue;
      }
      S->pending.erase(kv.second);
      launch(S, r, &n_ckpt, &n_rest);
      admitted = true;
      break;  // the candidates' iterators are stale now
    }
    if (!admitted) return;
  }
}

void admit(crum_server* S) {
  if (S->cfg.order == 1) {
    admit_by_size(S);
    return;
  }
  std::vector<bool> blocked(S->clients.size(), false);
  int n_ckpt = 0, n_rest = 0;
  for (uint64_t id : S->running) (S->reqs[id].kind == CRUM_REQ_RESTORE ? n_rest : n_ckpt)++;
  bool kind_full[2] = {false, false};  // a kind at its limit stops its queue, in order
  for (auto it = S->pending.begin(); it != S->pending.end();) {
    if (S->running.size() >= static_cast<size_t>(S->cfg.max_inflight)) break;
    Request& r = S->reqs[*it];
    Client& c = S->clients[r.client];
    const int k = r.kind == CRUM_REQ_RESTORE ? 1 : 0;
    const int lim = k ? S->cfg.max_restores : S->cfg.max_checkpoints;
    if (kind_full[k] || (lim > 0 && (k ? n_rest : n_ckpt) >= lim)) {
      kind_full[k] = true;
      blocked[r.client] = true;
      ++it;
      continue;
    }
    if (c.busy || blocked[r.client]) {
      blocked[r.client] = true;  // keep this client's later requests behind this one
      ++it;
      continue;
    }
    r.region_len = c.pages * crum::kPage;
    if (!region_alloc(S, r.region_len, &r.region_off)) break;  // wait for memory, in order
    it = S->pending.erase(it);
    launch(S, r, &n_ckpt, &n_rest);
  }
}

void server_main(crum_server* S) {
  cudaSetDevice(S->cfg.device);
  crum::trace_name_thread("crum server");
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    poll_running(S);
    admit(S);
    if (S->stop && S->pending.empty() && S->running.empty()) return;
    if (S->running.empty() && S->pending.empty())
      S->wake.wait_for(lk, std::chrono::milliseconds(50));
    else
      S->wake.wait_for(lk, std::chrono::microseconds(20));
  }
}

void fill_info(const Request& r, crum_request_info* info) {
  std::memset(info, 0, sizeof *info);
  info->id = r.id;
  info->client = r.client;
  info->kind = r.kind;
  info->done = r.state == 2;
  info->status = r.state == 2 ? r.status : CRUM_ETIMEOUT;
  info->n_dirty = r.n_dirty;
  info->bytes = r.bytes;
  info->image_seq = r.image_seq;
  info->checksum = r.checksum;
  if (r.state >= 1) info->t_queue_ms = ms_between(r.t_submit, r.t_admit);
  if (r.state == 2) info->t_total_ms = ms_between(r.t_submit, r.t_done);
}

}  // namespace

extern "C" {

crum_status crum_server_create(const crum_server_config* cfg, crum_server** out) {
  if (out == nullptr) return srv_fail(CRUM_EINVAL, "out is null");
  *out = nullptr;
  auto S = std::make_unique<crum_server>();
  if (cfg) S->cfg = *cfg;
  if (S->cfg.staging_budget == 0) S->cfg.staging_budget = 16ull << 30;
  if (S->cfg.max_inflight <= 0) S->cfg.max_inflight = 8;
  S->cfg.serialize_drains = S->cfg.serialize_drains >= 0 ? 1 : 0;
  // per-kind limits: 0 means the default (two checkpoints when their drains
  // are serialized, else one; one restore), negative means none
  if (S->cfg.max_checkpoints == 0) S->cfg.max_checkpoints = S->cfg.serialize_drains ? 2 : 1;
  if (S->cfg.max_restores == 0) S->cfg.max_restores = 1;
  if (S->cfg.max_checkpoints < 0) S->cfg.max_checkpoints = 0;
  if (S->cfg.max_restores < 0) S->cfg.max_restores = 0;
  S->cfg.staging_budget &= ~uint64_t(255);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || S->cfg.device < 0 || S->cfg.device >= ndev) {
    cudaGetLastError();
    return srv_fail(CRUM_EINVAL, "no such CUDA device");
  }
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(S->cfg.device);
  const cudaError_t e = cudaMalloc(&S->pool, S->cfg.staging_budget);
  cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return srv_fail(CRUM_ENOMEM, "cannot allocate the staging budget");
  }
  S->free_list.emplace(0, S->cfg.staging_budget);
  if (S->cfg.serialize_drains) S->sequencer = std::make_shared<crum::DrainSequencer>();
  crum_server* raw = S.release();
  raw->th = std::thread(server_main, raw);
  *out = raw;
  return CRUM_OK;
}

crum_status crum_server_destroy(crum_server* S) {
  if (S == nullptr) return CRUM_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->wake.notify_all();
  }
  if (S->th.joinable()) S->th.join();
  drop_kept_images(S);
  for (Client& c : S->clients) {
    if (c.newest) crum_image_release(c.newest);
    if (S->sequencer) crum::set_drain_sequencer(c.set, nullptr);
  }
  cudaFree(S->pool);
  delete S;
  return CRUM_OK;
}

crum_status crum_server_add_client(crum_server* S, crum_set* set, crum_stream_t app_stream,
                                   uint32_t* client_id) {
  if (S == nullptr || set == nullptr) return srv_fail(CRUM_EINVAL, "null server or set");
  if (!set->cfg.external_staging) return srv_fail(CRUM_EINVAL, "client set must use external staging");
  uint32_t n_allocs = 0;
  uint64_t pages = 0;
  crum_set_info(set, &n_allocs, &pages);
  if (pages == 0) return srv_fail(CRUM_EINVAL, "client set has no registrations");
  std::lock_guard<std::mutex> lk(S->mu);
  if (pages * crum::kPage > S->cfg.staging_budget)
    return srv_fail(CRUM_EINVAL, "client footprint exceeds the whole staging budget");
  if (S->sequencer && crum::set_drain_sequencer(set, S->sequencer) != CRUM_OK)
    return srv_fail(CRUM_EBUSY, "client set has checkpoints in flight");
  Client c;
  c.set = set;
  c.stream = static_cast<cudaStream_t>(app_stream);
  c.pages = pages;
  S->clients.push_back(c);
  if (client_id) *client_id = static_cast<uint32_t>(S->clients.size() - 1);
  return CRUM_OK;
}

crum_status crum_server_submit(crum_server* S, uint32_t client, int kind, uint64_t* request_id) {
  if (S == nullptr || kind < CRUM_REQ_CHECKPOINT || kind > CRUM_REQ_RESTORE)
    return srv_fail(CRUM_EINVAL, "bad server or request kind");
  std::lock_guard<std::mutex> lk(S->mu);
  if (client >= S->clients.size()) return srv_fail(CRUM_EINVAL, "unknown client");
  Request r;
  r.id = S->next_id++;
  r.client = client;
  r.kind = kind;
  r.t_submit = Clock::now();
  if (!S->have_first) {
    S->t_first = r.t_submit;
    S->have_first = true;
  }
  S->reqs.emplace(r.id, r);
  S->pending.push_back(r.id);
  S->submitted++;
  if (request_id) *request_id = r.id;
  S->wake.notify_all();
  return CRUM_OK;
}

crum_status crum_server_wait(crum_server* S, uint64_t id, int stage, int64_t timeout_ns,
                             crum_request_info* info) {
  if (S == nullptr) return srv_fail(CRUM_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return srv_fail(CRUM_EINVAL, "unknown request");
  auto ready = [&] {
    const Request& r = S->reqs[id];
    return r.state == 2 || (stage == CRUM_WAIT_CAPTURED && r.captured);
  };
  if (timeout_ns < 0) {
    S->done_cv.wait(lk, ready);
  } else if (!S->done_cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns), ready)) {
    if (info) fill_info(S->reqs[id], info);
    return srv_fail(CRUM_ETIMEOUT, "request still running");
  }
  const Request& r = S->reqs[id];
  if (info) fill_info(r, info);
  if (r.state != 2) return CRUM_OK;  // captured, still draining
  return r.status;
}

crum_status crum_server_take_image(crum_server* S, uint64_t id, crum_image** out) {
  if (S == nullptr || out == nullptr) return srv_fail(CRUM_EINVAL, "null server or out");
  *out = nullptr;
  std::lock_guard<std::mutex> lk(S->mu);
  if (!S->cfg.keep_images) return srv_fail(CRUM_EINVAL, "server created without keep_images");
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return srv_fail(CRUM_EINVAL, "unknown request");
  Request& r = it->second;
  if (r.kind == CRUM_REQ_RESTORE) return srv_fail(CRUM_EINVAL, "a restore request has no image");
  if (r.state != 2) return srv_fail(CRUM_EINVAL, "request not finished");
  if (r.img == nullptr) return srv_fail(CRUM_EINVAL, "image already taken, or the request failed");
  *out = r.img;  // the server's reference passes to the caller
  r.img = nullptr;
  return CRUM_OK;
}

crum_status crum_server_drain(crum_server* S, crum_server_stats* st) {
  if (S == nullptr) return srv_fail(CRUM_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(S->mu);
  S->done_cv.wait(lk, [&] { return S->pending.empty() && S->running.empty(); });
  if (st) {
    std::memset(st, 0, sizeof *st);
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->failed = S->failed;
    st->bytes_checkpointed = S->bytes_ckpt;
    st->bytes_restored = S->bytes_restored;
    st->p50_ms = percentile(S->lat_all, 50);
    st->p99_ms = percentile(S->lat_all, 99);
    st->p50_ckpt_ms = percentile(S->lat_ckpt, 50);
    st->p99_ckpt_ms = percentile(S->lat_ckpt, 99);
    st->p50_restore_ms = percentile(S->lat_restore, 50);
    st->p99_restore_ms = percentile(S->lat_restore, 99);
    st->wall_ms = S->have_first ? ms_between(S->t_first, S->t_last) : 0.0;
    st->peak_inflight = S->peak_inflight;
    st->peak_staging = S->peak_lent;
  }
  return CRUM_OK;
}

crum_status crum_server_reset_stats(crum_server* S) {
  if (S == nullptr) return srv_fail(CRUM_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(S->mu);
  S->done_cv.wait(lk, [&] { return S->pending.empty() && S->running.empty(); });
  drop_kept_images(S);
  S->reqs.clear();
  S->submitted = S->completed = S->failed = S->bytes_ckpt = S->bytes_restored = 0;
  S->lat_all.clear();
  S->lat_ckpt.clear();
  S->lat_restore.clear();
  S->have_first = false;
  S->peak_inflight = 0;
  S->peak_lent = S->lent;
  return CRUM_OK;
}

}  // extern "C"
