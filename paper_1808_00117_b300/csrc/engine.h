// Host-side state of registration sets and images (internal).
//
// The paper's checkpoint (Section 3.4) copies every region device -> host
// after draining the device, and its forked checkpoint (Section 3.3) lets a
// child process write the image while the application continues.  Here the
// "child" is three host threads per set:
//   planner  learns each capture's dirty count from a mapped pinned mailbox,
//            sizes the image and queues the device->host drain on the drain
//            stream;
//   drainer  marks each image DRAINED when its copies are done;
//   writer   persists drained images to files (memory and null sinks need
//            no writer), so slow storage never delays DRAINED.
// The application's stream only waits for the device-side capture (hash,
// scan, gather into staging); the staging buffer is split in two halves
// that alternate between consecutive checkpoints so a capture never waits
// for the previous checkpoint's drain unless both halves are busy.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>
#include <sys/syscall.h>
#include <unistd.h>

#include "crum.h"
#include "device.cuh"
#include "kernels.h"
#include "restore_codec.h"

namespace crum {

// A named range on the calling thread's NVTX timeline, for a profiler that
// records host ranges (Nsight Systems); without one attached, push and pop
// are a test of a function pointer.
class TraceRange {
 public:
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// Names the calling OS thread on that timeline.
inline void trace_name_thread(const char* name) {
  nvtxNameOsThreadA(static_cast<uint32_t>(syscall(SYS_gettid)), name);
}

// First-fit allocator over cudaHostAlloc arenas (pinning is slow: about
// 0.35 s per GiB, so images draw from a pool instead of pinning per image).
class PinnedPool {
 public:
  explicit PinnedPool(size_t initial);
  ~PinnedPool();
  uint8_t* alloc(size_t n);  // nullptr on failure
  void free(uint8_t* p, size_t n);
  size_t reserved() const { return reserved_; }

 private:
  struct Arena {
    uint8_t* base;
    size_t size;
    std::map<size_t, size_t> free_list;  // offset -> length
  };
  std::mutex mu_;
  std::vector<Arena> arenas_;
  size_t reserved_ = 0;
  size_t initial_;
};

struct Alloc {
  uint32_t id;
  uint8_t* ptr;
  uint64_t bytes;
  uint64_t n_pages;
  uint64_t first_page;
  bool managed = false;   // managed (unified) memory
  bool advised = false;   // the set added cudaMemAdviseSetAccessedBy for its device
};

struct Half {
  uint8_t* meta = nullptr;     // header, allocation table, page table, hashes
  size_t meta_cap = 0;
  uint8_t* payload = nullptr;  // half_slots pages
  uint64_t* scalars = nullptr; // device: [0] n_dirty, [1] trailer
  uint64_t* mailbox = nullptr; // mapped pinned host: [0] n_dirty
  uint64_t* mailbox_dev = nullptr;
  cudaEvent_t ev_scanned = nullptr;
  cudaEvent_t ev_drained = nullptr;  // last device->host copy out of this half
  bool drain_enqueued = true;        // host: ev_drained is recorded for its last user
  // compressed images (cfg.compress)
  uint8_t* cpay = nullptr;           // encoded payload
  uint32_t* enc_len = nullptr;       // encoded length of every slot
  uint8_t* alph = nullptr;           // every slot's alphabets, size kernel -> encoder
  uint64_t* ctotal = nullptr;        // device: encoded payload bytes
  uint64_t* cn = nullptr;            // device: [0] slots of a chunk, [1] scratch
  cudaEvent_t ev_sized = nullptr;    // encoded sizes, offsets and header written
  cudaEvent_t ev_encoded = nullptr;  // encoded payload and checksum written
};

// The capture sequence of one staging half as an instantiated CUDA graph:
// memset(bitmap), memset(counters), record k0, hash, record k1,
// wait(half drained), record k2, scan, record scanned, gather,
// record captured.  Kernel arguments and the per-image events are set on
// the executable graph before each launch; `epoch` says which registration
// and buffer layout it was built for.
struct CaptureGraph {
  cudaGraph_t graph = nullptr;  // kept: node handles below belong to it
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t k0 = nullptr, k1 = nullptr, k2 = nullptr, captured = nullptr;
  cudaGraphNode_t encoded = nullptr;  // compressed sets: end of the encoding stage
  cudaGraphNode_t hash = nullptr, scan = nullptr, gather = nullptr;
  KernelSpec hs{}, ss{}, gs{};
  // events the record nodes hold between launches (an image's events are
  // set only for its own launch: images, and their events, die earlier)
  cudaEvent_t placeholder[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  uint64_t epoch = 0;
};

// Orders the device->host drains of several sets (a server's clients) so
// they cross the link one at a time, in the order the checkpoints were
// submitted, while their captures may overlap.  Each drain waits on the
// device for the previous one (one event, re-recorded by each drain) and,
// on the host, for its turn to be queued.
struct DrainSequencer {
  std::mutex mu;
  std::condition_variable cv;
  uint64_t issued = 0;  // tickets handed out
  uint64_t next = 0;    // ticket whose drain may be queued now
  cudaEvent_t tail = nullptr;  // recorded after the last queued drain
  bool tail_recorded = false;
  ~DrainSequencer() {
    if (tail) cudaEventDestroy(tail);
  }
};

}  // namespace crum

struct crum_image {
  std::atomic<int> refs{1};
  std::shared_ptr<crum::PinnedPool> pool;
  crum_image* parent = nullptr;  // holds a reference
  int device = 0;
  uint64_t seq = 0, parent_seq = CRUM_NO_PARENT;
  bool full = false;
  uint32_t n_allocs = 0;
  uint64_t n_pages = 0;
  std::vector<std::pair<uint32_t, uint64_t>> table;  // (id, bytes) per allocation
  uint64_t n_dirty = 0, image_bytes = 0, checksum = 0, collisions = 0;
  uint8_t* host = nullptr;  // serialized image in pinned host memory
  size_t host_len = 0;
  std::mutex mu;
  std::condition_variable cv;
  int stage = 0;
  crum_status status = CRUM_OK;
  std::string err;
  cudaEvent_t ev_submit = nullptr, ev_captured = nullptr, ev_drained = nullptr;
  // phase timing: hash kernel [ev_k0, ev_k1], compaction [ev_k2, ev_captured]
  // (ev_k2 is taken once the staging half is free), drain [ev_d0, ev_drained]
  cudaEvent_t ev_k0 = nullptr, ev_k1 = nullptr, ev_k2 = nullptr, ev_d0 = nullptr;
  cudaEvent_t ev_e1 = nullptr;  // compressed: encoding stage done [ev_captured, ev_e1]
  std::chrono::steady_clock::time_point t_submit;
  double t_captured_ms = 0, t_drained_ms = 0, t_persisted_ms = 0;
  double t_hash_ms = 0, t_compact_ms = 0, t_drain_ms = 0, t_encode_ms = 0;
  int half = 0;
  bool drop_payload = false;  // null sink
  int64_t ticket = -1;        // drain order under a DrainSequencer
  bool compressed = false;    // version 2 image
  uint64_t payload_off = 0;   // compressed: where the encoded payload starts
  uint64_t payload_bytes = 0; // compressed: encoded payload bytes
  uint64_t host_pages = 0;    // pages read in place from host-placed managed memory
  std::string sink_path;
  bool do_fsync = false;
};

struct crum_set {
  crum_config cfg{};
  std::string sink_dir;
  int device = 0;
  uint32_t set_id = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::vector<crum::Alloc> allocs;
  uint32_t next_id = 0;
  uint64_t n_pages = 0;
  bool table_dirty = true;
  bool reg_changed = true;
  // device state
  crum::DevAlloc* d_allocs = nullptr;
  uint64_t* d_first_page = nullptr;
  size_t alloc_cap = 0;
  uint64_t* d_h = nullptr;
  size_t h_cap = 0;
  uint32_t* d_mask = nullptr;
  uint32_t* d_word_offset = nullptr;
  size_t words_cap = 0;
  unsigned long long* d_collisions = nullptr;
  uint8_t* d_shadow = nullptr;
  size_t shadow_cap = 0;  // pages
  uint64_t* d_owner = nullptr;  // merged restore: newest image slot of each page
  size_t owner_cap = 0;         // pages
  crum::ChainImage* d_chain = nullptr;
  size_t chain_cap = 0;         // images
  uint64_t* d_cur = nullptr;    // delta restore: current hash of every page
  size_t cur_cap = 0;           // pages
  unsigned long long* d_copied = nullptr;  // merged restore: pages copied across the link
  uint64_t restore_pages = 0;   // replay restore: pages copied across the link
  bool restore_counted_on_device = false;
  crum::Half half[2];
  int next_half = 0;
  uint64_t half_slots = 0;
  cudaStream_t cap_stream = nullptr, drain_stream = nullptr;
  cudaEvent_t ev_app = nullptr, ev_done = nullptr;
  int map_hash = 1, map_gather = 4;  // defaults until crum_autotune or the config
  crum::CaptureGraph graph[2];       // per staging half (cfg.use_graph)
  uint64_t graph_epoch = 1;          // bumped whenever a graph must be rebuilt
  // chain state
  uint64_t seq = 0;
  uint64_t chain_len = 0;  // incremental images since the newest full one
  crum_image* last = nullptr;
  bool needs_full = true;
  // background threads
  std::shared_ptr<crum::PinnedPool> pool;
  // pinned landing region of every payload that is not kept (null sink,
  // CRUM_NO_PAYLOAD): its bytes still cross the link, in region-sized
  // copies on the drain stream, and are overwritten by the next copy
  uint8_t* bounce = nullptr;
  std::mutex bounce_mu;
  std::shared_ptr<crum::DrainSequencer> sequencer;  // set by a server
  std::deque<crum_image*> plan_q, done_q, write_q;
  std::condition_variable plan_cv, done_cv, write_cv;
  std::thread planner, drainer, writer;
  bool stop = false;
  int inflight = 0;
};
