// C ABI of the PBD-R library: context, packed scene table, step plans and the
// host side of one substep.  See include/pbdr.h for the contract of every
// entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <vector>

#include "pbdr_internal.cuh"

using namespace pbdr;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

#define CUDA_TRY(expr)                                                              \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? PBDR_ERR_OOM : PBDR_ERR_CUDA,   \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));              \
  } while (0)

// page-locked host memory (grow-only staging for uploads)
struct PinnedBuf {
  void *p = nullptr;
  size_t bytes = 0;
  PinnedBuf() = default;
  PinnedBuf(const PinnedBuf &) = delete;
  PinnedBuf &operator=(const PinnedBuf &) = delete;
  ~PinnedBuf() {
    if (p) cudaFreeHost(p);
  }
  cudaError_t grow(size_t n) {
    if (bytes >= n) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    bytes = 0;
    const cudaError_t e = cudaHostAlloc(&p, n, cudaHostAllocDefault);
    if (e != cudaSuccess) {
      p = nullptr;
      return e;
    }
    bytes = n;
    return cudaSuccess;
  }
};

// Page-locked staging for the small host-to-device tables of a call (plan
// tables, segment tables, scene ids), used round-robin: a copy from pageable
// memory may make the driver synchronise with the stream it is issued on,
// which would hold the host until earlier work there (a substep) finishes.
// A slot is reused once the copy that last read it has completed.
// A few host threads kept for the lifetime of a context, so that scene
// set-up can split its per-particle pass without starting threads per call.
// run(n, f) calls f(0) .. f(n-1) on the workers and the calling thread and
// returns when all have finished.
class HostPool {
 public:
  explicit HostPool(int workers) {
    for (int i = 0; i < workers; ++i) th_.emplace_back([this] { loop(); });
  }
  HostPool(const HostPool &) = delete;
  HostPool &operator=(const HostPool &) = delete;
  ~HostPool() {
    {
      std::lock_guard<std::mutex> g(m_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto &t : th_) t.join();
  }
  int size() const { return (int)th_.size() + 1; }
  void run(int n, const std::function<void(int)> &f) {
    {
      std::lock_guard<std::mutex> g(m_);
      job_ = &f;
      n_ = n;
      next_ = 0;
      left_ = n;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> g(m_);
    done_.wait(g, [this] { return left_ == 0; });
    job_ = nullptr;
  }

 private:
  // takes and runs tasks of the current job until none is left
  void work() {
    for (;;) {
      const std::function<void(int)> *f;
      int t;
      {
        std::lock_guard<std::mutex> g(m_);
        if (!job_ || next_ >= n_) return;
        f = job_;
        t = next_++;
      }
      (*f)(t);
      std::lock_guard<std::mutex> g(m_);
      if (--left_ == 0) done_.notify_all();
    }
  }
  void loop() {
    for (;;) {
      {
        std::unique_lock<std::mutex> g(m_);
        cv_.wait(g, [this] { return stop_ || (job_ && next_ < n_); });
        if (stop_) return;
      }
      work();
    }
  }
  std::vector<std::thread> th_;
  std::mutex m_;
  std::condition_variable cv_, done_;
  const std::function<void(int)> *job_ = nullptr;
  int n_ = 0, next_ = 0, left_ = 0;
  bool stop_ = false;
};

struct StageRing {
  static constexpr int kSlots = 8;
  PinnedBuf buf[kSlots];
  cudaEvent_t ev[kSlots] = {};
  int next = 0;
  StageRing() = default;
  StageRing(const StageRing &) = delete;
  StageRing &operator=(const StageRing &) = delete;
  ~StageRing() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
  }
};

// owned device allocation
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class T>
  T *as() const { return reinterpret_cast<T *>(p); }
};

uint32_t table_size(int32_t n) {
  uint32_t want = (uint32_t)std::max(n, 1) * 2u;
  uint32_t t = 1;
  while (t < want) t <<= 1;
  return t;
}

// First-fit allocator of index ranges of the packed particle, body and chunk
// tables: destroyed scenes return their ranges, new scenes reuse them.
struct RangeAlloc {
  int32_t top = 0;                      // high-water mark
  std::map<int32_t, int32_t> free_;     // start -> length
  int32_t take(int32_t n) {             // first fit, or -1
    if (n <= 0) return top;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        const int32_t st = it->first, len = it->second;
        free_.erase(it);
        if (len > n) free_[st + n] = len - n;
        return st;
      }
    }
    return -1;
  }
  void give(int32_t st, int32_t n) {
    if (n <= 0) return;
    auto it = free_.emplace(st, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct SceneHost {
  bool alive = false;
  int32_t p0 = 0, np = 0, b0 = 0, nb = 0;
  ScenePar par{};
  int wrench_bodies = 0;
  int32_t c0 = 0, nc = 0;          // chunk range
  uint64_t last_step = 0;          // sequence number of the last step or asynchronous read of it (0: none)
};

// A step plan: the host-side description of one batched substep over a list
// of scenes.  Plans own no device memory: their small tables (hash bases,
// segment tables, wrench and class lists) live in `tab` and are copied into
// the context's table buffer, in stream order, when the plan becomes the
// active one; the streaming form's sort and cell scratch is the context's.
// size classes of the scene-resident kernel (particle capacities below)
constexpr int kNumClasses = 4;
constexpr int kStepRing = 64;      // step events kept for the per-scene idle test

struct Plan {
  std::vector<int32_t> ids;
  int32_t np = 0, nb = 0;
  int32_t pbase = 0, bbase = 0;
  bool pcontig = true, bcontig = true;
  uint32_t T_total = 0;
  int key_bits = 0;
  std::vector<int32_t> wrench_list;
  int kmax = 0;
  bool std_any = false;
  std::vector<int64_t> seg_off;    // per plan scene: first plan particle (n+1)
  std::vector<uint32_t> hbase_host;
  int sorted_in_b = 0;             // where the last sort left its result
  // device tables (int32 words); offsets into tab, -1 = absent.  pseg/bseg:
  // nseg + 1 segment starts (plan index) followed by nseg global bases
  std::vector<int32_t> tab;
  int32_t o_hbase = -1, o_wlist = -1, o_pseg = -1, o_bseg = -1, nseg = 0;
  int32_t o_iorder = -1;           // streaming solver iterations: body order (global ids)
  // scene-resident form: size classes of scenes, each one persistent launch
  bool fused = false;
  struct FClass {
    int ncap = 0;
    bool dx_shared = true;
    bool v_shared = true;
    int threads = 256;
    int grid = 0;
    int32_t n = 0;
    std::vector<int32_t> ids;
    int32_t o_list = -1;           // offset of the scene list in tab
  };
  std::array<FClass, kNumClasses> classes;
  std::unique_ptr<Plan> rest;      // scenes too large for a class (streaming form)
  bool tuned = false;              // launch shapes picked by the autotuner
  cudaGraphExec_t graph = nullptr; // one substep, captured
  uint64_t graph_gen = 0;          // context buffer generation the graph saw
  int64_t graph_launches = 0;
  uint64_t last_use = 0;           // for least-recently-used eviction
  int64_t substeps_run = 0;
  Plan() = default;
  Plan(const Plan &) = delete;
  Plan &operator=(const Plan &) = delete;
  ~Plan() {
    if (graph) cudaGraphExecDestroy(graph);
  }
};

constexpr size_t kMaxCachedPlans = 1024;
constexpr int64_t kTuneAfter = 128;   // default substeps of a plan before its launch shapes are tuned

constexpr int kClassCaps[kNumClasses] = {1024, 2048, 4096, 8192};
constexpr int kClassThreads[kNumClasses] = {256, 256, 512, 512};
// dynamic shared memory a class layout may use: the 227 KB a CTA may opt in
// to, less 1 KB for the kernel's static shared variables
constexpr size_t kFusedSmemLimit = 226 * 1024;

}  // namespace

namespace pbdr {
int set_last_error(int code, const char *msg) {
  g_err = msg;
  return code;
}
}  // namespace pbdr

struct pbdr_ctx {
  int device = 0;
  // Library work per stream: an event recorded after the last call that
  // enqueued work on that stream.  pbdr_destroy_scene queries them to tell
  // whether the ranges it frees may still be in use on the device.
  std::vector<std::pair<cudaStream_t, cudaEvent_t>> work_ev;
  bool work_pending = false;   // some recorded work may not have completed
  bool work_unknown = false;   // an event could not be recorded: assume work in flight
  bool free_dirty = false;     // freed ranges may still be used by work in flight
  bool async_other = false;    // a call other than pbdr_step may have left work in flight
  // one event per pbdr_step call, recorded after its work, in a ring: a
  // scene whose last step's event has completed is no longer in use
  uint64_t step_seq = 0;
  cudaEvent_t step_ev[kStepRing] = {};
  size_t budget = 0;
  size_t used = 0;
  int32_t pcap = 0, bcap = 0, scap = 0;
  int32_t np_used = 0, nb_used = 0;   // high-water marks of the packed tables
  RangeAlloc pa, ba, ca;               // free ranges of particles, bodies, chunks
  int nbr_cap = 32;
  DevBuf X[2], V[2], Q, Xinit, pbody, nbr_cnt, nbr;
  DevBuf Xd[2], Vd[2];             // tangents of X, V (forward-mode derivative), lazily allocated
  DevBuf Xb[2], Vb[2], Ub;         // adjoints of X, V and of the contact corrections (reverse mode)
  DevBuf dmu;                      // per scene: tangent of the friction coefficient
  DevBuf adj_store;                // saved states of the reverse sweep
  DevBuf bodies, wrench, quat, bcom, biter, border;
  DevBuf dx_scratch, tickets, chunks, partials;
  int32_t ccap = 0, nc_used = 0;   // chunk (and partial-slot) capacity / use
  cudaStream_t cls_stream[kNumClasses] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kNumClasses] = {};
  cudaStream_t rest_stream = nullptr;   // the streaming form of a mixed plan, beside the classes
  cudaEvent_t ev_rest_join = nullptr;
  int path = 0;                    // 0: scene-resident where a scene fits, 1: streaming only
  bool use_graphs = true;          // replay a captured CUDA graph per substep
  bool autotune = true;            // time launch shapes on the first step of a plan
  int64_t tune_after = kTuneAfter; // substeps of a plan before it is tuned
  int fused_threads = 0;           // 0: per-class default
  int num_sms = 0;
  Plan *last_fused_plan = nullptr;
  DevBuf scenes, scene_err;
  std::vector<SceneHost> sh;
  std::vector<BodyRec> bh;
  std::vector<BodyWrench> wh;
  std::map<std::vector<int32_t>, std::unique_ptr<Plan>> plans;
  uint64_t use_clock = 0;
  // autotuned launch shapes by (size class, scenes in it): threads, dx, v, grid
  std::map<std::pair<int, int32_t>, std::array<int, 4>> tune_memo;
  // tables of the active plan and the streaming form's scratch (grow-only)
  DevBuf tab, s_keys_a, s_keys_b, s_vals_a, s_vals_b, s_hist, s_cells, s_spos, s_pmap, s_bmap;
  DevBuf s_bounds, s_near;         // streaming neighbour culling: body boxes, near bodies
  DevBuf s_ilist, s_icount;        // ... and the particles it leaves to search, their number
  const Plan *active = nullptr;
  uint64_t gen = 1;                // bumped whenever a device buffer moves (graphs recapture)
  Plan *last_nbr_plan = nullptr;
  int64_t last_launches = 0;
  DevBuf stage_pos, stage_vel, seg_p0, seg_off, err_ids, err_out;
  // scene uploads: pinned staging
  PinnedBuf up_stage;
  StageRing h2d_ring;              // small tables of other calls
  std::unique_ptr<HostPool> pool;  // host threads of scene set-up (started on first use)
  // stage profiling
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Mark { int stage; size_t e0, e1; int64_t launches; };
  std::vector<Mark> marks;
  double stage_ms[PBDR_NUM_STAGES] = {0};
  int64_t stage_launches[PBDR_NUM_STAGES] = {0};
};

namespace {

int dev_alloc(pbdr_ctx *c, DevBuf &b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return PBDR_OK;
  size_t freed = b.bytes;
  if (c->budget && c->used - freed + bytes > c->budget)
    return fail(PBDR_ERR_BUDGET, "device memory budget exceeded (" + std::to_string(c->used - freed + bytes) +
                                     " > " + std::to_string(c->budget) + " bytes)");
  b.release();
  c->used -= freed;
  ++c->gen;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return fail(PBDR_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  b.bytes = bytes;
  c->used += bytes;
  return PBDR_OK;
}

// grow-only scratch with 50 % headroom (within the budget), so that a
// working set that grows a little at a time (a server's resident requests)
// reallocates rarely: freeing the old buffer waits for the device
int dev_reserve(pbdr_ctx *c, DevBuf &b, size_t bytes) {
  if (b.bytes >= bytes) return PBDR_OK;
  const size_t want = bytes + bytes / 2;
  if (!c->budget || c->used - b.bytes + want <= c->budget) return dev_alloc(c, b, want);
  return dev_alloc(c, b, bytes);
}

void dev_free(pbdr_ctx *c, DevBuf &b) {
  if (b.p) ++c->gen;
  c->used -= b.bytes;
  b.release();
}

// copies `bytes` from host memory `src` (any kind) to device memory `dst`
// on stream s through the next slot of the staging ring
int staged_h2d(pbdr_ctx *c, void *dst, const void *src, size_t bytes, cudaStream_t s) {
  if (!bytes) return PBDR_OK;
  StageRing &R = c->h2d_ring;
  const int k = R.next;
  R.next = (k + 1) % StageRing::kSlots;
  if (R.ev[k])
    CUDA_TRY(cudaEventSynchronize(R.ev[k]));   // the slot's last copy has read it
  else
    CUDA_TRY(cudaEventCreateWithFlags(&R.ev[k], cudaEventDisableTiming));
  CUDA_TRY(R.buf[k].grow(bytes));
  std::memcpy(R.buf[k].p, src, bytes);
  CUDA_TRY(cudaMemcpyAsync(dst, R.buf[k].p, bytes, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaEventRecord(R.ev[k], s));
  return PBDR_OK;
}

// records that library work was enqueued on stream s
void note_work(pbdr_ctx *c, cudaStream_t s) {
  cudaEvent_t e = nullptr;
  for (auto &w : c->work_ev)
    if (w.first == s) e = w.second;
  if (!e) {
    // streams come and go (a caller may destroy its own): forget those whose
    // last work has completed before the list grows long
    if (c->work_ev.size() >= 16) {
      for (size_t k = 0; k < c->work_ev.size();) {
        if (cudaEventQuery(c->work_ev[k].second) == cudaSuccess) {
          cudaEventDestroy(c->work_ev[k].second);
          c->work_ev[k] = c->work_ev.back();
          c->work_ev.pop_back();
        } else {
          cudaGetLastError();
          ++k;
        }
      }
    }
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      c->work_unknown = c->work_pending = true;
      return;
    }
    c->work_ev.push_back({s, e});
  }
  if (cudaEventRecord(e, s) != cudaSuccess) {
    cudaGetLastError();
    c->work_unknown = true;
  }
  c->work_pending = true;
}

// true when every library call's work has completed (queries, never waits)
bool work_done(pbdr_ctx *c) {
  if (!c->work_pending) return true;
  if (c->work_unknown) return false;
  for (auto &w : c->work_ev) {
    const cudaError_t q = cudaEventQuery(w.second);
    if (q == cudaSuccess) continue;
    if (q != cudaErrorNotReady) cudaGetLastError();
    return false;
  }
  c->work_pending = false;
  return true;
}

// notes, when a call that took a stream returns, the work it enqueued there;
// a call whose work is complete when it returns (a read that synchronises)
// or that stamped its scenes (a step) sets `quiet`
struct WorkNote {
  pbdr_ctx *c;
  cudaStream_t s;
  bool quiet = false;
  ~WorkNote() {
    if (!c) return;
    note_work(c, s);
    if (!quiet) c->async_other = true;
  }
};

// after a successful pbdr_step (or asynchronous read) on stream s: records
// the call's event and stamps its scenes with the call's sequence number
void stamp_use(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, cudaStream_t s) {
  const uint64_t seq = ++c->step_seq;
  cudaEvent_t &e = c->step_ev[seq % kStepRing];
  if ((!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) ||
      cudaEventRecord(e, s) != cudaSuccess) {
    cudaGetLastError();
    c->async_other = true;   // the scenes' stamps would be stale: fall back to the global test
    return;
  }
  for (int32_t i = 0; i < n; ++i) c->sh[ids[i]].last_step = seq;
}

// true when no work enqueued by an earlier call can still touch the ranges
// of scene S (queries, never waits): its last step has completed and every
// other call's work has too
bool scene_idle(pbdr_ctx *c, const SceneHost &S) {
  if (c->async_other) {
    if (!work_done(c)) return false;
    c->async_other = false;
  }
  if (S.last_step == 0) return true;
  if (c->step_seq - S.last_step >= (uint64_t)kStepRing) return work_done(c);   // its event was reused
  const cudaError_t q = cudaEventQuery(c->step_ev[S.last_step % kStepRing]);
  if (q == cudaSuccess) return true;
  if (q != cudaErrorNotReady) cudaGetLastError();
  return false;
}

// grow `b` to `bytes`, keeping the first `keep` bytes
int dev_grow(pbdr_ctx *c, DevBuf &b, size_t bytes, size_t keep) {
  if (b.bytes >= bytes) return PBDR_OK;
  if (c->budget && c->used + bytes > c->budget)
    return fail(PBDR_ERR_BUDGET, "device memory budget exceeded");
  // kernels in flight on any stream may still use the old buffer
  if (b.p) CUDA_TRY(cudaDeviceSynchronize());
  void *np = nullptr;
  cudaError_t e = cudaMalloc(&np, bytes);
  if (e != cudaSuccess) return fail(PBDR_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  if (b.p && keep) {
    e = cudaMemcpy(np, b.p, std::min(keep, b.bytes), cudaMemcpyDeviceToDevice);
    // a device-to-device copy may still run when cudaMemcpy returns: finish
    // it before anything else writes the new buffer on another stream
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      cudaFree(np);
      return fail(PBDR_ERR_CUDA, std::string("cudaMemcpy: ") + cudaGetErrorString(e));
    }
  }
  c->used += bytes;
  dev_free(c, b);
  b.p = np;
  b.bytes = bytes;
  return PBDR_OK;
}

int ensure_capacity(pbdr_ctx *c, int32_t np_need, int32_t nb_need, int32_t ns_need, int32_t nc_need) {
  int rc;
  if (nc_need > c->ccap) {
    int32_t cap = std::max(nc_need, std::max(256, c->ccap * 2));
    if ((rc = dev_grow(c, c->chunks, (size_t)cap * sizeof(Chunk), (size_t)c->nc_used * sizeof(Chunk)))) return rc;
    if ((rc = dev_grow(c, c->partials, (size_t)cap * kPartialFloats * sizeof(float), 0))) return rc;
    c->ccap = cap;
  }
  if (np_need > c->pcap) {
    int32_t cap = std::max(np_need, std::max(1024, c->pcap * 2));
    size_t keep4 = (size_t)c->np_used * sizeof(float4);
    for (int k = 0; k < 2; ++k) {
      if ((rc = dev_grow(c, c->X[k], (size_t)cap * sizeof(float4), keep4))) return rc;
      if ((rc = dev_grow(c, c->V[k], (size_t)cap * sizeof(float4), keep4))) return rc;
    }
    if ((rc = dev_grow(c, c->Q, (size_t)cap * sizeof(float4), keep4))) return rc;
    if ((rc = dev_grow(c, c->pbody, (size_t)cap * sizeof(int32_t), (size_t)c->np_used * 4))) return rc;
    if ((rc = dev_grow(c, c->nbr_cnt, (size_t)cap * sizeof(int32_t), 0))) return rc;
    // neighbour slots are rebuilt every substep: no copy
    dev_free(c, c->nbr);
    if ((rc = dev_alloc(c, c->nbr, (size_t)cap * c->nbr_cap * sizeof(int32_t)))) return rc;
    if (c->Xinit.p) {
      dev_free(c, c->Xinit);
      if ((rc = dev_alloc(c, c->Xinit, (size_t)cap * sizeof(float4)))) return rc;
    }
    if (c->dx_scratch.p) {
      dev_free(c, c->dx_scratch);
      if ((rc = dev_alloc(c, c->dx_scratch, (size_t)cap * sizeof(float4)))) return rc;
    }
    c->pcap = cap;
  }
  if (nb_need > c->bcap) {
    int32_t cap = std::max(nb_need, std::max(256, c->bcap * 2));
    if ((rc = dev_grow(c, c->bodies, (size_t)cap * sizeof(BodyRec), (size_t)c->nb_used * sizeof(BodyRec)))) return rc;
    if ((rc = dev_grow(c, c->wrench, (size_t)cap * sizeof(BodyWrench), (size_t)c->nb_used * sizeof(BodyWrench)))) return rc;
    if ((rc = dev_grow(c, c->quat, (size_t)cap * sizeof(float4), (size_t)c->nb_used * sizeof(float4)))) return rc;
    if ((rc = dev_grow(c, c->bcom, (size_t)cap * sizeof(float4), (size_t)c->nb_used * sizeof(float4)))) return rc;
    if ((rc = dev_grow(c, c->biter, (size_t)cap * kBodyScratch * sizeof(float4), 0))) return rc;
    if ((rc = dev_grow(c, c->border, (size_t)cap * sizeof(int32_t), (size_t)c->nb_used * sizeof(int32_t)))) return rc;
    c->bcap = cap;
  }
  if (ns_need > c->scap) {
    int32_t cap = std::max(ns_need, std::max(64, c->scap * 2));
    size_t ns = c->sh.size();
    if ((rc = dev_grow(c, c->scenes, (size_t)cap * sizeof(ScenePar), ns * sizeof(ScenePar)))) return rc;
    if ((rc = dev_grow(c, c->scene_err, (size_t)cap * sizeof(uint32_t), ns * sizeof(uint32_t)))) return rc;
    c->scap = cap;
  }
  return PBDR_OK;
}

bool finite3(const float *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

int check_scene(pbdr_ctx *c, pbdr_scene s) {
  if (!c) return fail(PBDR_ERR_INVALID, "NULL context");
  if (s < 0 || s >= (int32_t)c->sh.size() || !c->sh[s].alive)
    return fail(PBDR_ERR_INVALID, "invalid scene handle " + std::to_string(s));
  return PBDR_OK;
}

// Validates ids (alive, no duplicates).
int check_ids(pbdr_ctx *c, const pbdr_scene *ids, int32_t n) {
  if (!ids || n < 1) return fail(PBDR_ERR_INVALID, "need at least one scene id");
  std::vector<char> seen(c->sh.size(), 0);
  for (int32_t i = 0; i < n; ++i) {
    int rc = check_scene(c, ids[i]);
    if (rc) return rc;
    if (seen[ids[i]]) return fail(PBDR_ERR_INVALID, "duplicate scene id " + std::to_string(ids[i]));
    seen[ids[i]] = 1;
  }
  return PBDR_OK;
}

// streaming-form plan of ids[0..n); its tables are appended to `tab` (the
// plan's own, or the parent scene-resident plan's)
int fill_stream_plan(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, Plan &P, std::vector<int32_t> &tab) {
  P.ids.assign(ids, ids + n);
  P.hbase_host.assign(std::max<size_t>(c->sh.size(), 1), 0u);
  P.seg_off.assign(1, 0);
  std::vector<int32_t> pstart(1, 0), pb0, bstart(1, 0), bb0;
  uint64_t tsum = 0;
  int32_t next_p = -1, next_b = -1;
  for (int32_t i = 0; i < n; ++i) {
    const SceneHost &S = c->sh[ids[i]];
    if (i == 0) {
      P.pbase = S.p0;
      P.bbase = S.b0;
    } else {
      if (S.p0 != next_p) P.pcontig = false;
      if (S.b0 != next_b) P.bcontig = false;
    }
    next_p = S.p0 + S.np;
    next_b = S.b0 + S.nb;
    P.hbase_host[ids[i]] = (uint32_t)tsum;
    tsum += S.par.T;
    if (tsum > 0xF0000000ull) return fail(PBDR_ERR_INVALID, "hash tables of one step exceed 2^32 buckets");
    P.np += S.np;
    P.nb += S.nb;
    P.seg_off.push_back(P.np);
    pstart.push_back(P.np);
    pb0.push_back(S.p0);
    bstart.push_back(P.nb);
    bb0.push_back(S.b0);
    P.kmax = std::max(P.kmax, S.par.iterations);
    P.std_any |= (S.par.flags & kStdVelocity) != 0;
    if (S.wrench_bodies)
      for (int32_t b = S.b0; b < S.b0 + S.nb; ++b)
        if (c->bh[b].has_wrench) P.wrench_list.push_back(b);
  }
  P.T_total = (uint32_t)tsum;
  int bits = 1;
  while (bits < 32 && (1ull << bits) < tsum) ++bits;
  P.key_bits = bits;
  P.nseg = n;
  P.o_hbase = (int32_t)tab.size();
  for (uint32_t h : P.hbase_host) tab.push_back((int32_t)h);
  if (!P.pcontig) {
    P.o_pseg = (int32_t)tab.size();
    tab.insert(tab.end(), pstart.begin(), pstart.end());
    tab.insert(tab.end(), pb0.begin(), pb0.end());
  }
  if (!P.bcontig) {
    P.o_bseg = (int32_t)tab.size();
    tab.insert(tab.end(), bstart.begin(), bstart.end());
    tab.insert(tab.end(), bb0.begin(), bb0.end());
  }
  {  // solver-iteration order: bodies by size bucket (floor of log2 of the
     // particle count), largest first, so that each launch ends on small
     // bodies (a counting sort: linear in the bodies of the plan)
    auto bucket = [&](int32_t b) { return 31 - __builtin_clz((unsigned)std::max(c->bh[b].count, 1)); };
    int32_t at[33] = {0};
    for (int32_t i = 0; i < n; ++i) {
      const SceneHost &S = c->sh[ids[i]];
      for (int32_t b = S.b0; b < S.b0 + S.nb; ++b) ++at[bucket(b)];
    }
    for (int32_t k = 32, run = 0; k >= 0; --k) {
      const int32_t m = at[k];
      at[k] = run;
      run += m;
    }
    P.o_iorder = (int32_t)tab.size();
    tab.resize(tab.size() + P.nb);
    int32_t *o = tab.data() + P.o_iorder;
    for (int32_t i = 0; i < n; ++i) {
      const SceneHost &S = c->sh[ids[i]];
      for (int32_t b = S.b0; b < S.b0 + S.nb; ++b) o[at[bucket(b)]++] = b;
    }
  }
  if (!P.wrench_list.empty()) {
    P.o_wlist = (int32_t)tab.size();
    tab.insert(tab.end(), P.wrench_list.begin(), P.wrench_list.end());
  }
  int rc;
  if (P.std_any && !c->Xinit.p) {
    if ((rc = dev_alloc(c, c->Xinit, (size_t)c->pcap * sizeof(float4)))) return rc;
  }
  return PBDR_OK;
}

// default launch shape of size class k: scratch and velocities in shared
// memory where they fit, the class's thread count, every CTA the SMs hold
int default_shape(pbdr_ctx *c, int k, Plan::FClass &F) {
  F.ncap = kClassCaps[k];
  F.dx_shared = fused_layout(F.ncap, true, false, true).bytes <= kFusedSmemLimit;
  F.v_shared = F.dx_shared && fused_layout(F.ncap, true, true, true).bytes <= kFusedSmemLimit;
  F.threads = c->fused_threads ? c->fused_threads : kClassThreads[k];
  const int per_sm = fused_max_blocks_per_sm(F.ncap, F.dx_shared, F.v_shared, F.threads);
  if (per_sm < 1) return fail(PBDR_ERR_CUDA, "scene-resident kernel does not fit on an SM");
  F.grid = std::min<int>(std::max(F.n, 1), per_sm * c->num_sms);
  return PBDR_OK;
}

// scene-resident plan: scenes grouped by size class, the rest streamed
int fill_fused_plan(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, Plan &P) {
  P.ids.assign(ids, ids + n);
  P.fused = true;
  std::vector<int32_t> rest;
  for (int32_t i = 0; i < n; ++i) {
    const SceneHost &S = c->sh[ids[i]];
    int k = 0;
    while (k < kNumClasses && S.np > kClassCaps[k]) ++k;
    if (k < kNumClasses)
      P.classes[k].ids.push_back(ids[i]);
    else
      rest.push_back(ids[i]);
  }
  if (!c->num_sms) CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  int rc;
  for (int k = 0; k < kNumClasses; ++k) {
    Plan::FClass &F = P.classes[k];
    F.n = (int32_t)F.ids.size();
    F.ncap = kClassCaps[k];
    if (!F.n) continue;
    // largest scenes first: the persistent CTAs then finish together
    std::stable_sort(F.ids.begin(), F.ids.end(),
                     [&](int32_t a, int32_t b) { return c->sh[a].np > c->sh[b].np; });
    F.o_list = (int32_t)P.tab.size();
    P.tab.insert(P.tab.end(), F.ids.begin(), F.ids.end());
    if ((rc = default_shape(c, k, F))) return rc;
    if (!F.dx_shared && !c->dx_scratch.p) {
      if ((rc = dev_alloc(c, c->dx_scratch, (size_t)c->pcap * sizeof(float4)))) return rc;
    }
  }
  if (!c->tickets.p && (rc = dev_alloc(c, c->tickets, 64))) return rc;
  if (!rest.empty()) {
    P.rest = std::make_unique<Plan>();
    if ((rc = fill_stream_plan(c, rest.data(), (int32_t)rest.size(), *P.rest, P.tab))) return rc;
  }
  return PBDR_OK;
}

void erase_plan(pbdr_ctx *c, std::map<std::vector<int32_t>, std::unique_ptr<Plan>>::iterator it) {
  Plan *P = it->second.get();
  if (c->active == P) c->active = nullptr;
  if (c->last_fused_plan == P) c->last_fused_plan = nullptr;
  if (c->last_nbr_plan == P || (P->rest && c->last_nbr_plan == P->rest.get())) c->last_nbr_plan = nullptr;
  c->plans.erase(it);
}

// the plan for ids[0..n) (key prefix -2: scene-resident where scenes fit,
// -1: streaming form only), cached; least recently used plans are evicted
int build_plan(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, Plan **out, int streaming_only = 0) {
  if (!ids || n < 1) return fail(PBDR_ERR_INVALID, "need at least one scene id");
  const bool fused = !streaming_only && c->path == 0;
  std::vector<int32_t> key(ids, ids + n);
  key.insert(key.begin(), fused ? -2 : -1);
  auto it = c->plans.find(key);
  if (it != c->plans.end()) {
    it->second->last_use = ++c->use_clock;
    *out = it->second.get();
    return PBDR_OK;
  }
  int rc = check_ids(c, ids, n);
  if (rc) return rc;
  auto P = std::make_unique<Plan>();
  rc = fused ? fill_fused_plan(c, ids, n, *P) : fill_stream_plan(c, ids, n, *P, P->tab);
  if (rc) return rc;
  P->last_use = ++c->use_clock;
  Plan *raw = P.get();
  c->plans[key] = std::move(P);
  while (c->plans.size() > kMaxCachedPlans) {
    auto lru = c->plans.end();
    for (auto i = c->plans.begin(); i != c->plans.end(); ++i)
      if (i->second.get() != raw && (lru == c->plans.end() || i->second->last_use < lru->second->last_use)) lru = i;
    if (lru == c->plans.end()) break;
    erase_plan(c, lru);
  }
  *out = raw;
  return PBDR_OK;
}

void invalidate_plans(pbdr_ctx *c) {
  while (!c->plans.empty()) erase_plan(c, c->plans.begin());
  c->last_nbr_plan = nullptr;
  c->last_fused_plan = nullptr;
}

// drops the cached plans that contain scene s
void drop_plans_with(pbdr_ctx *c, pbdr_scene s) {
  for (auto it = c->plans.begin(); it != c->plans.end();) {
    auto nx = std::next(it);
    if (std::find(it->first.begin() + 1, it->first.end(), s) != it->first.end()) erase_plan(c, it);
    it = nx;
  }
}

// Makes P the active plan on stream s: sizes the streaming scratch, copies
// the plan's tables into the context's table buffer and expands the particle
// and body maps of non-contiguous scene lists.  Stream-ordered after every
// earlier use of those buffers on s.
int activate(pbdr_ctx *c, Plan *P, cudaStream_t s) {
  if (c->active == P) return PBDR_OK;
  Plan *S = P->fused ? P->rest.get() : P;
  int rc;
  if (S && S->np > 0) {
    const size_t npb = (size_t)S->np;
    if ((rc = dev_reserve(c, c->s_keys_a, npb * 4)) || (rc = dev_reserve(c, c->s_keys_b, npb * 4)) ||
        (rc = dev_reserve(c, c->s_vals_a, npb * 4)) || (rc = dev_reserve(c, c->s_vals_b, npb * 4)) ||
        (rc = dev_reserve(c, c->s_spos, npb * sizeof(float4))) ||
        (rc = dev_reserve(c, c->s_hist, radix_hist_words(S->np) * 4)) ||
        (rc = dev_reserve(c, c->s_cells, (size_t)std::max<uint32_t>(S->T_total, 1) * sizeof(uint4))))
      return rc;
    if (!S->pcontig && (rc = dev_reserve(c, c->s_pmap, npb * 4))) return rc;
    if (!S->bcontig && (rc = dev_reserve(c, c->s_bmap, (size_t)std::max(S->nb, 1) * 4))) return rc;
    const size_t nbod = (size_t)std::max(c->bcap, 1);
    if ((rc = dev_reserve(c, c->s_bounds, nbod * 2 * sizeof(float4))) ||
        (rc = dev_reserve(c, c->s_near, nbod * kNearMax * sizeof(int32_t))) ||
        (rc = dev_reserve(c, c->s_ilist, npb * sizeof(int32_t))) || (rc = dev_reserve(c, c->s_icount, 16)))
      return rc;
  }
  if (!P->tab.empty()) {
    if ((rc = dev_reserve(c, c->tab, P->tab.size() * 4))) return rc;
    if ((rc = staged_h2d(c, c->tab.p, P->tab.data(), P->tab.size() * 4, s))) return rc;
  }
  if (S && S->np > 0) {
    const int32_t *t = c->tab.as<int32_t>();
    if (!S->pcontig) launch_expand_map(t + S->o_pseg, t + S->o_pseg + S->nseg + 1, S->nseg, c->s_pmap.as<int32_t>(), s);
    if (!S->bcontig) launch_expand_map(t + S->o_bseg, t + S->o_bseg + S->nseg + 1, S->nseg, c->s_bmap.as<int32_t>(), s);
    CUDA_TRY(cudaGetLastError());
  }
  c->active = P;
  return PBDR_OK;
}

// event of the profiling pool, recorded on s (returns its pool index)
size_t prof_event(pbdr_ctx *c, cudaStream_t s) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->ev_pool.push_back(e);
  }
  cudaEventRecord(c->ev_pool[c->ev_used], s);
  return c->ev_used++;
}

struct StageTimer {
  pbdr_ctx *c;
  cudaStream_t s;
  int stage;
  size_t e0 = 0;
  int64_t l0 = 0;
  int64_t &launches;
  StageTimer(pbdr_ctx *c_, cudaStream_t s_, int st, int64_t &l) : c(c_), s(s_), stage(st), launches(l) {
    if (c->profiling) {
      e0 = prof_event(c, s);
      l0 = launches;
    }
  }
  ~StageTimer() {
    if (c->profiling) c->marks.push_back({stage, e0, prof_event(c, s), launches - l0});
  }
};

// neighbour stage on the positions Xp (keys already written by k_predict)
int neighbor_stage(pbdr_ctx *c, Plan &P, const float4 *Xp, cudaStream_t s, int64_t &launches) {
  int in_b = 0;
  {
  StageTimer tm(c, s, 2, launches);
  launches += radix_sort_pairs(c->s_keys_a.as<uint32_t>(), c->s_vals_a.as<uint32_t>(), c->s_keys_b.as<uint32_t>(),
                               c->s_vals_b.as<uint32_t>(), c->s_hist.as<uint32_t>(), P.np, P.key_bits, &in_b, s);
  }
  P.sorted_in_b = in_b;
  StageTimer tm(c, s, 3, launches);
  // body boxes and near bodies: particles far from every other body skip the search
  const bool cull = c->s_bounds.bytes >= (size_t)c->bcap * 2 * sizeof(float4) &&
                    c->s_near.bytes >= (size_t)c->bcap * kNearMax * sizeof(int32_t) &&
                    c->s_ilist.bytes >= (size_t)P.np * sizeof(int32_t) && c->s_icount.p;
  if (cull) {
    BoundArgs ba{};
    ba.Xp = Xp;
    ba.quat = c->quat.as<float4>();
    ba.bodies = c->bodies.as<BodyRec>();
    ba.scenes = c->scenes.as<ScenePar>();
    ba.bmap = P.bcontig ? nullptr : c->s_bmap.as<int32_t>();
    ba.bbase = P.bbase;
    ba.nbodies = P.nb;
    ba.bounds = c->s_bounds.as<float4>();
    ba.near = c->s_near.as<int32_t>();
    launches += launch_body_bounds(ba, s);
  }
  // every bucket record to all ones: empty, and the identities of its body minima
  CUDA_TRY(cudaMemsetAsync(c->s_cells.p, 0xFF, (size_t)std::max<uint32_t>(P.T_total, 1) * sizeof(uint4), s));
  const uint32_t *sk = in_b ? c->s_keys_b.as<uint32_t>() : c->s_keys_a.as<uint32_t>();
  const uint32_t *sv = in_b ? c->s_vals_b.as<uint32_t>() : c->s_vals_a.as<uint32_t>();
  CellArgs ca{};
  ca.skeys = sk;
  ca.svals = sv;
  ca.Xp = Xp;
  ca.pbody = c->pbody.as<int32_t>();
  ca.cells = c->s_cells.as<uint4>();
  ca.spos = c->s_spos.as<float4>();
  ca.np = P.np;
  launches += launch_cells(ca, s);
  NbrArgs na{};
  na.skeys = sk;
  na.svals = sv;
  na.Xp = Xp;
  na.pbody = c->pbody.as<int32_t>();
  na.pmap = P.pcontig ? nullptr : c->s_pmap.as<int32_t>();
  na.pbase = P.pbase;
  na.spos = c->s_spos.as<float4>();
  na.cells = c->s_cells.as<uint4>();
  na.bodies = c->bodies.as<BodyRec>();
  na.scenes = c->scenes.as<ScenePar>();
  na.hbase = reinterpret_cast<const uint32_t *>(c->tab.as<int32_t>() + P.o_hbase);
  na.nbr_cnt = c->nbr_cnt.as<int32_t>();
  na.nbr = c->nbr.as<int32_t>();
  na.nbr_stride = c->pcap;
  na.cap = c->nbr_cap;
  na.scene_err = c->scene_err.as<uint32_t>();
  na.np = P.np;
  if (cull) {
    na.bounds = c->s_bounds.as<float4>();
    na.near = c->s_near.as<int32_t>();
    na.quat = c->quat.as<float4>();
    na.ilist = c->s_ilist.as<int32_t>();
    na.icount = c->s_icount.as<uint32_t>();
    CUDA_TRY(cudaMemsetAsync(c->s_icount.p, 0, 4, s));
  }
  if (!c->num_sms) CUDA_TRY(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  launches += launch_neighbors(na, c->num_sms, s);
  c->last_nbr_plan = &P;
  return PBDR_OK;
}

PredictArgs predict_args(pbdr_ctx *c, Plan &P, const float4 *X0, const float4 *V0, float4 *Xp,
                         float4 *Vp, int predict) {
  PredictArgs a{};
  a.X0 = X0;
  a.V0 = V0;
  a.Xp = Xp;
  a.Vp = Vp;
  a.Xinit = (predict && P.std_any) ? c->Xinit.as<float4>() : nullptr;
  a.pbody = c->pbody.as<int32_t>();
  a.bodies = c->bodies.as<BodyRec>();
  a.scenes = c->scenes.as<ScenePar>();
  a.wrench = c->wrench.as<BodyWrench>();
  a.pmap = P.pcontig ? nullptr : c->s_pmap.as<int32_t>();
  a.pbase = P.pbase;
  a.np = P.np;
  a.hbase = reinterpret_cast<const uint32_t *>(c->tab.as<int32_t>() + P.o_hbase);
  a.keys = c->s_keys_a.as<uint32_t>();
  a.vals = c->s_vals_a.as<uint32_t>();
  a.predict = predict;
  return a;
}

int substep(pbdr_ctx *c, Plan &P, cudaStream_t s, int64_t &launches);

// one persistent launch of size class k of a scene-resident plan on stream st
int launch_class(pbdr_ctx *c, Plan &P, int k, cudaStream_t st) {
  Plan::FClass &F = P.classes[k];
  FusedArgs a{};
  a.X = c->X[0].as<float4>();
  a.V = c->V[0].as<float4>();
  a.Q = c->Q.as<float4>();
  a.pbody = c->pbody.as<int32_t>();
  a.bodies = c->bodies.as<BodyRec>();
  a.scenes = c->scenes.as<ScenePar>();
  a.wrench = c->wrench.as<BodyWrench>();
  a.quat = c->quat.as<float4>();
  a.bcom = c->bcom.as<float4>();
  a.biter = c->biter.as<float4>();
  a.chunks = c->chunks.as<Chunk>();
  a.border = c->border.as<int32_t>();
  a.partials = c->partials.as<float>();
  a.dx_scratch = F.dx_shared ? nullptr : c->dx_scratch.as<float4>();
  a.nbr_cnt = c->nbr_cnt.as<int32_t>();
  a.nbr = c->nbr.as<int32_t>();
  a.nbr_stride = c->pcap;
  a.nbr_cap = std::min(c->nbr_cap, kFusedNbrCap);
  a.scene_err = c->scene_err.as<uint32_t>();
  a.scene_list = c->tab.as<int32_t>() + F.o_list;
  a.nscenes = F.n;
  a.ticket = c->tickets.as<uint32_t>() + k;
  a.ncap = F.ncap;
  a.grid = F.grid;
  a.v_shared = F.v_shared ? 1 : 0;
  const FusedLayout L = fused_layout(F.ncap, F.dx_shared, F.v_shared, F.dx_shared);
  a.tcap = L.tcap;
  a.ccap = L.ccap;
  a.v_off = L.v_off;
  a.part_off = L.part_off;
  a.bcap = L.bcap;
  a.bt_off = L.bt_off;
  a.smem_bytes = L.bytes;
  return launch_scene_substep(a, F.threads, st);
}

int ensure_class_streams(pbdr_ctx *c) {
  if (c->ev_fork) return PBDR_OK;
  CUDA_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
  for (int k = 0; k < kNumClasses; ++k) {
    CUDA_TRY(cudaStreamCreateWithFlags(&c->cls_stream[k], cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&c->ev_join[k], cudaEventDisableTiming));
  }
  CUDA_TRY(cudaStreamCreateWithFlags(&c->rest_stream, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&c->ev_rest_join, cudaEventDisableTiming));
  return PBDR_OK;
}

int substep(pbdr_ctx *c, Plan &P, cudaStream_t s, int64_t &launches);

// tangent buffers sized to the particle capacity; new space is zero
int ensure_tangent(pbdr_ctx *c) {
  const size_t bytes = (size_t)std::max(c->pcap, 1) * sizeof(float4);
  for (DevBuf *b : {&c->Xd[0], &c->Xd[1], &c->Vd[0], &c->Vd[1]}) {
    if (b->bytes >= bytes) continue;
    const size_t old = b->p ? std::min(b->bytes, (size_t)c->np_used * sizeof(float4)) : 0;
    int rc = dev_grow(c, *b, bytes, old);
    if (rc) return rc;
    CUDA_TRY(cudaMemset(b->as<unsigned char>() + old, 0, bytes - old));
    CUDA_TRY(cudaDeviceSynchronize());   // grown rarely; later uploads use other streams
  }
  return PBDR_OK;
}

// one substep of a streaming plan with the tangent (forward-mode) kernels
int tangent_substep(pbdr_ctx *c, Plan &P, cudaStream_t s, int64_t &launches) {
  if (P.np == 0) return PBDR_OK;
  const int K = P.kmax;
  float4 *X0 = c->X[0].as<float4>(), *V0 = c->V[0].as<float4>();
  float4 *X1 = c->X[1].as<float4>(), *V1 = c->V[1].as<float4>();
  float4 *D0 = c->Xd[0].as<float4>(), *W0 = c->Vd[0].as<float4>();
  float4 *D1 = c->Xd[1].as<float4>(), *W1 = c->Vd[1].as<float4>();
  const bool odd = K % 2 == 1;
  float4 *Xp = odd ? X1 : X0, *Vp = odd ? V1 : V0, *Dp = odd ? D1 : D0, *Wp = odd ? W1 : W0;
  launches += launch_predict(predict_args(c, P, X0, V0, Xp, Vp, 1), s);
  TangentPredictArgs tp{};
  tp.Xd0 = D0;
  tp.Vd0 = W0;
  tp.Xdp = Dp;
  tp.Vdp = Wp;
  tp.pbody = c->pbody.as<int32_t>();
  tp.bodies = c->bodies.as<BodyRec>();
  tp.scenes = c->scenes.as<ScenePar>();
  tp.pmap = P.pcontig ? nullptr : c->s_pmap.as<int32_t>();
  tp.pbase = P.pbase;
  tp.np = P.np;
  launches += launch_predict_tangent(tp, s);
  int rc = neighbor_stage(c, P, Xp, s, launches);
  if (rc) return rc;
  IterArgs ia{};
  ia.Q = c->Q.as<float4>();
  ia.Xinit = nullptr;
  ia.nbr_cnt = c->nbr_cnt.as<int32_t>();
  ia.nbr = c->nbr.as<int32_t>();
  ia.nbr_stride = c->pcap;
  ia.bodies = c->bodies.as<BodyRec>();
  ia.scenes = c->scenes.as<ScenePar>();
  ia.quat = c->quat.as<float4>();
  ia.bcom = c->bcom.as<float4>();
  ia.bmap = P.bcontig ? nullptr : c->s_bmap.as<int32_t>();
  ia.bbase = P.bbase;
  ia.nbodies = P.nb;
  ia.scene_err = c->scene_err.as<uint32_t>();
  for (int k = 0; k < K; ++k) {
    const int out = (K - 1 - k) % 2;
    ia.Xin = out ? X0 : X1;
    ia.Vin = out ? V0 : V1;
    ia.Xout = out ? X1 : X0;
    ia.Vout = out ? V1 : V0;
    ia.k = k;
    TangentArgs ta{};
    ta.dmu = c->dmu.p ? c->dmu.as<float>() : nullptr;
    ta.Xdin = out ? D0 : D1;
    ta.Vdin = out ? W0 : W1;
    ta.Xdout = out ? D1 : D0;
    ta.Vdout = out ? W1 : W0;
    launches += launch_iterate_tangent(ia, ta, s);
  }
  CUDA_TRY(cudaGetLastError());
  return PBDR_OK;
}

// adjoint buffers sized to the particle capacity; new space is zero
int ensure_adjoint(pbdr_ctx *c) {
  const size_t bytes = (size_t)std::max(c->pcap, 1) * sizeof(float4);
  for (DevBuf *b : {&c->Xb[0], &c->Xb[1], &c->Vb[0], &c->Vb[1], &c->Ub}) {
    if (b->bytes >= bytes) continue;
    const size_t old = b->p ? std::min(b->bytes, (size_t)c->np_used * sizeof(float4)) : 0;
    int rc = dev_grow(c, *b, bytes, old);
    if (rc) return rc;
    CUDA_TRY(cudaMemset(b->as<unsigned char>() + old, 0, bytes - old));
    CUDA_TRY(cudaDeviceSynchronize());   // grown rarely; later uploads use other streams
  }
  return PBDR_OK;
}

// a saved state of the context: X, V of every particle, rotation warm start
// and sum anchor of every body
struct StateSlots {
  float4 *base = nullptr;
  size_t np = 0, nb = 0;
  float4 *slot(int k) const { return base + (size_t)k * (2 * np + 2 * nb); }
};

int save_state(pbdr_ctx *c, const StateSlots &S, int k, cudaStream_t s) {
  float4 *d = S.slot(k);
  CUDA_TRY(cudaMemcpyAsync(d, c->X[0].p, S.np * 16, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(d + S.np, c->V[0].p, S.np * 16, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(d + 2 * S.np, c->quat.p, S.nb * 16, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(d + 2 * S.np + S.nb, c->bcom.p, S.nb * 16, cudaMemcpyDeviceToDevice, s));
  return PBDR_OK;
}

int load_state(pbdr_ctx *c, const StateSlots &S, int k, cudaStream_t s) {
  const float4 *d = S.slot(k);
  CUDA_TRY(cudaMemcpyAsync(c->X[0].p, d, S.np * 16, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(c->V[0].p, d + S.np, S.np * 16, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(c->quat.p, d + 2 * S.np, S.nb * 16, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(c->bcom.p, d + 2 * S.np + S.nb, S.nb * 16, cudaMemcpyDeviceToDevice, s));
  return PBDR_OK;
}

// Reverse of one substep of a streaming plan, from the saved state at its
// start (loaded into X[0], V[0], quat, bcom) and the adjoint of its end state
// in Xb[0], Vb[0]; leaves the adjoint of its start state in Xb[0], Vb[0].
// The substep is run forward again, keeping the state before every
// iteration in slots it0 .. it0 + K - 1 of S.
int adjoint_substep(pbdr_ctx *c, Plan &P, const StateSlots &S, int it0, cudaStream_t s, int64_t &launches) {
  if (P.np == 0) return PBDR_OK;
  const int K = P.kmax;
  float4 *X0 = c->X[0].as<float4>(), *V0 = c->V[0].as<float4>();
  float4 *X1 = c->X[1].as<float4>(), *V1 = c->V[1].as<float4>();
  const bool odd = K % 2 == 1;
  float4 *Xp = odd ? X1 : X0, *Vp = odd ? V1 : V0;
  launches += launch_predict(predict_args(c, P, X0, V0, Xp, Vp, 1), s);
  int rc = neighbor_stage(c, P, Xp, s, launches);
  if (rc) return rc;
  IterArgs ia{};
  ia.Q = c->Q.as<float4>();
  ia.Xinit = nullptr;
  ia.nbr_cnt = c->nbr_cnt.as<int32_t>();
  ia.nbr = c->nbr.as<int32_t>();
  ia.nbr_stride = c->pcap;
  ia.bodies = c->bodies.as<BodyRec>();
  ia.scenes = c->scenes.as<ScenePar>();
  ia.bmap = P.bcontig ? nullptr : c->s_bmap.as<int32_t>();
  ia.bbase = P.bbase;
  ia.nbodies = P.nb;
  ia.scene_err = c->scene_err.as<uint32_t>();
  // forward, keeping the state before every iteration
  for (int k = 0; k < K; ++k) {
    const int out = (K - 1 - k) % 2;
    float4 *xin = out ? X0 : X1, *vin = out ? V0 : V1;
    float4 *d = S.slot(it0 + k);
    CUDA_TRY(cudaMemcpyAsync(d, xin, S.np * 16, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d + S.np, vin, S.np * 16, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d + 2 * S.np, c->quat.p, S.nb * 16, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d + 2 * S.np + S.nb, c->bcom.p, S.nb * 16, cudaMemcpyDeviceToDevice, s));
    ia.Xin = xin;
    ia.Vin = vin;
    ia.Xout = out ? X1 : X0;
    ia.Vout = out ? V1 : V0;
    ia.quat = c->quat.as<float4>();
    ia.bcom = c->bcom.as<float4>();
    ia.k = k;
    launches += launch_iterate(ia, 4, s);
  }
  // backward through the iterations; Xb/Vb ping-pong, ending in buffer `cur`
  int cur = 0;
  const int32_t *pmap = P.pcontig ? nullptr : c->s_pmap.as<int32_t>();
  for (int k = K - 1; k >= 0; --k) {
    float4 *d = S.slot(it0 + k);
    ia.Xin = d;
    ia.Vin = d + S.np;
    ia.quat = d + 2 * S.np;
    ia.bcom = d + 2 * S.np + S.nb;
    ia.Xout = X1;   // scratch for X_bsm, V_bsm
    ia.Vout = V1;
    ia.k = k;
    AdjointArgs ta{};
    ta.Xbin = c->Xb[cur].as<float4>();
    ta.Vbin = c->Vb[cur].as<float4>();
    ta.Xbout = c->Xb[1 - cur].as<float4>();
    ta.Vbout = c->Vb[1 - cur].as<float4>();
    ta.U = c->Ub.as<float4>();
    launches += launch_iterate_adjoint(ia, ta, c->pbody.as<int32_t>(), pmap, P.pbase, P.np, s);
    cur = 1 - cur;
  }
  TangentPredictArgs tp{};
  tp.Xd0 = c->Xb[cur].as<float4>();
  tp.Vd0 = c->Vb[cur].as<float4>();
  tp.Xdp = c->Xb[1 - cur].as<float4>();
  tp.Vdp = c->Vb[1 - cur].as<float4>();
  tp.pbody = c->pbody.as<int32_t>();
  tp.bodies = c->bodies.as<BodyRec>();
  tp.scenes = c->scenes.as<ScenePar>();
  tp.pmap = pmap;
  tp.pbase = P.pbase;
  tp.np = P.np;
  launches += launch_predict_adjoint(tp, s);
  cur = 1 - cur;
  if (cur != 0) {   // both buffers agree outside the plan's particles
    CUDA_TRY(cudaMemcpyAsync(c->Xb[0].p, c->Xb[1].p, S.np * 16, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->Vb[0].p, c->Vb[1].p, S.np * 16, cudaMemcpyDeviceToDevice, s));
  }
  CUDA_TRY(cudaGetLastError());
  return PBDR_OK;
}

int fused_substep(pbdr_ctx *c, Plan &P, cudaStream_t s, int64_t &launches) {
  int rc = ensure_class_streams(c);
  if (rc) return rc;
  // the scenes above the largest class (the streaming form, P.rest) touch
  // no scene, body or particle range of the classes: they run on a stream
  // of their own beside the classes and fill the SMs the classes' last
  // persistent CTAs leave idle.  With stage profiling on they run after the
  // classes instead, so that the stages' times stay apart.
  const bool rest_beside = P.rest && !c->profiling;
  {
    StageTimer tm(c, s, 5, launches);
    CUDA_TRY(cudaMemsetAsync(c->tickets.p, 0, 64, s));
    // the size classes are independent: one forked stream each
    CUDA_TRY(cudaEventRecord(c->ev_fork, s));
    for (int k = 0; k < (int)P.classes.size(); ++k) {
      if (!P.classes[k].n) continue;
      CUDA_TRY(cudaStreamWaitEvent(c->cls_stream[k], c->ev_fork, 0));
      launches += launch_class(c, P, k, c->cls_stream[k]);
      CUDA_TRY(cudaEventRecord(c->ev_join[k], c->cls_stream[k]));
    }
    if (rest_beside) {
      CUDA_TRY(cudaStreamWaitEvent(c->rest_stream, c->ev_fork, 0));
      if ((rc = substep(c, *P.rest, c->rest_stream, launches))) return rc;
      CUDA_TRY(cudaEventRecord(c->ev_rest_join, c->rest_stream));
      CUDA_TRY(cudaStreamWaitEvent(s, c->ev_rest_join, 0));
    }
    for (int k = 0; k < (int)P.classes.size(); ++k)
      if (P.classes[k].n) CUDA_TRY(cudaStreamWaitEvent(s, c->ev_join[k], 0));
    CUDA_TRY(cudaGetLastError());
  }
  c->last_fused_plan = &P;
  if (P.rest && !rest_beside) return substep(c, *P.rest, s, launches);
  return PBDR_OK;
}

// Autotuner of the scene-resident kernel.  The candidate launch shapes of a
// size class are: threads per CTA (128, 256, 512), the per-particle scratch
// (dX, x_asm) in shared or in global memory, velocities in shared memory or
// not, and the CTAs kept per SM (the occupancy limit or half of it).  Classes
// with at least as many scenes as SMs are tuned one after the other (largest
// work first) by timing whole substeps of the plan - all classes running
// concurrently as in production - with the other classes at their current
// shapes, and each keeps its fastest shape, remembered per (class, scene
// count) for later plans.  The kernel's results do not depend on its launch shape, and the
// state the trial substeps change is saved before and restored after, so
// tuning has no effect on the simulation.
int autotune_fused(pbdr_ctx *c, Plan &P, cudaStream_t s) {
  int rc;
  {  // classes with fewer scenes than SMs keep the defaults (one CTA per
     // scene anyway); shapes tuned before for the same class and scene count
     // are reused
    bool todo = false;
    for (int k = 0; k < (int)P.classes.size(); ++k) {
      Plan::FClass &F = P.classes[k];
      if (F.n < c->num_sms) continue;
      auto memo = c->tune_memo.find({k, F.n});
      if (memo == c->tune_memo.end()) {
        todo = true;
        continue;
      }
      F.threads = memo->second[0];
      F.dx_shared = memo->second[1] != 0;
      F.v_shared = memo->second[2] != 0;
      F.grid = memo->second[3];
    }
    if (!todo) {
      P.tuned = true;
      return PBDR_OK;
    }
  }
  if (!c->dx_scratch.p && (rc = dev_alloc(c, c->dx_scratch, (size_t)c->pcap * sizeof(float4)))) return rc;
  const size_t nX = (size_t)std::max(c->np_used, 1) * sizeof(float4);
  const size_t nB = (size_t)std::max(c->nb_used, 1) * sizeof(float4);
  const size_t nE = (size_t)std::max<size_t>(c->sh.size(), 1) * sizeof(uint32_t);
  DevBuf sX, sV, sQr, sCm, sE;
  if ((rc = dev_alloc(c, sX, nX)) || (rc = dev_alloc(c, sV, nX)) || (rc = dev_alloc(c, sQr, nB)) ||
      (rc = dev_alloc(c, sCm, nB)) || (rc = dev_alloc(c, sE, nE)))
    return rc;
  CUDA_TRY(cudaMemcpyAsync(sX.p, c->X[0].p, nX, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(sV.p, c->V[0].p, nX, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(sQr.p, c->quat.p, nB, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(sCm.p, c->bcom.p, nB, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(sE.p, c->scene_err.p, nE, cudaMemcpyDeviceToDevice, s));
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  auto restore = [&]() -> int {
    CUDA_TRY(cudaMemcpyAsync(c->X[0].p, sX.p, nX, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->V[0].p, sV.p, nX, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->quat.p, sQr.p, nB, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->bcom.p, sCm.p, nB, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->scene_err.p, sE.p, nE, cudaMemcpyDeviceToDevice, s));
    return PBDR_OK;
  };
  // every candidate starts from the same saved state: one warm substep,
  // then the fastest of three timed runs of three substeps
  auto time_substeps = [&](float *ms) -> int {
    int64_t l = 0;
    int r2 = restore();
    if (r2) return r2;
    if ((r2 = fused_substep(c, P, s, l))) return r2;
    *ms = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      CUDA_TRY(cudaEventRecord(e0, s));
      for (int k = 0; k < 3; ++k)
        if ((r2 = fused_substep(c, P, s, l))) return r2;
      CUDA_TRY(cudaEventRecord(e1, s));
      CUDA_TRY(cudaEventSynchronize(e1));
      CUDA_TRY(cudaGetLastError());
      float t = 0.f;
      CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
      *ms = std::min(*ms, t);
    }
    return PBDR_OK;
  };
  // classes by descending particle count
  std::vector<std::pair<int64_t, int>> work;
  for (int k = 0; k < (int)P.classes.size(); ++k) {
    int64_t w = 0;
    for (int32_t id : P.classes[k].ids) w += c->sh[id].np;
    if (P.classes[k].n) work.push_back({-w, k});
  }
  std::sort(work.begin(), work.end());
  std::vector<int> todo;
  for (auto &wk : work) {
    const Plan::FClass &F = P.classes[wk.second];
    if (F.n >= c->num_sms && !c->tune_memo.count({wk.second, F.n})) todo.push_back(wk.second);
  }
  // two coordinate-descent passes: the second revisits every class with the
  // others at their tuned shapes
  for (int pass = 0; pass < 2; ++pass)
  for (int kc : todo) {
    Plan::FClass &F = P.classes[kc];
    struct Cand {
      float ms;
      int threads, grid;
      bool dx, v;
    };
    std::vector<Cand> cands;
    const int threads_c[3] = {128, 256, 512};
    for (int dxi = 0; dxi < 2; ++dxi) {
      const bool dxs = dxi == 0;
      if (dxs && fused_layout(F.ncap, true, false, true).bytes > kFusedSmemLimit) continue;
      for (int vs = 0; vs < 2; ++vs) {
        const bool vsh = vs == 1;
        if (vsh && !(dxs && fused_layout(F.ncap, true, true, true).bytes <= kFusedSmemLimit)) continue;
        for (int ti = 0; ti < 3; ++ti) {
          const int per_sm = fused_max_blocks_per_sm(F.ncap, dxs, vsh, threads_c[ti]);
          if (per_sm < 1) continue;
          const int cps_c[2] = {per_sm, std::max(1, per_sm / 2)};
          for (int ci = 0; ci < (per_sm > 1 ? 2 : 1); ++ci)
            cands.push_back({0.f, threads_c[ti], std::min<int>(F.n, cps_c[ci] * c->num_sms), dxs, vsh});
        }
      }
    }
    if (cands.empty()) continue;
    auto apply = [&](const Cand &k) {
      F.threads = k.threads;
      F.grid = k.grid;
      F.dx_shared = k.dx;
      F.v_shared = k.v;
    };
    for (Cand &k : cands) {
      apply(k);
      if ((rc = time_substeps(&k.ms))) return rc;
    }
    // the three fastest are timed again, alternately, and keep their best
    // time: single trials differ by about as much as close candidates do
    std::sort(cands.begin(), cands.end(), [](const Cand &x, const Cand &y) { return x.ms < y.ms; });
    const size_t top = std::min<size_t>(3, cands.size());
    for (int round = 0; round < 3; ++round)
      for (size_t i = 0; i < top; ++i) {
        float ms = 0.f;
        apply(cands[i]);
        if ((rc = time_substeps(&ms))) return rc;
        cands[i].ms = std::min(cands[i].ms, ms);
      }
    std::sort(cands.begin(), cands.begin() + top, [](const Cand &x, const Cand &y) { return x.ms < y.ms; });
    apply(cands[0]);
  }
  // guard: keep the tuned shapes only if whole substeps beat the defaults
  if (!todo.empty()) {
    std::array<Plan::FClass, kNumClasses> tuned_shapes = P.classes, defaults = P.classes;
    for (int kc : todo)
      if ((rc = default_shape(c, kc, defaults[kc]))) return rc;
    auto set_shapes = [&](const std::array<Plan::FClass, kNumClasses> &src) {
      for (int kc : todo) {
        P.classes[kc].threads = src[kc].threads;
        P.classes[kc].grid = src[kc].grid;
        P.classes[kc].dx_shared = src[kc].dx_shared;
        P.classes[kc].v_shared = src[kc].v_shared;
      }
    };
    float t_tuned = 1e30f, t_default = 1e30f;
    for (int round = 0; round < 3; ++round) {
      float ms = 0.f;
      set_shapes(tuned_shapes);
      if ((rc = time_substeps(&ms))) return rc;
      t_tuned = std::min(t_tuned, ms);
      set_shapes(defaults);
      if ((rc = time_substeps(&ms))) return rc;
      t_default = std::min(t_default, ms);
    }
    set_shapes(t_tuned <= t_default ? tuned_shapes : defaults);
    for (int kc : todo) {
      const Plan::FClass &F = P.classes[kc];
      c->tune_memo[{kc, F.n}] = {F.threads, F.dx_shared ? 1 : 0, F.v_shared ? 1 : 0, F.grid};
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if ((rc = restore())) return rc;
  CUDA_TRY(cudaStreamSynchronize(s));
  for (DevBuf *b : {&sX, &sV, &sQr, &sCm, &sE}) dev_free(c, *b);
  P.tuned = true;
  return PBDR_OK;
}

// captures one substep of the plan into a CUDA graph (not on the legacy
// default stream, which cannot be captured)
int capture_plan(pbdr_ctx *c, Plan &P, cudaStream_t s) {
  int rc = ensure_class_streams(c);
  if (rc) return rc;
  int64_t launches = 0;
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  rc = substep(c, P, s, launches);
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return fail(PBDR_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&P.graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    P.graph = nullptr;
    return fail(PBDR_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  }
  P.graph_launches = launches;
  return PBDR_OK;
}

int substep(pbdr_ctx *c, Plan &P, cudaStream_t s, int64_t &launches) {
  if (P.fused) return fused_substep(c, P, s, launches);
  if (P.np == 0) return PBDR_OK;
  const int K = P.kmax;
  float4 *X0 = c->X[0].as<float4>(), *V0 = c->V[0].as<float4>();
  float4 *X1 = c->X[1].as<float4>(), *V1 = c->V[1].as<float4>();
  if (!P.wrench_list.empty()) {
    StageTimer tm(c, s, 0, launches);
    WrenchArgs wa{};
    wa.X = X0;
    wa.Q = c->Q.as<float4>();
    wa.bodies = c->bodies.as<BodyRec>();
    wa.wrench = c->wrench.as<BodyWrench>();
    wa.blist = c->tab.as<int32_t>() + P.o_wlist;
    wa.nb = (int32_t)P.wrench_list.size();
    launches += launch_wrench(wa, s);
  }
  // iteration k writes buffer (K-1-k) % 2, so the last one lands in buffer 0;
  // the prediction writes the buffer iteration 0 reads
  float4 *Xp = (K % 2 == 1) ? X1 : X0;
  float4 *Vp = (K % 2 == 1) ? V1 : V0;
  {
    StageTimer tm(c, s, 1, launches);
    launches += launch_predict(predict_args(c, P, X0, V0, Xp, Vp, 1), s);
  }
  int rc = neighbor_stage(c, P, Xp, s, launches);
  if (rc) return rc;
  StageTimer tm(c, s, 4, launches);
  IterArgs ia{};
  ia.Q = c->Q.as<float4>();
  ia.Xinit = P.std_any ? c->Xinit.as<float4>() : nullptr;
  ia.nbr_cnt = c->nbr_cnt.as<int32_t>();
  ia.nbr = c->nbr.as<int32_t>();
  ia.nbr_stride = c->pcap;
  ia.bodies = c->bodies.as<BodyRec>();
  ia.scenes = c->scenes.as<ScenePar>();
  ia.quat = c->quat.as<float4>();
  ia.bcom = c->bcom.as<float4>();
  ia.bmap = c->tab.as<int32_t>() + P.o_iorder;   // bodies largest first
  ia.bbase = P.bbase;
  ia.nbodies = P.nb;
  ia.scene_err = c->scene_err.as<uint32_t>();
  for (int k = 0; k < K; ++k) {
    const int out = (K - 1 - k) % 2;
    ia.Xin = out ? X0 : X1;
    ia.Vin = out ? V0 : V1;
    ia.Xout = out ? X1 : X0;
    ia.Vout = out ? V1 : V0;
    ia.k = k;
    launches += launch_iterate(ia, 1, s);   // one-warp CTAs: a finished body frees its slot at once
  }
  CUDA_TRY(cudaGetLastError());
  return PBDR_OK;
}

__global__ void k_errs(uint32_t *scene_err, const int32_t *ids, int32_t n, uint32_t *out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = scene_err[ids[i]];
  scene_err[ids[i]] = 0u;
}

// gather / scatter of xyz state for scenes ids[0..n) through device staging
int transfer_states(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, float *hpos, float *hvel,
                    const float *cpos, const float *cvel, uint32_t *err_bits, int unpack,
                    cudaStream_t s, float4 *bufX = nullptr, float4 *bufV = nullptr, bool sync = true) {
  if (!c) return fail(PBDR_ERR_INVALID, "NULL context");
  if (!ids || n < 1) return fail(PBDR_ERR_INVALID, "need at least one scene id");
  std::vector<int32_t> p0(n);
  std::vector<int64_t> off(n + 1, 0);
  for (int32_t i = 0; i < n; ++i) {
    int rc = check_scene(c, ids[i]);
    if (rc) return rc;
    p0[i] = c->sh[ids[i]].p0;
    off[i + 1] = off[i] + c->sh[ids[i]].np;
  }
  const int64_t total = off[n];
  int rc;
  const bool want_pos = unpack ? cpos != nullptr : hpos != nullptr;
  const bool want_vel = unpack ? cvel != nullptr : hvel != nullptr;
  if ((rc = dev_reserve(c, c->seg_p0, (size_t)n * 4))) return rc;
  if ((rc = dev_reserve(c, c->seg_off, (size_t)(n + 1) * 8))) return rc;
  if (want_pos && (rc = dev_reserve(c, c->stage_pos, (size_t)std::max<int64_t>(total, 1) * 12))) return rc;
  if (want_vel && (rc = dev_reserve(c, c->stage_vel, (size_t)std::max<int64_t>(total, 1) * 12))) return rc;
  if ((rc = staged_h2d(c, c->seg_p0.p, p0.data(), (size_t)n * 4, s))) return rc;
  if ((rc = staged_h2d(c, c->seg_off.p, off.data(), (size_t)(n + 1) * 8, s))) return rc;
  PackArgs pa{};
  pa.X = bufX ? bufX : c->X[0].as<float4>();
  pa.V = bufV ? bufV : c->V[0].as<float4>();
  pa.hpos = want_pos ? c->stage_pos.as<float>() : nullptr;
  pa.hvel = want_vel ? c->stage_vel.as<float>() : nullptr;
  pa.seg_p0 = c->seg_p0.as<int32_t>();
  pa.seg_off = c->seg_off.as<int64_t>();
  pa.nseg = n;
  pa.total = total;
  if (unpack) {
    if (want_pos) CUDA_TRY(cudaMemcpyAsync(pa.hpos, cpos, (size_t)total * 12, cudaMemcpyHostToDevice, s));
    if (want_vel) CUDA_TRY(cudaMemcpyAsync(pa.hvel, cvel, (size_t)total * 12, cudaMemcpyHostToDevice, s));
    launch_pack(pa, 1, s);
    CUDA_TRY(cudaGetLastError());
    return PBDR_OK;
  }
  launch_pack(pa, 0, s);
  if (want_pos) CUDA_TRY(cudaMemcpyAsync(hpos, pa.hpos, (size_t)total * 12, cudaMemcpyDeviceToHost, s));
  if (want_vel) CUDA_TRY(cudaMemcpyAsync(hvel, pa.hvel, (size_t)total * 12, cudaMemcpyDeviceToHost, s));
  if (err_bits) {
    if ((rc = dev_reserve(c, c->err_ids, (size_t)n * 4))) return rc;
    if ((rc = dev_reserve(c, c->err_out, (size_t)n * 4))) return rc;
    if ((rc = staged_h2d(c, c->err_ids.p, ids, (size_t)n * 4, s))) return rc;
    k_errs<<<(n + 255) / 256, 256, 0, s>>>(c->scene_err.as<uint32_t>(), c->err_ids.as<int32_t>(), n,
                                            c->err_out.as<uint32_t>());
    CUDA_TRY(cudaMemcpyAsync(err_bits, c->err_out.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
  }
  CUDA_TRY(cudaGetLastError());
  if (sync) CUDA_TRY(cudaStreamSynchronize(s));
  return PBDR_OK;
}

}  // namespace

extern "C" {

const char *pbdr_last_error(void) { return g_err.c_str(); }

int pbdr_ctx_create(int device, size_t hbm_budget_bytes, pbdr_ctx **out) {
  g_err.clear();
  if (!out) return fail(PBDR_ERR_INVALID, "NULL out");
  *out = nullptr;
  int ndev = 0;
  CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(PBDR_ERR_INVALID, "no CUDA device " + std::to_string(device));
  CUDA_TRY(cudaSetDevice(device));
  auto *c = new (std::nothrow) pbdr_ctx();
  if (!c) return fail(PBDR_ERR_OOM, "host allocation failed");
  c->device = device;
  c->budget = hbm_budget_bytes;
  *out = c;
  return PBDR_OK;
}

int pbdr_ctx_destroy(pbdr_ctx *c) {
  g_err.clear();
  if (!c) return PBDR_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  invalidate_plans(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : c->step_ev)
    if (e) cudaEventDestroy(e);
  for (auto &w : c->work_ev) cudaEventDestroy(w.second);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->rest_stream) cudaStreamDestroy(c->rest_stream);
  if (c->ev_rest_join) cudaEventDestroy(c->ev_rest_join);
  for (int k = 0; k < kNumClasses; ++k) {
    if (c->cls_stream[k]) cudaStreamDestroy(c->cls_stream[k]);
    if (c->ev_join[k]) cudaEventDestroy(c->ev_join[k]);
  }
  delete c;
  return PBDR_OK;
}

int pbdr_create_scene(pbdr_ctx *c, const pbdr_scene_desc *d, pbdr_scene *out) {
  g_err.clear();
  if (!c || !d || !out) return fail(PBDR_ERR_INVALID, "NULL argument");
  const int32_t N = d->num_particles, B = d->num_bodies;
  if (N < 0 || B < 0) return fail(PBDR_ERR_INVALID, "negative particle or body count");
  if ((N == 0) != (B == 0)) return fail(PBDR_ERR_INVALID, "a scene with particles needs bodies and vice versa");
  if (N > 0 && (!d->pos || !d->vel || !d->inv_mass || !d->body_off))
    return fail(PBDR_ERR_INVALID, "NULL array in descriptor");
  if (!(d->radius > 0.f) || !std::isfinite(d->radius)) return fail(PBDR_ERR_INVALID, "radius must be > 0");
  if (!(d->friction >= 0.f) || !std::isfinite(d->friction)) return fail(PBDR_ERR_INVALID, "friction must be >= 0");
  if (!(d->dt > 0.f) || !std::isfinite(d->dt)) return fail(PBDR_ERR_INVALID, "dt must be > 0");
  if (d->iterations < 1 || d->iterations > 1024) return fail(PBDR_ERR_INVALID, "iterations must be in 1..1024");
  if (!finite3(d->gravity) || !finite3(d->plane) || !std::isfinite(d->plane[3]))
    return fail(PBDR_ERR_INVALID, "gravity and plane must be finite");
  const uint32_t known = PBDR_STD_VELOCITY | PBDR_NO_LINMOM | PBDR_NO_ANGMOM | PBDR_CONTACT_AVG | PBDR_SM_FROM_XI;
  if (d->flags & ~known) return fail(PBDR_ERR_INVALID, "unknown flag bits");
  if (d->flags & PBDR_SM_FROM_XI) return fail(PBDR_ERR_UNSUPPORTED, "PBDR_SM_FROM_XI is not implemented on the GPU path");
  const double nl = std::sqrt((double)d->plane[0] * d->plane[0] + (double)d->plane[1] * d->plane[1] +
                              (double)d->plane[2] * d->plane[2]);
  if (!(std::fabs(nl - 1.0) < 1e-3)) return fail(PBDR_ERR_INVALID, "plane normal must be unit length");
  if (N > 0) {
    if (d->body_off[0] != 0 || d->body_off[B] != N) return fail(PBDR_ERR_INVALID, "body_off must start at 0 and end at N");
    for (int32_t b = 0; b < B; ++b) {
      const int32_t cnt = d->body_off[b + 1] - d->body_off[b];
      if (cnt <= 0) return fail(PBDR_ERR_INVALID, "body_off must be strictly increasing");
      if (cnt > kMaxBodyParticles) return fail(PBDR_ERR_INVALID, "body too large");
    }
    // the per-particle checks (finite, inverse mass > 0) run in the
    // rest-shape pass below, before anything is uploaded
  }
  if ((int64_t)c->pa.top + N > INT32_MAX / 2 || (int64_t)c->ba.top + B > INT32_MAX / 2)
    return fail(PBDR_ERR_INVALID, "context particle or body count overflow");
  // scene id: the first destroyed slot, else a new one
  int32_t sid = (int32_t)c->sh.size();
  for (int32_t i = 0; i < (int32_t)c->sh.size(); ++i)
    if (!c->sh[i].alive) {
      sid = i;
      break;
    }
  // work chunks of the scene-resident kernel: up to kChunk particles of one body
  int32_t nchunks = 0;
  for (int32_t b = 0; b < B; ++b) nchunks += (d->body_off[b + 1] - d->body_off[b] + kChunk - 1) / kChunk;
  // ranges of the packed tables: reuse freed ranges first (first fit)
  int32_t P0 = c->pa.take(N), B0 = c->ba.take(B), C0 = c->ca.take(nchunks);
  const bool p_top = P0 < 0, b_top = B0 < 0, c_top = C0 < 0;
  if (p_top) P0 = c->pa.top;
  if (b_top) B0 = c->ba.top;
  if (c_top) C0 = c->ca.top;
  auto give_back = [&]() {
    if (!p_top) c->pa.give(P0, N);
    if (!b_top) c->ba.give(B0, B);
    if (!c_top) c->ca.give(C0, nchunks);
  };
  std::vector<Chunk> chk;
  int32_t multi = 0;
  for (int32_t b = 0; b < B; ++b) {
    const int32_t n = d->body_off[b + 1] - d->body_off[b];
    const int32_t nk = (n + kChunk - 1) / kChunk;
    multi += nk > 1;
    for (int32_t k = 0; k < nk; ++k)
      chk.push_back(Chunk{B0 + b, P0 + d->body_off[b] + k * kChunk, std::min(kChunk, n - k * kChunk), k});
  }
  std::stable_sort(chk.begin(), chk.end(), [](const Chunk &x, const Chunk &y) { return x.count > y.count; });
  int rc = ensure_capacity(c, std::max(c->pa.top, P0 + N), std::max(c->ba.top, B0 + B),
                           std::max((int32_t)c->sh.size(), sid + 1), std::max(c->ca.top, C0 + nchunks));
  if (rc) {
    give_back();
    return rc;
  }

  // Staging of the scene's per-particle arrays in page-locked memory: the
  // rest-shape pass writes them in place and the upload is a handful of
  // copies at full link bandwidth.
  auto al16 = [](size_t v) { return (v + 15) & ~(size_t)15; };
  const size_t oX = 0, oV = oX + 16 * (size_t)N, oQ = oV + 16 * (size_t)N, oPB = oQ + 16 * (size_t)N;
  const size_t oBR = al16(oPB + 4 * (size_t)N), oQT = al16(oBR + sizeof(BodyRec) * (size_t)B);
  const size_t oCM = oQT + 16 * (size_t)B, oWR = oCM + 16 * (size_t)B;
  const size_t oCK = al16(oWR + sizeof(BodyWrench) * (size_t)B), oOR = al16(oCK + sizeof(Chunk) * chk.size());
  const size_t oSP = al16(oOR + 4 * (size_t)B), stage_bytes = al16(oSP + sizeof(ScenePar));
  {
    const cudaError_t e = c->up_stage.grow(stage_bytes);
    if (e != cudaSuccess) {
      give_back();
      return fail(PBDR_ERR_OOM, std::string("cudaHostAlloc: ") + cudaGetErrorString(e));
    }
  }
  unsigned char *stage = static_cast<unsigned char *>(c->up_stage.p);
  float4 *X = reinterpret_cast<float4 *>(stage + oX), *V = reinterpret_cast<float4 *>(stage + oV);
  float4 *Q = reinterpret_cast<float4 *>(stage + oQ);
  int32_t *pb = reinterpret_cast<int32_t *>(stage + oPB);
  std::vector<BodyRec> br(B);
  std::vector<float4> com(B);
  {
    int32_t slot_next = C0;
    for (int32_t b = 0; b < B; ++b) {
      BodyRec &r = br[b];
      const int32_t s0 = d->body_off[b], s1 = d->body_off[b + 1];
      r.slot0 = slot_next;
      r.nk = (s1 - s0 + kChunk - 1) / kChunk;
      slot_next += r.nk;
      r.start = P0 + s0;
      r.count = s1 - s0;
      r.scene = sid;
      r.has_wrench = 0;
    }
  }
  // host-side FP64 rest shape (Mueller et al. 2005): M, c0, q = x0 - c0;
  // bodies are independent, so large scenes split them over host threads
  auto rest_pass = [&](int32_t b_begin, int32_t b_end, int *bad) {
    std::vector<double> mb;   // particle masses of the current body
    for (int32_t b = b_begin; b < b_end; ++b) {
      const int32_t s0 = d->body_off[b], s1 = d->body_off[b + 1];
      mb.resize((size_t)(s1 - s0));
      double M = 0, cx = 0, cy = 0, cz = 0;
      for (int32_t p = s0; p < s1; ++p) {
        const float w = d->inv_mass[p];
        if (!(w > 0.f) || !std::isfinite(w)) bad[0] = 1;
        if (!finite3(d->pos + 3 * p) || !finite3(d->vel + 3 * p)) bad[1] = 1;
        const double m = 1.0 / (double)w;
        mb[p - s0] = m;
        M += m;
        cx += m * d->pos[3 * p];
        cy += m * d->pos[3 * p + 1];
        cz += m * d->pos[3 * p + 2];
      }
      if (bad[0] || bad[1]) return;
      cx /= M;
      cy /= M;
      cz /= M;
      com[b] = make_float4((float)cx, (float)cy, (float)cz, 0.f);
      double qs[3] = {0, 0, 0};
      for (int32_t p = s0; p < s1; ++p) {
        const double md = mb[p - s0];
        const float4 q = make_float4((float)(d->pos[3 * p] - cx), (float)(d->pos[3 * p + 1] - cy),
                                     (float)(d->pos[3 * p + 2] - cz), (float)md);
        Q[p] = q;
        qs[0] += md * q.x;
        qs[1] += md * q.y;
        qs[2] += md * q.z;
        X[p] = make_float4(d->pos[3 * p], d->pos[3 * p + 1], d->pos[3 * p + 2], d->inv_mass[p]);
        V[p] = make_float4(d->vel[3 * p], d->vel[3 * p + 1], d->vel[3 * p + 2], 0.f);
        pb[p] = B0 + b;
      }
      BodyRec &r = br[b];
      r.mass = (float)M;
      r.inv_mass = (float)(1.0 / M);
      r.qsx = (float)qs[0];
      r.qsy = (float)qs[1];
      r.qsz = (float)qs[2];
    }
  };
  {
    // scenes of 16k particles and more split their bodies over the
    // context's host threads (started once, kept with the context)
    int nthr = 1;
    if (N >= 16384 && B > 1) {
      if (!c->pool) {
        const int hw = std::max(1, (int)std::thread::hardware_concurrency());
        c->pool.reset(new HostPool(std::max(0, std::min(7, hw - 1))));
      }
      nthr = std::max(1, std::min({c->pool->size(), N / 8192, (int)B}));
    }
    std::vector<std::array<int, 2>> bad(nthr, std::array<int, 2>{0, 0});
    if (nthr == 1) {
      rest_pass(0, B, bad[0].data());
    } else {   // contiguous body ranges of about N / nthr particles each
      std::vector<int32_t> cut(nthr + 1, B);
      cut[0] = 0;
      for (int t = 0; t + 1 < nthr; ++t) {
        const int64_t target = (int64_t)N * (t + 1) / nthr;
        int32_t b = std::max(cut[t], (int32_t)0);
        while (b < B && d->body_off[b] < target) ++b;
        cut[t + 1] = b;
      }
      c->pool->run(nthr, [&](int t) {
        if (cut[t] < cut[t + 1]) rest_pass(cut[t], cut[t + 1], bad[t].data());
      });
    }
    int bad_mass = 0, bad_finite = 0;
    for (const auto &f : bad) {
      bad_mass |= f[0];
      bad_finite |= f[1];
    }
    if (bad_mass || bad_finite) {
      give_back();
      return fail(PBDR_ERR_INVALID, bad_mass ? "inverse masses must be finite and > 0"
                                             : "positions and velocities must be finite");
    }
  }
  SceneHost S;
  S.alive = true;
  S.p0 = P0;
  S.np = N;
  S.b0 = B0;
  S.c0 = C0;
  S.nc = nchunks;
  S.nb = B;
  ScenePar &P = S.par;
  P.radius = d->radius;
  P.friction = d->friction;
  P.dt = d->dt;
  P.inv_dt = (float)(1.0 / (double)d->dt);
  P.gx = d->gravity[0];
  P.gy = d->gravity[1];
  P.gz = d->gravity[2];
  P.nx = (float)(d->plane[0] / nl);
  P.ny = (float)(d->plane[1] / nl);
  P.nz = (float)(d->plane[2] / nl);
  P.nd = d->plane[3];
  {  // neighbour-grid constants (FP32): Rn = 2.2 r, cell h = Rn (1 + 2^-10)
    const float Rn = (float)(2.2 * (double)d->radius);
    const float h = (float)((double)Rn * (1.0 + 1.0 / 1024.0));
    volatile float rr = Rn * Rn;
    P.Rn2 = rr;
    P.inv_h = (float)(1.0 / (double)h);
  }
  P.iterations = d->iterations;
  P.flags = d->flags;
  P.T = table_size(N);
  P.c0 = C0;
  P.nc = (int32_t)chk.size();
  P.multi_chunk_bodies = multi;
  P.pad = 0;
  P.p0 = S.p0;
  P.np = N;
  P.b0 = S.b0;
  P.nb = B;
  std::vector<BodyWrench> wr(B);
  std::memset(wr.data(), 0, sizeof(BodyWrench) * (size_t)B);
  // the small per-body and per-scene tables into the staging area too
  std::memcpy(stage + oBR, br.data(), sizeof(BodyRec) * (size_t)B);
  for (int32_t b = 0; b < B; ++b) reinterpret_cast<float4 *>(stage + oQT)[b] = make_float4(0.f, 0.f, 0.f, 1.f);
  std::memcpy(stage + oCM, com.data(), 16 * (size_t)B);
  std::memcpy(stage + oWR, wr.data(), sizeof(BodyWrench) * (size_t)B);
  if (!chk.empty()) std::memcpy(stage + oCK, chk.data(), sizeof(Chunk) * chk.size());
  {  // the scene's bodies, largest first (owner-warp order of the scene-resident kernel)
    int32_t *ord = reinterpret_cast<int32_t *>(stage + oOR);
    for (int32_t b = 0; b < B; ++b) ord[b] = B0 + b;
    std::stable_sort(ord, ord + B, [&](int32_t x, int32_t y) { return br[x - B0].count > br[y - B0].count; });
  }
  std::memcpy(stage + oSP, &P, sizeof(ScenePar));
  // device uploads; on failure the taken ranges go back to the free lists
  auto upload = [&]() -> int {
    // a reused scene slot or table range may still be in use by work that was
    // in flight when it was freed: then wait for the device
    if ((!p_top || !b_top || !c_top || sid < (int32_t)c->sh.size()) && c->free_dirty) {
      CUDA_TRY(cudaDeviceSynchronize());
      c->free_dirty = c->work_pending = c->work_unknown = false;
    }
    // asynchronous copies from the pinned staging buffer on the legacy
    // stream, completed by one synchronisation below (measured: the same
    // copies on a separate non-blocking stream left the tuned substeps 5 %
    // slower; one synchronous copy per array cost 4.5 ns per particle more)
    cudaStream_t us = cudaStreamLegacy;
    auto h2d = [&](void *dst, size_t off, size_t bytes) -> cudaError_t {
      return bytes ? cudaMemcpyAsync(dst, stage + off, bytes, cudaMemcpyHostToDevice, us) : cudaSuccess;
    };
    if (N > 0) {
      CUDA_TRY(h2d(c->X[0].as<float4>() + S.p0, oX, (size_t)N * 16));
      CUDA_TRY(h2d(c->V[0].as<float4>() + S.p0, oV, (size_t)N * 16));
      CUDA_TRY(h2d(c->Q.as<float4>() + S.p0, oQ, (size_t)N * 16));
      CUDA_TRY(h2d(c->pbody.as<int32_t>() + S.p0, oPB, (size_t)N * 4));
      CUDA_TRY(h2d(c->bodies.as<BodyRec>() + S.b0, oBR, (size_t)B * sizeof(BodyRec)));
      CUDA_TRY(h2d(c->quat.as<float4>() + S.b0, oQT, (size_t)B * 16));
      CUDA_TRY(h2d(c->bcom.as<float4>() + S.b0, oCM, (size_t)B * 16));
      CUDA_TRY(h2d(c->wrench.as<BodyWrench>() + S.b0, oWR, (size_t)B * sizeof(BodyWrench)));
      CUDA_TRY(h2d(c->border.as<int32_t>() + B0, oOR, (size_t)B * 4));
    }
    CUDA_TRY(h2d(c->chunks.as<Chunk>() + C0, oCK, chk.size() * sizeof(Chunk)));
    CUDA_TRY(h2d(c->scenes.as<ScenePar>() + sid, oSP, sizeof(ScenePar)));
    CUDA_TRY(cudaMemsetAsync(c->scene_err.as<uint32_t>() + sid, 0, 4, us));
    if (c->dmu.p && (size_t)(sid + 1) * 4 <= c->dmu.bytes)
      CUDA_TRY(cudaMemsetAsync(c->dmu.as<float>() + sid, 0, 4, us));
    if (c->Xb[0].p && N > 0) {   // adjoints in use: the new scene starts with zero adjoints
      if ((rc = ensure_adjoint(c))) return rc;
      for (DevBuf *b : {&c->Xb[0], &c->Xb[1], &c->Vb[0], &c->Vb[1], &c->Ub})
        CUDA_TRY(cudaMemsetAsync(b->as<float4>() + S.p0, 0, (size_t)N * sizeof(float4), us));
    }
    if (c->Xd[0].p && N > 0) {   // tangents in use: the new scene starts with zero tangents
      if ((rc = ensure_tangent(c))) return rc;
      for (DevBuf *b : {&c->Xd[0], &c->Xd[1], &c->Vd[0], &c->Vd[1]})
        CUDA_TRY(cudaMemsetAsync(b->as<float4>() + S.p0, 0, (size_t)N * sizeof(float4), us));
    }
    // complete the uploads and memsets before returning: later work on any
    // stream then sees them, and the staging area may be reused by the next call
    CUDA_TRY(cudaStreamSynchronize(us));
    return PBDR_OK;
  };
  if ((rc = upload())) {
    cudaStreamSynchronize(cudaStreamLegacy);   // no copy still reads the staging area
    give_back();
    return rc;
  }
  if ((int32_t)c->bh.size() < B0 + B) {
    c->bh.resize(B0 + B);
    c->wh.resize(B0 + B);
  }
  std::copy(br.begin(), br.end(), c->bh.begin() + B0);
  std::copy(wr.begin(), wr.end(), c->wh.begin() + B0);
  if (sid == (int32_t)c->sh.size())
    c->sh.push_back(S);
  else
    c->sh[sid] = S;
  if (p_top) c->pa.top = P0 + N;
  if (b_top) c->ba.top = B0 + B;
  if (c_top) c->ca.top = C0 + nchunks;
  c->np_used = c->pa.top;
  c->nb_used = c->ba.top;
  c->nc_used = c->ca.top;
  *out = sid;
  return PBDR_OK;
}

int pbdr_destroy_scene(pbdr_ctx *c, pbdr_scene s) {
  g_err.clear();
  int rc = check_scene(c, s);
  if (rc) return rc;
  // the ranges freed here are clean when the scene's last step and every
  // other call's work have completed (e.g. after a read of its results),
  // even while steps of other scenes run; otherwise the next call that
  // reuses a freed range waits for the device first
  SceneHost &S = c->sh[s];
  c->free_dirty = work_done(c) ? false : (c->free_dirty || !scene_idle(c, S));
  S.alive = false;
  c->pa.give(S.p0, S.np);
  c->ba.give(S.b0, S.nb);
  c->ca.give(S.c0, S.nc);
  drop_plans_with(c, s);
  return PBDR_OK;
}

int pbdr_set_body_wrench(pbdr_ctx *c, pbdr_scene s, int32_t body, const float F[3], const float tau[3]) {
  g_err.clear();
  int rc = check_scene(c, s);
  if (rc) return rc;
  SceneHost &S = c->sh[s];
  if (body < 0 || body >= S.nb) return fail(PBDR_ERR_INVALID, "body index out of range");
  if (!F || !tau || !finite3(F) || !finite3(tau)) return fail(PBDR_ERR_INVALID, "force and torque must be finite");
  CUDA_TRY(cudaDeviceSynchronize());   // steps in flight keep the old wrench
  const int32_t gb = S.b0 + body;
  const bool on = F[0] != 0.f || F[1] != 0.f || F[2] != 0.f || tau[0] != 0.f || tau[1] != 0.f || tau[2] != 0.f;
  BodyWrench &w = c->wh[gb];
  w.force = make_float4(F[0], F[1], F[2], 0.f);
  w.torque = make_float4(tau[0], tau[1], tau[2], 0.f);
  const int was = c->bh[gb].has_wrench;
  c->bh[gb].has_wrench = on ? 1 : 0;
  S.wrench_bodies += (on ? 1 : 0) - was;
  CUDA_TRY(cudaMemcpy(c->wrench.as<BodyWrench>() + gb, &w, sizeof(BodyWrench), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(c->bodies.as<BodyRec>() + gb, &c->bh[gb], sizeof(BodyRec), cudaMemcpyHostToDevice));
  if (S.wrench_bodies)
    S.par.flags |= kSceneHasWrench;
  else
    S.par.flags &= ~kSceneHasWrench;
  CUDA_TRY(cudaMemcpy(c->scenes.as<ScenePar>() + s, &S.par, sizeof(ScenePar), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaStreamSynchronize(cudaStreamLegacy));   // the copies complete before later work on any stream
  if (was != c->bh[gb].has_wrench) drop_plans_with(c, s);
  return PBDR_OK;
}

int pbdr_step(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, int32_t substeps, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  if (!c) return fail(PBDR_ERR_INVALID, "NULL context");
  if (substeps < 0) return fail(PBDR_ERR_INVALID, "substeps must be >= 0");
  Plan *P = nullptr;
  int rc = build_plan(c, ids, n, &P);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = activate(c, P, s))) return rc;
  int64_t launches = 0;
  const bool graphs = c->use_graphs && !c->profiling && s != nullptr && substeps > 0;
  if (graphs && P->graph && P->graph_gen != c->gen) {   // a buffer it uses has moved
    cudaGraphExecDestroy(P->graph);
    P->graph = nullptr;
  }
  for (int32_t k = 0; k < substeps; ++k) {
    // launch shapes are tuned once the plan has run tune_after substeps,
    // on a state where contacts have formed
    if (P->fused && c->autotune && !P->tuned && P->substeps_run >= c->tune_after) {
      if ((rc = autotune_fused(c, *P, s))) return rc;
      if (P->graph) cudaGraphExecDestroy(P->graph);
      P->graph = nullptr;
    }
    if (graphs && !P->graph) {
      if ((rc = capture_plan(c, *P, s))) return rc;
      P->graph_gen = c->gen;
    }
    ++P->substeps_run;
    if (graphs) {
      CUDA_TRY(cudaGraphLaunch(P->graph, s));
      launches += P->graph_launches;
      if (P->fused) c->last_fused_plan = P;
      if (!P->fused || P->rest) c->last_nbr_plan = P->fused ? P->rest.get() : P;
    } else {
      rc = substep(c, *P, s, launches);
      if (rc) return rc;
    }
  }
  c->last_launches = launches;
  stamp_use(c, ids, n, s);
  work_note.quiet = true;
  return PBDR_OK;
}

int pbdr_read_state(pbdr_ctx *c, pbdr_scene s, float *pos, float *vel, uint32_t *err_bits, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  int rc = check_scene(c, s);
  if (rc) return rc;
  if (c->sh[s].np == 0) {
    if (err_bits) {
      CUDA_TRY(cudaMemcpy(err_bits, c->scene_err.as<uint32_t>() + s, 4, cudaMemcpyDeviceToHost));
      CUDA_TRY(cudaMemset(c->scene_err.as<uint32_t>() + s, 0, 4));
    }
    return PBDR_OK;
  }
  rc = transfer_states(c, &s, 1, pos, vel, nullptr, nullptr, err_bits, 0, (cudaStream_t)stream);
  work_note.quiet = rc == PBDR_OK;   // the read synchronised its stream
  return rc;
}

int pbdr_write_state(pbdr_ctx *c, pbdr_scene s, const float *pos, const float *vel, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  int rc = check_scene(c, s);
  if (rc) return rc;
  if (c->sh[s].np == 0) return PBDR_OK;
  return transfer_states(c, &s, 1, nullptr, nullptr, pos, vel, nullptr, 1, (cudaStream_t)stream);
}

int pbdr_read_states(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, float *pos, float *vel,
                     uint32_t *err_bits, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  const int rc = transfer_states(c, ids, n, pos, vel, nullptr, nullptr, err_bits, 0, (cudaStream_t)stream);
  work_note.quiet = rc == PBDR_OK;   // the read synchronised its stream
  return rc;
}

int pbdr_read_states_async(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, float *pos, float *vel,
                           uint32_t *err_bits, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  const int rc = transfer_states(c, ids, n, pos, vel, nullptr, nullptr, err_bits, 0, (cudaStream_t)stream,
                                 nullptr, nullptr, false);
  if (rc == PBDR_OK) {   // the scenes are in use until the stream reaches this point
    stamp_use(c, ids, n, (cudaStream_t)stream);
    work_note.quiet = true;
  }
  return rc;
}

int pbdr_write_states(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, const float *pos, const float *vel,
                      void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  return transfer_states(c, ids, n, nullptr, nullptr, pos, vel, nullptr, 1, (cudaStream_t)stream);
}

int pbdr_step_tangent(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, int32_t substeps, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  if (!c) return fail(PBDR_ERR_INVALID, "NULL context");
  if (substeps < 0) return fail(PBDR_ERR_INVALID, "substeps must be >= 0");
  int rc = check_ids(c, ids, n);
  if (rc) return rc;
  for (int32_t i = 0; i < n; ++i) {
    const SceneHost &S = c->sh[ids[i]];
    if (S.wrench_bodies) return fail(PBDR_ERR_UNSUPPORTED, "tangent substeps of scenes with a body wrench");
    if (S.par.flags & (kStdVelocity | PBDR_SM_FROM_XI))
      return fail(PBDR_ERR_UNSUPPORTED, "tangent substeps with PBDR_STD_VELOCITY or PBDR_SM_FROM_XI");
  }
  Plan *P = nullptr;
  if ((rc = build_plan(c, ids, n, &P, 1))) return rc;
  if ((rc = ensure_tangent(c))) return rc;
  if (c->dmu.p && c->dmu.bytes < (size_t)c->scap * 4) {
    const size_t old = c->dmu.bytes;
    if ((rc = dev_grow(c, c->dmu, (size_t)c->scap * 4, old))) return rc;
    CUDA_TRY(cudaMemset(c->dmu.as<unsigned char>() + old, 0, c->dmu.bytes - old));
  }
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = activate(c, P, s))) return rc;
  int64_t launches = 0;
  for (int32_t k = 0; k < substeps; ++k)
    if ((rc = tangent_substep(c, *P, s, launches))) return rc;
  c->last_launches = launches;
  return PBDR_OK;
}

int pbdr_write_tangent(pbdr_ctx *c, pbdr_scene s, const float *dpos, const float *dvel, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  int rc = check_scene(c, s);
  if (rc) return rc;
  if ((rc = ensure_tangent(c))) return rc;
  const SceneHost &S = c->sh[s];
  if (S.np == 0) return PBDR_OK;
  cudaStream_t st = (cudaStream_t)stream;
  for (DevBuf *b : {&c->Xd[0], &c->Vd[0]})
    CUDA_TRY(cudaMemsetAsync(b->as<float4>() + S.p0, 0, (size_t)S.np * sizeof(float4), st));
  if (!dpos && !dvel) return PBDR_OK;
  return transfer_states(c, &s, 1, nullptr, nullptr, dpos, dvel, nullptr, 1, st, c->Xd[0].as<float4>(),
                         c->Vd[0].as<float4>());
}

int pbdr_read_tangent(pbdr_ctx *c, pbdr_scene s, float *dpos, float *dvel, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  int rc = check_scene(c, s);
  if (rc) return rc;
  if (!c->Xd[0].p) return fail(PBDR_ERR_INVALID, "no tangent has been written");
  if (c->sh[s].np == 0) return PBDR_OK;
  return transfer_states(c, &s, 1, dpos, dvel, nullptr, nullptr, nullptr, 0, (cudaStream_t)stream,
                         c->Xd[0].as<float4>(), c->Vd[0].as<float4>());
}

int pbdr_write_tangent_friction(pbdr_ctx *c, pbdr_scene s, float dmu, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  int rc = check_scene(c, s);
  if (rc) return rc;
  if (!std::isfinite(dmu)) return fail(PBDR_ERR_INVALID, "friction tangent must be finite");
  const size_t need = (size_t)std::max(c->scap, 1) * 4;
  if (c->dmu.bytes < need) {
    const size_t old = c->dmu.p ? c->dmu.bytes : 0;
    if ((rc = dev_grow(c, c->dmu, need, old))) return rc;
    CUDA_TRY(cudaMemset(c->dmu.as<unsigned char>() + old, 0, c->dmu.bytes - old));
  }
  CUDA_TRY(cudaMemcpyAsync(c->dmu.as<float>() + s, &dmu, 4, cudaMemcpyHostToDevice, (cudaStream_t)stream));
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));   // the source is a stack value
  return PBDR_OK;
}

int pbdr_read_adjoint_friction(pbdr_ctx *c, pbdr_scene s, double *mubar, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  int rc = check_scene(c, s);
  if (rc) return rc;
  if (!mubar) return fail(PBDR_ERR_INVALID, "NULL mubar");
  if (!c->Xb[0].p) return fail(PBDR_ERR_INVALID, "no adjoint has been written");
  const SceneHost &S = c->sh[s];
  std::vector<float4> h((size_t)S.np);
  if (S.np > 0) {
    CUDA_TRY(cudaMemcpyAsync(h.data(), c->Xb[0].as<float4>() + S.p0, (size_t)S.np * sizeof(float4),
                             cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  }
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  double acc = 0.0;
  for (const float4 &v : h) acc += (double)v.w;
  *mubar = acc;
  return PBDR_OK;
}

int pbdr_adjoint(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, int32_t substeps, int32_t checkpoint_every,
                 void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  if (!c) return fail(PBDR_ERR_INVALID, "NULL context");
  if (substeps < 0) return fail(PBDR_ERR_INVALID, "substeps must be >= 0");
  if (checkpoint_every < 1) return fail(PBDR_ERR_INVALID, "checkpoint_every must be >= 1");
  int rc = check_ids(c, ids, n);
  if (rc) return rc;
  for (int32_t i = 0; i < n; ++i) {
    const SceneHost &S = c->sh[ids[i]];
    if (S.wrench_bodies) return fail(PBDR_ERR_UNSUPPORTED, "adjoint substeps of scenes with a body wrench");
    if (S.par.flags & (kStdVelocity | PBDR_SM_FROM_XI))
      return fail(PBDR_ERR_UNSUPPORTED, "adjoint substeps with PBDR_STD_VELOCITY or PBDR_SM_FROM_XI");
  }
  Plan *P = nullptr;
  if ((rc = build_plan(c, ids, n, &P, 1))) return rc;
  if ((rc = ensure_adjoint(c))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = activate(c, P, s))) return rc;
  if (substeps == 0) return PBDR_OK;
  const int T = substeps, C = std::min(checkpoint_every, substeps);
  const int nck = (T + C - 1) / C, K = std::max(P->kmax, 1);
  StateSlots S;
  S.np = (size_t)std::max(c->np_used, 1);
  S.nb = (size_t)std::max(c->nb_used, 1);
  const int slots = nck + C + K + 1;   // checkpoints | segment | iterations | final
  if ((rc = dev_alloc(c, c->adj_store, (size_t)slots * (2 * S.np + 2 * S.nb) * sizeof(float4)))) return rc;
  S.base = c->adj_store.as<float4>();
  const int seg0 = nck, it0 = nck + C, fin = nck + C + K;
  int64_t launches = 0;
  for (int t = 0; t < T; ++t) {   // forward, with checkpoints
    if (t % C == 0 && (rc = save_state(c, S, t / C, s))) return rc;
    if ((rc = substep(c, *P, s, launches))) return rc;
  }
  if ((rc = save_state(c, S, fin, s))) return rc;
  CUDA_TRY(cudaMemcpyAsync(c->Xb[1].p, c->Xb[0].p, S.np * 16, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(c->Vb[1].p, c->Vb[0].p, S.np * 16, cudaMemcpyDeviceToDevice, s));
  for (int sg = nck - 1; sg >= 0; --sg) {   // reverse, one segment at a time
    const int t0 = sg * C, t1 = std::min(T, t0 + C);
    if ((rc = load_state(c, S, sg, s))) return rc;
    for (int t = t0; t < t1; ++t) {
      if ((rc = save_state(c, S, seg0 + (t - t0), s))) return rc;
      if (t + 1 < t1 && (rc = substep(c, *P, s, launches))) return rc;
    }
    for (int t = t1 - 1; t >= t0; --t) {
      if ((rc = load_state(c, S, seg0 + (t - t0), s))) return rc;
      if ((rc = adjoint_substep(c, *P, S, it0, s, launches))) return rc;
    }
  }
  if ((rc = load_state(c, S, fin, s))) return rc;
  c->last_launches = launches;
  c->last_nbr_plan = nullptr;   // the lists now belong to a recomputed substep
  return PBDR_OK;
}

int pbdr_write_adjoint(pbdr_ctx *c, pbdr_scene s, const float *xbar, const float *vbar, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  int rc = check_scene(c, s);
  if (rc) return rc;
  if ((rc = ensure_adjoint(c))) return rc;
  const SceneHost &S = c->sh[s];
  if (S.np == 0) return PBDR_OK;
  cudaStream_t st = (cudaStream_t)stream;
  for (DevBuf *b : {&c->Xb[0], &c->Vb[0]})
    CUDA_TRY(cudaMemsetAsync(b->as<float4>() + S.p0, 0, (size_t)S.np * sizeof(float4), st));
  if (!xbar && !vbar) return PBDR_OK;
  return transfer_states(c, &s, 1, nullptr, nullptr, xbar, vbar, nullptr, 1, st, c->Xb[0].as<float4>(),
                         c->Vb[0].as<float4>());
}

int pbdr_read_adjoint(pbdr_ctx *c, pbdr_scene s, float *xbar, float *vbar, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  int rc = check_scene(c, s);
  if (rc) return rc;
  if (!c->Xb[0].p) return fail(PBDR_ERR_INVALID, "no adjoint has been written");
  if (c->sh[s].np == 0) return PBDR_OK;
  return transfer_states(c, &s, 1, xbar, vbar, nullptr, nullptr, nullptr, 0, (cudaStream_t)stream,
                         c->Xb[0].as<float4>(), c->Vb[0].as<float4>());
}

int pbdr_scene_info(pbdr_ctx *c, pbdr_scene s, int32_t *np, int32_t *nb) {
  g_err.clear();
  int rc = check_scene(c, s);
  if (rc) return rc;
  if (np) *np = c->sh[s].np;
  if (nb) *nb = c->sh[s].nb;
  return PBDR_OK;
}

int pbdr_build_neighbors(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  if (!c) return fail(PBDR_ERR_INVALID, "NULL context");
  Plan *P = nullptr;
  int rc = build_plan(c, ids, n, &P, 1);
  if (rc) return rc;
  if (P->np == 0) return PBDR_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = activate(c, P, s))) return rc;
  int64_t launches = 0;
  float4 *X0 = c->X[0].as<float4>();
  launches += launch_predict(predict_args(c, *P, X0, c->V[0].as<float4>(), X0, c->V[0].as<float4>(), 0), s);
  rc = neighbor_stage(c, *P, X0, s, launches);
  if (rc) return rc;
  CUDA_TRY(cudaGetLastError());
  c->last_launches = launches;
  return PBDR_OK;
}

int pbdr_read_neighbors(pbdr_ctx *c, pbdr_scene s, uint32_t *sorted_key, uint32_t *sorted_id, int32_t *off,
                        int32_t *idx, int64_t idx_cap, int64_t *idx_count, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  int rc = check_scene(c, s);
  if (rc) return rc;
  if (!idx_count) return fail(PBDR_ERR_INVALID, "NULL idx_count");
  Plan *P = c->last_nbr_plan;
  int pos_in_plan = -1;
  if (P)
    for (size_t i = 0; i < P->ids.size(); ++i)
      if (P->ids[i] == s) pos_in_plan = (int)i;
  bool fused = false;
  if (pos_in_plan < 0 && c->last_fused_plan) {
    for (auto &F : c->last_fused_plan->classes)
      for (int32_t id : F.ids) fused |= (id == s);
    if (fused && (sorted_key || sorted_id))
      return fail(PBDR_ERR_INVALID, "the scene-resident kernel keeps only the neighbour lists; "
                                    "sorted keys come from pbdr_build_neighbors");
  }
  if (pos_in_plan < 0 && !fused)
    return fail(PBDR_ERR_INVALID, "scene was not part of the last neighbour stage");
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(cudaStreamSynchronize(st));
  const SceneHost &S = c->sh[s];
  const int32_t N = S.np;
  std::vector<uint32_t> k(N), v(N);
  if (N > 0 && !fused) {
    const int64_t so = P->seg_off[pos_in_plan];
    const uint32_t *sk = P->sorted_in_b ? c->s_keys_b.as<uint32_t>() : c->s_keys_a.as<uint32_t>();
    const uint32_t *sv = P->sorted_in_b ? c->s_vals_b.as<uint32_t>() : c->s_vals_a.as<uint32_t>();
    CUDA_TRY(cudaMemcpy(k.data(), sk + so, (size_t)N * 4, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(v.data(), sv + so, (size_t)N * 4, cudaMemcpyDeviceToHost));
  }
  if (!fused) {
    const uint32_t hb = P->hbase_host[s];
    for (int32_t i = 0; i < N; ++i) {
      if (sorted_key) sorted_key[i] = k[i] - hb;
      if (sorted_id) sorted_id[i] = v[i] - (uint32_t)S.p0;
    }
  }
  std::vector<int32_t> cnt(N);
  if (N > 0) CUDA_TRY(cudaMemcpy(cnt.data(), c->nbr_cnt.as<int32_t>() + S.p0, (size_t)N * 4, cudaMemcpyDeviceToHost));
  int32_t maxc = 0;
  int64_t total = 0;
  for (int32_t i = 0; i < N; ++i) {
    maxc = std::max(maxc, cnt[i]);
    total += cnt[i];
  }
  *idx_count = total;
  if (off) {
    off[0] = 0;
    for (int32_t i = 0; i < N; ++i) off[i + 1] = off[i] + cnt[i];
  }
  if (idx && total > 0) {
    std::vector<int32_t> col((size_t)N);
    std::vector<int64_t> at(N + 1, 0);
    for (int32_t i = 0; i < N; ++i) at[i + 1] = at[i] + cnt[i];
    for (int32_t j = 0; j < maxc; ++j) {
      CUDA_TRY(cudaMemcpy(col.data(), c->nbr.as<int32_t>() + (int64_t)j * c->pcap + S.p0, (size_t)N * 4,
                          cudaMemcpyDeviceToHost));
      for (int32_t i = 0; i < N; ++i)
        if (j < cnt[i] && at[i] + j < idx_cap) idx[at[i] + j] = col[i] - S.p0;
    }
  }
  return PBDR_OK;
}

int pbdr_neighbor_total(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, int64_t *total, void *stream) {
  g_err.clear();
  WorkNote work_note{c, (cudaStream_t)stream};
  if (!c || !ids || !total || n < 1) return fail(PBDR_ERR_INVALID, "NULL argument");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int64_t t = 0;
  std::vector<int32_t> cnt;
  for (int32_t i = 0; i < n; ++i) {
    int rc = check_scene(c, ids[i]);
    if (rc) return rc;
    const SceneHost &S = c->sh[ids[i]];
    cnt.resize((size_t)S.np);
    if (S.np) CUDA_TRY(cudaMemcpy(cnt.data(), c->nbr_cnt.as<int32_t>() + S.p0, (size_t)S.np * 4, cudaMemcpyDeviceToHost));
    for (int32_t k = 0; k < S.np; ++k) t += cnt[k];
  }
  *total = t;
  return PBDR_OK;
}

int pbdr_set_profiling(pbdr_ctx *c, int enable) {
  g_err.clear();
  if (!c) return fail(PBDR_ERR_INVALID, "NULL context");
  c->profiling = enable != 0;
  return PBDR_OK;
}

int pbdr_read_profile(pbdr_ctx *c, double *stage_ms, int64_t *stage_launches, int32_t nstages) {
  g_err.clear();
  if (!c || nstages < 0 || nstages > PBDR_NUM_STAGES) return fail(PBDR_ERR_INVALID, "bad argument");
  for (const auto &m : c->marks) {
    CUDA_TRY(cudaEventSynchronize(c->ev_pool[m.e1]));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, c->ev_pool[m.e0], c->ev_pool[m.e1]));
    c->stage_ms[m.stage] += ms;
    c->stage_launches[m.stage] += m.launches;
  }
  c->marks.clear();
  c->ev_used = 0;
  for (int32_t k = 0; k < nstages; ++k) {
    if (stage_ms) stage_ms[k] = c->stage_ms[k];
    if (stage_launches) stage_launches[k] = c->stage_launches[k];
  }
  for (int k = 0; k < PBDR_NUM_STAGES; ++k) {
    c->stage_ms[k] = 0.0;
    c->stage_launches[k] = 0;
  }
  return PBDR_OK;
}

int pbdr_set_option(pbdr_ctx *c, int32_t option, int64_t value) {
  g_err.clear();
  if (!c) return fail(PBDR_ERR_INVALID, "NULL context");
  switch (option) {
    case PBDR_OPT_PATH:
      if (value != 0 && value != 1) return fail(PBDR_ERR_INVALID, "PBDR_OPT_PATH takes 0 or 1");
      c->path = (int)value;
      break;
    case PBDR_OPT_GRAPHS:
      c->use_graphs = value != 0;
      break;
    case PBDR_OPT_AUTOTUNE:
      c->autotune = value != 0;
      break;
    case PBDR_OPT_TUNE_AFTER:
      if (value < 1) return fail(PBDR_ERR_INVALID, "PBDR_OPT_TUNE_AFTER takes a substep count >= 1");
      c->tune_after = value;
      break;
    case PBDR_OPT_FUSED_THREADS:
      if (value != 0 && (value < 32 || value > 512 || value % 32))
        return fail(PBDR_ERR_INVALID, "PBDR_OPT_FUSED_THREADS takes 0 or a multiple of 32 in 32..512");
      c->fused_threads = (int)value;
      break;
    default:
      return fail(PBDR_ERR_INVALID, "unknown option " + std::to_string(option));
  }
  invalidate_plans(c);
  return PBDR_OK;
}

int pbdr_plan_config(pbdr_ctx *c, const pbdr_scene *ids, int32_t n, int32_t *out, int32_t cap) {
  g_err.clear();
  if (!c || !out || cap < 5 * kNumClasses)
    return fail(PBDR_ERR_INVALID, "need an output array of " + std::to_string(5 * kNumClasses) + " int32");
  Plan *P = nullptr;
  int rc = build_plan(c, ids, n, &P);
  if (rc) return rc;
  for (int k = 0; k < kNumClasses; ++k) {
    const bool has = P->fused;
    out[5 * k + 0] = has ? P->classes[k].ncap : 0;
    out[5 * k + 1] = has ? P->classes[k].n : 0;
    out[5 * k + 2] = has ? P->classes[k].threads : 0;
    out[5 * k + 3] = has ? ((P->classes[k].v_shared ? 1 : 0) | (P->classes[k].dx_shared ? 2 : 0)) : 0;
    out[5 * k + 4] = has ? P->classes[k].grid : 0;
  }
  return PBDR_OK;
}

int pbdr_last_launch_count(pbdr_ctx *c, int64_t *launches) {
  g_err.clear();
  if (!c || !launches) return fail(PBDR_ERR_INVALID, "NULL argument");
  *launches = c->last_launches;
  return PBDR_OK;
}

}  // extern "C"
