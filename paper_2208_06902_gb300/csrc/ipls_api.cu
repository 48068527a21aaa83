// Host runtime behind the C ABI of include/ipls.h: contexts, scratch memory,
// the level loop of the learned partitioning recursion, segmented sorting
// and request tickets.  Every step of the sort runs in the kernels of
// ipls_pass.cu and ipls_resident.cu; this file only plans and launches them.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ipls.h"
#include "ipls_device.cuh"

namespace {

using namespace ipls;

thread_local std::string g_last_error;

// Offsets inside a bucket are kept in 32 bits per tile.
constexpr int64_t kMaxKeys = (int64_t(1) << 32) - 1;
// Device-driven levels enqueued at most (deeper recursion continues with
// host-driven levels).
constexpr int kDevLevelsMax = 8;

iplsStatus fail(iplsStatus st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

iplsStatus cuda_fail(cudaError_t e, const char* where) {
  return fail(IPLS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define IPLS_CUDA(call)                                      \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);      \
  } while (0)

#define IPLS_TRY(call)                                       \
  do {                                                       \
    iplsStatus s_ = (call);                                  \
    if (s_ != IPLS_OK) return s_;                            \
  } while (0)

struct Slot {
  Sub* subs = nullptr;           int64_t sub_cap = 0;
  int32_t* tile2sub = nullptr;   int64_t tile_cap = 0;
  int32_t* chunk2sub = nullptr;  int64_t chunk_cap = 0;
  Model* models = nullptr;       int64_t model_cap = 0;
  ThrTable* tabs = nullptr;      int64_t tab_cap = 0;
  float* knots = nullptr;        int64_t knot_cap = 0;   // PL2 knots, when enabled
  uint64_t* counts = nullptr;    int64_t count_cap = 0;
  int64_t* bases = nullptr;      int64_t base_cap = 0;
  Group* groups = nullptr;       int64_t group_cap = 0;
  int32_t* fit_list = nullptr;   int64_t fit_cap = 0;
  TailModel* tails = nullptr;    int64_t tail_cap = 0;
  Fill* fills = nullptr;         int64_t fill_cap = 0;
};

// One sort in flight: its stream, the ping-pong buffer and per-level lists,
// the device counters and their pinned host copies.  A context has one
// workspace for its own synchronous calls and, once requests are submitted,
// one per in-flight batch slot, so that batches run side by side on the GPU.
struct Pending { int kind; int level; cudaEvent_t a, b; };
struct Workspace {
  iplsCtx c = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;            // created by the library (batch slots)
  bool main = false;                  // the context's own calls: traced and profiled
  char* scratch = nullptr;            int64_t scratch_cap = 0;   // bytes
  unsigned long long* status = nullptr; int64_t status_cap = 0;  // words
  uint32_t* tile_off = nullptr;       int64_t tile_off_cap = 0;  // words
  uint8_t* bids = nullptr;            int64_t bids_cap = 0;      // bytes
  uint32_t epoch = 0;
  Slot slot[2];
  LevelCtl* ctl = nullptr;
  RunStatus* run = nullptr;
  int64_t* root_bounds = nullptr;
  LevelCtl* h_ctl = nullptr;          // pinned
  RunStatus* h_run = nullptr;         // pinned
  // slow lists of the block-resident tail (children / whole tasks, one half each)
  SlowTask* slow = nullptr;           int64_t slow_cap = 0;
  SlowCtl* slow_ctl = nullptr;
  SlowCtl* h_slow = nullptr;          // pinned copy of *slow_ctl
  uint64_t* split_pool = nullptr;     int64_t split_pool_cap = 0;  // words
  // a batch of separate arrays: segment offsets and bases (device, pinned host)
  int64_t* seg_off = nullptr;         int64_t seg_off_cap = 0;
  uint64_t* seg_ubase = nullptr;      int64_t seg_ubase_cap = 0;
  int64_t* h_seg_off = nullptr;       uint64_t* h_seg_ubase = nullptr;  int64_t h_seg_cap = 0;
  iplsStats stats{};                  // the last sort on this workspace
  int64_t trace_grid_count = 0;
  std::vector<Pending> pending;       // profiling: event pairs per launch
  std::vector<cudaEvent_t> spare_events;
  // device-driven levels: one LevelCtl per level (entry 0: the segment
  // lists), their pinned copy, the grid trace counter, and the captured
  // graph of the last segmented call with its key
  LevelCtl* ctl_arr = nullptr;
  LevelCtl* h_ctl_arr = nullptr;
  long long* trace_ctr = nullptr;
  long long* h_trace_ctr = nullptr;
  bool capturing = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  struct GraphKey {
    void* keys; const int64_t* offsets; const uint64_t* ubase; int64_t n, nseg; int dtype, levels;
    bool operator==(const GraphKey& o) const {
      return keys == o.keys && offsets == o.offsets && ubase == o.ubase && n == o.n && nseg == o.nseg &&
             dtype == o.dtype && levels == o.levels;
    }
  } gkey{};
};

}  // namespace

struct iplsContext {
  iplsConfig cfg;
  iplsAllocFn alloc = nullptr;
  iplsFreeFn free_fn = nullptr;
  void* user = nullptr;
  int device = 0;
  int num_sms = 0;
  Workspace ws;                       // the context's own calls (its stream)
  iplsTraceRecDev* trace_grid = nullptr;
  iplsTraceRecDev* trace_res = nullptr;
  int64_t trace_alloc = 0;
  float* trace_knots = nullptr;       int64_t knot_cap = 0;       // records
  int knot_leaves = 0;
  int64_t calls = 0;
  // request serving (iplsSubmit): kServeSlots worker threads, each with its
  // own workspace and stream, take batches from the queue as they free up
  struct Request {
    void* keys;
    int64_t n;
    int dtype;
    iplsStatus st;
    bool done;
    std::string msg;     // the failure's message (set on the worker thread)
  };
  static constexpr int kServeSlots = 2;
  std::mutex exec_mu;                 // one synchronous sort at a time on the context
  std::mutex q_mu;                    // guards the queue, the requests and the batch log
  std::condition_variable q_cv;       // new request, a slot freed memory, or stop
  std::condition_variable done_cv;    // a request finished
  std::deque<uint64_t> queue;
  std::map<uint64_t, Request> reqs;
  std::thread workers[kServeSlots];
  Workspace serve_ws[kServeSlots];
  bool stop = false;
  uint64_t next_ticket = 1;
  int64_t inflight_bytes = 0;         // 2*w*n of the admitted requests not yet done
  cudaEvent_t serve_ref = nullptr;    // time origin of the batch log
  std::vector<iplsBatchRec> batch_log;
  std::atomic<int64_t> dev_bytes{0};
  std::mutex prof_mu;                 // guards the profile accumulators
  int64_t k_launches[16] = {};
  // per grid level (profile = 1): summed time of the level's grid kernels,
  // their launches, and the keys (and algorithmic bytes) its passes moved
  static constexpr int kLevels = 16;
  double lv_ms[kLevels] = {};
  int64_t lv_launches[kLevels] = {};
  int64_t lv_keys[kLevels] = {};
  int64_t lv_bytes[kLevels] = {};
  double k_ms[16] = {};
  int64_t k_bytes[16] = {};
  // host-buffer sorting
  char* host_stage = nullptr; int64_t host_stage_cap = 0;
  // pipelined host batches: three device buffers in rotation (one arriving,
  // one being sorted, one leaving), a copy stream each way, their events
  char* pipe_buf[3] = {}; int64_t pipe_cap[3] = {};
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t in_ev[3] = {}, sorted_ev[3] = {}, out_ev[3] = {};
};

namespace {

iplsStatus dev_alloc(iplsCtx c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (c->alloc) {
    *p = c->alloc(bytes, c->user);
    if (!*p) return fail(IPLS_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return fail(IPLS_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  c->dev_bytes += (int64_t)bytes;
  return IPLS_OK;
}

void dev_free(iplsCtx c, void* p, size_t bytes) {
  if (!p) return;
  if (c->free_fn) c->free_fn(p, c->user);
  else cudaFree(p);
  c->dev_bytes -= (int64_t)bytes;
}

// Grows a device array to hold at least `need` elements (contents dropped).
template <class T>
iplsStatus ensure(Workspace& w, T*& p, int64_t& cap, int64_t need) {
  if (need <= cap && p) return IPLS_OK;
  iplsCtx c = w.c;
  IPLS_CUDA(cudaStreamSynchronize(w.stream));
  dev_free(c, p, (size_t)cap * sizeof(T));
  p = nullptr;
  cap = 0;
  const int64_t want = need + need / 4 + 16;
  void* q;
  IPLS_TRY(dev_alloc(c, &q, (size_t)want * sizeof(T)));
  p = reinterpret_cast<T*>(q);
  cap = want;
  return IPLS_OK;
}

bool valid_dtype(int d) { return d >= 0 && d <= 3; }

enum KernelKind { kkFit, kkHist, kkCheck, kkRehist, kkScan, kkScatter, kkResident, kkFill,
                  kkInitSeg, kkInitTiles, kkTailFit, kkTileScan, kkSlow, kkSlowGroups, kkCount };
const char* const kKernelNames[kkCount] = {"k_fit", "k_hist", "k_check", "k_hist_redo", "k_scan",
                                           "k_scatter", "k_tail", "k_fill",
                                           "k_init_segments", "k_init_tiles", "k_tail_fit",
                                           "k_tilescan", "k_slow", "k_slow_groups"};

cudaEvent_t take_event(Workspace& w) {
  if (!w.spare_events.empty()) {
    cudaEvent_t e = w.spare_events.back();
    w.spare_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return e;
}

// Launches `fn` (which enqueues exactly one kernel) bracketed by CUDA events
// when profiling; every launch is counted.
template <class F>
cudaError_t timed(Workspace& w, int kind, F fn, int level = -1) {
  if (!w.c->cfg.profile || !w.main || w.capturing) {
    cudaError_t e = fn();
    return e;
  }
  cudaEvent_t a = take_event(w), b = take_event(w);
  if (a) cudaEventRecord(a, w.stream);
  cudaError_t e = fn();
  if (b) cudaEventRecord(b, w.stream);
  if (a && b) w.pending.push_back({kind, level, a, b});
  return e;
}

// Folds finished event pairs into the per-kernel totals (after a sync).
void resolve_events(Workspace& w) {
  iplsCtx c = w.c;
  std::lock_guard<std::mutex> lk(c->prof_mu);
  for (auto& p : w.pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->k_ms[p.kind] += ms;
      c->k_launches[p.kind] += 1;
      if (p.level >= 0 && p.level < iplsContext::kLevels) {
        c->lv_ms[p.level] += ms;
        c->lv_launches[p.level] += 1;
      }
    } else {
      cudaGetLastError();
    }
    w.spare_events.push_back(p.a);
    w.spare_events.push_back(p.b);
  }
  w.pending.clear();
}

// Grid kernels size their grids from the occupancy of the SMs they get.
int occupancy_grid(iplsCtx c, int, int) { return c->num_sms; }

// Group list of a slot with its fit list and fitted tail models.
iplsStatus ensure_groups(Workspace& w, Slot& s, int64_t need) {
  IPLS_TRY(ensure(w, s.groups, s.group_cap, need));
  IPLS_TRY(ensure(w, s.fit_list, s.fit_cap, s.group_cap));
  IPLS_TRY(ensure(w, s.tails, s.tail_cap, s.group_cap));
  return IPLS_OK;
}

// Splitter-pool slots for a tail sweep of nfit fitted tasks.
int64_t pool_slots(int64_t nfit) {
  return std::min<int64_t>(std::max<int64_t>(nfit, kSplitPoolMin), kSplitPoolMax);
}

// One sweep of k_tail_fit + k_tail over the groups in ra.
iplsStatus tail_sweep(Workspace& w, ResidentArgs& ra) {
  iplsCtx c = w.c;
  if (ra.nfit > 0) {
    IPLS_TRY(ensure(w, w.split_pool, w.split_pool_cap, pool_slots(ra.nfit) * 128));
    ra.split_pool = w.split_pool;
    ra.split_pool_slots = (int32_t)std::min<int64_t>(w.split_pool_cap / 128, kSplitPoolMax);
    IPLS_CUDA(timed(w, kkTailFit, [&] { return launch_tail_fit(ra, w.stream, c->num_sms); }));
  }
  if (ra.ngroups > 0)
    IPLS_CUDA(timed(w, kkResident, [&] { return launch_resident(ra, w.stream, 0, c->num_sms); }));
  if ((ra.large_from_end ? ra.nlarge : ra.ngroups) > 0)
    IPLS_CUDA(timed(w, kkResident, [&] { return launch_resident(ra, w.stream, 1, c->num_sms); }));
  return IPLS_OK;
}

// Fits and runs the block-resident tasks listed in slot s: one sweep over
// them, a second one over the children above the cutoff when the first
// queued many (in place in the user buffer; the slot's group list is free
// again once the first sweep ran), and k_slow for the rest.
// nsmall/nlarge: from a level's list (small tasks from the front, large ones
// from the back); with nlarge < 0 the nsmall groups are in plain order and
// both k_tail sizes walk them all.
iplsStatus launch_tail(Workspace& w, ResidentArgs& ra, Slot& s, int32_t nsmall, int32_t nlarge, int32_t nfit) {
  iplsCtx c = w.c;
  const bool from_end = nlarge >= 0;
  const int32_t ngroups = from_end ? nsmall + nlarge : nsmall;
  ra.groups = s.groups;
  ra.ngroups = nsmall;
  ra.nlarge = from_end ? nlarge : nsmall;
  ra.group_cap = (int32_t)std::min<int64_t>(s.group_cap, INT32_MAX);
  ra.large_from_end = from_end ? 1 : 0;
  ra.fit_list = s.fit_list;
  ra.nfit = nfit;
  ra.tail_models = s.tails;
  // disjoint ranges of more than `cutoff` keys each: both lists together
  // hold at most n / (cutoff + 1), and each half of the buffer holds that
  const int64_t half = w.slow_cap / 2;
  ra.slow = w.slow;
  ra.slow_cap = (int32_t)std::min<int64_t>(half, INT32_MAX);
  ra.whole = w.slow + half;
  ra.whole_cap = (int32_t)std::min<int64_t>(w.slow_cap - half, INT32_MAX);
  ra.slow_ctl = w.slow_ctl;
  ra.split_pool = w.split_pool;
  ra.split_pool_slots = (int32_t)std::min<int64_t>(w.split_pool_cap / 128, kSplitPoolMax);
  if (ngroups <= 0) return IPLS_OK;
  IPLS_CUDA(cudaMemsetAsync(w.slow_ctl, 0, sizeof(SlowCtl), w.stream));
  IPLS_TRY(tail_sweep(w, ra));
  if (ngroups >= kTailSweepMin) {
    IPLS_CUDA(cudaMemcpyAsync(w.h_slow, w.slow_ctl, sizeof(SlowCtl), cudaMemcpyDeviceToHost, w.stream));
    IPLS_CUDA(cudaStreamSynchronize(w.stream));
    const int32_t nc = w.h_slow->count;
    if (nc >= kTailSweepMin && nc <= ra.slow_cap) {
      IPLS_TRY(ensure_groups(w, s, nc));
      IPLS_CUDA(timed(w, kkSlowGroups, [&] { return launch_slow_groups(w.slow, nc, s.groups, s.fit_list, w.stream); }));
      // the child list starts again (count, ticket, pool_used, fit_ticket);
      // whole tasks stay
      IPLS_CUDA(cudaMemsetAsync(w.slow_ctl, 0, 4 * sizeof(int32_t), w.stream));
      ra.groups = s.groups;
      ra.ngroups = nc;
      ra.nlarge = nc;            // plain order: both sizes walk the list
      ra.large_from_end = 0;
      ra.fit_list = s.fit_list;
      ra.nfit = nc;
      ra.tail_models = s.tails;
      IPLS_TRY(tail_sweep(w, ra));
      w.stats.sweep_tasks += nc;
    }
  }
  IPLS_CUDA(timed(w, kkSlow, [&] { return launch_slow(ra, w.stream, c->num_sms); }));
  return IPLS_OK;
}

iplsStatus check_run(Workspace& w) {
  IPLS_CUDA(cudaMemcpyAsync(w.h_run, w.run, sizeof(RunStatus), cudaMemcpyDeviceToHost, w.stream));
  IPLS_CUDA(cudaStreamSynchronize(w.stream));
  if (w.h_run->error == IPLS_ERR_TIMEOUT)
    return fail(IPLS_ERR_TIMEOUT, "a device-side look-back wait exceeded spin_limit");
  if (w.h_run->error != 0)
    return fail((iplsStatus)w.h_run->error, "device reported status " + std::to_string(w.h_run->error));
  w.stats.resident_groups = w.h_run->resident_groups;
  w.stats.slow_tasks = w.h_run->slow_tasks;
  w.stats.slow_passes = w.h_run->slow_passes;
  w.stats.fallback_passes += w.h_run->resident_fallback;
  w.stats.trace_records = w.trace_grid_count + w.h_run->trace_count;
  return IPLS_OK;
}

// ---------------------------------------------------------------------------
// Device-driven levels (segmented sorts, cfg.flags & IPLS_FLAG_GRAPH): every
// buffer is sized for the worst case first, then the levels are enqueued
// with no host round trip -- each kernel reads its level's counts from the
// LevelCtl the previous level left on the device and loops over them with a
// fixed grid -- so that the whole sequence can be captured into a CUDA graph
// and replayed.  One readback at the end gives the statistics, any error,
// and whether the recursion needs more levels than were enqueued.
// ---------------------------------------------------------------------------
struct DevCaps {
  int64_t sub, tile, chunk, group, fill;
};

DevCaps dev_caps(const iplsConfig& cfg, int64_t n, int64_t nseg, int dtype) {
  const int rmax = resident_rmax(cfg.cutoff);
  DevCaps d;
  d.sub = n / (rmax + 1) + 2;
  d.tile = n / tile_keys(dtype) + d.sub + 2;
  d.chunk = d.tile / kChunkTiles + d.sub + 2;
  d.group = 2 * n / (cfg.cutoff + 1) + 257 * d.sub + 16 + nseg + 1024;
  d.fill = n / kFillChunk + 129 * d.sub + 16;
  return d;
}

// Subproblems a slot can hold in every per-subproblem array, and tiles and
// chunks the level arrays can hold (arrays grown by earlier calls may differ
// in capacity).
int64_t slot_sub_limit(const Workspace& w, const Slot& X) {
  const iplsConfig& cfg = w.c->cfg;
  int64_t m = std::min(X.sub_cap, X.model_cap);
  m = std::min(m, X.count_cap / kMaxK);
  m = std::min(m, X.base_cap / 257);
  if (cfg.flags & IPLS_FLAG_THRESHOLD_INDEX) m = std::min(m, X.tab_cap);
  if (cfg.pl2_leaves > 0) m = std::min(m, X.knot_cap / (cfg.pl2_leaves + 1));
  return std::min<int64_t>(m, INT32_MAX);
}
int64_t slot_tile_limit(const Workspace& w, const Slot& X) {
  return std::min(X.tile_cap, w.tile_off_cap / kMaxK);
}
int64_t slot_chunk_limit(const Workspace& w, const Slot& X) {
  return std::min(X.chunk_cap, w.status_cap / kMaxK);
}

iplsStatus device_prepare(Workspace& w, int64_t n, int64_t nseg, int dtype) {
  iplsCtx c = w.c;
  const iplsConfig& cfg = c->cfg;
  const DevCaps d = dev_caps(cfg, n, nseg, dtype);
  IPLS_TRY(ensure(w, w.scratch, w.scratch_cap, n * (int64_t)key_bytes(dtype)));
  IPLS_TRY(ensure(w, w.bids, w.bids_cap, n + 16));
  IPLS_TRY(ensure(w, w.slow, w.slow_cap, 2 * (n / (cfg.cutoff + 1)) + 4096));
  for (Slot& X : w.slot) {
    IPLS_TRY(ensure(w, X.subs, X.sub_cap, d.sub));
    IPLS_TRY(ensure(w, X.tile2sub, X.tile_cap, d.tile));
    IPLS_TRY(ensure(w, X.chunk2sub, X.chunk_cap, d.chunk));
    IPLS_TRY(ensure(w, X.models, X.model_cap, d.sub));
    IPLS_TRY(ensure(w, X.tabs, X.tab_cap, (cfg.flags & IPLS_FLAG_THRESHOLD_INDEX) ? d.sub : 1));
    if (cfg.pl2_leaves > 0) IPLS_TRY(ensure(w, X.knots, X.knot_cap, d.sub * (int64_t)(cfg.pl2_leaves + 1)));
    IPLS_TRY(ensure(w, X.counts, X.count_cap, d.sub * kMaxK));
    IPLS_TRY(ensure(w, X.bases, X.base_cap, d.sub * 257));
    IPLS_TRY(ensure_groups(w, X, d.group));
    IPLS_TRY(ensure(w, X.fills, X.fill_cap, d.fill));
  }
  IPLS_TRY(ensure(w, w.tile_off, w.tile_off_cap, d.tile * kMaxK));
  IPLS_TRY(ensure(w, w.status, w.status_cap, d.chunk * kMaxK));
  IPLS_TRY(ensure(w, w.split_pool, w.split_pool_cap, pool_slots(d.group) * 128));
  if (!w.ctl_arr) {
    void* p;
    IPLS_TRY(dev_alloc(c, &p, (kDevLevelsMax + 1) * sizeof(LevelCtl)));
    w.ctl_arr = (LevelCtl*)p;
    IPLS_TRY(dev_alloc(c, &p, sizeof(long long)));
    w.trace_ctr = (long long*)p;
    IPLS_CUDA(cudaMallocHost(&w.h_ctl_arr, (kDevLevelsMax + 1) * sizeof(LevelCtl)));
    IPLS_CUDA(cudaMallocHost(&w.h_trace_ctr, sizeof(long long)));
  }
  return IPLS_OK;
}

// The tail of one device-driven level: its groups in slot s, counted in
// *gcnt; a second sweep over the children above the cutoff when there are
// at least kTailSweepMin of them; k_slow for the rest.
// max_task: the largest task the groups can hold (tasks above kTailSmall
// keys need the large k_tail); sweep: whether a second sweep can occur (it
// needs kTailSweepMin children above the cutoff).  Launches that the sizes
// rule out are left out of the graph.
iplsStatus launch_tail_dev(Workspace& w, ResidentArgs ra, Slot& s, LevelCtl* gcnt, int64_t max_task,
                           bool sweep) {
  iplsCtx c = w.c;
  const int32_t cap = (int32_t)std::min<int64_t>(std::min(s.group_cap, std::min(s.fit_cap, s.tail_cap)), INT32_MAX);
  ra.groups = s.groups;
  ra.ngroups = cap;
  ra.nlarge = cap;
  ra.group_cap = cap;
  ra.large_from_end = 1;
  ra.fit_list = s.fit_list;
  ra.nfit = cap;
  ra.tail_models = s.tails;
  ra.gcnt = gcnt;
  ra.device_counts = 1;
  ra.sweep = 0;
  const int64_t half = w.slow_cap / 2;
  ra.slow = w.slow;
  ra.slow_cap = (int32_t)std::min<int64_t>(half, INT32_MAX);
  ra.whole = w.slow + half;
  ra.whole_cap = (int32_t)std::min<int64_t>(w.slow_cap - half, INT32_MAX);
  ra.slow_ctl = w.slow_ctl;
  ra.split_pool = w.split_pool;
  ra.split_pool_slots = (int32_t)std::min<int64_t>(w.split_pool_cap / 128, kSplitPoolMax);
  const bool large = max_task > kTailSmall;
  IPLS_CUDA(cudaMemsetAsync(w.slow_ctl, 0, sizeof(SlowCtl), w.stream));
  IPLS_CUDA(timed(w, kkTailFit, [&] { return launch_tail_fit(ra, w.stream, c->num_sms); }));
  IPLS_CUDA(timed(w, kkResident, [&] { return launch_resident(ra, w.stream, 0, c->num_sms); }));
  if (large) IPLS_CUDA(timed(w, kkResident, [&] { return launch_resident(ra, w.stream, 1, c->num_sms); }));
  if (sweep) {
    IPLS_CUDA(timed(w, kkSlowGroups, [&] {
      return launch_sweep_groups(w.slow, w.slow_ctl, ra.slow_cap, s.groups, s.fit_list, cap, w.stream);
    }));
    ResidentArgs rb = ra;
    rb.sweep = 1;
    rb.large_from_end = 0;
    IPLS_CUDA(timed(w, kkTailFit, [&] { return launch_tail_fit(rb, w.stream, c->num_sms); }));
    IPLS_CUDA(timed(w, kkResident, [&] { return launch_resident(rb, w.stream, 0, c->num_sms); }));
    if (large) IPLS_CUDA(timed(w, kkResident, [&] { return launch_resident(rb, w.stream, 1, c->num_sms); }));
  }
  IPLS_CUDA(timed(w, kkSlow, [&] { return launch_slow(ra, w.stream, c->num_sms); }));
  return IPLS_OK;
}

// Enqueues the segment lists and `levels` device-driven levels (buffers from
// device_prepare; no allocation and no host synchronisation), then copies
// the level counters, the run status and the trace counter to pinned memory.
iplsStatus device_enqueue(Workspace& w, int64_t n, int dtype, const int64_t* offsets, int64_t nseg,
                          const uint64_t* seg_ubase, uint64_t ubase, int levels) {
  iplsCtx c = w.c;
  const iplsConfig& cfg = c->cfg;
  const bool traced = w.main && cfg.trace_cap > 0;
  const int rmax = resident_rmax(cfg.cutoff);
  const int resident_root_ok = (cfg.root_sample <= 0 || cfg.root_sample <= kResidentSample);
  IPLS_CUDA(cudaMemsetAsync(w.run, 0, sizeof(RunStatus), w.stream));
  IPLS_CUDA(cudaMemsetAsync(w.ctl_arr, 0, (size_t)(levels + 1) * sizeof(LevelCtl), w.stream));
  IPLS_CUDA(cudaMemsetAsync(w.trace_ctr, 0, sizeof(long long), w.stream));
  ResidentArgs ra{};
  ra.dtype = dtype; ra.k = cfg.k; ra.cutoff = cfg.cutoff; ra.root_sample = cfg.root_sample;
  ra.seed = cfg.seed; ra.exact_only = cfg.exact_only; ra.buf[0] = nullptr; ra.buf[1] = w.scratch;
  ra.run = w.run; ra.trace = traced ? c->trace_res : nullptr; ra.trace_cap = traced ? cfg.trace_cap : 0;
  Slot& s0 = w.slot[0];
  Slot& s1 = w.slot[1];
  IPLS_CUDA(timed(w, kkInitSeg, [&] {
    return launch_init_segments(offsets, nseg, seg_ubase, ubase, rmax, cfg.cutoff, resident_root_ok, &w.ctl_arr[0],
                                s0.subs, (int32_t)slot_sub_limit(w, s0), s0.tile2sub,
                                slot_tile_limit(w, s0), s0.chunk2sub, slot_chunk_limit(w, s0), s1.groups,
                                (int32_t)std::min<int64_t>(std::min(s1.group_cap, std::min(s1.fit_cap, s1.tail_cap)),
                                                           INT32_MAX),
                                s1.fit_list, w.stream);
  }));
  // the second sweep needs kTailSweepMin children above the cutoff
  const bool sweep = n >= (int64_t)kTailSweepMin * (cfg.cutoff + 1);
  IPLS_TRY(launch_tail_dev(w, ra, s1, &w.ctl_arr[0], std::min<int64_t>(n, rmax), sweep));
  for (int level = 0; level < levels; ++level) {
    // the largest sample of the level: that of an n-key subproblem (level 0
    // may have its own root sample size)
    const int sample_bound = sample_size_host(std::max<int64_t>(n, 2), level == 0 ? 0 : 1, cfg.k, cfg.root_sample);
    Slot& X = w.slot[level & 1];
    Slot& Y = w.slot[(level + 1) & 1];
    // look-back words start from zero at every level (epoch 1 throughout),
    // so a replayed graph never meets words of an earlier replay
    IPLS_CUDA(cudaMemsetAsync(w.status, 0, (size_t)w.status_cap * 8, w.stream));
    LevelArgs a{};
    a.dtype = dtype; a.k = cfg.k; a.cutoff = cfg.cutoff; a.rmax = rmax;
    a.root_sample = cfg.root_sample; a.seed = cfg.seed; a.exact_only = cfg.exact_only;
    a.use_tables = (cfg.flags & IPLS_FLAG_THRESHOLD_INDEX) && !cfg.exact_only;
    a.spin_limit = cfg.spin_limit; a.epoch = 1; a.level = level;
    a.buf[0] = nullptr; a.buf[1] = w.scratch;
    a.nsub = (int32_t)slot_sub_limit(w, X);
    a.subs = X.subs; a.models = X.models; a.counts = X.counts; a.tabs = X.tabs; a.bases = X.bases;
    a.tile2sub = X.tile2sub; a.ntiles = slot_tile_limit(w, X); a.chunk2sub = X.chunk2sub;
    a.nchunks = slot_chunk_limit(w, X);
    a.status = w.status; a.tile_off = w.tile_off; a.bids = w.bids;
    a.ctl = &w.ctl_arr[level + 1]; a.run = w.run; a.cnt = &w.ctl_arr[level];
    a.next_subs = Y.subs; a.next_sub_cap = (int32_t)slot_sub_limit(w, Y);
    a.next_tile2sub = Y.tile2sub; a.next_tile_cap = slot_tile_limit(w, Y);
    a.next_chunk2sub = Y.chunk2sub; a.next_chunk_cap = slot_chunk_limit(w, Y);
    a.groups = X.groups;
    a.group_cap = (int32_t)std::min<int64_t>(std::min(X.group_cap, std::min(X.fit_cap, X.tail_cap)), INT32_MAX);
    a.fit_list = X.fit_list;
    a.fills = X.fills; a.fill_cap = (int32_t)std::min<int64_t>(X.fill_cap, INT32_MAX);
    a.trace = traced ? c->trace_grid : nullptr;
    a.trace_cap = traced ? cfg.trace_cap : 0;
    a.trace_base = 0;
    a.trace_ctr = traced ? w.trace_ctr : nullptr;
    a.trace_knots = traced ? c->trace_knots : nullptr;
    a.knot_cap = c->knot_cap;
    a.max_sample = sample_bound;
    a.pl2_leaves = cfg.pl2_leaves;
    a.pl2_depth = cfg.pl2_depth;
    a.knots = cfg.pl2_leaves > 0 ? X.knots : nullptr;
    const int sms = c->num_sms;
    IPLS_CUDA(timed(w, kkFit, [&] { return launch_fit(a, w.stream, sample_bound, sms); }, level));
    IPLS_CUDA(timed(w, kkHist, [&] { return launch_hist(a, w.stream, 0, sms); }, level));
    IPLS_CUDA(timed(w, kkCheck, [&] { return launch_check(a, w.stream, sample_bound, sms); }, level));
    IPLS_CUDA(timed(w, kkRehist, [&] { return launch_hist(a, w.stream, 1, sms); }, level));
    IPLS_CUDA(timed(w, kkScan, [&] { return launch_scan(a, w.stream, sms); }, level));
    IPLS_CUDA(timed(w, kkTileScan, [&] { return launch_tilescan(a, w.stream, sms * 8); }, level));
    IPLS_CUDA(timed(w, kkScatter, [&] { return launch_scatter(a, w.stream, sms); }, level));
    IPLS_TRY(launch_tail_dev(w, ra, X, &w.ctl_arr[level + 1], rmax, sweep));
    IPLS_CUDA(timed(w, kkFill, [&] {
      return launch_fill(X.fills, a.fill_cap, dtype, w.stream, &w.ctl_arr[level + 1], sms * 8, w.run);
    }));
  }
  IPLS_CUDA(cudaMemcpyAsync(w.h_ctl_arr, w.ctl_arr, (size_t)(levels + 1) * sizeof(LevelCtl),
                            cudaMemcpyDeviceToHost, w.stream));
  IPLS_CUDA(cudaMemcpyAsync(w.h_run, w.run, sizeof(RunStatus), cudaMemcpyDeviceToHost, w.stream));
  IPLS_CUDA(cudaMemcpyAsync(w.h_trace_ctr, w.trace_ctr, sizeof(long long), cudaMemcpyDeviceToHost, w.stream));
  return IPLS_OK;
}

// Levels enqueued for n keys: none when every segment fits a block-resident
// task, else one per factor of about 2^8 above that size, plus one.
int device_levels_for(int64_t n, int rmax) {
  if (n <= rmax) return 0;
  int L = 1;
  for (int64_t m = n; m > rmax && L < kDevLevelsMax; m >>= 8) ++L;
  return L;
}

// The level loop.  Level-0 subproblems are either the whole array or the
// segments; each level runs fit -> hist -> check -> (re)hist -> scan ->
// scatter over all its grid subproblems, then the block-resident kernel over
// the groups the level produced.
iplsStatus sort_impl(Workspace& w, void* keys, int64_t n, int dtype, const int64_t* offsets,
                     int64_t nseg, const uint64_t* seg_ubase = nullptr) {
  iplsCtx c = w.c;
  const int wb = key_bytes(dtype);
  const iplsConfig& cfg = c->cfg;
  const bool traced = w.main && cfg.trace_cap > 0;
  const uint64_t ubase = reinterpret_cast<uint64_t>(keys);
  const int rmax = resident_rmax(cfg.cutoff);
  const int resident_root_ok = (cfg.root_sample <= 0 || cfg.root_sample <= kResidentSample);
  const int tile = tile_keys(dtype);
  w.stats.grid_levels = 0;
  w.stats.grid_passes = 0;
  w.stats.keys_partitioned = 0;
  w.stats.resident_groups = 0;
  w.stats.fallback_passes = 0;
  w.stats.sweep_tasks = 0;
  w.stats.algorithmic_bytes = 0;
  w.stats.max_bucket_frac = 0.0;
  w.trace_grid_count = 0;
  IPLS_TRY(ensure(w, w.scratch, w.scratch_cap, n * (int64_t)wb));
  IPLS_TRY(ensure(w, w.bids, w.bids_cap, n + 16));
  IPLS_TRY(ensure(w, w.slow, w.slow_cap, 2 * (n / (cfg.cutoff + 1)) + 4096));
  if (traced && c->trace_alloc < cfg.trace_cap) {
    IPLS_CUDA(cudaStreamSynchronize(w.stream));
    dev_free(c, c->trace_grid, (size_t)c->trace_alloc * sizeof(iplsTraceRecDev));
    dev_free(c, c->trace_res, (size_t)c->trace_alloc * sizeof(iplsTraceRecDev));
    c->trace_grid = c->trace_res = nullptr;
    c->trace_alloc = 0;
    void* p;
    IPLS_TRY(dev_alloc(c, &p, (size_t)cfg.trace_cap * sizeof(iplsTraceRecDev)));
    c->trace_grid = (iplsTraceRecDev*)p;
    IPLS_TRY(dev_alloc(c, &p, (size_t)cfg.trace_cap * sizeof(iplsTraceRecDev)));
    c->trace_res = (iplsTraceRecDev*)p;
    c->trace_alloc = cfg.trace_cap;
  }
  if (traced && cfg.pl2_leaves > 0 && !c->trace_knots) {
    const int64_t cap = std::min<int64_t>(cfg.trace_cap, kKnotTraceMax);
    void* p;
    IPLS_TRY(dev_alloc(c, &p, (size_t)cap * (cfg.pl2_leaves + 1) * sizeof(float)));
    c->trace_knots = (float*)p;
    c->knot_cap = cap;
    c->knot_leaves = cfg.pl2_leaves;
  }
  IPLS_CUDA(cudaMemsetAsync(w.run, 0, sizeof(RunStatus), w.stream));
  void* bufs[2] = {keys, w.scratch};

  ResidentArgs ra{};
  ra.dtype = dtype; ra.k = cfg.k; ra.cutoff = cfg.cutoff; ra.root_sample = cfg.root_sample;
  ra.seed = cfg.seed; ra.exact_only = cfg.exact_only; ra.buf[0] = bufs[0]; ra.buf[1] = bufs[1];
  ra.run = w.run; ra.trace = traced ? c->trace_res : nullptr; ra.trace_cap = traced ? cfg.trace_cap : 0;

  int64_t nsub = 0, ntiles = 0, nchunks = 0;
  int64_t max_sub_n = n;  // bound on the size of this level's grid subproblems
  const int64_t sub_bound = n / (rmax + 1) + 2;
  const int64_t tile_bound = n / tile + sub_bound + 2;
  const int64_t chunk_bound = tile_bound / kChunkTiles + sub_bound + 2;
  int start_level = 0;
  int64_t moved = 0;
  if (offsets && (cfg.flags & IPLS_FLAG_GRAPH)) {
    // device-driven levels, captured once into a CUDA graph per (buffers,
    // sizes) and replayed
    const int levels = device_levels_for(n, rmax);
    IPLS_TRY(device_prepare(w, n, nseg, dtype));
    const Workspace::GraphKey key{keys, offsets, seg_ubase, n, nseg, dtype, levels};
    if (!(w.graph && w.gkey == key)) {
      if (w.graph) {
        cudaGraphExecDestroy(w.graph);
        w.graph = nullptr;
      }
      if (!w.cap_stream) IPLS_CUDA(cudaStreamCreateWithFlags(&w.cap_stream, cudaStreamNonBlocking));
      IPLS_CUDA(cudaStreamSynchronize(w.stream));
      const cudaStream_t keep = w.stream;
      w.stream = w.cap_stream;
      w.capturing = true;
      cudaError_t e = cudaStreamBeginCapture(w.stream, cudaStreamCaptureModeRelaxed);
      iplsStatus st = IPLS_OK;
      if (e == cudaSuccess) st = device_enqueue(w, n, dtype, offsets, nseg, seg_ubase, ubase, levels);
      cudaGraph_t g = nullptr;
      const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(w.stream, &g) : e;
      w.stream = keep;
      w.capturing = false;
      if (st != IPLS_OK) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st;
      }
      if (e2 != cudaSuccess) return cuda_fail(e2, "capturing the segmented sort");
      e = cudaGraphInstantiate(&w.graph, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        w.graph = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
      }
      w.gkey = key;
    }
    IPLS_CUDA(cudaGraphLaunch(w.graph, w.stream));
    IPLS_CUDA(cudaStreamSynchronize(w.stream));
    const LevelCtl* H = w.h_ctl_arr;
    const int64_t sub_cap = std::min(w.slot[0].sub_cap, w.slot[1].sub_cap);
    auto nsub_at = [&](int L) { return std::min<int64_t>(H[L].nsub_next, sub_cap); };
    if (w.h_run->error_level > 0) {
      // the level whose scatter stopped keeps its keys where its records say:
      // those in the ping-pong buffer go back to the caller's memory
      const int L = w.h_run->error_level - 1;
      IPLS_CUDA(launch_restore(w.slot[L & 1].subs, (int32_t)nsub_at(L), dtype, w.scratch, w.stream));
      IPLS_CUDA(cudaStreamSynchronize(w.stream));
      if (w.h_run->error == IPLS_ERR_TIMEOUT)
        return fail(IPLS_ERR_TIMEOUT, "a device-side look-back wait exceeded spin_limit; the keys "
                                      "hold a permutation of the input");
      return fail((iplsStatus)w.h_run->error, "device reported status " + std::to_string(w.h_run->error));
    }
    for (int L = 0; L <= levels; ++L) {
      if (!H[L].overflow) continue;
      // level L-1 listed more than fits: nothing after its scatter ran
      if (L > 0) {
        IPLS_CUDA(launch_restore(w.slot[(L - 1) & 1].subs, (int32_t)nsub_at(L - 1), dtype, w.scratch, w.stream));
        IPLS_CUDA(cudaStreamSynchronize(w.stream));
      }
      return fail(IPLS_ERR_INTERNAL, "a level list capacity was exceeded");
    }
    for (int L = 0; L < levels; ++L) {
      const int64_t ns = nsub_at(L);
      if (ns == 0) break;
      w.stats.grid_levels += 1;
      w.stats.grid_passes += ns;
      w.stats.fallback_passes += H[L + 1].fallback;
      moved += H[L + 1].keys_moved;
      w.stats.max_bucket_frac = std::max(w.stats.max_bucket_frac, (double)H[L + 1].max_bucket / 1048576.0);
      if (w.main) {
        std::lock_guard<std::mutex> lk(c->prof_mu);
        c->k_bytes[kkHist] += (int64_t)wb * H[L + 1].keys_level;
        c->k_bytes[kkScatter] += 2 * (int64_t)wb * H[L + 1].keys_moved;
      }
    }
    if (traced) w.trace_grid_count = *w.h_trace_ctr;
    nsub = nsub_at(levels);
    ntiles = H[levels].tiles_next;
    nchunks = H[levels].chunks_next;
    max_sub_n = H[levels].max_sub_n;
    start_level = levels;
    // the host-driven levels that follow start from clean look-back words
    IPLS_CUDA(cudaMemsetAsync(w.status, 0, (size_t)w.status_cap * 8, w.stream));
    w.epoch = 1;
  } else if (offsets) {
    // segments: big ones become level-0 grid subproblems, the rest groups
    Slot& s0 = w.slot[0];
    Slot& s1 = w.slot[1];
    IPLS_TRY(ensure(w, s0.subs, s0.sub_cap, sub_bound));
    IPLS_TRY(ensure(w, s0.tile2sub, s0.tile_cap, tile_bound));
    IPLS_TRY(ensure(w, s0.chunk2sub, s0.chunk_cap, chunk_bound));
    const int64_t gcap = 2 * n / (cfg.cutoff + 1) + 2 * (nseg / 64) + 1024 + 2 * sub_bound;
    IPLS_TRY(ensure_groups(w, s1, std::min<int64_t>(gcap, nseg + 1024)));
    IPLS_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(LevelCtl), w.stream));
    IPLS_CUDA(timed(w, kkInitSeg, [&] {
      return launch_init_segments(offsets, nseg, seg_ubase, ubase, rmax, cfg.cutoff, resident_root_ok, w.ctl,
                                  s0.subs, (int32_t)std::min<int64_t>(s0.sub_cap, INT32_MAX),
                                  s0.tile2sub, s0.tile_cap, s0.chunk2sub, s0.chunk_cap, s1.groups,
                                  (int32_t)std::min<int64_t>(s1.group_cap, INT32_MAX),
                                  s1.fit_list, w.stream);
    }));
    IPLS_CUDA(cudaMemcpyAsync(w.h_ctl, w.ctl, sizeof(LevelCtl), cudaMemcpyDeviceToHost, w.stream));
    IPLS_CUDA(cudaStreamSynchronize(w.stream));
    if (w.h_ctl->overflow) return fail(IPLS_ERR_INTERNAL, "segment list capacity exceeded");
    resolve_events(w);
    if ((int64_t)w.h_ctl->ngroups + w.h_ctl->ngroups_large > s1.group_cap)
      return fail(IPLS_ERR_INTERNAL, "segment list capacity exceeded");
    IPLS_TRY(launch_tail(w, ra, s1, w.h_ctl->ngroups, w.h_ctl->ngroups_large, w.h_ctl->nfit));
    nsub = w.h_ctl->nsub_next;
    ntiles = w.h_ctl->tiles_next;
    nchunks = w.h_ctl->chunks_next;
    max_sub_n = w.h_ctl->max_sub_n;
  } else if (n <= rmax && resident_root_ok) {
    // the whole array fits one block: one launch runs the whole recursion in
    // shared memory (the same sample, models and passes as the tail kernels)
    const SlowTask t{0, (int32_t)n, 0, ubase};
    IPLS_CUDA(timed(w, kkSlow, [&] { return launch_slow_one(ra, t, w.stream); }));
    IPLS_TRY(check_run(w));
    resolve_events(w);
    if (w.main) {
      std::lock_guard<std::mutex> lk(c->prof_mu);
      c->k_bytes[kkResident] += 2 * (int64_t)wb * n;
    }
    w.stats.algorithmic_bytes = 2 * (int64_t)wb * n;
    return IPLS_OK;
  } else {
    Slot& s0 = w.slot[0];
    IPLS_TRY(ensure(w, s0.subs, s0.sub_cap, 1));
    ntiles = (n + tile - 1) / tile;
    nchunks = (ntiles + kChunkTiles - 1) / kChunkTiles;
    IPLS_TRY(ensure(w, s0.tile2sub, s0.tile_cap, ntiles));
    IPLS_TRY(ensure(w, s0.chunk2sub, s0.chunk_cap, nchunks));
    const Sub root{0, n, 0, 0, 0, (int32_t)ntiles, 0, 0, (int32_t)nchunks, ubase};
    IPLS_CUDA(cudaMemcpyAsync(s0.subs, &root, sizeof(root), cudaMemcpyHostToDevice, w.stream));
    IPLS_CUDA(timed(w, kkInitTiles, [&] { return launch_init_tiles(s0.tile2sub, ntiles, 0, w.stream); }));
    IPLS_CUDA(timed(w, kkInitTiles, [&] { return launch_init_tiles(s0.chunk2sub, nchunks, 0, w.stream); }));
    nsub = 1;
  }

  int level = start_level;
  while (nsub > 0) {
    if (level > 4096) return fail(IPLS_ERR_INTERNAL, "recursion depth limit exceeded");
    Slot& X = w.slot[level & 1];
    Slot& Y = w.slot[(level + 1) & 1];
    IPLS_TRY(ensure(w, X.models, X.model_cap, nsub));
    IPLS_TRY(ensure(w, X.tabs, X.tab_cap, nsub));
    if (cfg.pl2_leaves > 0) IPLS_TRY(ensure(w, X.knots, X.knot_cap, nsub * (int64_t)(cfg.pl2_leaves + 1)));
    IPLS_TRY(ensure(w, X.counts, X.count_cap, nsub * kMaxK));
    IPLS_TRY(ensure(w, X.bases, X.base_cap, nsub * 257));
    IPLS_TRY(ensure_groups(w, X, 2 * n / (cfg.cutoff + 1) + 257 * nsub + 16));
    IPLS_TRY(ensure(w, X.fills, X.fill_cap, n / kFillChunk + 129 * nsub + 16));
    IPLS_TRY(ensure(w, Y.subs, Y.sub_cap, sub_bound));
    IPLS_TRY(ensure(w, Y.tile2sub, Y.tile_cap, tile_bound));
    IPLS_TRY(ensure(w, Y.chunk2sub, Y.chunk_cap, chunk_bound));
    IPLS_TRY(ensure(w, w.tile_off, w.tile_off_cap, ntiles * kMaxK));
    if (w.status_cap < nchunks * kMaxK) {
      IPLS_TRY(ensure(w, w.status, w.status_cap, nchunks * kMaxK));
      IPLS_CUDA(cudaMemsetAsync(w.status, 0, (size_t)w.status_cap * 8, w.stream));
      w.epoch = 0;
    }
    if (++w.epoch >= 0x10000) {
      IPLS_CUDA(cudaMemsetAsync(w.status, 0, (size_t)w.status_cap * 8, w.stream));
      w.epoch = 1;
    }
    IPLS_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(LevelCtl), w.stream));
    LevelArgs a{};
    a.dtype = dtype; a.k = cfg.k; a.cutoff = cfg.cutoff; a.rmax = rmax;
    a.root_sample = cfg.root_sample; a.seed = cfg.seed; a.exact_only = cfg.exact_only;
    a.use_tables = (cfg.flags & IPLS_FLAG_THRESHOLD_INDEX) && !cfg.exact_only;
    a.spin_limit = cfg.spin_limit; a.epoch = w.epoch; a.level = level;
    a.buf[0] = bufs[0]; a.buf[1] = bufs[1];
    a.nsub = (int32_t)nsub; a.subs = X.subs; a.models = X.models; a.counts = X.counts;
    a.tabs = X.tabs;
    a.bases = X.bases; a.tile2sub = X.tile2sub; a.ntiles = ntiles; a.status = w.status;
    a.chunk2sub = X.chunk2sub; a.nchunks = nchunks; a.tile_off = w.tile_off;
    a.bids = w.bids;
    a.ctl = w.ctl; a.run = w.run;
    a.next_subs = Y.subs; a.next_sub_cap = (int32_t)std::min<int64_t>(Y.sub_cap, INT32_MAX);
    a.next_tile2sub = Y.tile2sub; a.next_tile_cap = Y.tile_cap;
    a.next_chunk2sub = Y.chunk2sub; a.next_chunk_cap = Y.chunk_cap;
    a.groups = X.groups; a.group_cap = (int32_t)std::min<int64_t>(X.group_cap, INT32_MAX);
    a.fit_list = X.fit_list;
    a.fills = X.fills; a.fill_cap = (int32_t)std::min<int64_t>(X.fill_cap, INT32_MAX);
    a.trace = traced ? c->trace_grid : nullptr;
    a.trace_cap = traced ? cfg.trace_cap : 0;
    a.trace_base = w.trace_grid_count;
    a.trace_knots = traced ? c->trace_knots : nullptr;
    a.knot_cap = c->knot_cap;
    const int max_sample = sample_size_host(std::max<int64_t>(max_sub_n, 2), level, cfg.k, cfg.root_sample);
    a.max_sample = max_sample;
    a.pl2_leaves = cfg.pl2_leaves;
    a.pl2_depth = cfg.pl2_depth;
    a.knots = cfg.pl2_leaves > 0 ? X.knots : nullptr;
    IPLS_CUDA(timed(w, kkFit, [&] { return launch_fit(a, w.stream, max_sample, c->num_sms); }, level));
    IPLS_CUDA(timed(w, kkHist, [&] { return launch_hist(a, w.stream, 0, occupancy_grid(c, 0, dtype)); }, level));
    IPLS_CUDA(timed(w, kkCheck, [&] { return launch_check(a, w.stream, max_sample, c->num_sms); }, level));
    IPLS_CUDA(timed(w, kkRehist, [&] { return launch_hist(a, w.stream, 1, occupancy_grid(c, 0, dtype)); }, level));
    IPLS_CUDA(timed(w, kkScan, [&] { return launch_scan(a, w.stream, c->num_sms); }, level));
    IPLS_CUDA(timed(w, kkTileScan, [&] { return launch_tilescan(a, w.stream, c->num_sms * 8); }, level));
    IPLS_CUDA(timed(w, kkScatter, [&] { return launch_scatter(a, w.stream, occupancy_grid(c, 1, dtype)); }, level));
    IPLS_CUDA(cudaMemcpyAsync(w.h_ctl, w.ctl, sizeof(LevelCtl), cudaMemcpyDeviceToHost, w.stream));
    IPLS_CUDA(cudaMemcpyAsync(w.h_run, w.run, sizeof(RunStatus), cudaMemcpyDeviceToHost, w.stream));
    IPLS_CUDA(cudaStreamSynchronize(w.stream));
    const LevelCtl lc = *w.h_ctl;
    if (w.h_run->error != 0 || lc.overflow || (int64_t)lc.ngroups + lc.ngroups_large > X.group_cap) {
      // nothing of this level moved (k_scatter checks the status first):
      // put the level's keys back into the user buffer and stop
      IPLS_CUDA(launch_restore(X.subs, (int32_t)nsub, dtype, w.scratch, w.stream));
      IPLS_CUDA(cudaStreamSynchronize(w.stream));
      resolve_events(w);
      if (w.h_run->error == IPLS_ERR_TIMEOUT)
        return fail(IPLS_ERR_TIMEOUT, "a device-side look-back wait exceeded spin_limit; the keys "
                                      "hold a permutation of the input");
      if (w.h_run->error != 0)
        return fail((iplsStatus)w.h_run->error, "device reported status " + std::to_string(w.h_run->error));
      return fail(IPLS_ERR_INTERNAL, "a level list capacity was exceeded");
    }
    resolve_events(w);
    if (w.main) {
      std::lock_guard<std::mutex> lk(c->prof_mu);
      c->k_bytes[kkHist] += (int64_t)wb * lc.keys_level;
      c->k_bytes[kkScatter] += 2 * (int64_t)wb * lc.keys_moved;
      if (level < iplsContext::kLevels) {
        c->lv_keys[level] += lc.keys_moved;
        c->lv_bytes[level] += 2 * (int64_t)wb * lc.keys_moved;
      }
    }
    w.stats.grid_levels += 1;
    w.stats.grid_passes += nsub;
    w.stats.fallback_passes += lc.fallback;
    moved += lc.keys_moved;
    w.stats.max_bucket_frac = std::max(w.stats.max_bucket_frac, (double)lc.max_bucket / 1048576.0);
    w.trace_grid_count += nsub;
    IPLS_TRY(launch_tail(w, ra, X, lc.ngroups, lc.ngroups_large, lc.nfit));
    if (lc.nfill > 0)
      IPLS_CUDA(timed(w, kkFill, [&] { return launch_fill(X.fills, lc.nfill, dtype, w.stream); }));
    nsub = lc.nsub_next;
    ntiles = lc.tiles_next;
    nchunks = lc.chunks_next;
    max_sub_n = lc.max_sub_n;
    ++level;
  }
  IPLS_TRY(check_run(w));
  resolve_events(w);
  if (w.main) {
    std::lock_guard<std::mutex> lk(c->prof_mu);
    c->k_bytes[kkResident] += 2 * (int64_t)wb * w.h_run->resident_keys;
  }
  w.stats.keys_partitioned = moved;
  w.stats.algorithmic_bytes = 2 * (int64_t)wb * (moved + w.h_run->resident_keys);
  return IPLS_OK;
}

iplsStatus check_common(int64_t n, int dtype) {
  if (!valid_dtype(dtype)) return fail(IPLS_ERR_ARG, "unknown dtype");
  if (n < 0 || n > kMaxKeys) return fail(IPLS_ERR_ARG, "n out of range [0, 2^32 - 1]");
  return IPLS_OK;
}

// Device keys must be aligned to the key width.
iplsStatus check_keys_ptr(const void* keys, int dtype) {
  if (reinterpret_cast<uintptr_t>(keys) % (uintptr_t)key_bytes(dtype) != 0)
    return fail(IPLS_ERR_ARG, "keys must be aligned to the key width");
  return IPLS_OK;
}

iplsStatus validate_cfg(const iplsConfig& c) {
  if (c.k < 3 || c.k > 256) return fail(IPLS_ERR_ARG, "k must be in [3, 256]");
  if (c.cutoff < 1 || c.cutoff > kResidentMax) return fail(IPLS_ERR_ARG, "cutoff must be in [1, 8192]");
  if (c.root_sample < 0 || c.root_sample > 16384)
    return fail(IPLS_ERR_ARG, "root_sample must be in [0, 16384]");
  if (c.spin_limit < 1) return fail(IPLS_ERR_ARG, "spin_limit must be >= 1");
  if (c.max_batch < 0) return fail(IPLS_ERR_ARG, "max_batch must be >= 0");
  if (c.pl2_leaves != 0 && (c.pl2_leaves < 2 || c.pl2_leaves > kPL2MaxLeaves || (c.pl2_leaves & (c.pl2_leaves - 1))))
    return fail(IPLS_ERR_ARG, "pl2_leaves must be 0 or a power of two in [2, 1024]");
  if (c.budget_bytes < 0) return fail(IPLS_ERR_ARG, "budget_bytes must be >= 0");
  if (c.serve_slots < 0 || c.serve_slots > 2) return fail(IPLS_ERR_ARG, "serve_slots must be 0, 1 or 2");
  if (c.pl2_depth < 0) return fail(IPLS_ERR_ARG, "pl2_depth must be >= 0");
  return IPLS_OK;
}



}  // namespace

namespace ipls {
void set_last_error(const char* msg) { g_last_error = msg; }
}  // namespace ipls

// ---------------------------------------------------------------------------
// Segment lists for iplsSortSegmented: windows of 64 consecutive segments,
// each packed greedily by one thread (same rule as k_scan's bucket packing).
// ---------------------------------------------------------------------------
namespace ipls {

constexpr int kSegWindow = 64;

__global__ void k_init_segments(const int64_t* off, int64_t nseg, const uint64_t* seg_ubase, uint64_t ubase,
                                int rmax, int cutoff,
                                int resident_ok, LevelCtl* ctl, Sub* subs, int32_t sub_cap,
                                int32_t* tile2sub, int64_t tile_cap, int32_t* chunk2sub,
                                int64_t chunk_cap, Group* groups, int32_t group_cap,
                                int32_t* fit_list) {
  const int64_t wnd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t q0 = wnd * kSegWindow;
  if (q0 >= nseg) return;
  const int64_t q1 = q0 + kSegWindow < nseg ? q0 + kSegWindow : nseg;
  int64_t g0 = -1, glast = -1, tot = 0;
  uint64_t gbase = 0;
  for (int64_t q = q0; q <= q1; ++q) {
    const int64_t cq = (q < q1) ? off[q + 1] - off[q] : 0;
    const uint64_t ub = (seg_ubase && q < q1) ? seg_ubase[q] : ubase;
    const bool big = cq > cutoff && (cq > rmax || !resident_ok);
    const bool mid = cq > cutoff && !big;
    const bool brk = (q == q1) || big || mid;
    const bool fits = (cq > 0) && !brk;
    // segments share a task only when they lie one after another in one array
    if (g0 >= 0 && (brk || (fits && (tot + cq > rmax || ub != gbase)))) {
      const int g = group_slot(ctl, tot, group_cap);
      if (g < 0) ctl->overflow = 1;
      else groups[g] = Group{off[g0], off + g0, (int32_t)tot, 0, 0, (int32_t)(glast - g0 + 1), -1, 0, gbase};
      g0 = -1;
      tot = 0;
    }
    if (mid) {
      const int g = group_slot(ctl, cq, group_cap);
      if (g < 0) {
        ctl->overflow = 1;
      } else {
        groups[g] = Group{off[q], nullptr, (int32_t)cq, 0, 0, 1, g, 0, ub};
        const int f = atomicAdd(&ctl->nfit, 1);
        if (f < group_cap) fit_list[f] = g;
        else ctl->overflow = 1;
      }
    }
    if (big) {
      const int i = atomicAdd(&ctl->nsub_next, 1);
      if (i >= sub_cap) {
        ctl->overflow = 1;
      } else {
        Sub ns{off[q], cq, 0, 0, 0, 0, 0, 0, 0, ub};
        if (reserve_tiles(ctl, i, ns, tile2sub, tile_cap, chunk2sub, chunk_cap)) subs[i] = ns;
      }
    }
    if (fits) {
      if (g0 < 0) { g0 = q; gbase = ub; }
      tot += cq;
      glast = q;
    }
  }
}

cudaError_t launch_init_segments(const int64_t* offsets, int64_t nseg, const uint64_t* seg_ubase,
                                 uint64_t ubase, int rmax, int cutoff,
                                 int resident_ok, LevelCtl* ctl, Sub* subs, int32_t sub_cap,
                                 int32_t* tile2sub, int64_t tile_cap, int32_t* chunk2sub,
                                 int64_t chunk_cap, Group* groups, int32_t group_cap,
                                 int32_t* fit_list, cudaStream_t s) {
  const int64_t windows = (nseg + kSegWindow - 1) / kSegWindow;
  if (windows <= 0) return cudaSuccess;
  const int threads = 128;
  const int64_t blocks = (windows + threads - 1) / threads;
  k_init_segments<<<(unsigned)blocks, threads, 0, s>>>(offsets, nseg, seg_ubase, ubase, rmax, cutoff, resident_ok,
                                                       ctl, subs, sub_cap, tile2sub, tile_cap,
                                                       chunk2sub, chunk_cap, groups, group_cap,
                                                       fit_list);
  return cudaGetLastError();
}

}  // namespace ipls

// ---------------------------------------------------------------------------
// Workspaces.
// ---------------------------------------------------------------------------
namespace {

iplsStatus ws_init(iplsCtx c, Workspace& w, cudaStream_t stream, bool own_stream, bool main) {
  w.c = c;
  w.stream = stream;
  w.own_stream = own_stream;
  w.main = main;
  cudaError_t e = cudaMallocHost(&w.h_ctl, sizeof(LevelCtl));
  if (e == cudaSuccess) e = cudaMallocHost(&w.h_run, sizeof(RunStatus));
  if (e == cudaSuccess) e = cudaMallocHost(&w.h_slow, sizeof(SlowCtl));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "cudaMallocHost");
  }
  void* p;
  IPLS_TRY(dev_alloc(c, &p, sizeof(LevelCtl)));
  w.ctl = (LevelCtl*)p;
  IPLS_TRY(dev_alloc(c, &p, sizeof(RunStatus)));
  w.run = (RunStatus*)p;
  IPLS_TRY(dev_alloc(c, &p, 2 * sizeof(int64_t)));
  w.root_bounds = (int64_t*)p;
  IPLS_TRY(dev_alloc(c, &p, sizeof(SlowCtl)));
  w.slow_ctl = (SlowCtl*)p;
  return IPLS_OK;
}

// Releases everything a workspace holds (waits for its stream first).
void ws_free(Workspace& w) {
  iplsCtx c = w.c;
  if (!c) return;
  if (w.stream || !w.own_stream) cudaStreamSynchronize(w.stream);
  dev_free(c, w.scratch, (size_t)w.scratch_cap);
  dev_free(c, w.status, (size_t)w.status_cap * 8);
  dev_free(c, w.tile_off, (size_t)w.tile_off_cap * 4);
  dev_free(c, w.bids, (size_t)w.bids_cap);
  for (Slot& s : w.slot) {
    dev_free(c, s.subs, s.sub_cap * sizeof(Sub));
    dev_free(c, s.tile2sub, s.tile_cap * sizeof(int32_t));
    dev_free(c, s.chunk2sub, s.chunk_cap * sizeof(int32_t));
    dev_free(c, s.models, s.model_cap * sizeof(Model));
    dev_free(c, s.tabs, s.tab_cap * sizeof(ThrTable));
    dev_free(c, s.knots, s.knot_cap * sizeof(float));
    dev_free(c, s.counts, s.count_cap * sizeof(uint64_t));
    dev_free(c, s.bases, s.base_cap * sizeof(int64_t));
    dev_free(c, s.groups, s.group_cap * sizeof(Group));
    dev_free(c, s.fit_list, s.fit_cap * sizeof(int32_t));
    dev_free(c, s.tails, s.tail_cap * sizeof(TailModel));
    dev_free(c, s.fills, s.fill_cap * sizeof(Fill));
    s = Slot{};
  }
  dev_free(c, w.ctl, sizeof(LevelCtl));
  dev_free(c, w.run, sizeof(RunStatus));
  dev_free(c, w.root_bounds, 2 * sizeof(int64_t));
  dev_free(c, w.slow, (size_t)w.slow_cap * sizeof(SlowTask));
  dev_free(c, w.slow_ctl, sizeof(SlowCtl));
  dev_free(c, w.split_pool, (size_t)w.split_pool_cap * 8);
  dev_free(c, w.seg_off, (size_t)w.seg_off_cap * 8);
  dev_free(c, w.seg_ubase, (size_t)w.seg_ubase_cap * 8);
  if (w.h_ctl) cudaFreeHost(w.h_ctl);
  if (w.h_run) cudaFreeHost(w.h_run);
  if (w.h_slow) cudaFreeHost(w.h_slow);
  if (w.h_seg_off) cudaFreeHost(w.h_seg_off);
  if (w.h_seg_ubase) cudaFreeHost(w.h_seg_ubase);
  dev_free(c, w.ctl_arr, (kDevLevelsMax + 1) * sizeof(LevelCtl));
  dev_free(c, w.trace_ctr, sizeof(long long));
  if (w.h_ctl_arr) cudaFreeHost(w.h_ctl_arr);
  if (w.h_trace_ctr) cudaFreeHost(w.h_trace_ctr);
  if (w.graph) cudaGraphExecDestroy(w.graph);
  if (w.cap_stream) cudaStreamDestroy(w.cap_stream);
  for (auto& p : w.pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (cudaEvent_t e : w.spare_events) cudaEventDestroy(e);
  if (w.own_stream && w.stream) cudaStreamDestroy(w.stream);
  w = Workspace{};
}

// Sorts `count` separate device arrays, keys[i][0..n[i]), each in place and
// each a level-0 subproblem of its own: one segmented sort over an index
// space in which array i occupies [off_i, off_i + n[i]), with its own base
// (keys[i] - off_i), so nothing is gathered or copied back.
iplsStatus sort_arrays(Workspace& w, void* const* keys, const int64_t* n, int64_t count, int dtype) {
  if (count == 1) return sort_impl(w, keys[0], n[0], dtype, nullptr, 0);
  const int64_t wb = key_bytes(dtype);
  if (w.h_seg_cap < count + 1) {
    if (w.h_seg_off) cudaFreeHost(w.h_seg_off);
    if (w.h_seg_ubase) cudaFreeHost(w.h_seg_ubase);
    w.h_seg_off = nullptr;
    w.h_seg_ubase = nullptr;
    w.h_seg_cap = 0;
    const int64_t cap = 2 * count + 16;
    IPLS_CUDA(cudaMallocHost(&w.h_seg_off, (size_t)cap * 8));
    IPLS_CUDA(cudaMallocHost(&w.h_seg_ubase, (size_t)cap * 8));
    w.h_seg_cap = cap;
  }
  IPLS_TRY(ensure(w, w.seg_off, w.seg_off_cap, count + 1));
  IPLS_TRY(ensure(w, w.seg_ubase, w.seg_ubase_cap, count));
  // the previous batch's copies read these host arrays: wait for them
  IPLS_CUDA(cudaStreamSynchronize(w.stream));
  int64_t total = 0;
  for (int64_t i = 0; i < count; ++i) {
    w.h_seg_off[i] = total;
    w.h_seg_ubase[i] = reinterpret_cast<uint64_t>(keys[i]) - (uint64_t)(total * wb);
    total += n[i];
  }
  w.h_seg_off[count] = total;
  if (total > kMaxKeys) return fail(IPLS_ERR_ARG, "a batch holds at most 2^32 - 1 keys");
  IPLS_CUDA(cudaMemcpyAsync(w.seg_off, w.h_seg_off, (size_t)(count + 1) * 8, cudaMemcpyHostToDevice, w.stream));
  IPLS_CUDA(cudaMemcpyAsync(w.seg_ubase, w.h_seg_ubase, (size_t)count * 8, cudaMemcpyHostToDevice, w.stream));
  return sort_impl(w, nullptr, total, dtype, w.seg_off, count, w.seg_ubase);
}

}  // namespace

// ---------------------------------------------------------------------------
// Request serving (iplsSubmit): kServeSlots worker threads per context, each
// with its own workspace and stream.  A worker that is free takes the oldest
// queued request's dtype and, in arrival order, the queued requests of that
// dtype while the bytes of all admitted requests (2*w*n each) stay within
// cfg.budget_bytes and the batch within cfg.max_batch, and sorts them with
// one batched sort (each request a segment in its own memory).  While one
// batch runs the other worker admits the next, so batches of different sizes
// and dtypes overlap on the device, and memory freed by a finished batch
// lets waiting requests in.
// ---------------------------------------------------------------------------
namespace {

void serve_loop(iplsCtx c, int slot) {
  cudaSetDevice(c->device);
  Workspace& w = c->serve_ws[slot];
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  std::vector<uint64_t> batch;
  std::vector<void*> ptrs;
  std::vector<int64_t> sizes;
  for (;;) {
    batch.clear();
    ptrs.clear();
    sizes.clear();
    int dtype = 0;
    int64_t bytes = 0;
    {
      std::unique_lock<std::mutex> lk(c->q_mu);
      const int64_t budget = c->cfg.budget_bytes;
      auto need_of = [&](uint64_t t) {
        const iplsContext::Request& r = c->reqs[t];
        return 2 * r.n * (int64_t)key_bytes(r.dtype);
      };
      c->q_cv.wait(lk, [&] {
        if (c->queue.empty()) return c->stop;
        return budget <= 0 || c->inflight_bytes + need_of(c->queue.front()) <= budget ||
               c->inflight_bytes == 0;
      });
      if (c->queue.empty()) break;  // stop requested and nothing pending
      dtype = c->reqs[c->queue.front()].dtype;
      const int max_batch = c->cfg.max_batch;
      for (auto it = c->queue.begin(); it != c->queue.end();) {
        const iplsContext::Request& r = c->reqs[*it];
        if (r.dtype != dtype) { ++it; continue; }
        const int64_t need = need_of(*it);
        if (!batch.empty() && budget > 0 && c->inflight_bytes + bytes + need > budget) break;
        if (max_batch > 0 && (int)batch.size() >= max_batch) break;
        batch.push_back(*it);
        ptrs.push_back(r.keys);
        sizes.push_back(r.n);
        bytes += need;
        it = c->queue.erase(it);
      }
      c->inflight_bytes += bytes;
    }
    if (ev0) cudaEventRecord(ev0, w.stream);
    iplsStatus st = sort_arrays(w, ptrs.data(), sizes.data(), (int64_t)batch.size(), dtype);
    if (ev1) cudaEventRecord(ev1, w.stream);
    if (cudaStreamSynchronize(w.stream) != cudaSuccess && st == IPLS_OK) {
      cudaGetLastError();
      st = IPLS_ERR_CUDA;
    }
    iplsBatchRec rec{};
    rec.first_ticket = batch.front();
    rec.requests = (int32_t)batch.size();
    rec.slot = slot;
    rec.dtype = dtype;
    rec.status = (int32_t)st;
    for (int64_t x : sizes) rec.keys += x;
    float t0 = 0.f, t1 = 0.f;
    if (ev0 && ev1 && c->serve_ref && cudaEventElapsedTime(&t0, c->serve_ref, ev0) == cudaSuccess &&
        cudaEventElapsedTime(&t1, c->serve_ref, ev1) == cudaSuccess) {
      rec.start_ms = t0;
      rec.end_ms = t1;
    } else {
      cudaGetLastError();
      rec.start_ms = rec.end_ms = -1.0;
    }
    {
      std::lock_guard<std::mutex> lk(c->q_mu);
      for (uint64_t t : batch) {
        c->reqs[t].st = st;
        c->reqs[t].done = true;
        if (st != IPLS_OK) c->reqs[t].msg = g_last_error;
      }
      c->inflight_bytes -= bytes;
      if (c->batch_log.size() < 65536) c->batch_log.push_back(rec);
    }
    c->done_cv.notify_all();
    c->q_cv.notify_all();  // memory was freed: a waiting worker may admit more
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
}

// Starts the workers (first iplsSubmit; q_mu held).
iplsStatus start_workers(iplsCtx c) {
  if (c->workers[0].joinable()) return IPLS_OK;
  const int slots = c->cfg.serve_slots > 0 ? c->cfg.serve_slots : iplsContext::kServeSlots;
  for (int i = 0; i < slots; ++i) {
    cudaStream_t s = nullptr;
    IPLS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    IPLS_TRY(ws_init(c, c->serve_ws[i], s, true, false));
  }
  if (!c->serve_ref) {
    IPLS_CUDA(cudaEventCreate(&c->serve_ref));
    IPLS_CUDA(cudaEventRecord(c->serve_ref, c->serve_ws[0].stream));
    IPLS_CUDA(cudaEventSynchronize(c->serve_ref));
  }
  for (int i = 0; i < slots; ++i) c->workers[i] = std::thread(serve_loop, c, i);
  return IPLS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

iplsStatus iplsDefaultConfig(iplsConfig* cfg) {
  if (!cfg) return fail(IPLS_ERR_ARG, "cfg is NULL");
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->k = 256;
  cfg->cutoff = 32;
  cfg->root_sample = 0;
  cfg->seed = 0;
  cfg->sync = 1;
  cfg->exact_only = 0;
  cfg->spin_limit = int64_t(1) << 26;
  cfg->trace_cap = 0;
  cfg->budget_bytes = 0;
  cfg->pl2_depth = 1;
  return IPLS_OK;
}

iplsStatus iplsCreate(iplsCtx* out, const iplsConfig* cfg, iplsAllocFn alloc, iplsFreeFn free_fn,
                      void* user, void* stream) {
  if (!out) return fail(IPLS_ERR_ARG, "ctx is NULL");
  *out = nullptr;
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(IPLS_ERR_ARG, "alloc and free must both be given or both be NULL");
  iplsContext* c = new iplsContext();
  if (cfg) c->cfg = *cfg; else iplsDefaultConfig(&c->cfg);
  iplsStatus st = validate_cfg(c->cfg);
  if (st != IPLS_OK) { delete c; return st; }
  c->alloc = alloc;
  c->free_fn = free_fn;
  c->user = user;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return cuda_fail(e, "iplsCreate");
  }
  if ((st = ws_init(c, c->ws, reinterpret_cast<cudaStream_t>(stream), false, true)) != IPLS_OK) {
    iplsDestroy(c);
    return st;
  }
  *out = c;
  return IPLS_OK;
}

iplsStatus iplsDestroy(iplsCtx c) {
  if (!c) return fail(IPLS_ERR_ARG, "ctx is NULL");
  {
    std::lock_guard<std::mutex> lk(c->q_mu);
    c->stop = true;
  }
  c->q_cv.notify_all();
  for (std::thread& t : c->workers)
    if (t.joinable()) t.join();
  for (Workspace& w : c->serve_ws) ws_free(w);
  ws_free(c->ws);
  if (c->serve_ref) cudaEventDestroy(c->serve_ref);
  dev_free(c, c->trace_grid, (size_t)c->trace_alloc * sizeof(iplsTraceRecDev));
  dev_free(c, c->trace_res, (size_t)c->trace_alloc * sizeof(iplsTraceRecDev));
  dev_free(c, c->trace_knots, (size_t)c->knot_cap * (c->knot_leaves + 1) * sizeof(float));
  dev_free(c, c->host_stage, (size_t)c->host_stage_cap);
  for (int k = 0; k < 3; ++k) {
    dev_free(c, c->pipe_buf[k], (size_t)c->pipe_cap[k]);
    if (c->in_ev[k]) cudaEventDestroy(c->in_ev[k]);
    if (c->sorted_ev[k]) cudaEventDestroy(c->sorted_ev[k]);
    if (c->out_ev[k]) cudaEventDestroy(c->out_ev[k]);
  }
  if (c->h2d) cudaStreamDestroy(c->h2d);
  if (c->d2h) cudaStreamDestroy(c->d2h);
  delete c;
  return IPLS_OK;
}

iplsStatus iplsScratchBytes(iplsCtx c, int64_t n, iplsDtype dtype, size_t* bytes) {
  if (!bytes) return fail(IPLS_ERR_ARG, "bytes is NULL");
  IPLS_TRY(check_common(n, dtype));
  const int cutoff = c ? c->cfg.cutoff : 32;
  const int rmax = resident_rmax(cutoff);
  const int64_t subs = n / (rmax + 1) + 2;
  const int64_t tiles = n / tile_keys(dtype) + subs + 2;
  size_t b = (size_t)n * key_bytes(dtype);                         // ping-pong keys
  b += (size_t)n;                                                  // bucket ids
  b += (size_t)pool_slots(n / (cutoff + 1)) * 128 * 8;             // splitter pool
  b += (size_t)tiles * kMaxK * 8;                                  // look-back words
  b += 2 * (size_t)subs * (sizeof(Sub) + sizeof(Model) + kMaxK * 8 + 257 * 8);
  if (c && c->cfg.pl2_leaves > 0) b += 2 * (size_t)subs * (c->cfg.pl2_leaves + 1) * sizeof(float);
  b += 2 * (size_t)tiles * 4;
  b += 2 * (size_t)(2 * n / rmax + 257 * subs + 16) * (sizeof(Group) + 4 + sizeof(TailModel));
  b += 2 * (size_t)(n / kFillChunk + 129 * subs + 16) * sizeof(Fill);
  *bytes = b + b / 4 + 4096;
  return IPLS_OK;
}

static iplsCtx default_ctx(iplsStatus* st) {
  static thread_local std::map<int, iplsCtx> ctxs;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    *st = fail(IPLS_ERR_CUDA, "no current CUDA device");
    return nullptr;
  }
  auto it = ctxs.find(dev);
  if (it != ctxs.end()) { *st = IPLS_OK; return it->second; }
  iplsCtx c = nullptr;
  *st = iplsCreate(&c, nullptr, nullptr, nullptr, nullptr, nullptr);
  if (*st != IPLS_OK) return nullptr;
  ctxs[dev] = c;
  return c;
}

iplsStatus iplsSort(iplsCtx c, void* keys, int64_t n, iplsDtype dtype) {
  IPLS_TRY(check_common(n, dtype));
  if (n > 1 && !keys) return fail(IPLS_ERR_ARG, "keys is NULL");
  IPLS_TRY(check_keys_ptr(keys, dtype));
  iplsStatus st = IPLS_OK;
  if (!c) { c = default_ctx(&st); if (!c) return st; }
  std::lock_guard<std::mutex> ex(c->exec_mu);
  c->calls += 1;
  if (n <= 1) return IPLS_OK;
  g_last_error.clear();
  return sort_impl(c->ws, keys, n, dtype, nullptr, 0);
}

iplsStatus iplsSortSegmented(iplsCtx c, void* keys, const int64_t* offsets, int64_t nseg,
                             iplsDtype dtype) {
  if (!valid_dtype(dtype)) return fail(IPLS_ERR_ARG, "unknown dtype");
  if (nseg < 0) return fail(IPLS_ERR_ARG, "nseg < 0");
  if (nseg == 0) return IPLS_OK;
  if (!offsets || !keys) return fail(IPLS_ERR_ARG, "keys or offsets is NULL");
  IPLS_TRY(check_keys_ptr(keys, dtype));
  if (reinterpret_cast<uintptr_t>(offsets) % 8 != 0) return fail(IPLS_ERR_ARG, "offsets must be 8-byte aligned");
  iplsStatus st = IPLS_OK;
  if (!c) { c = default_ctx(&st); if (!c) return st; }
  std::lock_guard<std::mutex> ex(c->exec_mu);
  // validate the offsets on the host (non-decreasing ends, within 2^32 - 1)
  int64_t first = 0, last = 0;
  IPLS_CUDA(cudaMemcpyAsync(&first, offsets, 8, cudaMemcpyDeviceToHost, c->ws.stream));
  IPLS_CUDA(cudaMemcpyAsync(&last, offsets + nseg, 8, cudaMemcpyDeviceToHost, c->ws.stream));
  IPLS_CUDA(cudaStreamSynchronize(c->ws.stream));
  if (first < 0 || last < first || last > kMaxKeys)
    return fail(IPLS_ERR_ARG, "offsets out of range");
  c->calls += 1;
  g_last_error.clear();
  return sort_impl(c->ws, keys, last, dtype, offsets, nseg);
}

iplsStatus iplsSortBatch(iplsCtx c, void* const* keys, const int64_t* n, int64_t count, iplsDtype dtype) {
  if (!valid_dtype(dtype)) return fail(IPLS_ERR_ARG, "unknown dtype");
  if (count < 0) return fail(IPLS_ERR_ARG, "count < 0");
  if (count == 0) return IPLS_OK;
  if (!keys || !n) return fail(IPLS_ERR_ARG, "keys or n is NULL");
  int64_t total = 0;
  std::vector<void*> ptrs;
  std::vector<int64_t> sizes;
  for (int64_t i = 0; i < count; ++i) {
    if (n[i] < 0) return fail(IPLS_ERR_ARG, "a size is negative");
    if (n[i] > 1 && !keys[i]) return fail(IPLS_ERR_ARG, "a keys pointer is NULL");
    if (n[i] > 1) IPLS_TRY(check_keys_ptr(keys[i], dtype));
    total += n[i];
    if (total > kMaxKeys) return fail(IPLS_ERR_ARG, "a batch holds at most 2^32 - 1 keys");
    if (n[i] > 1) { ptrs.push_back(keys[i]); sizes.push_back(n[i]); }
  }
  iplsStatus st = IPLS_OK;
  if (!c) { c = default_ctx(&st); if (!c) return st; }
  std::lock_guard<std::mutex> ex(c->exec_mu);
  c->calls += 1;
  if (ptrs.empty()) return IPLS_OK;
  g_last_error.clear();
  IPLS_TRY(sort_arrays(c->ws, ptrs.data(), sizes.data(), (int64_t)ptrs.size(), dtype));
  IPLS_CUDA(cudaStreamSynchronize(c->ws.stream));
  return IPLS_OK;
}

iplsStatus iplsSortHost(iplsCtx c, void* host_keys, int64_t n, iplsDtype dtype) {
  IPLS_TRY(check_common(n, dtype));
  if (n > 1 && !host_keys) return fail(IPLS_ERR_ARG, "host_keys is NULL");
  iplsStatus st = IPLS_OK;
  if (!c) { c = default_ctx(&st); if (!c) return st; }
  std::lock_guard<std::mutex> ex(c->exec_mu);
  c->calls += 1;
  if (n <= 1) return IPLS_OK;
  g_last_error.clear();
  const size_t bytes = (size_t)n * key_bytes(dtype);
  Workspace& w = c->ws;
  IPLS_TRY(ensure(w, c->host_stage, c->host_stage_cap, (int64_t)bytes));
  IPLS_CUDA(cudaMemcpyAsync(c->host_stage, host_keys, bytes, cudaMemcpyHostToDevice, w.stream));
  IPLS_TRY(sort_impl(w, c->host_stage, n, dtype, nullptr, 0));
  IPLS_CUDA(cudaMemcpyAsync(host_keys, c->host_stage, bytes, cudaMemcpyDeviceToHost, w.stream));
  IPLS_CUDA(cudaStreamSynchronize(w.stream));
  return IPLS_OK;
}

iplsStatus iplsSortHostBatch(iplsCtx c, void* const* host_keys, const int64_t* n, int64_t count,
                             iplsDtype dtype) {
  if (!valid_dtype(dtype)) return fail(IPLS_ERR_ARG, "unknown dtype");
  if (count < 0) return fail(IPLS_ERR_ARG, "count < 0");
  if (count == 0) return IPLS_OK;
  if (!host_keys || !n) return fail(IPLS_ERR_ARG, "host_keys or n is NULL");
  int64_t max_n = 0;
  for (int64_t i = 0; i < count; ++i) {
    IPLS_TRY(check_common(n[i], dtype));
    if (n[i] > 1 && !host_keys[i]) return fail(IPLS_ERR_ARG, "host_keys[i] is NULL");
    max_n = std::max(max_n, n[i]);
  }
  iplsStatus st = IPLS_OK;
  if (!c) { c = default_ctx(&st); if (!c) return st; }
  std::lock_guard<std::mutex> ex(c->exec_mu);
  c->calls += count;
  g_last_error.clear();
  const int wb = key_bytes(dtype);
  Workspace& w = c->ws;
  for (int k = 0; k < 3; ++k) IPLS_TRY(ensure(w, c->pipe_buf[k], c->pipe_cap[k], max_n * wb));
  if (!c->h2d) {
    IPLS_CUDA(cudaStreamCreateWithFlags(&c->h2d, cudaStreamNonBlocking));
    IPLS_CUDA(cudaStreamCreateWithFlags(&c->d2h, cudaStreamNonBlocking));
    for (int k = 0; k < 3; ++k) {
      IPLS_CUDA(cudaEventCreateWithFlags(&c->in_ev[k], cudaEventDisableTiming));
      IPLS_CUDA(cudaEventCreateWithFlags(&c->sorted_ev[k], cudaEventDisableTiming));
      IPLS_CUDA(cudaEventCreateWithFlags(&c->out_ev[k], cudaEventDisableTiming));
    }
  }
  // array i uses buffer i % 3; its copy in may start once array i - 3 has
  // left that buffer, its sort once it has arrived, its copy out once it is
  // sorted.  The copies in and out of neighbouring arrays run on their own
  // streams while array i is sorted.
  auto copy_in = [&](int64_t i) -> cudaError_t {
    const int k = (int)(i % 3);
    cudaError_t e = cudaSuccess;
    if (i >= 3) e = cudaStreamWaitEvent(c->h2d, c->out_ev[k], 0);
    if (e == cudaSuccess && n[i] > 1)
      e = cudaMemcpyAsync(c->pipe_buf[k], host_keys[i], (size_t)n[i] * wb, cudaMemcpyHostToDevice, c->h2d);
    if (e == cudaSuccess) e = cudaEventRecord(c->in_ev[k], c->h2d);
    return e;
  };
  iplsStatus result = IPLS_OK;
  cudaError_t e = copy_in(0);
  for (int64_t i = 0; i < count && e == cudaSuccess && result == IPLS_OK; ++i) {
    const int k = (int)(i % 3);
    if (i + 1 < count) e = copy_in(i + 1);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(w.stream, c->in_ev[k], 0);
    if (e != cudaSuccess) break;
    if (n[i] > 1) result = sort_impl(w, c->pipe_buf[k], n[i], dtype, nullptr, 0);
    if (result != IPLS_OK) break;
    e = cudaEventRecord(c->sorted_ev[k], w.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->d2h, c->sorted_ev[k], 0);
    if (e == cudaSuccess && n[i] > 1)
      e = cudaMemcpyAsync(host_keys[i], c->pipe_buf[k], (size_t)n[i] * wb, cudaMemcpyDeviceToHost, c->d2h);
    if (e == cudaSuccess) e = cudaEventRecord(c->out_ev[k], c->d2h);
  }
  // every copy this call queued has finished before it returns
  const cudaError_t e1 = cudaStreamSynchronize(c->h2d);
  const cudaError_t e2 = cudaStreamSynchronize(c->d2h);
  if (result != IPLS_OK) return result;
  if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
  if (e != cudaSuccess) return cuda_fail(e, "iplsSortHostBatch");
  return IPLS_OK;
}

iplsStatus iplsGetKernelStats(iplsCtx c, iplsKernelStat* out, int32_t cap, int32_t* count,
                              int32_t reset) {
  if (!c || !count || (cap > 0 && !out)) return fail(IPLS_ERR_ARG, "bad kernel-stats arguments");
  std::lock_guard<std::mutex> ex(c->exec_mu);
  IPLS_CUDA(cudaStreamSynchronize(c->ws.stream));
  resolve_events(c->ws);
  std::lock_guard<std::mutex> lk(c->prof_mu);
  int m = 0;
  for (int k = 0; k < kkCount && m < cap; ++k) {
    std::memset(&out[m], 0, sizeof(out[m]));
    std::strncpy(out[m].name, kKernelNames[k], sizeof(out[m].name) - 1);
    out[m].launches = c->k_launches[k];
    out[m].total_ms = c->k_ms[k];
    out[m].bytes = c->k_bytes[k];
    ++m;
  }
  *count = m;
  if (reset) {
    for (int k = 0; k < 16; ++k) { c->k_launches[k] = 0; c->k_ms[k] = 0.0; c->k_bytes[k] = 0; }
  }
  return IPLS_OK;
}

iplsStatus iplsGetLevelStats(iplsCtx c, iplsLevelStat* out, int32_t cap, int32_t* count, int32_t reset) {
  if (!c || !count || (cap > 0 && !out)) return fail(IPLS_ERR_ARG, "bad level-stats arguments");
  std::lock_guard<std::mutex> ex(c->exec_mu);
  IPLS_CUDA(cudaStreamSynchronize(c->ws.stream));
  resolve_events(c->ws);
  std::lock_guard<std::mutex> lk(c->prof_mu);
  int m = 0;
  for (int l = 0; l < iplsContext::kLevels && m < cap; ++l) {
    if (c->lv_launches[l] == 0 && c->lv_keys[l] == 0) continue;
    out[m].level = l;
    out[m].pad = 0;
    out[m].launches = c->lv_launches[l];
    out[m].keys = c->lv_keys[l];
    out[m].grid_ms = c->lv_ms[l];
    out[m].bytes = c->lv_bytes[l];
    ++m;
  }
  *count = m;
  if (reset)
    for (int l = 0; l < iplsContext::kLevels; ++l) {
      c->lv_ms[l] = 0.0;
      c->lv_launches[l] = c->lv_keys[l] = c->lv_bytes[l] = 0;
    }
  return IPLS_OK;
}

iplsStatus iplsSubmit(iplsCtx c, void* keys, int64_t n, iplsDtype dtype, uint64_t* ticket) {
  if (!c || !ticket) return fail(IPLS_ERR_ARG, "ctx or ticket is NULL");
  IPLS_TRY(check_common(n, dtype));
  if (n > 1 && !keys) return fail(IPLS_ERR_ARG, "keys is NULL");
  IPLS_TRY(check_keys_ptr(keys, dtype));
  if (c->cfg.budget_bytes > 0 && 2 * n * (int64_t)key_bytes(dtype) > c->cfg.budget_bytes)
    return fail(IPLS_ERR_BUDGET, "request exceeds the memory budget");
  {
    std::lock_guard<std::mutex> lk(c->q_mu);
    const uint64_t t = c->next_ticket++;
    c->reqs[t] = iplsContext::Request{keys, n, (int)dtype, n <= 1 ? IPLS_OK : IPLS_PENDING, n <= 1, {}};
    if (n > 1) c->queue.push_back(t);
    const iplsStatus ws = start_workers(c);
    if (ws != IPLS_OK) {
      c->queue.pop_back();
      c->reqs.erase(t);
      return ws;
    }
    *ticket = t;
  }
  c->q_cv.notify_all();
  return IPLS_OK;
}

iplsStatus iplsPoll(iplsCtx c, uint64_t ticket) {
  if (!c) return fail(IPLS_ERR_ARG, "ctx is NULL");
  std::lock_guard<std::mutex> lk(c->q_mu);
  auto it = c->reqs.find(ticket);
  if (it == c->reqs.end()) return fail(IPLS_ERR_ARG, "unknown ticket");
  if (it->second.done && it->second.st != IPLS_OK) g_last_error = it->second.msg;
  return it->second.done ? it->second.st : IPLS_PENDING;
}

iplsStatus iplsWait(iplsCtx c, uint64_t ticket, int64_t timeout_us) {
  if (!c) return fail(IPLS_ERR_ARG, "ctx is NULL");
  std::unique_lock<std::mutex> lk(c->q_mu);
  auto it = c->reqs.find(ticket);
  if (it == c->reqs.end()) return fail(IPLS_ERR_ARG, "unknown ticket");
  auto done = [&] { return it->second.done; };
  if (timeout_us < 0) c->done_cv.wait(lk, done);
  else c->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), done);
  if (it->second.done && it->second.st != IPLS_OK) g_last_error = it->second.msg;
  return it->second.done ? it->second.st : IPLS_PENDING;
}

iplsStatus iplsGetStats(iplsCtx c, iplsStats* out) {
  if (!c || !out) return fail(IPLS_ERR_ARG, "ctx or stats is NULL");
  std::lock_guard<std::mutex> ex(c->exec_mu);
  IPLS_CUDA(cudaStreamSynchronize(c->ws.stream));
  *out = c->ws.stats;
  out->calls = c->calls;
  out->scratch_bytes = c->dev_bytes.load();
  return IPLS_OK;
}

iplsStatus iplsGetBatchLog(iplsCtx c, iplsBatchRec* out, int64_t cap, int64_t* count) {
  if (!c || !count || (cap > 0 && !out)) return fail(IPLS_ERR_ARG, "bad batch-log arguments");
  std::lock_guard<std::mutex> lk(c->q_mu);
  const int64_t m = std::min<int64_t>(cap, (int64_t)c->batch_log.size());
  for (int64_t i = 0; i < m; ++i) out[i] = c->batch_log[i];
  *count = m;
  return IPLS_OK;
}

iplsStatus iplsGetTrace(iplsCtx c, iplsTraceRec* out, int64_t cap, int64_t* count) {
  if (!c || !count || (cap > 0 && !out)) return fail(IPLS_ERR_ARG, "bad trace arguments");
  static_assert(sizeof(iplsTraceRec) == sizeof(iplsTraceRecDev), "trace layout");
  std::lock_guard<std::mutex> ex(c->exec_mu);
  IPLS_CUDA(cudaStreamSynchronize(c->ws.stream));
  *count = 0;
  if (c->cfg.trace_cap <= 0) return IPLS_OK;
  IPLS_CUDA(cudaMemcpy(c->ws.h_run, c->ws.run, sizeof(RunStatus), cudaMemcpyDeviceToHost));
  const int64_t ng = std::min(c->ws.trace_grid_count, c->cfg.trace_cap);
  const int64_t nr = std::min<int64_t>(c->ws.h_run->trace_count, c->cfg.trace_cap);
  const int64_t a = std::min(ng, cap);
  const int64_t b = std::min(nr, cap - a);
  if (a > 0) IPLS_CUDA(cudaMemcpy(out, c->trace_grid, a * sizeof(iplsTraceRec), cudaMemcpyDeviceToHost));
  if (b > 0) IPLS_CUDA(cudaMemcpy(out + a, c->trace_res, b * sizeof(iplsTraceRec), cudaMemcpyDeviceToHost));
  *count = a + b;
  return IPLS_OK;
}

iplsStatus iplsGetTraceKnots(iplsCtx c, float* out, int64_t cap, int64_t* count) {
  if (!c || !count || (cap > 0 && !out)) return fail(IPLS_ERR_ARG, "bad trace-knot arguments");
  std::lock_guard<std::mutex> ex(c->exec_mu);
  IPLS_CUDA(cudaStreamSynchronize(c->ws.stream));
  *count = 0;
  if (c->cfg.trace_cap <= 0 || c->cfg.pl2_leaves <= 0 || !c->trace_knots) return IPLS_OK;
  const int64_t ng = std::min(std::min(c->ws.trace_grid_count, c->cfg.trace_cap), c->knot_cap);
  const int64_t a = std::min(ng, cap);
  if (a > 0)
    IPLS_CUDA(cudaMemcpy(out, c->trace_knots, (size_t)a * (c->cfg.pl2_leaves + 1) * sizeof(float),
                         cudaMemcpyDeviceToHost));
  *count = a;
  return IPLS_OK;
}

const char* iplsLastError(void) { return g_last_error.c_str(); }

}  // extern "C"
