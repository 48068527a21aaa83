// Host runtime behind the C ABI of include/ipls.h: contexts, scratch memory,
// the level loop of the learned partitioning recursion, segmented sorting
// and request tickets.  Every step of the sort runs in the kernels of
// ipls_pass.cu and ipls_resident.cu; this file only plans and launches them.
#include <algorithm>
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

}  // namespace

struct iplsContext {
  iplsConfig cfg;
  iplsAllocFn alloc = nullptr;
  iplsFreeFn free_fn = nullptr;
  void* user = nullptr;
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  char* scratch = nullptr;            int64_t scratch_cap = 0;   // bytes
  unsigned long long* status = nullptr; int64_t status_cap = 0;  // words
  uint32_t* tile_off = nullptr;       int64_t tile_off_cap = 0;  // words
  uint8_t* bids = nullptr;            int64_t bids_cap = 0;      // bytes
  uint32_t epoch = 0;
  Slot slot[2];
  LevelCtl* ctl = nullptr;
  RunStatus* run = nullptr;
  int64_t* root_bounds = nullptr;
  LevelCtl* h_ctl = nullptr;
  RunStatus* h_run = nullptr;
  iplsTraceRecDev* trace_grid = nullptr;
  iplsTraceRecDev* trace_res = nullptr;
  int64_t trace_alloc = 0;
  float* trace_knots = nullptr;       int64_t knot_cap = 0;       // records
  int knot_leaves = 0;
  int64_t trace_grid_count = 0;
  iplsStats stats{};
  // request queue (iplsSubmit): a worker thread batches pending requests
  struct Request {
    void* keys;
    int64_t n;
    int dtype;
    iplsStatus st;
    bool done;
  };
  std::mutex exec_mu;                 // one sort at a time on the context
  std::mutex q_mu;                    // guards the queue and the requests
  std::condition_variable q_cv;       // new request, or stop
  std::condition_variable done_cv;    // a request finished
  std::deque<uint64_t> queue;
  std::map<uint64_t, Request> reqs;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  char* batch_buf = nullptr;          int64_t batch_cap = 0;     // bytes
  int64_t* batch_off = nullptr;       int64_t batch_off_cap = 0; // words
  int64_t* h_batch_off = nullptr;     int64_t h_batch_off_cap = 0;
  int hist_grid[4] = {0, 0, 0, 0};
  int scatter_grid[4] = {0, 0, 0, 0};
  int64_t dev_bytes = 0;
  // profiling (cfg.profile): event pairs per launch, resolved at sync points
  struct Pending { int kind; int level; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> spare_events;
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
  // slow lists of the block-resident tail (children / whole tasks, one half each)
  SlowTask* slow = nullptr; int64_t slow_cap = 0;
  SlowCtl* slow_ctl = nullptr;
  SlowCtl* h_slow = nullptr;          // pinned copy of *slow_ctl
  uint64_t* split_pool = nullptr;     int64_t split_pool_cap = 0;  // words
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
iplsStatus ensure(iplsCtx c, T*& p, int64_t& cap, int64_t need) {
  if (need <= cap && p) return IPLS_OK;
  IPLS_CUDA(cudaStreamSynchronize(c->stream));
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

cudaEvent_t take_event(iplsCtx c) {
  if (!c->spare_events.empty()) {
    cudaEvent_t e = c->spare_events.back();
    c->spare_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return e;
}

// Launches `fn` (which enqueues exactly one kernel) bracketed by CUDA events
// when profiling; every launch is counted.
template <class F>
cudaError_t timed(iplsCtx c, int kind, F fn, int level = -1) {
  if (!c->cfg.profile) {
    cudaError_t e = fn();
    return e;
  }
  cudaEvent_t a = take_event(c), b = take_event(c);
  if (a) cudaEventRecord(a, c->stream);
  cudaError_t e = fn();
  if (b) cudaEventRecord(b, c->stream);
  if (a && b) c->pending.push_back({kind, level, a, b});
  return e;
}

// Folds finished event pairs into the per-kernel totals (after a sync).
void resolve_events(iplsCtx c) {
  for (auto& p : c->pending) {
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
    c->spare_events.push_back(p.a);
    c->spare_events.push_back(p.b);
  }
  c->pending.clear();
}

// Grid kernels size their grids from the occupancy of the SMs they get.
int occupancy_grid(iplsCtx c, int, int) { return c->num_sms; }

// Group list of a slot with its fit list and fitted tail models.
iplsStatus ensure_groups(iplsCtx c, Slot& s, int64_t need) {
  IPLS_TRY(ensure(c, s.groups, s.group_cap, need));
  IPLS_TRY(ensure(c, s.fit_list, s.fit_cap, s.group_cap));
  IPLS_TRY(ensure(c, s.tails, s.tail_cap, s.group_cap));
  return IPLS_OK;
}

// Splitter-pool slots for a tail sweep of nfit fitted tasks.
int64_t pool_slots(int64_t nfit) {
  return std::min<int64_t>(std::max<int64_t>(nfit, kSplitPoolMin), kSplitPoolMax);
}

// One sweep of k_tail_fit + k_tail over the groups in ra.
iplsStatus tail_sweep(iplsCtx c, ResidentArgs& ra) {
  if (ra.nfit > 0) {
    IPLS_TRY(ensure(c, c->split_pool, c->split_pool_cap, pool_slots(ra.nfit) * 128));
    ra.split_pool = c->split_pool;
    ra.split_pool_slots = (int32_t)std::min<int64_t>(c->split_pool_cap / 128, kSplitPoolMax);
    IPLS_CUDA(timed(c, kkTailFit, [&] { return launch_tail_fit(ra, c->stream, c->num_sms); }));
  }
  if (ra.ngroups > 0)
    IPLS_CUDA(timed(c, kkResident, [&] { return launch_resident(ra, c->stream, 0); }));
  if ((ra.large_from_end ? ra.nlarge : ra.ngroups) > 0)
    IPLS_CUDA(timed(c, kkResident, [&] { return launch_resident(ra, c->stream, 1); }));
  return IPLS_OK;
}

// Fits and runs the block-resident tasks listed in slot s: one sweep over
// them, a second one over the children above the cutoff when the first
// queued many (in place in the user buffer; the slot's group list is free
// again once the first sweep ran), and k_slow for the rest.
// nsmall/nlarge: from a level's list (small tasks from the front, large ones
// from the back); with nlarge < 0 the nsmall groups are in plain order and
// both k_tail sizes walk them all.
iplsStatus launch_tail(iplsCtx c, ResidentArgs& ra, Slot& s, int32_t nsmall, int32_t nlarge, int32_t nfit) {
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
  const int64_t half = c->slow_cap / 2;
  ra.slow = c->slow;
  ra.slow_cap = (int32_t)std::min<int64_t>(half, INT32_MAX);
  ra.whole = c->slow + half;
  ra.whole_cap = (int32_t)std::min<int64_t>(c->slow_cap - half, INT32_MAX);
  ra.slow_ctl = c->slow_ctl;
  ra.split_pool = c->split_pool;
  ra.split_pool_slots = (int32_t)std::min<int64_t>(c->split_pool_cap / 128, kSplitPoolMax);
  if (ngroups <= 0) return IPLS_OK;
  IPLS_CUDA(cudaMemsetAsync(c->slow_ctl, 0, sizeof(SlowCtl), c->stream));
  IPLS_TRY(tail_sweep(c, ra));
  if (ngroups >= kTailSweepMin) {
    IPLS_CUDA(cudaMemcpyAsync(c->h_slow, c->slow_ctl, sizeof(SlowCtl), cudaMemcpyDeviceToHost, c->stream));
    IPLS_CUDA(cudaStreamSynchronize(c->stream));
    const int32_t nc = c->h_slow->count;
    if (nc >= kTailSweepMin && nc <= ra.slow_cap) {
      IPLS_TRY(ensure_groups(c, s, nc));
      IPLS_CUDA(timed(c, kkSlowGroups, [&] { return launch_slow_groups(c->slow, nc, s.groups, s.fit_list, c->stream); }));
      // the child list starts again (count, ticket, pool_used, fit_ticket);
      // whole tasks stay
      IPLS_CUDA(cudaMemsetAsync(c->slow_ctl, 0, 4 * sizeof(int32_t), c->stream));
      ra.groups = s.groups;
      ra.ngroups = nc;
      ra.nlarge = nc;            // plain order: both sizes walk the list
      ra.large_from_end = 0;
      ra.fit_list = s.fit_list;
      ra.nfit = nc;
      ra.tail_models = s.tails;
      IPLS_TRY(tail_sweep(c, ra));
      c->stats.sweep_tasks += nc;
    }
  }
  IPLS_CUDA(timed(c, kkSlow, [&] { return launch_slow(ra, c->stream, c->num_sms); }));
  return IPLS_OK;
}

iplsStatus check_run(iplsCtx c) {
  IPLS_CUDA(cudaMemcpyAsync(c->h_run, c->run, sizeof(RunStatus), cudaMemcpyDeviceToHost, c->stream));
  IPLS_CUDA(cudaStreamSynchronize(c->stream));
  if (c->h_run->error == IPLS_ERR_TIMEOUT)
    return fail(IPLS_ERR_TIMEOUT, "a device-side look-back wait exceeded spin_limit");
  if (c->h_run->error != 0)
    return fail((iplsStatus)c->h_run->error, "device reported status " + std::to_string(c->h_run->error));
  c->stats.resident_groups = c->h_run->resident_groups;
  c->stats.slow_tasks = c->h_run->slow_tasks;
  c->stats.slow_passes = c->h_run->slow_passes;
  c->stats.fallback_passes += c->h_run->resident_fallback;
  c->stats.trace_records = c->trace_grid_count + c->h_run->trace_count;
  return IPLS_OK;
}

// The level loop.  Level-0 subproblems are either the whole array or the
// segments; each level runs fit -> hist -> check -> (re)hist -> scan ->
// scatter over all its grid subproblems, then the block-resident kernel over
// the groups the level produced.
iplsStatus sort_impl(iplsCtx c, void* keys, int64_t n, int dtype, const int64_t* offsets,
                     int64_t nseg) {
  const int w = key_bytes(dtype);
  const iplsConfig& cfg = c->cfg;
  const int rmax = resident_rmax(cfg.cutoff);
  const int resident_root_ok = (cfg.root_sample <= 0 || cfg.root_sample <= kResidentSample);
  const int tile = tile_keys(dtype);
  c->stats.grid_levels = 0;
  c->stats.grid_passes = 0;
  c->stats.keys_partitioned = 0;
  c->stats.resident_groups = 0;
  c->stats.fallback_passes = 0;
  c->stats.sweep_tasks = 0;
  c->stats.algorithmic_bytes = 0;
  c->stats.max_bucket_frac = 0.0;
  c->trace_grid_count = 0;
  IPLS_TRY(ensure(c, c->scratch, c->scratch_cap, n * (int64_t)w));
  IPLS_TRY(ensure(c, c->bids, c->bids_cap, n));
  IPLS_TRY(ensure(c, c->slow, c->slow_cap, 2 * (n / (cfg.cutoff + 1)) + 4096));
  if (cfg.trace_cap > 0 && c->trace_alloc < cfg.trace_cap) {
    IPLS_CUDA(cudaStreamSynchronize(c->stream));
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
  if (cfg.trace_cap > 0 && cfg.pl2_leaves > 0 && !c->trace_knots) {
    const int64_t cap = std::min<int64_t>(cfg.trace_cap, kKnotTraceMax);
    void* p;
    IPLS_TRY(dev_alloc(c, &p, (size_t)cap * (cfg.pl2_leaves + 1) * sizeof(float)));
    c->trace_knots = (float*)p;
    c->knot_cap = cap;
    c->knot_leaves = cfg.pl2_leaves;
  }
  IPLS_CUDA(cudaMemsetAsync(c->run, 0, sizeof(RunStatus), c->stream));
  void* bufs[2] = {keys, c->scratch};

  ResidentArgs ra{};
  ra.dtype = dtype; ra.k = cfg.k; ra.cutoff = cfg.cutoff; ra.root_sample = cfg.root_sample;
  ra.seed = cfg.seed; ra.exact_only = cfg.exact_only; ra.buf[0] = bufs[0]; ra.buf[1] = bufs[1];
  ra.run = c->run; ra.trace = cfg.trace_cap > 0 ? c->trace_res : nullptr; ra.trace_cap = cfg.trace_cap;

  int64_t nsub = 0, ntiles = 0, nchunks = 0;
  int64_t max_sub_n = n;  // bound on the size of this level's grid subproblems
  const int64_t sub_bound = n / (rmax + 1) + 2;
  const int64_t tile_bound = n / tile + sub_bound + 2;
  const int64_t chunk_bound = tile_bound / kChunkTiles + sub_bound + 2;
  if (offsets) {
    // segments: big ones become level-0 grid subproblems, the rest groups
    Slot& s0 = c->slot[0];
    Slot& s1 = c->slot[1];
    IPLS_TRY(ensure(c, s0.subs, s0.sub_cap, sub_bound));
    IPLS_TRY(ensure(c, s0.tile2sub, s0.tile_cap, tile_bound));
    IPLS_TRY(ensure(c, s0.chunk2sub, s0.chunk_cap, chunk_bound));
    const int64_t gcap = 2 * n / (cfg.cutoff + 1) + 2 * (nseg / 64) + 1024 + 2 * sub_bound;
    IPLS_TRY(ensure_groups(c, s1, std::min<int64_t>(gcap, nseg + 1024)));
    IPLS_CUDA(cudaMemsetAsync(c->ctl, 0, sizeof(LevelCtl), c->stream));
    IPLS_CUDA(timed(c, kkInitSeg, [&] {
      return launch_init_segments(offsets, nseg, rmax, cfg.cutoff, resident_root_ok, c->ctl,
                                  s0.subs, (int32_t)std::min<int64_t>(s0.sub_cap, INT32_MAX),
                                  s0.tile2sub, s0.tile_cap, s0.chunk2sub, s0.chunk_cap, s1.groups,
                                  (int32_t)std::min<int64_t>(s1.group_cap, INT32_MAX),
                                  s1.fit_list, c->stream);
    }));
    IPLS_CUDA(cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(LevelCtl), cudaMemcpyDeviceToHost, c->stream));
    IPLS_CUDA(cudaStreamSynchronize(c->stream));
    if (c->h_ctl->overflow) return fail(IPLS_ERR_INTERNAL, "segment list capacity exceeded");
    resolve_events(c);
    if ((int64_t)c->h_ctl->ngroups + c->h_ctl->ngroups_large > s1.group_cap)
      return fail(IPLS_ERR_INTERNAL, "segment list capacity exceeded");
    IPLS_TRY(launch_tail(c, ra, s1, c->h_ctl->ngroups, c->h_ctl->ngroups_large, c->h_ctl->nfit));
    nsub = c->h_ctl->nsub_next;
    ntiles = c->h_ctl->tiles_next;
    nchunks = c->h_ctl->chunks_next;
    max_sub_n = c->h_ctl->max_sub_n;
  } else if (n <= rmax && resident_root_ok) {
    // the whole array is one block-resident task (base case only when n is
    // at most the cutoff, otherwise a fitted pass first)
    Slot& s1 = c->slot[1];
    IPLS_TRY(ensure_groups(c, s1, 1));
    const int64_t hb[2] = {0, n};
    const int fitted = n > cfg.cutoff ? 1 : 0;
    IPLS_CUDA(cudaMemcpyAsync(c->root_bounds, hb, sizeof(hb), cudaMemcpyHostToDevice, c->stream));
    const Group g{0, c->root_bounds, (int32_t)n, 0, 0, 1, fitted ? 0 : -1, 0};
    IPLS_CUDA(cudaMemcpyAsync(s1.groups, &g, sizeof(g), cudaMemcpyHostToDevice, c->stream));
    if (fitted) {
      const int32_t zero = 0;
      IPLS_CUDA(cudaMemcpyAsync(s1.fit_list, &zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream));
    }
    IPLS_TRY(launch_tail(c, ra, s1, 1, -1, fitted));
    IPLS_TRY(check_run(c));
    resolve_events(c);
    c->k_bytes[kkResident] += 2 * (int64_t)w * n;
    c->stats.algorithmic_bytes = 2 * (int64_t)w * n;
    return IPLS_OK;
  } else {
    Slot& s0 = c->slot[0];
    IPLS_TRY(ensure(c, s0.subs, s0.sub_cap, 1));
    ntiles = (n + tile - 1) / tile;
    nchunks = (ntiles + kChunkTiles - 1) / kChunkTiles;
    IPLS_TRY(ensure(c, s0.tile2sub, s0.tile_cap, ntiles));
    IPLS_TRY(ensure(c, s0.chunk2sub, s0.chunk_cap, nchunks));
    const Sub root{0, n, 0, 0, 0, (int32_t)ntiles, 0, 0, (int32_t)nchunks};
    IPLS_CUDA(cudaMemcpyAsync(s0.subs, &root, sizeof(root), cudaMemcpyHostToDevice, c->stream));
    IPLS_CUDA(timed(c, kkInitTiles, [&] { return launch_init_tiles(s0.tile2sub, ntiles, 0, c->stream); }));
    IPLS_CUDA(timed(c, kkInitTiles, [&] { return launch_init_tiles(s0.chunk2sub, nchunks, 0, c->stream); }));
    nsub = 1;
  }

  int level = 0;
  int64_t moved = 0;
  while (nsub > 0) {
    if (level > 4096) return fail(IPLS_ERR_INTERNAL, "recursion depth limit exceeded");
    Slot& X = c->slot[level & 1];
    Slot& Y = c->slot[(level + 1) & 1];
    IPLS_TRY(ensure(c, X.models, X.model_cap, nsub));
    IPLS_TRY(ensure(c, X.tabs, X.tab_cap, nsub));
    if (cfg.pl2_leaves > 0) IPLS_TRY(ensure(c, X.knots, X.knot_cap, nsub * (int64_t)(cfg.pl2_leaves + 1)));
    IPLS_TRY(ensure(c, X.counts, X.count_cap, nsub * kMaxK));
    IPLS_TRY(ensure(c, X.bases, X.base_cap, nsub * 257));
    IPLS_TRY(ensure_groups(c, X, 2 * n / (cfg.cutoff + 1) + 257 * nsub + 16));
    IPLS_TRY(ensure(c, X.fills, X.fill_cap, n / kFillChunk + 129 * nsub + 16));
    IPLS_TRY(ensure(c, Y.subs, Y.sub_cap, sub_bound));
    IPLS_TRY(ensure(c, Y.tile2sub, Y.tile_cap, tile_bound));
    IPLS_TRY(ensure(c, Y.chunk2sub, Y.chunk_cap, chunk_bound));
    IPLS_TRY(ensure(c, c->tile_off, c->tile_off_cap, ntiles * kMaxK));
    if (c->status_cap < nchunks * kMaxK) {
      IPLS_TRY(ensure(c, c->status, c->status_cap, nchunks * kMaxK));
      IPLS_CUDA(cudaMemsetAsync(c->status, 0, (size_t)c->status_cap * 8, c->stream));
      c->epoch = 0;
    }
    if (++c->epoch >= 0x10000) {
      IPLS_CUDA(cudaMemsetAsync(c->status, 0, (size_t)c->status_cap * 8, c->stream));
      c->epoch = 1;
    }
    IPLS_CUDA(cudaMemsetAsync(c->ctl, 0, sizeof(LevelCtl), c->stream));
    LevelArgs a{};
    a.dtype = dtype; a.k = cfg.k; a.cutoff = cfg.cutoff; a.rmax = rmax;
    a.root_sample = cfg.root_sample; a.seed = cfg.seed; a.exact_only = cfg.exact_only;
    a.use_tables = (cfg.flags & IPLS_FLAG_THRESHOLD_INDEX) && !cfg.exact_only;
    a.spin_limit = cfg.spin_limit; a.epoch = c->epoch; a.level = level;
    a.buf[0] = bufs[0]; a.buf[1] = bufs[1];
    a.nsub = (int32_t)nsub; a.subs = X.subs; a.models = X.models; a.counts = X.counts;
    a.tabs = X.tabs;
    a.bases = X.bases; a.tile2sub = X.tile2sub; a.ntiles = ntiles; a.status = c->status;
    a.chunk2sub = X.chunk2sub; a.nchunks = nchunks; a.tile_off = c->tile_off;
    a.bids = c->bids;
    a.ctl = c->ctl; a.run = c->run;
    a.next_subs = Y.subs; a.next_sub_cap = (int32_t)std::min<int64_t>(Y.sub_cap, INT32_MAX);
    a.next_tile2sub = Y.tile2sub; a.next_tile_cap = Y.tile_cap;
    a.next_chunk2sub = Y.chunk2sub; a.next_chunk_cap = Y.chunk_cap;
    a.groups = X.groups; a.group_cap = (int32_t)std::min<int64_t>(X.group_cap, INT32_MAX);
    a.fit_list = X.fit_list;
    a.fills = X.fills; a.fill_cap = (int32_t)std::min<int64_t>(X.fill_cap, INT32_MAX);
    a.trace = cfg.trace_cap > 0 ? c->trace_grid : nullptr;
    a.trace_cap = cfg.trace_cap;
    a.trace_base = c->trace_grid_count;
    a.trace_knots = cfg.trace_cap > 0 ? c->trace_knots : nullptr;
    a.knot_cap = c->knot_cap;
    const int max_sample = sample_size_host(std::max<int64_t>(max_sub_n, 2), level, cfg.k, cfg.root_sample);
    a.max_sample = max_sample;
    a.pl2_leaves = cfg.pl2_leaves;
    a.knots = cfg.pl2_leaves > 0 ? X.knots : nullptr;
    IPLS_CUDA(timed(c, kkFit, [&] { return launch_fit(a, c->stream, max_sample); }, level));
    IPLS_CUDA(timed(c, kkHist, [&] { return launch_hist(a, c->stream, 0, occupancy_grid(c, 0, dtype)); }, level));
    IPLS_CUDA(timed(c, kkCheck, [&] { return launch_check(a, c->stream, max_sample); }, level));
    IPLS_CUDA(timed(c, kkRehist, [&] { return launch_hist(a, c->stream, 1, occupancy_grid(c, 0, dtype)); }, level));
    IPLS_CUDA(timed(c, kkScan, [&] { return launch_scan(a, c->stream); }, level));
    IPLS_CUDA(timed(c, kkTileScan, [&] { return launch_tilescan(a, c->stream, c->num_sms * 8); }, level));
    IPLS_CUDA(timed(c, kkScatter, [&] { return launch_scatter(a, c->stream, occupancy_grid(c, 1, dtype)); }, level));
    IPLS_CUDA(cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(LevelCtl), cudaMemcpyDeviceToHost, c->stream));
    IPLS_CUDA(cudaMemcpyAsync(c->h_run, c->run, sizeof(RunStatus), cudaMemcpyDeviceToHost, c->stream));
    IPLS_CUDA(cudaStreamSynchronize(c->stream));
    const LevelCtl lc = *c->h_ctl;
    if (c->h_run->error != 0 || lc.overflow || (int64_t)lc.ngroups + lc.ngroups_large > X.group_cap) {
      // nothing of this level moved (k_scatter checks the status first):
      // put the level's keys back into the user buffer and stop
      IPLS_CUDA(launch_restore(X.subs, (int32_t)nsub, dtype, keys, c->scratch, c->stream));
      IPLS_CUDA(cudaStreamSynchronize(c->stream));
      resolve_events(c);
      if (c->h_run->error == IPLS_ERR_TIMEOUT)
        return fail(IPLS_ERR_TIMEOUT, "a device-side look-back wait exceeded spin_limit; the keys "
                                      "hold a permutation of the input");
      if (c->h_run->error != 0)
        return fail((iplsStatus)c->h_run->error, "device reported status " + std::to_string(c->h_run->error));
      return fail(IPLS_ERR_INTERNAL, "a level list capacity was exceeded");
    }
    resolve_events(c);
    c->k_bytes[kkHist] += (int64_t)w * lc.keys_level;
    c->k_bytes[kkScatter] += 2 * (int64_t)w * lc.keys_moved;
    if (level < iplsContext::kLevels) {
      c->lv_keys[level] += lc.keys_moved;
      c->lv_bytes[level] += 2 * (int64_t)w * lc.keys_moved;
    }
    c->stats.grid_levels += 1;
    c->stats.grid_passes += nsub;
    c->stats.fallback_passes += lc.fallback;
    moved += lc.keys_moved;
    c->stats.max_bucket_frac = std::max(c->stats.max_bucket_frac, (double)lc.max_bucket / 1048576.0);
    c->trace_grid_count += nsub;
    IPLS_TRY(launch_tail(c, ra, X, lc.ngroups, lc.ngroups_large, lc.nfit));
    if (lc.nfill > 0)
      IPLS_CUDA(timed(c, kkFill, [&] { return launch_fill(X.fills, lc.nfill, dtype, keys, c->stream); }));
    nsub = lc.nsub_next;
    ntiles = lc.tiles_next;
    nchunks = lc.chunks_next;
    max_sub_n = lc.max_sub_n;
    ++level;
  }
  IPLS_TRY(check_run(c));
  resolve_events(c);
  c->k_bytes[kkResident] += 2 * (int64_t)w * c->h_run->resident_keys;
  c->stats.keys_partitioned = moved;
  c->stats.algorithmic_bytes = 2 * (int64_t)w * (moved + c->h_run->resident_keys);
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

__global__ void k_init_segments(const int64_t* off, int64_t nseg, int rmax, int cutoff,
                                int resident_ok, LevelCtl* ctl, Sub* subs, int32_t sub_cap,
                                int32_t* tile2sub, int64_t tile_cap, int32_t* chunk2sub,
                                int64_t chunk_cap, Group* groups, int32_t group_cap,
                                int32_t* fit_list) {
  const int64_t wnd = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t q0 = wnd * kSegWindow;
  if (q0 >= nseg) return;
  const int64_t q1 = q0 + kSegWindow < nseg ? q0 + kSegWindow : nseg;
  int64_t g0 = -1, glast = -1, tot = 0;
  for (int64_t q = q0; q <= q1; ++q) {
    const int64_t cq = (q < q1) ? off[q + 1] - off[q] : 0;
    const bool big = cq > cutoff && (cq > rmax || !resident_ok);
    const bool mid = cq > cutoff && !big;
    const bool brk = (q == q1) || big || mid;
    const bool fits = (cq > 0) && !brk;
    if (g0 >= 0 && (brk || (fits && tot + cq > rmax))) {
      const int g = group_slot(ctl, tot, group_cap);
      if (g < 0) ctl->overflow = 1;
      else groups[g] = Group{off[g0], off + g0, (int32_t)tot, 0, 0, (int32_t)(glast - g0 + 1), -1, 0};
      g0 = -1;
      tot = 0;
    }
    if (mid) {
      const int g = group_slot(ctl, cq, group_cap);
      if (g < 0) {
        ctl->overflow = 1;
      } else {
        groups[g] = Group{off[q], nullptr, (int32_t)cq, 0, 0, 1, g, 0};
        fit_list[atomicAdd(&ctl->nfit, 1)] = g;
      }
    }
    if (big) {
      const int i = atomicAdd(&ctl->nsub_next, 1);
      if (i >= sub_cap) {
        ctl->overflow = 1;
      } else {
        Sub ns{off[q], cq, 0, 0, 0, 0, 0, 0, 0};
        if (reserve_tiles(ctl, i, ns, tile2sub, tile_cap, chunk2sub, chunk_cap)) subs[i] = ns;
      }
    }
    if (fits) {
      if (g0 < 0) g0 = q;
      tot += cq;
      glast = q;
    }
  }
}

cudaError_t launch_init_segments(const int64_t* offsets, int64_t nseg, int rmax, int cutoff,
                                 int resident_ok, LevelCtl* ctl, Sub* subs, int32_t sub_cap,
                                 int32_t* tile2sub, int64_t tile_cap, int32_t* chunk2sub,
                                 int64_t chunk_cap, Group* groups, int32_t group_cap,
                                 int32_t* fit_list, cudaStream_t s) {
  const int64_t windows = (nseg + kSegWindow - 1) / kSegWindow;
  if (windows <= 0) return cudaSuccess;
  const int threads = 128;
  const int64_t blocks = (windows + threads - 1) / threads;
  k_init_segments<<<(unsigned)blocks, threads, 0, s>>>(offsets, nseg, rmax, cutoff, resident_ok,
                                                       ctl, subs, sub_cap, tile2sub, tile_cap,
                                                       chunk2sub, chunk_cap, groups, group_cap,
                                                       fit_list);
  return cudaGetLastError();
}

}  // namespace ipls

// ---------------------------------------------------------------------------
// Request serving (iplsSubmit): one worker thread per context forms batches
// from the pending requests -- the oldest request's dtype, in arrival order,
// while they fit the memory budget (cfg.budget_bytes) and cfg.max_batch --
// and sorts a batch with one segmented sort: each request is a segment, so
// the partition passes of all of them share the same launches.  Requests
// that arrive while a batch runs join the next one.
// ---------------------------------------------------------------------------
namespace {

iplsStatus run_batch(iplsCtx c, const std::vector<uint64_t>& batch, int dtype,
                     const std::vector<iplsContext::Request>& rs) {
  std::lock_guard<std::mutex> ex(c->exec_mu);
  const int64_t w = key_bytes(dtype);
  if (rs.size() == 1) {  // alone: in place
    IPLS_TRY(sort_impl(c, rs[0].keys, rs[0].n, dtype, nullptr, 0));
    IPLS_CUDA(cudaStreamSynchronize(c->stream));
    return IPLS_OK;
  }
  const int64_t nseg = (int64_t)rs.size();
  if (c->h_batch_off_cap < nseg + 1) {
    if (c->h_batch_off) cudaFreeHost(c->h_batch_off);
    c->h_batch_off = nullptr;
    c->h_batch_off_cap = 0;
    IPLS_CUDA(cudaMallocHost(&c->h_batch_off, (size_t)(2 * nseg + 16) * 8));
    c->h_batch_off_cap = 2 * nseg + 16;
  }
  int64_t total = 0;
  for (int64_t i = 0; i < nseg; ++i) { c->h_batch_off[i] = total; total += rs[i].n; }
  c->h_batch_off[nseg] = total;
  IPLS_TRY(ensure(c, c->batch_buf, c->batch_cap, total * w));
  IPLS_TRY(ensure(c, c->batch_off, c->batch_off_cap, nseg + 1));
  for (int64_t i = 0; i < nseg; ++i)
    if (rs[i].n > 0)
      IPLS_CUDA(cudaMemcpyAsync(c->batch_buf + c->h_batch_off[i] * w, rs[i].keys, (size_t)(rs[i].n * w),
                                cudaMemcpyDeviceToDevice, c->stream));
  IPLS_CUDA(cudaMemcpyAsync(c->batch_off, c->h_batch_off, (size_t)(nseg + 1) * 8, cudaMemcpyHostToDevice,
                            c->stream));
  IPLS_TRY(sort_impl(c, c->batch_buf, total, dtype, c->batch_off, nseg));
  for (int64_t i = 0; i < nseg; ++i)
    if (rs[i].n > 0)
      IPLS_CUDA(cudaMemcpyAsync(rs[i].keys, c->batch_buf + c->h_batch_off[i] * w, (size_t)(rs[i].n * w),
                                cudaMemcpyDeviceToDevice, c->stream));
  IPLS_CUDA(cudaStreamSynchronize(c->stream));
  (void)batch;
  return IPLS_OK;
}

void serve_loop(iplsCtx c) {
  cudaSetDevice(c->device);
  for (;;) {
    std::vector<uint64_t> batch;
    std::vector<iplsContext::Request> rs;
    int dtype = 0;
    {
      std::unique_lock<std::mutex> lk(c->q_mu);
      c->q_cv.wait(lk, [&] { return c->stop || !c->queue.empty(); });
      if (c->queue.empty()) return;  // stop requested and nothing pending
      dtype = c->reqs[c->queue.front()].dtype;
      const int64_t budget = c->cfg.budget_bytes;
      const int max_batch = c->cfg.max_batch;
      int64_t bytes = 0;
      for (auto it = c->queue.begin(); it != c->queue.end();) {
        const iplsContext::Request& r = c->reqs[*it];
        if (r.dtype != dtype) { ++it; continue; }
        const int64_t need = 2 * r.n * (int64_t)key_bytes(dtype);
        if (!batch.empty() && budget > 0 && bytes + need > budget) break;
        if (max_batch > 0 && (int)batch.size() >= max_batch) break;
        batch.push_back(*it);
        rs.push_back(r);
        bytes += need;
        it = c->queue.erase(it);
      }
    }
    const iplsStatus st = run_batch(c, batch, dtype, rs);
    {
      std::lock_guard<std::mutex> lk(c->q_mu);
      for (uint64_t t : batch) {
        c->reqs[t].st = st;
        c->reqs[t].done = true;
      }
    }
    c->done_cv.notify_all();
  }
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
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_ctl, sizeof(LevelCtl));
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_run, sizeof(RunStatus));
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_slow, sizeof(SlowCtl));
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    if (c->h_run) cudaFreeHost(c->h_run);
    if (c->h_slow) cudaFreeHost(c->h_slow);
    delete c;
    return cuda_fail(e, "iplsCreate");
  }
  void* p;
  if ((st = dev_alloc(c, &p, sizeof(LevelCtl))) != IPLS_OK) { iplsDestroy(c); return st; }
  c->ctl = (LevelCtl*)p;
  if ((st = dev_alloc(c, &p, sizeof(RunStatus))) != IPLS_OK) { iplsDestroy(c); return st; }
  c->run = (RunStatus*)p;
  if ((st = dev_alloc(c, &p, 2 * sizeof(int64_t))) != IPLS_OK) { iplsDestroy(c); return st; }
  c->root_bounds = (int64_t*)p;
  if ((st = dev_alloc(c, &p, sizeof(SlowCtl))) != IPLS_OK) { iplsDestroy(c); return st; }
  c->slow_ctl = (SlowCtl*)p;
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
  if (c->worker.joinable()) c->worker.join();
  cudaStreamSynchronize(c->stream);
  dev_free(c, c->batch_buf, (size_t)c->batch_cap);
  dev_free(c, c->batch_off, (size_t)c->batch_off_cap * 8);
  if (c->h_batch_off) cudaFreeHost(c->h_batch_off);
  dev_free(c, c->scratch, (size_t)c->scratch_cap);
  dev_free(c, c->status, (size_t)c->status_cap * 8);
  dev_free(c, c->tile_off, (size_t)c->tile_off_cap * 4);
  dev_free(c, c->bids, (size_t)c->bids_cap);
  for (Slot& s : c->slot) {
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
  }
  dev_free(c, c->ctl, sizeof(LevelCtl));
  dev_free(c, c->run, sizeof(RunStatus));
  dev_free(c, c->root_bounds, 2 * sizeof(int64_t));
  dev_free(c, c->trace_grid, (size_t)c->trace_alloc * sizeof(iplsTraceRecDev));
  dev_free(c, c->trace_res, (size_t)c->trace_alloc * sizeof(iplsTraceRecDev));
  dev_free(c, c->trace_knots, (size_t)c->knot_cap * (c->knot_leaves + 1) * sizeof(float));
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
  if (c->h_run) cudaFreeHost(c->h_run);
  if (c->h_slow) cudaFreeHost(c->h_slow);
  for (auto& p : c->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
  for (cudaEvent_t e : c->spare_events) cudaEventDestroy(e);
  dev_free(c, c->host_stage, (size_t)c->host_stage_cap);
  dev_free(c, c->slow, (size_t)c->slow_cap * sizeof(SlowTask));
  dev_free(c, c->slow_ctl, sizeof(SlowCtl));
  dev_free(c, c->split_pool, (size_t)c->split_pool_cap * 8);
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
  c->stats.calls += 1;
  if (n <= 1) return IPLS_OK;
  g_last_error.clear();
  std::lock_guard<std::mutex> ex(c->exec_mu);
  return sort_impl(c, keys, n, dtype, nullptr, 0);
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
  // validate the offsets on the host (non-decreasing, within 2^40)
  int64_t first = 0, last = 0;
  IPLS_CUDA(cudaMemcpyAsync(&first, offsets, 8, cudaMemcpyDeviceToHost, c->stream));
  IPLS_CUDA(cudaMemcpyAsync(&last, offsets + nseg, 8, cudaMemcpyDeviceToHost, c->stream));
  IPLS_CUDA(cudaStreamSynchronize(c->stream));
  if (first < 0 || last < first || last > kMaxKeys)
    return fail(IPLS_ERR_ARG, "offsets out of range");
  c->stats.calls += 1;
  g_last_error.clear();
  std::lock_guard<std::mutex> ex(c->exec_mu);
  return sort_impl(c, keys, last, dtype, offsets, nseg);
}

iplsStatus iplsSortHost(iplsCtx c, void* host_keys, int64_t n, iplsDtype dtype) {
  IPLS_TRY(check_common(n, dtype));
  if (n > 1 && !host_keys) return fail(IPLS_ERR_ARG, "host_keys is NULL");
  iplsStatus st = IPLS_OK;
  if (!c) { c = default_ctx(&st); if (!c) return st; }
  c->stats.calls += 1;
  if (n <= 1) return IPLS_OK;
  g_last_error.clear();
  const size_t bytes = (size_t)n * key_bytes(dtype);
  std::lock_guard<std::mutex> ex(c->exec_mu);
  IPLS_TRY(ensure(c, c->host_stage, c->host_stage_cap, (int64_t)bytes));
  IPLS_CUDA(cudaMemcpyAsync(c->host_stage, host_keys, bytes, cudaMemcpyHostToDevice, c->stream));
  IPLS_TRY(sort_impl(c, c->host_stage, n, dtype, nullptr, 0));
  IPLS_CUDA(cudaMemcpyAsync(host_keys, c->host_stage, bytes, cudaMemcpyDeviceToHost, c->stream));
  IPLS_CUDA(cudaStreamSynchronize(c->stream));
  return IPLS_OK;
}

iplsStatus iplsGetKernelStats(iplsCtx c, iplsKernelStat* out, int32_t cap, int32_t* count,
                              int32_t reset) {
  if (!c || !count || (cap > 0 && !out)) return fail(IPLS_ERR_ARG, "bad kernel-stats arguments");
  IPLS_CUDA(cudaStreamSynchronize(c->stream));
  resolve_events(c);
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
  IPLS_CUDA(cudaStreamSynchronize(c->stream));
  resolve_events(c);
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
    c->reqs[t] = iplsContext::Request{keys, n, (int)dtype, n <= 1 ? IPLS_OK : IPLS_PENDING, n <= 1};
    if (n > 1) c->queue.push_back(t);
    if (!c->worker.joinable()) c->worker = std::thread(serve_loop, c);
    *ticket = t;
  }
  c->q_cv.notify_one();
  return IPLS_OK;
}

iplsStatus iplsPoll(iplsCtx c, uint64_t ticket) {
  if (!c) return fail(IPLS_ERR_ARG, "ctx is NULL");
  std::lock_guard<std::mutex> lk(c->q_mu);
  auto it = c->reqs.find(ticket);
  if (it == c->reqs.end()) return fail(IPLS_ERR_ARG, "unknown ticket");
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
  return it->second.done ? it->second.st : IPLS_PENDING;
}

iplsStatus iplsGetStats(iplsCtx c, iplsStats* out) {
  if (!c || !out) return fail(IPLS_ERR_ARG, "ctx or stats is NULL");
  IPLS_CUDA(cudaStreamSynchronize(c->stream));
  c->stats.scratch_bytes = c->dev_bytes;
  *out = c->stats;
  return IPLS_OK;
}

iplsStatus iplsGetTrace(iplsCtx c, iplsTraceRec* out, int64_t cap, int64_t* count) {
  if (!c || !count || (cap > 0 && !out)) return fail(IPLS_ERR_ARG, "bad trace arguments");
  static_assert(sizeof(iplsTraceRec) == sizeof(iplsTraceRecDev), "trace layout");
  IPLS_CUDA(cudaStreamSynchronize(c->stream));
  *count = 0;
  if (c->cfg.trace_cap <= 0) return IPLS_OK;
  IPLS_CUDA(cudaMemcpy(c->h_run, c->run, sizeof(RunStatus), cudaMemcpyDeviceToHost));
  const int64_t ng = std::min(c->trace_grid_count, c->cfg.trace_cap);
  const int64_t nr = std::min<int64_t>(c->h_run->trace_count, c->cfg.trace_cap);
  const int64_t a = std::min(ng, cap);
  const int64_t b = std::min(nr, cap - a);
  if (a > 0) IPLS_CUDA(cudaMemcpy(out, c->trace_grid, a * sizeof(iplsTraceRec), cudaMemcpyDeviceToHost));
  if (b > 0) IPLS_CUDA(cudaMemcpy(out + a, c->trace_res, b * sizeof(iplsTraceRec), cudaMemcpyDeviceToHost));
  *count = a + b;
  return IPLS_OK;
}

iplsStatus iplsGetTraceKnots(iplsCtx c, float* out, int64_t cap, int64_t* count) {
  if (!c || !count || (cap > 0 && !out)) return fail(IPLS_ERR_ARG, "bad trace-knot arguments");
  IPLS_CUDA(cudaStreamSynchronize(c->stream));
  *count = 0;
  if (c->cfg.trace_cap <= 0 || c->cfg.pl2_leaves <= 0 || !c->trace_knots) return IPLS_OK;
  const int64_t ng = std::min(std::min(c->trace_grid_count, c->cfg.trace_cap), c->knot_cap);
  const int64_t a = std::min(ng, cap);
  if (a > 0)
    IPLS_CUDA(cudaMemcpy(out, c->trace_knots, (size_t)a * (c->cfg.pl2_leaves + 1) * sizeof(float),
                         cudaMemcpyDeviceToHost));
  *count = a;
  return IPLS_OK;
}

const char* iplsLastError(void) { return g_last_error.c_str(); }

}  // extern "C"
