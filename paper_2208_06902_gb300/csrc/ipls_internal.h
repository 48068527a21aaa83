// Internal layouts shared by the host runtime and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ipls {

constexpr int kMaxK = 256;        // buckets per pass (paper: 256)
constexpr int kMaxSplit = 127;    // splitters: 2*127+1 = 255 buckets
constexpr int kTileKeys = 4096;   // keys per grid-pass tile
constexpr int kPassThreads = 256; // threads of the grid-pass kernels
constexpr int kResidentMax = 8192;      // keys of one block-resident group
constexpr int kResidentThreads = 512;
constexpr int kResidentSample = 1024;   // sample capacity inside a resident block
// Block-resident tasks of at most kTailSmall keys run in 256-thread blocks
// (four per SM), larger ones in 512-thread blocks (two per SM).
constexpr int kTailSmall = 4096;
constexpr int kResidentTasks = 2048;    // pending ranges inside a resident block
constexpr int kFitThreads = 1024;
constexpr int kFillChunk = 65536;

enum ModelKind : int32_t { kLinear = 0, kSplitter = 1, kPL2 = 2 };

// PL2 (piecewise-linear CDF): used, when enabled, for subproblems larger
// than kPL2MinKeys whose sample has at most kPL2MaxSample keys; trained for
// kPL2Steps steps.  Model layout: l.kind = kPL2, l.nb = k, l.S, l.D = leaf
// shift, l.rho, l.qlo = X(sample minimum); nsplit = leaves M.  The knot values
// y_0..y_M (binary32) are in the level's knot buffer, M + 1 per subproblem.
constexpr int64_t kPL2MinKeys = 8192;
constexpr int kPL2MaxSample = 4096;
constexpr int kPL2Steps = 8;
constexpr int kPL2MaxLeaves = 1024;
// Grid-pass trace records whose PL2 knots are kept (iplsGetTraceKnots).
constexpr int64_t kKnotTraceMax = 16384;

// Linear partition model of one subproblem: b(x) = clamp(floor(fma(A,
// x (-) x_lo, Bc)), 0, nb-1) (Ch.3 model equation, centred form).
// kind == kSplitter means the sample does not support the linear model and
// the splitter tree has to be built (Ch.3 "Decision Trees").
struct LinModel {
  int32_t kind;
  int32_t nb;
  int32_t capped;
  int32_t fast;   // the fixed-point / FP32 estimate applies (see Classifier)
  int64_t S;
  int64_t D;
  double A;
  double Bc;
  double ud;
  uint64_t xlo_bits;
  int32_t rho;    // fixed-point scale: X(x) = trunc(x / 2^rho)
  int32_t pad;
  int64_t qlo;    // X(x_lo)
  float af;       // RN32(A * 2^rho)
  float bcf;      // RN32(Bc)
  float crel;     // certified bound = crel*|v| + cabs
  float cabs;
  // Same-binade estimate: for a key in the binade of x_lo (integer keys:
  // within 2^62 of it), x (-) x_lo = (u - u_lo) * q exactly, with u the
  // totalOrder bits and q the binade's spacing (1 for integers), so the model
  // value is estimated from D = (u - u_lo) >> ushift as fmaf(auf, D, bcf),
  // auf = RN32(A * q * 2^ushift), certified by crel*|v| + ucabs.
  int32_t ufast;
  int32_t ushift;
  float auf;
  float ucabs;
  // Uncentred estimate (float keys whose binary32 truncation xf is a normal
  // number): v = fmaf(gaf, xf, gbf) with gaf = RN32(A), gbf = RN32(Bc - A x_lo),
  // certified by gc1*|xf| + crel*|v| + gcabs.
  int32_t gfast;
  float gaf;
  float gbf;
  float gc1;
  float gcabs;
  int32_t gpad;
};

// Full model: the linear part, or unique splitters s_1 < ... < s_m as
// totalOrder keys with equality buckets at odd ids.
struct Model {
  LinModel l;
  int32_t nsplit;
  int32_t pad;
  uint64_t split[128];
};

// Model of a block-resident tail task as k_tail_fit leaves it: the linear
// part, or (kind kSplitter) the unique splitters built from the same sorted
// sample -- up to kTailSplit inline, more in slot `pool` of the splitter
// pool (pool < 0: none was free, the task takes the slow path).
constexpr int kTailSplit = 8;
struct TailModel {
  LinModel l;
  int32_t nsplit;
  int32_t pool;
  uint64_t split[kTailSplit];
};

// Exact bucket thresholds of a linear model and a two-level index over them
// (grid-level subproblems).  thr[j] (j = 1..nb-1) is the smallest
// totalOrder key whose bucket under the binary64 model is at least j, so the
// bucket of a key u is the number of thresholds <= u.  Float keys: l1 is
// indexed by the key's sign and exponent (one entry per binade between thr[1]
// and thr[nb-1]); an entry is either a constant bucket or, with bit 15 set,
// (m << 11 | offset) for 2^m cells of l2 indexed by the top m mantissa bits,
// each cell holding the bucket at its start.  Integer keys: one entry whose
// cells are (u - thr[1]) >> ishift.
constexpr int kL1Max = 4096;
constexpr int kL2Max = 2048;
struct ThrTable {
  uint64_t thr[kMaxK + 1];
  uint16_t l1[kL1Max];
  uint8_t l2[kL2Max];
  int32_t ok;       // 1: use the tables; 0: classify with the model
  int32_t e_lo;     // coarse index of l1[0]
  int32_t n_l1;
  int32_t ishift;   // integer keys: cell shift
};

// Every record below names its subproblem's keys by `off`, a position in the
// sort's index space (the whole array, or the segments one after another), and
// by `ubase`, the address such that, while the keys are in the caller's
// memory (buffer 0), key `off + i` is at ((Bits*)ubase)[off + i].  One array
// has one ubase; a batch of separate arrays has one per array, so each is
// sorted where it lives.  Buffer 1 (the context's ping-pong buffer) is indexed
// by `off` directly.
// A grid-level subproblem.
struct Sub {
  int64_t off;     // first key in the index space
  int64_t n;
  int32_t level;
  int32_t buf;     // 0 = user keys, 1 = scratch
  int64_t tile0;   // first tile of this subproblem in the level's tile space
  int32_t ntiles;
  int32_t flags;
  int32_t chunk0;  // first tile chunk (kChunkTiles tiles) of this subproblem
  int32_t nchunks;
  uint64_t ubase;  // caller's memory of this subproblem (see above)
};
constexpr int kChunkTiles = 32;  // tiles per decoupled look-back chunk
enum SubFlags : int32_t { kRehist = 1, kSkipScatter = 2 };

// A block-resident task.  fit < 0: consecutive children [off, off+n) of one
// parent (or consecutive segments), each of at most `cutoff` keys, child c
// spanning [bounds[c]-bounds[0], bounds[c+1]-bounds[0]); they only need the
// base case.  fit >= 0: one subproblem [off, off+n) at `level` whose model
// was fitted by k_tail_fit into tail_models[fit].
struct Group {
  int64_t off;
  const int64_t* bounds;
  int32_t n;
  int32_t level;
  int32_t buf;
  int32_t nchild;
  int32_t fit;
  int32_t pad;
  uint64_t ubase;
};

// Keys [off, off+n) of the user buffer all equal to `bits`.
struct Fill {
  int64_t off;
  int64_t n;
  uint64_t bits;
  uint64_t ubase;
};

// Device-side counters of one level (zeroed before the level).
struct LevelCtl {
  int32_t nsub_next;
  int32_t ngroups;
  int32_t nfill;
  int32_t nrehist;
  int32_t nfit;          // tasks needing a tail fit
  int32_t ngroups_large; // tasks of more than kTailSmall keys (listed from the back)
  int64_t tiles_next;
  int64_t chunks_next;
  uint32_t ticket;
  int32_t overflow;      // a list capacity was exceeded
  int64_t fallback;      // splitter passes
  int64_t max_bucket;    // max over passes of largest bucket / n, scaled by 2^20
  int64_t keys_moved;    // keys scattered by this level's grid passes
  int64_t keys_level;    // keys in this level's grid subproblems
  int64_t max_sub_n;     // largest grid subproblem created for the next level
  uint32_t tile_ticket[2];  // next tile group of [0] k_hist, [1] k_scatter
};

// Run-wide device status (persists across levels of one call).
struct RunStatus {
  int32_t error;         // 0 or a negative iplsStatus
  int32_t where;         // which wait gave up (diagnostics)
  int32_t error_level;   // 1 + the first grid level whose scatter moved nothing
                         // because of an error (0: none)
  int32_t pad;
  int64_t trace_count;
  int64_t resident_passes;
  int64_t resident_fallback;
  int64_t resident_keys;
  int64_t resident_groups;
  int64_t slow_tasks;
  int64_t slow_passes;
};

// A range of the user buffer that needs the in-block recursion (a bucket
// above the cutoff, or a task whose model is the splitter tree or made no
// progress): keys [off, off+n) form one subproblem at `level`.
struct SlowTask {
  int64_t off;
  int32_t n;
  int32_t level;
  uint64_t ubase;
};

// Counters of the slow lists (zeroed before each tail launch).  `count`
// children above the cutoff wait in the child list, `wcount` whole tasks
// (no progress, or no pool slot for their splitters) in the whole list.
struct SlowCtl {
  int32_t count;
  uint32_t ticket;
  int32_t pool_used;   // splitter-pool slots taken by this tail sweep
  int32_t fit_ticket;  // next task of k_tail_fit's persistent warps
  int32_t wcount;
  int32_t sweep;       // device-driven levels: tasks of the second sweep (0: none)
  int32_t tticket[2];  // device-driven levels: next task of the small / large k_tail
};

// Splitters of a tail task whose tree has more than kTailSplit of them (one
// pool slot per such task; a task that finds the pool full takes the slow
// path).  The pool has a slot for every fitted task of a round, at least
// kSplitPoolMin and at most kSplitPoolMax of them.
constexpr int kSplitPoolMin = 16384;
constexpr int kSplitPoolMax = 1 << 18;
// A second tail sweep takes the children above the cutoff when the first
// round queued at least this many (fewer go straight to k_slow).
constexpr int kTailSweepMin = 1024;

// Per-level device arrays (all device pointers).
struct LevelArgs {
  int dtype;
  int k;
  int cutoff;
  int rmax;              // children above this size stay grid-level
  int64_t root_sample;
  uint64_t seed;
  int exact_only;
  int use_tables;        // build and use the exact threshold index
  int pl2_leaves;        // 0, or PL2 leaves for subproblems above kPL2MinKeys
  int pl2_depth;         // PL2 only at levels below this (0: every level)
  float* knots;          // [nsub][pl2_leaves + 1] PL2 knot values (when pl2_leaves > 0)
  int max_sample;        // largest sample of the level (k_fit's shared-memory layout)
  int64_t spin_limit;
  uint32_t epoch;        // look-back epoch of this level's scatter
  int level;
  int src_buf;           // buffer this level's subproblems live in
  void* buf[2];          // buf[1] = the ping-pong buffer (buffer 0 is each record's ubase)
  int32_t nsub;
  Sub* subs;
  Model* models;
  ThrTable* tabs;        // [nsub]
  uint64_t* counts;      // [nsub][256]
  int64_t* bases;        // [nsub][257]
  int32_t* tile2sub;     // this level's tiles
  int64_t ntiles;
  int32_t* chunk2sub;    // this level's tile chunks
  int64_t nchunks;
  uint32_t* tile_off;    // [ntiles][256]: tile histogram, then offsets in bucket
  uint8_t* bids;         // bucket of every key of this level (by key position)
  unsigned long long* status;  // look-back words [nchunks][256]
  LevelCtl* ctl;
  RunStatus* run;
  // outputs for the next level
  Sub* next_subs;
  int32_t next_sub_cap;
  int32_t* next_tile2sub;
  int64_t next_tile_cap;
  int32_t* next_chunk2sub;
  int64_t next_chunk_cap;
  Group* groups;
  int32_t group_cap;
  int32_t* fit_list;     // groups[fit_list[i]] need a tail fit
  Fill* fills;
  int32_t fill_cap;
  // trace: grid passes of this level take records trace_base + s
  struct iplsTraceRecDev* trace;
  int64_t trace_cap;
  int64_t trace_base;
  float* trace_knots;    // PL2 knots of grid records (pl2_leaves + 1 each), or NULL
  int64_t knot_cap;      // records with room in trace_knots
  // Device-driven levels (no host round trip between levels): when cnt is
  // set, this level's subproblem, tile and chunk counts are the previous
  // level's nsub_next, tiles_next and chunks_next (written by k_scan or
  // k_init_segments), capped by nsub, ntiles and nchunks, which are then
  // capacities; a level after an overflow or a device error does nothing.
  const LevelCtl* cnt;
  long long* trace_ctr;  // device-driven levels: next free grid trace record
};

struct ResidentArgs {
  int dtype;
  int k;
  int cutoff;
  int64_t root_sample;
  uint64_t seed;
  int exact_only;
  void* buf[2];                    // buf[1] = the ping-pong buffer (buffer 0: each record's ubase)
  const Group* groups;
  int32_t ngroups;                 // groups[0, ngroups) (the small ones when large_from_end)
  int32_t nlarge;                  // tasks for the large blocks
  int32_t group_cap;
  int32_t large_from_end;          // 1: the large tasks are groups[group_cap-1-i], i < nlarge;
                                   // 0: both sizes walk groups[0, ngroups) and skip the other's
  const int32_t* fit_list;
  int32_t nfit;
  TailModel* tail_models;          // indexed by Group::fit
  SlowTask* slow;                  // child list (capacity slow_cap)
  int32_t slow_cap;
  int32_t whole_cap;
  SlowTask* whole;                 // whole-task list (capacity whole_cap)
  SlowCtl* slow_ctl;
  uint64_t* split_pool;            // [split_pool_slots][128] splitters
  int32_t split_pool_slots;
  RunStatus* run;
  struct iplsTraceRecDev* trace;   // block-resident passes append here
  int64_t trace_cap;
  // Device-driven levels: the group counts are those gcnt (the level's
  // LevelCtl) holds, or for a second sweep (sweep = 1) slow_ctl->sweep; the
  // kernels then loop over the tasks with a fixed grid.
  LevelCtl* gcnt;
  int32_t sweep;
  int32_t device_counts;
};

// Tasks of a tail launch: host-given counts, or (device-driven levels) the
// counts the level's k_scan left in *gcnt -- none once the level overflowed,
// a device error was raised, or the two ends of the group list met (which
// marks the level as overflowed for the host to see).
__device__ __forceinline__ int32_t tail_count(const ResidentArgs& a, bool large) {
  if (!a.device_counts) return (large && a.large_from_end) ? a.nlarge : a.ngroups;
  // a level whose scatter stopped on an error has nothing to finish
  if (*reinterpret_cast<const volatile int32_t*>(&a.run->error_level) != 0) return 0;
  if (a.sweep) return *reinterpret_cast<const volatile int32_t*>(&a.slow_ctl->sweep);
  const volatile LevelCtl* g = a.gcnt;
  if (g->overflow) return 0;
  if ((int64_t)g->ngroups + g->ngroups_large > a.group_cap) {
    a.gcnt->overflow = 1;
    return 0;
  }
  return large ? g->ngroups_large : g->ngroups;
}
__device__ __forceinline__ int32_t tail_nfit(const ResidentArgs& a) {
  if (!a.device_counts) return a.nfit;
  if (a.sweep) return tail_count(a, false);
  return tail_count(a, false) > 0 || tail_count(a, true) > 0 ? a.gcnt->nfit : 0;
}

// Same layout as iplsTraceRec in the public header.
struct iplsTraceRecDev {
  int64_t off, n;
  int32_t level, kind, capped, nbuckets;
  int64_t S, D;
  double A, Bc, ud;
  uint64_t xlo_bits;
  int32_t nsplit, where;
  int64_t counts[256];
};

// Counts of a level (device-driven levels read them from the device).
__device__ __forceinline__ bool level_dead(const LevelArgs& a) {
  // (after an error the level still launches its scatter, which moves
  // nothing and records that it stopped there)
  return a.cnt && (*reinterpret_cast<const volatile int32_t*>(&a.cnt->overflow) != 0 ||
                   *reinterpret_cast<const volatile int32_t*>(&a.run->error_level) != 0);
}
__device__ __forceinline__ int32_t level_nsub(const LevelArgs& a) {
  if (!a.cnt) return a.nsub;
  if (level_dead(a)) return 0;
  const int32_t v = a.cnt->nsub_next;
  return v < a.nsub ? v : a.nsub;
}
__device__ __forceinline__ int64_t level_ntiles(const LevelArgs& a) {
  if (!a.cnt) return a.ntiles;
  if (level_dead(a)) return 0;
  const int64_t v = a.cnt->tiles_next;
  return v < a.ntiles ? v : a.ntiles;
}
__device__ __forceinline__ int64_t level_nchunks(const LevelArgs& a) {
  if (!a.cnt) return a.nchunks;
  if (level_dead(a)) return 0;
  const int64_t v = a.cnt->chunks_next;
  return v < a.nchunks ? v : a.nchunks;
}

// Keys of a record: the caller's memory (buf 0, at ubase) or the ping-pong buffer.
template <class B>
__host__ __device__ __forceinline__ B* keys_of(int buf, uint64_t ubase, void* const* bufs) {
  return buf == 0 ? reinterpret_cast<B*>(ubase) : reinterpret_cast<B*>(bufs[1]);
}

// Kernel launchers (defined in the .cu files).
cudaError_t launch_fit(const LevelArgs& a, cudaStream_t s, int max_sample, int sms);
cudaError_t launch_hist(const LevelArgs& a, cudaStream_t s, int rehist_only, int sms);
cudaError_t launch_check(const LevelArgs& a, cudaStream_t s, int max_sample, int sms);
cudaError_t launch_scan(const LevelArgs& a, cudaStream_t s, int sms);
cudaError_t launch_tilescan(const LevelArgs& a, cudaStream_t s, int grid);
cudaError_t launch_scatter(const LevelArgs& a, cudaStream_t s, int sms);
cudaError_t launch_tail_fit(const ResidentArgs& a, cudaStream_t s, int sms);
// large = 0: tasks of up to 4096 keys (256-thread blocks); 1: the rest.
cudaError_t launch_resident(const ResidentArgs& a, cudaStream_t s, int large, int sms);
cudaError_t launch_slow(const ResidentArgs& a, cudaStream_t s, int sms);
// groups[i] = the fitted tail task of list[i], fit_list[i] = i (i < n).
cudaError_t launch_slow_groups(const SlowTask* list, int32_t n, Group* groups, int32_t* fit_list,
                               cudaStream_t s);
// One block sorts keys[t.off, t.off + t.n) (t.n <= resident_rmax(a.cutoff));
// it reads and writes only the keys and *a.run.
cudaError_t launch_slow_one(const ResidentArgs& a, const SlowTask& t, cudaStream_t s);
// Sets the message iplsLastError() returns on this thread.
void set_last_error(const char* msg);
// seg_ubase: per-segment ubase (device array), or NULL for `ubase` everywhere.
cudaError_t launch_init_segments(const int64_t* offsets, int64_t nseg, const uint64_t* seg_ubase,
                                 uint64_t ubase, int rmax, int cutoff,
                                 int resident_ok, LevelCtl* ctl, Sub* subs, int32_t sub_cap,
                                 int32_t* tile2sub, int64_t tile_cap, int32_t* chunk2sub,
                                 int64_t chunk_cap, Group* groups, int32_t group_cap,
                                 int32_t* fit_list, cudaStream_t s);
int resident_rmax(int cutoff);
// cnt (device-driven levels): nfill is then a capacity and the count is
// cnt->nfill (nothing once the level overflowed).
cudaError_t launch_fill(const Fill* fills, int32_t nfill, int dtype, cudaStream_t s,
                        const LevelCtl* cnt = nullptr, int grid = 0, const RunStatus* run = nullptr);
// Device-driven second sweep: when the first sweep queued at least
// kTailSweepMin children (and the list fits), turns them into the sweep's
// groups, sets ctl->sweep to their number and restarts the child list;
// otherwise sets ctl->sweep = 0 and leaves them to k_slow.
cudaError_t launch_sweep_groups(const SlowTask* list, SlowCtl* ctl, int32_t list_cap, Group* groups,
                                int32_t* fit_list, int32_t group_cap, cudaStream_t s);
cudaError_t launch_init_tiles(int32_t* tile2sub, int64_t ntiles, int32_t value, cudaStream_t s);
// Copies the keys of the level's subproblems held in the scratch buffer back
// into the caller's memory (after a device-side error).
cudaError_t launch_restore(const Sub* subs, int32_t nsub, int dtype, const void* scratch, cudaStream_t s);

int tile_keys(int dtype);
int key_bytes(int dtype);
int sample_size_host(int64_t n, int level, int k, int64_t root_sample);

}  // namespace ipls
