/* ipls.h -- C ABI of the GB300 learned-sort library.
 *
 * The library sorts numeric keys on one GPU with the learned partitioning
 * pass of In-Place Parallel Learned Sort (IPLS, arxiv 2208.06902): fit a
 * linear partition model by FMCD on a sample, classify every key into one
 * of k buckets, histogram and prefix-sum the buckets, scatter the keys into
 * contiguous bucket runs, recurse into large buckets and base-case-sort
 * small ones.  Every step runs in this library's own CUDA kernels.
 *
 * Conventions shared by every entry point:
 *   - Keys are plain device arrays of one dtype, no payload.  The result is
 *     ascending under IEEE 754 totalOrder for float dtypes (-NaN < -inf < ...
 *     < -0 < +0 < ... < +inf < +NaN) and natural order for integers.  The
 *     sorted permutation is unique, so the output is bit-exact.
 *   - Sizes are counts of keys (int64).  n = 0 or 1 is a no-op returning
 *     IPLS_OK.  n < 0, n > 2^32 - 1, a NULL pointer, or an unknown dtype
 *     return IPLS_ERR_ARG without touching memory.
 *   - Device pointers must be valid for the GPU the context was created on
 *     and aligned to the key width.  The caller owns `keys`; the context
 *     owns all scratch memory (one ping-pong key buffer of n keys, one bucket
 *     id byte per key, and per-level bookkeeping), allocated through the
 *     context's allocator.
 *   - Work is enqueued on the context's stream.  With cfg.sync = 1 (the
 *     default) a call waits for its work and returns the device status;
 *     with cfg.sync = 0 it returns after enqueueing and a device-side error
 *     surfaces at the next synchronising call (iplsGetStats, iplsWait, or a
 *     synchronous sort).
 *   - IPLS_ERR_ARG and IPLS_ERR_BUDGET leave the key array untouched.
 *     IPLS_ERR_TIMEOUT and IPLS_ERR_INTERNAL (device-side conditions) leave
 *     it holding a permutation of its input: keys are only ever moved, a
 *     partition level that sees the error moves nothing, and the keys of
 *     that level still in the context's ping-pong buffer are copied back.
 *     After IPLS_ERR_OOM or IPLS_ERR_CUDA its contents are unspecified.  The
 *     context stays usable; its next call starts from a clean state.
 *   - iplsLastError() returns a thread-local message for the last failure.
 */
#ifndef IPLS_H_
#define IPLS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { IPLS_F64 = 0, IPLS_F32 = 1, IPLS_U64 = 2, IPLS_U32 = 3 } iplsDtype;

typedef enum {
  IPLS_OK = 0,
  IPLS_PENDING = 1,          /* iplsPoll: the request has not finished */
  IPLS_ERR_ARG = -1,         /* invalid argument; nothing was enqueued */
  IPLS_ERR_OOM = -2,         /* the allocator returned NULL */
  IPLS_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  IPLS_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
  IPLS_ERR_BUDGET = -5,      /* a request exceeds the context's memory budget */
  IPLS_ERR_INTERNAL = -6     /* an internal limit (recursion depth) was hit */
} iplsStatus;

/* Parameters of the method and of the run.  iplsDefaultConfig() fills the
 * paper's values: k = 256 buckets per pass and a sample of alpha*k - 1 keys
 * with alpha = 0.2 log2 n (Ch.4 "Proposed Algorithm"). */
typedef struct iplsConfig {
  int32_t k;              /* buckets per pass, 3..256 (paper: 256) */
  int32_t cutoff;         /* subproblems of <= cutoff keys are base-cased (>= 1) */
  int64_t root_sample;    /* sample size of the top-level subproblem; 0 = formula */
  uint64_t seed;          /* seed of the counter-based sampling stream */
  int32_t sync;           /* 1: calls wait for the device and check its status */
  int32_t exact_only;     /* 1: evaluate the model in binary64 for every key
                             (same result, slower; for testing) */
  int64_t spin_limit;     /* polls of a device-side wait before IPLS_ERR_TIMEOUT */
  int64_t trace_cap;      /* records kept by iplsGetTrace (0 = tracing off) */
  int64_t budget_bytes;   /* iplsSubmit admission budget (0 = unlimited) */
  int32_t profile;        /* 1: time every kernel launch with CUDA events
                             (read with iplsGetKernelStats) */
  int32_t flags;          /* IPLS_FLAG_* bits (tuning switches; results do not change) */
  int32_t max_batch;      /* iplsSubmit: requests sorted together at most (0 = no limit,
                             1 = one at a time) */
  int32_t pl2_leaves;     /* 0: the FMCD linear model everywhere (the paper's IPLS).
                             2..1024 (a power of two): subproblems of more than 8192 keys
                             whose sample has at most 4096 keys use the two-level
                             piecewise-linear CDF model PL2 with this many leaves
                             (Ch.2 Learned Sort, Ch.3 RMI: a learned CDF trained on
                             the sample against its empirical CDF), falling back to
                             the splitter tree when a bucket gets more than 4n/k keys.
                             The sorted result is the same either way. */
  int32_t serve_slots;    /* iplsSubmit: batches in flight at once, 1 or 2 (0 = 2) */
  int32_t pl2_depth;      /* with pl2_leaves: PL2 only at recursion levels below this
                             (default 1: the whole array or each segment; 0 = every level) */
  int32_t reserved[2];
} iplsConfig;

/* cfg.flags: classify grid-level passes through the exact threshold index
 * instead of the certified fixed-point estimate (same buckets, different
 * speed; off by default). */
#define IPLS_FLAG_THRESHOLD_INDEX 1

/* cfg.flags: iplsSortSegmented runs its recursion levels without host round
 * trips -- every kernel reads its level's counts from device memory -- and
 * captures them into a CUDA graph, replayed while the keys pointer, offsets
 * pointer, segment count and total stay the same (deeper recursion than the
 * graph holds continues level by level from the host).  Buffers are sized
 * for the worst case up front, so the context holds more scratch.  Same
 * sorted result. */
#define IPLS_FLAG_GRAPH 2

/* Accumulated device time of one kernel of the library (profile = 1).
 * bytes = algorithmic bytes: keys read + keys written by the launches, in
 * bytes (the classify/histogram sweep reads every live key once, the scatter
 * reads and writes every live key once, the block-resident kernel reads and
 * writes each of its keys once). */
typedef struct iplsKernelStat {
  char name[24];
  int64_t launches;
  double total_ms;        /* sum of CUDA-event durations of the launches */
  int64_t bytes;          /* algorithmic bytes moved by those launches */
} iplsKernelStat;

/* Device time of the grid-level partition passes of one recursion level
 * (profile = 1), accumulated over calls: grid_ms sums the CUDA-event
 * durations of that level's grid kernels (fit, classify + histogram, check,
 * scans, scatter); keys counts the keys those passes moved and bytes their
 * algorithmic bytes, 2 * w * keys (every moved key read once and written
 * once, Ch.2 IPS4o partitioning step). */
typedef struct iplsLevelStat {
  int32_t level;
  int32_t pad;
  int64_t launches;
  int64_t keys;
  double grid_ms;
  int64_t bytes;
} iplsLevelStat;

/* One partition pass as recorded by the trace (see iplsGetTrace). */
typedef struct iplsTraceRec {
  int64_t off;            /* first key of the subproblem in the whole array */
  int64_t n;              /* keys in the subproblem */
  int32_t level;          /* recursion level (0 = whole array or segment) */
  int32_t kind;           /* 0 = FMCD linear model, 1 = splitter tree, 2 = PL2 */
  int32_t capped;         /* FMCD stopped at its 3D > N break */
  int32_t nbuckets;       /* k, or 2*nsplit+1 for the splitter tree */
  int64_t S;              /* sample size */
  int64_t D;              /* FMCD's conflict-degree parameter */
  double A;               /* slope of the centred model */
  double Bc;              /* intercept of the centred model */
  double ud;              /* the u_d the slope came from */
  uint64_t xlo_bits;      /* raw bits of the centre key x[D] */
  int32_t nsplit;         /* splitters (kind 1) */
  int32_t where;          /* 0 = grid-wide pass, 1 = block-resident pass */
  int64_t counts[256];    /* keys per bucket */
} iplsTraceRec;

typedef struct iplsStats {
  int64_t calls;              /* sort calls since the context was created */
  int64_t grid_levels;        /* grid-wide partition levels in the last call */
  int64_t grid_passes;        /* grid-wide partition passes in the last call */
  int64_t keys_partitioned;   /* keys moved by grid-wide passes, last call */
  int64_t resident_groups;    /* block-resident groups, last call */
  int64_t fallback_passes;    /* splitter-tree passes, last call */
  int64_t algorithmic_bytes;  /* 2*w*(keys moved) over all passes, last call */
  int64_t scratch_bytes;      /* device scratch held by the context */
  int64_t trace_records;      /* passes recorded (may exceed trace_cap) */
  double max_bucket_frac;     /* largest bucket / subproblem size, grid passes */
  int64_t slow_tasks;         /* ranges recursed inside one block (slow lists), last call */
  int64_t slow_passes;        /* partition passes run by that in-block recursion, last call */
  int64_t sweep_tasks;        /* children above the cutoff taken by a second block-resident
                                 sweep (fit + pass + base case) instead, last call */
} iplsStats;

/* One batch of served requests (iplsGetBatchLog).  start_ms / end_ms are
 * CUDA-event times of the batch's work on its slot's stream, in ms after a
 * reference event recorded when the serving slots started (-1 if unknown). */
typedef struct iplsBatchRec {
  uint64_t first_ticket;  /* ticket of the batch's oldest request */
  int32_t requests;       /* requests in the batch */
  int32_t slot;           /* in-flight slot (worker and stream) that ran it */
  int64_t keys;           /* keys of all its requests */
  int32_t dtype;
  int32_t status;         /* the batch's iplsStatus */
  double start_ms;
  double end_ms;
} iplsBatchRec;

typedef struct iplsContext* iplsCtx;
typedef void* (*iplsAllocFn)(size_t bytes, void* user);  /* device memory */
typedef void (*iplsFreeFn)(void* ptr, void* user);

/* Fills *cfg with the defaults (k=256, cutoff=32, formula sample, seed 0,
 * sync=1, spin_limit=2^26).  IPLS_ERR_ARG if cfg is NULL. */
iplsStatus iplsDefaultConfig(iplsConfig* cfg);

/* Creates a context on the current CUDA device.  cfg NULL = defaults.
 * alloc/free NULL = cudaMalloc/cudaFree; otherwise every device allocation
 * goes through them with `user` passed back.  stream = cudaStream_t (NULL =
 * the legacy default stream).  The context is not thread-safe. */
iplsStatus iplsCreate(iplsCtx* ctx, const iplsConfig* cfg, iplsAllocFn alloc,
                      iplsFreeFn free_fn, void* user, void* stream);

/* Waits for the context's stream, releases all scratch, frees the context. */
iplsStatus iplsDestroy(iplsCtx ctx);

/* Device scratch bytes a sort of n keys of `dtype` needs (upper bound). */
iplsStatus iplsScratchBytes(iplsCtx ctx, int64_t n, iplsDtype dtype, size_t* bytes);

/* Sorts keys[0..n) in place (device pointer).  ctx NULL = a per-thread
 * default context on the current device with default configuration.
 * The whole IPLS recursion of the paper (Ch.2 IPS4o framework, Ch.3 FMCD
 * model, Ch.4 IPLS parameters) runs on the device. */
iplsStatus iplsSort(iplsCtx ctx, void* keys, int64_t n, iplsDtype dtype);

/* Sorts nseg independent segments keys[offsets[i]..offsets[i+1]) in place.
 * offsets is a DEVICE array of nseg+1 non-decreasing int64 values with
 * offsets[0] >= 0; nseg = 0 is a no-op.  Each segment is a level-0
 * subproblem of its own (its sample stream is keyed by its offset), so a
 * segment sorts to the same bytes alone or in the batch. */
iplsStatus iplsSortSegmented(iplsCtx ctx, void* keys, const int64_t* offsets,
                             int64_t nseg, iplsDtype dtype);

/* Sorts keys[0..n) that live in HOST memory: copies them to a
 * context-owned device buffer, sorts them there with iplsSort's kernels and
 * copies the result back into the same host array.  Pinned (page-locked)
 * host memory gives full copy bandwidth; pageable memory works too. */
iplsStatus iplsSortHost(iplsCtx ctx, void* host_keys, int64_t n, iplsDtype dtype);

/* Sorts `count` separate HOST arrays host_keys[i][0..n[i]) in place, one
 * after another, with the copies overlapped: while array i is sorted on the
 * device, array i+1 is copied in and array i-1 copied out, on two copy
 * streams of the context, through three context-owned device buffers of the
 * largest n[i] keys each.  host_keys and n are host arrays of count
 * entries; the arrays must not overlap.  Each array ends up exactly as
 * iplsSortHost leaves it.  The copies overlap only for pinned (page-locked)
 * host memory; pageable memory gives the same result without overlap.  The
 * call returns when every array is back in host memory; on an error the
 * arrays not yet copied back keep their input. */
iplsStatus iplsSortHostBatch(iplsCtx ctx, void* const* host_keys, const int64_t* n, int64_t count,
                             iplsDtype dtype);

/* Sorts `count` separate device arrays keys[i][0..n[i]) in place (keys and
 * n are HOST arrays of count entries; each keys[i] is a device pointer
 * aligned to the key width).  All arrays are sorted together: each is a
 * level-0 subproblem of its own, addressed in its own memory (nothing is
 * gathered or copied), and every partition pass of every array shares the
 * same kernel launches.  Each array ends up sorted exactly as iplsSort
 * alone would sort it.  The sum of the sizes must not exceed 2^32 - 1.
 * The arrays must not overlap. */
iplsStatus iplsSortBatch(iplsCtx ctx, void* const* keys, const int64_t* n, int64_t count,
                         iplsDtype dtype);

/* Asynchronous sort request for keys[0..n) (device memory, already
 * written): queues it and returns a ticket at once.  The context serves
 * requests with cfg.serve_slots in-flight slots (two by default), each a
 * worker thread with its own
 * stream and scratch: a free slot takes the oldest queued request's dtype
 * and, in arrival order, further queued requests of that dtype while the
 * bytes of all requests in flight, 2*w*n each, stay within cfg.budget_bytes
 * (0 = unlimited) and the batch within cfg.max_batch, and sorts them with one
 * batched sort in place (as iplsSortBatch).  While one slot's batch runs the
 * other admits the next, so requests that arrive meanwhile are served as
 * memory frees up and their work overlaps on the GPU; batches of different
 * dtypes may run side by side.  The result is the same sorted array whatever
 * the batch.  Returns IPLS_ERR_BUDGET if one request alone exceeds the
 * budget.  `keys` must stay alive and untouched until the request completes.
 * The slots' streams are created by the library; work submitted through the
 * context's own stream is not ordered with them.  Allocator callbacks given
 * to iplsCreate are also called from the slots' worker threads. */
iplsStatus iplsSubmit(iplsCtx ctx, void* keys, int64_t n, iplsDtype dtype,
                      uint64_t* ticket);

/* IPLS_PENDING while the request is queued or running, then its final
 * status (IPLS_ERR_ARG for an unknown ticket). */
iplsStatus iplsPoll(iplsCtx ctx, uint64_t ticket);

/* Waits up to timeout_us microseconds (< 0 = forever) for a request; returns
 * its final status, or IPLS_PENDING if it is still running. */
iplsStatus iplsWait(iplsCtx ctx, uint64_t ticket, int64_t timeout_us);

/* Copies up to cap records of the batches served so far (oldest first, at
 * most 65536 kept) to host memory and sets *count. */
iplsStatus iplsGetBatchLog(iplsCtx ctx, iplsBatchRec* out, int64_t cap, int64_t* count);

/* Statistics of the context (synchronises its stream). */
iplsStatus iplsGetStats(iplsCtx ctx, iplsStats* stats);

/* Per-kernel device time and algorithmic bytes accumulated while
 * cfg.profile = 1 (synchronises the stream).  Writes up to cap entries and
 * sets *count; reset = 1 clears the accumulators after reading. */
iplsStatus iplsGetKernelStats(iplsCtx ctx, iplsKernelStat* out, int32_t cap, int32_t* count,
                              int32_t reset);

/* Per-level grid-pass time and bytes accumulated while cfg.profile = 1
 * (synchronises the stream).  Writes up to cap entries, one per level that
 * ran grid passes, and sets *count; reset = 1 clears the accumulators. */
iplsStatus iplsGetLevelStats(iplsCtx ctx, iplsLevelStat* out, int32_t cap, int32_t* count,
                             int32_t reset);

/* Copies up to cap trace records of the last sort to host memory `out`
 * (requires cfg.trace_cap > 0) and sets *count to the records kept. */
iplsStatus iplsGetTrace(iplsCtx ctx, iplsTraceRec* out, int64_t cap, int64_t* count);

/* Sorts keys[0..n) in place (device pointer) WITHOUT allocating any memory:
 * no cudaMalloc/cudaFree, no allocator callback, no context.  The paper has
 * no counterpart; it exists for callers that cannot allocate when they sort
 * (a framework pool holding the device's memory, a latency-critical loop in
 * which cudaMalloc/cudaFree could synchronise the device, a pipeline that
 * must not fail for lack of memory half-way).
 *   - n <= 8192 (resident_rmax: 8192 for cfg->cutoff >= 7, 1024*(cutoff+1)
 *     below); a larger n returns IPLS_ERR_ARG with a message naming the
 *     limit, before any CUDA call.  One block sorts the keys; the result
 *     equals iplsSort's on the same keys and configuration.
 *   - cfg NULL = iplsDefaultConfig; k, cutoff, root_sample (<= 1024), seed
 *     and exact_only are used.  stream = cudaStream_t (NULL = legacy
 *     default stream).
 *   - The call synchronises its stream (it copies the device status back
 *     and waits for it), so it cannot be made while that stream is being
 *     captured into a CUDA graph.
 *   - Its only device scratch is a 256-byte status block in a file-scope
 *     __device__ array of the library, cleared on the stream at the start
 *     of every call.  The first call on each device looks up that array's
 *     address (cudaGetSymbolAddress, with the device current).
 *   - The status block is shared by every call on a device: calls that
 *     overlap in time (other threads or streams) race on it and must be
 *     serialised by the caller. */
iplsStatus iplsSortSmallNoAlloc(void* keys, int64_t n, iplsDtype dtype, const iplsConfig* cfg,
                                void* stream);

/* Copies the PL2 knot values of the grid-level pass records of the last sort
 * (the records iplsGetTrace lists first, in the same order) to host memory:
 * (cfg.pl2_leaves + 1) binary32 values y_0..y_M per record, zeros for a pass
 * whose model is not PL2.  Requires cfg.trace_cap > 0 and cfg.pl2_leaves > 0
 * (otherwise *count = 0); knots are kept for at most the first 16384 grid
 * records.  out holds cap records; *count is set to the records written.
 * (PL2: Ch.2 "Learned Sort" and Ch.3 "Recursive Model Index", a learned
 * CDF fitted to the sample's empirical CDF.) */
iplsStatus iplsGetTraceKnots(iplsCtx ctx, float* out, int64_t cap, int64_t* count);

/* The PL2 model's training loss and gradient, computed on the device by the
 * same forward and backward functions that train PL2 inside the sort (Ch.3:
 * the mean squared error of a learned CDF against the empirical CDF).
 *   sample: DEVICE array of S keys of `dtype`, ascending in totalOrder
 *           (2 <= S <= 4096), the sample the model is fitted on;
 *   leaves: M, a power of two in [2, 1024];
 *   knots:  DEVICE array of M + 1 binary32 knot values y_0..y_M;
 *   out:    DEVICE array of 2(M + 1) + 2 floats, written on `stream`
 *           (cudaStream_t, NULL = legacy default stream; the call returns
 *           after enqueueing): out[j] = G_j = sum_i r_i dF(x_i)/dy_j and
 *           out[M+1+j] = H_j = sum_i (dF(x_i)/dy_j)^2 for j = 0..M, with
 *           F the model's CDF at sample i and r_i = F(x_i) - (i + 1/2)/S;
 *           the loss gradient is 2 G_j / S.  out[2M+2] = the loss
 *           (1/S) sum r_i^2 and out[2M+3] = 1, or all zeros when the
 *           sample's range cannot carry PL2 (equal or non-finite extremes).
 * Binary32 throughout, sums over each leaf in sample order.  Allocates
 * nothing.  IPLS_ERR_ARG for an out-of-range S, leaves or dtype, or a NULL
 * pointer; IPLS_ERR_CUDA if the launch fails. */
iplsStatus iplsPL2LossGrad(const void* sample, int64_t S, iplsDtype dtype, int32_t leaves,
                           const float* knots, float* out, void* stream);

/* Message of the last failure on this thread ("" if none). */
const char* iplsLastError(void);

#ifdef __cplusplus
}  /* extern "C" */
#endif

#endif  /* IPLS_H_ */
