// Block-resident tail of the IPLS recursion (Ch.2 IPS4o recursion into
// independent buckets; Ch.4 IPLS), for subproblems of at most kResidentMax
// keys.
//
//   k_tail_fit   persistent warps, one subproblem at a time: sample
//                alpha*k-1 keys, sort them (warp radix sort on the digits the
//                sample's keys set), fit FMCD -- many fits in flight per SM
//                hide the latency of the sort and of the binary64 steps.
//   k_tail       one block per task, in two sizes: 256 threads (four blocks
//                per SM) for tasks of up to kTailSmall keys, 512 threads for
//                larger ones.  A fitted subproblem is read from HBM
//                once, classified with its model, ranked stably per bucket
//                and placed into shared memory in bucket order; each bucket
//                of at most `cutoff` keys is then base-cased by rank counting
//                (the position of a key inside its bucket is the number of
//                smaller keys, ties broken by position), and the subproblem
//                is written to the user buffer once.  A task of small children
//                (consecutive buckets or segments of at most `cutoff` keys)
//                goes straight to the base case.  Buckets above the cutoff
//                are written out in place and queued on the child list;
//                tasks without progress, or whose splitter tree found no
//                pool slot, on the whole-task list.
//   (2nd sweep)  when many children were queued, k_tail_fit and k_tail run
//                once more over them, in place in the user buffer; what
//                they queue in turn is left to k_slow.
//   k_slow       persistent blocks drain both lists: each range recurses
//                inside one block (sample, sort, fit, classify, stable
//                scatter, base case) and is written back in place.
//
// The paper's base case is SkaSort for n <= 2^12 (Ch.4); any exact sort
// gives the same, unique result.
#include <algorithm>

#include "ipls_device.cuh"

namespace ipls {

constexpr int kRW = kResidentThreads / 32;  // warps
constexpr int kRKPT = kResidentMax / kResidentThreads;
constexpr int kFitWarps = 8;
// k_tail_fit: sample sort by warp radix sort up to this many keys (every
// tail task: n <= 8192 gives at most 664), bitonic network above
constexpr int kRadixSteps = 22;
constexpr int kRadixMax = 32 * kRadixSteps;
// Per warp: the sample (kRadixMax keys), then kRadixMax 8-byte words that
// hold first the radix sort's second buffer and then the sample's
// fixed-point images.  A bitonic-sorted sample (up to kResidentSample keys)
// uses the whole slot.
template <class Ord>
__host__ __device__ constexpr size_t fit_slot_bytes() { return (size_t)kRadixMax * sizeof(Ord) + (size_t)kRadixMax * 8; }
static_assert(fit_slot_bytes<unsigned int>() >= kResidentSample * 4, "slot must hold the largest sample");
static_assert(fit_slot_bytes<unsigned long long>() >= kResidentSample * 8, "slot must hold the largest sample");

// ---------------------------------------------------------------------------
// k_tail_fit
// ---------------------------------------------------------------------------
template <class K>
__global__ void __launch_bounds__(kFitWarps * 32) k_tail_fit(ResidentArgs a) {
  using T = KT<K>;
  using Ord = typename T::Ord;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ FitShared fs[kFitWarps];
  __shared__ TailModel tm[kFitWarps];
  __shared__ unsigned rcnt[kFitWarps][256], rpeer[kFitWarps][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nfit = tail_nfit(a);
  for (int i = lane; i < 256; i += 32) rpeer[warp][i] = 0u;
  unsigned char* slot = smem_raw + (size_t)warp * fit_slot_bytes<Ord>();
  Ord* so = reinterpret_cast<Ord*>(slot);
  Ord* rtmp = reinterpret_cast<Ord*>(slot + (size_t)kRadixMax * sizeof(Ord));
  long long* qimg = reinterpret_cast<long long*>(slot + (size_t)kRadixMax * sizeof(Ord));
  // persistent warps: each takes the next task until none is left
  for (;;) {
    int task = 0;
    if (lane == 0) task = atomicAdd(&a.slow_ctl->fit_ticket, 1);
    task = __shfl_sync(0xffffffffu, task, 0);
    if (task >= nfit) break;
    const Group g = a.groups[a.fit_list[task]];
    int S = (int)sample_size(g.n, g.level, a.k, a.root_sample);
    if (S > kResidentSample) S = kResidentSample;  // never planned by the host
    const uint64_t stream = stream_key(a.seed, g.off, g.n, g.level);
    const typename T::Bits* src = keys_of<const typename T::Bits>(g.buf, g.ubase, a.buf) + g.off;
    for (int j = lane; j < S; j += 32) so[j] = T::ord(src[sample_offset(stream, j, g.n)]);
    __syncwarp();
    if (S <= kRadixMax) warp_radix_sort<kRadixSteps>(so, rtmp, rcnt[warp], rpeer[warp], S);
    else group_sort<WarpG, Ord>(so, S);
    TailModel& m = tm[warp];
    // after the radix sort its second buffer holds the fixed-point images
    fit_linear<WarpG, K>(so, S, a.k, &m.l, fs[warp], S <= kRadixMax ? qimg : nullptr);
    if (lane == 0) {
      m.nsplit = 0;
      m.pool = -1;
    }
    __syncwarp();
    if (m.l.kind == kSplitter) {
      // splitter tree from the same sorted sample: (k-1)/2 equidistant sample
      // keys, duplicates dropped (Ch.3 "Decision Trees"; equality buckets).
      // First count them, then store them inline or in a pool slot.
      const int want = (a.k - 1) / 2;
      int cnt = 0;
      for (int base = 0; base < want; base += 32) {
        const int i = base + lane;
        const bool keep = i < want && (i == 0 || so[(int64_t)(i + 1) * S / (want + 1)] !=
                                                     so[(int64_t)i * S / (want + 1)]);
        cnt += __popc(__ballot_sync(0xffffffffu, keep));
      }
      int slot = -1;
      if (cnt > kTailSplit && lane == 0) {
        slot = atomicAdd(&a.slow_ctl->pool_used, 1);
        if (slot >= a.split_pool_slots) slot = -1;
      }
      slot = __shfl_sync(0xffffffffu, slot, 0);
      uint64_t* out = cnt <= kTailSplit ? m.split : (slot >= 0 ? a.split_pool + (size_t)slot * 128 : nullptr);
      if (out) {
        int pos0 = 0;
        for (int base = 0; base < want; base += 32) {
          const int i = base + lane;
          bool keep = false;
          uint64_t u = 0;
          if (i < want) {
            u = (uint64_t)so[(int64_t)(i + 1) * S / (want + 1)];
            keep = (i == 0) || (u != (uint64_t)so[(int64_t)i * S / (want + 1)]);
          }
          const unsigned bal = __ballot_sync(0xffffffffu, keep);
          if (keep) out[pos0 + __popc(bal & lanemask_lt())] = u;
          pos0 += __popc(bal);
        }
      }
      if (lane == 0) {
        m.nsplit = cnt;
        m.pool = slot;
        m.l.nb = 2 * cnt + 1;
        m.l.fast = 0;
      }
      __syncwarp();
    }
    const unsigned long long* s = reinterpret_cast<const unsigned long long*>(&m);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(&a.tail_models[g.fit]);
    if (lane < (int)(sizeof(TailModel) / 8)) d[lane] = s[lane];
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// In-block recursion (the slow path)
// ---------------------------------------------------------------------------
template <class K>
struct ResSmem {
  typename KT<K>::Ord keys[kResidentMax];
  union {
    struct {
      typename KT<K>::Ord samp[kResidentSample];
      unsigned short wcnt[kRW][kMaxK];
      unsigned long long tasks[kResidentTasks];  // small list from 0 up, stack from the top
    } s;
  } u;
  int bstart[kMaxK + 1];
  int tot[kMaxK];
  int hom[kMaxK];
  Model model;
  FitShared fs;
  int nsmall, nstack, redo, err, slow_all;
  unsigned long long popped;
  long long rec;
};

__device__ __forceinline__ unsigned long long enc_task(int start, int len, int level) {
  return ((unsigned long long)(unsigned)level << 32) | ((unsigned long long)start << 16) | (unsigned)len;
}
__device__ __forceinline__ int task_start(unsigned long long e) { return (int)((e >> 16) & 0xFFFF); }
__device__ __forceinline__ int task_len(unsigned long long e) { return (int)(e & 0xFFFF); }
__device__ __forceinline__ int task_level(unsigned long long e) { return (int)(e >> 32); }

// Writes one trace record for a pass (thread 0 writes the header).
template <class K>
__device__ void trace_pass(ResSmem<K>& sh, const ResidentArgs& a, int64_t off, int n, int level,
                           const Model& m) {
  if (a.trace_cap <= 0) return;
  if (threadIdx.x == 0) {
    sh.rec = (long long)atomicAdd((unsigned long long*)&a.run->trace_count, 1ULL);
    if (sh.rec < a.trace_cap) {
      iplsTraceRecDev& r = a.trace[sh.rec];
      r.off = off; r.n = n; r.level = level; r.kind = m.l.kind; r.capped = m.l.capped;
      r.nbuckets = m.l.nb; r.S = m.l.S; r.D = m.l.D; r.A = m.l.A; r.Bc = m.l.Bc; r.ud = m.l.ud;
      r.xlo_bits = m.l.xlo_bits; r.nsplit = m.nsplit; r.where = 1;
    }
  }
  __syncthreads();
  if (sh.rec < a.trace_cap && threadIdx.x < kMaxK)
    a.trace[sh.rec].counts[threadIdx.x] = (threadIdx.x < m.l.nb) ? sh.tot[threadIdx.x] : 0;
  __syncthreads();
}

// For every bucket b with more than `cutoff` keys (stored contiguously from
// keys[start[b]]), hom[b] = 1 when all of them are the same key (compared
// after a right shift by `shift`, which drops the position bits of packed
// words).  Such a
// bucket is done: its own pass would draw a homogeneous sample, take the
// splitter tree with that one key as its only splitter and put every key
// into the equality bucket, moving nothing (the rule for duplicates).
template <class Ord>
__device__ void mark_homogeneous(const Ord* keys, const int* start, const int* tot, int nb,
                                 int cutoff, int* hom, int shift = 0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) hom[b] = tot[b] > cutoff ? 1 : 0;
  __syncthreads();
  for (int b = warp; b < nb; b += blockDim.x >> 5) {
    if (!hom[b]) continue;
    const Ord first = keys[start[b]] >> shift;
    bool diff = false;
    for (int i = start[b] + lane; i < start[b] + tot[b]; i += 32) diff |= (keys[i] >> shift) != first;
    if (__any_sync(0xffffffffu, diff) && lane == 0) hom[b] = 0;
  }
  __syncthreads();
}

// The pass record of such a homogeneous subproblem (one thread): splitter
// tree with one splitter, every key in its equality bucket.
__device__ void record_homogeneous(const ResidentArgs& a, int64_t off, int n, int level) {
  atomicAdd((unsigned long long*)&a.run->resident_passes, 1ULL);
  atomicAdd((unsigned long long*)&a.run->resident_fallback, 1ULL);
  if (a.trace_cap <= 0) return;
  const long long rec = (long long)atomicAdd((unsigned long long*)&a.run->trace_count, 1ULL);
  if (rec >= a.trace_cap) return;
  iplsTraceRecDev& r = a.trace[rec];
  r.off = off; r.n = n; r.level = level; r.kind = kSplitter; r.capped = 0; r.nbuckets = 3;
  r.S = sample_size(n, level, a.k, a.root_sample); r.D = 0; r.A = 0.0; r.Bc = 0.0; r.ud = 0.0;
  r.xlo_bits = 0; r.nsplit = 1; r.where = 1;
  for (int b = 0; b < kMaxK; ++b) r.counts[b] = (b == 1) ? n : 0;
}

// Exclusive scan of sh.tot into sh.bstart (one warp, 8 values per lane).
template <class K>
__device__ __forceinline__ void scan_totals(ResSmem<K>& sh) {
  if ((threadIdx.x >> 5) == 0) {
    const int lane = threadIdx.x & 31;
    int loc[8];
    int sum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) { loc[q] = sh.tot[lane * 8 + q]; sum += loc[q]; }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += x;
    }
    int run = incl - sum;
#pragma unroll
    for (int q = 0; q < 8; ++q) { sh.bstart[lane * 8 + q] = run; run += loc[q]; }
    if (lane == 31) sh.bstart[kMaxK] = run;
  }
  __syncthreads();
}

// Totals per bucket from the per-warp counters (into sh.tot); turns wcnt
// into per-warp exclusive offsets.
template <class K>
__device__ __forceinline__ void warp_counts_to_offsets(ResSmem<K>& sh) {
  if (threadIdx.x < kMaxK) {
    const int b = threadIdx.x;
    int run = 0;
    for (int w = 0; w < kRW; ++w) {
      const int x = sh.u.s.wcnt[w][b];
      sh.u.s.wcnt[w][b] = (unsigned short)run;
      run += x;
    }
    sh.tot[b] = run;
  }
  __syncthreads();
}

// Base-cases every pending small range of the slow path (warp bitonic up to
// 32 keys in registers, above that one warp's bitonic network in shared
// memory per range).
template <class K>
__device__ void flush_small(ResSmem<K>& sh) {
  using Ord = typename KT<K>::Ord;
  __syncthreads();
  const int ns = sh.nsmall;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = warp; q < ns; q += kRW) {
    const unsigned long long e = sh.u.s.tasks[q];
    const int st = task_start(e), len = task_len(e);
    if (len > 32) continue;
    Ord v = (lane < len) ? sh.keys[st + lane] : (Ord)~(Ord)0;
    v = warp_sort32(v);
    if (lane < len) sh.keys[st + lane] = v;
  }
  // larger ranges (up to the cutoff): one warp each, many at a time
  for (int q = warp; q < ns; q += kRW) {
    const unsigned long long e = sh.u.s.tasks[q];
    if (task_len(e) > 32) group_sort<WarpG>(sh.keys + task_start(e), task_len(e));
  }
  __syncthreads();
  if (threadIdx.x == 0) sh.nsmall = 0;
  __syncthreads();
}

template <class K>
__device__ __forceinline__ void push_child(ResSmem<K>& sh, int start, int len, int level, int cutoff) {
  if (len < 2) return;
  if (len <= cutoff) {
    const int i = atomicAdd(&sh.nsmall, 1);
    if (i < kResidentTasks / 2) sh.u.s.tasks[i] = enc_task(start, len, level);
    else sh.err = 1;
  } else {
    const int i = atomicAdd(&sh.nstack, 1);
    if (i < kResidentTasks / 2) sh.u.s.tasks[kResidentTasks - 1 - i] = enc_task(start, len, level);
    else sh.err = 1;
  }
}

// Slow path: one learned partition pass on keys[s0, s0+c) inside shared
// memory, fitting the model in the block (sample, sort, FMCD or splitter
// tree, no-progress rule), then queueing the children.
template <class K>
__device__ void resident_pass(ResSmem<K>& sh, const ResidentArgs& a, int64_t goff, int s0, int c,
                              int level) {
  using T = KT<K>;
  using Ord = typename T::Ord;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int S = (int)sample_size(c, level, a.k, a.root_sample);
  if (S > kResidentSample) {  // never planned by the host; keep the block in bounds
    if (threadIdx.x == 0) sh.err = 1;
    S = kResidentSample;
  }
  const uint64_t stream = stream_key(a.seed, goff + s0, c, level);
  for (int j = threadIdx.x; j < S; j += blockDim.x) sh.u.s.samp[j] = sh.keys[s0 + sample_offset(stream, j, c)];
  __syncthreads();
  block_sort(sh.u.s.samp, S);
  fit_model<BlockG, K>(sh.u.s.samp, S, a.k, &sh.model, sh.fs);
  const int chunk = ((c + kRW * 32 - 1) / (kRW * 32)) * 32;
  const int steps = chunk / 32;
  Ord v[kRKPT];
  unsigned int br[kRKPT];
  for (int attempt = 0; attempt < 2; ++attempt) {
    Classifier<K> cls;
    cls.load(sh.model, a.exact_only);
    for (int i = threadIdx.x; i < kRW * kMaxK; i += blockDim.x) (&sh.u.s.wcnt[0][0])[i] = 0;
    if (threadIdx.x == 0) sh.redo = 0;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRKPT; ++j) {
      if (j < steps) {
        const int i = warp * chunk + j * 32 + lane;
        const bool ok = i < c;
        v[j] = ok ? sh.keys[s0 + i] : (Ord)0;
        const int bk = ok ? cls.bucket(T::unord(v[j])) : kMaxK;
        const unsigned peers = same_bucket_lanes(bk, bk < kMaxK);
        const int lt = __popc(peers & lanemask_lt());
        const int leader = __ffs(peers) - 1;
        const int basec = (bk < kMaxK) ? sh.u.s.wcnt[warp][bk] : 0;
        br[j] = ((unsigned)bk << 16) | (unsigned)(basec + lt);
        __syncwarp();
        if (lane == leader && bk < kMaxK) sh.u.s.wcnt[warp][bk] = (unsigned short)(basec + __popc(peers));
        __syncwarp();
      }
    }
    __syncthreads();
    warp_counts_to_offsets(sh);
    if (threadIdx.x < kMaxK && attempt == 0 && sh.model.l.kind == kLinear && sh.tot[threadIdx.x] == c)
      sh.redo = 1;
    __syncthreads();
    if (!sh.redo) break;
    // no progress: redo the pass with the splitter tree of the same sample
    build_splitters<BlockG, K>(sh.u.s.samp, S, a.k, &sh.model);
  }
  scan_totals(sh);
#pragma unroll
  for (int j = 0; j < kRKPT; ++j) {
    if (j < steps) {
      const int bk = (int)(br[j] >> 16);
      if (bk < kMaxK) sh.keys[s0 + sh.bstart[bk] + sh.u.s.wcnt[warp][bk] + (int)(br[j] & 0xFFFF)] = v[j];
    }
  }
  __syncthreads();
  const Model& m = sh.model;
  trace_pass(sh, a, goff + s0, c, level, m);
  if (threadIdx.x == 0) {
    atomicAdd((unsigned long long*)&a.run->resident_passes, 1ULL);
    atomicAdd((unsigned long long*)&a.run->slow_passes, 1ULL);
    if (m.l.kind == kSplitter) atomicAdd((unsigned long long*)&a.run->resident_fallback, 1ULL);
  }
  // children (equality buckets of the splitter tree are homogeneous: done;
  // so is any other child whose keys are all equal, after its record)
  mark_homogeneous(sh.keys + s0, sh.bstart, sh.tot, m.l.nb, a.cutoff, sh.hom);
  if (threadIdx.x < m.l.nb) {
    const int b = threadIdx.x;
    const bool eq = (m.l.kind == kSplitter) && (b & 1);
    if (!eq) {
      if (sh.hom[b]) record_homogeneous(a, goff + s0 + sh.bstart[b], sh.tot[b], level + 1);
      else push_child(sh, s0 + sh.bstart[b], sh.tot[b], level + 1, a.cutoff);
    }
  }
  __syncthreads();
}

// Runs the slow-path stack to completion (all threads).
template <class K>
__device__ void run_stack(ResSmem<K>& sh, const ResidentArgs& a, int64_t goff) {
  for (;;) {
    __syncthreads();
    if (sh.nstack == 0 || sh.err) break;
    if (sh.nsmall + kMaxK > kResidentTasks / 2) flush_small(sh);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int i = --sh.nstack;
      sh.popped = sh.u.s.tasks[kResidentTasks - 1 - i];
    }
    __syncthreads();
    const unsigned long long e = sh.popped;
    if (task_level(e) > 4096) {
      if (threadIdx.x == 0) { atomicExch(&a.run->error, -6); sh.nstack = 0; }
      continue;
    }
    resident_pass<K>(sh, a, goff, task_start(e), task_len(e), task_level(e));
  }
  if (sh.err) {
    if (threadIdx.x == 0) { atomicExch(&a.run->error, -6); sh.nsmall = 0; }
    __syncthreads();
  }
  flush_small(sh);
}

template <class K>
__global__ void __launch_bounds__(kResidentThreads, 2) k_slow(ResidentArgs a) {
  using T = KT<K>;
  using Bits = typename T::Bits;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ResSmem<K>& sh = *reinterpret_cast<ResSmem<K>*>(smem_raw);
  __shared__ int s_i;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_i = (int)atomicAdd(&a.slow_ctl->ticket, 1u);
    __syncthreads();
    // the whole tasks first, then the children
    const int i = s_i;
    const int nw = min(a.slow_ctl->wcount, a.whole_cap);
    const int nc = min(a.slow_ctl->count, a.slow_cap);
    if (i >= nw + nc) break;
    const SlowTask st = i < nw ? a.whole[i] : a.slow[i - nw];
    if (threadIdx.x == 0) atomicAdd((unsigned long long*)&a.run->slow_tasks, 1ULL);
    Bits* src = reinterpret_cast<Bits*>(st.ubase) + st.off;
    for (int p = threadIdx.x; p < st.n; p += blockDim.x) sh.keys[p] = T::ord(src[p]);
    if (threadIdx.x == 0) {
      sh.nsmall = 0;
      sh.err = 0;
      sh.nstack = 1;
      sh.u.s.tasks[kResidentTasks - 1] = enc_task(0, st.n, st.level);
    }
    __syncthreads();
    run_stack<K>(sh, a, st.off);
    for (int p = threadIdx.x; p < st.n; p += blockDim.x) src[p] = T::unord(sh.keys[p]);
  }
}

// ---------------------------------------------------------------------------
// k_tail
// ---------------------------------------------------------------------------
template <class K, int kCap, int kW>
struct TailSmem {
  typename KT<K>::Ord keys[kCap];
  // segment of each position: a bucket or child, or (large tasks) a bucket
  // eighth (bucket * 8 + refinement)
  typename std::conditional<kCap == kResidentMax, unsigned short, unsigned char>::type seg[kCap];
  unsigned short wcnt[kW][kMaxK];   // each warp's offset inside every bucket (stable placement)
  unsigned int peer[kW][kMaxK];     // per-warp bucket counts, then placement cursors (or, for
                                    // stable placement, lanes of the current step per bucket)
  int bstart[kMaxK + 1];
  int segb[kMaxK + 1];
  int tot[kMaxK];
  int hom[kMaxK];
  TailModel tm;
  uint64_t split[128];   // a tree too large for the record, from the pool
  typename KT<K>::Ord seglo[kMaxK];  // smallest key of each base-cased segment
  unsigned char segpk[kMaxK];        // 1: the segment is ranked on packed words
  typename KT<K>::Ord wlo[kW], whi[kW];    // per-warp key range of a fitted task
  typename KT<K>::Ord tlo;           // smallest key of a fitted task
  int tpk;                           // 1: the fitted task's keys are placed packed
  int slow_all;
  int any_big;   // some bucket above the cutoff would be queued
  int any_mid;   // some bucket (bit 0) or eighth (bit 1) of kSameMin+1 .. cutoff keys
  long long rec;
};
// two (four) blocks per SM, each with its 1 KB of reserved shared memory
static_assert(2 * (sizeof(TailSmem<double, kResidentMax, kRW>) + 1024) <= 233472,
              "the large k_tail must keep two blocks per SM");
static_assert(4 * (sizeof(TailSmem<double, kTailSmall, kRW / 2>) + 1024) <= 233472,
              "the small k_tail must keep four blocks per SM");

// A child above the cutoff (it may take another tail round).
__device__ __forceinline__ void push_slow(const ResidentArgs& a, int64_t off, int n, int level,
                                          uint64_t ubase) {
  const int i = atomicAdd(&a.slow_ctl->count, 1);
  if (i < a.slow_cap) a.slow[i] = SlowTask{off, n, level, ubase};
  else atomicExch(&a.run->error, -6);
}

// A whole task that recurses inside one block (k_slow).
__device__ __forceinline__ void push_whole(const ResidentArgs& a, int64_t off, int n, int level,
                                           uint64_t ubase) {
  const int i = atomicAdd(&a.slow_ctl->wcount, 1);
  if (i < a.whole_cap) a.whole[i] = SlowTask{off, n, level, ubase};
  else atomicExch(&a.run->error, -6);
}

// Base case on packed words: a key whose group of keys spans fewer than
// 2^(bits - kPosBits) values is held as (key - min) << kPosBits | position,
// and one unsigned compare of two words gives their (key, position) order.
constexpr int kPosBits = 13;
static_assert(kResidentMax <= (1 << kPosBits), "positions must fit the packed word");

// Large tail tasks cut their buckets into eighths only when the keys fill
// at least this many buckets.
constexpr int kFineMinBuckets = 64;

// Base case: a segment of more than this many keys is first checked for
// copies of one key, which keep their places (any order of equal keys gives
// the same bytes); ranking them by counting would cost the square of the
// segment's size.  The mark is bit 31 of the segment's start (starts are
// below 2^13), so that the base case reads it with the bounds.
constexpr int kSameMin = 32;
constexpr unsigned kSameBit = 0x80000000u;
constexpr unsigned kStartMask = 0x7FFFFFFFu;

// Number of words in keys[s, e) below kp (the rank of a packed word in its
// segment; packed words are distinct).  Two (8-byte) or four (4-byte)
// words per shared-memory load; the array is 16-byte aligned.
template <class Ord>
__device__ __forceinline__ int count_below(const Ord* keys, int s, int e, Ord kp) {
  int cnt = 0;
  int r = s;
  if (sizeof(Ord) == 8) {
    if ((r & 1) && r < e) cnt += keys[r++] < kp ? 1 : 0;
#pragma unroll 2
    for (; r + 2 <= e; r += 2) {
      const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(keys + r);
      cnt += ((Ord)w.x < kp ? 1 : 0) + ((Ord)w.y < kp ? 1 : 0);
    }
  } else {
    for (; (r & 3) && r < e; ++r) cnt += keys[r] < kp ? 1 : 0;
#pragma unroll 2
    for (; r + 4 <= e; r += 4) {
      const uint4 w = *reinterpret_cast<const uint4*>(keys + r);
      cnt += ((Ord)w.x < kp ? 1 : 0) + ((Ord)w.y < kp ? 1 : 0) + ((Ord)w.z < kp ? 1 : 0) + ((Ord)w.w < kp ? 1 : 0);
    }
  }
  for (; r < e; ++r) cnt += keys[r] < kp ? 1 : 0;
  return cnt;
}

// 1 when keys[s, e) hold two different keys (compared after a right shift
// by `shift`, which drops the position bits of packed words).  Stops at the
// first difference.
template <class Ord>
__device__ __forceinline__ int differs(const Ord* keys, int s, int e, int shift) {
  const Ord k0 = keys[s];
  int r = s + 1;
  for (; r + 4 <= e; r += 4)
    if (((keys[r] ^ k0) | (keys[r + 1] ^ k0) | (keys[r + 2] ^ k0) | (keys[r + 3] ^ k0)) >> shift) return 1;
  for (; r < e; ++r)
    if ((keys[r] ^ k0) >> shift) return 1;
  return 0;
}

// kThreads threads, tasks of at most kCap keys; the small size takes tasks
// of up to kTailSmall keys, the large one the rest (each skips the other's).
// One task: the group at list position gi (all threads of the block).
template <class K, int kThreads, int kCap>
__device__ __forceinline__ void tail_task(const ResidentArgs& a, int gi, unsigned char* smem_raw) {
  using T = KT<K>;
  using Bits = typename T::Bits;
  using Ord = typename T::Ord;
  constexpr int kW = kThreads / 32;     // warps
  constexpr int kPT = kCap / kThreads;  // keys per thread
  constexpr Ord kSpan = (Ord)1 << (sizeof(Ord) * 8 - kPosBits);
  TailSmem<K, kCap, kW>& sh = *reinterpret_cast<TailSmem<K, kCap, kW>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool large = kCap == kResidentMax;
  const Group g = a.groups[large && a.large_from_end ? a.group_cap - 1 - gi : gi];
  if (large ? g.n <= kTailSmall : g.n > kCap) return;
  const int n = g.n;
  const Bits* src = keys_of<const Bits>(g.buf, g.ubase, a.buf) + g.off;
  Bits* dst = reinterpret_cast<Bits*>(g.ubase) + g.off;
  int nseg;
  bool split_tree = false;  // children at odd ids are equality buckets
  bool fine = false;        // segments are bucket eighths (starts in fstart)
  unsigned* const fstart = &sh.peer[0][0];
  if (g.fit >= 0) {
    // the model: a copy in shared memory for the phases after the first
    // barrier; until then every thread reads it from global memory, and each
    // warp zeroes its own bucket-count row, so no barrier is needed to start
    const TailModel& gm = a.tail_models[g.fit];
    if (threadIdx.x < (int)(sizeof(TailModel) / 8))
      reinterpret_cast<unsigned long long*>(&sh.tm)[threadIdx.x] =
          reinterpret_cast<const unsigned long long*>(&gm)[threadIdx.x];
    for (int i = lane; i < kMaxK; i += 32) sh.peer[warp][i] = 0u;
    if (threadIdx.x == 0) {
      sh.slow_all = 0;
      sh.any_big = 0;
      sh.any_mid = 0;
    }
    __syncwarp();
    const TailModel* gmp = &gm;
    split_tree = gm.l.kind == kSplitter;
    // a large splitter tree comes from its pool slot; without one the task
    // recurses in k_slow
    bool slow = split_tree && gm.nsplit > kTailSplit && gm.pool < 0;
    const uint64_t* splits = gm.split;
    if (split_tree && gm.nsplit > kTailSplit && !slow) {
      for (int i = threadIdx.x; i < gm.nsplit; i += blockDim.x)
        sh.split[i] = a.split_pool[(size_t)gm.pool * 128 + i];
      __syncthreads();
      splits = sh.split;
    }
    const int nsplit = gmp->nsplit;
    if (!slow) {
      Classifier<K> cls;
      cls.load(gmp->l, a.exact_only);
      const int chunk = ((n + kW * 32 - 1) / (kW * 32)) * 32;
      const int steps = chunk / 32;
      Bits v[kPT];
      unsigned int br[kPT];
#pragma unroll
      for (int j = 0; j < kPT; ++j) {
        const int i = warp * chunk + j * 32 + lane;
        v[j] = (j < steps && i < n) ? src[i] : Bits(0);
      }
      // classify; keys that need the binary64 model are deferred; the
      // task's key range on the side
      unsigned dmask = 0;
      Ord klo = ~(Ord)0, khi = 0;
      // a linear model with a same-binade or uncentred estimate is evaluated
      // without branches (undecided keys are deferred); the rest through the
      // general dispatch
      const int path = split_tree || gmp->l.kind != kLinear ? 0 : cls.ufast ? 1 : cls.gfast ? 2 : 0;
      if (path != 0) {
#pragma unroll
        for (int j = 0; j < kPT; ++j) {
          if (j < steps) {
            const int i = warp * chunk + j * 32 + lane;
            int bk = kMaxK;
            if (i < n) {
              const Ord o = T::ord(v[j]);
              klo = o < klo ? o : klo;
              khi = o > khi ? o : khi;
              bool ok;
              bk = path == 1 ? cls.ord_bf(v[j], ok) : cls.flt_bf(v[j], ok);
              if (!ok) dmask |= 1u << j;
            }
            br[j] = (unsigned)bk;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < kPT; ++j) {
          if (j < steps) {
            const int i = warp * chunk + j * 32 + lane;
            int bk = kMaxK;
            if (i < n) {
              const Ord o = T::ord(v[j]);
              klo = o < klo ? o : klo;
              khi = o > khi ? o : khi;
              bk = split_tree ? splitter_bucket((uint64_t)o, splits, nsplit)
                              : cls.bucket_or_defer(v[j]);
              if (bk < 0) dmask |= 1u << j;
            }
            br[j] = (unsigned)bk;
          }
        }
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        const Ord l2 = __shfl_xor_sync(0xffffffffu, klo, o), h2 = __shfl_xor_sync(0xffffffffu, khi, o);
        klo = l2 < klo ? l2 : klo;
        khi = h2 > khi ? h2 : khi;
      }
      if (lane == 0) {
        sh.wlo[warp] = klo;
        sh.whi[warp] = khi;
      }
      if (__any_sync(0xffffffffu, dmask != 0)) {
        // queue them (in the key area, free until the tile is placed) and
        // evaluate 32 at a time
        static_assert(kW * kPT * 32 * 3 <= (int)sizeof(sh.keys), "deferred queue must fit in the key area");
        unsigned short* xq = reinterpret_cast<unsigned short*>(sh.keys) + warp * kPT * 32;
        unsigned char* xr = reinterpret_cast<unsigned char*>(sh.keys) + kW * kPT * 32 * 2 + warp * kPT * 32;
        int nq = 0;
        for (int j = 0; j < steps; ++j) {
          const bool d = (dmask >> j) & 1u;
          const unsigned dm = __ballot_sync(0xffffffffu, d);
          if (d) xq[nq + __popc(dm & lanemask_lt())] = (unsigned short)(j * 32 + lane);
          nq += __popc(dm);
        }
        __syncwarp();
        for (int q = lane; q < nq; q += 32) {
          const int code = xq[q];
          xr[code] = (unsigned char)cls.exact(src[warp * chunk + code]);
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < kPT; ++j)
          if (j < steps && ((dmask >> j) & 1u)) br[j] = xr[j * 32 + lane];
        __syncwarp();
      }
      // per-warp bucket counts (one shared atomic per key)
#pragma unroll
      for (int j = 0; j < kPT; ++j)
        if (j < steps && br[j] < (unsigned)kMaxK) atomicAdd(&sh.peer[warp][br[j]], 1u);
      __syncthreads();
      if (threadIdx.x < kMaxK) {
        // bucket totals; each warp's offset inside the bucket (placement
        // cursors in peer, the same offsets in wcnt for stable placement)
        const int b = threadIdx.x;
        unsigned run = 0;
#pragma unroll
        for (int w = 0; w < kW; ++w) {
          const unsigned x = sh.peer[w][b];
          sh.peer[w][b] = run;
          sh.wcnt[w][b] = (unsigned short)run;
          run += x;
        }
        sh.tot[b] = (int)run;
        // no progress of the linear model: the splitter tree decides (the
        // splitter tree itself always progresses or leaves one equality run)
        if ((int)run == n && !split_tree) sh.slow_all = 1;
        if ((int)run > a.cutoff && b < sh.tm.l.nb && !(split_tree && (b & 1))) sh.any_big = 1;
        if ((int)run > kSameMin && (int)run <= a.cutoff) sh.any_mid = 1;
      }
      if (threadIdx.x == 0) {  // the task's key range
        Ord lo = ~(Ord)0, hi = 0;
#pragma unroll
        for (int w = 0; w < kW; ++w) {
          lo = sh.wlo[w] < lo ? sh.wlo[w] : lo;
          hi = sh.whi[w] > hi ? sh.whi[w] : hi;
        }
        sh.tlo = lo;
        sh.tpk = (Ord)(hi - lo) < kSpan ? 1 : 0;
      }
      // non-empty buckets (keys spread over few buckets are mostly copies
      // of few values, which eighths would not separate)
      const int nonempty = __syncthreads_count(threadIdx.x < kMaxK && sh.tot[threadIdx.x] > 0);
      slow = sh.slow_all != 0;
      if (!slow) {
        if (warp == 0) {
          int loc[8];
          int sum = 0;
#pragma unroll
          for (int q = 0; q < 8; ++q) { loc[q] = sh.tot[lane * 8 + q]; sum += loc[q]; }
          int incl = sum;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
          }
          int run = incl - sum;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            sh.bstart[lane * 8 + q] = run;
            sh.segb[lane * 8 + q] = run;
            run += loc[q];
          }
          if (lane == 31) { sh.bstart[kMaxK] = run; sh.segb[kMaxK] = run; }
        }
        __syncthreads();
        const bool tpk = sh.tpk != 0;
        const Ord tlo = sh.tlo;
        const bool stable = sh.any_big != 0;
        if (stable) {
          // a bucket above the cutoff becomes a subproblem of its own, whose
          // sample is drawn by position: keys keep their input order inside
          // every bucket (rank within the warp from per-bucket lane masks,
          // one shared OR per key, after the warp's offset in wcnt)
          for (int i = lane; i < kMaxK; i += 32) sh.peer[warp][i] = 0u;
          __syncwarp();
#pragma unroll
          for (int j = 0; j < kPT; ++j) {
            if (j < steps) {
              const int bk = (int)br[j];
              const bool valid = bk < kMaxK;
              const int bq = valid ? bk : 0;
              if (valid) atomicOr(&sh.peer[warp][bq], 1u << lane);
              __syncwarp();
              const unsigned peers = valid ? sh.peer[warp][bq] : 0u;
              const int lt = __popc(peers & lanemask_lt());
              const int basec = sh.wcnt[warp][bq];
              br[j] = ((unsigned)bk << 16) | (unsigned)(basec + lt);
              __syncwarp();
              if (valid && lt == 0) {  // the first lane of the bucket
                sh.wcnt[warp][bq] = (unsigned short)(basec + __popc(peers));
                sh.peer[warp][bq] = 0u;
              }
              __syncwarp();
            }
          }
        }
        // large tasks of a linear model with an estimate: every bucket is
        // cut into eighths by a refinement that never decreases inside the
        // bucket, so that the base case ranks each key among about an
        // eighth of its bucket
        fine = kCap == kResidentMax && path != 0 && !stable && nonempty >= kFineMinBuckets;
        if (fine) {
          unsigned* const fcur = reinterpret_cast<unsigned*>(&sh.wcnt[0][0]);
          static_assert(kCap != kResidentMax || sizeof(sh.wcnt) >= kMaxK * 8 * sizeof(unsigned), "eighth cursors must fit");
          static_assert(kCap != kResidentMax || sizeof(sh.peer) >= (kMaxK * 8 + 1) * sizeof(unsigned), "eighth starts must fit");
          for (int i = threadIdx.x; i < kMaxK * 8; i += kThreads) fcur[i] = 0u;
          __syncthreads();
#pragma unroll
          for (int j = 0; j < kPT; ++j) {
            if (j < steps) {
              const int bk = (int)br[j];
              unsigned id = 0xFFFFu;
              if (bk < kMaxK) {
                id = (unsigned)(bk * 8 + cls.sub8(src[warp * chunk + j * 32 + lane], bk, path));
                atomicAdd(&fcur[id], 1u);
              }
              br[j] = id;
            }
          }
          __syncthreads();
          if (threadIdx.x < kMaxK) {
            const int b = threadIdx.x;
            unsigned run = (unsigned)sh.bstart[b];
            bool mid = false;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const unsigned c = fcur[b * 8 + q];
              fcur[b * 8 + q] = run;
              fstart[b * 8 + q] = run;
              run += c;
              mid = mid || c > (unsigned)kSameMin;
            }
            if (mid) sh.any_mid = 3;
          }
          if (threadIdx.x == 0) fstart[kMaxK * 8] = (unsigned)n;
          __syncthreads();
#pragma unroll
          for (int j = 0; j < kPT; ++j) {
            if (j < steps) {
              const unsigned id = br[j];
              if (id < (unsigned)(kMaxK * 8)) {
                const int p = (int)atomicAdd(&fcur[id], 1u);
                const Ord o = T::ord(src[warp * chunk + j * 32 + lane]);
                sh.keys[p] = tpk ? (Ord)((Ord)(o - tlo) << kPosBits) | (Ord)p : o;
                sh.seg[p] = (unsigned short)id;
              }
            }
          }
        } else {
          // every bucket is base-cased unless `stable`: the order inside a
          // bucket does not matter, and a shared cursor per (warp, bucket)
          // gives each key its place
#pragma unroll
          for (int j = 0; j < kPT; ++j) {
            if (j < steps) {
              const int bk = stable ? (int)(br[j] >> 16) : (int)br[j];
              if (bk < kMaxK) {
                const int p = sh.bstart[bk] + (stable ? (int)(br[j] & 0xFFFF)
                                                      : (int)atomicAdd(&sh.peer[warp][bk], 1u));
                // read again (from cache) rather than held in registers
                const Ord o = T::ord(src[warp * chunk + j * 32 + lane]);
                sh.keys[p] = tpk ? (Ord)((Ord)(o - tlo) << kPosBits) | (Ord)p : o;
                sh.seg[p] = (unsigned char)bk;
              }
            }
          }
        }
        if (threadIdx.x == 0) {
          atomicAdd((unsigned long long*)&a.run->resident_passes, 1ULL);
          if (split_tree) atomicAdd((unsigned long long*)&a.run->resident_fallback, 1ULL);
        }
        // trace record of this pass (the model was fitted by k_tail_fit)
        if (a.trace_cap > 0) {
          if (threadIdx.x == 0) {
            sh.rec = (long long)atomicAdd((unsigned long long*)&a.run->trace_count, 1ULL);
            if (sh.rec < a.trace_cap) {
              iplsTraceRecDev& r = a.trace[sh.rec];
              r.off = g.off; r.n = n; r.level = g.level; r.kind = sh.tm.l.kind;
              r.capped = sh.tm.l.capped; r.nbuckets = sh.tm.l.nb; r.S = sh.tm.l.S; r.D = sh.tm.l.D;
              r.A = sh.tm.l.A; r.Bc = sh.tm.l.Bc; r.ud = sh.tm.l.ud; r.xlo_bits = sh.tm.l.xlo_bits;
              r.nsplit = split_tree ? nsplit : 0; r.where = 1;
            }
          }
          __syncthreads();
          if (sh.rec < a.trace_cap && threadIdx.x < kMaxK)
            a.trace[sh.rec].counts[threadIdx.x] = (threadIdx.x < sh.tm.l.nb) ? sh.tot[threadIdx.x] : 0;
        }
        // buckets above the cutoff are queued as children; an equality
        // bucket is done, and so is a bucket of equal keys after its record
        // (most tasks have no bucket above the cutoff and skip this)
        if (sh.any_big) {
          __syncthreads();
          mark_homogeneous(sh.keys, sh.bstart, sh.tot, sh.tm.l.nb, a.cutoff, sh.hom,
                           sh.tpk ? kPosBits : 0);
          if (threadIdx.x < sh.tm.l.nb && sh.tot[threadIdx.x] > a.cutoff && !(split_tree && (threadIdx.x & 1))) {
            const int b = threadIdx.x;
            if (sh.hom[b]) record_homogeneous(a, g.off + sh.bstart[b], sh.tot[b], g.level + 1);
            else push_slow(a, g.off + sh.bstart[b], sh.tot[b], g.level + 1, g.ubase);
          }
          __syncthreads();
        }
      }
    }
    if (slow) {
      // the whole task recurses in the slow kernel (the in-block fit draws the
      // same sample and makes the same model), from the user buffer
      if (g.buf != 0)
        for (int p = threadIdx.x; p < n; p += blockDim.x) dst[p] = src[p];
      if (threadIdx.x == 0) push_whole(a, g.off, n, g.level, g.ubase);
      if (threadIdx.x == 0) atomicAdd((unsigned long long*)&a.run->resident_groups, 1ULL);
      return;
    }
    nseg = sh.tm.l.nb;
  } else {
    for (int i = threadIdx.x; i < n; i += blockDim.x) sh.keys[i] = T::ord(src[i]);
    const int64_t b0 = g.bounds[0];
    for (int q = threadIdx.x; q <= g.nchild; q += blockDim.x) sh.segb[q] = (int)(g.bounds[q] - b0);
    __syncthreads();
    for (int q = warp; q < g.nchild; q += kW)
      for (int i = sh.segb[q] + lane; i < sh.segb[q + 1]; i += 32) sh.seg[i] = (unsigned char)q;
    nseg = g.nchild;
  }
  __syncthreads();
  // ---- base case: rank counting inside every segment of <= cutoff keys ----
  // The position of a key in its segment is the number of keys before it in
  // (key, position) order, counted on packed words where they fit: a fitted
  // task was placed packed when its whole key range fits; a group of small
  // children is packed here, segment by segment.
  const int cutoff = a.cutoff;
  const bool task_pk = g.fit >= 0 && sh.tpk != 0;
  if (g.fit < 0) {
    for (int q = threadIdx.x; q < nseg; q += blockDim.x) {
      Ord mn = 0;
      bool pk = false, eq = false;
      const int s = sh.segb[q] & (int)kStartMask, e = sh.segb[q + 1] & (int)kStartMask;
      if (e - s >= 2 && e - s <= cutoff) {
        mn = sh.keys[s];
        Ord mx = mn;
        for (int r = s + 1; r < e; ++r) {
          const Ord k = sh.keys[r];
          mn = k < mn ? k : mn;
          mx = k > mx ? k : mx;
        }
        pk = (Ord)(mx - mn) < kSpan;
        eq = mx == mn;
      }
      sh.seglo[q] = mn;
      sh.segpk[q] = pk ? 1 : 0;
      // only this thread writes segb[q]; readers mask the mark off
      if (eq) sh.segb[q] = s | (int)kSameBit;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      const int q = sh.seg[p];
      if (sh.segpk[q]) sh.keys[p] = (Ord)((Ord)(sh.keys[p] - sh.seglo[q]) << kPosBits) | (Ord)p;
    }
    __syncthreads();
  } else if (sh.any_mid & (fine ? 2 : 1)) {
    // segments of kSameMin+1 .. cutoff keys that hold copies of one key
    const int ncell = fine ? kMaxK * 8 : nseg;
    const int sshift = task_pk ? kPosBits : 0;
    unsigned* const st = fine ? fstart : reinterpret_cast<unsigned*>(sh.segb);
    for (int q = threadIdx.x; q < ncell; q += blockDim.x) {
      const int s = (int)(st[q] & kStartMask), e = (int)(st[q + 1] & kStartMask);
      if (e - s > kSameMin && e - s <= cutoff && !differs(sh.keys, s, e, sshift)) st[q] = (unsigned)s | kSameBit;
    }
    __syncthreads();
  }
  for (int p = threadIdx.x; p < n; p += blockDim.x) {
    const int q = sh.seg[p];
    const unsigned s0 = fine ? fstart[q] : (unsigned)sh.segb[q];
    const int s = (int)(s0 & kStartMask);
    const int e = (int)((fine ? fstart[q + 1] : (unsigned)sh.segb[q + 1]) & kStartMask);
    const Ord kp = sh.keys[p];
    // copies of one key keep their places
    const bool based = e - s <= cutoff && !(split_tree && (q & 1)) && !(s0 & kSameBit);
    int d = p;
    Ord out = kp;
    if (task_pk || (g.fit < 0 && sh.segpk[q])) {
      if (based) d = s + count_below(sh.keys, s, e, kp);
      out = (Ord)((task_pk ? sh.tlo : sh.seglo[q]) + (kp >> kPosBits));
    } else if (based) {
      int cnt = 0;
      for (int r = s; r < e; ++r) {
        const Ord kr = sh.keys[r];
        cnt += (kr < kp) || (kr == kp && r < p);
      }
      d = s + cnt;
    }
    dst[d] = T::unord(out);
  }
  if (threadIdx.x == 0) {
    atomicAdd((unsigned long long*)&a.run->resident_keys, (unsigned long long)n);
    atomicAdd((unsigned long long*)&a.run->resident_groups, 1ULL);
  }
}

// kThreads threads, tasks of at most kCap keys; the small size takes tasks
// of up to kTailSmall keys, the large one the rest (each skips the other's).
// Host-driven levels: one block per task.  Device-driven levels (kTicket):
// one wave of blocks takes the tasks from a ticket.
template <class K, int kThreads, int kCap, bool kTicket>
__global__ void __launch_bounds__(kThreads, kCap == kResidentMax ? 2 : 4) k_tail(ResidentArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool large = kCap == kResidentMax;
  if (!kTicket) {
    tail_task<K, kThreads, kCap>(a, blockIdx.x, smem_raw);
    return;
  }
  __shared__ int s_gi;
  const int32_t count = tail_count(a, large);
  for (;;) {
    if (threadIdx.x == 0) s_gi = atomicAdd(&a.slow_ctl->tticket[large ? 1 : 0], 1);
    __syncthreads();
    const int gi = s_gi;
    if (gi >= count) break;
    tail_task<K, kThreads, kCap>(a, gi, smem_raw);
    __syncthreads();  // the task is done with shared memory (and s_gi read)
  }
}

template <class Bits>
__global__ void k_fill(const Fill* fills, const LevelCtl* cnt, int32_t cap, const RunStatus* run) {
  int32_t nf = cap;
  if (cnt) nf = (cnt->overflow || run->error_level) ? 0 : (cnt->nfill < cap ? cnt->nfill : cap);
  for (int32_t fi = blockIdx.x; fi < nf; fi += gridDim.x) {
  const Fill f = fills[fi];
  Bits* keys = reinterpret_cast<Bits*>(f.ubase);
  const Bits v = (Bits)f.bits;
  for (int64_t i = threadIdx.x; i < f.n; i += blockDim.x) keys[f.off + i] = v;
  }
}

template <class F>
static cudaError_t by_dtype_r(int dtype, F f) {
  switch (dtype) {
    case 0: return f((double*)nullptr);
    case 1: return f((float*)nullptr);
    case 2: return f((unsigned long long*)nullptr);
    case 3: return f((unsigned int*)nullptr);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_tail_fit(const ResidentArgs& a, cudaStream_t s, int sms) {
  if (a.nfit <= 0) return cudaSuccess;
  return by_dtype_r(a.dtype, [&](auto* tag) {
    using K = std::remove_pointer_t<decltype(tag)>;
    const size_t smem = (size_t)kFitWarps * fit_slot_bytes<typename KT<K>::Ord>();
    cudaFuncSetAttribute(k_tail_fit<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tail_fit<K>, kFitWarps * 32, smem) != cudaSuccess || per < 1) {
      cudaGetLastError();
      per = 1;
    }
    const int64_t need = (a.nfit + kFitWarps - 1) / kFitWarps;
    const int blocks = (int)std::min<int64_t>(need, (int64_t)per * sms);
    k_tail_fit<K><<<blocks, kFitWarps * 32, smem, s>>>(a);
    return cudaGetLastError();
  });
}

template <class K, bool kTicket>
static cudaError_t launch_resident_t(const ResidentArgs& a, cudaStream_t s, int large, int sms) {
  // tasks of up to kTailSmall keys in the small blocks, the rest in the
  // large ones; on device-driven levels the counts are capacities and one
  // wave of resident blocks takes the tasks from a ticket
  if (!large) {
    if (a.ngroups <= 0) return cudaSuccess;
    const size_t ss = sizeof(TailSmem<K, kTailSmall, kRW / 2>);
    cudaFuncSetAttribute(k_tail<K, kResidentThreads / 2, kTailSmall, kTicket>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ss);
    const int g = a.device_counts ? std::min(a.ngroups, sms * 4) : a.ngroups;
    k_tail<K, kResidentThreads / 2, kTailSmall, kTicket><<<g, kResidentThreads / 2, ss, s>>>(a);
    return cudaGetLastError();
  }
  const size_t sl = sizeof(TailSmem<K, kResidentMax, kRW>);
  cudaFuncSetAttribute(k_tail<K, kResidentThreads, kResidentMax, kTicket>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sl);
  const int nl = a.large_from_end ? a.nlarge : a.ngroups;
  if (nl <= 0) return cudaSuccess;
  const int g = a.device_counts ? std::min(nl, sms * 2) : nl;
  k_tail<K, kResidentThreads, kResidentMax, kTicket><<<g, kResidentThreads, sl, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_resident(const ResidentArgs& a, cudaStream_t s, int large, int sms) {
  return by_dtype_r(a.dtype, [&](auto* tag) {
    using K = std::remove_pointer_t<decltype(tag)>;
    return a.device_counts ? launch_resident_t<K, true>(a, s, large, sms)
                           : launch_resident_t<K, false>(a, s, large, sms);
  });
}

cudaError_t launch_slow(const ResidentArgs& a, cudaStream_t s, int sms) {
  return by_dtype_r(a.dtype, [&](auto* tag) {
    using K = std::remove_pointer_t<decltype(tag)>;
    const size_t smem = sizeof(ResSmem<K>);
    cudaFuncSetAttribute(k_slow<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_slow<K>, kResidentThreads, smem) != cudaSuccess || per < 1) {
      cudaGetLastError();
      per = 1;
    }
    k_slow<K><<<per * sms, kResidentThreads, smem, s>>>(a);
    return cudaGetLastError();
  });
}

__global__ void k_slow_groups(const SlowTask* list, int32_t n, Group* groups, int32_t* fit_list) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const SlowTask t = list[i];
  groups[i] = Group{t.off, nullptr, t.n, t.level, 0, 1, i, 0, t.ubase};
  fit_list[i] = i;
}

cudaError_t launch_slow_groups(const SlowTask* list, int32_t n, Group* groups, int32_t* fit_list,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_slow_groups<<<(n + 255) / 256, 256, 0, s>>>(list, n, groups, fit_list);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(1024) k_sweep_groups(const SlowTask* list, SlowCtl* ctl, int32_t list_cap,
                                                      Group* groups, int32_t* fit_list, int32_t group_cap) {
  __shared__ int32_t s_n;
  if (threadIdx.x == 0) {
    int32_t n = ctl->count;
    if (n < kTailSweepMin || n > list_cap || n > group_cap) n = 0;
    s_n = n;
  }
  __syncthreads();
  const int32_t n = s_n;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const SlowTask t = list[i];
    groups[i] = Group{t.off, nullptr, t.n, t.level, 0, 1, i, 0, t.ubase};
    fit_list[i] = i;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl->sweep = n;
    if (n > 0) {  // the child list starts again; whole tasks stay
      ctl->count = 0;
      ctl->ticket = 0;
      ctl->pool_used = 0;
      ctl->fit_ticket = 0;
      ctl->tticket[0] = 0;
      ctl->tticket[1] = 0;
    }
  }
}

cudaError_t launch_sweep_groups(const SlowTask* list, SlowCtl* ctl, int32_t list_cap, Group* groups,
                                int32_t* fit_list, int32_t group_cap, cudaStream_t s) {
  k_sweep_groups<<<1, 1024, 0, s>>>(list, ctl, list_cap, groups, fit_list, group_cap);
  return cudaGetLastError();
}

cudaError_t launch_fill(const Fill* fills, int32_t nfill, int dtype, cudaStream_t s, const LevelCtl* cnt,
                        int grid, const RunStatus* run) {
  if (nfill <= 0) return cudaSuccess;
  const int g = cnt ? (grid < nfill ? grid : nfill) : nfill;
  if (dtype == 0 || dtype == 2)
    k_fill<unsigned long long><<<g, 256, 0, s>>>(fills, cnt, nfill, run);
  else
    k_fill<unsigned int><<<g, 256, 0, s>>>(fills, cnt, nfill, run);
  return cudaGetLastError();
}

// One range sorted by one block with the in-block recursion of k_slow, the
// range passed by value instead of through the slow lists: the only device
// memory it touches besides the keys is a.run.
template <class K>
__global__ void __launch_bounds__(kResidentThreads, 1) k_slow_one(ResidentArgs a, SlowTask st) {
  using T = KT<K>;
  using Bits = typename T::Bits;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ResSmem<K>& sh = *reinterpret_cast<ResSmem<K>*>(smem_raw);
  Bits* src = reinterpret_cast<Bits*>(st.ubase) + st.off;
  for (int p = threadIdx.x; p < st.n; p += blockDim.x) sh.keys[p] = T::ord(src[p]);
  if (threadIdx.x == 0) {
    sh.nsmall = 0;
    sh.err = 0;
    sh.nstack = st.n > a.cutoff ? 1 : 0;
    sh.u.s.tasks[kResidentTasks - 1] = enc_task(0, st.n, st.level);
    if (st.n <= a.cutoff && st.n > 1) {
      sh.nsmall = 1;
      sh.u.s.tasks[0] = enc_task(0, st.n, st.level);
    }
  }
  __syncthreads();
  run_stack<K>(sh, a, st.off);
  for (int p = threadIdx.x; p < st.n; p += blockDim.x) src[p] = T::unord(sh.keys[p]);
}

cudaError_t launch_slow_one(const ResidentArgs& a, const SlowTask& t, cudaStream_t s) {
  return by_dtype_r(a.dtype, [&](auto* tag) {
    using K = std::remove_pointer_t<decltype(tag)>;
    const size_t smem = sizeof(ResSmem<K>);
    cudaError_t e = cudaFuncSetAttribute(k_slow_one<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_slow_one<K><<<1, kResidentThreads, smem, s>>>(a, t);
    return cudaGetLastError();
  });
}

// Largest task a block can hold for this cutoff: every pending range of more
// than `cutoff` keys must fit in half of the task array.
int resident_rmax(int cutoff) {
  const long long lim = (long long)(kResidentTasks / 2) * (cutoff + 1);
  return lim < kResidentMax ? (int)lim : kResidentMax;
}

}  // namespace ipls
