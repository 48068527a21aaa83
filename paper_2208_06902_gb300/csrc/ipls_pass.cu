// Grid-wide learned partition pass over all subproblems of one level.
//
//   k_fit      sample alpha*k-1 keys, sort them, fit FMCD (Ch.3 listing) or
//              the splitter tree -- or, when enabled, train the PL2 learned
//              CDF -- and zero the counts: one warp per subproblem
//              (k_fit_warp) when the sample fits, else one block.
//   k_hist     every tile of every subproblem: classify each key with the
//              model (Ch.3 model equation) and store its bucket id, per-warp
//              shared histograms; the tile's histogram goes to memory, the
//              subproblem's totals are accumulated with one atomic per
//              bucket per block.
//   k_check    no-progress rule: a linear pass that puts every key into one
//              bucket (or a PL2 pass with a bucket above 4n/k) is redone with
//              the splitter tree from the same sample.
//   k_scan     exclusive scan of the bucket counts -> bucket bases; children
//              become next-level subproblems, block-resident groups (tasks of
//              up to kTailSmall keys from the front of the list, larger ones
//              from the back), or (equality buckets) fills; records the trace.
//   k_tilescan exclusive scan of the tile histograms of every subproblem,
//              per bucket, over its tiles: chunks of kChunkTiles tiles in
//              ticket order, each chunk's prefix found by decoupled look-back
//              over the chunks before it.
//   k_scatter  every tile: read the keys and the bucket ids k_hist stored,
//              rank each key stably inside the tile (per-bucket peer masks +
//              per-warp counters), stage the tile in bucket order in shared
//              memory and write the bucket runs out with coalesced stores at
//              bucket base + tile offset (Ch.2 IPS4o: move every key into the
//              region of its bucket).
#include <cuda/atomic>

#include "ipls_device.cuh"

namespace ipls {

constexpr int kTile = kTileKeys;
constexpr int kWarps = kPassThreads / 32;
// k_scatter: 512 threads per tile, 8 keys each
constexpr int kScatterThreads = 512;
constexpr int kSWarps = kScatterThreads / 32;
constexpr int kSKPT = kTile / kScatterThreads;
constexpr int kSKPW = kTile / kSWarps;

int tile_keys(int) { return kTile; }
int key_bytes(int dtype) { return (dtype == 0 || dtype == 2) ? 8 : 4; }
int sample_size_host(int64_t n, int level, int k, int64_t root_sample) {
  return (int)sample_size(n, level, k, root_sample);
}

template <class K>
__device__ __forceinline__ const typename KT<K>::Bits* buf_ptr(const LevelArgs& a, const Sub& sub) {
  return keys_of<const typename KT<K>::Bits>(sub.buf, sub.ubase, a.buf);
}

// Copies a Model between memories with all threads of the block.
__device__ __forceinline__ void copy_model(Model* dst, const Model* src) {
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(Model) / 8); i += blockDim.x) d[i] = s[i];
}

// Copies a ThrTable between memories with all threads of the block.
__device__ __forceinline__ void copy_table(ThrTable* dst, const ThrTable* src) {
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(ThrTable) / 8); i += blockDim.x) d[i] = s[i];
}

// Gathers and sorts the sample of one subproblem (all threads).
template <class K>
__device__ int gather_sorted_sample(const LevelArgs& a, const Sub& sub,
                                    typename KT<K>::Ord* so) {
  using T = KT<K>;
  const int S = (int)sample_size(sub.n, sub.level, a.k, a.root_sample);
  const uint64_t st = stream_key(a.seed, sub.off, sub.n, sub.level);
  const typename T::Bits* src = buf_ptr<K>(a, sub);
  for (int j = threadIdx.x; j < S; j += blockDim.x)
    so[j] = T::ord(src[sub.off + sample_offset(st, j, sub.n)]);
  __syncthreads();
  block_sort(so, S);
  return S;
}

// Subproblems whose sample fits a warp's share of shared memory are fitted
// by one warp each (k_fit_warp), many at a time; the others (the root and
// very large subproblems, or all when the threshold index is built) by one
// block each (k_fit).
// A level with fewer subproblems than kWarpFitMin keeps one block per fit
// (eight fits per block would leave most SMs idle).
constexpr int kFitWarpsG = 8;
constexpr int kWarpFitMin = 1024;
__host__ __device__ __forceinline__ bool warp_fits(const LevelArgs& a, int32_t nsub) {
  return !a.use_tables && nsub >= kWarpFitMin;
}
// Subproblems that take PL2 (when enabled) are fitted by a block.
__device__ __forceinline__ bool takes_pl2(const LevelArgs& a, const Sub& sub, int S) {
  // (a level whose largest sample exceeds kPL2MaxSample is a level-0 launch
  // in which every sample does; it reserves no PL2 scratch)
  return a.pl2_leaves > 0 && sub.n > kPL2MinKeys && S <= kPL2MaxSample && a.max_sample <= kPL2MaxSample &&
         (a.pl2_depth == 0 || sub.level < a.pl2_depth);
}
__device__ __forceinline__ bool fit_by_warp(const LevelArgs& a, const Sub& sub, int32_t nsub) {
  const int S = (int)sample_size(sub.n, sub.level, a.k, a.root_sample);
  return warp_fits(a, nsub) && S <= kResidentSample && !takes_pl2(a, sub, S);
}

template <class K>
__global__ void __launch_bounds__(kFitWarpsG * 32) k_fit_warp(LevelArgs a) {
  using T = KT<K>;
  using Ord = typename T::Ord;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ FitShared fs[kFitWarpsG];
  __shared__ Model mod[kFitWarpsG];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t nsub = level_nsub(a);
  for (int s = blockIdx.x * kFitWarpsG + warp; s < nsub; s += gridDim.x * kFitWarpsG) {
  const Sub sub = a.subs[s];
  if (!fit_by_warp(a, sub, nsub)) continue;
  const int S = (int)sample_size(sub.n, sub.level, a.k, a.root_sample);
  Ord* so = reinterpret_cast<Ord*>(smem_raw) + warp * kResidentSample;
  const uint64_t st = stream_key(a.seed, sub.off, sub.n, sub.level);
  const typename T::Bits* src = buf_ptr<K>(a, sub) + sub.off;
  for (int j = lane; j < S; j += 32) so[j] = T::ord(src[sample_offset(st, j, sub.n)]);
  __syncwarp();
  group_sort<WarpG, Ord>(so, S);
  Model& m = mod[warp];
  fit_model<WarpG, K>(so, S, a.k, &m, fs[warp]);
  const unsigned long long* ms = reinterpret_cast<const unsigned long long*>(&m);
  unsigned long long* md = reinterpret_cast<unsigned long long*>(&a.models[s]);
  for (int i = lane; i < (int)(sizeof(Model) / 8); i += 32) md[i] = ms[i];
  for (int b = lane; b < kMaxK; b += 32) a.counts[(size_t)s * kMaxK + b] = 0;
  if (lane == 0) {
    if (a.use_tables) a.tabs[s].ok = 0;
    a.subs[s].flags = 0;
    atomicAdd((unsigned long long*)&a.ctl->keys_level, (unsigned long long)sub.n);
  }
  __syncwarp();
  }
}

// ---------------------------------------------------------------------------
template <class K>
__global__ void __launch_bounds__(kFitThreads) k_fit(LevelArgs a) {
  using Ord = typename KT<K>::Ord;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Model sm;
  __shared__ FitShared fs;
  __shared__ ThrTable tab;
  __shared__ int scan_tmp[kL1Max];
  Ord* so = reinterpret_cast<Ord*>(smem);
  const int32_t nsub = level_nsub(a);
  for (int s = blockIdx.x; s < nsub; s += gridDim.x) {
  __syncthreads();  // the previous subproblem is done with shared memory
  const Sub sub = a.subs[s];
  if (fit_by_warp(a, sub, nsub)) continue;  // k_fit_warp fits this one
  const int S = gather_sorted_sample<K>(a, sub, so);
  bool pl2 = false;
  if (takes_pl2(a, sub, S)) {
    // scratch after the sample: leaf, w and r per sample
    unsigned char* base = smem + (((size_t)a.max_sample * sizeof(Ord) + 15) & ~(size_t)15);
    PL2Scratch sc{reinterpret_cast<int32_t*>(base + (size_t)kPL2MaxSample * 8),
                  reinterpret_cast<float*>(base), reinterpret_cast<float*>(base + (size_t)kPL2MaxSample * 4)};
    __shared__ float py[kPL2MaxLeaves + 1];
    __shared__ int pstart[kPL2MaxLeaves + 1];
    __shared__ int pflag, prho, psh;
    __shared__ long long px0;
    if (threadIdx.x == 0) sm.nsplit = 0;
    pl2 = fit_pl2<K>(so, S, a.pl2_leaves, a.k, &sm, a.knots + (size_t)s * (a.pl2_leaves + 1), sc, py,
                     pstart, &pflag, &px0, &prho, &psh);
  }
  if (!pl2) fit_model<BlockG, K>(so, S, a.k, &sm, fs);
  copy_model(&a.models[s], &sm);
  if (sm.l.kind == kLinear && a.use_tables) {
    build_thr_table<K>(sm.l, &tab, scan_tmp);
    copy_table(&a.tabs[s], &tab);
  } else if (threadIdx.x == 0 && a.use_tables) {
    a.tabs[s].ok = 0;
  }
  for (int b = threadIdx.x; b < kMaxK; b += blockDim.x) a.counts[(size_t)s * kMaxK + b] = 0;
  if (threadIdx.x == 0) {
    a.subs[s].flags = 0;
    atomicAdd((unsigned long long*)&a.ctl->keys_level, (unsigned long long)sub.n);
  }
  }
}

// ---------------------------------------------------------------------------
// How k_hist classifies the keys of a subproblem: the branch-free
// same-binade or uncentred estimate of a linear model, or the general
// dispatch (fixed-point estimate, splitter tree, PL2, binary64 only).
constexpr int kPathGeneric = 0, kPathOrd = 1, kPathFlt = 2;
constexpr int kHistGrab = 4;  // tiles k_hist takes per ticket
constexpr int kScatterGrab = 4;  // tiles k_scatter takes per ticket

template <class K>
__global__ void __launch_bounds__(kPassThreads, 4) k_hist(LevelArgs a, int rehist_only) {
  using T = KT<K>;
  using Bits = typename T::Bits;
  constexpr int kChunk = 8;  // keys per thread in flight
  __shared__ Model sm;
  __shared__ ThrTable tab;
  __shared__ unsigned int hist[kWarps][kMaxK];
  __shared__ unsigned int acc[kMaxK];
  __shared__ ExactQueue<kChunk * 32> xq[kWarps];
  __shared__ float pl_yf[kPL2MaxLeaves + 1];
  __shared__ int pl_lo[kPL2MaxLeaves + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kWarps * kMaxK; i += blockDim.x) (&hist[0][0])[i] = 0;
  for (int i = threadIdx.x; i < kMaxK; i += blockDim.x) acc[i] = 0;
  const int64_t nt = level_ntiles(a);
  int cur = -1;
  bool use_tab = false;
  int path = kPathGeneric;
  Classifier<K> cls;
  // groups of kHistGrab tiles from a level-wide ticket: tiles of some
  // subproblems classify slower (the general dispatch, deferred keys), and
  // a fixed share per block would leave the level waiting for the slowest
  // (the re-histogram pass, which skips most tiles, keeps one fixed range
  // per block)
  unsigned* const ticket = &a.ctl->tile_ticket[0];
  __shared__ long long s_tg;
  bool first = true;
  for (;;) {
  __syncthreads();  // the previous group is done before the ticket is read again
  if (!rehist_only && threadIdx.x == 0) s_tg = (long long)atomicAdd(ticket, (unsigned)kHistGrab);
  __syncthreads();
  int64_t tg, tge;
  if (rehist_only) {
    if (!first) break;
    first = false;
    tg = nt * blockIdx.x / gridDim.x;
    tge = nt * (blockIdx.x + 1) / gridDim.x;
  } else {
    tg = s_tg;
    if (tg >= nt) break;
    tge = tg + kHistGrab < nt ? tg + kHistGrab : nt;
  }
  for (int64_t t = tg; t < tge; ++t) {
    const int s = a.tile2sub[t];
    if (s != cur) {
      __syncthreads();
      if (cur >= 0) {
        for (int b = threadIdx.x; b < kMaxK; b += blockDim.x) {
          if (acc[b]) atomicAdd((unsigned long long*)&a.counts[(size_t)cur * kMaxK + b], (unsigned long long)acc[b]);
          acc[b] = 0;
        }
      }
      __syncthreads();
      copy_model(&sm, &a.models[s]);
      if (threadIdx.x == 0) tab.ok = 0;
      __syncthreads();
      if (a.use_tables && a.tabs[s].ok) copy_table(&tab, &a.tabs[s]);
      cur = s;
      __syncthreads();
      cls.load(sm, a.exact_only);
      use_tab = a.use_tables && sm.l.kind == kLinear && tab.ok;
      path = sm.l.kind != kLinear ? kPathGeneric : cls.ufast ? kPathOrd : cls.gfast ? kPathFlt : kPathGeneric;
      if (sm.l.kind == kPL2) {
        pl2_tables(sm, a.knots + (size_t)s * (a.pl2_leaves + 1), pl_yf, pl_lo, threadIdx.x, blockDim.x);
        __syncthreads();
      }
    }
    const Sub sub = a.subs[s];
    if (rehist_only && !(sub.flags & kRehist)) continue;
    const int64_t ti = t - sub.tile0;
    const int64_t base = sub.off + ti * kTile;
    const int64_t rem = sub.n - ti * kTile;
    const int tn = rem < kTile ? (int)rem : kTile;
    const Bits* src = buf_ptr<K>(a, sub) + base;
    for (int c0 = 0; c0 < kTile; c0 += kChunk * kPassThreads) {
      Bits v[kChunk];
#pragma unroll
      for (int j = 0; j < kChunk; ++j) {
        const int i = c0 + j * kPassThreads + threadIdx.x;
        v[j] = (i < tn) ? src[i] : Bits(0);
      }
      uint8_t* ids = a.bids + base;
      if (use_tab) {
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
          const int i = c0 + j * kPassThreads + threadIdx.x;
          if (i < tn) {
            const int bk = table_bucket<K>(T::ord(v[j]), tab, sm.l.nb);
            ids[i] = (uint8_t)bk;
            atomicAdd(&hist[warp][bk], 1u);
          }
        }
      } else {
        unsigned dmask = 0;  // steps whose key needs the binary64 model
        if (path != kPathGeneric) {
          // the estimate of the whole subproblem, without branches; keys it
          // cannot decide go to the binary64 batch below
#pragma unroll
          for (int j = 0; j < kChunk; ++j) {
            const int i = c0 + j * kPassThreads + threadIdx.x;
            if (i < tn) {
              bool ok;
              const int bk = path == kPathOrd ? cls.ord_bf(v[j], ok) : cls.flt_bf(v[j], ok);
              if (ok) {
                ids[i] = (uint8_t)bk;
                atomicAdd(&hist[warp][bk], 1u);
              } else {
                dmask |= 1u << j;
              }
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < kChunk; ++j) {
            const int i = c0 + j * kPassThreads + threadIdx.x;
            if (i < tn) {
              const int bk = sm.l.kind == kPL2 ? pl2_bucket<K>(v[j], sm, pl_yf, pl_lo) : cls.bucket_or_defer(v[j]);
              if (bk >= 0) {
                ids[i] = (uint8_t)bk;
                atomicAdd(&hist[warp][bk], 1u);
              } else {
                dmask |= 1u << j;
              }
            }
          }
        }
        if (__any_sync(0xffffffffu, dmask != 0)) {
          // queue them and evaluate 32 at a time
          int nq = 0;
          for (int j = 0; j < kChunk; ++j) {
            const bool d = (dmask >> j) & 1u;
            const unsigned dm = __ballot_sync(0xffffffffu, d);
            if (d) xq[warp].idx[nq + __popc(dm & lanemask_lt())] = (unsigned short)(c0 + j * kPassThreads + threadIdx.x);
            nq += __popc(dm);
          }
          __syncwarp();
          for (int q = lane; q < nq; q += 32) {
            const int i = xq[warp].idx[q];
            const int e = cls.exact(src[i]);
            ids[i] = (uint8_t)e;
            atomicAdd(&hist[warp][e], 1u);
          }
          __syncwarp();
        }
      }
    }
    __syncthreads();
    // the tile's histogram (all 256 bins) to memory; subproblem totals in acc
    uint32_t* th = a.tile_off + (size_t)t * kMaxK;
    for (int b = threadIdx.x; b < kMaxK; b += blockDim.x) {
      unsigned int tot = 0;
      for (int w = 0; w < kWarps; ++w) { tot += hist[w][b]; hist[w][b] = 0; }
      th[b] = tot;
      acc[b] += tot;
    }
    // the rows are zero again before any warp counts the next tile
    __syncthreads();
  }
  }
  __syncthreads();
  if (cur >= 0) {
    for (int b = threadIdx.x; b < kMaxK; b += blockDim.x)
      if (acc[b]) atomicAdd((unsigned long long*)&a.counts[(size_t)cur * kMaxK + b], (unsigned long long)acc[b]);
  }
}

// ---------------------------------------------------------------------------
template <class K>
__global__ void __launch_bounds__(kFitThreads) k_check(LevelArgs a) {
  using Ord = typename KT<K>::Ord;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Model sm;
  __shared__ int s_redo;
  Ord* so = reinterpret_cast<Ord*>(smem);
  const int32_t nsub = level_nsub(a);
  for (int s = blockIdx.x; s < nsub; s += gridDim.x) {
  __syncthreads();  // the previous subproblem is done with shared memory
  const Sub sub = a.subs[s];
  if (threadIdx.x == 0) s_redo = 0;
  __syncthreads();
  const Model& gm = a.models[s];
  if (gm.l.kind == kLinear) {
    for (int b = threadIdx.x; b < gm.l.nb; b += blockDim.x)
      if ((int64_t)a.counts[(size_t)s * kMaxK + b] == sub.n) s_redo = 1;
  } else if (gm.l.kind == kPL2) {
    // no progress, or one bucket above 4n/k: the splitter tree instead
    for (int b = threadIdx.x; b < gm.l.nb; b += blockDim.x) {
      const int64_t c = (int64_t)a.counts[(size_t)s * kMaxK + b];
      if (c == sub.n || c * gm.l.nb > 4 * sub.n) s_redo = 1;
    }
  }
  __syncthreads();
  if (!s_redo) continue;
  copy_model(&sm, &gm);
  __syncthreads();
  const int S = gather_sorted_sample<K>(a, sub, so);
  build_splitters<BlockG, K>(so, S, a.k, &sm);
  copy_model(&a.models[s], &sm);
  for (int b = threadIdx.x; b < kMaxK; b += blockDim.x) a.counts[(size_t)s * kMaxK + b] = 0;
  if (threadIdx.x == 0) {
    if (a.use_tables) a.tabs[s].ok = 0;
    a.subs[s].flags |= kRehist;
    atomicAdd(&a.ctl->nrehist, 1);
  }
  }
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t block_exclusive_scan256(int64_t v, int64_t* tmp) {
  // 256 threads; returns the exclusive prefix of v over thread order.
  const int t = threadIdx.x;
  tmp[t] = v;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    const int64_t x = (t >= off) ? tmp[t - off] : 0;
    __syncthreads();
    tmp[t] += x;
    __syncthreads();
  }
  const int64_t incl = tmp[t];
  __syncthreads();
  return incl - v;
}

template <class K>
__device__ void append_fill(const LevelArgs& a, int64_t off, int64_t n, uint64_t bits, uint64_t ubase) {
  for (int64_t o = 0; o < n; o += kFillChunk) {
    const int i = atomicAdd(&a.ctl->nfill, 1);
    if (i >= a.fill_cap) { a.ctl->overflow = 1; return; }
    a.fills[i] = Fill{off + o, (n - o) < kFillChunk ? (n - o) : (int64_t)kFillChunk, bits, ubase};
  }
}

template <class K>
__global__ void __launch_bounds__(256) k_scan(LevelArgs a) {
  using T = KT<K>;
  __shared__ int64_t tmp[256];
  __shared__ int64_t cnt[256];
  __shared__ int64_t bas[257];
  __shared__ int s_skip;
  __shared__ long long s_rec;
  const int b = threadIdx.x;
  const int32_t nsub = level_nsub(a);
  for (int s = blockIdx.x; s < nsub; s += gridDim.x) {
  __syncthreads();  // the previous subproblem is done with shared memory
  const Sub sub = a.subs[s];
  const Model& m = a.models[s];
  const int nb = m.l.nb;
  const bool splitter = m.l.kind == kSplitter;
  const int dst_buf = 1 - sub.buf;
  const int64_t c = (b < nb) ? (int64_t)a.counts[(size_t)s * kMaxK + b] : 0;
  cnt[b] = c;
  const int64_t ex = block_exclusive_scan256(c, tmp);
  bas[b] = ex;
  if (b == 255) bas[256] = ex + c;
  if (b == 0) {
    s_skip = 0;
    // trace record of this pass: trace_base + s, or (device-driven levels)
    // the next free record
    s_rec = a.trace_cap <= 0 ? 0
            : a.trace_ctr ? (long long)atomicAdd((unsigned long long*)a.trace_ctr, 1ULL)
                          : a.trace_base + s;
  }
  __syncthreads();
  int64_t* gb = a.bases + (size_t)s * 257;
  gb[b] = bas[b];
  if (b == 0) gb[256] = bas[256];
  const bool eq = splitter && (b & 1) && b < nb;
  if (eq && c == sub.n) s_skip = 1;
  const long long rec = s_rec;
  if (a.trace_cap > 0 && rec < a.trace_cap) {
    iplsTraceRecDev& r = a.trace[rec];
    if (b == 0) {
      r.off = sub.off; r.n = sub.n; r.level = sub.level; r.kind = m.l.kind;
      r.capped = m.l.capped; r.nbuckets = nb; r.S = m.l.S; r.D = m.l.D; r.A = m.l.A;
      r.Bc = m.l.Bc; r.ud = m.l.ud; r.xlo_bits = m.l.xlo_bits; r.nsplit = m.nsplit; r.where = 0;
    }
    r.counts[b] = c;
    // the PL2 knots of the pass (zeros for another kind of model)
    if (a.trace_knots && a.pl2_leaves > 0 && rec < a.knot_cap) {
      const int M1 = a.pl2_leaves + 1;
      float* kr = a.trace_knots + (size_t)rec * M1;
      const float* kn = a.knots + (size_t)s * M1;
      for (int j = b; j < M1; j += 256) kr[j] = m.l.kind == kPL2 ? kn[j] : 0.0f;
    }
  }
  __syncthreads();
  // every splitter-tree pass counts, a homogeneous one too
  if (b == 0 && splitter) atomicAdd((unsigned long long*)&a.ctl->fallback, 1ULL);
  if (s_skip) {
    // homogeneous subproblem: every key equals one splitter; nothing moves
    if (b == 0) {
      a.subs[s].flags |= kSkipScatter;
      if (sub.buf != 0) {
        int j = 1;
        for (int q = 1; q < nb; q += 2) if (cnt[q] == sub.n) j = q;
        append_fill<K>(a, sub.off, sub.n, (uint64_t)T::unord((typename T::Ord)m.split[(j - 1) / 2]),
                       sub.ubase);
      }
    }
  } else if (c > 0) {
    if (eq) {
      if (dst_buf != 0)
        append_fill<K>(a, sub.off + bas[b], c, (uint64_t)T::unord((typename T::Ord)m.split[(b - 1) / 2]),
                       sub.ubase);
    } else if (c > a.rmax) {
      const int i = atomicAdd(&a.ctl->nsub_next, 1);
      if (i >= a.next_sub_cap) {
        a.ctl->overflow = 1;
      } else {
        Sub ns{sub.off + bas[b], c, sub.level + 1, dst_buf, 0, 0, 0, 0, 0, sub.ubase};
        if (reserve_tiles(a.ctl, i, ns, a.next_tile2sub, a.next_tile_cap, a.next_chunk2sub,
                          a.next_chunk_cap))
          a.next_subs[i] = ns;
      }
    } else if (c > a.cutoff) {
      // a block-resident subproblem whose model k_tail_fit fits
      const int g = group_slot(a.ctl, c, a.group_cap);
      if (g < 0) {
        a.ctl->overflow = 1;
      } else {
        a.groups[g] = Group{sub.off + bas[b], nullptr, (int32_t)c, sub.level + 1, dst_buf, 1, g, 0, sub.ubase};
        const int f = atomicAdd(&a.ctl->nfit, 1);
        if (f < a.group_cap) a.fit_list[f] = g;
        else a.ctl->overflow = 1;
      }
    }
  }
  if (!s_skip && b == 0) {
    // pack consecutive base-case buckets into groups of <= rmax keys
    int b0 = -1, blast = -1;
    int64_t tot = 0;
    for (int q = 0; q <= nb; ++q) {
      const int64_t cq = (q < nb) ? cnt[q] : 0;
      const bool eqq = (q < nb) && splitter && (q & 1);
      const bool brk = (q == nb) || (cq > 0 && (eqq || cq > a.cutoff));
      const bool fits = (cq > 0) && !brk;
      if (b0 >= 0 && (brk || (fits && tot + cq > a.rmax))) {
        const int g = group_slot(a.ctl, tot, a.group_cap);
        if (g < 0) a.ctl->overflow = 1;
        else a.groups[g] = Group{sub.off + bas[b0], gb + b0, (int32_t)tot, sub.level + 1,
                                 dst_buf, blast - b0 + 1, -1, 0, sub.ubase};
        b0 = -1;
        tot = 0;
      }
      if (fits) {
        if (b0 < 0) b0 = q;
        tot += cq;
        blast = q;
      }
    }
    atomicAdd((unsigned long long*)&a.ctl->keys_moved, (unsigned long long)sub.n);
    int64_t mx = 0;
    for (int q = 0; q < nb; ++q) mx = cnt[q] > mx ? cnt[q] : mx;
    const long long frac = (long long)((double)mx * 1048576.0 / (double)sub.n);
    atomicMax((unsigned long long*)&a.ctl->max_bucket, (unsigned long long)frac);
  }  }
}

// ---------------------------------------------------------------------------
// Look-back status word: [63:48] epoch, [47:46] flag (1 aggregate, 2
// inclusive prefix), [45:0] count.
constexpr unsigned long long kFlagAgg = 1ULL << 46;
constexpr unsigned long long kFlagPre = 2ULL << 46;
constexpr unsigned long long kValMask = (1ULL << 46) - 1;

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> r(*p);
  r.store(v, cuda::memory_order_release);
}
__device__ __forceinline__ unsigned long long ld_acquire(unsigned long long* p) {
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> r(*p);
  return r.load(cuda::memory_order_acquire);
}

// One block of 256 threads per chunk (thread b = bucket b), chunks in ticket
// order so that a chunk only waits for chunks already being processed.
__global__ void __launch_bounds__(256) k_tilescan(LevelArgs a) {
  __shared__ int s_c;
  const int b = threadIdx.x;
  const unsigned long long ep = (unsigned long long)(a.epoch & 0xFFFF) << 48;
  const int64_t nchunks = level_nchunks(a);
  for (;;) {
    __syncthreads();
    if (b == 0) s_c = (int)atomicAdd(&a.ctl->ticket, 1u);
    __syncthreads();
    const int c = s_c;
    if (c >= nchunks) break;
    const Sub sub = a.subs[a.chunk2sub[c]];
    if (sub.flags & kSkipScatter) continue;
    const int ci = c - sub.chunk0;
    const int64_t tb = sub.tile0 + (int64_t)ci * kChunkTiles;
    const int64_t te0 = tb + kChunkTiles, tend = sub.tile0 + sub.ntiles;
    const int cnt = (int)((te0 < tend ? te0 : tend) - tb);
    uint32_t h[kChunkTiles];
    unsigned long long agg = 0;
#pragma unroll
    for (int q = 0; q < kChunkTiles; ++q) {
      h[q] = (q < cnt) ? a.tile_off[(size_t)(tb + q) * kMaxK + b] : 0u;
      agg += h[q];
    }
    unsigned long long* st = a.status + (size_t)c * kMaxK;
    unsigned long long excl = 0;
    if (ci == 0) {
      st_release(&st[b], ep | kFlagPre | agg);
    } else {
      st_release(&st[b], ep | kFlagAgg | agg);
      int64_t j = c - 1;
      long long spins = 0;
      for (;;) {
        const unsigned long long w = ld_acquire(&a.status[(size_t)j * kMaxK + b]);
        if ((w & ~((1ULL << 48) - 1)) == ep && (w & (3ULL << 46))) {
          excl += w & kValMask;
          if (w & kFlagPre) break;
          --j;
          continue;
        }
        if (++spins > a.spin_limit) {
          atomicExch(&a.run->error, -4);
          atomicExch(&a.run->where, 1);
          break;
        }
        __nanosleep(64);
      }
      st_release(&st[b], ep | kFlagPre | (excl + agg));
    }
    unsigned long long run = excl;
#pragma unroll
    for (int q = 0; q < kChunkTiles; ++q) {
      if (q < cnt) {
        a.tile_off[(size_t)(tb + q) * kMaxK + b] = (uint32_t)run;
        run += h[q];
      }
    }
  }
}

// The tile staged in bucket order, and the block's ranking state.
template <class K>
struct ScatterSmem {
  typename KT<K>::Bits stage[kTile];
  unsigned char sbid[kTile];
  unsigned short wcnt[kSWarps][kMaxK];
  unsigned int peer[kSWarps][kMaxK];   // lanes of the current step per bucket (kept zero between steps)
  int tile_start[kMaxK];
  int tile_tot[kMaxK];
  long long gbase[kMaxK];
};

// Stable scatter of every tile of the level: each block owns a contiguous
// range of tiles; 512 threads, 8 keys each, read straight into registers.
template <class K>
__global__ void __launch_bounds__(kScatterThreads, 2) k_scatter(LevelArgs a) {
  using T = KT<K>;
  using Bits = typename T::Bits;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem<K>& sh = *reinterpret_cast<ScatterSmem<K>*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // an earlier kernel gave up (bounded wait): move nothing, so that every
  // key of the level stays in its source buffer for the host to restore
  if (*reinterpret_cast<volatile int32_t*>(&a.run->error) != 0) {
    // the first level that moved nothing (its keys are where its records say)
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&a.run->error_level, 0, a.level + 1);
    return;
  }
  const int64_t nt = level_ntiles(a);
  for (int i = threadIdx.x; i < kSWarps * kMaxK; i += blockDim.x) (&sh.peer[0][0])[i] = 0u;
  // groups of kScatterGrab tiles from a level-wide ticket: tiles of skipped
  // subproblems cost nothing and the last tile of a subproblem is short, so
  // a fixed share per block would leave the level waiting for the slowest
  unsigned* const ticket = &a.ctl->tile_ticket[1];
  __shared__ long long s_tg;
  for (;;) {
  __syncthreads();  // the previous group is done before the ticket is read again
  if (threadIdx.x == 0) s_tg = (long long)atomicAdd(ticket, (unsigned)kScatterGrab);
  __syncthreads();
  const int64_t tg = s_tg;
  if (tg >= nt) break;
  const int64_t tge = tg + kScatterGrab < nt ? tg + kScatterGrab : nt;
  for (int64_t t = tg; t < tge; ++t) {
    const int s = a.tile2sub[t];
    const Sub sub = a.subs[s];
    if (sub.flags & kSkipScatter) continue;
    __syncthreads();
    for (int i = threadIdx.x; i < kSWarps * kMaxK; i += blockDim.x) (&sh.wcnt[0][0])[i] = 0;
    const int64_t ti = t - sub.tile0;
    const int64_t kbase = sub.off + ti * kTile;
    const int64_t rem = sub.n - ti * kTile;
    const int tn = rem < kTile ? (int)rem : kTile;
    const Bits* src = keys_of<const Bits>(sub.buf, sub.ubase, a.buf) + kbase;
    const uint8_t* ids = a.bids + kbase;
    Bits v[kSKPT];
    unsigned int br[kSKPT];   // bucket id, then bucket << 16 | rank within warp
#pragma unroll
    for (int j = 0; j < kSKPT; ++j) {
      const int i = warp * kSKPW + j * 32 + lane;
      v[j] = (i < tn) ? src[i] : Bits(0);
      br[j] = (i < tn) ? (unsigned)ids[i] : (unsigned)kMaxK;
    }
    __syncthreads();  // wcnt zeroed
#pragma unroll
    for (int j = 0; j < kSKPT; ++j) {
      const int bk = (int)br[j];
      const bool valid = bk < kMaxK;
      const int bq = valid ? bk : 0;
      // the lanes of this step with the same bucket: one shared OR each
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
    __syncthreads();
    if (threadIdx.x < kMaxK) {
      const int b = threadIdx.x;
      int run = 0;
#pragma unroll
      for (int w = 0; w < kSWarps; ++w) {
        const int x = sh.wcnt[w][b];
        sh.wcnt[w][b] = (unsigned short)run;
        run += x;
      }
      sh.tile_tot[b] = run;
    } else {
      // meanwhile: this tile's base of every bucket in the destination
      const int b = threadIdx.x - kMaxK;
      sh.gbase[b] = sub.off + a.bases[(size_t)s * 257 + b] + (long long)a.tile_off[(size_t)t * kMaxK + b];
    }
    __syncthreads();
    if (warp == 0) {
      // exclusive scan of the tile's bucket totals: 8 buckets per lane
      int loc[8];
      int sum = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) { loc[q] = sh.tile_tot[lane * 8 + q]; sum += loc[q]; }
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
      }
      int run = incl - sum;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        sh.tile_start[lane * 8 + q] = run;
        sh.gbase[lane * 8 + q] -= run;
        run += loc[q];
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kSKPT; ++j) {
      const int bk = (int)(br[j] >> 16);
      if (bk < kMaxK) {
        const int lp = sh.tile_start[bk] + sh.wcnt[warp][bk] + (int)(br[j] & 0xFFFF);
        sh.stage[lp] = v[j];
        sh.sbid[lp] = (unsigned char)bk;
      }
    }
    __syncthreads();
    Bits* dst = keys_of<Bits>(1 - sub.buf, sub.ubase, a.buf) + sub.off;
    const uint64_t span = (uint64_t)sub.n;
    for (int i = threadIdx.x; i < tn; i += blockDim.x) {
      const uint64_t p = (uint64_t)(sh.gbase[sh.sbid[i]] - sub.off + i);
      if (p < span) dst[p] = sh.stage[i];
    }
  }
  }
}

// ---------------------------------------------------------------------------
// After a level stopped on an error: copies the keys of every subproblem of
// the level that live in the scratch buffer back into the user buffer, so
// that the user buffer holds a permutation of its input.  One block per
// subproblem.
template <class Bits>
__global__ void k_restore(const Sub* subs, const Bits* scratch) {
  const Sub sub = subs[blockIdx.x];
  if (sub.buf != 1) return;
  Bits* user = reinterpret_cast<Bits*>(sub.ubase);
  for (int64_t i = threadIdx.x; i < sub.n; i += blockDim.x) user[sub.off + i] = scratch[sub.off + i];
}

cudaError_t launch_restore(const Sub* subs, int32_t nsub, int dtype, const void* scratch, cudaStream_t s) {
  if (nsub <= 0) return cudaSuccess;
  if (dtype == 0 || dtype == 2)
    k_restore<unsigned long long><<<nsub, 256, 0, s>>>(subs, reinterpret_cast<const unsigned long long*>(scratch));
  else
    k_restore<unsigned int><<<nsub, 256, 0, s>>>(subs, reinterpret_cast<const unsigned int*>(scratch));
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
__global__ void k_init_tiles(int32_t* tile2sub, int64_t ntiles, int32_t value) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ntiles;
       i += (int64_t)gridDim.x * blockDim.x)
    tile2sub[i] = value;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <class F>
static cudaError_t by_dtype(int dtype, F f) {
  switch (dtype) {
    case 0: return f((double*)nullptr);
    case 1: return f((float*)nullptr);
    case 2: return f((unsigned long long*)nullptr);
    case 3: return f((unsigned int*)nullptr);
  }
  return cudaErrorInvalidValue;
}

// The dynamic shared memory of k_fit and k_check depends on the level's
// largest sample; their limit is set once to the largest any call can ask
// for (a root sample of 16384 keys), never lowered, since it is a property of
// the kernel shared by every thread and stream of the process.
constexpr int kRootSampleMax = 16384;
template <class K>
size_t fit_smem_max() {
  return (size_t)kRootSampleMax * sizeof(typename KT<K>::Ord);
}

// Device-driven levels (a.cnt set) launch a fixed grid over the level's
// capacity; the kernels loop over the subproblems the device counted.
static int64_t loop_grid(const LevelArgs& a, int64_t per_block, int64_t fixed) {
  const int64_t need = (a.nsub + per_block - 1) / per_block;
  return a.cnt ? (need < fixed ? need : fixed) : need;
}

cudaError_t launch_fit(const LevelArgs& a, cudaStream_t s, int max_sample, int sms) {
  if (a.nsub <= 0) return cudaSuccess;
  return by_dtype(a.dtype, [&](auto* tag) {
    using K = std::remove_pointer_t<decltype(tag)>;
    using Ord = typename KT<K>::Ord;
    if (a.cnt || warp_fits(a, a.nsub)) {
      const size_t wsmem = (size_t)kFitWarpsG * kResidentSample * sizeof(Ord);
      cudaFuncSetAttribute(k_fit_warp<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem);
      k_fit_warp<K><<<(unsigned)loop_grid(a, kFitWarpsG, (int64_t)sms * 4), kFitWarpsG * 32, wsmem, s>>>(a);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
      if (!a.cnt && max_sample <= kResidentSample && a.pl2_leaves == 0) return cudaSuccess;  // all went to warps
    }
    size_t smem = (size_t)max_sample * sizeof(Ord);
    if (a.pl2_leaves > 0 && max_sample <= kPL2MaxSample)
      smem = ((smem + 15) & ~(size_t)15) + (size_t)kPL2MaxSample * 12;
    if (smem > fit_smem_max<K>()) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(k_fit<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fit_smem_max<K>());
    k_fit<K><<<(unsigned)loop_grid(a, 1, (int64_t)sms * 2), kFitThreads, smem, s>>>(a);
    return cudaGetLastError();
  });
}

cudaError_t launch_check(const LevelArgs& a, cudaStream_t s, int max_sample, int sms) {
  if (a.nsub <= 0) return cudaSuccess;
  return by_dtype(a.dtype, [&](auto* tag) {
    using K = std::remove_pointer_t<decltype(tag)>;
    const size_t smem = (size_t)max_sample * sizeof(typename KT<K>::Ord);
    if (smem > fit_smem_max<K>()) return cudaErrorInvalidValue;
    cudaFuncSetAttribute(k_check<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fit_smem_max<K>());
    k_check<K><<<(unsigned)loop_grid(a, 1, (int64_t)sms * 2), kFitThreads, smem, s>>>(a);
    return cudaGetLastError();
  });
}

static int resident_blocks(const void* fn, int threads, size_t smem, int sms) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess || per < 1) {
    cudaGetLastError();
    per = 1;
  }
  return per * sms;
}

cudaError_t launch_hist(const LevelArgs& a, cudaStream_t s, int rehist_only, int sms) {
  if (a.ntiles <= 0) return cudaSuccess;
  return by_dtype(a.dtype, [&](auto* tag) {
    using K = std::remove_pointer_t<decltype(tag)>;
    int g = resident_blocks((const void*)k_hist<K>, kPassThreads, 0, sms);
    if (g > a.ntiles) g = (int)a.ntiles;
    k_hist<K><<<g, kPassThreads, 0, s>>>(a, rehist_only);
    return cudaGetLastError();
  });
}

cudaError_t launch_scan(const LevelArgs& a, cudaStream_t s, int sms) {
  if (a.nsub <= 0) return cudaSuccess;
  return by_dtype(a.dtype, [&](auto* tag) {
    using K = std::remove_pointer_t<decltype(tag)>;
    k_scan<K><<<(unsigned)loop_grid(a, 1, (int64_t)sms * 8), 256, 0, s>>>(a);
    return cudaGetLastError();
  });
}

cudaError_t launch_tilescan(const LevelArgs& a, cudaStream_t s, int grid) {
  if (a.nchunks <= 0) return cudaSuccess;
  int g = grid;
  if (g > a.nchunks) g = (int)a.nchunks;
  k_tilescan<<<g, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_scatter(const LevelArgs& a, cudaStream_t s, int grid) {
  if (a.ntiles <= 0) return cudaSuccess;
  return by_dtype(a.dtype, [&](auto* tag) {
    using K = std::remove_pointer_t<decltype(tag)>;
    const size_t smem = sizeof(ScatterSmem<K>);
    cudaFuncSetAttribute(k_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int g = resident_blocks((const void*)k_scatter<K>, kScatterThreads, smem, grid);
    if (g > a.ntiles) g = (int)a.ntiles;
    k_scatter<K><<<g, kScatterThreads, smem, s>>>(a);
    return cudaGetLastError();
  });
}

cudaError_t launch_init_tiles(int32_t* tile2sub, int64_t ntiles, int32_t value, cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  int g = (int)((ntiles + 255) / 256);
  if (g > 4096) g = 4096;
  k_init_tiles<<<g, 256, 0, s>>>(tile2sub, ntiles, value);
  return cudaGetLastError();
}

}  // namespace ipls
