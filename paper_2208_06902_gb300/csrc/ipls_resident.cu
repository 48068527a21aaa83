// Block-resident IPLS: a group of small subproblems (consecutive buckets of
// one parent, or consecutive segments) is loaded into one block's shared
// memory once, the whole remaining recursion runs there -- sample, sort the
// sample, fit, classify, stable scatter, recurse (Ch.2 IPS4o recursion into
// independent buckets; Ch.4 IPLS) -- and the sorted keys are written to the
// user buffer once.  Subproblems of at most `cutoff` keys are base-cased:
// a warp-wide bitonic sort for up to 32 keys, a block-wide sorting network
// above that (the paper's base case is SkaSort for n <= 2^12, Ch.4; any exact
// sort gives the same, unique result).
#include "ipls_device.cuh"

namespace ipls {

constexpr int kRW = kResidentThreads / 32;  // warps
constexpr int kRKPT = kResidentMax / kResidentThreads;

template <class K>
struct ResSmem {
  typename KT<K>::Ord keys[kResidentMax];
  typename KT<K>::Ord samp[kResidentSample];
  unsigned short wcnt[kRW][kMaxK];
  unsigned long long tasks[kResidentTasks];  // small list from 0 up, stack from the top down
  int bstart[kMaxK + 1];
  int tot[kMaxK];
  Model model;
  FitShared fs;
  int nsmall, nstack, redo, err;
  unsigned long long popped;
  long long rec;
};

__device__ __forceinline__ unsigned long long enc_task(int start, int len, int level) {
  return ((unsigned long long)(unsigned)level << 32) | ((unsigned long long)start << 16) | (unsigned)len;
}
__device__ __forceinline__ int task_start(unsigned long long e) { return (int)((e >> 16) & 0xFFFF); }
__device__ __forceinline__ int task_len(unsigned long long e) { return (int)(e & 0xFFFF); }
__device__ __forceinline__ int task_level(unsigned long long e) { return (int)(e >> 32); }

// Base-cases every pending small range (all threads).
template <class K>
__device__ void flush_small(ResSmem<K>& sh) {
  using Ord = typename KT<K>::Ord;
  __syncthreads();
  const int ns = sh.nsmall;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int q = warp; q < ns; q += kRW) {
    const unsigned long long e = sh.tasks[q];
    const int st = task_start(e), len = task_len(e);
    if (len > 32) continue;
    Ord v = (lane < len) ? sh.keys[st + lane] : (Ord)~(Ord)0;
    v = warp_sort32(v);
    if (lane < len) sh.keys[st + lane] = v;
  }
  __syncthreads();
  for (int q = 0; q < ns; ++q) {
    const unsigned long long e = sh.tasks[q];
    if (task_len(e) > 32) block_sort(sh.keys + task_start(e), task_len(e));
  }
  __syncthreads();
  if (threadIdx.x == 0) sh.nsmall = 0;
  __syncthreads();
}

// Queues a child range: small ones for the base case, large ones on the stack.
template <class K>
__device__ __forceinline__ void push_child(ResSmem<K>& sh, int start, int len, int level, int cutoff) {
  if (len < 2) return;
  if (len <= cutoff) {
    const int i = atomicAdd(&sh.nsmall, 1);
    if (i < kResidentTasks / 2) sh.tasks[i] = enc_task(start, len, level);
    else sh.err = 1;
  } else {
    const int i = atomicAdd(&sh.nstack, 1);
    if (i < kResidentTasks / 2) sh.tasks[kResidentTasks - 1 - i] = enc_task(start, len, level);
    else sh.err = 1;
  }
}

// One learned partition pass on keys[s0, s0+c) inside shared memory.
template <class K>
__device__ void resident_pass(ResSmem<K>& sh, const ResidentArgs& a, int64_t goff, int s0, int c,
                              int level) {
  using T = KT<K>;
  using Ord = typename T::Ord;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // sample (with replacement) and sort it
  int S = (int)sample_size(c, level, a.k, a.root_sample);
  if (S > kResidentSample) {  // never planned by the host; keep the block in bounds
    if (threadIdx.x == 0) sh.err = 1;
    S = kResidentSample;
  }
  const uint64_t stream = stream_key(a.seed, goff + s0, c, level);
  for (int j = threadIdx.x; j < S; j += blockDim.x) sh.samp[j] = sh.keys[s0 + sample_offset(stream, j, c)];
  __syncthreads();
  block_sort(sh.samp, S);
  fit_model<K>(sh.samp, S, a.k, &sh.model, sh.fs);
  // each warp owns a contiguous chunk of the range, in 32-key steps
  const int chunk = ((c + kRW * 32 - 1) / (kRW * 32)) * 32;
  const int steps = chunk / 32;
  Ord v[kRKPT];
  unsigned int br[kRKPT];
  for (int attempt = 0; attempt < 2; ++attempt) {
    Classifier<K> cls;
    cls.load(sh.model, a.exact_only);
    for (int i = threadIdx.x; i < kRW * kMaxK; i += blockDim.x) (&sh.wcnt[0][0])[i] = 0;
    if (threadIdx.x == 0) sh.redo = 0;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kRKPT; ++j) {
      if (j < steps) {
        const int i = warp * chunk + j * 32 + lane;
        const bool ok = i < c;
        v[j] = ok ? sh.keys[s0 + i] : (Ord)0;
        const int bk = ok ? cls.bucket(T::unord(v[j])) : kMaxK;
        const unsigned peers = __match_any_sync(0xffffffffu, bk);
        const int lt = __popc(peers & lanemask_lt());
        const int leader = __ffs(peers) - 1;
        const int basec = (bk < kMaxK) ? sh.wcnt[warp][bk] : 0;
        br[j] = ((unsigned)bk << 16) | (unsigned)(basec + lt);
        __syncwarp();
        if (lane == leader && bk < kMaxK) sh.wcnt[warp][bk] = (unsigned short)(basec + __popc(peers));
        __syncwarp();
      }
    }
    __syncthreads();
    if (threadIdx.x < kMaxK) {
      const int b = threadIdx.x;
      int run = 0;
      for (int w = 0; w < kRW; ++w) {
        const int x = sh.wcnt[w][b];
        sh.wcnt[w][b] = (unsigned short)run;
        run += x;
      }
      sh.tot[b] = run;
      if (attempt == 0 && sh.model.kind == kLinear && run == c) sh.redo = 1;
    }
    __syncthreads();
    if (!sh.redo) break;
    // no progress: redo the pass with the splitter tree of the same sample
    if (threadIdx.x == 0) {
      Model& m = sh.model;
      const int want = (a.k - 1) / 2;
      int cnt = 0;
      for (int i = 0; i < want; ++i) {
        const uint64_t u = (uint64_t)sh.samp[(int64_t)(i + 1) * S / (want + 1)];
        if (cnt == 0 || m.split[cnt - 1] != u) m.split[cnt++] = u;
      }
      m.kind = kSplitter;
      m.nsplit = cnt;
      m.nb = 2 * cnt + 1;
      m.fast = 0;
    }
    __syncthreads();
  }
  // exclusive scan of the bucket totals (one warp, 8 values per lane)
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
    for (int q = 0; q < 8; ++q) { sh.bstart[lane * 8 + q] = run; run += loc[q]; }
    if (lane == 31) sh.bstart[kMaxK] = run;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kRKPT; ++j) {
    if (j < steps) {
      const int bk = (int)(br[j] >> 16);
      if (bk < kMaxK) sh.keys[s0 + sh.bstart[bk] + sh.wcnt[warp][bk] + (int)(br[j] & 0xFFFF)] = v[j];
    }
  }
  __syncthreads();
  const Model& m = sh.model;
  if (a.trace_cap > 0) {
    if (threadIdx.x == 0) {
      sh.rec = (long long)atomicAdd((unsigned long long*)&a.run->trace_count, 1ULL);
      if (sh.rec < a.trace_cap) {
        iplsTraceRecDev& r = a.trace[sh.rec];
        r.off = goff + s0; r.n = c; r.level = level; r.kind = m.kind; r.capped = m.capped;
        r.nbuckets = m.nb; r.S = m.S; r.D = m.D; r.A = m.A; r.Bc = m.Bc; r.ud = m.ud;
        r.xlo_bits = m.xlo_bits; r.nsplit = m.nsplit; r.where = 1;
      }
    }
    __syncthreads();
    if (sh.rec < a.trace_cap && threadIdx.x < kMaxK)
      a.trace[sh.rec].counts[threadIdx.x] = (threadIdx.x < m.nb) ? sh.tot[threadIdx.x] : 0;
  }
  if (threadIdx.x == 0) {
    atomicAdd((unsigned long long*)&a.run->resident_passes, 1ULL);
    if (m.kind == kSplitter) atomicAdd((unsigned long long*)&a.run->resident_fallback, 1ULL);
  }
  // children (equality buckets of the splitter tree are homogeneous: done)
  if (threadIdx.x < m.nb) {
    const int b = threadIdx.x;
    const bool eq = (m.kind == kSplitter) && (b & 1);
    if (!eq) push_child(sh, s0 + sh.bstart[b], sh.tot[b], level + 1, a.cutoff);
  }
  __syncthreads();
}

template <class K>
__global__ void __launch_bounds__(kResidentThreads, 2) k_resident(ResidentArgs a) {
  using T = KT<K>;
  using Bits = typename T::Bits;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ResSmem<K>& sh = *reinterpret_cast<ResSmem<K>*>(smem_raw);
  const Group g = a.groups[blockIdx.x];
  const Bits* src = reinterpret_cast<const Bits*>(a.buf[g.buf]) + g.off;
  for (int i = threadIdx.x; i < g.n; i += blockDim.x) sh.keys[i] = T::ord(src[i]);
  if (threadIdx.x == 0) { sh.nsmall = 0; sh.nstack = 0; sh.err = 0; }
  __syncthreads();
  const int64_t b0 = g.bounds[0];
  for (int q0 = 0; q0 < g.nchild; q0 += kMaxK) {
    if (sh.nsmall + kMaxK > kResidentTasks / 2) flush_small(sh);
    const int q = q0 + threadIdx.x;
    if (threadIdx.x < kMaxK && q < g.nchild) {
      const int st = (int)(g.bounds[q] - b0);
      const int len = (int)(g.bounds[q + 1] - g.bounds[q]);
      push_child(sh, st, len, g.level, a.cutoff);
    }
    __syncthreads();
  }
  for (;;) {
    __syncthreads();
    if (sh.nstack == 0 || sh.err) break;
    if (sh.nsmall + kMaxK > kResidentTasks / 2) flush_small(sh);
    __syncthreads();
    if (threadIdx.x == 0) {
      const int i = --sh.nstack;
      sh.popped = sh.tasks[kResidentTasks - 1 - i];
    }
    __syncthreads();
    const unsigned long long e = sh.popped;
    if (task_level(e) > 4096) {
      if (threadIdx.x == 0) { atomicExch(&a.run->error, -6); sh.nstack = 0; }
      continue;
    }
    resident_pass<K>(sh, a, g.off, task_start(e), task_len(e), task_level(e));
  }
  if (sh.err) {
    if (threadIdx.x == 0) atomicExch(&a.run->error, -6);
    if (threadIdx.x == 0) sh.nsmall = 0;
    __syncthreads();
  }
  flush_small(sh);
  Bits* dst = reinterpret_cast<Bits*>(a.buf[0]) + g.off;
  for (int i = threadIdx.x; i < g.n; i += blockDim.x) dst[i] = T::unord(sh.keys[i]);
  if (threadIdx.x == 0) {
    atomicAdd((unsigned long long*)&a.run->resident_keys, (unsigned long long)g.n);
    atomicAdd((unsigned long long*)&a.run->resident_groups, 1ULL);
  }
}

// Largest group a block can hold for this cutoff: every pending range of
// more than `cutoff` keys, plus one pass's worth of children, must fit in
// the task array.
int resident_rmax(int cutoff) {
  const long long lim = (long long)(kResidentTasks / 2) * (cutoff + 1);
  return lim < kResidentMax ? (int)lim : kResidentMax;
}

template <class Bits>
__global__ void k_fill(const Fill* fills, Bits* keys) {
  const Fill f = fills[blockIdx.x];
  const Bits v = (Bits)f.bits;
  for (int64_t i = threadIdx.x; i < f.n; i += blockDim.x) keys[f.off + i] = v;
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

cudaError_t launch_resident(const ResidentArgs& a, cudaStream_t s) {
  if (a.ngroups <= 0) return cudaSuccess;
  return by_dtype_r(a.dtype, [&](auto* tag) {
    using K = std::remove_pointer_t<decltype(tag)>;
    const size_t smem = sizeof(ResSmem<K>);
    cudaFuncSetAttribute(k_resident<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_resident<K><<<a.ngroups, kResidentThreads, smem, s>>>(a);
    return cudaGetLastError();
  });
}

cudaError_t launch_fill(const Fill* fills, int32_t nfill, int dtype, void* keys, cudaStream_t s) {
  if (nfill <= 0) return cudaSuccess;
  if (dtype == 0 || dtype == 2)
    k_fill<unsigned long long><<<nfill, 256, 0, s>>>(fills, reinterpret_cast<unsigned long long*>(keys));
  else
    k_fill<unsigned int><<<nfill, 256, 0, s>>>(fills, reinterpret_cast<unsigned int*>(keys));
  return cudaGetLastError();
}

}  // namespace ipls
