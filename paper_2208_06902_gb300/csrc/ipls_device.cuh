// Device building blocks of the learned partitioning pass.
//
//  * key traits: IEEE totalOrder keys ("ord"), binary64 values, exact
//    differences, fixed-point images of keys;
//  * SplitMix64 counter-based sampling (Steele, Lea and Flood 2014);
//  * a block-wide sorting network for samples and small runs, and a warp
//    LSD radix sort for the samples of block-resident tasks;
//  * the FMCD fit (Ch.3 "Linear Models", its listing) as a binary search over
//    the conflict-degree parameter D with a certified integer filter;
//  * classification by the clamped linear model (Ch.3 model equation) or by
//    the splitter tree with equality buckets (Ch.3 "Decision Trees");
//  * the PL2 learned CDF (training and classification);
//  * the slots of block-resident tasks in a level's group list.
#pragma once

#include <cfloat>
#include <cstdint>
#include <cuda_runtime.h>

#include "ipls_internal.h"

namespace ipls {

constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;

// ---------------------------------------------------------------------------
// SplitMix64 and the sample stream of one subproblem.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// Stream of the subproblem (seed, offset, size, level): one finaliser per
// field.  Sample j is output j+1 of a SplitMix64 generator seeded with it,
// mapped to [off, off+n) by a 64x64 multiply-high.
__device__ __forceinline__ uint64_t stream_key(uint64_t seed, int64_t off, int64_t n,
                                               int32_t level) {
  uint64_t t = mix64(seed + kGamma);
  t = mix64((t ^ (uint64_t)off) + kGamma);
  t = mix64((t ^ (uint64_t)n) + kGamma);
  t = mix64((t ^ (uint64_t)(uint32_t)level) + kGamma);
  return t;
}

__device__ __forceinline__ int64_t sample_offset(uint64_t stream, int64_t j, int64_t n) {
  const uint64_t r = mix64(stream + (uint64_t)(j + 1) * kGamma);
  return (int64_t)__umul64hi(r, (uint64_t)n);
}

// alpha*k - 1 sample keys with alpha = 0.2*floor(log2 n) (Ch.4), at least 3;
// the top level may override it.
__host__ __device__ __forceinline__ int64_t sample_size(int64_t n, int level, int k,
                                                       int64_t root_sample) {
  if (level == 0 && root_sample > 0) return root_sample;
#ifdef __CUDA_ARCH__
  const int64_t L = 63 - __clzll((long long)n);
#else
  const int64_t L = 63 - __builtin_clzll((unsigned long long)n);
#endif
  int64_t S = (L * k) / 5 - 1;
  return S < 3 ? 3 : S;
}

// ---------------------------------------------------------------------------
// Key traits.
// ---------------------------------------------------------------------------
template <class K> struct KT;

template <> struct KT<double> {
  using Bits = unsigned long long;
  using Ord = unsigned long long;
  static constexpr int W = 8;
  static constexpr int kMant = 52;   // low ord bits linear inside a binade
  static constexpr int kBias = 1075; // spacing of biased exponent e: 2^(max(e,1) - kBias)
  static constexpr int kExpMask = 0x7FF;
  __device__ static __forceinline__ Ord ord(Bits b) {
    return (b >> 63) ? ~b : (b | (1ULL << 63));
  }
  __device__ static __forceinline__ Bits unord(Ord u) {
    return (u >> 63) ? (u & ~(1ULL << 63)) : ~u;
  }
  __device__ static __forceinline__ double value(Bits b) { return __longlong_as_double((long long)b); }
  __device__ static __forceinline__ bool special(Bits b) { return ((b >> 52) & 0x7FF) == 0x7FF; }
  __device__ static __forceinline__ bool is_nan(Bits b) { return (b & ~(1ULL << 63)) > 0x7FF0000000000000ULL; }
  __device__ static __forceinline__ bool negative(Bits b) { return (b >> 63) != 0; }
  // a (-) b: one binary64 subtraction
  __device__ static __forceinline__ double diff(Bits a, Bits b) { return __dsub_rn(value(a), value(b)); }
  __device__ static __forceinline__ void mant_exp(Bits b, uint64_t& M, int& E, bool& neg) {
    const int e = (int)((b >> 52) & 0x7FF);
    const uint64_t m = b & 0xFFFFFFFFFFFFFULL;
    M = e ? (m | (1ULL << 52)) : m;
    E = (e ? e : 1) - 1075;
    neg = (b >> 63) != 0;
  }
};

template <> struct KT<float> {
  using Bits = unsigned int;
  using Ord = unsigned int;
  static constexpr int W = 4;
  static constexpr int kMant = 23;
  static constexpr int kBias = 150;
  static constexpr int kExpMask = 0xFF;
  __device__ static __forceinline__ Ord ord(Bits b) { return (b >> 31) ? ~b : (b | 0x80000000u); }
  __device__ static __forceinline__ Bits unord(Ord u) { return (u >> 31) ? (u & 0x7FFFFFFFu) : ~u; }
  __device__ static __forceinline__ double value(Bits b) { return (double)__uint_as_float(b); }
  __device__ static __forceinline__ bool special(Bits b) { return ((b >> 23) & 0xFF) == 0xFF; }
  __device__ static __forceinline__ bool is_nan(Bits b) { return (b & 0x7FFFFFFFu) > 0x7F800000u; }
  __device__ static __forceinline__ bool negative(Bits b) { return (b >> 31) != 0; }
  __device__ static __forceinline__ double diff(Bits a, Bits b) { return __dsub_rn(value(a), value(b)); }
  __device__ static __forceinline__ void mant_exp(Bits b, uint64_t& M, int& E, bool& neg) {
    const int e = (int)((b >> 23) & 0xFF);
    const uint64_t m = b & 0x7FFFFFu;
    M = e ? (m | (1u << 23)) : m;
    E = (e ? e : 1) - 150;
    neg = (b >> 31) != 0;
  }
};

template <class U, int WB> struct KTInt {
  using Bits = U;
  using Ord = U;
  static constexpr int W = WB;
  static constexpr int kMant = 0;    // integer keys: the value is linear in u
  static constexpr int kBias = 0;
  static constexpr int kExpMask = 0;
  __device__ static __forceinline__ Ord ord(Bits b) { return b; }
  __device__ static __forceinline__ Bits unord(Ord u) { return u; }
  __device__ static __forceinline__ double value(Bits b) { return __ull2double_rn((unsigned long long)b); }
  __device__ static __forceinline__ bool special(Bits) { return false; }
  __device__ static __forceinline__ bool is_nan(Bits) { return false; }
  __device__ static __forceinline__ bool negative(Bits) { return false; }
  // exact integer difference, rounded once to binary64
  __device__ static __forceinline__ double diff(Bits a, Bits b) {
    return a >= b ? __ull2double_rn((unsigned long long)(a - b))
                  : -__ull2double_rn((unsigned long long)(b - a));
  }
  __device__ static __forceinline__ void mant_exp(Bits b, uint64_t& M, int& E, bool& neg) {
    M = (uint64_t)b;
    E = 0;
    neg = false;
  }
};
template <> struct KT<unsigned long long> : KTInt<unsigned long long, 8> {};
template <> struct KT<unsigned int> : KTInt<unsigned int, 4> {};

// X(x) = x / 2^rho truncated toward zero, as int64; |X - x/2^rho| < 1.
// Saturates (sat = true, |X| = 2^62) when |x| >= 2^(62+rho).
template <class K>
__device__ __forceinline__ int64_t fixed_point(typename KT<K>::Bits b, int rho, bool& sat) {
  uint64_t M;
  int E;
  bool neg;
  KT<K>::mant_exp(b, M, E, neg);
  const int sh = E - rho;
  uint64_t U;
  sat = false;
  if (sh >= 0) {
    if (sh >= 62 || (M >> (62 - sh)) != 0) {
      sat = (M != 0);
      U = (M != 0) ? (1ULL << 62) : 0;
    } else {
      U = M << sh;
    }
  } else {
    const int r = -sh;
    U = (r >= 64) ? 0 : (M >> r);
    if (U >> 62) { sat = true; U = 1ULL << 62; }
  }
  const int64_t X = (int64_t)U;
  return neg ? -X : X;
}

// Smallest L with |x| < 2^L (kNoBits for x = 0): X(x) at rho = L - 61 stays
// below 2^61.  Integer operations only.
constexpr int kNoBits = -100000;
template <class K>
__device__ __forceinline__ int magnitude_bits(typename KT<K>::Bits b) {
  uint64_t M;
  int E;
  bool neg;
  KT<K>::mant_exp(b, M, E, neg);
  return M ? E + (64 - __clzll((long long)M)) : kNoBits;
}

// ---------------------------------------------------------------------------
// Cooperating groups: a whole block or a single warp.
// ---------------------------------------------------------------------------
struct BlockG {
  __device__ static __forceinline__ int tid() { return threadIdx.x; }
  __device__ static __forceinline__ int size() { return blockDim.x; }
  __device__ static __forceinline__ void sync() { __syncthreads(); }
  __device__ static __forceinline__ bool any(bool p) { return __syncthreads_or(p) != 0; }
};
// Bits of the lanes below this one.
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

struct WarpG {
  __device__ static __forceinline__ int tid() { return threadIdx.x & 31; }
  __device__ static __forceinline__ int size() { return 32; }
  __device__ static __forceinline__ void sync() { __syncwarp(); }
  __device__ static __forceinline__ bool any(bool p) { return __any_sync(0xffffffffu, p) != 0; }
};

// ---------------------------------------------------------------------------
// Sorting network on a shared-memory array a[0..n): a bitonic sorter whose
// merges open with the mirrored comparator, so every comparator puts the
// minimum at the lower index and positions >= n act as +infinity without
// being stored.  Every member of the group must call it.
// ---------------------------------------------------------------------------
template <class G, class T>
__device__ void group_sort(T* a, int n) {
  if (n <= 1) return;
  int P = 1, lp = 0;
  while (P < n) { P <<= 1; ++lp; }
  const int pairs = P >> 1;
  for (int ls = 1; ls <= lp; ++ls) {
    const int size = 1 << ls, lhalf = ls - 1, half = size >> 1;
    for (int t = G::tid(); t < pairs; t += G::size()) {
      const int blk = t >> lhalf, j = t & (half - 1);
      const int lo = blk * size + j, hi = blk * size + size - 1 - j;
      if (hi < n) {
        T x = a[lo], y = a[hi];
        if (y < x) { a[lo] = y; a[hi] = x; }
      }
    }
    G::sync();
    for (int lst = lhalf - 1; lst >= 0; --lst) {
      const int stride = 1 << lst;
      for (int t = G::tid(); t < pairs; t += G::size()) {
        const int lo = ((t >> lst) << (lst + 1)) + (t & (stride - 1));
        const int hi = lo + stride;
        if (hi < n) {
          T x = a[lo], y = a[hi];
          if (y < x) { a[lo] = y; a[hi] = x; }
        }
      }
      G::sync();
    }
  }
}

template <class T>
__device__ __forceinline__ void block_sort(T* a, int n) { group_sort<BlockG, T>(a, n); }

// One stable counting-sort pass of a warp radix sort: src[0..n) by the 8-bit
// digit ((key - lo) >> shift) & 255 into dst.  The in-warp rank of a key
// among the keys of its step with the same digit comes from a shared OR of
// lane bits; cnt holds the digit counts, peer is zero on entry and on exit.
template <int kSteps, class Ord>
__device__ __forceinline__ void radix_pass(const Ord* src, Ord* dst, unsigned* cnt, unsigned* peer, int n,
                                           Ord lo, int shift) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < 256; i += 32) cnt[i] = 0;
  __syncwarp();
  unsigned rk[kSteps];  // digit << 16 | rank among the equal digits before it
#pragma unroll
  for (int t = 0; t < kSteps; ++t) {
    if (t * 32 < n) {
      const int i = t * 32 + lane;
      const bool valid = i < n;
      const int d = valid ? (int)(((src[i] - lo) >> shift) & 255) : 0;
      if (valid) atomicOr(&peer[d], 1u << lane);
      __syncwarp();
      const unsigned pm = valid ? peer[d] : 0u;
      const int lt = __popc(pm & lanemask_lt());
      const unsigned base = cnt[d];
      rk[t] = ((unsigned)d << 16) | (base + (unsigned)lt);
      __syncwarp();
      if (valid && lt == 0) {
        cnt[d] = base + (unsigned)__popc(pm);
        peer[d] = 0u;
      }
      __syncwarp();
    }
  }
  {  // exclusive scan of the 256 digit counts, 8 per lane
    unsigned loc[8], sum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) { loc[q] = cnt[lane * 8 + q]; sum += loc[q]; }
    unsigned incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned x = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += x;
    }
    unsigned run = incl - sum;
#pragma unroll
    for (int q = 0; q < 8; ++q) { cnt[lane * 8 + q] = run; run += loc[q]; }
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < kSteps; ++t) {
    if (t * 32 < n) {
      const int i = t * 32 + lane;
      if (i < n) dst[cnt[rk[t] >> 16] + (rk[t] & 0xFFFFu)] = src[i];
    }
  }
  __syncwarp();
}

// Digits of the first try of warp_radix_sort (the highest ones).
constexpr int kRadixTop = 3;

// LSD radix sort of a[0..n) (n <= 32*kSteps) by one warp, on 8-bit digits of
// (key - min): a sample drawn from one subproblem spans a narrow range, so
// few passes are needed (none when all keys are equal).  tmp holds n more
// keys; cnt and peer are 256 words each, peer zero on entry and on exit.
// The passes run over the kRadixTop highest digits that some key sets
// first; keys whose top digits differ are then in order, and when every
// key is at most its right neighbour the array is sorted.  Otherwise (two
// keys that agree on the top digits were left out of order) every digit is
// sorted again, from the lowest.
template <int kSteps, class Ord>
__device__ void warp_radix_sort(Ord* a, Ord* tmp, unsigned* cnt, unsigned* peer, int n) {
  const int lane = threadIdx.x & 31;
  Ord lo = ~(Ord)0;
  for (int i = lane; i < n; i += 32) {
    const Ord v = a[i];
    lo = v < lo ? v : lo;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const Ord l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    lo = l2 < lo ? l2 : lo;
  }
  // bits set in some key minus lo (the smallest key has none): a digit that
  // is zero for every key leaves the order as it is, so its pass is skipped
  // (keys with trailing zero bits, such as integer-valued doubles, skip the
  // low digits)
  Ord vary = 0;
  for (int i = lane; i < n; i += 32) vary |= a[i] - lo;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) vary |= __shfl_xor_sync(0xffffffffu, vary, o);
  const int bits = vary == 0 ? 0 : (int)(sizeof(Ord) * 8) - (sizeof(Ord) == 8 ? __clzll((long long)vary) : __clz((int)vary));
  const int passes = (bits + 7) / 8;
  Ord* src = a;
  Ord* dst = tmp;
  // the lowest of the kRadixTop highest digits that some key sets
  int p0 = 0;
  for (int p = passes - 1, live = 0; p >= 0; --p) {
    if (((vary >> (8 * p)) & 255) == 0) continue;
    if (++live == kRadixTop) {
      p0 = p;
      break;
    }
  }
  for (;;) {
    for (int p = p0; p < passes; ++p) {
      if (((vary >> (8 * p)) & 255) == 0) continue;
      radix_pass<kSteps>(src, dst, cnt, peer, n, lo, 8 * p);
      Ord* sw = src;
      src = dst;
      dst = sw;
    }
    if (p0 == 0) break;
    bool bad = false;
    for (int i = lane; i + 1 < n; i += 32) bad = bad || src[i] > src[i + 1];
    if (!__any_sync(0xffffffffu, bad)) break;
    p0 = 0;
  }
  if (src != a) {
    for (int i = lane; i < n; i += 32) a[i] = src[i];
    __syncwarp();
  }
}

// Warp-wide bitonic sort of up to 32 values (one per lane; absent lanes hold
// the maximum value).  Returns this lane's value of the sorted sequence.
template <class T>
__device__ __forceinline__ T warp_sort32(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const T o = __shfl_xor_sync(0xffffffffu, v, stride);
      const bool up = ((lane & size) == 0);          // ascending block
      const bool lower = ((lane & stride) == 0);
      const bool take_min = (lower == up);
      v = take_min ? (o < v ? o : v) : (o < v ? v : o);
    }
  }
  return v;
}

// ---------------------------------------------------------------------------
// FMCD on the sorted sample so[0..N) (ord keys in shared memory).
//
// The loop of the paper's listing returns the smallest D >= 1 such that every
// window of D+1 consecutive sample points spans at least
// u_d(D) = (x[N-1-D] (-) x[D]) / (K-2), or, if no D with 3D <= N has that
// property, the first D with 3D > N together with u_d of the D before it.
// The property is monotone in D (the rounded gap grows with D, u_d shrinks),
// which is why the listing never moves its window start back; here it is
// found by binary search, one group reduction per probe.
//
// A probe first compares fixed-point images of the keys, which decide a
// window with certainty unless its gap lies within a few units of u_d; only
// those windows are re-checked with the binary64 subtraction.
// ---------------------------------------------------------------------------
struct FitShared {
  double ud;
  int rho;
  int filter;
  int linear;
  int pad;
};

// Fields of the same-binade estimate (LinModel::ufast ...).  q is the spacing
// of the binade of x_lo; ushift is chosen so that in-range keys (model value
// within nb + |Bc| + 1 of zero) have |D >> ushift| < 2^30 while keys with
// |D >> ushift| >= 2^30 are certainly clamped.  The bound ucabs covers the
// truncation by the shift (at most auf), the rounding of Bc and a margin;
// crel*|v| covers the binary32 roundings of D, auf and the fma (three units
// of 2^-24 and the binary64 model's own rounding, with room to spare).
// The estimate is used only when the whole sample (so[0] .. so[N-1]) lies in
// x_lo's binade, so that most keys take it; otherwise the fixed-point estimate
// alone serves.
template <class K>
__device__ void same_binade_model(typename KT<K>::Bits xlo, typename KT<K>::Ord s_first,
                                  typename KT<K>::Ord s_last, int nb, double A, double Bc, LinModel* m) {
  using T = KT<K>;
  int ok = !T::special(xlo);
  const typename T::Ord ulo = T::ord(xlo);
  if (T::kMant > 0)
    ok = ok && ((s_first ^ ulo) >> T::kMant) == 0 && ((s_last ^ ulo) >> T::kMant) == 0;
  else
    ok = ok && (uint64_t)(s_last - s_first) < (1ULL << 62);
  double q = 1.0;
  if (T::kMant > 0) {
    const int e = (int)(((uint64_t)xlo >> T::kMant) & T::kExpMask);
    q = ldexp(1.0, (e ? e : 1) - T::kBias);
  }
  const double aq = __dmul_rn(A, q);  // exact: q is a power of two (unless it underflows)
  ok = ok && isfinite(aq) && aq >= DBL_MIN;
  const double width = ok ? __dmul_rn(__ddiv_ru(__dadd_ru((double)nb + 1.0, fabs(Bc)), aq), 1.0 + 0x1.0p-50) : 0.0;
  ok = ok && isfinite(width);
  int s = ok ? ilogb(width) + 1 - 29 : 0;
  if (s < 0) s = 0;
  const double a2s = ldexp(aq, s);
  const float auf = __double2float_rn(a2s);
  ok = ok && s < 64 && auf >= FLT_MIN && isfinite(auf);
  const float ucabs = __double2float_ru((fabs(Bc) * 0x1.0p-21 + 2.0 * a2s + 0x1.0p-40) * (1.0 + 0x1.0p-20));
  ok = ok && ucabs < 0x1.0p-8f;
  m->ufast = ok;
  m->ushift = s;
  m->auf = auf;
  m->ucabs = ucabs;
}

// Fields of the uncentred estimate (LinModel::gfast ...), float keys only.
// With xf the key truncated to binary32 (23 mantissa bits; exact for f32
// keys), B = Bc - A x_lo in binary64 and v_f = RN32(RN32(A) xf + RN32(B)):
//   |v_f - v64| <= |A||xf|(2^-23 + 2^-24)(1 + 2^-22)   (truncation, RN32(A))
//                + 2^-23 |B| + 2^-23 |v_f|              (RN32(B), the fma)
//                + 2^-52 |A| (|xf| + |x_lo|) + 2^-53 |v64| (the binary64 model's
//                                                       own roundings)
// so gc1 = |A| 2^-21.9, crel = 2^-21 and gcabs = 2^-22 |B| + 2^-51 |A x_lo|
// + 2^-40 (rounded up) bound it, and the FP32 evaluation of the bound and of
// v_f +- del stays within the margin.  Used only when the bound at the
// sample's extremes stays below 2^-8 of a bucket.
template <class K>
__device__ void uncentred_model(typename KT<K>::Bits xlo, typename KT<K>::Bits s_first,
                                typename KT<K>::Bits s_last, double A, double Bc, LinModel* m) {
  using T = KT<K>;
  m->gfast = 0;
  m->gaf = m->gbf = m->gc1 = m->gcabs = 0.0f;
  m->gpad = 0;
  if (T::kMant == 0 || T::special(xlo)) return;
  const double x0 = T::value(xlo);
  const double B = __fma_rn(-A, x0, Bc);
  const float gaf = __double2float_rn(A), gbf = __double2float_rn(B);
  const double c1 = fabs(A) * 0x1.1p-22 * (1.0 + 0x1.0p-20);
  const float gc1 = __double2float_ru(c1);
  const float gcabs = __double2float_ru((fabs(B) * 0x1.0p-22 + fabs(A * x0) * 0x1.0p-51 + 0x1.0p-40) *
                                        (1.0 + 0x1.0p-20));
  const double xm = fmax(fabs(T::value(s_first)), fabs(T::value(s_last)));
  const bool ok = isfinite(B) && isfinite(gaf) && isfinite(gbf) && isfinite(gc1) && gaf != 0.0f &&
                  isfinite(xm) && (double)gc1 * xm + gcabs < 0x1.0p-8;
  if (!ok) return;
  m->gfast = 1;
  m->gaf = gaf;
  m->gbf = gbf;
  m->gc1 = gc1;
  m->gcabs = gcabs;
}

// One probe: does every window of D+1 consecutive sample points span at
// least u_d(D)?  The thresholds of the fixed-point test come from the
// fixed-point span q[N-1-D] - q[D]: with |q(x) - x/2^rho| < 1 and binary64
// rounding errors of at most 2^-53 per operation, a window whose image gap
// dq reaches t_hi certainly passes and one below t_lo certainly fails (the
// margins cover both the truncations and the roundings).  Only windows in
// between are decided with u_d and the gap computed in binary64.
// q, when given, holds the sample's fixed-point images (q[i] = X(so[i]) at
// fs.rho), computed once per fit instead of once per window and probe.
template <class K>
__device__ __forceinline__ long long fixed_of(const typename KT<K>::Ord* so, const long long* q, int i,
                                              int rho) {
  if (q) return q[i];
  bool sat;
  return fixed_point<K>(KT<K>::unord(so[i]), rho, sat);
}

template <class G, class K>
__device__ bool fmcd_probe(const typename KT<K>::Ord* so, const long long* q, int N, int D, int K_,
                           FitShared& fs) {
  using T = KT<K>;
  int fail = 0, amb = 0;
  const int W = N - D;  // windows i = 0 .. N-1-D
  const int filter = fs.filter;
  const int rho = fs.rho;
  long long t_lo = -1, t_hi = 0;
  if (filter) {
    const long long Sq = fixed_of<K>(so, q, N - 1 - D, rho) - fixed_of<K>(so, q, D, rho);
    const long long km2 = K_ - 2;
    const long long marg = (Sq >> 48) + 8;
    t_hi = (Sq + 2 + marg) / km2 + 3;
    const long long lo_num = Sq - 2 - marg;
    t_lo = lo_num > 0 ? lo_num / km2 - 3 : -1;
    for (int i = G::tid(); i < W; i += G::size()) {
      const long long dq = fixed_of<K>(so, q, i + D, rho) - fixed_of<K>(so, q, i, rho);
      if (dq < t_lo) fail = 1;
      else if (dq < t_hi) amb = 1;
    }
  } else {
    amb = 1;
  }
  if (G::any(fail)) return false;
  if (!G::any(amb)) return true;
  if (G::tid() == 0)
    fs.ud = __ddiv_rn(T::diff(T::unord(so[N - 1 - D]), T::unord(so[D])), (double)(K_ - 2));
  G::sync();
  const double ud = fs.ud;
  if (amb) {
    for (int i = G::tid(); i < W; i += G::size()) {
      if (filter) {
        const long long dq = fixed_of<K>(so, q, i + D, rho) - fixed_of<K>(so, q, i, rho);
        if (dq < t_lo || dq >= t_hi) continue;
      }
      if (!(T::diff(T::unord(so[i + D]), T::unord(so[i])) >= ud)) { fail = 1; break; }
    }
  }
  return !G::any(fail);
}

// Fits the linear model of one subproblem from its sorted sample (every
// member of the group calls it).  m->kind = kLinear, or kSplitter when the
// sample's extremes are equal or not finite or FMCD degenerates (u_d <= 0
// or not finite, A or Bc not finite); the FMCD fields are kept either way.
template <class G, class K>
__device__ void fit_linear(const typename KT<K>::Ord* so, int N, int K_, LinModel* m, FitShared& fs,
                           long long* q = nullptr) {
  using T = KT<K>;
  using Bits = typename T::Bits;
  if (G::tid() == 0) {
    const Bits first = T::unord(so[0]), last = T::unord(so[N - 1]);
    const bool lin = (so[0] != so[N - 1]) && !T::special(first) && !T::special(last);
    fs.linear = lin ? 1 : 0;
    m->kind = kSplitter;
    m->nb = K_;
    m->capped = 0;
    m->fast = 0;
    m->S = N;
    m->D = 0;
    m->A = 0.0;
    m->Bc = 0.0;
    m->ud = 0.0;
    m->xlo_bits = 0;
    m->rho = 0;
    m->qlo = 0;
    m->ufast = 0;
    m->ushift = 0;
    m->auf = 0.0f;
    m->ucabs = 0.0f;
    m->gfast = 0;
    m->gaf = m->gbf = m->gc1 = m->gcabs = 0.0f;
    m->gpad = 0;
    if (lin) {
      // certified filter: fixed point at rho = L - 61 with |x| < 2^L for every
      // sample key; off when the keys are all zero or so large that a
      // binary64 difference could overflow
      const int L1 = magnitude_bits<K>(first), L2 = magnitude_bits<K>(last);
      const int L = L1 > L2 ? L1 : L2;
      fs.filter = (L != kNoBits && L <= 1022) ? 1 : 0;
      fs.rho = fs.filter ? L - 61 : 0;
    }
  }
  G::sync();
  if (fs.linear && q && fs.filter) {  // fixed-point images, once
    for (int i = G::tid(); i < N; i += G::size()) {
      bool sat;
      q[i] = fixed_point<K>(T::unord(so[i]), fs.rho, sat);
    }
    G::sync();
  }
  if (!fs.filter) q = nullptr;
  if (fs.linear) {
    const int Dcap = N / 3 + 1;  // smallest D with 3D > N
    int D;
    int capped = 0;
    if (!fmcd_probe<G, K>(so, q, N, Dcap - 1, K_, fs)) {
      capped = 1;
      D = Dcap;
    } else {
      int lo = 1, hi = Dcap - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (fmcd_probe<G, K>(so, q, N, mid, K_, fs)) hi = mid; else lo = mid + 1;
      }
      D = lo;
    }
    if (G::tid() == 0) {
      // the slope comes from u_d at D (or at D-1 after the 3D > N break)
      const int Du = capped ? Dcap - 1 : D;
      const double ud = __ddiv_rn(T::diff(T::unord(so[N - 1 - Du]), T::unord(so[Du])), (double)(K_ - 2));
      const double A = __ddiv_rn(1.0, ud);
      const Bits xhi = T::unord(so[N - 1 - D]), xlo = T::unord(so[D]);
      const double span = T::diff(xhi, xlo);
      const double prod = __dmul_rn(A, span);
      const double Bc = __dmul_rn(__dsub_rn((double)K_, prod), 0.5);
      m->D = D;
      m->capped = capped;
      m->ud = ud;
      m->A = A;
      m->Bc = Bc;
      m->xlo_bits = (uint64_t)xlo;
      const bool ok = isfinite(ud) && ud > 0.0 && isfinite(A) && isfinite(Bc);
      if (ok) {
        m->kind = kLinear;
        // fast path: rho so that the in-range half-width (nb+|Bc|)/A, bounded
        // above by (nb+|Bc|)*u_d*(1+2^-50), stays below 2^(rho+29)
        const double tmax = __dmul_rn(__dmul_rn(__dadd_rn((double)K_, fabs(Bc)), ud), 1.0 + 0x1.0p-50);
        int fast = isfinite(tmax) && tmax > 0.0;
        const int rho = fast ? ilogb(tmax) - 28 : 0;
        bool sat = false;
        const long long qlo = fast ? fixed_point<K>(xlo, rho, sat) : 0;
        if (sat || qlo >= (1LL << 61) || qlo <= -(1LL << 61)) fast = 0;
        const double a2r = ldexp(A, rho);
        const float af = __double2float_rn(a2r);
        if (!(af >= FLT_MIN) || !isfinite(af)) fast = 0;
        const double cabs_d = fabs(Bc) * 0x1.0p-21 + 4.0 * a2r + 0x1.0p-40;
        const float cabs = __double2float_ru(cabs_d * (1.0 + 0x1.0p-20));
        if (!(cabs < 0x1.0p-8f)) fast = 0;
        m->fast = fast;
        m->rho = rho;
        m->qlo = qlo;
        m->af = af;
        m->bcf = __double2float_rn(Bc);
        m->crel = 0x1.0p-21f;
        m->cabs = cabs;
        same_binade_model<K>(xlo, so[0], so[N - 1], K_, A, Bc, m);
        uncentred_model<K>(xlo, T::unord(so[0]), T::unord(so[N - 1]), A, Bc, m);
      }
    }
  }
  G::sync();
}

// Splitter tree with equality buckets from the sorted sample: the (k-1)/2
// equidistant sample keys, deduplicated, so that the tree with equality
// buckets has at most k buckets.
template <class G, class K>
__device__ void build_splitters(const typename KT<K>::Ord* so, int N, int K_, Model* m) {
  if (G::tid() == 0) {
    const int want = (K_ - 1) / 2;
    int cnt = 0;
    for (int i = 0; i < want; ++i) {
      const uint64_t u = (uint64_t)so[(int64_t)(i + 1) * N / (want + 1)];
      if (cnt == 0 || m->split[cnt - 1] != u) m->split[cnt++] = u;
    }
    m->l.kind = kSplitter;
    m->l.fast = 0;
    m->nsplit = cnt;
    m->l.nb = 2 * cnt + 1;
  }
  G::sync();
}

template <class G, class K>
__device__ void fit_model(const typename KT<K>::Ord* so, int N, int K_, Model* m, FitShared& fs) {
  if (G::tid() == 0) m->nsplit = 0;
  fit_linear<G, K>(so, N, K_, &m->l, fs);
  if (m->l.kind == kSplitter) build_splitters<G, K>(so, N, K_, m);
}

// Splitter tree with equality buckets: p = #{s_i <= u}; bucket 2p-1 if
// s_p == u, else bucket 2p.
__device__ __forceinline__ int splitter_bucket(uint64_t u, const uint64_t* split, int nsplit) {
  int lo = 0, hi = nsplit;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (split[mid] <= u) lo = mid + 1; else hi = mid;
  }
  if (lo > 0 && split[lo - 1] == u) return 2 * lo - 1;
  return 2 * lo;
}

// The model equation in binary64 (reading: one fma, floor, clamp, cast).
template <class K>
__device__ __forceinline__ int classify_exact(typename KT<K>::Bits b, double A, double Bc,
                                              typename KT<K>::Bits xlo, int nb) {
  using T = KT<K>;
  if (T::is_nan(b)) return T::negative(b) ? 0 : nb - 1;
  const double d = T::diff(b, xlo);
  const double v = floor(__fma_rn(A, d, Bc));
  if (v < 0.0) return 0;
  if (v >= (double)nb) return nb - 1;
  return (int)v;
}

// Register copy of what one key's classification needs.
template <class K>
struct Classifier {
  using Bits = typename KT<K>::Bits;
  using Ord = typename KT<K>::Ord;
  int kind, nb, fast, rho, nsplit, ufast, ushift, gfast;
  long long qlo;
  float af, bcf, crel, cabs, auf, ucabs, gaf, gbf, gc1, gcabs;
  float nbm1f;      // nb - 1 as binary32
  float aufs;       // auf with the sign of x_lo's binade folded in (float keys)
  unsigned xl32, xh32;  // x_lo's bits, low and high words
  bool neg_binade;  // x_lo is negative (float keys)
  double A, Bc;
  Bits xlo;
  Ord ulo;
  const uint64_t* split;

  __device__ __forceinline__ void load(const LinModel& m, int exact_only) {
    kind = m.kind;
    nb = m.nb;
    fast = m.fast && !exact_only;
    rho = m.rho;
    qlo = m.qlo;
    af = m.af;
    bcf = m.bcf;
    crel = m.crel;
    cabs = m.cabs;
    A = m.A;
    Bc = m.Bc;
    xlo = (Bits)m.xlo_bits;
    ulo = KT<K>::ord(xlo);
    ufast = m.ufast && !exact_only;
    ushift = m.ushift;
    auf = m.auf;
    ucabs = m.ucabs;
    gfast = m.gfast && !exact_only;
    gaf = m.gaf;
    gbf = m.gbf;
    gc1 = m.gc1;
    gcabs = m.gcabs;
    nbm1f = (float)(nb - 1);
    neg_binade = KT<K>::kMant > 0 && KT<K>::negative(xlo);
    aufs = neg_binade ? -auf : auf;
    xl32 = (unsigned)(unsigned long long)xlo;
    xh32 = (unsigned)((unsigned long long)xlo >> 32);
    nsplit = 0;
    split = nullptr;
  }
  __device__ __forceinline__ void load(const Model& m, int exact_only) {
    load(m.l, exact_only);
    nsplit = m.nsplit;
    split = m.split;
  }

  // Fixed-point / FP32 evaluation; -1 when the certified interval around the
  // FP32 value contains a bucket boundary.
  __device__ __forceinline__ int fast_bucket(Bits b) const {
    using T = KT<K>;
    if (T::special(b)) return T::negative(b) ? 0 : nb - 1;
    bool sat;
    const long long X = fixed_point<K>(b, rho, sat);
    if (sat) return X > 0 ? nb - 1 : 0;
    const long long d = X - qlo;
    if (d >= (1LL << 30)) return nb - 1;
    if (d <= -(1LL << 30)) return 0;
    const float df = __int2float_rn((int)d);
    const float v = fmaf(af, df, bcf);
    const float del = fmaf(crel, fabsf(v), cabs);
    const float hi = v + del, lo = v - del;
    if (hi < 1.0f) return 0;
    if (lo >= (float)(nb - 1)) return nb - 1;
    const float fl = floorf(lo), fh = floorf(hi);
    if (fl == fh) return __float_as_int(fl + 8388608.0f) - 0x4B000000;
    return -1;
  }

  // The certified binary32 decision on an estimate v with bound del: the
  // bucket, or -1 when [v - del, v + del] contains a bucket boundary.
  __device__ __forceinline__ int decide(float v, float del) const {
    const float hi = v + del, lo = v - del;
    if (hi < 1.0f) return 0;
    if (lo >= (float)(nb - 1)) return nb - 1;
    const float fl = floorf(lo), fh = floorf(hi);
    if (fl == fh) return __float_as_int(fl + 8388608.0f) - 0x4B000000;
    return -1;
  }

  // Same-binade estimate from the order bits u of the key: -1 when the key
  // is not in x_lo's binade (or not within 2^62 of it, for integers) or the
  // certified interval contains a bucket boundary.
  __device__ __forceinline__ int ord_bucket(Ord u) const {
    using T = KT<K>;
    long long D;
    if (T::kMant > 0) {
      if (((u ^ ulo) >> T::kMant) != 0) return -1;  // another sign or exponent
      D = (long long)((uint64_t)u - (uint64_t)ulo); // |D| < 2^52: the wrap gives its sign
    } else {
      const uint64_t du = (uint64_t)u - (uint64_t)ulo;
      D = (long long)du;
      if ((u >= ulo) != (D >= 0)) return -1;        // |u - u_lo| >= 2^63
    }
    const long long Ds = D >> ushift;
    if (Ds >= (1LL << 30)) return nb - 1;
    if (Ds <= -(1LL << 30)) return 0;
    const float v = fmaf(auf, __int2float_rn((int)Ds), bcf);
    return decide(v, fmaf(crel, fabsf(v), ucabs));
  }

  // Uncentred estimate for float keys: -1 when the key's binary32
  // truncation is not a normal number or the certified interval contains a
  // bucket boundary.
  __device__ __forceinline__ int flt_bucket(Bits b) const {
    float xf;
    if (sizeof(Bits) == 8) {
      const unsigned long long u = (unsigned long long)b;
      const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
      const unsigned e = (hi >> 20) & 0x7FFu;
      if (e - 897u > 253u) return -1;  // beyond binary32's normal range (or inf/NaN)
      const unsigned mant = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;
      xf = __uint_as_float((hi & 0x80000000u) | ((e - 896u) << 23) | mant);
    } else {
      const unsigned u = (unsigned)b;
      const unsigned e = (u >> 23) & 0xFFu;
      if (e - 1u > 253u) return -1;
      xf = __uint_as_float(u);
    }
    const float v = fmaf(gaf, xf, gbf);
    return decide(v, fmaf(gc1, fabsf(xf), fmaf(crel, fabsf(v), gcabs)));
  }

  // decide() without branches: the bucket (valid when ok) and whether the
  // certified interval [v - del, v + del] holds no bucket boundary.  Both
  // ends are floored and clamped to [0, nb - 1] (clamp∘floor is monotone),
  // so equal results decide every point of the interval, the clamped ends
  // included.  v and del are finite here (keys they would not be finite
  // for are excluded by the caller's range checks).
  __device__ __forceinline__ int decide_bf(float v, float del, bool& ok) const {
    const float fl = fminf(fmaxf(floorf(v - del), 0.0f), nbm1f);
    const float fh = fminf(fmaxf(floorf(v + del), 0.0f), nbm1f);
    ok = fl == fh;
    return __float2int_rz(fl);
  }

  // ord_bucket() without branches, on the key's own bits.  Float keys: in
  // x_lo's binade the totalOrder difference is the raw-bits difference, with
  // its sign flipped for negative binades (folded into aufs); the shift
  // truncates toward -inf either way, within the same bound.  A shifted
  // difference beyond int32 lies far outside the model's range (|D >> s| >=
  // 2^31 > 2^30): clamped by its sign.  ok = false for a key outside the
  // binade (integers: whose difference from x_lo overflows) or whose
  // interval holds a boundary.
  __device__ __forceinline__ int ord_bf(Bits b, bool& ok) const {
    using T = KT<K>;
    if (T::kMant == 23) {
      // binary32: |bits - x_lo bits| < 2^23 in the binade
      const unsigned u = (unsigned)b, x = (unsigned)xlo;
      const bool in = ((u ^ x) >> 23) == 0;
      const int ds = (int)(u - x) >> ushift;
      const float v = fmaf(aufs, __int2float_rn(ds), bcf);
      bool okd;
      const int r = decide_bf(v, fmaf(crel, fabsf(v), ucabs), okd);
      ok = in && okd;
      return r;
    }
    unsigned dl, dh;
    bool in;
    if (T::kMant == 52) {
      // binary64 on 32-bit halves: same binade iff the top 12 bits agree
      const unsigned bl = (unsigned)(unsigned long long)b, bh = (unsigned)((unsigned long long)b >> 32);
      in = ((bh ^ xh32) >> 20) == 0;
      asm("sub.cc.u32 %0, %2, %3;\n\tsubc.u32 %1, %4, %5;" : "=r"(dl), "=r"(dh) : "r"(bl), "r"(xl32), "r"(bh), "r"(xh32));
    } else {
      const uint64_t du = (uint64_t)b - (uint64_t)ulo;
      dl = (unsigned)du;
      dh = (unsigned)(du >> 32);
      in = ((uint64_t)b >= (uint64_t)ulo) == ((long long)du >= 0);
    }
    // the low word of D >> s, and whether D >> s fits in it
    int ds;
    bool fits;
    if (ushift < 32) {
      ds = (int)__funnelshift_r(dl, dh, ushift);
      fits = ((int)dh >> ushift) == (ds >> 31);
    } else {
      ds = (int)dh >> (ushift - 32);
      fits = true;
    }
    const float v = fmaf(aufs, __int2float_rn(ds), bcf);
    bool okd;
    int r = decide_bf(v, fmaf(crel, fabsf(v), ucabs), okd);
    const bool above = ((int)dh >= 0) != neg_binade;  // the key's value is above x_lo's
    r = fits ? r : (above ? nb - 1 : 0);
    ok = in && (okd || !fits);
    return r;
  }

  // A refinement of bucket bk for ordering inside it: an index in [0, 8)
  // that never decreases as the key grows among the keys of bucket bk --
  // the eighth of [bk, bk + 1) the estimate of path 1 (same-binade) or 2
  // (uncentred) puts the key in, clamped; a key that estimate does not
  // cover takes the end it lies on (below or above x_lo's binade, beyond
  // int32 after the shift, or outside binary32's normal range, where zero
  // and the tiny values sit between the negative and the positive keys).
  // It only orders keys inside their (exact) bucket, so it needs no
  // certificate.
  __device__ __forceinline__ int sub8(Bits b, int bk, int path) const {
    using T = KT<K>;
    float v;
    if (path == 1) {
      bool cover;
      if (T::kMant == 23) {
        const unsigned u = (unsigned)b, x = (unsigned)xlo;
        cover = ((u ^ x) >> 23) == 0;
        v = fmaf(aufs, __int2float_rn((int)(u - x) >> ushift), bcf);
      } else {
        unsigned dl, dh;
        bool in;
        if (T::kMant == 52) {
          const unsigned bl = (unsigned)(unsigned long long)b, bh = (unsigned)((unsigned long long)b >> 32);
          in = ((bh ^ xh32) >> 20) == 0;
          asm("sub.cc.u32 %0, %2, %3;\n\tsubc.u32 %1, %4, %5;" : "=r"(dl), "=r"(dh) : "r"(bl), "r"(xl32), "r"(bh), "r"(xh32));
        } else {
          const uint64_t du = (uint64_t)b - (uint64_t)ulo;
          dl = (unsigned)du;
          dh = (unsigned)(du >> 32);
          in = ((uint64_t)b >= (uint64_t)ulo) == ((long long)du >= 0);
        }
        int ds;
        bool fits;
        if (ushift < 32) {
          ds = (int)__funnelshift_r(dl, dh, ushift);
          fits = ((int)dh >> ushift) == (ds >> 31);
        } else {
          ds = (int)dh >> (ushift - 32);
          fits = true;
        }
        cover = in && fits;
        v = fmaf(aufs, __int2float_rn(ds), bcf);
      }
      if (!cover) return T::ord(b) < ulo ? 0 : 7;
    } else {
      float xf;
      if (sizeof(Bits) == 8) {
        const unsigned long long u = (unsigned long long)b;
        const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
        const unsigned e = (hi >> 20) & 0x7FFu;
        const float inf = __uint_as_float((hi & 0x80000000u) | 0x7F800000u);
        const unsigned mant = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;
        xf = e < 897u ? 0.0f
             : e > 1150u ? inf
                         : __uint_as_float((hi & 0x80000000u) | ((e - 896u) << 23) | mant);
      } else {
        const unsigned u = (unsigned)b;
        const unsigned e = (u >> 23) & 0xFFu;
        xf = e == 0u ? 0.0f : e == 255u ? __uint_as_float((u & 0x80000000u) | 0x7F800000u) : __uint_as_float(u);
      }
      v = fmaf(gaf, xf, gbf);
    }
    const float t = fminf(fmaxf(floorf((v - (float)bk) * 8.0f), 0.0f), 7.0f);
    return (int)t;
  }

  // flt_bucket() without branches.
  __device__ __forceinline__ int flt_bf(Bits b, bool& ok) const {
    float xf;
    bool in;
    if (sizeof(Bits) == 8) {
      const unsigned long long u = (unsigned long long)b;
      const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
      const unsigned e = (hi >> 20) & 0x7FFu;
      in = e - 897u <= 253u;
      const unsigned mant = __funnelshift_l(lo, hi, 3) & 0x7FFFFFu;
      xf = __uint_as_float((hi & 0x80000000u) | ((e - 896u) << 23) | mant);
    } else {
      const unsigned u = (unsigned)b;
      const unsigned e = (u >> 23) & 0xFFu;
      in = e - 1u <= 253u;
      xf = __uint_as_float(u);
    }
    const float v = fmaf(gaf, xf, gbf);
    bool okd;
    const int r = decide_bf(v, fmaf(gc1, fabsf(xf), fmaf(crel, fabsf(v), gcabs)), okd);
    ok = in && okd;
    return r;
  }

  __device__ __forceinline__ int bucket(Bits b) const {
    if (kind == kSplitter) return splitter_bucket((uint64_t)KT<K>::ord(b), split, nsplit);
    if (ufast) {
      const int r = ord_bucket(KT<K>::ord(b));
      if (r >= 0) return r;
    } else if (gfast) {
      const int r = flt_bucket(b);
      if (r >= 0) return r;
    }
    if (fast) {
      const int r = fast_bucket(b);
      if (r >= 0) return r;
    }
    return classify_exact<K>(b, A, Bc, xlo, nb);
  }
  // The fixed-point / FP32 estimate when it decides, -1 when the key needs
  // the binary64 model (the caller may batch those), the full answer for
  // the splitter tree or when the estimate is off.
  __device__ __forceinline__ int bucket_or_defer(Bits b) const {
    if (kind == kSplitter) return splitter_bucket((uint64_t)KT<K>::ord(b), split, nsplit);
    if (ufast) {
      const int r = ord_bucket(KT<K>::ord(b));
      if (r >= 0) return r;
    } else if (gfast) {
      const int r = flt_bucket(b);
      if (r >= 0) return r;
    }
    if (fast) return fast_bucket(b);
    return classify_exact<K>(b, A, Bc, xlo, nb);
  }
  __device__ __forceinline__ int exact(Bits b) const { return classify_exact<K>(b, A, Bc, xlo, nb); }
};

// Tile positions of the keys of one warp whose bucket needs the binary64
// model, queued so that the FP64 instructions run with all 32 lanes busy
// (on this GPU an FP64 warp instruction costs the same with one active lane
// as with 32).
template <int kCap>
struct ExactQueue {
  unsigned short idx[kCap];
};

// ---------------------------------------------------------------------------
// PL2: two-level piecewise-linear CDF (learned CDF of Ch.2 "Learned Sort" /
// Ch.3 "Recursive Model Index", mean squared error against the empirical
// CDF as in Ch.3).  The root maps a key to fixed point X = trunc(x/2^rho)
// and to leaf j = (X - X0) >> sh of M equal-width leaves over the sample's
// range; leaf j interpolates between knot values y_j and y_{j+1}.
// Training: knots start at the empirical CDF, then kPL2Steps red-black sweeps
// of coordinate descent: every odd knot, then every even one, moves to the
// exact minimiser of the loss along its coordinate (y_j - G_j / H_j),
// clamped to [y_{j-1}, y_{j+1}] (0 and 1 at the ends); knots of one parity
// share no sample, so a half-sweep is parallel, the loss does not rise (in
// exact arithmetic) and the knots stay in [0, 1], non-decreasing.  Binary32
// throughout; every sum runs over sample indices in order (the samples of a
// leaf are contiguous), with one rounding per operation, so the model is the
// same bit for bit wherever it is computed.
// ---------------------------------------------------------------------------
struct PL2Scratch {
  int32_t* leaf;    // [S]
  float* w;         // [S]
  float* r;         // [S]
};

__device__ __forceinline__ int exponent_of(double r) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(r);
  const int e = (int)((b >> 52) & 0x7FF);
  return e == 0 ? -1022 : e - 1023;
}

// Geometry of a PL2 model from the sorted sample so[0..S) (thread 0 of the
// block; the result is read after a barrier): the fixed-point scale rho of
// the sample's range, X0 = X(sample minimum) and the leaf shift sh, so that
// leaf j = (X - X0) >> sh of M leaves covers the range.  *s_flag = 0 when the
// range cannot carry PL2 (equal or non-finite extremes, saturation).
template <class K>
__device__ void pl2_geometry(const typename KT<K>::Ord* so, int S, int M, int* s_flag, long long* s_x0,
                             int* s_rho, int* s_sh) {
  using T = KT<K>;
  *s_flag = 0;
  const typename T::Bits b0 = T::unord(so[0]), b1 = T::unord(so[S - 1]);
  if (so[0] != so[S - 1] && !T::special(b0) && !T::special(b1)) {
    const double range = T::diff(b1, b0);
    if (range > 0.0 && isfinite(range)) {
      const int rho = exponent_of(range) - 30;
      bool s0, s1;
      const long long X0 = fixed_point<K>(b0, rho, s0), X1 = fixed_point<K>(b1, rho, s1);
      if (!s0 && !s1) {
        int mlog = 0;
        while ((1 << mlog) < M) ++mlog;
        const unsigned long long umax = (unsigned long long)(X1 - X0);
        const int bl = umax == 0 ? 0 : 64 - __clzll((long long)umax);
        *s_sh = bl - mlog > 0 ? bl - mlog : 0;
        *s_rho = rho;
        *s_x0 = X0;
        *s_flag = 1;
      }
    }
  }
}

// Per-sample features (block-wide): the leaf of every sample and its position
// w in [0, 1) inside the leaf, then the first sample of every leaf (start[M]
// = S).  with_init: the knots start at the empirical CDF, y_j = start_j / S.
template <class K>
__device__ void pl2_features(const typename KT<K>::Ord* so, int S, int M, int rho, int sh, long long X0,
                             PL2Scratch sc, int* start, float* y, bool with_init) {
  using T = KT<K>;
  const int tid = threadIdx.x, nt = blockDim.x;
  const float inv = __int_as_float((127 - sh) << 23);  // 2^-sh
  for (int i = tid; i < S; i += nt) {
    bool sat;
    const long long U = fixed_point<K>(T::unord(so[i]), rho, sat) - X0;
    long long j = U >> sh;
    if (j > M - 1) j = M - 1;
    sc.leaf[i] = (int32_t)j;
    sc.w[i] = __fmul_rn(__ll2float_rn(U - (j << sh)), inv);
  }
  __syncthreads();
  // leaf starts: the first sample of every leaf (leaves are non-decreasing)
  for (int j = tid; j <= M; j += nt) {
    int lo = 0, hi = S;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sc.leaf[mid] < j) lo = mid + 1; else hi = mid;
    }
    start[j] = (j == M) ? S : lo;
    if (with_init) y[j] = __fdiv_rn((float)((j == M) ? S : lo), (float)S);
  }
  __syncthreads();
}

// Forward (block-wide): the model's CDF at every sample and its residual
// against the empirical CDF, r_i = F(x_i) - (i + 1/2)/S, binary32.
__device__ __forceinline__ void pl2_forward(int S, const PL2Scratch& sc, const float* y) {
  for (int i = threadIdx.x; i < S; i += blockDim.x) {
    const int a = sc.leaf[i];
    const float t1 = __fsub_rn(1.0f, sc.w[i]);
    const float F = __fadd_rn(__fmul_rn(y[a], t1), __fmul_rn(y[a + 1], sc.w[i]));
    const float tau = __fdiv_rn(__fadd_rn((float)i, 0.5f), (float)S);
    sc.r[i] = __fsub_rn(F, tau);
  }
}

// Backward for knot j (one thread): G_j = sum r_i dF(x_i)/dy_j and H_j =
// sum (dF(x_i)/dy_j)^2 over the samples of leaf j (weight 1 - w) then of
// leaf j-1 (weight w), in sample order; the loss gradient is 2 G_j / S and
// the loss is quadratic in y_j with curvature 2 H_j / S.
__device__ __forceinline__ void pl2_knot_gh(int j, int M, const PL2Scratch& sc, const int* start, float* G,
                                            float* H) {
  float g = 0.0f, h = 0.0f;
  if (j < M)
    for (int i = start[j]; i < start[j + 1]; ++i) {
      const float t1 = __fsub_rn(1.0f, sc.w[i]);
      g = __fadd_rn(g, __fmul_rn(sc.r[i], t1));
      h = __fadd_rn(h, __fmul_rn(t1, t1));
    }
  if (j > 0)
    for (int i = start[j - 1]; i < start[j]; ++i) {
      g = __fadd_rn(g, __fmul_rn(sc.r[i], sc.w[i]));
      h = __fadd_rn(h, __fmul_rn(sc.w[i], sc.w[i]));
    }
  *G = g;
  *H = h;
}

// Block-wide (all threads).  so[0..S) is the sorted sample (order bits).
// Returns false (m untouched) when the sample's range cannot carry PL2; else
// the knots y_0..y_M go to kout.  Training: kPL2Steps red-black sweeps, each
// half-sweep a forward pass over the samples and a backward step per knot of
// one parity (y_j -= G_j / H_j, clamped between its neighbours).
template <class K>
__device__ bool fit_pl2(const typename KT<K>::Ord* so, int S, int M, int K_, Model* m, float* kout,
                        PL2Scratch sc, float* y, int* start, int* s_flag, long long* s_x0,
                        int* s_rho, int* s_sh) {
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) pl2_geometry<K>(so, S, M, s_flag, s_x0, s_rho, s_sh);
  __syncthreads();
  if (!*s_flag) return false;
  const int rho = *s_rho, sh = *s_sh;
  const long long X0 = *s_x0;
  pl2_features<K>(so, S, M, rho, sh, X0, sc, start, y, true);
  for (int step = 0; step < kPL2Steps; ++step) {
    for (int parity = 1; parity >= 0; --parity) {
      pl2_forward(S, sc, y);
      __syncthreads();
      // the knots of this parity (they read only knots of the other one)
      for (int j = 2 * tid + parity; j <= M; j += 2 * nt) {
        float g, h;
        pl2_knot_gh(j, M, sc, start, &g, &h);
        if (h > 0.0f) {
          const float lo = j > 0 ? y[j - 1] : 0.0f, hi = j < M ? y[j + 1] : 1.0f;
          y[j] = fminf(fmaxf(__fsub_rn(y[j], __fdiv_rn(g, h)), lo), hi);
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    m->l.kind = kPL2;
    m->l.nb = K_;
    m->l.capped = 0;
    m->l.fast = 0;
    m->l.S = S;
    m->l.D = sh;
    m->l.rho = rho;
    m->l.qlo = X0;
    m->nsplit = M;
  }
  for (int j = tid; j <= M; j += nt) kout[j] = y[j];
  __syncthreads();
  return true;
}

// Per-model tables for classifying with a PL2 model: its binary32 knots
// (from the level's knot buffer) and the first bucket of every leaf.
__device__ __forceinline__ void pl2_tables(const Model& m, const float* knots, float* yf, int* lo,
                                           int nthreads_tid, int nthreads) {
  const int M = m.nsplit, K = m.l.nb;
  const float kf = (float)K;
  for (int j = nthreads_tid; j <= M; j += nthreads) {
    yf[j] = knots[j];
    int b = (int)floorf(__fmul_rn(yf[j], kf));
    lo[j] = b > K - 1 ? K - 1 : b;
  }
}

// Bucket under a PL2 model: floor(k F(x)) in binary32, clamped to the
// leaf's range [lo_j, lo_{j+1}], so monotone in x.
template <class K>
__device__ __forceinline__ int pl2_bucket(typename KT<K>::Bits b, const Model& m, const float* yf,
                                          const int* lo) {
  using T = KT<K>;
  const int K_ = m.l.nb, M = m.nsplit, sh = (int)m.l.D;
  if (T::is_nan(b)) return T::negative(b) ? 0 : K_ - 1;
  bool sat;
  const long long X = fixed_point<K>(b, m.l.rho, sat);
  if (sat) return X > 0 ? K_ - 1 : 0;
  const long long U = X - m.l.qlo;
  if (U < 0) return 0;
  const long long j = U >> sh;
  if (j >= M) return K_ - 1;
  const float inv = __int_as_float((127 - sh) << 23);  // 2^-sh
  const float w = __fmul_rn(__ll2float_rn(U - (j << sh)), inv);
  const float F = __fadd_rn(yf[j], __fmul_rn(__fsub_rn(yf[j + 1], yf[j]), w));
  int bk = (int)floorf(__fmul_rn(F, (float)K_));
  if (bk < lo[j]) bk = lo[j];
  if (bk > lo[j + 1]) bk = lo[j + 1];
  return bk;
}

// ---------------------------------------------------------------------------
// Exact thresholds of the linear model and the two-level index (ThrTable).
// ---------------------------------------------------------------------------
template <class K>
__device__ __forceinline__ int exact_bucket_ord(typename KT<K>::Ord u, const LinModel& m) {
  using T = KT<K>;
  return classify_exact<K>(T::unord(u), m.A, m.Bc, (typename T::Bits)m.xlo_bits, m.nb);
}

// An ord key near the value x_lo + (j - Bc) * u_d, where the model's value
// crosses j (a starting point only; the search below is exact).
template <class K>
__device__ __forceinline__ typename KT<K>::Ord threshold_estimate(int j, const LinModel& m) {
  using T = KT<K>;
  using Ord = typename T::Ord;
  const double x0 = T::value((typename T::Bits)m.xlo_bits);
  const double est = __fma_rn(__dsub_rn((double)j, m.Bc), m.ud, x0);
  if (!(est == est)) return T::ord((typename T::Bits)m.xlo_bits);
  if (T::kMant == 52) {
    return (Ord)T::ord((typename T::Bits)__double_as_longlong(est));
  } else if (T::kMant == 23) {
    return (Ord)T::ord((typename T::Bits)__float_as_uint(__double2float_rn(est)));
  } else {
    const double top = T::W == 8 ? 18446744073709551615.0 : 4294967295.0;
    if (est <= 0.0) return (Ord)0;
    if (est >= top) return (Ord)~(Ord)0;
    return (Ord)__double2ull_rz(est);
  }
}

// Smallest ord key u with bucket(u) >= j (1 <= j <= nb-1), by galloping from
// the estimate and bisection; the bucket map is monotone in u.
template <class K>
__device__ typename KT<K>::Ord exact_threshold(int j, const LinModel& m) {
  using Ord = typename KT<K>::Ord;
  const Ord top = ~(Ord)0;
  Ord u0 = threshold_estimate<K>(j, m);
  Ord lo, hi;
  if (exact_bucket_ord<K>(u0, m) >= j) {
    hi = u0;
    Ord step = 1;
    for (;;) {
      if (hi == 0) return 0;
      const Ord cand = hi > step ? hi - step : (Ord)0;
      if (exact_bucket_ord<K>(cand, m) < j) { lo = cand; break; }
      hi = cand;
      step = step << 1 ? step << 1 : step;
    }
  } else {
    lo = u0;
    Ord step = 1;
    for (;;) {
      if (lo == top) return top;
      const Ord cand = (Ord)(top - lo) > step ? (Ord)(lo + step) : top;
      if (exact_bucket_ord<K>(cand, m) >= j) { hi = cand; break; }
      lo = cand;
      step = step << 1 ? step << 1 : step;
    }
  }
  while ((Ord)(hi - lo) > 1) {  // bucket(lo) < j <= bucket(hi)
    const Ord mid = lo + (Ord)((hi - lo) / 2);
    if (exact_bucket_ord<K>(mid, m) >= j) hi = mid; else lo = mid;
  }
  return hi;
}

// Number of thresholds thr[1..nt] that are <= u (thr ascending).
__device__ __forceinline__ int count_le(const uint64_t* thr, int nt, uint64_t u) {
  int lo = 0, hi = nt;  // answer in [0, nt]
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (thr[mid] <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Builds the thresholds and the index of a linear model into `t` (shared
// memory), with every thread of the block.  t->ok = 0 when the index would
// not fit (the model is then evaluated directly).
template <class K>
__device__ void build_thr_table(const LinModel& m, ThrTable* t, int* scan_tmp) {
  using T = KT<K>;
  constexpr int MB = T::kMant;
  const int nb = m.nb, nt = nb - 1;
  for (int j = threadIdx.x; j <= kMaxK; j += blockDim.x) {
    if (j == 0) t->thr[0] = 0;
    else if (j <= nt) t->thr[j] = (uint64_t)exact_threshold<K>(j, m);
    else t->thr[j] = ~0ULL;
  }
  __syncthreads();
  __shared__ int s_nl1, s_ok, s_elo;
  if (threadIdx.x == 0) {
    s_ok = 1;
    if (MB > 0) {
      const int elo = (int)(t->thr[1] >> MB), ehi = (int)(t->thr[nt] >> MB);
      s_elo = elo;
      s_nl1 = ehi - elo + 1;
      if (s_nl1 > kL1Max) s_ok = 0;
      t->ishift = 0;
    } else {
      s_elo = 0;
      s_nl1 = 1;
      const uint64_t span = t->thr[nt] - t->thr[1];
      const int bits = span ? 64 - __clzll((long long)span) : 0;
      t->ishift = bits > 10 ? bits - 10 : 0;
    }
    t->e_lo = s_elo;
    t->n_l1 = s_nl1;
  }
  __syncthreads();
  if (!s_ok) {
    if (threadIdx.x == 0) t->ok = 0;
    __syncthreads();
    return;
  }
  const int nl1 = s_nl1, elo = s_elo;
  // sizes of the cell tables, per coarse entry (scan_tmp: kL1Max ints)
  for (int e = threadIdx.x; e < nl1; e += blockDim.x) {
    int size = 0;
    if (MB > 0) {
      const uint64_t lo_u = (uint64_t)(elo + e) << MB;
      const uint64_t hi_u = lo_u + ((1ULL << MB) - 1);
      const int c = count_le(t->thr, nt, hi_u) - count_le(t->thr, nt, lo_u);
      if (c > 0) {
        int mm = 2;
        while ((1 << mm) < 4 * c && mm < 10) ++mm;
        size = 1 << mm;
      }
    } else {
      size = (int)((t->thr[nt] - t->thr[1]) >> t->ishift) + 1;
    }
    scan_tmp[e] = size;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive scan (n_l1 <= 4096, once per subproblem)
    int run = 0;
    for (int e = 0; e < nl1; ++e) { const int x = scan_tmp[e]; scan_tmp[e] = run; run += x; }
    if (run > kL2Max) s_ok = 0;
  }
  __syncthreads();
  if (!s_ok) {
    if (threadIdx.x == 0) t->ok = 0;
    __syncthreads();
    return;
  }
  for (int e = threadIdx.x; e < nl1; e += blockDim.x) {
    const int off = scan_tmp[e];
    if (MB > 0) {
      const uint64_t lo_u = (uint64_t)(elo + e) << MB;
      const uint64_t hi_u = lo_u + ((1ULL << MB) - 1);
      const int b0 = count_le(t->thr, nt, lo_u);
      const int c = count_le(t->thr, nt, hi_u) - b0;
      if (c == 0) {
        t->l1[e] = (uint16_t)b0;
      } else {
        int mm = 2;
        while ((1 << mm) < 4 * c && mm < 10) ++mm;
        t->l1[e] = (uint16_t)(0x8000 | (mm << 11) | off);
      }
    } else {
      t->l1[0] = 0x8000;
    }
  }
  __syncthreads();
  // cells in parallel: each finds its entry by binary search over the offsets
  __shared__ int s_total;
  if (threadIdx.x == 0) {
    int total = 0;
    if (MB > 0) {
      const unsigned last = t->l1[nl1 - 1];
      total = scan_tmp[nl1 - 1] + ((last & 0x8000) ? (1 << ((last >> 11) & 15)) : 0);
    } else {
      total = (int)((t->thr[nt] - t->thr[1]) >> t->ishift) + 1;
    }
    s_total = total;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < s_total; q += blockDim.x) {
    if (MB > 0) {
      int lo = 0, hi = nl1 - 1;  // last entry with offset <= q and a cell table
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (scan_tmp[mid] <= q) lo = mid; else hi = mid - 1;
      }
      while (lo > 0 && !(t->l1[lo] & 0x8000)) --lo;  // entries without cells have size 0
      const unsigned ent = t->l1[lo];
      const int mm = (ent >> 11) & 15;
      const int k = q - scan_tmp[lo];
      const uint64_t lo_u = (uint64_t)(elo + lo) << MB;
      t->l2[q] = (uint8_t)count_le(t->thr, nt, lo_u + ((uint64_t)k << (MB - mm)));
    } else {
      t->l2[q] = (uint8_t)count_le(t->thr, nt, t->thr[1] + ((uint64_t)q << t->ishift));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) t->ok = 1;
  __syncthreads();
}

// Bucket of ord key u from the thresholds and their index (t->ok == 1).
template <class K>
__device__ __forceinline__ int table_bucket(typename KT<K>::Ord u, const ThrTable& t, int nb) {
  constexpr int MB = KT<K>::kMant;
  const uint64_t uu = (uint64_t)u;
  if (uu < t.thr[1]) return 0;
  if (uu >= t.thr[nb - 1]) return nb - 1;
  int g;
  if (MB > 0) {
    const unsigned ent = t.l1[(int)(uu >> MB) - t.e_lo];
    if (!(ent & 0x8000)) return (int)ent;
    const int mm = (ent >> 11) & 15, off = ent & 0x7FF;
    g = t.l2[off + (int)((uu >> (MB - mm)) & ((1u << mm) - 1))];
  } else {
    g = t.l2[(int)((uu - t.thr[1]) >> t.ishift)];
  }
  while (uu >= t.thr[g + 1]) ++g;
  return g;
}

// Reserves the tiles of a new grid subproblem of n keys, and the chunks of
// kChunkTiles tiles the look-back scan walks, in the next level's tile and
// chunk spaces; fills the Sub fields.  False (and ctl->overflow) when a
// capacity is exceeded.
// Slot of a new block-resident task in the level's group list: tasks of up
// to kTailSmall keys from the front, larger ones from the back (so each
// k_tail size launches exactly its own).  -1 when that end is full; the host
// also checks that the two ends did not meet.
__device__ __forceinline__ int group_slot(LevelCtl* ctl, int64_t n, int32_t cap) {
  if (n <= kTailSmall) {
    const int i = atomicAdd(&ctl->ngroups, 1);
    return i < cap ? i : -1;
  }
  const int j = atomicAdd(&ctl->ngroups_large, 1);
  return j < cap ? cap - 1 - j : -1;
}

__device__ __forceinline__ bool reserve_tiles(LevelCtl* ctl, int32_t idx, Sub& sub, int32_t* tile2sub,
                                              int64_t tile_cap, int32_t* chunk2sub,
                                              int64_t chunk_cap) {
  const int nt = (int)((sub.n + kTileKeys - 1) / kTileKeys);
  const int nc = (nt + kChunkTiles - 1) / kChunkTiles;
  const long long t0 = (long long)atomicAdd((unsigned long long*)&ctl->tiles_next, (unsigned long long)nt);
  const long long c0 = (long long)atomicAdd((unsigned long long*)&ctl->chunks_next, (unsigned long long)nc);
  if (t0 + nt > tile_cap || c0 + nc > chunk_cap || c0 + nc > 0x7FFFFFFFLL) {
    ctl->overflow = 1;
    return false;
  }
  atomicMax((unsigned long long*)&ctl->max_sub_n, (unsigned long long)sub.n);
  sub.tile0 = t0;
  sub.ntiles = nt;
  sub.chunk0 = (int32_t)c0;
  sub.nchunks = nc;
  for (int q = 0; q < nt; ++q) tile2sub[t0 + q] = idx;
  for (int q = 0; q < nc; ++q) chunk2sub[c0 + q] = idx;
  return true;
}


// Lanes of the warp holding the same bucket id (0..255) as this lane, from
// eight ballots (cheaper than a match instruction on this GPU); lanes with
// valid == false are in no set and get 0.
__device__ __forceinline__ unsigned same_bucket_lanes(int bk, bool valid) {
  unsigned peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
  for (int bit = 0; bit < 8; ++bit) {
    const bool on = (bk >> bit) & 1;
    const unsigned m = __ballot_sync(0xffffffffu, on);
    peers &= on ? m : ~m;
  }
  return valid ? peers : 0u;
}

}  // namespace ipls
