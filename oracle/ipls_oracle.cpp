// Serial CPU oracle of In-Place Parallel Learned Sort (IPLS), arxiv 2208.06902.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file; only the test suite, the smoke check and the timed CPU
// baseline of bench.py do.  It shares no code, header, table or constant
// generator with the CUDA library: every formula below is written out again
// from the paper.
//
// What it computes, and where the paper defines it:
//   * the partition model F(x) = clamp(floor(a*x + b), 0, k-1)
//       (Ch.3 "Linear Models", the model equation and the clamping rule);
//   * FMCD, the Fastest Minimum Conflict Degree fit (Ch.3 "Linear Models"),
//       from its definition (the smallest conflict-degree parameter D whose
//       windows all span the bucket width u_d(D)), in binary64;
//   * the IPLS pass: sample alpha*k-1 random keys with alpha = 0.2 log N and
//       k = 256, sort the sample, train FMCD, predict the bucket of every key
//       and move the keys into contiguous bucket regions (Ch.2 IPS4o section,
//       Ch.3 four phases, Ch.4 "Proposed Algorithm");
//   * recursion into every bucket as an independent subproblem, with a base
//       case below a size cutoff (Ch.2 IPS4o, Ch.4);
//   * the sampled-splitter decision tree with equality buckets (Ch.3
//       "Decision Trees") as the fallback when the linear model cannot split.
//
// Readings where the paper is silent or ambiguous (each one is listed, with
// its reason, in the design notes of the repository):
//   R1  FMCD arithmetic is binary64, not long double.
//   R2  When FMCD stops at 3D > N, the slope keeps the u_d of the D before
//       the stop (the paper's search leaves before recomputing it).
//   R3  The model is evaluated in the centred form
//         b(x) = clamp(floor(fma(A, x (-) x_lo, Bc)), 0, k-1),
//       x_lo = x[D], Bc = (K - A*(x[N-1-D] (-) x[D])) / 2, which equals
//       A*x + B of the listing in exact arithmetic; (-) is a binary64
//       subtraction for float keys and the exact integer difference rounded
//       once to binary64 for integer keys.
//   R4  One correctly rounded fma, then floor, then the clamp in binary64,
//       then the conversion to an integer bucket.  NaN keys go to bucket 0
//       when their sign bit is set and to bucket k-1 otherwise.
//   R5  alpha = 0.2*floor(log2 n): S = max(3, floor(floor(log2 n)*k/5) - 1);
//       the root may override S.
//   R6  k is the same at every level.
//   R7  Duplicates: a sample whose extremes are equal or not finite, a
//       degenerate FMCD result (u_d <= 0 or not finite, A not finite), or a
//       linear pass that puts every key into one bucket, re-partitions the
//       subproblem with the splitter tree with equality buckets built from
//       the same sorted sample.  An equality bucket is homogeneous and done.
//   R8  Keys keep their input order inside a bucket (stable scatter).
//   R9  Samples are drawn with replacement from a counter-based SplitMix64
//       stream keyed by (seed, offset, size, level); see sample_indices().
//
// Keys are ordered by IEEE 754 totalOrder for floats (-NaN < -inf < ... <
// -0 < +0 < ... < +inf < +NaN) and naturally for integers.
//
// Build: g++ -O2 -ffp-contract=off -fPIC -shared (no fast-math, no FMA
// contraction: every rounding is the one written here).

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

enum { OR_F64 = 0, OR_F32 = 1, OR_U64 = 2, OR_U32 = 3 };

// ---------------------------------------------------------------------------
// Configuration, model record and trace record (oracle-private layouts).
// ---------------------------------------------------------------------------
struct OracleCfg {
  int32_t k;            // buckets per pass (paper: 256, Ch.4)
  int32_t cutoff;       // subproblems of at most this many keys are base-cased
  int64_t root_sample;  // sample size at level 0; 0 = the alpha*k-1 formula
  uint64_t seed;        // seed of the sampling stream
  int32_t pl2_leaves;   // 0: FMCD everywhere; else PL2 with this many leaves
                        // (a power of two, 2..1024) for subproblems of more
                        // than kPL2MinKeys keys
  int32_t pl2_depth;    // PL2 only at levels below this (0: at every level)
};

// PL2 is used for subproblems larger than this (smaller ones keep FMCD).
const int64_t kPL2MinKeys = 8192;
// Samples longer than this keep FMCD (the device trains PL2 in shared memory).
const int64_t kPL2MaxSample = 4096;
// Training steps of PL2.
const int kPL2Steps = 8;

struct OracleModel {
  int32_t kind;     // 0 = FMCD linear model, 1 = splitter tree, 2 = homogeneous
  int32_t capped;   // FMCD left its loop at the 3D > N break (stale u_d)
  int64_t S;        // sample size
  int64_t D;        // conflict-degree parameter returned by FMCD
  double A;         // slope 1/u_d
  double Bc;        // centred intercept (K - A*span)/2
  double xlo;       // x[D]: the centre of the centred form (as binary64)
  uint64_t xlo_bits;  // x[D] as raw key bits (integer keys: the exact key)
  double B;         // the listing's own intercept (K - A*(x_hi + x_lo))/2
  double ud;        // the u_d the slope came from
  int32_t nsplit;   // splitter count (kind 1); leaves M (kind 2)
  int32_t nbuckets; // buckets of this pass: k, or 2*nsplit+1 for splitters
  uint64_t split[128];  // splitters as totalOrder bits, ascending, unique
                        // (kind 2 keeps its knots y_0..y_M beside the model)
  int32_t pl2_sh;   // kind 2: leaf width 2^sh in fixed-point units
  int32_t pl2_rho;  // kind 2: fixed-point scale, X(x) = trunc(x / 2^rho)
  int64_t pl2_x0;   // kind 2: X(x_0), the sample minimum
};

struct OracleTrace {
  int64_t off, n;
  int32_t level, pad;
  OracleModel model;
  int64_t counts[512];
};

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): golden-gamma increment
// followed by the 64-bit finaliser.  Used as a counter-based generator.
// ---------------------------------------------------------------------------
const uint64_t kGamma = 0x9e3779b97f4a7c15ULL;

uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

uint64_t mulhi64(uint64_t a, uint64_t b) {
  return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

// The stream of one subproblem: seed, offset, size and level folded in, one
// finaliser per field.  Sample j is the (j+1)-th SplitMix64 output of that
// stream, reduced to [0, n) by a multiply-high.
uint64_t stream_key(uint64_t seed, int64_t off, int64_t n, int32_t level) {
  uint64_t t = mix64(seed + kGamma);
  t = mix64((t ^ (uint64_t)off) + kGamma);
  t = mix64((t ^ (uint64_t)n) + kGamma);
  t = mix64((t ^ (uint64_t)(uint32_t)level) + kGamma);
  return t;
}

void sample_indices(uint64_t seed, int64_t off, int64_t n, int32_t level,
                    int64_t S, int64_t* idx) {
  uint64_t t = stream_key(seed, off, n, level);
  for (int64_t j = 0; j < S; ++j) {
    uint64_t r = mix64(t + (uint64_t)(j + 1) * kGamma);
    idx[j] = off + (int64_t)mulhi64(r, (uint64_t)n);
  }
}

// Sample size, reading R5 of alpha = 0.2 log N, S = alpha*k - 1 (Ch.4).
int64_t sample_size(int64_t n, int32_t level, const OracleCfg& cfg) {
  if (level == 0 && cfg.root_sample > 0) return cfg.root_sample;
  int64_t L = 0;
  while ((int64_t(1) << (L + 1)) <= n) ++L;  // floor(log2 n)
  int64_t S = (L * cfg.k) / 5 - 1;
  return S < 3 ? 3 : S;
}

// ---------------------------------------------------------------------------
// Key traits: totalOrder bits, value as binary64, exact difference.
// ---------------------------------------------------------------------------
template <class T> struct Key;

template <> struct Key<double> {
  static uint64_t ord(double x) {
    uint64_t b; std::memcpy(&b, &x, 8);
    return (b >> 63) ? ~b : (b | (uint64_t(1) << 63));
  }
  static uint64_t bits(double x) { uint64_t b; std::memcpy(&b, &x, 8); return b; }
  static double val(double x) { return x; }
  static bool is_nan(double x) { return std::isnan(x); }
  static bool neg_sign(double x) { return std::signbit(x); }
  static bool finite(double x) { return std::isfinite(x); }
  // a (-) b: one binary64 subtraction.
  static double diff(double a, double b) { return a - b; }
};

template <> struct Key<float> {
  static uint64_t ord(float x) {
    uint32_t b; std::memcpy(&b, &x, 4);
    return (b >> 31) ? (uint32_t)~b : (b | 0x80000000u);
  }
  static uint64_t bits(float x) { uint32_t b; std::memcpy(&b, &x, 4); return b; }
  static double val(float x) { return (double)x; }   // exact promotion
  static bool is_nan(float x) { return std::isnan(x); }
  static bool neg_sign(float x) { return std::signbit(x); }
  static bool finite(float x) { return std::isfinite(x); }
  static double diff(float a, float b) { return (double)a - (double)b; }
};

template <class U> struct IntKey {
  static uint64_t ord(U x) { return (uint64_t)x; }
  static uint64_t bits(U x) { return (uint64_t)x; }
  static double val(U x) { return (double)x; }
  static bool is_nan(U) { return false; }
  static bool neg_sign(U) { return false; }
  static bool finite(U) { return true; }
  // Exact integer difference, rounded once to binary64 (reading R3).
  static double diff(U a, U b) {
    return a >= b ? (double)(uint64_t)(a - b) : -(double)(uint64_t)(b - a);
  }
};
template <> struct Key<uint64_t> : IntKey<uint64_t> {};
template <> struct Key<uint32_t> : IntKey<uint32_t> {};

// ---------------------------------------------------------------------------
// FMCD (Ch.3 "Linear Models"), in binary64 (reading R1).
//
// x[0..N) is the sorted sample and K the number of buckets.  For a conflict
// degree parameter D the bucket width is u_d(D) = (x[N-1-D] (-) x[D])/(K-2),
// and D "holds" when every window of D+1 consecutive sample points spans at
// least u_d(D) (then no bucket of width u_d receives more than D+1 sample
// points).  FMCD returns the smallest D that holds; it stops looking once
// 3D > N, and then (reading R2) keeps the u_d of the D before the stop.
// The slope of the model is A = 1/u_d; the centred intercept is
// Bc = (K - A*(x[N-1-D] (-) x[D]))/2, and the uncentred intercept of the
// paper, B = (K - A*(x[N-1-D] + x[D]))/2, is kept for comparison.
// ---------------------------------------------------------------------------
template <class T>
double fmcd_width(const T* x, int64_t N, int32_t K, int64_t D) {
  return Key<T>::diff(x[N - 1 - D], x[D]) / (double)(K - 2);
}

// D holds: every window of D+1 consecutive points spans at least u_d(D).
template <class T>
bool fmcd_holds(const T* x, int64_t N, int32_t K, int64_t D) {
  const double ud = fmcd_width<T>(x, N, K, D);
  for (int64_t i = 0; i + D < N; ++i)
    if (!(Key<T>::diff(x[i + D], x[i]) >= ud)) return false;
  return true;
}

// The model record for a chosen D (capped: u_d is taken at D-1).
template <class T>
void fmcd_model(const T* x, int64_t N, int32_t K, int64_t D, int capped, OracleModel* m) {
  typedef Key<T> KT;
  const double ud = fmcd_width<T>(x, N, K, capped ? D - 1 : D);
  const double A = 1.0 / ud;
  const double span = KT::diff(x[N - 1 - D], x[D]);
  const double prod = A * span;
  const double sum = KT::val(x[N - 1 - D]) + KT::val(x[D]);
  const double prod2 = A * sum;
  m->kind = 0;
  m->capped = capped;
  m->S = N;
  m->D = D;
  m->ud = ud;
  m->A = A;
  m->Bc = ((double)K - prod) / 2.0;
  m->B = ((double)K - prod2) / 2.0;
  m->xlo = KT::val(x[D]);
  m->xlo_bits = KT::bits(x[D]);
  m->nsplit = 0;
  m->nbuckets = K;
}

// FMCD from its definition: try D = 1, 2, ... while 3D <= N.
template <class T>
void fmcd(const T* x, int64_t N, int32_t K, OracleModel* m) {
  const int64_t Dstop = N / 3 + 1;  // smallest D with 3D > N
  for (int64_t D = 1; D < Dstop; ++D)
    if (fmcd_holds<T>(x, N, K, D)) { fmcd_model<T>(x, N, K, D, 0, m); return; }
  fmcd_model<T>(x, N, K, Dstop, 1, m);
}

// The same result by one walk over the window starts, the way the paper's
// O(S) search finds it: a window that is too narrow for the current D raises
// D (and u_d) until it is wide enough, and the walk never steps back, since
// a window's span grows with D while u_d(D) does not (so a window that passed
// for a smaller D still passes).  Kept only to be checked against fmcd().
template <class T>
void fmcd_incremental(const T* x, int64_t N, int32_t K, OracleModel* m) {
  int64_t D = 1, start = 0;
  double ud = fmcd_width<T>(x, N, K, D);
  for (;;) {
    if (start + D >= N) { fmcd_model<T>(x, N, K, D, 0, m); return; }
    if (Key<T>::diff(x[start + D], x[start]) >= ud) { ++start; continue; }
    ++D;
    if (3 * D > N) { fmcd_model<T>(x, N, K, D, 1, m); return; }
    ud = fmcd_width<T>(x, N, K, D);
  }
}

// Model equation of Ch.3 "Linear Models" in the centred form (R3, R4).
template <class T>
int32_t linear_bucket(T x, const OracleModel& m, T xlo) {
  typedef Key<T> KT;
  const int32_t k = m.nbuckets;
  if (KT::is_nan(x)) return KT::neg_sign(x) ? 0 : k - 1;
  const double d = KT::diff(x, xlo);
  double v = std::fma(m.A, d, m.Bc);
  v = std::floor(v);
  if (v < 0.0) return 0;
  if (v >= (double)k) return k - 1;
  return (int32_t)v;
}

// Splitter tree with equality buckets (Ch.3 "Decision Trees"): with unique
// splitters s_1 < ... < s_m, bucket 2p for keys strictly between s_p and
// s_{p+1}, bucket 2p-1 for keys equal to s_p.
int32_t splitter_bucket(uint64_t u, const OracleModel& m) {
  int32_t p = 0;
  while (p < m.nsplit && m.split[p] <= u) ++p;   // p = #{s_i <= u}
  if (p > 0 && m.split[p - 1] == u) return 2 * p - 1;
  return 2 * p;
}

template <class T>
void build_splitters(const T* samp, int64_t S, int32_t k, OracleModel* m) {
  typedef Key<T> KT;
  const int64_t want = (k - 1) / 2;
  int32_t cnt = 0;
  for (int64_t i = 0; i < want; ++i) {
    uint64_t u = KT::ord(samp[(i + 1) * S / (want + 1)]);
    if (cnt == 0 || m->split[cnt - 1] != u) m->split[cnt++] = u;
  }
  m->kind = 1;
  m->nsplit = cnt;
  m->nbuckets = 2 * cnt + 1;
}

// ---------------------------------------------------------------------------
// PL2: a two-level piecewise-linear CDF model (the learned-CDF view of Ch.2
// "Learned Sort" and Ch.3 "Recursive Model Index", with the loss of Ch.3 --
// the mean squared error against the empirical CDF).  The root routes a key
// to one of M equal-width leaves of the sample's range; the leaves
// interpolate linearly between knot values y_0..y_M, so the CDF is
// continuous, and the knots are kept non-decreasing, so it is monotone
// (RMIs need not be; a bucket map must be).  Trained and evaluated in
// binary32.  Bucket = floor(k F(x)), clamped per leaf to
// [floor(k y_j), floor(k y_{j+1})].
// ---------------------------------------------------------------------------

// X(x) = trunc(x / 2^rho) as an integer, saturating (sat = true) when
// |x / 2^rho| >= 2^62.  Exact: scaling by a power of two, then truncation;
// integer keys use integer shifts.
template <class T> struct Fixed;
template <> struct Fixed<double> {
  static int64_t X(double x, int rho, bool& sat) {
    sat = false;
    if (std::isnan(x)) { sat = true; return 0; }
    const double v = std::ldexp(x, -rho);
    if (!(std::fabs(v) < 4611686018427387904.0)) { sat = true; return v > 0 ? (int64_t(1) << 62) : -(int64_t(1) << 62); }
    return (int64_t)std::trunc(v);
  }
};
template <> struct Fixed<float> {
  static int64_t X(float x, int rho, bool& sat) { return Fixed<double>::X((double)x, rho, sat); }
};
template <class U> struct FixedInt {
  static int64_t X(U x, int rho, bool& sat) {
    sat = false;
    const uint64_t u = (uint64_t)x;
    if (rho >= 0) {
      const uint64_t v = rho >= 64 ? 0 : (u >> rho);
      if (v >> 62) { sat = true; return int64_t(1) << 62; }
      return (int64_t)v;
    }
    const int l = -rho;
    if (l >= 62 || (u >> (62 - l)) != 0) { sat = u != 0; return u ? (int64_t(1) << 62) : 0; }
    return (int64_t)(u << l);
  }
};
template <> struct Fixed<uint64_t> : FixedInt<uint64_t> {};
template <> struct Fixed<uint32_t> : FixedInt<uint32_t> {};

// Unbiased exponent of a finite positive binary64 (denormals: -1022).
static int exponent_of(double r) {
  uint64_t b; std::memcpy(&b, &r, 8);
  const int e = (int)((b >> 52) & 0x7FF);
  return e == 0 ? -1022 : e - 1023;
}

static int bit_length(uint64_t v) {
  int b = 0;
  while (v) { ++b; v >>= 1; }
  return b;
}

// Per-sample features of PL2 on the sorted sample: leaf, position in it.
template <class R>
struct PL2Feat {
  std::vector<int32_t> leaf;
  std::vector<R> w;
  std::vector<int64_t> start;  // start[j]: first sample of leaf j; start[M] = S
};

// Fits PL2 on the sorted sample x[0..S) with M leaves, every operation in
// the arithmetic type R with one rounding each and every sum in sample order.
// R = float is the model the sort uses (binary32); R = double is the same
// training in binary64, kept as a reference for the loss it reaches.
// Returns false (and leaves m alone) when the sample's range cannot be used:
// equal or non-finite extremes (the duplicate rule takes over) or a range
// that does not fit the fixed point (FMCD takes over).
template <class T, class R>
bool pl2_train(const T* x, int64_t S, int32_t M, int32_t K, OracleModel* m, std::vector<R>* knots,
               PL2Feat<R>* feat_out, std::vector<double>* loss_trace) {
  typedef Key<T> KT;
  if (KT::ord(x[0]) == KT::ord(x[S - 1]) || !KT::finite(x[0]) || !KT::finite(x[S - 1])) return false;
  const double range = KT::diff(x[S - 1], x[0]);
  if (!(range > 0.0) || !std::isfinite(range)) return false;
  const int rho = exponent_of(range) - 30;
  bool s0, s1;
  const int64_t X0 = Fixed<T>::X(x[0], rho, s0);
  const int64_t X1 = Fixed<T>::X(x[S - 1], rho, s1);
  if (s0 || s1) return false;
  int mlog = 0;
  while ((1 << mlog) < M) ++mlog;
  const int64_t umax = X1 - X0;
  const int sh = std::max(0, bit_length((uint64_t)umax) - mlog);
  PL2Feat<R> f;
  f.leaf.resize(S);
  f.w.resize(S);
  const R inv = std::ldexp((R)1, -sh);
  for (int64_t i = 0; i < S; ++i) {
    bool sat;
    const int64_t U = Fixed<T>::X(x[i], rho, sat) - X0;
    int64_t j = U >> sh;
    if (j > M - 1) j = M - 1;
    f.leaf[i] = (int32_t)j;
    f.w[i] = (R)(U - (j << sh)) * inv;   // the position the classifier uses
  }
  // leaf starts: samples are sorted, so leaf j is one index range
  f.start.assign(M + 1, S);
  for (int32_t j = 0; j < M; ++j) {
    int64_t c = 0;
    while (c < S && f.leaf[c] < j) ++c;
    f.start[j] = c;
  }
  std::vector<R> y(M + 1), tau(S), r(S);
  for (int64_t i = 0; i < S; ++i) tau[i] = ((R)i + (R)0.5) / (R)S;
  // initial knots: the empirical CDF at the knots
  for (int32_t j = 0; j <= M; ++j) y[j] = (R)f.start[j] / (R)S;
  auto loss = [&]() {
    double L = 0.0;
    for (int64_t i = 0; i < S; ++i) L += (double)r[i] * (double)r[i];
    return L / (double)S;
  };
  auto forward = [&]() {  // F and the residual of every sample
    for (int64_t i = 0; i < S; ++i) {
      const int32_t a = f.leaf[i];
      const R t1 = (R)1 - f.w[i];
      const R p = y[a] * t1;
      const R q = y[a + 1] * f.w[i];
      const R F = p + q;
      r[i] = F - tau[i];
    }
  };
  for (int step = 0; step <= kPL2Steps; ++step) {
    if (loss_trace) {
      forward();
      loss_trace->push_back(loss());
    }
    if (step == kPL2Steps) break;
    // red-black coordinate descent: the odd knots, then the even ones.  Knots
    // of one parity share no sample, so each moves to the exact minimiser of
    // the loss along its own coordinate, y_j - G_j / H_j (the 1-D quadratic's
    // Newton step), clamped to [y_{j-1}, y_{j+1}] (0 and 1 at the ends): in
    // exact arithmetic the loss never rises, and the knots stay in [0, 1],
    // non-decreasing.  G_j and H_j sum leaf j (weight 1-w) then leaf j-1
    // (weight w) in sample order.
    for (int parity = 1; parity >= 0; --parity) {
      forward();
      for (int32_t j = parity; j <= M; j += 2) {
        R g = 0, h = 0;
        if (j < M)
          for (int64_t i = f.start[j]; i < f.start[j + 1]; ++i) {
            const R t1 = (R)1 - f.w[i];
            g = g + r[i] * t1;
            h = h + t1 * t1;
          }
        if (j > 0)
          for (int64_t i = f.start[j - 1]; i < f.start[j]; ++i) {
            g = g + r[i] * f.w[i];
            h = h + f.w[i] * f.w[i];
          }
        if (h > (R)0) {
          const R lo = j > 0 ? y[j - 1] : (R)0, hi = j < M ? y[j + 1] : (R)1;
          y[j] = std::min(std::max(y[j] - g / h, lo), hi);
        }
      }
    }
  }
  m->kind = 2;
  m->capped = 0;
  m->S = S;
  m->D = sh;
  m->nsplit = M;
  m->nbuckets = K;
  m->pl2_sh = sh;
  m->pl2_rho = rho;
  m->pl2_x0 = X0;
  *knots = y;
  if (feat_out) *feat_out = f;
  return true;
}

// The model's training: binary32 (the sort's PL2 model).
template <class T>
bool pl2_fit(const T* x, int64_t S, int32_t M, int32_t K, OracleModel* m, std::vector<float>* knots,
             std::vector<double>* loss_trace) {
  return pl2_train<T, float>(x, S, M, K, m, knots, nullptr, loss_trace);
}

// Bucket of key x under a PL2 model: floor(k F(x)) in binary32, clamped to
// the leaf's range.  Monotone in x: the leaf index and the position in the
// leaf are, F is within a leaf (non-negative slope, monotone roundings),
// and the leaf ranges [floor(k y_j), floor(k y_{j+1})] follow each other.
template <class T>
int32_t pl2_bucket(T x, const OracleModel& m, const float* y) {
  typedef Key<T> KT;
  const int32_t K = m.nbuckets, M = m.nsplit;
  if (KT::is_nan(x)) return KT::neg_sign(x) ? 0 : K - 1;
  bool sat;
  const int64_t X = Fixed<T>::X(x, m.pl2_rho, sat);
  if (sat) return X > 0 ? K - 1 : 0;
  const int64_t U = X - m.pl2_x0;
  if (U < 0) return 0;
  const int64_t j = U >> m.pl2_sh;
  if (j >= M) return K - 1;
  const float y0 = y[j], y1 = y[j + 1];
  const float kf = (float)K;
  const float inv = std::ldexp(1.0f, -m.pl2_sh);
  const float w = (float)(U - (j << m.pl2_sh)) * inv;
  const float d = y1 - y0;
  const float F = y0 + d * w;
  int32_t b = (int32_t)std::floor(F * kf);
  int32_t lo = (int32_t)std::floor(y0 * kf), hi = (int32_t)std::floor(y1 * kf);
  if (lo > K - 1) lo = K - 1;
  if (hi > K - 1) hi = K - 1;
  if (b < lo) b = lo;
  if (b > hi) b = hi;
  return b;
}

template <class T>
int32_t bucket_of(T x, const OracleModel& m, T xlo, const float* knots = nullptr) {
  if (m.kind == 0) return linear_bucket<T>(x, m, xlo);
  if (m.kind == 2) return pl2_bucket<T>(x, m, knots);
  return splitter_bucket(Key<T>::ord(x), m);
}

// One IPLS partition pass on src[0..n) (the subproblem at offset `off` of the
// whole array, at recursion level `level`): sample, sort the sample, fit,
// classify, histogram, exclusive scan, stable scatter into dst[0..n).
template <class T>
void partition_pass(const T* src, int64_t n, int64_t off, int32_t level,
                    const OracleCfg& cfg, T* dst, int64_t* counts,
                    OracleModel* m, std::vector<float>* knots_out = nullptr) {
  typedef Key<T> KT;
  const int64_t S = sample_size(n, level, cfg);
  std::vector<int64_t> idx(S);
  sample_indices(cfg.seed, off, n, level, S, idx.data());
  std::vector<T> samp(S);
  for (int64_t j = 0; j < S; ++j) samp[j] = src[idx[j] - off];
  std::stable_sort(samp.begin(), samp.end(),
                   [](T a, T b) { return KT::ord(a) < KT::ord(b); });
  std::memset(m, 0, sizeof(*m));
  m->S = S;
  const bool usable = KT::ord(samp[0]) != KT::ord(samp[S - 1]) &&
                      KT::finite(samp[0]) && KT::finite(samp[S - 1]);
  bool linear = usable;
  T xlo = samp[0];
  std::vector<int32_t> b(n);
  // PL2 for large subproblems when enabled; its pass falls back to the
  // splitter tree on no progress or when a bucket holds more than 4n/k keys
  std::vector<float> knots;
  if (usable && cfg.pl2_leaves > 0 && n > kPL2MinKeys && S <= kPL2MaxSample &&
      (cfg.pl2_depth == 0 || level < cfg.pl2_depth) &&
      pl2_fit<T>(samp.data(), S, cfg.pl2_leaves, cfg.k, m, &knots, nullptr)) {
    linear = false;
    std::fill(counts, counts + m->nbuckets, 0);
    for (int64_t i = 0; i < n; ++i) counts[b[i] = pl2_bucket<T>(src[i], *m, knots.data())]++;
    bool bad = false;
    for (int32_t j = 0; j < m->nbuckets; ++j)
      if (counts[j] == n || counts[j] * (int64_t)m->nbuckets > 4 * n) bad = true;
    if (!bad) {
      std::vector<int64_t> base(m->nbuckets + 1, 0);
      for (int32_t j = 0; j < m->nbuckets; ++j) base[j + 1] = base[j] + counts[j];
      for (int64_t i = 0; i < n; ++i) dst[base[b[i]]++] = src[i];
      if (knots_out) *knots_out = knots;
      return;
    }
  } else if (linear) {
    fmcd<T>(samp.data(), S, cfg.k, m);
    const bool ok = std::isfinite(m->ud) && m->ud > 0.0 &&
                    std::isfinite(m->A) && std::isfinite(m->Bc);
    if (ok) xlo = samp[m->D]; else linear = false;
  }
  if (linear) {
    std::fill(counts, counts + m->nbuckets, 0);
    for (int64_t i = 0; i < n; ++i) counts[b[i] = linear_bucket<T>(src[i], *m, xlo)]++;
    bool all_one = false;
    for (int32_t j = 0; j < m->nbuckets; ++j) if (counts[j] == n) all_one = true;
    if (all_one) linear = false;      // no progress: splitter fallback (R7)
  }
  if (!linear) {
    OracleModel keep = *m;
    build_splitters<T>(samp.data(), S, cfg.k, m);
    m->S = S; m->D = keep.D; m->capped = keep.capped; m->A = keep.A;
    m->Bc = keep.Bc; m->B = keep.B; m->ud = keep.ud; m->xlo = keep.xlo;
    m->xlo_bits = keep.xlo_bits;
    std::fill(counts, counts + m->nbuckets, 0);
    for (int64_t i = 0; i < n; ++i) counts[b[i] = splitter_bucket(KT::ord(src[i]), *m)]++;
  }
  std::vector<int64_t> base(m->nbuckets + 1, 0);
  for (int32_t j = 0; j < m->nbuckets; ++j) base[j + 1] = base[j] + counts[j];
  for (int64_t i = 0; i < n; ++i) dst[base[b[i]]++] = src[i];
}

// Base case: insertion sort by totalOrder (the paper uses SkaSort for
// n <= 2^12, Ch.4; any exact sort gives the same, unique result).
template <class T>
void base_sort(T* a, int64_t n) {
  typedef Key<T> KT;
  for (int64_t i = 1; i < n; ++i) {
    T v = a[i];
    int64_t j = i - 1;
    while (j >= 0 && KT::ord(a[j]) > KT::ord(v)) { a[j + 1] = a[j]; --j; }
    a[j + 1] = v;
  }
}

struct Sub { int64_t off, n; };

// IPLS by levels: every subproblem at level L lives in buffer L%2 (0 = keys,
// 1 = scratch); a pass writes its buckets into the other buffer; buckets
// become level L+1 subproblems (Ch.2 IPS4o recursion; Ch.4).
// `roots` are the level-0 subproblems: the whole array, or independent
// segments each keyed by its own offset.
// knots_out (optional): (pl2_leaves + 1) floats per trace record, the knots
// of that pass's PL2 model (zero for passes of another kind).
template <class T>
int ipls_sort(T* keys, int64_t n, const std::vector<Sub>& roots, const OracleCfg& cfg,
              OracleTrace* trace, int64_t trace_cap, int64_t* trace_count, int32_t* levels_out,
              float* knots_out = nullptr) {
  if (trace_count) *trace_count = 0;
  if (levels_out) *levels_out = 0;
  if (cfg.k < 3 || cfg.k > 256 || cfg.cutoff < 1) return -1;
  if (n <= 1) return 0;
  std::vector<T> scratch(n);
  T* buf[2] = {keys, scratch.data()};
  std::vector<Sub> cur, next;
  for (const Sub& r : roots) if (r.n > 1) cur.push_back(r);
  int32_t level = 0;
  std::vector<int64_t> counts(512);
  OracleModel m;
  while (!cur.empty()) {
    if (level > 4096) return -6;
    next.clear();
    T* src = buf[level & 1];
    T* dst = buf[(level + 1) & 1];
    for (const Sub& s : cur) {
      if (s.n <= cfg.cutoff) {
        if (src != keys) std::memcpy(keys + s.off, src + s.off, s.n * sizeof(T));
        base_sort<T>(keys + s.off, s.n);
        continue;
      }
      std::vector<float> kn;
      partition_pass<T>(src + s.off, s.n, s.off, level, cfg, dst + s.off,
                        counts.data(), &m, &kn);
      if (trace && trace_count && *trace_count < trace_cap) {
        if (knots_out && cfg.pl2_leaves > 0) {
          float* kr = knots_out + *trace_count * (int64_t)(cfg.pl2_leaves + 1);
          for (int32_t j = 0; j <= cfg.pl2_leaves; ++j)
            kr[j] = (m.kind == 2 && j < (int32_t)kn.size()) ? kn[j] : 0.0f;
        }
        OracleTrace& t = trace[(*trace_count)++];
        t.off = s.off; t.n = s.n; t.level = level; t.pad = 0; t.model = m;
        std::memset(t.counts, 0, sizeof(t.counts));
        std::copy(counts.begin(), counts.begin() + m.nbuckets, t.counts);
      }
      int64_t pos = s.off;
      for (int32_t j = 0; j < m.nbuckets; ++j) {
        const int64_t c = counts[j];
        if (c == 0) continue;
        const bool equal_bucket = (m.kind == 1) && (j & 1);
        if (equal_bucket) {
          if (dst != keys) std::memcpy(keys + pos, dst + pos, c * sizeof(T));
        } else {
          next.push_back(Sub{pos, c});
        }
        pos += c;
      }
    }
    cur.swap(next);
    ++level;
  }
  if (levels_out) *levels_out = level;
  return 0;
}

template <class F>
int dispatch(int dtype, F f) {
  switch (dtype) {
    case OR_F64: return f((double*)nullptr);
    case OR_F32: return f((float*)nullptr);
    case OR_U64: return f((uint64_t*)nullptr);
    case OR_U32: return f((uint32_t*)nullptr);
  }
  return -1;
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (loaded by the tests through ctypes).
// ---------------------------------------------------------------------------
extern "C" {

int oracle_record_sizes(int64_t* model_bytes, int64_t* trace_bytes) {
  *model_bytes = sizeof(OracleModel);
  *trace_bytes = sizeof(OracleTrace);
  return 0;
}

uint64_t oracle_mix64(uint64_t z) { return mix64(z); }

void oracle_sample_indices(uint64_t seed, int64_t off, int64_t n, int32_t level,
                           int64_t S, int64_t* idx) {
  sample_indices(seed, off, n, level, S, idx);
}

int64_t oracle_sample_size(int64_t n, int32_t level, int32_t k, int64_t root_sample) {
  OracleCfg c{k, 1, root_sample, 0};
  return sample_size(n, level, c);
}

int oracle_total_order(int dtype, const void* keys, int64_t n, uint64_t* out) {
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    const T* k = (const T*)keys;
    for (int64_t i = 0; i < n; ++i) out[i] = Key<T>::ord(k[i]);
    return 0;
  });
}

// FMCD on an already sorted sample (from its definition).
int oracle_fmcd(int dtype, const void* sorted, int64_t N, int32_t K, OracleModel* m) {
  if (N < 3 || K < 3) return -1;
  std::memset(m, 0, sizeof(*m));
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    fmcd<T>((const T*)sorted, N, K, m);
    return 0;
  });
}

// FMCD by the one-walk search (for checking it against the definition).
int oracle_fmcd_incremental(int dtype, const void* sorted, int64_t N, int32_t K, OracleModel* m) {
  if (N < 3 || K < 3) return -1;
  std::memset(m, 0, sizeof(*m));
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    fmcd_incremental<T>((const T*)sorted, N, K, m);
    return 0;
  });
}

// Bucket of every key under a given model (kind 0 uses A, Bc and the key
// whose raw bits are xlo_bits; kind 1 uses the splitters).  A PL2 model
// (kind 2) needs its knots: oracle_pl2_classify.
int oracle_classify(int dtype, const void* keys, int64_t n, const OracleModel* m,
                    int32_t* out) {
  if (m->kind == 2) return 2;
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    T xlo;
    uint64_t b = m->xlo_bits;
    if (sizeof(T) == 8) std::memcpy(&xlo, &b, 8);
    else { uint32_t b32 = (uint32_t)b; std::memcpy(&xlo, &b32, 4); }
    const T* k = (const T*)keys;
    for (int64_t i = 0; i < n; ++i) out[i] = bucket_of<T>(k[i], *m, xlo);
    return 0;
  });
}

// Partition keys[0..n) by a given model: stable scatter into dst, counts out.
int oracle_partition_with_model(int dtype, const void* keys, int64_t n,
                                const OracleModel* m, void* dst, int64_t* counts) {
  std::vector<int32_t> b(n);
  int rc = oracle_classify(dtype, keys, n, m, b.data());
  if (rc) return rc;
  std::fill(counts, counts + m->nbuckets, 0);
  for (int64_t i = 0; i < n; ++i) counts[b[i]]++;
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    std::vector<int64_t> base(m->nbuckets + 1, 0);
    for (int32_t j = 0; j < m->nbuckets; ++j) base[j + 1] = base[j] + counts[j];
    const T* s = (const T*)keys;
    T* d = (T*)dst;
    for (int64_t i = 0; i < n; ++i) d[base[b[i]]++] = s[i];
    return 0;
  });
}

// One full IPLS pass (sample, sort, fit, classify, scan, stable scatter) on
// the subproblem src[0..n) that sits at `off` of the whole array, `level`.
int oracle_partition_pass(int dtype, const void* src, int64_t n, int64_t off,
                          int32_t level, const OracleCfg* cfg, void* dst,
                          int64_t* counts, OracleModel* m) {
  if (n < 2 || cfg->k < 3 || cfg->k > 256) return -1;
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    partition_pass<T>((const T*)src, n, off, level, *cfg, (T*)dst, counts, m);
    return 0;
  });
}

// Whole IPLS sort, in place.  Returns 0, or a negative status.
int oracle_sort(int dtype, void* keys, int64_t n, const OracleCfg* cfg,
                OracleTrace* trace, int64_t trace_cap, int64_t* trace_count,
                int32_t* levels) {
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    std::vector<Sub> roots(1, Sub{0, n});
    return ipls_sort<T>((T*)keys, n, roots, *cfg, trace, trace_cap, trace_count, levels);
  });
}

// oracle_sort that also writes the PL2 knots of every traced pass
// ((pl2_leaves + 1) floats per record into knots).
int oracle_sort_knots(int dtype, void* keys, int64_t n, const OracleCfg* cfg,
                      OracleTrace* trace, int64_t trace_cap, int64_t* trace_count,
                      int32_t* levels, float* knots) {
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    std::vector<Sub> roots(1, Sub{0, n});
    return ipls_sort<T>((T*)keys, n, roots, *cfg, trace, trace_cap, trace_count, levels, knots);
  });
}

// Sorts each segment keys[off[i]..off[i+1]) as its own level-0 subproblem.
int oracle_sort_segments(int dtype, void* keys, const int64_t* off, int64_t nseg,
                         const OracleCfg* cfg, OracleTrace* trace, int64_t trace_cap,
                         int64_t* trace_count, int32_t* levels) {
  if (nseg < 0) return -1;
  std::vector<Sub> roots;
  for (int64_t i = 0; i < nseg; ++i) {
    if (off[i + 1] < off[i]) return -1;
    roots.push_back(Sub{off[i], off[i + 1] - off[i]});
  }
  const int64_t n = nseg > 0 ? off[nseg] : 0;
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    return ipls_sort<T>((T*)keys, n, roots, *cfg, trace, trace_cap, trace_count, levels);
  });
}

// Reference sort for the pins: std::sort under totalOrder.
// PL2 on a sorted sample: the fitted model, its knots y_0..y_M (M + 1
// floats into `knots`) and the loss after each of the training steps
// (kPL2Steps + 1 values).  Returns 1 when the sample's range could not be
// used.
int oracle_pl2_fit(int dtype, const void* sorted, int64_t S, int32_t M, int32_t K, OracleModel* m,
                   double* losses, float* knots) {
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    std::memset(m, 0, sizeof(*m));
    std::vector<double> lt;
    std::vector<float> y;
    if (!pl2_fit<T>((const T*)sorted, S, M, K, m, &y, &lt)) return 1;
    for (size_t i = 0; i < lt.size(); ++i) losses[i] = lt[i];
    for (size_t j = 0; j < y.size(); ++j) knots[j] = y[j];
    return 0;
  });
}

// The same training in binary64 (a reference for the loss the binary32
// model reaches): its knots (M + 1 doubles) and losses after each step.
int oracle_pl2_fit_f64(int dtype, const void* sorted, int64_t S, int32_t M, int32_t K, OracleModel* m,
                       double* losses, double* knots) {
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    std::memset(m, 0, sizeof(*m));
    std::vector<double> lt, y;
    if (!pl2_train<T, double>((const T*)sorted, S, M, K, m, &y, nullptr, &lt)) return 1;
    for (size_t i = 0; i < lt.size(); ++i) losses[i] = lt[i];
    for (size_t j = 0; j < y.size(); ++j) knots[j] = y[j];
    return 0;
  });
}

// Buckets of keys[0..n) under a PL2 model with knots y_0..y_M.
int oracle_pl2_classify(int dtype, const void* keys, int64_t n, const OracleModel* m,
                        const float* knots, int32_t* out) {
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    const T* x = (const T*)keys;
    for (int64_t i = 0; i < n; ++i) out[i] = pl2_bucket<T>(x[i], *m, knots);
    return 0;
  });
}

// The PL2 loss (1/S) sum (F(x_i) - (i+1/2)/S)^2 and its gradient in the knot
// values y[0..M], for the leaves and positions a model assigns to the sorted
// sample (summed in sample order).  For checking training steps.
// absg (optional): per knot, the sum of the magnitudes of the terms of its
// gradient, (2/S) sum |r_i| * weight_i (a scale for rounding-error bounds).
int oracle_pl2_loss_grad(int dtype, const void* sorted, int64_t S, const OracleModel* m,
                         const double* y, double* loss, double* grad, double* absg) {
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    const T* x = (const T*)sorted;
    const int32_t M = m->nsplit;
    const double inv = std::ldexp(1.0, -m->pl2_sh);
    std::vector<double> r(S), w(S);
    std::vector<int32_t> leaf(S);
    double L = 0.0;
    for (int64_t i = 0; i < S; ++i) {
      bool sat;
      const int64_t U = Fixed<T>::X(x[i], m->pl2_rho, sat) - m->pl2_x0;
      int64_t j = U >> m->pl2_sh;
      if (j > M - 1) j = M - 1;
      if (j < 0) j = 0;
      leaf[i] = (int32_t)j;
      w[i] = (double)(U - (j << m->pl2_sh)) * inv;
      const double F = y[j] * (1.0 - w[i]) + y[j + 1] * w[i];
      r[i] = F - ((double)i + 0.5) / (double)S;
      L += r[i] * r[i];
    }
    *loss = L / (double)S;
    for (int32_t j = 0; j <= M; ++j) grad[j] = 0.0;
    for (int64_t i = 0; i < S; ++i) {
      grad[leaf[i]] += 2.0 * r[i] * (1.0 - w[i]) / (double)S;
      grad[leaf[i] + 1] += 2.0 * r[i] * w[i] / (double)S;
    }
    if (absg) {
      for (int32_t j = 0; j <= M; ++j) absg[j] = 0.0;
      for (int64_t i = 0; i < S; ++i) {
        absg[leaf[i]] += 2.0 * std::fabs(r[i]) * (1.0 - w[i]) / (double)S;
        absg[leaf[i] + 1] += 2.0 * std::fabs(r[i]) * w[i] / (double)S;
      }
    }
    return 0;
  });
}

int oracle_std_sort(int dtype, void* keys, int64_t n) {
  return dispatch(dtype, [&](auto* tag) {
    typedef std::remove_pointer_t<decltype(tag)> T;
    T* k = (T*)keys;
    std::sort(k, k + n, [](T a, T b) { return Key<T>::ord(a) < Key<T>::ord(b); });
    return 0;
  });
}

// Multiset fingerprint: sum and xor of mix64 over the raw bits of every key.
void oracle_multiset_hash(int dtype, const void* keys, int64_t n, uint64_t* sum_out,
                          uint64_t* xor_out) {
  uint64_t s = 0, x = 0;
  const int w = (dtype == OR_F64 || dtype == OR_U64) ? 8 : 4;
  const unsigned char* p = (const unsigned char*)keys;
  for (int64_t i = 0; i < n; ++i) {
    uint64_t b = 0;
    std::memcpy(&b, p + i * w, w);
    uint64_t h = mix64(b + kGamma);
    s += h; x ^= h;
  }
  *sum_out = s; *xor_out = x;
}

}  // extern "C"
