/* Seeded synthetic key generators (inputs only: no sorting arithmetic here).
 *
 * They stand in for the synthetic datasets of the paper's benchmark (Ch.5,
 * "Synthetic Datasets") and for the duplicate-heavy sets; the real-world
 * datasets are not available and are not imitated.
 *
 * Every key i of a stream is a pure function of (seed, distribution, i):
 * r_i = mix64(stream + (i+1)*gamma) with SplitMix64 (Steele, Lea and Flood
 * 2014), so the output does not depend on how many threads produce it.
 * Floating-point draws use the host libm (log, exp, cos, sqrt, pow); a last-bit
 * difference between two hosts' libm can change a key, never the way the
 * same bytes are fed to both sides of a comparison.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GAMMA 0x9e3779b97f4a7c15ULL

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
static uint64_t draw(uint64_t stream, uint64_t i) { return mix64(stream + (i + 1) * GAMMA); }
static double unit01(uint64_t r) { return (double)(r >> 11) * 0x1.0p-53; }          /* [0,1) */
static double unit01_open0(uint64_t r) { return (double)((r >> 11) + 1) * 0x1.0p-53; } /* (0,1] */
static uint64_t mulhi(uint64_t a, uint64_t b) {
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
}

enum {
  G_UNIFORM = 0, G_NORMAL = 1, G_LOGNORMAL = 2, G_EXPONENTIAL = 3, G_MIXGAUSS = 4,
  G_ZIPF = 5, G_ROOTDUPS = 6, G_TWODUPS = 7, G_EIGHTDUPS = 8, G_RAW64 = 9
};
enum { T_F64 = 0, T_F32 = 1, T_U64 = 2, T_U32 = 3 };

typedef struct {
  int dist, dtype;
  int64_t n;          /* size that defines index formulas (root/two dups) */
  uint64_t seed;
  double zipf_s;
  int64_t zipf_n;
  const double* zipf_cdf;
  double mu[5], sd[5];
  void* out;
  int64_t lo, hi;     /* index range to produce */
} Job;

/* Box-Muller (1958): one standard normal from two independent uniforms. */
static double normal01(uint64_t stream, uint64_t i) {
  double u1 = unit01_open0(draw(stream, 2 * i));
  double u2 = unit01(draw(stream, 2 * i + 1));
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* Smallest k in [1, N] with cdf[k-1] >= u (inverse CDF by binary search). */
static int64_t zipf_draw(const double* cdf, int64_t N, double u) {
  int64_t lo = 0, hi = N - 1;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (cdf[mid] >= u) hi = mid; else lo = mid + 1;
  }
  return lo + 1;
}

static void put(const Job* j, int64_t i, double v, uint64_t iv, int is_int) {
  switch (j->dtype) {
    case T_F64: ((double*)j->out)[i - j->lo] = is_int ? (double)iv : v; break;
    case T_F32: ((float*)j->out)[i - j->lo] = is_int ? (float)iv : (float)v; break;
    case T_U64: {
      uint64_t u;
      if (is_int) u = iv;
      else {  /* order-preserving map of the binary64 draw to 64-bit keys */
        uint64_t b; memcpy(&b, &v, 8);
        u = (b >> 63) ? ~b : (b | (1ULL << 63));
      }
      ((uint64_t*)j->out)[i - j->lo] = u;
      break;
    }
    case T_U32: {
      uint32_t u;
      if (is_int) u = (uint32_t)iv;
      else {
        float f = (float)v; uint32_t b; memcpy(&b, &f, 4);
        u = (b >> 31) ? ~b : (b | 0x80000000u);
      }
      ((uint32_t*)j->out)[i - j->lo] = u;
      break;
    }
  }
}

static void* run(void* arg) {
  const Job* j = (const Job*)arg;
  const uint64_t stream = mix64(j->seed * 0x100000001b3ULL + (uint64_t)j->dist + GAMMA);
  const uint64_t mstream = mix64(stream ^ 0x5bd1e995ULL);
  int64_t root = 1;
  if (j->dist == G_ROOTDUPS) { root = (int64_t)sqrt((double)j->n);
    while (root * root > j->n) --root; while ((root + 1) * (root + 1) <= j->n) ++root; }
  for (int64_t i = j->lo; i < j->hi; ++i) {
    switch (j->dist) {
      case G_UNIFORM: put(j, i, unit01(draw(stream, i)), 0, 0); break;
      case G_NORMAL: put(j, i, normal01(stream, i), 0, 0); break;
      case G_LOGNORMAL: put(j, i, exp(0.5 * normal01(stream, i)), 0, 0); break;
      case G_EXPONENTIAL: put(j, i, -log1p(-unit01(draw(stream, i))) / 2.0, 0, 0); break;
      case G_MIXGAUSS: {
        int c = (int)mulhi(draw(mstream, i), 5);
        put(j, i, j->mu[c] + j->sd[c] * normal01(stream, i), 0, 0);
        break;
      }
      case G_ZIPF: put(j, i, 0, (uint64_t)zipf_draw(j->zipf_cdf, j->zipf_n, unit01(draw(stream, i))), 1); break;
      case G_ROOTDUPS: put(j, i, 0, (uint64_t)(i % root), 1); break;
      case G_TWODUPS: {
        uint64_t n = (uint64_t)j->n, ii = (uint64_t)i;
        put(j, i, 0, (uint64_t)(((unsigned __int128)ii * ii + n / 2) % n), 1);
        break;
      }
      case G_EIGHTDUPS: put(j, i, 0, (uint64_t)(i % 8), 1); break;
      case G_RAW64: put(j, i, 0, draw(stream, i), 1); break;
    }
  }
  return 0;
}

/* Normalised CDF of Zipf(s) over 1..N, summed in index order. */
static double* zipf_table(double s, int64_t N) {
  double* cdf = (double*)malloc((size_t)N * sizeof(double));
  if (!cdf) return 0;
  double acc = 0;
  for (int64_t k = 1; k <= N; ++k) { acc += pow((double)k, -s); cdf[k - 1] = acc; }
  for (int64_t k = 0; k < N; ++k) cdf[k] /= acc;
  cdf[N - 1] = 1.0;
  return cdf;
}

/* Generate keys [lo, hi) of a stream of size n into out (hi-lo keys).
 * Returns 0, or -1 on a bad argument / allocation failure. */
int datagen_fill(int dist, int dtype, int64_t n, uint64_t seed, double zipf_s,
                 int64_t zipf_n, int64_t lo, int64_t hi, void* out, int threads) {
  if (lo < 0 || hi < lo || hi > n || dist < 0 || dist > G_RAW64) return -1;
  Job base;
  memset(&base, 0, sizeof(base));
  base.dist = dist; base.dtype = dtype; base.n = n; base.seed = seed;
  base.zipf_s = zipf_s; base.zipf_n = zipf_n; base.out = out;
  double* cdf = 0;
  if (dist == G_ZIPF) {
    if (zipf_n < 1) return -1;
    cdf = zipf_table(zipf_s, zipf_n);
    if (!cdf) return -1;
    base.zipf_cdf = cdf;
  }
  if (dist == G_MIXGAUSS) {   /* five components: mean U[-100,100], sd U[1,10] */
    uint64_t ps = mix64(seed + 0x6a09e667f3bcc909ULL);
    for (int c = 0; c < 5; ++c) {
      base.mu[c] = -100.0 + 200.0 * unit01(draw(ps, 2 * c));
      base.sd[c] = 1.0 + 9.0 * unit01(draw(ps, 2 * c + 1));
    }
  }
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  int64_t total = hi - lo;
  if (total < 65536) threads = 1;
  pthread_t tid[256];
  Job jobs[256];
  int started = 0;
  for (int t = 0; t < threads; ++t) {
    jobs[t] = base;
    jobs[t].lo = lo + total * t / threads;
    jobs[t].hi = lo + total * (t + 1) / threads;
    jobs[t].out = (char*)out + (jobs[t].lo - lo) * (int64_t)((dtype == T_F64 || dtype == T_U64) ? 8 : 4);
    /* each job writes relative to its own lo */
  }
  for (int t = 0; t < threads; ++t) {
    if (threads == 1 || pthread_create(&tid[t], 0, run, &jobs[t]) != 0) { run(&jobs[t]); tid[t] = 0; }
    else ++started;
  }
  for (int t = 0; t < threads; ++t) if (tid[t]) pthread_join(tid[t], 0);
  (void)started;
  free(cdf);
  return 0;
}

/* Job of one whole stream (a segment): the same keys datagen_fill gives for
 * [0, n) with this seed. */
static void init_job(Job* j, int dist, int dtype, int64_t n, uint64_t seed, const double* cdf,
                     int64_t zipf_n, void* out) {
  memset(j, 0, sizeof(*j));
  j->dist = dist; j->dtype = dtype; j->n = n; j->seed = seed;
  j->zipf_s = 0.75; j->zipf_n = zipf_n; j->zipf_cdf = cdf; j->out = out;
  j->lo = 0; j->hi = n;
  if (dist == G_MIXGAUSS) {
    uint64_t ps = mix64(seed + 0x6a09e667f3bcc909ULL);
    for (int c = 0; c < 5; ++c) {
      j->mu[c] = -100.0 + 200.0 * unit01(draw(ps, 2 * c));
      j->sd[c] = 1.0 + 9.0 * unit01(draw(ps, 2 * c + 1));
    }
  }
}

typedef struct {
  const int64_t* offsets;
  const int32_t* dist;
  int64_t s0, s1;
  uint64_t seed;
  int dtype;
  const double* cdf;
  void* out;
} SegJob;

static void* run_segments(void* arg) {
  const SegJob* sj = (const SegJob*)arg;
  const int64_t w = (sj->dtype == T_F64 || sj->dtype == T_U64) ? 8 : 4;
  for (int64_t s = sj->s0; s < sj->s1; ++s) {
    const int64_t a = sj->offsets[s], n = sj->offsets[s + 1] - a;
    if (n <= 0) continue;
    Job j;
    init_job(&j, sj->dist[s], sj->dtype, n, sj->seed * 1000003ULL + (uint64_t)s, sj->cdf, 1000000,
             (char*)sj->out + a * w);
    run(&j);
  }
  return 0;
}

/* Segment s of a batch: keys [offsets[s], offsets[s+1]) from distribution
 * dist[s] with stream seed seed*1000003+s (Zipf with s=0.75 over 1..1e6), i.e.
 * what datagen_fill gives for the whole segment.  Segments are shared out
 * over threads; the keys do not depend on the thread count. */
int datagen_fill_segments(const int64_t* offsets, int64_t nseg, const int32_t* dist, uint64_t seed,
                          int dtype, void* out, int threads) {
  if (nseg < 0) return -1;
  for (int64_t s = 0; s < nseg; ++s)
    if (dist[s] < 0 || dist[s] > G_RAW64 || offsets[s + 1] < offsets[s]) return -1;
  double* cdf = zipf_table(0.75, 1000000);
  if (!cdf) return -1;
  if (threads < 1) threads = 1;
  if (threads > 256) threads = 256;
  pthread_t tid[256];
  SegJob jobs[256];
  for (int t = 0; t < threads; ++t) {
    jobs[t].offsets = offsets; jobs[t].dist = dist; jobs[t].seed = seed; jobs[t].dtype = dtype;
    jobs[t].cdf = cdf; jobs[t].out = out;
    jobs[t].s0 = nseg * t / threads;
    jobs[t].s1 = nseg * (t + 1) / threads;
  }
  for (int t = 0; t < threads; ++t)
    if (threads == 1 || pthread_create(&tid[t], 0, run_segments, &jobs[t]) != 0) { run_segments(&jobs[t]); tid[t] = 0; }
  for (int t = 0; t < threads; ++t) if (tid[t]) pthread_join(tid[t], 0);
  free(cdf);
  return 0;
}
