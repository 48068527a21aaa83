// iplsSortSmallNoAlloc: a sort entry point that allocates no memory at all.
//
// Every other entry point runs through a context whose scratch (ping-pong
// buffer, bucket ids, level lists, status words) comes from cudaMalloc or
// the caller's allocator.  Some callers cannot allocate at the moment they
// need a sort:
//   - a framework whose caching allocator already holds nearly all of the
//     device's memory in its own pool, where a cudaMalloc from a library
//     fails or forces the pool to release memory;
//   - a latency-critical loop, where cudaMalloc/cudaFree may synchronise the
//     whole device and stall unrelated streams;
//   - code that must not meet an out-of-memory error half-way through a
//     pipeline (the allocation is the only step here that could fail for
//     lack of memory).
// For those callers this entry point sorts a small array (at most
// resident_rmax(cutoff) keys, 8192 with the default cutoff) in one block,
// with the in-block learned partition recursion (the same sample, model,
// passes and result as iplsSort).  Its only device scratch is the run status
// block below, a file-scope __device__ array: no cudaMalloc, cudaFree, torch
// or other allocating call is made, on the first call or any later one.
#include <cstdint>
#include <cstring>
#include <mutex>

#include "ipls.h"
#include "ipls_internal.h"

namespace {

using namespace ipls;

// Scratch of the no-allocation path: one RunStatus (error word and
// counters), rounded up to its 256-byte maximum.  It must be zero when the
// kernel starts; every call clears it on its stream first.
constexpr size_t kNoAllocScratchBytes = 256;
static_assert(sizeof(RunStatus) <= kNoAllocScratchBytes, "RunStatus outgrew the static scratch");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

iplsStatus fail_na(iplsStatus st, const char* msg) {
  set_last_error(msg);
  return st;
}

// Device address of the static scratch on the current device, looked up once
// per device while that device is current.
iplsStatus scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_na(IPLS_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail_na(IPLS_ERR_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_last_error(e != cudaSuccess ? cudaGetErrorString(e) : "cudaGetSymbolAddress returned NULL");
      return IPLS_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return IPLS_OK;
}

}  // namespace

extern "C" {

iplsStatus iplsSortSmallNoAlloc(void* keys, int64_t n, iplsDtype dtype, const iplsConfig* cfg,
                                void* stream) {
  if ((int)dtype < 0 || (int)dtype > 3) return fail_na(IPLS_ERR_ARG, "unknown dtype");
  if (n < 0) return fail_na(IPLS_ERR_ARG, "n must be >= 0");
  iplsConfig c;
  if (cfg) {
    c = *cfg;
  } else {
    iplsDefaultConfig(&c);
  }
  if (c.k < 3 || c.k > 256) return fail_na(IPLS_ERR_ARG, "k must be in [3, 256]");
  if (c.cutoff < 1 || c.cutoff > kResidentMax) return fail_na(IPLS_ERR_ARG, "cutoff must be in [1, 8192]");
  if (c.root_sample < 0 || c.root_sample > kResidentSample)
    return fail_na(IPLS_ERR_ARG, "root_sample must be in [0, 1024] for iplsSortSmallNoAlloc");
  const int64_t limit = resident_rmax(c.cutoff);
  if (n > limit)
    return fail_na(IPLS_ERR_ARG,
                   "iplsSortSmallNoAlloc sorts at most resident_rmax(cutoff) keys (8192 for "
                   "cutoff >= 7, 1024*(cutoff+1) below); use iplsSort for larger arrays");
  if (n > 0 && !keys) return fail_na(IPLS_ERR_ARG, "keys is NULL");
  const size_t w = (dtype == IPLS_F64 || dtype == IPLS_U64) ? 8 : 4;
  if (reinterpret_cast<uintptr_t>(keys) % w != 0)
    return fail_na(IPLS_ERR_ARG, "keys must be aligned to the key width");

  void* scratch = nullptr;
  iplsStatus st = scratch_address(&scratch);
  if (st != IPLS_OK) return st;
  if (n < 2) return IPLS_OK;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RunStatus* run = static_cast<RunStatus*>(scratch);
  cudaError_t e = cudaMemsetAsync(run, 0, sizeof(RunStatus), s);
  if (e != cudaSuccess) return fail_na(IPLS_ERR_CUDA, cudaGetErrorString(e));

  ResidentArgs a;
  std::memset(&a, 0, sizeof(a));
  a.dtype = (int)dtype;
  a.k = c.k;
  a.cutoff = c.cutoff;
  a.root_sample = c.root_sample;
  a.seed = c.seed;
  a.exact_only = c.exact_only;
  a.buf[0] = keys;
  a.buf[1] = nullptr;
  a.run = run;
  a.trace = nullptr;
  a.trace_cap = 0;
  const SlowTask t{0, (int32_t)n, 0, reinterpret_cast<uint64_t>(keys)};
  e = launch_slow_one(a, t, s);
  if (e != cudaSuccess) return fail_na(IPLS_ERR_CUDA, cudaGetErrorString(e));

  RunStatus h;
  e = cudaMemcpyAsync(&h, run, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_na(IPLS_ERR_CUDA, cudaGetErrorString(e));
  if (h.error != 0) return fail_na((iplsStatus)h.error, "device reported an error in the in-block recursion");
  return IPLS_OK;
}

}  // extern "C"
