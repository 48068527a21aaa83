// iplsPL2LossGrad: the PL2 learned CDF's loss and gradient on the device.
//
// The PL2 model (a two-level piecewise-linear CDF, the learned CDF of Ch.2
// "Learned Sort" and Ch.3 "Recursive Model Index" trained against the
// empirical CDF with the mean squared error of Ch.3) is trained inside k_fit
// by red-black coordinate descent.  Each half-sweep of that training is a
// forward pass (the CDF and the residual of every sample) and a backward pass
// (per knot j, G_j = sum r_i dF_i/dy_j and H_j = sum (dF_i/dy_j)^2).  This
// file runs exactly those two device functions (pl2_forward, pl2_knot_gh from
// ipls_device.cuh) for knot values the caller supplies, so that the device's
// gradient can be compared with an independent computation.
#include <cstdint>

#include "ipls.h"
#include "ipls_device.cuh"

namespace ipls {

constexpr int kPL2GradThreads = 1024;

// One block: out[0..M] = G_j, out[M+1..2M+1] = H_j, out[2M+2] = loss
// (1/S) sum r_i^2 (binary32, block-reduced), out[2M+3] = 1 when the sample's
// range carries PL2 (else everything is 0).
template <class K>
__global__ void __launch_bounds__(kPL2GradThreads) k_pl2_loss_grad(const typename KT<K>::Bits* sample, int S,
                                                                   int M, const float* knots, float* out) {
  using T = KT<K>;
  using Ord = typename T::Ord;
  // dynamic: the sample (S keys) then leaf, w and r (S entries each)
  extern __shared__ __align__(16) unsigned char smem[];
  Ord* so = reinterpret_cast<Ord*>(smem);
  int32_t* leaf = reinterpret_cast<int32_t*>(smem + (size_t)kPL2MaxSample * sizeof(Ord));
  float* w = reinterpret_cast<float*>(leaf + kPL2MaxSample);
  float* r = w + kPL2MaxSample;
  __shared__ float y[kPL2MaxLeaves + 1];
  __shared__ int start[kPL2MaxLeaves + 1];
  __shared__ int s_flag, s_rho, s_sh;
  __shared__ long long s_x0;
  __shared__ float part[kPL2GradThreads / 32];
  for (int i = threadIdx.x; i < S; i += blockDim.x) so[i] = T::ord(sample[i]);
  for (int j = threadIdx.x; j <= M; j += blockDim.x) y[j] = knots[j];
  __syncthreads();
  if (threadIdx.x == 0) pl2_geometry<K>(so, S, M, &s_flag, &s_x0, &s_rho, &s_sh);
  __syncthreads();
  if (!s_flag) {
    for (int j = threadIdx.x; j < 2 * (M + 1) + 2; j += blockDim.x) out[j] = 0.0f;
    return;
  }
  const PL2Scratch sc{leaf, w, r};
  pl2_features<K>(so, S, M, s_rho, s_sh, s_x0, sc, start, y, false);
  pl2_forward(S, sc, y);
  __syncthreads();
  for (int j = threadIdx.x; j <= M; j += blockDim.x) pl2_knot_gh(j, M, sc, start, &out[j], &out[M + 1 + j]);
  float acc = 0.0f;
  for (int i = threadIdx.x; i < S; i += blockDim.x) acc = __fadd_rn(acc, __fmul_rn(r[i], r[i]));
  for (int o = 16; o >= 1; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.0f;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) tot = __fadd_rn(tot, part[q]);
    out[2 * (M + 1)] = __fdiv_rn(tot, (float)S);
    out[2 * (M + 1) + 1] = 1.0f;
  }
}

}  // namespace ipls

extern "C" iplsStatus iplsPL2LossGrad(const void* sample, int64_t S, iplsDtype dtype, int32_t leaves,
                                      const float* knots, float* out, void* stream) {
  using namespace ipls;
  if ((int)dtype < 0 || (int)dtype > 3) {
    set_last_error("unknown dtype");
    return IPLS_ERR_ARG;
  }
  if (S < 2 || S > kPL2MaxSample) {
    set_last_error("iplsPL2LossGrad: S must be in [2, 4096]");
    return IPLS_ERR_ARG;
  }
  if (leaves < 2 || leaves > kPL2MaxLeaves || (leaves & (leaves - 1))) {
    set_last_error("iplsPL2LossGrad: leaves must be a power of two in [2, 1024]");
    return IPLS_ERR_ARG;
  }
  if (!sample || !knots || !out) {
    set_last_error("iplsPL2LossGrad: NULL pointer");
    return IPLS_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n = (int)S;
  cudaError_t e = cudaSuccess;
  const size_t smem8 = (size_t)kPL2MaxSample * 20, smem4 = (size_t)kPL2MaxSample * 16;
  switch ((int)dtype) {
    case 0:
      e = cudaFuncSetAttribute(k_pl2_loss_grad<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem8);
      if (e == cudaSuccess)
        k_pl2_loss_grad<double><<<1, kPL2GradThreads, smem8, s>>>(static_cast<const unsigned long long*>(sample),
                                                                  n, leaves, knots, out);
      break;
    case 1:
      e = cudaFuncSetAttribute(k_pl2_loss_grad<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem4);
      if (e == cudaSuccess)
        k_pl2_loss_grad<float><<<1, kPL2GradThreads, smem4, s>>>(static_cast<const unsigned int*>(sample), n,
                                                                 leaves, knots, out);
      break;
    case 2:
      e = cudaFuncSetAttribute(k_pl2_loss_grad<unsigned long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem8);
      if (e == cudaSuccess)
        k_pl2_loss_grad<unsigned long long><<<1, kPL2GradThreads, smem8, s>>>(
            static_cast<const unsigned long long*>(sample), n, leaves, knots, out);
      break;
    default:
      e = cudaFuncSetAttribute(k_pl2_loss_grad<unsigned int>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem4);
      if (e == cudaSuccess)
        k_pl2_loss_grad<unsigned int><<<1, kPL2GradThreads, smem4, s>>>(static_cast<const unsigned int*>(sample),
                                                                        n, leaves, knots, out);
      break;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return IPLS_ERR_CUDA;
  }
  return IPLS_OK;
}
