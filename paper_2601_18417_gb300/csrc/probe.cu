// probe.cu -- measured arithmetic peaks of the device: FP64 and FP32
// fused-multiply-add throughput, the denominators of the ALU rooflines the
// benchmark reports (the FP64 face kernels are bound by the FP64 pipe, the
// double-float ones by FP32 issue).  No counterpart in the paper.
#include "hofv_internal.cuh"

namespace hofv {

// CHAINS independent FMA chains per thread, x <- x a + b (a < 1, so every
// value stays normal and bounded); the sum is written only if it takes an
// impossible value, which keeps the chains alive without a store per thread
template <typename T, int CHAINS>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T a, T b, T* out) {
  T x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x % 7 + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  if (s == (T)-1) out[0] = s;
}

template <typename T>
static int time_fma(hofv_ctx* c, int iters, T* scratch, double* tflops) {
  constexpr int kChains = 8;
  const unsigned grid = (unsigned)c->sm_count * 8, block = 256;
  cudaEvent_t e0, e1;
  HOFV_CUDA(c, cudaEventCreate(&e0));
  HOFV_CUDA(c, cudaEventCreate(&e1));
  k_fma_probe<T, kChains><<<grid, block, 0, c->stream>>>(iters / 8, (T)0.999999, (T)1e-6, scratch);
  HOFV_CUDA(c, cudaEventRecord(e0, c->stream));
  k_fma_probe<T, kChains><<<grid, block, 0, c->stream>>>(iters, (T)0.999999, (T)1e-6, scratch);
  HOFV_CUDA(c, cudaEventRecord(e1, c->stream));
  HOFV_CUDA(c, cudaEventSynchronize(e1));
  float ms = 0.f;
  HOFV_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HOFV_CUDA(c, cudaGetLastError());
  const double fmas = (double)grid * block * kChains * iters;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return 0;
}

__global__ void k_inv_cbrt(const double* __restrict__ J, double* __restrict__ own,
                           double* __restrict__ lib, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = J[i];
  if (own) own[i] = inv_cbrt(x);
  if (lib) lib[i] = rcbrt(x);
}

}  // namespace hofv

using namespace hofv;

extern "C" int hofv_probe_inv_cbrt(hofv_ctx* c, const double* J, double* r_own, double* r_lib,
                                   int64_t n) {
  if (!c || n < 0 || (n > 0 && !J)) return HOFV_EINVAL;
  if (n == 0) return 0;
  HOFV_CUDA(c, cudaSetDevice(c->device));
  k_inv_cbrt<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(J, r_own, r_lib, n);
  HOFV_CUDA(c, cudaGetLastError());
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  return 0;
}

extern "C" int hofv_probe_peaks(hofv_ctx* c, double* fp64_tflops, double* fp32_tflops,
                                int32_t* sm_count) {
  if (!c) return HOFV_EINVAL;
  HOFV_CUDA(c, cudaSetDevice(c->device));
  if (sm_count) *sm_count = c->sm_count;
  void* scratch = nullptr;
  HOFV_CUDA(c, cudaMalloc(&scratch, 64));
  int rc = 0;
  if (fp64_tflops) rc = time_fma<double>(c, 4096, static_cast<double*>(scratch), fp64_tflops);
  if (rc == 0 && fp32_tflops) rc = time_fma<float>(c, 262144, static_cast<float*>(scratch), fp32_tflops);
  cudaFree(scratch);
  return rc;
}
