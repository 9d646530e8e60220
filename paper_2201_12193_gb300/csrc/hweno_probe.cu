// Arithmetic throughput probe (measurement only; the paper has no counterpart):
// the FP64 or FP32 fused multiply-add rate one GPU sustains, the denominator of
// the ALU roofline the reconstruction kernels are measured against.
//
// Every thread runs 8 independent chains x <- x * a + b (no dependence between
// chains, so the pipe, not latency, sets the rate) over 4 resident blocks of
// 256 threads per multiprocessor; a = 1 - 2^-20 and b = 2^-24 keep the values
// bounded and normal.  Timed with CUDA events around one launch after a
// warm-up launch; one FMA counts 2 flop.
#include <stdio.h>

#include "hweno.h"
#include "hweno_device.cuh"

namespace {

constexpr int PT = 256;
constexpr int CHAINS = 8;

// Sink: the chains' sum is stored only when it equals an impossible value, so
// the compiler keeps the arithmetic without any store in practice.
__device__ double g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(PT) fma_probe_kernel(long long iters, T a, T b) {
  T x[CHAINS];
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < CHAINS; ++k) s += x[k];
  if (s == T(-1.0)) g_probe_sink = (double)s;
}

template <typename T>
cudaError_t run_probe(long long iters, double* flop_per_s, cudaStream_t st) {
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int blocks = 4 * nsm;
  const T a = T(1.0 - 1.0 / 1048576.0), b = T(1.0 / 16777216.0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return e; }
  fma_probe_kernel<T><<<blocks, PT, 0, st>>>(iters / 8 + 1, a, b);    // warm-up
  cudaEventRecord(e0, st);
  fma_probe_kernel<T><<<blocks, PT, 0, st>>>(iters, a, b);
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  const double flop = 2.0 * CHAINS * (double)iters * (double)blocks * PT;
  *flop_per_s = ms > 0.f ? flop / (ms * 1e-3) : 0.0;
  return cudaSuccess;
}

// The fused FP32 kernel's double -> float rounding (hw::f32_rn) applied to n values.
__global__ void f32_round_kernel(const double* __restrict__ in, float* __restrict__ out, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    out[t] = hw::f32_rn(in[t]);
}

}  // namespace

extern "C" hweno_status hweno_f32_round(const double* in, float* out, long long n, void* cuda_stream) {
  if ((!in || !out) && n > 0) return HWENO_EINVAL;
  if (n < 0) return HWENO_EINVAL;
  if (n == 0) return HWENO_OK;
  const long long blocks = (n + PT - 1) / PT < 4096 ? (n + PT - 1) / PT : 4096;
  f32_round_kernel<<<(int)blocks, PT, 0, (cudaStream_t)cuda_stream>>>(in, out, n);
  return cudaGetLastError() == cudaSuccess ? HWENO_OK : HWENO_ECUDA;
}

extern "C" hweno_status hweno_alu_probe(int precision, long long iters, double* flop_per_s, void* cuda_stream) {
  if (!flop_per_s || iters < 1 || (precision != 0 && precision != 1)) return HWENO_EINVAL;
  const cudaError_t e = precision == 0 ? run_probe<double>(iters, flop_per_s, (cudaStream_t)cuda_stream)
                                       : run_probe<float>(iters, flop_per_s, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) {
    fprintf(stderr, "hweno_alu_probe: %s\n", cudaGetErrorString(e));
    return HWENO_ECUDA;
  }
  return HWENO_OK;
}
