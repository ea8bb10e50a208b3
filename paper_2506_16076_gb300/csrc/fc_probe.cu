// FP64 throughput probes of the GPU the library runs on: the denominators against which
// the line kernels' FP64 work is read. DFMA: independent fused multiply-add chains on the
// FP64 pipe; DMMA: the FP64 matrix instruction (m8n8k4), the only FP64 tensor path, which
// the dense per-length derivative operator would have used.
#include <cuda_runtime.h>

#include "fc_internal.h"

namespace {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_THREADS = 256;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dfma(double* out, int iters, double a, double b) {
  double x[PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
  if (s == 12345.678) out[0] = s;  // keeps the chains live; never true for the inputs used
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dmma(double* out, int iters) {
  // 4 independent accumulators of one warp-wide 8 x 8 x 4 FP64 product each
  double a = 1e-3 * (threadIdx.x & 31), b = 1.0 - 1e-3 * (threadIdx.x & 31);
  double c[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                   : "+d"(c[k][0]), "+d"(c[k][1])
                   : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) s += c[k][0] + c[k][1];
  if (s == 12345.678) out[0] = s;
}

}  // namespace

extern "C" fc_status fc_probe_fp64(double* dfma_gflops, double* dmma_gflops, void* stream) {
  if (!dfma_gflops || !dmma_gflops) return FC_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FC_ERR_CUDA;
  double* sink = nullptr;
  if (cudaMallocAsync(&sink, sizeof(double), st) != cudaSuccess) return FC_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = sms * 8;
  const int it_fma = 20000, it_mma = 4000;
  float ms_fma = 0.0f, ms_mma = 0.0f;
  for (int rep = 0; rep < 2; ++rep) {  // the first round warms up clocks and caches
    cudaEventRecord(e0, st);
    k_probe_dfma<<<blocks, PROBE_THREADS, 0, st>>>(sink, it_fma, 0.999999, 1e-7);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms_fma, e0, e1);
    cudaEventRecord(e0, st);
    k_probe_dmma<<<blocks, PROBE_THREADS, 0, st>>>(sink, it_mma);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms_mma, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, st);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return FC_ERR_CUDA;
  const double threads = (double)blocks * PROBE_THREADS;
  *dfma_gflops = 2.0 * PROBE_CHAINS * (double)it_fma * threads / (ms_fma * 1e-3) / 1e9;
  const double warps = threads / 32.0;
  *dmma_gflops = 2.0 * 8 * 8 * 4 * 4.0 * (double)it_mma * warps / (ms_mma * 1e-3) / 1e9;
  return FC_OK;
}
