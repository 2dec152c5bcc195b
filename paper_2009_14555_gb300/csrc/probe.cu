// probe.cu - measured arithmetic peaks of the device (diagnostic; the paper
// has no counterpart).
//
// The roofline of the FP32-bulk and float64 stage kernels is an ALU one, so
// their fractions need the device's own fused-multiply-add rates, not unit
// counts times a nominal clock.  Each thread runs NCH independent FMA chains
// (enough to cover the pipeline latency) for a fixed number of iterations on
// a grid of several CTAs per SM; the result is written out so that no chain
// is dead code.  FLOPs = 2 per FMA.
#include <cuda_runtime.h>

#include "../../include/dis.h"

int dis_internal_error(int code, const char* fmt, ...);

namespace {

constexpr int NCH = 8;

__device__ __forceinline__ float fma_t(float x, float a, float b) { return fmaf(x, a, b); }
__device__ __forceinline__ double fma_t(double x, double a, double b) { return fma(x, a, b); }

template <class T>
__global__ void __launch_bounds__(512) k_fma_loop(T a, T b, int iters, T* out) {
  T x[NCH];
#pragma unroll
  for (int c = 0; c < NCH; ++c) x[c] = a + (T)(threadIdx.x + c);
  for (int n = 0; n < iters; ++n) {
#pragma unroll
    for (int c = 0; c < NCH; ++c) x[c] = fma_t(x[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < NCH; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
int time_fma(cudaStream_t st, int iters, double* tflops, double* ms_out) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 512, blocks = sms * 4;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)threads * blocks) != cudaSuccess)
    return dis_internal_error(DIS_ENOMEM, "dis_alu_peaks: cannot allocate the output");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // a (0.999...) keeps the chains bounded: x -> a x + b converges to b / (1 - a)
  const T a = (T)0.9999, b = (T)1e-3;
  k_fma_loop<T><<<blocks, threads, 0, st>>>(a, b, 64, out);  // warm-up
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(e0, st);
    k_fma_loop<T><<<blocks, threads, 0, st>>>(a, b, iters, out);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return dis_internal_error(DIS_ECUDA, "dis_alu_peaks: %s", cudaGetErrorString(e));
  const double flop = 2.0 * NCH * (double)iters * threads * blocks;
  *tflops = flop / (best * 1e-3) / 1e12;
  if (ms_out) *ms_out = best;
  return DIS_OK;
}

}  // namespace

extern "C" int dis_alu_peaks(void* stream, double* fp32_tflops, double* fp64_tflops, double* ms) {
  if (!fp32_tflops || !fp64_tflops) return dis_internal_error(DIS_EINVAL, "dis_alu_peaks: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  int rc = time_fma<float>(st, 1 << 14, fp32_tflops, ms ? ms : nullptr);
  if (rc) return rc;
  return time_fma<double>(st, 1 << 9, fp64_tflops, ms ? ms + 1 : nullptr);
}
