// probe.cu -- throughput probe of the units the k-sum is bound by: the MUFU
// (ex2, lg2, rsqrt, rcp), the FP32 FMA pipe and the FP64 FMA pipe.  Eight
// independent dependency chains per thread, a persistent grid of resident
// blocks, timed with CUDA events; the result is operations per second.
#include <cstring>

#include "../../include/ffe.h"
#include "ffe_internal.cuh"

namespace ffe {

enum { kOpEx2 = 0, kOpLg2, kOpRsq, kOpRcp, kOpFma32, kOpFma64 };

template <int OP>
__global__ void __launch_bounds__(256) probe_kernel(float* sink, int iters) {
  if constexpr (OP == kOpFma64) {
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 1.0 + threadIdx.x * 1e-7 + j * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) x[j] = fma(x[j], 0.999999, 1e-6);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 12345.0) sink[0] = (float)s;
  } else {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 1.0f + threadIdx.x * 1e-6f + j * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (OP == kOpEx2) x[j] = ex2a(-x[j]);
        if (OP == kOpLg2) x[j] = lg2a(x[j] + 2.0f);
        if (OP == kOpRsq) x[j] = rsqa(x[j]);
        if (OP == kOpRcp) x[j] = rcpa(x[j]);
        if (OP == kOpFma32) x[j] = fmaf(x[j], 0.999999f, 1e-6f);
      }
    }
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 12345.0f) sink[0] = s;
  }
}

template <int OP>
static cudaError_t probe_one(int grid, int iters, float* sink, cudaEvent_t e0, cudaEvent_t e1, double* rate) {
  probe_kernel<OP><<<grid, 256>>>(sink, iters / 8);  // warm-up
  cudaEventRecord(e0);
  probe_kernel<OP><<<grid, 256>>>(sink, iters);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e != cudaSuccess) return e;
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  *rate = (double)grid * 256.0 * 8.0 * (double)iters / (ms * 1e-3);
  return cudaSuccess;
}

}  // namespace ffe

extern "C" ffe_status ffe_probe_peaks(ffe_peaks* out) {
  using namespace ffe;
  if (!out) return FFE_EINVAL;
  std::memset(out, 0, sizeof *out);
  int dev = 0, nsm = 0, clk = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return FFE_ECUDA;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev);
  out->n_sm = nsm;
  out->sm_khz_max = clk;
  float* sink = nullptr;
  if (cudaMalloc(&sink, sizeof(float)) != cudaSuccess) return FFE_ENOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int grid = nsm * 8;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = probe_one<kOpEx2>(grid, 4096, sink, e0, e1, &out->ex2);
  if (e == cudaSuccess) e = probe_one<kOpLg2>(grid, 4096, sink, e0, e1, &out->lg2);
  if (e == cudaSuccess) e = probe_one<kOpRsq>(grid, 4096, sink, e0, e1, &out->rsqrt);
  if (e == cudaSuccess) e = probe_one<kOpRcp>(grid, 4096, sink, e0, e1, &out->rcp);
  if (e == cudaSuccess) e = probe_one<kOpFma32>(grid, 16384, sink, e0, e1, &out->fma32);
  if (e == cudaSuccess) e = probe_one<kOpFma64>(grid, 256, sink, e0, e1, &out->fma64);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  return e == cudaSuccess ? FFE_OK : FFE_ECUDA;
}
