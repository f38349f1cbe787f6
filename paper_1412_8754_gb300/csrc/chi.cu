// chi.cu -- the static Cooper pair susceptibility of App. C as one k-space
// map-reduce per pair momentum, in FP64.
//
//   chi_{e e'}(q) = (1/N^2) sum_k eta(-k-q)^2 S(E_{e,k,up}, E_{e',-k-q,down}),
//   S(a, b) = [1 - f(a) - f(b)] / (a + b),
// with E_{e,k,up} = E_e(k) - mu - h, E_{e',-k-q,down} = E_e'(-k-q) - mu + h,
// f the Fermi function at T and eta the s+- structure factor.  (App. C writes
// G = [f(-E_up) - f(E_down)] / (omega - E_up - E_down) at omega -> 0 and
// chi = -(1/N) sum eta^2 G; f(-x) = 1 - f(x) gives the form above.)
//
// S is evaluated without cancellation or overflow: with x = a/2T, z = b/2T,
// 1 - f(a) - f(b) = (tanh x + tanh z)/2 and tanh x + tanh z =
// sinh(x+z)/(cosh x cosh z), so S = sinhc(x+z) / (4 T cosh x cosh z), taken
// as the exponential of ln sinhc(x+z) - ln cosh x - ln cosh z: finite through
// a + b = 0 (where it is the limit f(a) f(-a)/T) and for any |a|/T.
#include <cmath>
#include <vector>

#include "plan.h"

namespace ffe {

namespace {

__device__ __forceinline__ double ln_cosh(double x) {
  const double ax = fabs(x);
  return ax + log1p(exp(-2.0 * ax)) - 0.69314718055994530942;
}

// ln(sinh(y)/y)
__device__ __forceinline__ double ln_sinhc(double y) {
  const double ay = fabs(y);
  if (ay < 1e-3) {
    const double y2 = y * y;
    return y2 / 6.0 - y2 * y2 / 180.0;
  }
  return ay + log1p(-exp(-2.0 * ay)) - 0.69314718055994530942 - log(ay);
}

__device__ __forceinline__ double pair_s(double a, double b, double T) {
  const double x = 0.5 * a / T, z = 0.5 * b / T;
  return exp(ln_sinhc(x + z) - ln_cosh(x) - ln_cosh(z)) / (4.0 * T);
}

// Band energies at momentum (kx, ky) of either model, ascending.
__device__ __forceinline__ int bands_at(const ModelParams& m, double kx, double ky, double (&e)[3]) {
  double sx, cx, sy, cy;
  sincos(kx, &sx, &cx);
  sincos(ky, &sy, &cy);
  if (m.nbands == 3) {
    bands3_at(m, cx, sx, cy, sy, e[0], e[1], e[2]);
    return 3;
  }
  band_pair<double>(m, cx, cy, sx, sy, e[0], e[1]);
  e[2] = 0.0;
  return 2;
}

constexpr int kChiChunk = 16384;  // k-points per block
constexpr int kChiThreads = 256;

__global__ void __launch_bounds__(kChiThreads) chi_kernel(const ModelParams m, int N, const double* __restrict__ qx,
                                                          const double* __restrict__ qy, double h, double T,
                                                          int n_chunks, double* partials, int32_t* counters,
                                                          double* chi) {
  const int q = blockIdx.y, chunk = blockIdx.x;
  const int64_t nk = (int64_t)N * N;
  const int64_t k0 = (int64_t)chunk * kChiChunk, k1 = min(nk, k0 + kChiChunk);
  const int nb = m.nbands;
  const double two_pi_n = 2.0 * 3.14159265358979323846 / (double)N;
  double acc[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) acc[p] = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const int iy = (int)(k / N), ix = (int)(k - (int64_t)iy * N);
    const double kx = two_pi_n * ix, ky = two_pi_n * iy;
    double eu[3], ed[3];
    bands_at(m, kx, ky, eu);
    bands_at(m, -kx - qx[q], -ky - qy[q], ed);
    const double eta = m.eta_amp * cos(kx + qx[q]) * cos(ky + qy[q]);
    const double eta2 = eta * eta;
    for (int e = 0; e < nb; ++e)
      for (int f = 0; f < nb; ++f) acc[e * 3 + f] += eta2 * pair_s(eu[e] - m.mu - h, ed[f] - m.mu + h, T);
  }
  // block reduction of the 9 sums
  __shared__ double red[kChiThreads / 32][9];
  __shared__ int last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    double v = acc[p];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0) red[warp][p] = v;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    double v = 0.0;
    for (int w = 0; w < kChiThreads / 32; ++w) v += red[w][threadIdx.x];
    partials[((int64_t)q * n_chunks + chunk) * 9 + threadIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counters + q, 1) == n_chunks - 1);
  __syncthreads();
  if (last && threadIdx.x < 9) {  // the last block of q adds the chunks in order
    __threadfence();
    double v = 0.0;
    for (int c = 0; c < n_chunks; ++c) v += __ldcg(partials + ((int64_t)q * n_chunks + c) * 9 + threadIdx.x);
    const int e = threadIdx.x / 3, f = threadIdx.x - 3 * (threadIdx.x / 3);
    if (e < nb && f < nb) chi[((int64_t)q * nb + e) * nb + f] = v / (double)nk;
  }
}

}  // namespace
}  // namespace ffe

using namespace ffe;

extern "C" ffe_status ffe_pair_susceptibility(ffe_context* ctx, int32_t N, int32_t n_q, const double* qx,
                                              const double* qy, double h, double T, double* chi, void* stream) {
  if (!ctx) return FFE_EINVAL;
  if (!qx || !qy || !chi || n_q < 1 || n_q > 65535)
    return set_err(ctx, "ffe_pair_susceptibility: NULL array or n_q outside [1, 65535]"), FFE_EINVAL;
  if (N < 2 || N > 8192 || (N % 2) != 0) return set_err(ctx, "N=%d must be even in [2, 8192]", N), FFE_EINVAL;
  if (!(T > 0.0) || !std::isfinite(T) || !std::isfinite(h)) return set_err(ctx, "T <= 0 or non-finite h"), FFE_EINVAL;
  for (int i = 0; i < n_q; ++i)
    if (!std::isfinite(qx[i]) || !std::isfinite(qy[i])) return set_err(ctx, "q %d not finite", i), FFE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = ctx->mp.nbands;
  const int64_t nk = (int64_t)N * N;
  const int n_chunks = (int)((nk + kChiChunk - 1) / kChiChunk);
  double *d_q = nullptr, *d_part = nullptr, *d_chi = nullptr;
  int32_t* d_cnt = nullptr;
  cudaError_t e = cudaMalloc(&d_q, 2 * n_q * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_part, (size_t)n_q * n_chunks * 9 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_chi, (size_t)n_q * nb * nb * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_cnt, n_q * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_q, qx, n_q * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_q + n_q, qy, n_q * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, n_q * sizeof(int32_t), s);
  if (e == cudaSuccess) {
    chi_kernel<<<dim3(n_chunks, n_q), kChiThreads, 0, s>>>(ctx->mp, N, d_q, d_q + n_q, h, T, n_chunks, d_part, d_cnt,
                                                            d_chi);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(chi, d_chi, (size_t)n_q * nb * nb * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (void* p : {(void*)d_q, (void*)d_part, (void*)d_chi, (void*)d_cnt})
    if (p) cudaFree(p);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pair susceptibility");
  return FFE_OK;
}
