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

// Band energies at a momentum given by (cos, sin) of each component, ascending.
__device__ __forceinline__ int bands_at(const ModelParams& m, double cx, double sx, double cy, double sy,
                                        double (&e)[3]) {
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

// (cos, sin) of both components of a pair momentum.
struct __align__(16) QTrig {
  double cx, sx, cy, sy;
};

// cs[i] = (cos, sin)(2 pi i / N), i < N; cq[q] = (cos qx, sin qx, cos qy, sin qy).
// The momenta k and -k-q take their cosines and sines from these by the
// angle-sum identities; ln cosh is formed once per band and momentum.
__global__ void __launch_bounds__(kChiThreads) chi_kernel(const ModelParams m, int N, const double2* __restrict__ cs,
                                                          const QTrig* __restrict__ cq, double h, double T,
                                                          int n_chunks, double* partials, int32_t* counters,
                                                          double* chi) {
  const int q = blockIdx.y, chunk = blockIdx.x;
  const int64_t nk = (int64_t)N * N;
  const int64_t k0 = (int64_t)chunk * kChiChunk, k1 = min(nk, k0 + kChiChunk);
  const int nb = m.nbands;
  const QTrig qq = cq[q];
  const double half_inv_t = 0.5 / T;
  double acc[9];
#pragma unroll
  for (int p = 0; p < 9; ++p) acc[p] = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const int iy = (int)(k / N), ix = (int)(k - (int64_t)iy * N);
    const double2 tx = cs[ix], ty = cs[iy];
    // k + q: cos(a + b) = ca cb - sa sb, sin(a + b) = sa cb + ca sb; -k-q: cos even, sin odd
    const double cxq = tx.x * qq.cx - tx.y * qq.sx, sxq = tx.y * qq.cx + tx.x * qq.sx;
    const double cyq = ty.x * qq.cy - ty.y * qq.sy, syq = ty.y * qq.cy + ty.x * qq.sy;
    double eu[3], ed[3];
    bands_at(m, tx.x, tx.y, ty.x, ty.y, eu);
    bands_at(m, cxq, -sxq, cyq, -syq, ed);
    const double eta = m.eta_amp * cxq * cyq;
    const double eta2 = eta * eta;
    double xu[3], lu[3], zd[3], ld[3];
    for (int e = 0; e < nb; ++e) {
      xu[e] = (eu[e] - m.mu - h) * half_inv_t;
      zd[e] = (ed[e] - m.mu + h) * half_inv_t;
      lu[e] = ln_cosh(xu[e]);
      ld[e] = ln_cosh(zd[e]);
    }
    const double w = eta2 / (4.0 * T);
    for (int e = 0; e < nb; ++e)
      for (int f = 0; f < nb; ++f) acc[e * 3 + f] += w * exp(ln_sinhc(xu[e] + zd[f]) - lu[e] - ld[f]);
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
  std::vector<double2> cs(N);
  std::vector<QTrig> cq(n_q);
  const double two_pi_n = 2.0 * 3.14159265358979323846 / (double)N;
  for (int i = 0; i < N; ++i) cs[i] = make_double2(std::cos(two_pi_n * i), std::sin(two_pi_n * i));
  for (int i = 0; i < n_q; ++i) cq[i] = QTrig{std::cos(qx[i]), std::sin(qx[i]), std::cos(qy[i]), std::sin(qy[i])};
  double2* d_cs = nullptr;
  QTrig* d_cq = nullptr;
  double *d_part = nullptr, *d_chi = nullptr;
  int32_t* d_cnt = nullptr;
  cudaError_t e = cudaMalloc(&d_cs, N * sizeof(double2));
  if (e == cudaSuccess) e = cudaMalloc(&d_cq, n_q * sizeof(QTrig));
  if (e == cudaSuccess) e = cudaMalloc(&d_part, (size_t)n_q * n_chunks * 9 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_chi, (size_t)n_q * nb * nb * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_cnt, n_q * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_cs, cs.data(), N * sizeof(double2), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_cq, cq.data(), n_q * sizeof(QTrig), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, n_q * sizeof(int32_t), s);
  if (e == cudaSuccess) {
    chi_kernel<<<dim3(n_chunks, n_q), kChiThreads, 0, s>>>(ctx->mp, N, d_cs, d_cq, h, T, n_chunks, d_part, d_cnt,
                                                            d_chi);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(chi, d_chi, (size_t)n_q * nb * nb * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (void* p : {(void*)d_cs, (void*)d_cq, (void*)d_part, (void*)d_chi, (void*)d_cnt})
    if (p) cudaFree(p);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pair susceptibility");
  return FFE_OK;
}
