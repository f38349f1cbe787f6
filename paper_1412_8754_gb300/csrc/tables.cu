// tables.cu -- per-group trig tables (the k-lattice and momentum shifts of
// Alg. 1) and the Delta-independent normal-state sum M of the reformulated
// Eq. freeene.
#include "ffe_internal.cuh"
#include "ksum.cuh"

namespace ffe {

// Row t of a group: axis = t / N (0: x, 1: y), i = t % N.  Stores
// cos/sin(2 pi i/N + q/2), cos/sin(2 pi i/N - q/2) and cos(2 pi i/N), computed
// in FP64 and rounded once to FP32 for the FP32 path.
__global__ void tables_kernel(const GroupDesc* __restrict__ groups, TabRowF* tabf, float* c0f,
                              TabRowD* tabd, double* c0d) {
  const GroupDesc g = groups[blockIdx.y];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * g.N) return;
  const int axis = t / g.N;
  const int i = t - axis * g.N;
  const double q = axis == 0 ? g.qx : g.qy;
  const double ang = (2.0 * 3.14159265358979323846) * (double)i / (double)g.N;
  double sp, cp, sm, cm;
  sincos(ang + 0.5 * q, &sp, &cp);
  sincos(ang - 0.5 * q, &sm, &cm);
  const double c0 = cos(ang);
  const int64_t row = g.tab_off + t;
  tabd[row] = TabRowD{cp, sp, cm, sm};
  c0d[row] = c0;
  tabf[row] = TabRowF{(float)cp, (float)sp, (float)cm, (float)sm};
  c0f[row] = (float)c0;
}

cudaError_t tables_launch(const ModelParams&, const GroupDesc* groups, int n_groups, int max_n,
                          TabRowF* tabf, float* c0f, TabRowD* tabd, double* c0d, cudaStream_t s) {
  if (n_groups <= 0) return cudaSuccess;
  dim3 grid((2 * max_n + 255) / 256, n_groups);
  tables_kernel<<<grid, 256, 0, s>>>(groups, tabf, c0f, tabd, c0d);
  return cudaGetLastError();
}

// FP32 / FP64 parameter forms derived from the authoritative FP64 inputs.
__global__ void prep_params_kernel(const double* __restrict__ delta, int64_t n_delta, float* d2f,
                                   const HT* __restrict__ ht, int64_t n_ht, HTf* htf, HTd* htd) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_delta; i += stride) {
    const double d = delta[i];
    d2f[i] = (float)(d * d);
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_ht; i += stride) {
    const HT e = ht[i];
    const double ln2 = 0.69314718055994530942;
    htf[i] = HTf{(float)e.h, (float)(1.0 / (e.T * ln2)), (float)(e.T * ln2), 0.0f};
    htd[i] = HTd{e.h, 1.0 / e.T, e.T, 0.0};
  }
}

cudaError_t prep_params_launch(const double* delta, int64_t n_delta, float* d2f, const HT* ht,
                               int64_t n_ht, HTf* htf, HTd* htd, cudaStream_t s) {
  const int64_t n = n_delta > n_ht ? n_delta : n_ht;
  if (n <= 0) return cudaSuccess;
  int grid = (int)((n + 255) / 256);
  if (grid > 4096) grid = 4096;
  prep_params_kernel<<<grid, 256, 0, s>>>(delta, n_delta, d2f, ht, n_ht, htf, htd);
  return cudaGetLastError();
}

// M(h) = sum_k sum_eps [min(E_eps(k+Q/2) - mu - h, 0) + min(E_eps(-k+Q/2) - mu + h, 0)]
// for up to 32 h values per item, over the item's k range, in FP64.
//
// With u = E(k+Q/2) - mu and d = E(-k+Q/2) - mu the summand is
// min(u, h) + min(d, -h) - 0, so each band value contributes either itself or
// +-h.  Lane j of a warp owns h_j.  A value below every h of the item (u) or
// below every -h (d) adds itself to every h: it goes to a per-lane total S.
// A value above all of them adds +h_j (u) or -h_j (d) to every h: it goes to
// a per-lane integer count C, so that S + C h_j is its contribution to h_j.
// Only the few values inside [h_min, h_max) (or its mirror) need a choice per
// h: they are broadcast to the warp and lane j adds min(value, +-h_j).  Every
// choice is made on FP32 copies; where the copies tie, the two candidates
// differ by at most one FP32 ulp of h.
__global__ void __launch_bounds__(256) normal_kernel(const ModelParams m,
                                                     const GroupDesc* __restrict__ groups,
                                                     const MItem* __restrict__ items,
                                                     const double* __restrict__ hlist,
                                                     const TabRowD* __restrict__ tabd,
                                                     double* partials, int32_t* counters, double* M) {
  __shared__ double red[8][32];
  __shared__ int last_flag;
  const MItem it = items[blockIdx.x];
  const GroupDesc g = groups[it.group];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h0 = it.hb * 32;
  const int nh = min(32, g.n_h - h0);
  const double hj = hlist[g.h_off + h0 + min(lane, nh - 1)];
  const float hjf = (float)hj;
  float hminf = hjf, hmaxf = hjf;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    hminf = fminf(hminf, __shfl_xor_sync(kFull, hminf, s));
    hmaxf = fmaxf(hmaxf, __shfl_xor_sync(kFull, hmaxf, s));
  }
  double S = 0.0, acc = 0.0;
  int C = 0;
  // warp-uniform trip count: every lane takes part in the ballots
  for (int64_t kb = it.k0 + (threadIdx.x & ~31); kb < it.k1; kb += blockDim.x) {
    const int64_t k = kb + lane;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    unsigned rare = 0;
    if (k < it.k1) {
      const int iy = (int)(k / g.N);
      const int ix = (int)(k - (int64_t)iy * g.N);
      const TabRowD rx = tabd[g.tab_off + ix];
      const TabRowD ry = tabd[g.tab_off + g.N + iy];
      band_pair<double>(m, rx.cp, ry.cp, rx.sp, ry.sp, v[0], v[1]);
      band_pair<double>(m, rx.cm, ry.cm, rx.sm, ry.sm, v[2], v[3]);
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] -= m.mu;
      double below = 0.0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float f = (float)v[i];
        // u (i < 2) against h; d (i >= 2) against -h
        const float lo = i < 2 ? hminf : -hmaxf, hi = i < 2 ? hmaxf : -hminf;
        if (f < lo) {
          below += v[i];
        } else if (f >= hi) {
          C += i < 2 ? 1 : -1;
        } else {
          rare |= 1u << i;
        }
      }
      S += below;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      unsigned mask = __ballot_sync(kFull, (rare >> i) & 1u);
      while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        const double x = __shfl_sync(kFull, v[i], src);
        const float xf = (float)x;
        if (i < 2)
          acc += xf < hjf ? x : hj;
        else
          acc += xf < -hjf ? x : -hj;
      }
    }
  }
  // warp totals of S and C, then this lane's M contribution for h_j
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    S += __shfl_xor_sync(kFull, S, s);
    C += __shfl_xor_sync(kFull, C, s);
  }
  red[warp][lane] = (S + (double)C * hj) + acc;
  __syncthreads();
  if (warp == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][lane];
    partials[it.partial_off + (int64_t)it.chunk * 32 + lane] = s;
    __threadfence();
    __syncwarp();
    int prev = 0;
    if (lane == 0) prev = atomicAdd(counters + it.counter, 1);
    prev = __shfl_sync(kFull, prev, 0);
    if (lane == 0) last_flag = (prev == it.n_chunks - 1);
  }
  __syncthreads();
  if (last_flag && warp == 0) {
    __threadfence();
    double s = 0.0;
    for (int c = 0; c < it.n_chunks; ++c) s += __ldcg(partials + it.partial_off + (int64_t)c * 32 + lane);
    if (lane < nh) M[g.h_off + h0 + lane] = s;
    if (lane == 0) counters[it.counter] = 0;
  }
}

cudaError_t normal_launch(const ModelParams& m, const GroupDesc* groups, const MItem* items,
                          int n_items, const double* hlist, const TabRowD* tabd, double* partials,
                          int32_t* counters, double* M, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  normal_kernel<<<n_items, 256, 0, s>>>(m, groups, items, hlist, tabd, partials, counters, M);
  return cudaGetLastError();
}

}  // namespace ffe
