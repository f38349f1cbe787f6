// tables.cu -- per-group trig tables (the k-lattice and momentum shifts of
// Alg. 1) and the Delta-independent normal-state sum M of the reformulated
// Eq. freeene.
#include "ffe_internal.cuh"
#include "ksum.cuh"

namespace ffe {

// Row t of a group: axis = t / N (0: x, 1: y), i = t % N.  Stores
// cos/sin(2 pi i/N + q/2), cos/sin(2 pi i/N - q/2) and cos(2 pi i/N), computed
// in FP64 and rounded once to FP32 for the FP32 path.
__device__ __forceinline__ float2 split_df(double x) {
  const float hi = (float)x;
  return make_float2(hi, (float)(x - (double)hi));
}

__global__ void tables_kernel(const GroupDesc* __restrict__ groups, TabRowF* tabf, float* c0f,
                              TabRowD* tabd, double* c0d, TabRowDF* tabdf) {
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
  if (tabdf) tabdf[row] = TabRowDF{split_df(cp), split_df(sp), split_df(cm), split_df(sm)};
}

cudaError_t tables_launch(const ModelParams&, const GroupDesc* groups, int n_groups, int max_n,
                          TabRowF* tabf, float* c0f, TabRowD* tabd, double* c0d, TabRowDF* tabdf,
                          cudaStream_t s) {
  if (n_groups <= 0) return cudaSuccess;
  dim3 grid((2 * max_n + 255) / 256, n_groups);
  tables_kernel<<<grid, 256, 0, s>>>(groups, tabf, c0f, tabd, c0d, tabdf);
  return cudaGetLastError();
}

// ---- three-band model (App. B): band tables (bands3_at, ffe_internal.cuh) --
// Row (group g, momentum m, lattice point k): m = 0 is k + Q/2 (spin up),
// m = 1 is -k + Q/2 (spin down).  The second is the first at the lattice
// point -k (mod N), so each thread diagonalises k + Q/2 once and writes it to
// row (0, k) and row (1, -k).
__global__ void bands3_kernel(const ModelParams m, const GroupDesc* __restrict__ groups,
                              const TabRowD* __restrict__ tabd, E3D* e3d, float4* e3f) {
  const GroupDesc g = groups[blockIdx.z];
  const int64_t nk = (int64_t)g.N * g.N;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nk) return;
  const int iy = (int)(k / g.N);
  const int ix = (int)(k - (int64_t)iy * g.N);
  const TabRowD rx = tabd[g.tab_off + ix], ry = tabd[g.tab_off + g.N + iy];
  double e0, e1, e2;
  bands3_at(m, rx.cp, rx.sp, ry.cp, ry.sp, e0, e1, e2);
  const int mx = ix == 0 ? 0 : g.N - ix, my = iy == 0 ? 0 : g.N - iy;
  const int64_t row0 = g.e3_off + k, row1 = g.e3_off + nk + (int64_t)my * g.N + mx;
  e3d[row0] = E3D{e0, e1, e2, 0.0};
  e3d[row1] = E3D{e0, e1, e2, 0.0};
  const float4 f = make_float4((float)e0, (float)e1, (float)e2, 0.0f);
  e3f[row0] = f;
  e3f[row1] = f;
}

cudaError_t bands3_launch(const ModelParams& m, const GroupDesc* groups, int n_groups, int max_n,
                          const TabRowD* tabd, E3D* e3d, float4* e3f, cudaStream_t s) {
  if (n_groups <= 0 || m.nbands != 3) return cudaSuccess;
  const int64_t nk = (int64_t)max_n * max_n;
  dim3 grid((unsigned)((nk + 255) / 256), 1, n_groups);
  bands3_kernel<<<grid, 256, 0, s>>>(m, groups, tabd, e3d, e3f);
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

// ---- double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2 (Dekker 1971; Knuth's two-sum; the fused
// multiply-add two-product of Ogita, Rump and Oishi 2005).  About 44 bits of
// precision at FP32-pipe throughput, which on this GPU is ~77x the FP64 pipe's.
struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return DF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  DF s = df_two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return df_quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_neg(DF x) { return DF{-x.hi, -x.lo}; }
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return df_quick_two_sum(p, e);
}
// sqrt by one Newton step from the FP32 root r: r + (x - r^2) / (2 r)
__device__ __forceinline__ DF df_sqrt(DF x) {
  if (!(x.hi > 0.0f)) return DF{0.0f, 0.0f};
  const float r = sqrtf(x.hi);
  const float p = __fmul_rn(r, r);
  const float pe = fmaf(r, r, -p);
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p), pe), x.lo);
  return df_quick_two_sum(r, __fdiv_rn(d, __fmul_rn(2.0f, r)));
}
__device__ __forceinline__ DF df_from(double x) {
  const float hi = (float)x;
  return DF{hi, (float)(x - (double)hi)};
}

struct ModelDF {
  DF a_sum, a_diff, a_c, a_s, mu;  // -(t1+t2), -(t1-t2), -4 t3, -4 t4, mu
};

// App. A eigenvalues at one momentum in double-float (as band_pair).
__device__ __forceinline__ void band_pair_df(const ModelDF& m, DF cx, DF cy, DF sx, DF sy, DF& lo, DF& hi) {
  const DF mean = df_add(df_mul(m.a_sum, df_add(cx, cy)), df_mul(m.a_c, df_mul(cx, cy)));
  const DF half = df_mul(m.a_diff, df_add(cx, df_neg(cy)));
  const DF t12 = df_mul(m.a_s, df_mul(sx, sy));
  const DF root = df_sqrt(df_add(df_mul(half, half), df_mul(t12, t12)));
  lo = df_add(mean, df_neg(root));
  hi = df_add(mean, root);
}

__device__ __forceinline__ double df_to_double(DF x) { return (double)x.hi + (double)x.lo; }

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
// Values of the M sum: FP64, or double-float for FP32 plans.
template <bool DFM>
struct MVal;
template <>
struct MVal<false> {
  using T = double;
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double neg(double a) { return -a; }
  static __device__ __forceinline__ float f32(double a) { return (float)a; }
  static __device__ __forceinline__ double to_double(double a) { return a; }
  static __device__ __forceinline__ double shfl(double a, int src) { return __shfl_sync(kFull, a, src); }
};
template <>
struct MVal<true> {
  using T = DF;
  static __device__ __forceinline__ DF zero() { return DF{0.0f, 0.0f}; }
  static __device__ __forceinline__ DF add(DF a, DF b) { return df_add(a, b); }
  static __device__ __forceinline__ DF neg(DF a) { return df_neg(a); }
  static __device__ __forceinline__ float f32(DF a) { return a.hi; }
  static __device__ __forceinline__ double to_double(DF a) { return df_to_double(a); }
  static __device__ __forceinline__ DF shfl(DF a, int src) {
    return DF{__shfl_sync(kFull, a.hi, src), __shfl_sync(kFull, a.lo, src)};
  }
};

// The band values u_lo, u_hi at k+Q/2, minus mu, in v[0], v[1], and copies of
// them in v[2], v[3] for the sum against -h: M sums min(d, -h) over every k,
// with d = E(-k+Q/2) - mu = u(-k), and k -> -k is a bijection of the lattice
// (the bands are 2 pi-periodic), so that sum equals the sum of min(u, -h).
__device__ __forceinline__ void band_values(const ModelParams& m, const ModelDF&, const TabRowD& rx,
                                            const TabRowD& ry, const TabRowDF&, const TabRowDF&, double (&v)[4]) {
  band_pair<double>(m, rx.cp, ry.cp, rx.sp, ry.sp, v[0], v[1]);
  v[0] -= m.mu;
  v[1] -= m.mu;
  v[2] = v[0];
  v[3] = v[1];
}
__device__ __forceinline__ void band_values(const ModelParams&, const ModelDF& md, const TabRowD&, const TabRowD&,
                                            const TabRowDF& rx, const TabRowDF& ry, DF (&v)[4]) {
  auto f = [](float2 a) { return DF{a.x, a.y}; };
  band_pair_df(md, f(rx.cp), f(ry.cp), f(rx.sp), f(ry.sp), v[0], v[1]);
  const DF nmu = df_neg(md.mu);
  v[0] = df_add(v[0], nmu);
  v[1] = df_add(v[1], nmu);
  v[2] = v[0];
  v[3] = v[1];
}

// M(h) for up to 32 h values per item, over the item's k range.
//
// With u = E(k+Q/2) - mu and d = E(-k+Q/2) - mu the summand is
// min(u, h) + min(d, -h); summed over the lattice, the d of point k is the u
// of point -k, so every d is taken as a copy of u (band_values: one band
// evaluation per k-point), and each value contributes either itself or
// +-h.  Lane j of a warp owns h_j.  A value below every h of the item (u) or
// below every -h (d) adds itself to every h: it goes to a per-lane total S.
// A value above all of them adds +h_j (u) or -h_j (d) to every h: it goes to
// a per-lane integer count C, so that S + C h_j is its contribution to h_j.
// Only the few values inside [h_min, h_max) (or its mirror) need a choice per
// h: they are broadcast to the warp and lane j adds min(value, +-h_j).  Every
// choice is made on FP32 copies; where the copies tie, the two candidates
// differ by at most one FP32 ulp of h.  FP64 plans compute the band values and
// sums in FP64; FP32 plans in double-float (~44 bits), far below their error
// bound, at FP32-pipe speed.
template <bool DFM, bool NB3>
__global__ void __launch_bounds__(256) normal_kernel(const ModelParams m,
                                                     const GroupDesc* __restrict__ groups,
                                                     const MItem* __restrict__ items,
                                                     const double* __restrict__ hlist,
                                                     const TabRowD* __restrict__ tabd,
                                                     const TabRowDF* __restrict__ tabdf,
                                                     const E3D* __restrict__ e3d,
                                                     double* partials, int32_t* counters, double* M) {
  // NU band values at k + Q/2 (u) and NU at -k + Q/2 (d)
  constexpr int NU = NB3 ? 3 : 2;
  constexpr int NV = 2 * NU;
  using V = MVal<DFM>;
  using T = typename V::T;
  __shared__ double red[8][32];
  __shared__ int last_flag;
  const MItem it = items[blockIdx.x];
  const GroupDesc g = groups[it.group];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int h0 = it.hb * 32;
  const int nh = min(32, g.n_h - h0);
  const double hj = hlist[g.h_off + h0 + min(lane, nh - 1)];
  const float hjf = (float)hj;
  T hjv, nhjv;
  if constexpr (DFM) {
    hjv = df_from(hj);
  } else {
    hjv = hj;
  }
  nhjv = V::neg(hjv);
  ModelDF md;
  if constexpr (DFM) {
    md.a_sum = df_from(-(m.t1 + m.t2));
    md.a_diff = df_from(-(m.t1 - m.t2));
    md.a_c = df_from(-4.0 * m.t3);
    md.a_s = df_from(-4.0 * m.t4);
    md.mu = df_from(m.mu);
  }
  float hminf = hjf, hmaxf = hjf;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    hminf = fminf(hminf, __shfl_xor_sync(kFull, hminf, s));
    hmaxf = fmaxf(hmaxf, __shfl_xor_sync(kFull, hmaxf, s));
  }
  T S = V::zero(), acc = V::zero();
  int C = 0;
  const int k1 = (int)it.k1;
  // warp-uniform trip count: every lane takes part in the ballots
  for (int kb = (int)it.k0 + (threadIdx.x & ~31); kb < k1; kb += blockDim.x) {
    const int k = kb + lane;
    T v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = V::zero();
    unsigned rare = 0;
    if (k < k1) {
      if constexpr (NB3) {  // the -k+Q/2 values by the same relabelling (band_values)
        const E3D eu = e3d[g.e3_off + k];
        v[0] = eu.x - m.mu;
        v[1] = eu.y - m.mu;
        v[2] = eu.z - m.mu;
        v[3] = v[0];
        v[4] = v[1];
        v[5] = v[2];
      } else {
        const int iy = k / g.N;
        const int ix = k - iy * g.N;
        TabRowD rx, ry;
        TabRowDF fx, fy;
        if constexpr (DFM) {
          fx = tabdf[g.tab_off + ix];
          fy = tabdf[g.tab_off + g.N + iy];
        } else {
          rx = tabd[g.tab_off + ix];
          ry = tabd[g.tab_off + g.N + iy];
        }
        band_values(m, md, rx, ry, fx, fy, v);
      }
      if (g.band_only) {  // other bands: u, d far above every +-h, min(u, h) + min(d, -h) = 0
#pragma unroll
        for (int b = 0; b < NU; ++b)
          if (b != g.band_only - 1) {
            if constexpr (DFM) {
              v[b] = DF{1e30f, 0.0f};
              v[b + NU] = DF{1e30f, 0.0f};
            } else {
              v[b] = 1e30;
              v[b + NU] = 1e30;
            }
          }
      }
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const float f = V::f32(v[i]);
        // u (i < NU) against h; d (i >= NU) against -h
        const float lo = i < NU ? hminf : -hmaxf, hi = i < NU ? hmaxf : -hminf;
        if (f < lo) {
          S = V::add(S, v[i]);
        } else if (f >= hi) {
          C += i < NU ? 1 : -1;
        } else {
          rare |= 1u << i;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      unsigned mask = __ballot_sync(kFull, (rare >> i) & 1u);
      while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        const T x = V::shfl(v[i], src);
        const float xf = V::f32(x);
        if (i < NU)
          acc = V::add(acc, xf < hjf ? x : hjv);
        else
          acc = V::add(acc, xf < -hjf ? x : nhjv);
      }
    }
  }
  // warp totals of S and C, then this lane's M contribution for h_j
  double Sd = V::to_double(S);
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    Sd += __shfl_xor_sync(kFull, Sd, s);
    C += __shfl_xor_sync(kFull, C, s);
  }
  red[warp][lane] = (Sd + (double)C * hj) + V::to_double(acc);
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
                          int n_items, const double* hlist, const TabRowD* tabd, const TabRowDF* tabdf,
                          const E3D* e3d, double* partials, int32_t* counters, double* M, cudaStream_t s) {
  if (n_items <= 0) return cudaSuccess;
  if (m.nbands == 3)  // FP64 band tables, either precision
    normal_kernel<false, true><<<n_items, 256, 0, s>>>(m, groups, items, hlist, tabd, tabdf, e3d, partials,
                                                       counters, M);
  else if (tabdf)
    normal_kernel<true, false><<<n_items, 256, 0, s>>>(m, groups, items, hlist, tabd, tabdf, e3d, partials,
                                                       counters, M);
  else
    normal_kernel<false, false><<<n_items, 256, 0, s>>>(m, groups, items, hlist, tabd, tabdf, e3d, partials,
                                                        counters, M);
  return cudaGetLastError();
}

}  // namespace ffe
