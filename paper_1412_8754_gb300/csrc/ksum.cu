// ksum.cu -- the k-sum of Eq. freeene (Sec. 2) as one persistent map-reduce.
//
// Each warp repeatedly takes a work item (group, k-set range, output-batch
// range) from a global atomic queue.  For every k-set of 32*KPT lattice points
// it builds the per-k band state in registers from the trig tables (App. A
// band energies at k+Q/2 and -k+Q/2: no band energies are stored in memory),
// then for every batch of 32 outputs evaluates the k-point term v_k of each
// output (see ffe_internal.cuh), sums it over the warp's k-points, and folds
// the 32 per-lane sums into one value per output with a butterfly
// reduce-scatter.  The warp keeps FP64 accumulators per output in shared
// memory; at the end of the item it writes them as one partial per output and
// the last warp to finish a segment (a fixed output range) adds the partials
// of all its k-chunks in a fixed order (deterministic) and writes
//   Omega = M + V + 2 N^2 Delta^2 / U
// together with an error bound for FP32 evaluation.  This replaces the
// paper's per-block partial sums + second reduction kernel + host-side
// remainder (Sec. 3, Alg. 2 and the three steps around it) by one launch.
#include <type_traits>

#include "ffe_internal.cuh"
#include "ksum.cuh"

namespace ffe {

// Batch parameters staged in shared memory, one entry per output of a batch.
struct BParF {  // FP32: Delta^2 (LIST only), h, c = 1/(T ln 2), T ln 2
  float d2, h, c, tl;
};
struct BParD {  // FP64: Delta^2 (LIST only), h, 1/T, T
  double d2, h, inv_t, t;
};

template <typename Real>
using BPar = typename std::conditional<std::is_same<Real, float>::value, BParF, BParD>::type;

template <typename Real>
__device__ __forceinline__ void load_row(const KsumArgs& a, int64_t row, TabRowF& r, float& c0) {
  r = a.tabf[row];
  c0 = a.c0f[row];
}
template <typename Real>
__device__ __forceinline__ void load_row(const KsumArgs& a, int64_t row, TabRowD& r, double& c0) {
  r = a.tabd[row];
  c0 = a.c0d[row];
}

template <typename Real, int KPT>
__device__ __forceinline__ void build_states(const KsumArgs& a, const GroupDesc& g, int ks, int lane,
                                             KState<Real> (&st)[KPT]) {
  using Row = typename std::conditional<std::is_same<Real, float>::value, TabRowF, TabRowD>::type;
  const int64_t nk = (int64_t)g.N * g.N;
#pragma unroll
  for (int j = 0; j < KPT; ++j) {
    const int64_t kidx = (int64_t)ks * (32 * KPT) + j * 32 + lane;
    if (kidx < nk) {
      const int iy = (int)(kidx / g.N);
      const int ix = (int)(kidx - (int64_t)iy * g.N);
      Row rx, ry;
      Real c0x, c0y;
      load_row<Real>(a, g.tab_off + ix, rx, c0x);
      load_row<Real>(a, g.tab_off + g.N + iy, ry, c0y);
      kstate_make<Real, Row>(a.m, rx, ry, c0x, c0y, st[j]);
    } else {
      kstate_invalid<Real>(st[j]);
    }
  }
}

// Stage the parameters of batch b (32 outputs) into this warp's shared slot.
// Returns the number of valid outputs in the batch.
template <typename Real, int LAYOUT>
__device__ __forceinline__ int stage_batch(const KsumArgs& a, const GroupDesc& g, int b, int lane,
                                           BPar<Real>* bp, int& delta_i) {
  int nvalid;
  int64_t ht_e, d_e;
  if (LAYOUT == kLayoutProduct) {
    delta_i = b / g.n_hblk;
    const int j0 = (b - delta_i * g.n_hblk) * 32;
    nvalid = min(32, g.n_ht - j0);
    ht_e = g.ht_off + j0 + lane;
    d_e = g.delta_off + delta_i;
  } else {
    delta_i = -1;
    const int o0 = b * 32;
    nvalid = min(32, g.n_out - o0);
    ht_e = g.ht_off + o0 + lane;
    d_e = g.delta_off + o0 + lane;
  }
  __syncwarp();
  BPar<Real> p;
  if (lane < nvalid) {
    if constexpr (std::is_same<Real, float>::value) {
      const HTf q = a.htf[ht_e];
      p.d2 = (LAYOUT == kLayoutList) ? a.d2f[d_e] : 0.0f;
      p.h = q.h;
      p.c = q.c;
      p.tl = q.tl;
    } else {
      const HTd q = a.htd[ht_e];
      const double dd = (LAYOUT == kLayoutList) ? a.delta[d_e] : 0.0;
      p.d2 = dd * dd;
      p.h = q.h;
      p.inv_t = q.inv_t;
      p.t = q.t;
    }
  } else {
    p.d2 = 0;
    p.h = 0;
    if constexpr (std::is_same<Real, float>::value) {
      p.c = 0;
      p.tl = 0;
    } else {
      p.inv_t = 0;
      p.t = 0;
    }
  }
  bp[lane] = p;
  __syncwarp();
  return nvalid;
}

// v_k summed over this lane's KPT k-points for one output (both bands).
template <int KPT>
__device__ __forceinline__ float v_sum_f32(const KState<float> (&st)[KPT], const float (&R)[KPT][2],
                                           const float (&A)[KPT][2], const BParF& p) {
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    float p0, f0, p1, f1;
    band_term_f32(R[k][0], A[k][0], st[k].as[0], st[k].d0[0], p.h, p.c, p0, f0);
    band_term_f32(R[k][1], A[k][1], st[k].as[1], st[k].d0[1], p.h, p.c, p1, f1);
    const float v = fmaf(-p.tl, lg2a(p0 * p1), f0 + f1);
    s += v;
  }
  return s;
}

template <int KPT>
__device__ __forceinline__ double v_sum_f64(const KState<double> (&st)[KPT], const double (&R)[KPT][2],
                                            const double (&A)[KPT][2], const BParD& p) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    double q0, f0, q1, f1;
    band_term_f64(R[k][0], A[k][0], st[k].as[0], st[k].d0[0], p.h, p.inv_t, q0, f0);
    band_term_f64(R[k][1], A[k][1], st[k].as[1], st[k].d0[1], p.h, p.inv_t, q1, f1);
    const double Q = q0 + q1 + q0 * q1;  // (1+q0)(1+q1) - 1
    s += (f0 + f1) - p.t * log1p(Q);
  }
  return s;
}

template <typename Real, int KPT>
__device__ __forceinline__ void ra_all(const KState<Real> (&st)[KPT], Real d2, Real (&R)[KPT][2],
                                       Real (&A)[KPT][2]) {
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const Real D = d2 * st[k].eta2;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if constexpr (std::is_same<Real, float>::value)
        ra_f32(D, st[k].s2[b], st[k].as[b], R[k][b], A[k][b]);
      else
        ra_f64(D, st[k].s2[b], st[k].as[b], R[k][b], A[k][b]);
    }
  }
}

// One batch: returns, in lane l, the warp's sum for output l of the batch.
template <typename Real, int KPT, int LAYOUT>
__device__ __forceinline__ Real eval_batch(const KsumArgs& a, const KState<Real> (&st)[KPT],
                                           const BPar<Real>* bp, int nvalid, Real d2_product, int lane) {
  Real part[32];
  if (LAYOUT == kLayoutProduct) {
    Real R[KPT][2], A[KPT][2];
    ra_all<Real, KPT>(st, d2_product, R, A);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      Real s = (Real)0;
      if (j < nvalid) {
        const BPar<Real> p = bp[j];
        if constexpr (std::is_same<Real, float>::value)
          s = v_sum_f32<KPT>(st, R, A, p);
        else
          s = v_sum_f64<KPT>(st, R, A, p);
      }
      part[j] = s;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      Real s = (Real)0;
      if (j < nvalid) {
        const BPar<Real> p = bp[j];
        Real R[KPT][2], A[KPT][2];
        ra_all<Real, KPT>(st, (Real)p.d2, R, A);
        if constexpr (std::is_same<Real, float>::value)
          s = v_sum_f32<KPT>(st, R, A, p);
        else
          s = v_sum_f64<KPT>(st, R, A, p);
      }
      part[j] = s;
    }
  }
  return reduce_scatter32<Real>(part, lane);
}

// Output index (within the group) of lane `lane` in batch b, or -1.
__device__ __forceinline__ int batch_output(const GroupDesc& g, int b, int lane, int& delta_i,
                                            int& ht_i) {
  if (g.layout == kLayoutProduct) {
    delta_i = b / g.n_hblk;
    ht_i = (b - delta_i * g.n_hblk) * 32 + lane;
    if (ht_i >= g.n_ht) return -1;
    return delta_i * g.n_ht + ht_i;
  }
  const int o = b * 32 + lane;
  if (o >= g.n_out) return -1;
  delta_i = o;
  ht_i = o;
  return o;
}

// Last warp of a segment: add the chunk partials in chunk order and finish.
__device__ void finalize_segment(const KsumArgs& a, const Segment& sg, const GroupDesc& g, int lane) {
  const int nb = sg.b1 - sg.b0;
  const double n2 = (double)g.N * (double)g.N;
  for (int b = sg.b0; b < sg.b1; ++b) {
    int di, hi;
    const int o = batch_output(g, b, lane, di, hi);
    if (o < 0) continue;
    const double* src = a.partials + sg.partial_off + (int64_t)(b - sg.b0) * 32 + lane;
    double V = 0.0;
    for (int c = 0; c < sg.n_chunks; ++c) V += __ldcg(src + (int64_t)c * nb * 32);
    const double dl = a.delta[g.delta_off + di];
    const HT ht = a.ht[g.ht_off + hi];
    const double M = a.M[g.h_off + ht.h_idx];
    const int64_t out = g.out_off + o;
    a.V[out] = V;
    a.omega[out] = M + V + 2.0 * n2 * dl * dl / a.m.U;
    a.ebound[out] = a.eb_rel * fabs(V) + a.eb_abs * n2 * ht.T;
  }
}

template <typename Real, int KPT, int LAYOUT>
__global__ void __launch_bounds__(256) ksum_kernel(const KsumArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  double* acc = reinterpret_cast<double*>(smem_raw) + (size_t)warp * (kMaxBatchesPerItem * 32);
  BPar<Real>* bp = reinterpret_cast<BPar<Real>*>(smem_raw + (size_t)nwarps * kMaxBatchesPerItem * 32 *
                                                               sizeof(double)) +
                   warp * 32;
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(a.queue, 1);
    it = __shfl_sync(kFull, it, 0);
    if (it >= a.n_items) break;
    const WorkItem w = a.items[it];
    const GroupDesc g = a.groups[w.group];
    const int nb = w.b1 - w.b0;
    if (nb > kMaxBatchesPerItem || g.layout != LAYOUT) {
      if (lane == 0) atomicOr(a.status, 1);
      continue;
    }
    for (int b = 0; b < nb; ++b) acc[b * 32 + lane] = 0.0;
    for (int ks = w.kset0; ks < w.kset1; ++ks) {
      KState<Real> st[KPT];
      build_states<Real, KPT>(a, g, ks, lane, st);
      for (int b = w.b0; b < w.b1; ++b) {
        int di;
        const int nvalid = stage_batch<Real, LAYOUT>(a, g, b, lane, bp, di);
        Real d2p = (Real)0;
        if (LAYOUT == kLayoutProduct) {
          if constexpr (std::is_same<Real, float>::value)
            d2p = a.d2f[g.delta_off + di];
          else {
            const double dd = a.delta[g.delta_off + di];
            d2p = dd * dd;
          }
        }
        const Real tot = eval_batch<Real, KPT, LAYOUT>(a, st, bp, nvalid, d2p, lane);
        acc[(b - w.b0) * 32 + lane] += (double)tot;
      }
    }
    const Segment sg = a.segs[w.seg];
    double* dst = a.partials + sg.partial_off + (int64_t)w.chunk * nb * 32;
    for (int b = 0; b < nb; ++b) dst[b * 32 + lane] = acc[b * 32 + lane];
    __threadfence();
    __syncwarp();
    int prev = 0;
    if (lane == 0) prev = atomicAdd(a.seg_count + w.seg, 1);
    prev = __shfl_sync(kFull, prev, 0);
    if (prev == sg.n_chunks - 1) {
      __threadfence();
      finalize_segment(a, sg, g, lane);
      __syncwarp();
      if (lane == 0) a.seg_count[w.seg] = 0;  // ready for the next launch
    }
  }
}

size_t ksum_smem_bytes(int prec, int block_threads) {
  const int nw = block_threads / 32;
  const size_t par = (prec == 1) ? sizeof(BParF) : sizeof(BParD);
  return (size_t)nw * (kMaxBatchesPerItem * 32 * sizeof(double) + 32 * par);
}

template <typename Real, int KPT, int LAYOUT>
static cudaError_t launch_one(const KsumArgs& a, int grid, int block, size_t smem, cudaStream_t s) {
  auto k = ksum_kernel<Real, KPT, LAYOUT>;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  if (cs == cudaStreamCaptureStatusNone) {  // during capture the attribute is already set (occupancy query)
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename Real, int KPT, int LAYOUT>
static cudaError_t occupancy_one(int block, size_t smem, int* blocks_per_sm) {
  auto k = ksum_kernel<Real, KPT, LAYOUT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, block, smem);
}

#define FFE_KSUM_DISPATCH(FN, ...)                                                         \
  do {                                                                                     \
    if (prec == 1) {                                                                       \
      if (layout == kLayoutProduct) {                                                      \
        if (kpt == 2) return FN<float, 2, kLayoutProduct>(__VA_ARGS__);                    \
        if (kpt == 4) return FN<float, 4, kLayoutProduct>(__VA_ARGS__);                    \
        if (kpt == 8) return FN<float, 8, kLayoutProduct>(__VA_ARGS__);                    \
      } else {                                                                             \
        if (kpt == 2) return FN<float, 2, kLayoutList>(__VA_ARGS__);                       \
        if (kpt == 4) return FN<float, 4, kLayoutList>(__VA_ARGS__);                       \
        if (kpt == 8) return FN<float, 8, kLayoutList>(__VA_ARGS__);                       \
      }                                                                                    \
    } else {                                                                               \
      if (layout == kLayoutProduct) {                                                      \
        if (kpt == 1) return FN<double, 1, kLayoutProduct>(__VA_ARGS__);                   \
        if (kpt == 2) return FN<double, 2, kLayoutProduct>(__VA_ARGS__);                   \
      } else {                                                                             \
        if (kpt == 1) return FN<double, 1, kLayoutList>(__VA_ARGS__);                      \
        if (kpt == 2) return FN<double, 2, kLayoutList>(__VA_ARGS__);                      \
      }                                                                                    \
    }                                                                                      \
    return cudaErrorInvalidValue;                                                          \
  } while (0)

cudaError_t ksum_launch(int prec, int layout, int kpt, const KsumArgs& a, int grid, int block,
                        cudaStream_t s) {
  const size_t smem = ksum_smem_bytes(prec, block);
  FFE_KSUM_DISPATCH(launch_one, a, grid, block, smem, s);
}

cudaError_t ksum_occupancy(int prec, int layout, int kpt, int block, int* blocks_per_sm) {
  const size_t smem = ksum_smem_bytes(prec, block);
  FFE_KSUM_DISPATCH(occupancy_one, block, smem, blocks_per_sm);
}

bool ksum_kpt_supported(int prec, int kpt) {
  return prec == 1 ? (kpt == 2 || kpt == 4 || kpt == 8) : (kpt == 1 || kpt == 2);
}

}  // namespace ffe
