// direct.cu -- Omega at the points of one (N, Q) from device arrays, the job
// table written on the device (see direct.cuh).  Eq. freeene summed over the
// lattice by the same kernels as every other entry point (tables, normal-state
// sums, k-sum); only the planning moves from the host to three small kernels.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/ffe.h"
#include "direct.cuh"
#include "ffe_internal.cuh"
#include "plan.h"

namespace ffe {
namespace {

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr int kWinFloats = 8;  // far window of a segment: hlo, hhi, tgap, d2max, d2min, sgl_r (+2 spare)

template <typename T>
__device__ __forceinline__ T* at(unsigned char* base, size_t off) {
  return reinterpret_cast<T*>(base + off);
}

// Per point: validation, (h, T) entry, Delta, the h list of every group; and
// the counters cleared.
__global__ void direct_pack_kernel(DirectShape sh, DirectLayout L, const double* __restrict__ h,
                                   const double* __restrict__ T, const double* __restrict__ delta,
                                   unsigned char* base) {
  const int n_hb = (sh.n + 31) / 32;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t o = i0; o < sh.n; o += stride) {
    const double hv = h[o], tv = T[o], dv = delta[o];
    const bool ok = isfinite(hv) && isfinite(dv) && isfinite(tv) && tv > 0.0;
    at<HT>(base, L.ht)[o] = HT{ok ? hv : 0.0, ok ? tv : 1.0, (int32_t)o, 0};
    at<double>(base, L.delta)[o] = ok ? dv : 0.0;
    at<int32_t>(base, L.bad)[o] = ok ? 0 : 1;
    for (int g = 0; g < sh.n_grp; ++g) at<double>(base, L.hlist)[(int64_t)g * sh.n + o] = ok ? hv : 0.0;
  }
  for (int64_t i = i0; i < 8; i += stride) at<int32_t>(base, L.cnt)[i] = 0;
  for (int64_t i = i0; i < (int64_t)sh.n_grp * sh.n_segs; i += stride) at<int32_t>(base, L.segcnt)[i] = 0;
  for (int64_t i = i0; i < (int64_t)sh.n_grp * n_hb; i += stride) at<int32_t>(base, L.mcnt)[i] = 0;
}

// One warp per segment: the far window of its outputs, as the host planner
// sets it for a LIST group (FP32: h range, 27 ln2 T_max, Delta^2 range; FP64:
// h range, kExpNegligible T_max and the largest Delta^2), rounded outward to float.
__global__ void direct_window_kernel(DirectShape sh, DirectLayout L, unsigned char* base) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) / 32, lane = threadIdx.x & 31;
  if (warp >= sh.n_segs) return;
  const HT* ht = at<HT>(base, L.ht);
  const double* dl = at<double>(base, L.delta);
  const int o0 = warp * kMaxBatchesList * 32, o1 = min(sh.n, (warp + 1) * kMaxBatchesList * 32);
  double hlo = INFINITY, hhi = -INFINITY, tmax = 0.0, d2lo = INFINITY, d2hi = 0.0;
  for (int o = o0 + lane; o < o1; o += 32) {
    const HT e = ht[o];
    hlo = fmin(hlo, e.h);
    hhi = fmax(hhi, e.h);
    tmax = fmax(tmax, e.T);
    const double d2 = dl[o] * dl[o];
    d2lo = fmin(d2lo, d2);
    d2hi = fmax(d2hi, d2);
  }
  for (int m = 16; m > 0; m >>= 1) {
    hlo = fmin(hlo, __shfl_xor_sync(kFull, hlo, m));
    hhi = fmax(hhi, __shfl_xor_sync(kFull, hhi, m));
    tmax = fmax(tmax, __shfl_xor_sync(kFull, tmax, m));
    d2lo = fmin(d2lo, __shfl_xor_sync(kFull, d2lo, m));
    d2hi = fmax(d2hi, __shfl_xor_sync(kFull, d2hi, m));
  }
  if (lane != 0) return;
  float* w = at<float>(base, L.win) + (size_t)warp * kWinFloats;
  const bool f32 = sh.prec == FFE_FP32C;
  const double ln2 = 0.69314718055994530942;
  w[0] = nextafterf(__double2float_rn(hlo), -INFINITY);
  w[1] = nextafterf(__double2float_rn(hhi), INFINITY);
  w[2] = f32 ? nextafterf(__double2float_rn(27.0 * ln2 * tmax + 1e-5), INFINITY)
             : nextafterf(__double2float_rn(kExpNegligible * tmax), INFINITY);
  w[3] = nextafterf(__double2float_rn(d2hi), INFINITY);
  w[4] = f32 ? nextafterf(__double2float_rn(d2lo), 0.0f) : 0.0f;
  w[5] = f32 ? w[2] : INFINITY;
}

// Groups, segments, k-sum work items and normal-state items.
__global__ void direct_table_kernel(DirectShape sh, DirectLayout L, unsigned char* base) {
  const int n_batches = (sh.n + 31) / 32;
  const int64_t nk = (int64_t)sh.N * sh.N;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t i = i0; i < sh.n_grp; i += stride) {
    GroupDesc g;
    memset(&g, 0, sizeof g);
    g.N = sh.N;
    g.layout = kLayoutList;
    g.n_out = sh.n;
    g.n_delta = sh.n;
    g.n_ht = sh.n;
    g.n_hblk = 1;
    g.n_batches = n_batches;
    g.n_h = sh.n;
    g.out_off = i * sh.n;
    g.h_off = i * sh.n;
    g.qx = sh.qx;
    g.qy = sh.qy;
    g.band_only = sh.n_grp > 1 ? (int32_t)i + 1 : 0;
    at<GroupDesc>(base, L.group)[i] = g;
  }
  const int64_t per_grp = (int64_t)sh.n_chunks * n_batches * 32;  // partial sums of one group
  for (int64_t i = i0; i < (int64_t)sh.n_grp * sh.n_segs; i += stride) {
    const int grp = (int)(i / sh.n_segs), sg = (int)(i % sh.n_segs);
    const int b0 = sg * kMaxBatchesList, b1 = min(n_batches, b0 + kMaxBatchesList);
    // every earlier segment of the group has kMaxBatchesList batches
    at<Segment>(base, L.seg)[i] = Segment{grp, b0, b1, sh.n_chunks, grp * per_grp + (int64_t)sh.n_chunks * b0 * 32};
  }
  const float* win = at<float>(base, L.win);
  for (int64_t i = i0; i < sh.n_items; i += stride) {
    const int per = sh.n_segs * sh.n_chunks;
    const int grp = (int)(i / per), r = (int)(i % per);
    const int sg = r / sh.n_chunks, c = r % sh.n_chunks;
    const int b0 = sg * kMaxBatchesList, b1 = min(n_batches, b0 + kMaxBatchesList);
    const float* w = win + (size_t)sg * kWinFloats;
    at<WorkItem>(base, L.items)[i] = WorkItem{grp, grp * sh.n_segs + sg, c, c * sh.ck,
                                              min(sh.n_ksets, (c + 1) * sh.ck), b0, b1, w[0], w[1], w[2], w[3],
                                              w[4], w[5]};
  }
  for (int64_t i = i0; i < sh.n_mitems; i += stride) {
    const int per = n_batches * sh.m_chunks;
    const int grp = (int)(i / per), r = (int)(i % per);
    const int hb = r / sh.m_chunks, c = r % sh.m_chunks;
    const int counter = grp * n_batches + hb;
    at<MItem>(base, L.mitems)[i] = MItem{grp, hb, c, sh.m_chunks, (int64_t)c * kDirectMChunk,
                                         min(nk, (int64_t)(c + 1) * kDirectMChunk),
                                         (int64_t)counter * sh.m_chunks * 32, counter, 0};
  }
}

__global__ void direct_finish_kernel(DirectShape sh, DirectLayout L, const unsigned char* base, double* omega,
                                     double* omega_band) {
  const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= sh.n) return;
  const int32_t status = reinterpret_cast<const int32_t*>(base + L.cnt)[7];
  const bool nan = status != 0 || reinterpret_cast<const int32_t*>(base + L.bad)[o] != 0;
  const double* om = reinterpret_cast<const double*>(base + L.omega);
  if (sh.n_grp == 1) {
    omega[o] = nan ? NAN : om[o];
    return;
  }
  double tot = 0.0;  // the bands in ascending order, as ffe_omega adds them
  for (int b = 0; b < sh.n_grp; ++b) {
    const double v = om[(int64_t)b * sh.n + o];
    if (omega_band) omega_band[o * sh.n_grp + b] = nan ? NAN : v;
    tot += v;
  }
  omega[o] = nan ? NAN : tot;
}

}  // namespace

DirectShape direct_shape(int N, int n, int prec, int nbands, bool per_band, double qx, double qy, int max_items,
                         double n_warps) {
  DirectShape sh;
  std::memset(&sh, 0, sizeof sh);
  sh.N = N;
  sh.n = n;
  sh.prec = prec;
  sh.nbands = nbands;
  sh.n_grp = per_band ? nbands : 1;
  sh.kpt = prec == FFE_FP32C ? 4 : 1;
  sh.qx = qx;
  sh.qy = qy;
  const int n_batches = (n + 31) / 32;
  const int64_t nk = (int64_t)N * N;
  const int kset_pts = 32 * sh.kpt;
  sh.n_ksets = (int)((nk + kset_pts - 1) / kset_pts);
  sh.n_segs = (n_batches + kMaxBatchesList - 1) / kMaxBatchesList;
  const int seg_b = std::min(n_batches, kMaxBatchesList);
  double target = prec == FFE_FP32C ? 8388608.0 : 262144.0;
  if (n_warps > 0.0) {  // a small job gets smaller items, so that every warp finds work
    const double work = (double)sh.n_grp * n_batches * 32.0 * (double)sh.n_ksets * kset_pts;
    target = std::max((double)kset_pts * 32.0, std::min(target, work / (4.0 * n_warps)));
  }
  const int64_t units = (int64_t)sh.n_segs * sh.n_grp;  // item rows, each split into the same k-chunks
  int64_t ck = (int64_t)(target / ((double)seg_b * 32.0 * kset_pts));
  ck = std::max<int64_t>(ck, ((int64_t)sh.n_ksets * units + max_items - 1) / max_items);
  ck = std::max<int64_t>(1, std::min<int64_t>(ck, sh.n_ksets));
  while (((sh.n_ksets + ck - 1) / ck) * units > max_items && ck < sh.n_ksets) ++ck;
  sh.ck = (int)ck;
  sh.n_chunks = (int)((sh.n_ksets + ck - 1) / ck);
  sh.n_items = (int)(sh.n_chunks * units);
  sh.m_chunks = (int)((nk + kDirectMChunk - 1) / kDirectMChunk);
  sh.n_mitems = sh.n_grp * n_batches * sh.m_chunks;
  return sh;
}

DirectLayout direct_layout(const DirectShape& sh) {
  DirectLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at_off = off;
    off = align256(off + std::max<size_t>(bytes, 1));
    return at_off;
  };
  const size_t rows = 2 * (size_t)sh.N;
  const size_t nk = (size_t)sh.N * sh.N;
  const size_t n = sh.n, ng = sh.n_grp;
  const size_t n_batches = (n + 31) / 32;
  L.tabf = take(rows * sizeof(TabRowF));
  L.c0f = take(rows * sizeof(float));
  L.tabd = take(rows * sizeof(TabRowD));
  L.c0d = take(rows * sizeof(double));
  L.tabdf = take(rows * sizeof(TabRowDF));
  const size_t e3 = sh.nbands == 3 ? 2 * nk : 0;
  L.e3d = take(e3 * sizeof(E3D));
  L.e3f = take(e3 * sizeof(float4));
  L.group = take(ng * sizeof(GroupDesc));
  L.seg = take(ng * sh.n_segs * sizeof(Segment));
  L.items = take((size_t)sh.n_items * sizeof(WorkItem));
  L.mitems = take((size_t)sh.n_mitems * sizeof(MItem));
  L.win = take((size_t)sh.n_segs * kWinFloats * sizeof(float));
  L.d2f = take(n * sizeof(float));
  L.ht = take(n * sizeof(HT));
  L.htf = take(n * sizeof(HTf));
  L.htd = take(n * sizeof(HTd));
  L.hlist = take(ng * n * sizeof(double));
  L.delta = take(n * sizeof(double));
  L.bad = take(n * sizeof(int32_t));
  L.M = take(ng * n * sizeof(double));
  L.mpart = take((size_t)sh.n_mitems * 32 * sizeof(double));
  L.mcnt = take(ng * n_batches * sizeof(int32_t));
  L.part = take(ng * (size_t)sh.n_chunks * n_batches * 32 * sizeof(double));
  L.V = take(ng * n * sizeof(double));
  L.eb = take(ng * n * sizeof(double));
  L.omega = take(ng * n * sizeof(double));
  L.cnt = take(8 * sizeof(int32_t));
  L.segcnt = take(ng * sh.n_segs * sizeof(int32_t));
  L.total = off;
  return L;
}

cudaError_t direct_enqueue(const ModelParams& mp, const DirectShape& sh, const DirectLayout& L, unsigned char* base,
                           const double* h, const double* T, const double* delta, double* omega, double* omega_band,
                           int ksum_grid, cudaStream_t s) {
  const int n = sh.n;
  const int pack_grid = std::min(1024, std::max(1, (n + 255) / 256));
  direct_pack_kernel<<<pack_grid, 256, 0, s>>>(sh, L, h, T, delta, base);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  direct_window_kernel<<<(sh.n_segs + 7) / 8, 256, 0, s>>>(sh, L, base);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t rows = std::max<int64_t>({(int64_t)sh.n_items, (int64_t)sh.n_mitems, (int64_t)sh.n_grp * sh.n_segs});
  direct_table_kernel<<<(int)std::min<int64_t>(1024, (rows + 255) / 256), 256, 0, s>>>(sh, L, base);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const GroupDesc* groups = reinterpret_cast<const GroupDesc*>(base + L.group);
  HT* ht = reinterpret_cast<HT*>(base + L.ht);
  e = prep_params_launch(reinterpret_cast<const double*>(base + L.delta), n, reinterpret_cast<float*>(base + L.d2f),
                         ht, n, reinterpret_cast<HTf*>(base + L.htf), reinterpret_cast<HTd*>(base + L.htd), s);
  if (e != cudaSuccess) return e;
  // every group shares the tables of group 0 (same N and Q)
  e = tables_launch(mp, groups, 1, sh.N, reinterpret_cast<TabRowF*>(base + L.tabf),
                    reinterpret_cast<float*>(base + L.c0f), reinterpret_cast<TabRowD*>(base + L.tabd),
                    reinterpret_cast<double*>(base + L.c0d), reinterpret_cast<TabRowDF*>(base + L.tabdf), s);
  if (e != cudaSuccess) return e;
  if (mp.nbands == 3) {
    e = bands3_launch(mp, groups, 1, sh.N, reinterpret_cast<const TabRowD*>(base + L.tabd),
                      reinterpret_cast<E3D*>(base + L.e3d), reinterpret_cast<float4*>(base + L.e3f), s);
    if (e != cudaSuccess) return e;
  }
  e = normal_launch(mp, groups, reinterpret_cast<const MItem*>(base + L.mitems), sh.n_mitems,
                    reinterpret_cast<const double*>(base + L.hlist), reinterpret_cast<const TabRowD*>(base + L.tabd),
                    sh.prec == FFE_FP32C ? reinterpret_cast<const TabRowDF*>(base + L.tabdf) : nullptr,
                    reinterpret_cast<const E3D*>(base + L.e3d), reinterpret_cast<double*>(base + L.mpart),
                    reinterpret_cast<int32_t*>(base + L.mcnt), reinterpret_cast<double*>(base + L.M), s);
  if (e != cudaSuccess) return e;
  KsumArgs a;
  std::memset(&a, 0, sizeof a);
  a.m = mp;
  a.groups = groups;
  a.items = reinterpret_cast<const WorkItem*>(base + L.items);
  a.n_items = sh.n_items;
  a.segs = reinterpret_cast<const Segment*>(base + L.seg);
  a.queue = reinterpret_cast<int32_t*>(base + L.cnt);
  a.seg_count = reinterpret_cast<int32_t*>(base + L.segcnt);
  a.partials = reinterpret_cast<double*>(base + L.part);
  a.tabf = reinterpret_cast<const TabRowF*>(base + L.tabf);
  a.c0f = reinterpret_cast<const float*>(base + L.c0f);
  a.tabd = reinterpret_cast<const TabRowD*>(base + L.tabd);
  a.c0d = reinterpret_cast<const double*>(base + L.c0d);
  a.delta = reinterpret_cast<const double*>(base + L.delta);
  a.d2f = reinterpret_cast<const float*>(base + L.d2f);
  a.ht = ht;
  a.htf = reinterpret_cast<const HTf*>(base + L.htf);
  a.htd = reinterpret_cast<const HTd*>(base + L.htd);
  a.M = reinterpret_cast<const double*>(base + L.M);
  a.V = reinterpret_cast<double*>(base + L.V);
  a.omega = reinterpret_cast<double*>(base + L.omega);
  a.ebound = reinterpret_cast<double*>(base + L.eb);
  a.eb_rel = 0.0;
  a.eb_abs = 0.0;
  a.status = reinterpret_cast<int32_t*>(base + L.cnt) + 7;
  a.w_scaled = sh.prec == FFE_FP32C ? 1 : 0;
  a.e3f = reinterpret_cast<const float4*>(base + L.e3f);
  a.e3d = reinterpret_cast<const E3D*>(base + L.e3d);
  e = ksum_launch(sh.prec, kLayoutList, sh.kpt, a, ksum_grid, 256, s);
  if (e != cudaSuccess) return e;
  direct_finish_kernel<<<(n + 127) / 128, 128, 0, s>>>(sh, L, base, omega, omega_band);
  return cudaGetLastError();
}

}  // namespace ffe

using namespace ffe;

extern "C" ffe_status ffe_omega_async(ffe_context* ctx, int32_t N, double qx, double qy, const double* h,
                                      const double* T, const double* delta, int64_t n, double* omega,
                                      double* omega_band, void* stream) {
  if (!ctx) return FFE_EINVAL;
  if (!h || !T || !delta || !omega) return set_err(ctx, "ffe_omega_async: NULL array"), FFE_EINVAL;
  if (N < 2 || N > 8192 || N % 2) return set_err(ctx, "N=%d must be even in [2, 8192]", N), FFE_EINVAL;
  if (n < 1 || n > ((int64_t)1 << 24)) return set_err(ctx, "n=%lld out of [1, 2^24]", (long long)n), FFE_EINVAL;
  if (!std::isfinite(qx) || !std::isfinite(qy)) return set_err(ctx, "Q not finite"), FFE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int prec = ctx->model.prec;
  int bps = 0;
  cudaError_t e = ksum_occupancy(prec, kLayoutList, prec == FFE_FP32C ? 4 : 1, 256, &bps);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "occupancy");
  bps = std::max(1, bps);
  const DirectShape sh = direct_shape(N, (int)n, prec, ctx->mp.nbands, omega_band != nullptr, qx, qy, 1 << 20,
                                      (double)ctx->n_sm * bps * 8);
  const DirectLayout L = direct_layout(sh);
  if (L.total > ctx->direct_bytes) {  // grow the context's scratch (cudaFree waits for the device)
    if (ctx->direct) cudaFree(ctx->direct);
    ctx->direct = nullptr;
    ctx->direct_bytes = 0;
    e = cudaMalloc(&ctx->direct, L.total);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
    ctx->direct_bytes = L.total;
  }
  e = direct_enqueue(ctx->mp, sh, L, static_cast<unsigned char*>(ctx->direct), h, T, delta, omega, omega_band,
                     ctx->n_sm * bps, s);
  return e == cudaSuccess ? FFE_OK : cuda_fail(ctx, e, "ffe_omega_async");
}
