// noalloc.cu -- Omega at up to 512 points of one (N, Q) with no allocation.
//
// Some callers cannot allocate device memory at the moment they need a free
// energy: a service that has handed all free device memory to its own pool
// (a cudaMalloc there fails or evicts its cache), or a latency-critical loop
// in which cudaMalloc/cudaFree would synchronise the device and stall the
// other streams.  ffe_omega_noalloc serves them: the caller passes its own
// device arrays for the inputs and the output, and every intermediate (trig
// tables, work queue, partial sums, normal-state sums) lives in one
// file-scope __device__ array of fixed size.  Nothing is allocated, on the
// device or the host, during a call.
//
// The array is shared by every call on a device and keeps the contents of
// the last call; all counters are cleared at the start of each call.  Calls
// that overlap on the GPU (on different streams, or from different host
// threads) race on it and must be serialised by the caller.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/ffe.h"
#include "ffe_internal.cuh"
#include "ksum.cuh"

namespace ffe {
namespace {

constexpr int kNAMaxN = 2048;     // largest lattice
constexpr int kNAMaxOut = 512;    // most points per call
constexpr int kNAMaxItems = 256;  // k-sum work items
constexpr int kNAMaxMItems = 2048;
constexpr int64_t kNAMChunk = 32768;  // k-points per normal-state work item
constexpr size_t kNAScratchBytes = size_t(4) << 20;  // 4 MiB

static __device__ __align__(256) unsigned char g_na_scratch[kNAScratchBytes];

constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte offsets of the regions inside the scratch array.
constexpr size_t kOffTabF = 0;
constexpr size_t kOffC0F = align256(kOffTabF + 2 * kNAMaxN * sizeof(TabRowF));
constexpr size_t kOffTabD = align256(kOffC0F + 2 * kNAMaxN * sizeof(float));
constexpr size_t kOffC0D = align256(kOffTabD + 2 * kNAMaxN * sizeof(TabRowD));
constexpr size_t kOffTabDF = align256(kOffC0D + 2 * kNAMaxN * sizeof(double));
constexpr size_t kOffGroup = align256(kOffTabDF + 2 * kNAMaxN * sizeof(TabRowDF));
constexpr size_t kOffSeg = align256(kOffGroup + sizeof(GroupDesc));
constexpr int kNAMaxSegs = (kNAMaxOut / 32 + kMaxBatchesList - 1) / kMaxBatchesList;
constexpr size_t kOffItems = align256(kOffSeg + kNAMaxSegs * sizeof(Segment));
constexpr size_t kOffMItems = align256(kOffItems + kNAMaxItems * sizeof(WorkItem));
constexpr size_t kOffD2F = align256(kOffMItems + kNAMaxMItems * sizeof(MItem));
constexpr size_t kOffHT = align256(kOffD2F + kNAMaxOut * sizeof(float));
constexpr size_t kOffHTF = align256(kOffHT + kNAMaxOut * sizeof(HT));
constexpr size_t kOffHTD = align256(kOffHTF + kNAMaxOut * sizeof(HTf));
constexpr size_t kOffHList = align256(kOffHTD + kNAMaxOut * sizeof(HTd));
constexpr size_t kOffM = align256(kOffHList + kNAMaxOut * sizeof(double));
constexpr size_t kOffMPart = align256(kOffM + kNAMaxOut * sizeof(double));
constexpr size_t kOffMCnt = align256(kOffMPart + size_t(kNAMaxMItems) * 32 * sizeof(double));
constexpr size_t kOffPart = align256(kOffMCnt + 64 * sizeof(int32_t));
// partials: every k-chunk of every batch: <= kNAMaxItems items of <= kMaxBatchesList batches
constexpr size_t kOffV = align256(kOffPart + size_t(kNAMaxItems) * kMaxBatchesList * 32 * sizeof(double));
constexpr size_t kOffEB = align256(kOffV + kNAMaxOut * sizeof(double));
constexpr size_t kOffCnt = align256(kOffEB + kNAMaxOut * sizeof(double));
constexpr size_t kOffSegCnt = align256(kOffCnt + 8 * sizeof(int32_t));
constexpr size_t kOffBad = align256(kOffSegCnt + kNAMaxSegs * sizeof(int32_t));
constexpr size_t kOffDelta = align256(kOffBad + kNAMaxOut * sizeof(int32_t));
constexpr size_t kNAUsed = align256(kOffDelta + kNAMaxOut * sizeof(double));
static_assert(kNAUsed <= kNAScratchBytes, "scratch regions exceed the static array");

// Device address of g_na_scratch per device, obtained once with that device current.
constexpr int kNAMaxDevices = 64;
void* g_na_addr[kNAMaxDevices] = {};
std::mutex g_na_mutex;

// Shape of one call's job table, computed on the host from (N, n) alone; the
// tables themselves are written on the device by na_setup_kernel.
struct NAShape {
  int32_t N, n, prec;
  int32_t n_segs, n_chunks, ck, n_ksets, n_items;
  int32_t m_chunks, n_mitems;
  double qx, qy;
};

// One block of kNAMaxOut threads: validates the points, writes the (h, T)
// entries, the job table (group, segments, work items with the far windows of
// their outputs, normal-state items) and clears the counters.  An invalid
// point (T <= 0 or a non-finite h, T or Delta) is computed as (h, T, Delta) =
// (0, 1, 0), flagged, and gets Omega = NaN from na_finish_kernel.
__global__ void __launch_bounds__(kNAMaxOut) na_setup_kernel(NAShape sh, const double* __restrict__ h,
                                                            const double* __restrict__ T,
                                                            const double* __restrict__ delta, unsigned char* base) {
  HT* ht = reinterpret_cast<HT*>(base + kOffHT);
  double* hlist = reinterpret_cast<double*>(base + kOffHList);
  double* dl = reinterpret_cast<double*>(base + kOffDelta);
  int32_t* bad = reinterpret_cast<int32_t*>(base + kOffBad);
  const int o = threadIdx.x;
  if (o < sh.n) {
    const double hv = h[o], tv = T[o], dv = delta[o];
    const bool ok = isfinite(hv) && isfinite(dv) && isfinite(tv) && tv > 0.0;
    ht[o] = HT{ok ? hv : 0.0, ok ? tv : 1.0, o, 0};
    hlist[o] = ok ? hv : 0.0;
    dl[o] = ok ? dv : 0.0;
    bad[o] = ok ? 0 : 1;
  }
  int32_t* cnt = reinterpret_cast<int32_t*>(base + kOffCnt);
  int32_t* segcnt = reinterpret_cast<int32_t*>(base + kOffSegCnt);
  int32_t* mcnt = reinterpret_cast<int32_t*>(base + kOffMCnt);
  if (o < 8) cnt[o] = 0;
  if (o < kNAMaxSegs) segcnt[o] = 0;
  if (o < 64) mcnt[o] = 0;
  __syncthreads();
  // the far window of each segment (item_far_window of the plans, LIST layout)
  __shared__ float w_hlo[kNAMaxSegs], w_hhi[kNAMaxSegs], w_tgap[kNAMaxSegs], w_d2max[kNAMaxSegs],
      w_d2min[kNAMaxSegs], w_sglr[kNAMaxSegs];
  if (o < sh.n_segs) {
    const int o0 = o * kMaxBatchesList * 32, o1 = min(sh.n, (o + 1) * kMaxBatchesList * 32);
    double hlo = INFINITY, hhi = -INFINITY, tmax = 0.0, d2lo = INFINITY, d2hi = 0.0;
    for (int i = o0; i < o1; ++i) {
      const HT e = ht[i];
      hlo = fmin(hlo, e.h);
      hhi = fmax(hhi, e.h);
      tmax = fmax(tmax, e.T);
      const double d2 = dl[i] * dl[i];
      d2lo = fmin(d2lo, d2);
      d2hi = fmax(d2hi, d2);
    }
    const bool f32 = sh.prec == FFE_FP32C;
    w_hlo[o] = nextafterf(__double2float_rn(hlo), -INFINITY);
    w_hhi[o] = nextafterf(__double2float_rn(hhi), INFINITY);
    const double ln2 = 0.69314718055994530942;
    w_tgap[o] = f32 ? nextafterf(__double2float_rn(27.0 * ln2 * tmax + 1e-5), INFINITY)
                    : nextafterf(__double2float_rn(750.0 * tmax), INFINITY);
    w_d2max[o] = f32 ? nextafterf(__double2float_rn(d2hi), INFINITY) : INFINITY;
    w_d2min[o] = f32 ? nextafterf(__double2float_rn(d2lo), 0.0f) : 0.0f;
    w_sglr[o] = f32 ? w_tgap[o] : INFINITY;
  }
  __syncthreads();
  const int n_batches = (sh.n + 31) / 32;
  if (o == 0) {
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
    g.qx = sh.qx;
    g.qy = sh.qy;
    *reinterpret_cast<GroupDesc*>(base + kOffGroup) = g;
  }
  Segment* segs = reinterpret_cast<Segment*>(base + kOffSeg);
  if (o < sh.n_segs) {
    const int b0 = o * kMaxBatchesList, b1 = min(n_batches, b0 + kMaxBatchesList);
    // every earlier segment has kMaxBatchesList batches
    segs[o] = Segment{0, b0, b1, sh.n_chunks, (int64_t)sh.n_chunks * b0 * 32};
  }
  WorkItem* items = reinterpret_cast<WorkItem*>(base + kOffItems);
  for (int i = o; i < sh.n_items; i += blockDim.x) {
    const int sg = i / sh.n_chunks, c = i % sh.n_chunks;
    const int b0 = sg * kMaxBatchesList, b1 = min(n_batches, b0 + kMaxBatchesList);
    items[i] = WorkItem{0, sg, c, c * sh.ck, min(sh.n_ksets, (c + 1) * sh.ck), b0, b1, w_hlo[sg], w_hhi[sg],
                        w_tgap[sg], w_d2max[sg], w_d2min[sg], w_sglr[sg]};
  }
  MItem* mitems = reinterpret_cast<MItem*>(base + kOffMItems);
  const int64_t nk = (int64_t)sh.N * sh.N;
  for (int i = o; i < sh.n_mitems; i += blockDim.x) {
    const int hb = i / sh.m_chunks, c = i % sh.m_chunks;
    mitems[i] = MItem{0, hb, c, sh.m_chunks, (int64_t)c * kNAMChunk, min(nk, (int64_t)(c + 1) * kNAMChunk),
                      (int64_t)hb * sh.m_chunks * 32, hb, 0};
  }
}

// Omega = NaN for flagged points, and for every point when a kernel of the
// call reported an internal inconsistency in the status word.
__global__ void na_finish_kernel(int n, const unsigned char* base, double* omega) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  const int32_t status = reinterpret_cast<const int32_t*>(base + kOffCnt)[7];
  if (status != 0 || reinterpret_cast<const int32_t*>(base + kOffBad)[o] != 0) omega[o] = NAN;
}

}  // namespace
}  // namespace ffe

using namespace ffe;

extern "C" ffe_status ffe_omega_noalloc(const ffe_model* m, int32_t N, double qx, double qy, const double* h,
                                        const double* T, const double* delta, int32_t n, double* omega,
                                        void* stream) {
  if (!m || !h || !T || !delta || !omega) return FFE_EINVAL;
  if (m->kind != FFE_MODEL_RAGHU2) return FFE_EUNSUPPORTED;
  if (m->prec != FFE_FP64 && m->prec != FFE_FP32C) return FFE_EINVAL;
  if (!(m->U > 0.0)) return FFE_EINVAL;
  for (int b = 0; b < 3; ++b)
    if (!std::isfinite(m->U_band[b]) || m->U_band[b] < 0.0 || (b == 2 && m->U_band[b] != 0.0)) return FFE_EINVAL;
  if (N < 2 || N > kNAMaxN || (N % 2) != 0) return FFE_EINVAL;  // beyond the static scratch
  if (n < 1 || n > kNAMaxOut) return FFE_EINVAL;                 // beyond the static scratch
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNAMaxDevices) return FFE_ECUDA;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {  // set-up, once per device, with that device current
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_na_scratch) != cudaSuccess || !ptr) return FFE_ECUDA;
    g_na_addr[dev] = ptr;
  }
  unsigned char* base = static_cast<unsigned char*>(g_na_addr[dev]);
  const int prec = m->prec;
  const int kpt = prec == FFE_FP32C ? 4 : 1;
  int n_sm = 0, bps = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FFE_ECUDA;
  if (ksum_occupancy(prec, kLayoutList, kpt, 256, &bps) != cudaSuccess) return FFE_ECUDA;
  if (bps < 1) bps = 1;

  // job table shape: one LIST group, segments of <= kMaxBatchesList batches,
  // each split into the same <= kNAMaxItems / n_segs k-chunks
  NAShape sh;
  std::memset(&sh, 0, sizeof sh);
  sh.N = N;
  sh.n = n;
  sh.prec = prec;
  sh.qx = qx;
  sh.qy = qy;
  const int n_batches = (n + 31) / 32;
  const int64_t nk = (int64_t)N * N;
  const int kset_pts = 32 * kpt;
  sh.n_ksets = (int)((nk + kset_pts - 1) / kset_pts);
  sh.n_segs = (n_batches + kMaxBatchesList - 1) / kMaxBatchesList;
  const int seg_b = std::min(n_batches, kMaxBatchesList);
  const double target = prec == FFE_FP32C ? 8388608.0 : 262144.0;
  int ck = (int)(target / ((double)seg_b * 32.0 * kset_pts));
  ck = std::max(ck, (sh.n_ksets * sh.n_segs + kNAMaxItems - 1) / kNAMaxItems);
  ck = std::max(1, std::min(ck, sh.n_ksets));
  while ((int64_t)((sh.n_ksets + ck - 1) / ck) * sh.n_segs > kNAMaxItems) ++ck;
  sh.ck = ck;
  sh.n_chunks = (sh.n_ksets + ck - 1) / ck;
  sh.n_items = sh.n_chunks * sh.n_segs;
  sh.m_chunks = (int)((nk + kNAMChunk - 1) / kNAMChunk);
  sh.n_mitems = n_batches * sh.m_chunks;
  if (sh.n_mitems > kNAMaxMItems || n_batches > 64) return FFE_EINTERNAL;

  ModelParams mp{m->t1, m->t2, m->t3, m->t4, m->mu, m->U, m->eta_amp, FFE_MODEL_RAGHU2, 2};
  for (int b = 0; b < 2; ++b) {
    mp.Ub[b] = m->U_band[b] > 0.0 ? m->U_band[b] : m->U;
    if (mp.Ub[b] != m->U) mp.per_band_u = 1;
  }
  const GroupDesc* d_group = reinterpret_cast<const GroupDesc*>(base + kOffGroup);
  HT* d_ht = reinterpret_cast<HT*>(base + kOffHT);
  double* d_hlist = reinterpret_cast<double*>(base + kOffHList);
  const double* d_delta = reinterpret_cast<const double*>(base + kOffDelta);
  na_setup_kernel<<<1, kNAMaxOut, 0, s>>>(sh, h, T, delta, base);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = prep_params_launch(d_delta, n, reinterpret_cast<float*>(base + kOffD2F), d_ht, n,
                           reinterpret_cast<HTf*>(base + kOffHTF), reinterpret_cast<HTd*>(base + kOffHTD), s);
  if (e == cudaSuccess)
    e = tables_launch(mp, d_group, 1, N, reinterpret_cast<TabRowF*>(base + kOffTabF),
                      reinterpret_cast<float*>(base + kOffC0F), reinterpret_cast<TabRowD*>(base + kOffTabD),
                      reinterpret_cast<double*>(base + kOffC0D), reinterpret_cast<TabRowDF*>(base + kOffTabDF), s);
  if (e == cudaSuccess)
    e = normal_launch(mp, d_group, reinterpret_cast<const MItem*>(base + kOffMItems), sh.n_mitems, d_hlist,
                      reinterpret_cast<const TabRowD*>(base + kOffTabD),
                      prec == FFE_FP32C ? reinterpret_cast<const TabRowDF*>(base + kOffTabDF) : nullptr,
                      nullptr, reinterpret_cast<double*>(base + kOffMPart),
                      reinterpret_cast<int32_t*>(base + kOffMCnt), reinterpret_cast<double*>(base + kOffM), s);
  if (e != cudaSuccess) return FFE_ECUDA;
  KsumArgs a;
  std::memset(&a, 0, sizeof a);
  a.m = mp;
  a.groups = d_group;
  a.items = reinterpret_cast<const WorkItem*>(base + kOffItems);
  a.n_items = sh.n_items;
  a.segs = reinterpret_cast<const Segment*>(base + kOffSeg);
  a.queue = reinterpret_cast<int32_t*>(base + kOffCnt);
  a.seg_count = reinterpret_cast<int32_t*>(base + kOffSegCnt);
  a.partials = reinterpret_cast<double*>(base + kOffPart);
  a.tabf = reinterpret_cast<const TabRowF*>(base + kOffTabF);
  a.c0f = reinterpret_cast<const float*>(base + kOffC0F);
  a.tabd = reinterpret_cast<const TabRowD*>(base + kOffTabD);
  a.c0d = reinterpret_cast<const double*>(base + kOffC0D);
  a.delta = d_delta;
  a.d2f = reinterpret_cast<const float*>(base + kOffD2F);
  a.ht = d_ht;
  a.htf = reinterpret_cast<const HTf*>(base + kOffHTF);
  a.htd = reinterpret_cast<const HTd*>(base + kOffHTD);
  a.M = reinterpret_cast<const double*>(base + kOffM);
  a.V = reinterpret_cast<double*>(base + kOffV);
  a.omega = omega;
  a.ebound = reinterpret_cast<double*>(base + kOffEB);
  a.eb_rel = 0.0;
  a.eb_abs = 0.0;
  a.status = reinterpret_cast<int32_t*>(base + kOffCnt) + 7;
  a.w_scaled = prec == FFE_FP32C ? 1 : 0;
  e = ksum_launch(prec, kLayoutList, kpt, a, n_sm * bps, 256, s);
  if (e != cudaSuccess) return FFE_ECUDA;
  na_finish_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, base, omega);
  return cudaGetLastError() == cudaSuccess ? FFE_OK : FFE_ECUDA;
}
