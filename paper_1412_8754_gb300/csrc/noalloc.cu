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
constexpr size_t kNAUsed = align256(kOffSegCnt + kNAMaxSegs * sizeof(int32_t));
static_assert(kNAUsed <= kNAScratchBytes, "scratch regions exceed the static array");

// Device address of g_na_scratch per device, obtained once with that device current.
constexpr int kNAMaxDevices = 64;
void* g_na_addr[kNAMaxDevices] = {};
std::mutex g_na_mutex;

// Host staging of the job table (static storage: no heap use per call).
GroupDesc g_na_group;
Segment g_na_segs[kNAMaxSegs];
WorkItem g_na_items[kNAMaxItems];
MItem g_na_mitems[kNAMaxMItems];

__global__ void na_pack_kernel(const double* __restrict__ h, const double* __restrict__ T, int n, HT* ht,
                               double* hlist) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  ht[o] = HT{h[o], T[o], o, 0};
  hlist[o] = h[o];
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

  // job table: one LIST group, one segment of all batches, <= 256 k-chunks
  GroupDesc& g = g_na_group;
  std::memset(&g, 0, sizeof g);
  g.N = N;
  g.layout = kLayoutList;
  g.n_out = n;
  g.n_delta = n;
  g.n_ht = n;
  g.n_hblk = 1;
  g.n_batches = (n + 31) / 32;
  g.n_h = n;
  g.qx = qx;
  g.qy = qy;
  const int64_t nk = (int64_t)N * N;
  const int kset_pts = 32 * kpt;
  const int n_ksets = (int)((nk + kset_pts - 1) / kset_pts);
  // segments of <= kMaxBatchesList batches, each split into the same k-chunks
  const int n_segs = (g.n_batches + kMaxBatchesList - 1) / kMaxBatchesList;
  const int seg_b = std::min(g.n_batches, kMaxBatchesList);
  const double target = prec == FFE_FP32C ? 8388608.0 : 262144.0;
  int ck = (int)(target / ((double)seg_b * 32.0 * kset_pts));
  ck = std::max(ck, (n_ksets * n_segs + kNAMaxItems - 1) / kNAMaxItems);
  ck = std::max(1, std::min(ck, n_ksets));
  while ((int64_t)((n_ksets + ck - 1) / ck) * n_segs > kNAMaxItems) ++ck;
  const int n_chunks = (n_ksets + ck - 1) / ck;
  int n_items = 0;
  int64_t poff = 0;
  for (int sg = 0; sg < n_segs; ++sg) {
    const int b0 = sg * kMaxBatchesList, b1 = std::min(g.n_batches, b0 + kMaxBatchesList);
    g_na_segs[sg] = Segment{0, b0, b1, n_chunks, poff};
    poff += (int64_t)n_chunks * (b1 - b0) * 32;
    for (int c = 0; c < n_chunks; ++c)
      g_na_items[n_items++] = WorkItem{0, sg, c, c * ck, std::min(n_ksets, (c + 1) * ck), b0, b1, 0.0f, 0.0f,
                                       INFINITY, INFINITY, 0.0f, INFINITY};
  }
  const int64_t mchunk = 32768;
  const int m_chunks = (int)((nk + mchunk - 1) / mchunk);
  const int n_hb = (n + 31) / 32;
  int n_mitems = 0;
  for (int hb = 0; hb < n_hb; ++hb)
    for (int c = 0; c < m_chunks; ++c)
      g_na_mitems[n_mitems++] =
          MItem{0, hb, c, m_chunks, (int64_t)c * mchunk, std::min(nk, (int64_t)(c + 1) * mchunk),
                (int64_t)hb * m_chunks * 32, hb, 0};

  // clear what must start at zero; stage the job table
  cudaError_t e = cudaMemsetAsync(base + kOffCnt, 0, 8 * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffSegCnt, 0, n_segs * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffMCnt, 0, 64 * sizeof(int32_t), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + kOffGroup, &g, sizeof g, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + kOffSeg, g_na_segs, n_segs * sizeof(Segment), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + kOffItems, g_na_items, n_items * sizeof(WorkItem), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + kOffMItems, g_na_mitems, n_mitems * sizeof(MItem), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return FFE_ECUDA;

  const ModelParams mp{m->t1, m->t2, m->t3, m->t4, m->mu, m->U, m->eta_amp, FFE_MODEL_RAGHU2, 2};
  const GroupDesc* d_group = reinterpret_cast<const GroupDesc*>(base + kOffGroup);
  HT* d_ht = reinterpret_cast<HT*>(base + kOffHT);
  double* d_hlist = reinterpret_cast<double*>(base + kOffHList);
  na_pack_kernel<<<(n + 127) / 128, 128, 0, s>>>(h, T, n, d_ht, d_hlist);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = prep_params_launch(delta, n, reinterpret_cast<float*>(base + kOffD2F), d_ht, n,
                           reinterpret_cast<HTf*>(base + kOffHTF), reinterpret_cast<HTd*>(base + kOffHTD), s);
  if (e == cudaSuccess)
    e = tables_launch(mp, d_group, 1, N, reinterpret_cast<TabRowF*>(base + kOffTabF),
                      reinterpret_cast<float*>(base + kOffC0F), reinterpret_cast<TabRowD*>(base + kOffTabD),
                      reinterpret_cast<double*>(base + kOffC0D), reinterpret_cast<TabRowDF*>(base + kOffTabDF), s);
  if (e == cudaSuccess)
    e = normal_launch(mp, d_group, reinterpret_cast<const MItem*>(base + kOffMItems), n_mitems, d_hlist,
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
  a.n_items = n_items;
  a.segs = reinterpret_cast<const Segment*>(base + kOffSeg);
  a.queue = reinterpret_cast<int32_t*>(base + kOffCnt);
  a.seg_count = reinterpret_cast<int32_t*>(base + kOffSegCnt);
  a.partials = reinterpret_cast<double*>(base + kOffPart);
  a.tabf = reinterpret_cast<const TabRowF*>(base + kOffTabF);
  a.c0f = reinterpret_cast<const float*>(base + kOffC0F);
  a.tabd = reinterpret_cast<const TabRowD*>(base + kOffTabD);
  a.c0d = reinterpret_cast<const double*>(base + kOffC0D);
  a.delta = delta;
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
  return e == cudaSuccess ? FFE_OK : FFE_ECUDA;
}
