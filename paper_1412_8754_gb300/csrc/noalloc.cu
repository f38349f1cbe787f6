// noalloc.cu -- Omega at up to 512 points of one (N, Q) with no allocation.
//
// Some callers cannot allocate device memory at the moment they need a free
// energy: a service that has handed all free device memory to its own pool
// (a cudaMalloc there fails or evicts its cache), or a latency-critical loop
// in which cudaMalloc/cudaFree would synchronise the device and stall the
// other streams.  ffe_omega_noalloc serves them: the caller passes its own
// device arrays for the inputs and the output, and every intermediate (job
// table, trig tables, work queue, partial sums, normal-state sums) lives in
// one file-scope __device__ array of fixed size, written by the call's own
// kernels (direct.cu).  Nothing is allocated, on the device or the host, and
// nothing is copied from the host during a call.
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
#include "direct.cuh"
#include "ffe_internal.cuh"
#include "ksum.cuh"

namespace ffe {
namespace {

constexpr int kNAMaxN = 2048;     // largest lattice
constexpr int kNAMaxOut = 512;    // most points per call
constexpr int kNAMaxItems = 256;  // k-sum work items
constexpr size_t kNAScratchBytes = size_t(4) << 20;  // 4 MiB

static __device__ __align__(256) unsigned char g_na_scratch[kNAScratchBytes];

// Device address of g_na_scratch per device, obtained once with that device current.
constexpr int kNAMaxDevices = 64;
void* g_na_addr[kNAMaxDevices] = {};
std::mutex g_na_mutex;

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
  if (!std::isfinite(qx) || !std::isfinite(qy)) return FFE_EINVAL;
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
  int n_sm = 0, bps = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return FFE_ECUDA;
  if (ksum_occupancy(prec, kLayoutList, prec == FFE_FP32C ? 4 : 1, 256, &bps) != cudaSuccess) return FFE_ECUDA;
  bps = std::max(1, bps);
  const DirectShape sh = direct_shape(N, n, prec, 2, false, qx, qy, kNAMaxItems, (double)n_sm * bps * 8);
  const DirectLayout L = direct_layout(sh);
  if (L.total > kNAScratchBytes || sh.n_items > kNAMaxItems) return FFE_EINTERNAL;
  ModelParams mp;
  std::memset(&mp, 0, sizeof mp);
  mp.t1 = m->t1;
  mp.t2 = m->t2;
  mp.t3 = m->t3;
  mp.t4 = m->t4;
  mp.mu = m->mu;
  mp.U = m->U;
  mp.eta_amp = m->eta_amp;
  mp.kind = FFE_MODEL_RAGHU2;
  mp.nbands = 2;
  for (int b = 0; b < 2; ++b) {
    mp.Ub[b] = m->U_band[b] > 0.0 ? m->U_band[b] : m->U;
    if (mp.Ub[b] != m->U) mp.per_band_u = 1;
  }
  const cudaError_t e =
      direct_enqueue(mp, sh, L, base, h, T, delta, omega, nullptr, n_sm * bps, s);
  return e == cudaSuccess ? FFE_OK : FFE_ECUDA;
}
