// direct.cuh -- Omega at the points of one (N, Q) read from device arrays, with
// the job table written on the device (internal; used by ffe_omega_async and
// ffe_omega_noalloc).
//
// The points become one LIST group (or one per band, band_only = b + 1, when
// the per-band values are wanted), every group sharing the trig tables and
// (three-band model) band tables of group 0.  Every point is its own (h, T)
// entry of its group.  A setup sequence of three small kernels validates the
// points, writes the job table (groups, segments, work items with the far
// windows of their outputs, normal-state items) and clears the counters; the
// usual kernels follow (parameter forms, tables, normal-state sums, k-sum), and
// a finish kernel writes the results: NaN for an invalid point (T <= 0 or a
// non-finite h, T or Delta, computed as (0, 1, 0) meanwhile) and for every
// point when a kernel reported an inconsistency in the status word.
#pragma once

#include <cstddef>
#include <cstdint>

#include "ksum.cuh"

namespace ffe {

struct DirectShape {
  int32_t N, n, prec, nbands;
  int32_t n_grp;       // 1: Omega over all bands; nbands: one group per band
  int32_t kpt;         // k-points per thread of the k-sum
  int32_t n_segs;      // segments per group (<= kMaxBatchesList batches each)
  int32_t n_ksets, ck, n_chunks;
  int32_t n_items;     // k-sum work items, all groups
  int32_t m_chunks;    // normal-state k-chunks per (group, block of 32 points)
  int32_t n_mitems;    // normal-state items, all groups
  int32_t pad;
  double qx, qy;
};

// Byte offsets of the regions inside one scratch block (each 256-aligned).
struct DirectLayout {
  size_t tabf, c0f, tabd, c0d, tabdf, e3d, e3f;
  size_t group, seg, items, mitems, win;
  size_t d2f, ht, htf, htd, hlist, delta, bad;
  size_t M, mpart, mcnt, part, V, eb, omega, cnt, segcnt;
  size_t total;
};

constexpr int64_t kDirectMChunk = 32768;  // k-points per normal-state work item

// The job table's shape for n points of one (N, Q); max_items caps the k-sum's
// work items (the k-chunks grow to fit); n_warps > 0, the resident warps of
// the k-sum's grid: items small enough for about four per warp.
DirectShape direct_shape(int N, int n, int prec, int nbands, bool per_band, double qx, double qy, int max_items,
                         double n_warps);
DirectLayout direct_layout(const DirectShape& sh);
// Enqueues the whole computation on s.  omega[n] receives Omega (all bands);
// omega_band (NULL or [n][nbands], needs sh.n_grp == nbands) each band's.
cudaError_t direct_enqueue(const ModelParams& mp, const DirectShape& sh, const DirectLayout& L, unsigned char* base,
                           const double* h, const double* T, const double* delta, double* omega, double* omega_band,
                           int ksum_grid, cudaStream_t s);

}  // namespace ffe
