// ksum.cuh -- launch interface of the kernels (host side, internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ffe_internal.cuh"

namespace ffe {

struct KsumArgs {
  ModelParams m;
  const GroupDesc* groups;
  const WorkItem* items;
  int32_t n_items;
  int32_t pad0;
  const Segment* segs;
  int32_t* queue;      // work counter, zeroed before each launch
  int32_t* seg_count;  // per-segment completion counters (self-resetting)
  double* partials;
  const TabRowF* tabf;
  const float* c0f;
  const TabRowD* tabd;
  const double* c0d;
  const double* delta;  // Delta values (authoritative, FP64)
  const float* d2f;     // Delta^2 in FP32
  const HT* ht;
  const HTf* htf;
  const HTd* htd;
  const double* M;      // normal-state sums per (group, h)
  double* V;            // per-output sum_k v_k
  double* omega;        // per-output Omega
  double* ebound;       // per-output FP32 error bound (0 for FP64)
  double eb_rel, eb_abs;
  int32_t* status;
  int32_t w_scaled;  // 1: partial sums hold W (FP32 path), V = -T ln2 W; 0: they hold V
  int32_t pad1;
  unsigned long long* near_evals;  // FP32 path: band evaluations with the full term, [1] those with one
                                   // exponential, [2] far ones in the closed form (NULL: not counted)
  const float4* e3f;               // three-band model: band tables (GroupDesc::e3_off), FP32
  const E3D* e3d;                  // and FP64
  // FP32 k-state table (NULL: states are built from the trig tables): per
  // (group, band pair, lattice point) |s| and d0 of both slots, and eta^2
  float4* kst4;
  float* kste;
};

size_t ksum_smem_bytes(int prec, int layout, int kpt, int block_threads);
cudaError_t kstate_table_launch(const KsumArgs& a, int n_groups, int max_n, cudaStream_t s);
cudaError_t ksum_launch(int prec, int layout, int kpt, const KsumArgs& a, int grid, int block,
                        cudaStream_t s);
cudaError_t ksum_occupancy(int prec, int layout, int kpt, int block, int* blocks_per_sm);
bool ksum_kpt_supported(int prec, int kpt);

// ---- tables and the normal-state sum (tables.cu)
// Work item of the M kernel: k range [k0, k1) of one group, h block hb (32 h).
struct MItem {
  int32_t group;
  int32_t hb;
  int32_t chunk;
  int32_t n_chunks;
  int64_t k0, k1;
  int64_t partial_off;  // partials[partial_off + chunk*32 + j]
  int32_t counter;      // index of the (group, hb) completion counter
  int32_t pad;
};

cudaError_t tables_launch(const ModelParams& m, const GroupDesc* groups, int n_groups, int max_n,
                          TabRowF* tabf, float* c0f, TabRowD* tabd, double* c0d, TabRowDF* tabdf,
                          cudaStream_t s);
cudaError_t prep_params_launch(const double* delta, int64_t n_delta, float* d2f, const HT* ht,
                               int64_t n_ht, HTf* htf, HTd* htd, cudaStream_t s);
// tabdf non-NULL: band energies in double-float arithmetic from tabdf (FP32
// plans); NULL: in FP64 from tabd.
cudaError_t normal_launch(const ModelParams& m, const GroupDesc* groups, const MItem* items,
                          int n_items, const double* hlist, const TabRowD* tabd, const TabRowDF* tabdf,
                          const E3D* e3d, double* partials, int32_t* counters, double* M, cudaStream_t s);
// Three-band model: its band tables (GroupDesc::e3_off) from the FP64 trig tables.
cudaError_t bands3_launch(const ModelParams& m, const GroupDesc* groups, int n_groups, int max_n,
                          const TabRowD* tabd, E3D* e3d, float4* e3f, cudaStream_t s);

// ---- search, rescoring and labels (search.cu)
struct Line {          // one Delta search: outputs out0 + i*stride, i < count
  int64_t out0;
  int32_t stride;
  int32_t count;
  int32_t group;
  int32_t pad;
  int64_t delta0;      // Delta entry of i = 0 (entries delta0 + i)
  int64_t ht;          // (h,T) entry
};

struct LineResult {
  double delta_star, omega_star, eb_star;
  double omega_lo, eb_lo;
  double delta_lo;     // the Delta of omega_lo (the lower end of the range)
  int64_t out_star;
  int32_t idx_star;
  int32_t flags;
};

struct Rescore {       // FP64 re-evaluation request
  int32_t group;
  int32_t kind;        // 0: omega/ebound[dst]; 1: line best; 2: line lo
  int64_t dst;
  int64_t ht;
  double delta;
};

// Golden-section search state of one line (one (q, h, T) point).
struct GoldenState {
  double a, b;          // current bracket
  double x1, x2;        // interior points
  double f1, f2;        // Omega at x1, x2
  double eb1, eb2;      // their FP32 error bounds (0 once FP64)
  double xb, fb, ebb;   // lowest Omega seen so far (ties -> smaller Delta)
  double flo, eblo;     // Omega at the reference point x0
  double lo, hi;        // the search range (bracket at the start)
  double x0;            // reference point, evaluated first: the normal state
                        // Delta = 0; equal to lo except for a window bracket
  double wide;          // interior points farther apart than this may lie in
                        // different basins (0: 1 % of hi - lo)
  int32_t side;         // 0: the pending evaluation is x1, 1: x2
  int32_t pad;
};

struct RescoreArgs {
  ModelParams m;
  const GroupDesc* groups;
  const TabRowD* tabd;
  const double* c0d;
  const HT* ht;
  const double* M;
  const Rescore* req;
  const int32_t* n_req;
  int32_t chunk_k;      // k-points per chunk
  int32_t max_chunks;   // chunks per request (covers the largest N^2)
  int32_t* queue;
  int32_t* counters;    // per request (self-resetting)
  double* partials;     // [cap][max_chunks]
  double* omega;
  double* ebound;
  LineResult* lines;
  int32_t* rescored;    // per output flag (kind 0)
  GoldenState* golden;  // kinds 3 (x1) and 4 (x2)
  int32_t cap;
  int32_t n_groups;     // groups of the plan (the requests' group ids are below it)
  const E3D* e3d;       // three-band model: FP64 band tables (GroupDesc::e3_off)
  // grouping of the requests (rescore_sort_kernel): request indices ordered
  // by group [cap], runs of at most kRescoreRun of them within one group
  // (first, count) [cap], and per group its request count, request offset,
  // run offset and a fill counter [4 (n_groups + 1)]; the run count in total
  // is gcount[n_groups]
  int32_t* order;
  int2* runs;
  int32_t* gcount;
};
// Requests of one group evaluated together (one pass over its band energies).
constexpr int kRescoreRun = 6;

enum { kGoldenInit = 0, kGoldenLo, kGoldenX1, kGoldenX2, kGoldenMark, kGoldenDecide, kGoldenRecord,
       kGoldenMarkFinal, kGoldenFinish };
cudaError_t golden_launch(int mode, const Line* lines, int n_lines, GoldenState* gs, const double* omega,
                          const double* ebound, double* delta, float* d2f, Rescore* req, int32_t* n_req,
                          int32_t cap, LineResult* res, cudaStream_t s);

cudaError_t argmin_launch(const Line* lines, int n_lines, const double* omega, const double* ebound,
                          const double* delta, const int32_t* rescored, int mode, Rescore* req,
                          int32_t* n_req, int32_t cap, LineResult* res, cudaStream_t s);
cudaError_t rescore_launch(const RescoreArgs& a, int grid, cudaStream_t s);
cudaError_t rescore_occupancy(int* blocks_per_sm);  // resident rescore blocks (128 threads) per SM
// LineResult -> ffe_result (include/ffe.h) of n lines on the device.
cudaError_t results_launch(const LineResult* lr, int64_t n, const int32_t* counters, int32_t cap, void* out,
                           cudaStream_t s);
cudaError_t labels_launch(LineResult* res, int n_q, int n_pts, const int32_t* q_is_zero,
                          const Line* lines, const double* delta, int mode, Rescore* req,
                          int32_t* n_req, int32_t cap, int8_t* labels, int32_t* best_q,
                          cudaStream_t s);

}  // namespace ffe
