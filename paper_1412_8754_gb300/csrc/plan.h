// plan.h -- host-side structures behind the opaque handles of include/ffe.h.
#pragma once

#include <map>
#include <string>
#include <vector>

#include "../../include/ffe.h"
#include "ksum.cuh"

namespace ffe {

constexpr int kRing = 256;                          // timing event pairs per plan
constexpr double kEbRel = 7.62939453125e-06;        // 2^-17: FP32 bound, relative to |sum_k v_k|
constexpr double kEbAbs = 1.6527e-07;               // 2^-22 ln 2: log2 error per k-point, times T
// The FP32 k-state table of a plan (20 bytes per group, band pair and lattice
// point) is kept when it fits in this many bytes (the environment variable
// FFE_KSTATE_TABLE_MAX_BYTES, read when a plan is allocated, overrides it);
// larger plans build the states inside the k-sum instead.
constexpr int64_t kKstateTableMaxBytes = int64_t(32) << 30;
// The largest freed plan block a context keeps for reuse.
constexpr size_t kSpareMaxBytes = size_t(16) << 30;

enum { kPlanScanGrid = 1, kPlanMinGrid = 2, kPlanOmega = 3, kPlanScanGolden = 4, kPlanMinGolden = 5 };

struct Tuning {
  int kpt;
  int block;
  double item_target;  // k-point evaluations per warp work item
};

}  // namespace ffe

struct ffe_context {
  ffe_model model;
  ffe::ModelParams mp;
  int device = 0;
  int n_sm = 0;
  std::string device_name;
  std::string err;
  std::vector<ffe_plan*> plans;               // user plans (ffe_plan_*)
  std::map<std::string, ffe_plan*> cache;     // plans reused by the host-buffer calls
  std::map<std::string, ffe::Tuning> tuned;   // autotuner results
  std::string tune_path;
  // the device block of the last plan freed (at most kSpareMaxBytes), reused
  // by the next plan that fits in it: short-lived plans (the surrogate-guided
  // passes, the autotuner's trials) then skip cudaMalloc and cudaFree
  void* spare = nullptr;
  size_t spare_bytes = 0;
  // scratch of the stream-ordered point evaluation (ffe_omega_async), grown
  // to the largest call
  void* direct = nullptr;
  size_t direct_bytes = 0;
};

struct ffe_plan {
  ffe_context* ctx = nullptr;
  int kind = 0;
  int prec = 0;
  int layout = 0;
  // host tables
  std::vector<ffe::GroupDesc> groups;
  std::vector<ffe::WorkItem> items;
  std::vector<ffe::Segment> segs;
  std::vector<int64_t> item_sig;  // the shapes items/segs were built for (item_signature)
  std::vector<ffe::MItem> mitems;
  std::vector<ffe::Line> lines;
  std::vector<double> delta;
  std::vector<ffe::HT> ht;
  std::vector<double> hlist;
  std::vector<int32_t> q_is_zero;
  std::vector<int64_t> order;  // input index of each output (point plans)
  int64_t n_out = 0;
  int64_t n_partials = 0;
  int64_t n_mpartials = 0;
  int n_mcounters = 0;
  int64_t tab_rows = 0;
  int n_q = 0, n_pts = 0, max_n = 2;
  // golden-section state sizes
  int golden_steps = 0;
  // launch configuration
  int kpt = 4, block = 256, grid = 0, rescore_grid = 0;
  int variant = 0;  // k-sum kernel variant (kLayoutProduct / kLayoutProductUT / kLayoutList)
  bool forced = false;  // use `tuning` instead of the context's choice
  ffe::Tuning tuning{4, 256, 8388608.0};
  double item_target = 8388608.0;
  int rescore_chunk = 16384, rescore_chunks = 1;
  int32_t cap = 0;
  double k_evals = 0.0;
  int launches = 0;
  size_t bytes = 0;
  size_t h2d_bytes = 0, d2h_bytes = 0;
  // device buffers: one block (`arena`, arena_bytes) holds them all
  void* arena = nullptr;
  size_t arena_bytes = 0;
  ffe::GroupDesc* d_groups = nullptr;
  ffe::WorkItem* d_items = nullptr;
  ffe::Segment* d_segs = nullptr;
  ffe::MItem* d_mitems = nullptr;
  ffe::Line* d_lines = nullptr;
  double* d_delta = nullptr;
  float* d_d2f = nullptr;
  ffe::HT* d_ht = nullptr;
  ffe::HTf* d_htf = nullptr;
  ffe::HTd* d_htd = nullptr;
  double* d_hlist = nullptr;
  int32_t* d_qzero = nullptr;
  ffe::TabRowF* d_tabf = nullptr;
  float* d_c0f = nullptr;
  ffe::TabRowD* d_tabd = nullptr;
  ffe::TabRowDF* d_tabdf = nullptr;  // double-float copy (normal-state sums of FP32 plans)
  ffe::E3D* d_e3d = nullptr;          // three-band model: band tables, FP64
  float4* d_e3f = nullptr;            // and FP32
  float4* d_kst4 = nullptr;           // FP32 k-state table (|s|, d0 of both slots) and eta^2;
  float* d_kste = nullptr;            // none when kst_rows == 0
  int64_t kst_rows = 0;
  int64_t e3_rows = 0;                // rows of the three-band band tables
  double* d_c0d = nullptr;
  double* d_M = nullptr;
  double* d_Mpart = nullptr;
  int32_t* d_Mcnt = nullptr;
  double* d_partials = nullptr;
  int32_t* d_segcnt = nullptr;
  int32_t* d_counters = nullptr;
  unsigned long long* d_near = nullptr;  // full-term k-evaluations of the last execution (FP32)
  double* d_V = nullptr;
  double* d_omega = nullptr;
  double* d_eb = nullptr;
  int32_t* d_rescored = nullptr;
  ffe::Rescore* d_req = nullptr;
  double* d_rpart = nullptr;
  int32_t* d_rcnt = nullptr;
  int32_t* d_rorder = nullptr;  // requests sorted by (group, dst) [cap]
  int2* d_rruns = nullptr;      // runs of requests of one group [cap]
  int32_t* d_rgcount = nullptr; // per-group request counts, offsets, run offsets, fill [4 (n_groups + 1)]
  ffe::LineResult* d_lres = nullptr;
  int8_t* d_labels = nullptr;
  int32_t* d_bestq = nullptr;
  ffe::GoldenState* d_golden = nullptr;   // golden-section state per line (golden.cu)
  std::vector<ffe::GoldenState> golden0;  // its initial value (search range per line)
  // execution
  cudaStream_t stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t node_ev0 = nullptr, node_ev1 = nullptr;
  cudaEvent_t ev_cap0 = nullptr, ev_cap1 = nullptr;
  cudaEvent_t ring0[ffe::kRing] = {};
  cudaEvent_t ring1[ffe::kRing] = {};
  int64_t exec_count = 0;
  int64_t timed_upto = 0;
  int32_t last_rescored[2] = {0, 0};  // FP64 requests of the last fetched execution
  // page-locked staging of a refill's uploads (stream-ordered calls) and the
  // event after its copies
  void* staging = nullptr;
  size_t staging_bytes = 0;
  cudaEvent_t staged_ev = nullptr;
};

namespace ffe {

struct HostCopy {
  void* dst;
  const void* src;
  size_t bytes;
};

void set_err(ffe_context* c, const char* fmt, ...);
ffe_status cuda_fail(ffe_context* c, cudaError_t e, const char* what);
void linspace(double lo, double hi, int n, double* out);

ffe_plan* plan_new(ffe_context* ctx, int kind);
void plan_free(ffe_plan* p);
ffe_status plan_configure(ffe_context* ctx, ffe_plan* p);
ffe_status plan_finish(ffe_context* ctx, ffe_plan* p, bool use_graph);
ffe_status plan_upload_params(ffe_context* ctx, ffe_plan* p, cudaStream_t s);
ffe_status plan_refill(ffe_context* ctx, ffe_plan* p, cudaStream_t s, bool pinned);
void fill_scan(ffe_plan* p, const ffe_scan* sc);
ffe_status check_scan(ffe_context* ctx, const ffe_scan* sc);
ffe_status plan_run(ffe_context* ctx, ffe_plan* p, cudaStream_t s);
ffe_status plan_check_status(ffe_context* ctx, ffe_plan* p, cudaStream_t s);
double plan_k_evals(const ffe_plan* p);
void build_items(ffe_plan* p);
void build_mitems(ffe_plan* p);
bool batches_share_T(const ffe_plan* p);
void apply_tiles(ffe_plan* p, bool shared_t);
ffe_status fetch_scan(ffe_context* ctx, ffe_plan* p, ffe_result* per_point, int8_t* labels, int32_t* best_q,
                      cudaStream_t s);
// MLP inference on device arrays (mlp.cu): y[n] (network units) at raw x[n][4].
ffe_status surrogate_infer_device(ffe_surrogate* s, const float* x, int64_t n, float* y, cudaStream_t st);
float surrogate_y_scale(const ffe_surrogate* s);

Tuning tuning_for(ffe_context* ctx, const ffe_plan* p);
void tuning_load(ffe_context* ctx);

}  // namespace ffe
