// api.cu -- the C ABI of include/ffe.h: argument checking, packing of job
// tables, device buffers, the launch sequence of one scan, its CUDA graph and
// the timing ring.  Every arithmetic step of the method runs in the kernels
// of ksum.cu / tables.cu / search.cu; this file only plans and launches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/ffe.h"
#include "ffe_internal.cuh"
#include "ksum.cuh"
#include "plan.h"

using namespace ffe;

// ------------------------------------------------------------------ helpers
namespace ffe {

void set_err(ffe_context* c, const char* fmt, ...) {
  if (!c) return;
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  c->err = buf;
}

ffe_status cuda_fail(ffe_context* c, cudaError_t e, const char* what) {
  set_err(c, "%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? FFE_ENOMEM : FFE_ECUDA;
}

#define FFE_CU(call, what)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

// A plan's buffers are carved from one device allocation: plan_alloc runs its
// list of requests twice, first to add up the sizes (arena == nullptr), then
// to hand out 256-byte aligned pieces of the arena.
struct Arena {
  unsigned char* base = nullptr;
  size_t off = 0;
};

template <typename T>
static ffe_status dev_alloc(ffe_context*, ffe_plan* p, Arena& a, T** ptr, size_t count) {
  if (count == 0) count = 1;
  const size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
  *ptr = a.base ? reinterpret_cast<T*>(a.base + a.off) : nullptr;
  a.off += bytes;
  if (a.base) p->bytes += count * sizeof(T);
  return FFE_OK;
}

template <typename T>
static ffe_status upload(ffe_context* ctx, T* dst, const std::vector<T>& src, cudaStream_t s) {
  if (src.empty()) return FFE_OK;
  FFE_CU(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s), "upload");
  return FFE_OK;
}

// numpy.linspace(lo, hi, n): i*step + lo, last point exactly hi.
void linspace(double lo, double hi, int n, double* out) {
  if (n == 1) {
    out[0] = lo;
    return;
  }
  const double step = (hi - lo) / (double)(n - 1);
  for (int i = 0; i < n; ++i) out[i] = (double)i * step + lo;
  out[n - 1] = hi;
}

static bool valid_N(int32_t N) { return N >= 2 && N <= 8192 && (N % 2) == 0; }
static bool finite(double x) { return std::isfinite(x); }

}  // namespace ffe

// ------------------------------------------------------------- planning
namespace ffe {

// Split every group's (batches x k-sets) into warp work items of roughly
// `target` k-point evaluations, segments of <= max_batches(layout) batches.
// FP32 path: a band is "far" for an item when, with h in [hlo, hhi] and
// T <= Tmax over the item's outputs,
// |s| - max(|d0 - hlo|, |d0 - hhi|) >= tgap = 27 ln2 Tmax (+1e-5 against FP32
// rounding): then every output has c |R -+ d| >= 27, each factor
// (1 + 2^-c|R-+d|) leaves the FP32 product unchanged (P + P e with P e below
// half an ulp of P: the same bits as the full term), and its clamp term is c a.
// FP64 path: tgap = kExpNegligible Tmax, so that every exp(-|R -+ d|/T) of
// the band has an argument of at least kExpNegligible, is taken as 0 (as in
// band_term_f64) and the band's term is the clamp term -a alone.
static void item_far_window(const ffe_plan* p, const GroupDesc& g, int b0, int b1, double golden_d2, WorkItem& w) {
  w.far_hlo = 0.0f;
  w.far_hhi = 0.0f;
  w.far_tgap = INFINITY;
  w.far_d2max = INFINITY;
  w.sgl_d2min = 0.0f;
  w.sgl_r = INFINITY;
  const bool f32 = p->prec == FFE_FP32C;
  // the item's Delta entries [d0, d1) and (h, T) entries [e0, e1): PRODUCT
  // items are consecutive batches of one h-block (tile_pos), LIST items their
  // outputs
  int64_t d0, d1, e0, e1;
  if (g.layout == kLayoutProduct) {
    const int hb = tile_hb(g), db = tile_db(g), nd = tile_n_dblk(g);
    const int hblk = b0 / nd, dblk0 = b0 - hblk * nd;
    d0 = (int64_t)dblk0 * db;
    d1 = std::min<int64_t>(g.n_delta, (int64_t)(dblk0 + (b1 - b0)) * db);
    e0 = (int64_t)hblk * hb;
    e1 = std::min<int64_t>(g.n_ht, e0 + hb);
  } else {
    d0 = e0 = (int64_t)b0 * 32;
    d1 = e1 = std::min<int64_t>(g.n_out, (int64_t)b1 * 32);
  }
  if (f32 && p->golden_steps == 0) {  // the smallest Delta^2 of the item's outputs (golden: 0)
    double d2 = INFINITY;
    for (int64_t i = d0; i < d1; ++i) d2 = std::min(d2, p->delta[g.delta_off + i] * p->delta[g.delta_off + i]);
    if (d2 < INFINITY) w.sgl_d2min = std::nextafter((float)d2, 0.0f);
  }
  {  // the largest Delta^2 of the item's outputs (far series, blocked bands)
    double d2 = 0.0;
    if (p->golden_steps > 0)  // golden brackets stay inside each line's [lo, hi]
      d2 = golden_d2;
    else
      for (int64_t i = d0; i < d1; ++i) d2 = std::max(d2, p->delta[g.delta_off + i] * p->delta[g.delta_off + i]);
    w.far_d2max = std::nextafter((float)d2, INFINITY);
  }
  double hlo = INFINITY, hhi = -INFINITY, tmax = 0.0;
  for (int64_t e = e0; e < e1; ++e) {
    const HT& x = p->ht[g.ht_off + e];
    hlo = std::min(hlo, x.h);
    hhi = std::max(hhi, x.h);
    tmax = std::max(tmax, x.T);
  }
  if (!(hlo <= hhi)) return;
  // float bounds that contain the FP64 ones
  w.far_hlo = std::nextafter((float)hlo, -INFINITY);
  w.far_hhi = std::nextafter((float)hhi, INFINITY);
  if (!f32) {
    w.far_tgap = std::nextafter((float)(kExpNegligible * tmax), INFINITY);
    return;
  }
  w.far_tgap = std::nextafter((float)(27.0 * 0.69314718055994530942 * tmax + 1e-5), INFINITY);
  w.sgl_r = std::nextafter((float)(27.0 * 0.69314718055994530942 * tmax + 1e-5), INFINITY);
}

// Golden plans: the largest Delta^2 any bracket can reach (brackets stay in
// [lo, hi]; x0 may lie outside); 0 for grid plans.
static double golden_reach(const ffe_plan* p) {
  double d2 = 0.0;
  for (const GoldenState& gs : p->golden0) d2 = std::max({d2, gs.lo * gs.lo, gs.hi * gs.hi, gs.x0 * gs.x0});
  return d2;
}

// What the structure of the work items depends on: the launch shape and, per
// group, its lattice, layout, output counts and tiles -- not the parameter
// values, which enter only through each segment's windows.
static std::vector<int64_t> item_signature(const ffe_plan* p) {
  std::vector<int64_t> s = {p->prec, p->kpt, p->grid, p->block, (int64_t)std::llround(p->item_target),
                            (int64_t)p->groups.size()};
  for (const GroupDesc& g : p->groups)
    s.insert(s.end(), {g.N, g.layout, g.n_delta, g.n_ht, g.n_hblk, g.n_batches, g.hb, g.n_out});
  return s;
}

// The far and single-band windows of every segment from the plan's current
// parameter values, written into the segment's items (their structure stays):
// the same windows build_items gives.
static void refresh_item_windows(ffe_plan* p) {
  const double golden_d2 = golden_reach(p);
  std::vector<WorkItem> win(p->segs.size());
  for (size_t i = 0; i < p->segs.size(); ++i) {
    const Segment& sg = p->segs[i];
    item_far_window(p, p->groups[sg.group], sg.b0, sg.b1, golden_d2, win[i]);
  }
  for (WorkItem& w : p->items) {
    const WorkItem& x = win[w.seg];
    w.far_hlo = x.far_hlo;
    w.far_hhi = x.far_hhi;
    w.far_tgap = x.far_tgap;
    w.far_d2max = x.far_d2max;
    w.sgl_d2min = x.sgl_d2min;
    w.sgl_r = x.sgl_r;
  }
}

void build_items(ffe_plan* p) {
  p->items.clear();
  p->segs.clear();
  const int kset_pts = 32 * p->kpt;
  const double golden_d2 = golden_reach(p);
  // A small plan gets smaller items, so that the persistent grid's warps all
  // find work: at least about four items per resident warp.
  double work = 0.0;
  for (const GroupDesc& g : p->groups) {
    const int64_t nk = (int64_t)g.N * g.N;
    work += (double)g.n_batches * 32.0 * (double)((nk + kset_pts - 1) / kset_pts) * kset_pts;
  }
  const double n_warps = std::max(1.0, (double)p->grid * (double)(p->block / 32));
  const double target = std::max((double)kset_pts * 32.0, std::min(p->item_target, work / (4.0 * n_warps)));
  int64_t poff = 0;
  for (int gi = 0; gi < (int)p->groups.size(); ++gi) {
    const GroupDesc& g = p->groups[gi];
    const int64_t nk = (int64_t)g.N * g.N;
    const int n_ksets = (int)((nk + kset_pts - 1) / kset_pts);
    // segments: LIST, <= kMaxBatchesList batches; PRODUCT, consecutive batches of one h-block
    // spanning at most kMaxTileDeltas Delta values (FP32: the warp's far sums per Delta)
    const bool prod = g.layout == kLayoutProduct;
    const bool f32 = p->prec == FFE_FP32C;
    const int sb = prod ? std::min(max_batches(g.layout, f32), (f32 ? kMaxTileDeltas : 32) / tile_db(g))
                        : max_batches(g.layout, f32);
    const int run = prod ? tile_n_dblk(g) : std::max(1, g.n_batches);  // batches per h-block
    // one k-chunk length for all segments of the group (sized for the widest), so that
    // chunk c of every segment reads the same k-states
    int ck = (int)std::max(1.0, std::floor(target / ((double)std::min(sb, g.n_batches) * 32.0 * kset_pts)));
    ck = std::min(ck, n_ksets);
    const int n_chunks = (n_ksets + ck - 1) / ck;
    const size_t first_item = p->items.size();
    for (int b0 = 0; b0 < g.n_batches;) {
      const int b1 = std::min(b0 - b0 % run + run, b0 + sb);
      const int nb = b1 - b0;
      Segment sg;
      sg.group = gi;
      sg.b0 = b0;
      sg.b1 = b1;
      sg.n_chunks = n_chunks;
      sg.partial_off = poff;
      const int seg_id = (int)p->segs.size();
      p->segs.push_back(sg);
      WorkItem proto;
      std::memset(&proto, 0, sizeof proto);
      item_far_window(p, g, b0, b1, golden_d2, proto);
      poff += (int64_t)n_chunks * nb * 32;
      for (int c = 0; c < n_chunks; ++c) {
        WorkItem w;
        w.group = gi;
        w.seg = seg_id;
        w.chunk = c;
        w.kset0 = c * ck;
        w.kset1 = std::min(n_ksets, (c + 1) * ck);
        w.b0 = b0;
        w.b1 = b1;
        w.far_hlo = proto.far_hlo;
        w.far_hhi = proto.far_hhi;
        w.far_tgap = proto.far_tgap;
        w.far_d2max = proto.far_d2max;
        w.sgl_d2min = proto.sgl_d2min;
        w.sgl_r = proto.sgl_r;
        p->items.push_back(w);
      }
      b0 = b1;
    }
    // chunk-major within the group: the segments of one k-chunk run side by side and share
    // the chunk's k-states in L2
    std::stable_sort(p->items.begin() + first_item, p->items.end(),
                     [](const WorkItem& a, const WorkItem& b) { return a.chunk < b.chunk; });
  }
  p->n_partials = poff;
  // longest first: the queue hands out big items early, small ones fill the tail; items
  // of one size keep their group and chunk order
  auto cost = [](const WorkItem& w) { return (double)(w.kset1 - w.kset0) * (w.b1 - w.b0); };
  std::stable_sort(p->items.begin(), p->items.end(),
                   [&](const WorkItem& a, const WorkItem& b) { return cost(a) > cost(b); });
  p->item_sig = item_signature(p);
}

void build_mitems(ffe_plan* p) {
  p->mitems.clear();
  const int64_t chunk = 32768;
  int64_t poff = 0;
  int counter = 0;
  for (int gi = 0; gi < (int)p->groups.size(); ++gi) {
    const GroupDesc& g = p->groups[gi];
    const int64_t nk = (int64_t)g.N * g.N;
    const int n_chunks = (int)((nk + chunk - 1) / chunk);
    for (int hb = 0; hb * 32 < g.n_h; ++hb) {
      for (int c = 0; c < n_chunks; ++c) {
        MItem m;
        m.group = gi;
        m.hb = hb;
        m.chunk = c;
        m.n_chunks = n_chunks;
        m.k0 = (int64_t)c * chunk;
        m.k1 = std::min(nk, m.k0 + chunk);
        m.partial_off = poff;
        m.counter = counter;
        m.pad = 0;
        p->mitems.push_back(m);
      }
      poff += (int64_t)n_chunks * 32;
      ++counter;
    }
  }
  p->n_mpartials = poff;
  p->n_mcounters = counter;
}

// The tile width of a PRODUCT group under the shared-T kernel: 8 (h,T)
// entries x 4 Delta rows per batch -- a work item then spans the h range of 8
// entries, so fewer bands are near for some output of it -- or, for a short
// (h,T) list, the smallest power of two that holds it.
static int tile_width(const GroupDesc& g) {
  int hb = 8;
  while (hb > 1 && hb / 2 >= g.n_ht) hb /= 2;
  return hb;
}

// True when every tile's (h,T) entries of every PRODUCT group share one T.
bool batches_share_T(const ffe_plan* p) {
  for (const GroupDesc& g : p->groups) {
    if (g.layout != kLayoutProduct) return false;
    const int hb = tile_width(g);
    for (int j0 = 0; j0 < g.n_ht; j0 += hb) {
      const int j1 = std::min(g.n_ht, j0 + hb);
      for (int j = j0 + 1; j < j1; ++j)
        if (p->ht[g.ht_off + j].T != p->ht[g.ht_off + j0].T) return false;
    }
  }
  return true;
}

// PRODUCT batch shapes: tiles (tile_width entries x 32 / tile_width Delta rows)
// for the shared-T kernel, else 32 entries of one Delta.
void apply_tiles(ffe_plan* p, bool shared_t) {
  for (GroupDesc& g : p->groups) {
    if (g.layout != kLayoutProduct) continue;
    g.hb = shared_t ? tile_width(g) : 32;
    g.n_hblk = (g.n_ht + g.hb - 1) / g.hb;
    g.n_batches = g.n_hblk * tile_n_dblk(g);
  }
}

double plan_k_evals(const ffe_plan* p) {
  double s = 0.0;
  for (const GroupDesc& g : p->groups) s += (double)g.N * (double)g.N * (double)g.n_out;
  // a golden-section execution evaluates every line 3 + steps times
  return p->golden_steps > 0 ? s * (3.0 + p->golden_steps) : s;
}

// Each group's first row in the three-band band tables and in the k-state
// table (set again whenever the groups are refilled); the row totals.
static void table_offsets(const ffe_context* ctx, ffe_plan* p, int64_t& e3_rows, int64_t& kst_rows) {
  e3_rows = 0;
  kst_rows = 0;
  const int64_t npairs = (ctx->mp.nbands + 1) / 2;
  for (GroupDesc& g : p->groups) {
    const int64_t nk = (int64_t)g.N * g.N;
    g.e3_off = e3_rows;
    if (ctx->mp.nbands == 3) e3_rows += 2 * nk;
    g.kst_off = kst_rows;
    kst_rows += npairs * nk;
  }
}

// The buffers of a plan (sizes from the host tables already in *p).
static ffe_status plan_alloc_requests(ffe_context* ctx, ffe_plan* p, Arena& arena) {
  ffe_status st;
#define ALLOC(ptr, n)                               \
  if ((st = dev_alloc(ctx, p, arena, &p->ptr, (n))) != FFE_OK) return st;
  int64_t tab_rows = 0, hcount = 0;
  for (const GroupDesc& g : p->groups) {
    tab_rows = std::max<int64_t>(tab_rows, g.tab_off + 2 * (int64_t)g.N);
    hcount = std::max<int64_t>(hcount, g.h_off + g.n_h);
  }
  p->tab_rows = tab_rows;
  ALLOC(d_groups, p->groups.size());
  ALLOC(d_items, p->items.size());
  ALLOC(d_segs, p->segs.size());
  ALLOC(d_mitems, p->mitems.size());
  ALLOC(d_lines, p->lines.size());
  ALLOC(d_delta, p->delta.size());
  ALLOC(d_d2f, p->delta.size());
  ALLOC(d_ht, p->ht.size());
  ALLOC(d_htf, p->ht.size());
  ALLOC(d_htd, p->ht.size());
  ALLOC(d_hlist, p->hlist.size());
  ALLOC(d_qzero, p->q_is_zero.size());
  ALLOC(d_tabf, tab_rows);
  ALLOC(d_c0f, tab_rows);
  ALLOC(d_tabd, tab_rows);
  ALLOC(d_tabdf, tab_rows);
  ALLOC(d_c0d, tab_rows);
  ALLOC(d_M, hcount);
  ALLOC(d_Mpart, p->n_mpartials);
  ALLOC(d_Mcnt, p->n_mcounters);
  ALLOC(d_partials, p->n_partials);
  ALLOC(d_segcnt, p->segs.size());
  ALLOC(d_counters, 8);
  ALLOC(d_near, 3);
  ALLOC(d_V, p->n_out);
  ALLOC(d_omega, p->n_out);
  ALLOC(d_eb, p->n_out);
  ALLOC(d_rescored, p->n_out);
  p->cap = (int32_t)std::min<int64_t>(p->n_out + 2 * (int64_t)p->lines.size() + 64, 1 << 16);
  ALLOC(d_req, p->cap);
  int max_n = 2;
  for (const GroupDesc& g : p->groups) max_n = std::max(max_n, g.N);
  p->max_n = max_n;
  // at most 64 chunks per FP64 request: bounded partial storage for any N
  const int64_t nk_max = (int64_t)max_n * max_n;
  p->rescore_chunk = (int)std::max<int64_t>(16384, (nk_max + 63) / 64);
  p->rescore_chunks = (int)((nk_max + p->rescore_chunk - 1) / p->rescore_chunk);
  ALLOC(d_rpart, (int64_t)p->cap * p->rescore_chunks);
  ALLOC(d_rcnt, p->cap);
  ALLOC(d_rorder, p->cap);
  ALLOC(d_rruns, p->cap);
  ALLOC(d_rgcount, 4 * (p->groups.size() + 1));
  ALLOC(d_lres, p->lines.size());
  ALLOC(d_labels, std::max<size_t>(1, p->n_pts));
  ALLOC(d_bestq, std::max<size_t>(1, p->n_pts));
  ALLOC(d_golden, p->golden0.size());
  // three-band model: band tables, two momenta x N^2 rows per group; FP32
  // plans: the k-state table, built once per execution and read by each of
  // its k-sum launches (a golden search has 3 + steps of them)
  int64_t e3_rows, kst_rows;
  table_offsets(ctx, p, e3_rows, kst_rows);
  p->e3_rows = e3_rows;
  ALLOC(d_e3d, e3_rows);
  ALLOC(d_e3f, e3_rows);
  int64_t kst_max = kKstateTableMaxBytes;  // FFE_KSTATE_TABLE_MAX_BYTES overrides (0: never a table)
  if (const char* env = getenv("FFE_KSTATE_TABLE_MAX_BYTES")) kst_max = std::strtoll(env, nullptr, 10);
  if (p->prec != FFE_FP32C || kst_rows * (int64_t)(sizeof(float4) + sizeof(float)) > kst_max) kst_rows = 0;
  p->kst_rows = kst_rows;
  ALLOC(d_kst4, kst_rows);
  ALLOC(d_kste, kst_rows);
#undef ALLOC
  return FFE_OK;
}

// Clears counters and uploads the host tables into the plan's buffers.
static ffe_status plan_upload_tables(ffe_context* ctx, ffe_plan* p) {
  ffe_status st;
  cudaStream_t s = p->stream;
  FFE_CU(cudaMemsetAsync(p->d_Mcnt, 0, sizeof(int32_t) * std::max(1, p->n_mcounters), s), "memset");
  FFE_CU(cudaMemsetAsync(p->d_segcnt, 0, sizeof(int32_t) * std::max<size_t>(1, p->segs.size()), s), "memset");
  FFE_CU(cudaMemsetAsync(p->d_rcnt, 0, sizeof(int32_t) * p->cap, s), "memset");
  if ((st = upload(ctx, p->d_groups, p->groups, s)) != FFE_OK) return st;
  if ((st = upload(ctx, p->d_items, p->items, s)) != FFE_OK) return st;
  if ((st = upload(ctx, p->d_segs, p->segs, s)) != FFE_OK) return st;
  if ((st = upload(ctx, p->d_mitems, p->mitems, s)) != FFE_OK) return st;
  if ((st = upload(ctx, p->d_lines, p->lines, s)) != FFE_OK) return st;
  return plan_upload_params(ctx, p, s);
}

// Allocate device buffers for the host tables already in *p and upload them.
ffe_status plan_alloc(ffe_context* ctx, ffe_plan* p) {
  ffe_status st = FFE_OK;
  Arena arena;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {  // one allocation for every buffer of the plan
      const size_t need = std::max<size_t>(arena.off, 256);
      void* raw = nullptr;
      if (ctx->spare && ctx->spare_bytes >= need && ctx->spare_bytes <= 2 * need + (size_t(64) << 20)) {
        raw = ctx->spare;  // the context's kept block fits (and is not far larger)
        p->arena_bytes = ctx->spare_bytes;
        ctx->spare = nullptr;
        ctx->spare_bytes = 0;
      } else {
        cudaError_t e = cudaMalloc(&raw, need);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc");
        p->arena_bytes = need;
      }
      p->arena = raw;
      arena.base = static_cast<unsigned char*>(raw);
      arena.off = 0;
    }
    if ((st = plan_alloc_requests(ctx, p, arena)) != FFE_OK) return st;
  }
  return plan_upload_tables(ctx, p);
}


// The per-call inputs -- Delta values, (h, T) entries, distinct h lists, Q,
// golden-section ranges -- as a list of host-to-device copies.
static ffe_status plan_param_copies(ffe_context* ctx, ffe_plan* p, std::vector<HostCopy>& out) {
  int64_t e3_rows, kst_rows;
  table_offsets(ctx, p, e3_rows, kst_rows);  // refilled groups: offsets again
  if (e3_rows > p->e3_rows || (p->kst_rows > 0 && kst_rows > p->kst_rows))
    return set_err(ctx, "plan groups outgrew their table buffers"), FFE_EINTERNAL;
  auto add = [&](void* dst, const void* src, size_t bytes) {
    if (bytes) out.push_back(HostCopy{dst, src, bytes});
  };
  add(p->d_delta, p->delta.data(), p->delta.size() * sizeof(double));
  add(p->d_ht, p->ht.data(), p->ht.size() * sizeof(HT));
  add(p->d_hlist, p->hlist.data(), p->hlist.size() * sizeof(double));
  add(p->d_groups, p->groups.data(), p->groups.size() * sizeof(GroupDesc));
  add(p->d_qzero, p->q_is_zero.data(), p->q_is_zero.size() * sizeof(int32_t));
  add(p->d_golden, p->golden0.data(), p->golden0.size() * sizeof(GoldenState));
  p->h2d_bytes = p->delta.size() * sizeof(double) + p->ht.size() * sizeof(HT) +
                 p->hlist.size() * sizeof(double) + p->groups.size() * sizeof(GroupDesc) +
                 p->golden0.size() * sizeof(GoldenState);
  return FFE_OK;
}

ffe_status plan_upload_params(ffe_context* ctx, ffe_plan* p, cudaStream_t s) {
  std::vector<HostCopy> copies;
  ffe_status st = plan_param_copies(ctx, p, copies);
  if (st != FFE_OK) return st;
  for (const HostCopy& c : copies)
    FFE_CU(cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, s), "upload");
  return FFE_OK;
}

// A plan refilled with new values of the same shape (a cached plan): the work
// items' far windows depend on the values (h range, T_max, Delta range), so
// they are rebuilt and uploaded with the parameters.  pinned: stage the copies
// in the plan's page-locked buffer so that the call does not wait for the
// device (the buffer is reused once the previous refill's copies are done).
ffe_status plan_refill(ffe_context* ctx, ffe_plan* p, cudaStream_t s, bool pinned) {
  const size_t n_items = p->items.size();
  apply_tiles(p, p->variant == kLayoutProductUT);
  if (!p->item_sig.empty() && item_signature(p) == p->item_sig)
    refresh_item_windows(p);  // same shapes: only the windows follow the new values
  else
    build_items(p);
  if (p->items.size() != n_items) return set_err(ctx, "plan refill changed its work items"), FFE_EINTERNAL;
  std::vector<HostCopy> copies;
  copies.push_back(HostCopy{p->d_items, p->items.data(), p->items.size() * sizeof(WorkItem)});
  ffe_status st = plan_param_copies(ctx, p, copies);
  if (st != FFE_OK) return st;
  if (!pinned) {
    for (const HostCopy& c : copies)
      FFE_CU(cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, s), "upload");
    return FFE_OK;
  }
  size_t need = 0;
  for (const HostCopy& c : copies) need += (c.bytes + 255) & ~size_t(255);
  if (p->staged_ev) FFE_CU(cudaEventSynchronize(p->staged_ev), "staging wait");
  else FFE_CU(cudaEventCreateWithFlags(&p->staged_ev, cudaEventDisableTiming), "event");
  if (need > p->staging_bytes) {
    if (p->staging) cudaFreeHost(p->staging);
    p->staging = nullptr;
    p->staging_bytes = 0;
    FFE_CU(cudaHostAlloc(&p->staging, need, cudaHostAllocDefault), "cudaHostAlloc");
    p->staging_bytes = need;
  }
  unsigned char* buf = static_cast<unsigned char*>(p->staging);
  size_t off = 0;
  for (const HostCopy& c : copies) {
    std::memcpy(buf + off, c.src, c.bytes);
    FFE_CU(cudaMemcpyAsync(c.dst, buf + off, c.bytes, cudaMemcpyHostToDevice, s), "upload");
    off += (c.bytes + 255) & ~size_t(255);
  }
  FFE_CU(cudaEventRecord(p->staged_ev, s), "event");
  return FFE_OK;
}

static KsumArgs make_ksum_args(ffe_plan* p) {
  KsumArgs a;
  a.m = p->ctx->mp;
  a.groups = p->d_groups;
  a.items = p->d_items;
  a.n_items = (int32_t)p->items.size();
  a.pad0 = 0;
  a.segs = p->d_segs;
  a.queue = p->d_counters + 0;
  a.near_evals = p->d_near;
  a.e3f = p->d_e3f;
  a.e3d = p->d_e3d;
  a.kst4 = p->kst_rows > 0 ? p->d_kst4 : nullptr;
  a.kste = p->kst_rows > 0 ? p->d_kste : nullptr;
  a.seg_count = p->d_segcnt;
  a.partials = p->d_partials;
  a.tabf = p->d_tabf;
  a.c0f = p->d_c0f;
  a.tabd = p->d_tabd;
  a.c0d = p->d_c0d;
  a.delta = p->d_delta;
  a.d2f = p->d_d2f;
  a.ht = p->d_ht;
  a.htf = p->d_htf;
  a.htd = p->d_htd;
  a.M = p->d_M;
  a.V = p->d_V;
  a.omega = p->d_omega;
  a.ebound = p->d_eb;
  a.eb_rel = p->prec == FFE_FP32C ? kEbRel : 0.0;
  a.eb_abs = p->prec == FFE_FP32C ? kEbAbs : 0.0;
  a.status = p->d_counters + 7;
  a.w_scaled = p->prec == FFE_FP32C ? 1 : 0;
  a.pad1 = 0;
  return a;
}

static RescoreArgs make_rescore_args(ffe_plan* p, int queue_slot, int count_slot) {
  RescoreArgs r;
  r.m = p->ctx->mp;
  r.groups = p->d_groups;
  r.tabd = p->d_tabd;
  r.e3d = p->d_e3d;
  r.c0d = p->d_c0d;
  r.ht = p->d_ht;
  r.M = p->d_M;
  r.req = p->d_req;
  r.n_req = p->d_counters + count_slot;
  r.chunk_k = p->rescore_chunk;
  r.max_chunks = p->rescore_chunks;
  r.queue = p->d_counters + queue_slot;
  r.counters = p->d_rcnt;
  r.partials = p->d_rpart;
  r.omega = p->d_omega;
  r.ebound = p->d_eb;
  r.lines = p->d_lres;
  r.rescored = p->d_rescored;
  r.golden = p->d_golden;
  r.cap = p->cap;
  r.n_groups = (int32_t)p->groups.size();
  r.order = p->d_rorder;
  r.runs = p->d_rruns;
  r.gcount = p->d_rgcount;
  return r;
}

// The whole device-side sequence of one execution, on stream s.
// counters: [0] k-sum queue, [1] rescore queue A, [2] rescore queue B,
//           [3] requests of the Delta search, [4] requests of the labels,
//           [5] requests of a golden step, [6] its rescore queue,
//           [7] status word.
ffe_status plan_enqueue(ffe_context* ctx, ffe_plan* p, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1,
                        unsigned ev_flags) {
  int launches = 0;
  FFE_CU(cudaMemsetAsync(p->d_counters, 0, 8 * sizeof(int32_t), s), "memset counters");
  FFE_CU(cudaMemsetAsync(p->d_near, 0, 3 * sizeof(unsigned long long), s), "memset counters");
  FFE_CU(cudaMemsetAsync(p->d_rescored, 0, sizeof(int32_t) * std::max<int64_t>(1, p->n_out), s), "memset");
  FFE_CU(prep_params_launch(p->d_delta, (int64_t)p->delta.size(), p->d_d2f, p->d_ht, (int64_t)p->ht.size(),
                            p->d_htf, p->d_htd, s),
         "prep_params");
  ++launches;
  FFE_CU(tables_launch(ctx->mp, p->d_groups, (int)p->groups.size(), p->max_n, p->d_tabf, p->d_c0f, p->d_tabd,
                       p->d_c0d, p->d_tabdf, s),
         "tables");
  ++launches;
  if (ctx->mp.nbands == 3) {
    FFE_CU(bands3_launch(ctx->mp, p->d_groups, (int)p->groups.size(), p->max_n, p->d_tabd, p->d_e3d, p->d_e3f, s),
           "bands3");
    ++launches;
  }
  FFE_CU(normal_launch(ctx->mp, p->d_groups, p->d_mitems, (int)p->mitems.size(), p->d_hlist, p->d_tabd,
                       p->prec == FFE_FP32C ? p->d_tabdf : nullptr, p->d_e3d, p->d_Mpart, p->d_Mcnt, p->d_M, s),
         "normal");
  ++launches;
  KsumArgs ka = make_ksum_args(p);
  if (ka.kst4) {
    FFE_CU(kstate_table_launch(ka, (int)p->groups.size(), p->max_n, s), "k-state table");
    ++launches;
  }
  const int n_lines = (int)p->lines.size();
  if (p->golden_steps > 0) {
    // lockstep golden-section: one k-sum launch per evaluation of every line
    auto golden = [&](int mode) -> ffe_status {
      FFE_CU(golden_launch(mode, p->d_lines, n_lines, p->d_golden, p->d_omega, p->d_eb, p->d_delta, p->d_d2f,
                           p->d_req, p->d_counters + 5, p->cap, p->d_lres, s),
             "golden");
      ++launches;
      return FFE_OK;
    };
    auto ksum = [&]() -> ffe_status {
      FFE_CU(cudaMemsetAsync(p->d_counters + 0, 0, sizeof(int32_t), s), "memset");
      FFE_CU(ksum_launch(p->prec, p->variant, p->kpt, ka, p->grid, p->block, s), "ksum");
      ++launches;
      return FFE_OK;
    };
    ffe_status st;
    if ((st = golden(kGoldenInit)) != FFE_OK) return st;
    if (ev0) FFE_CU(cudaEventRecordWithFlags(ev0, s, ev_flags), "event");
    const int first[3] = {kGoldenLo, kGoldenX1, kGoldenX2};
    for (int i = 0; i < 3; ++i) {
      if ((st = ksum()) != FFE_OK) return st;
      if ((st = golden(first[i])) != FFE_OK) return st;
    }
    for (int step = 0; step < p->golden_steps; ++step) {
      FFE_CU(cudaMemsetAsync(p->d_counters + 5, 0, 2 * sizeof(int32_t), s), "memset");
      if ((st = golden(kGoldenMark)) != FFE_OK) return st;
      FFE_CU(rescore_launch(make_rescore_args(p, 6, 5), p->rescore_grid, s), "rescore golden");
      launches += 2;
      if ((st = golden(kGoldenDecide)) != FFE_OK) return st;
      if ((st = ksum()) != FFE_OK) return st;
      if ((st = golden(kGoldenRecord)) != FFE_OK) return st;
    }
    if (ev1) FFE_CU(cudaEventRecordWithFlags(ev1, s, ev_flags), "event");
    FFE_CU(cudaMemsetAsync(p->d_counters + 5, 0, 2 * sizeof(int32_t), s), "memset");
    if ((st = golden(kGoldenMarkFinal)) != FFE_OK) return st;
    FFE_CU(rescore_launch(make_rescore_args(p, 6, 5), p->rescore_grid, s), "rescore golden");
    launches += 2;
    if ((st = golden(kGoldenFinish)) != FFE_OK) return st;
  } else {
    if (ev0) FFE_CU(cudaEventRecordWithFlags(ev0, s, ev_flags), "event");
    FFE_CU(ksum_launch(p->prec, p->variant, p->kpt, ka, p->grid, p->block, s), "ksum");
    ++launches;
    if (ev1) FFE_CU(cudaEventRecordWithFlags(ev1, s, ev_flags), "event");
  }
  if (!p->lines.empty()) {
    if (p->golden_steps == 0) {
    FFE_CU(argmin_launch(p->d_lines, n_lines, p->d_omega, p->d_eb, p->d_delta, p->d_rescored, 0, p->d_req,
                         p->d_counters + 3, p->cap, p->d_lres, s),
           "argmin A");
    FFE_CU(rescore_launch(make_rescore_args(p, 1, 3), p->rescore_grid, s), "rescore A");
    FFE_CU(argmin_launch(p->d_lines, n_lines, p->d_omega, p->d_eb, p->d_delta, p->d_rescored, 1, p->d_req,
                         p->d_counters + 3, p->cap, p->d_lres, s),
           "argmin B");
    launches += 4;  // argmin A, request grouping, rescore, argmin B
    }
    if (p->n_q > 0) {
      // the request slots are reused once pass A's requests are done (stream order)
      FFE_CU(labels_launch(p->d_lres, p->n_q, p->n_pts, p->d_qzero, p->d_lines, p->d_delta, 0, p->d_req,
                           p->d_counters + 4, p->cap, p->d_labels, p->d_bestq, s),
             "labels 0");
      FFE_CU(rescore_launch(make_rescore_args(p, 2, 4), p->rescore_grid, s), "rescore B");
      FFE_CU(labels_launch(p->d_lres, p->n_q, p->n_pts, p->d_qzero, p->d_lines, p->d_delta, 1, p->d_req,
                           p->d_counters + 4, p->cap, p->d_labels, p->d_bestq, s),
             "labels 1");
      launches += 4;  // labels 0, request grouping, rescore, labels 1
    }
  }
  p->launches = launches;
  return FFE_OK;
}

ffe_status plan_configure(ffe_context* ctx, ffe_plan* p) {
  p->variant = p->layout;
  if (p->prec == FFE_FP32C && p->layout == kLayoutProduct && batches_share_T(p)) p->variant = kLayoutProductUT;
  apply_tiles(p, p->variant == kLayoutProductUT);
  // launch shape: persistent grid of resident blocks
  const Tuning t = tuning_for(ctx, p);
  p->kpt = t.kpt;
  p->block = t.block;
  p->item_target = t.item_target;
  p->tuning = t;
  int bps = 0;
  cudaError_t e = ksum_occupancy(p->prec, p->variant, p->kpt, p->block, &bps);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "occupancy");
  if (bps < 1) bps = 1;
  p->grid = ctx->n_sm * bps;
  int rbps = 0;
  e = rescore_occupancy(&rbps);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "occupancy");
  p->rescore_grid = ctx->n_sm * std::max(1, rbps);
  build_items(p);
  build_mitems(p);
  p->k_evals = plan_k_evals(p);
  return FFE_OK;
}

ffe_status plan_finish(ffe_context* ctx, ffe_plan* p, bool use_graph) {
  ffe_status st = plan_alloc(ctx, p);
  if (st != FFE_OK) return st;
  FFE_CU(cudaStreamSynchronize(p->stream), "sync");
  if (!use_graph) return FFE_OK;
  cudaGraph_t graph = nullptr;
  FFE_CU(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  st = plan_enqueue(ctx, p, p->stream, p->ev_cap0, p->ev_cap1, cudaEventRecordExternal);
  cudaError_t e = cudaStreamEndCapture(p->stream, &graph);
  if (st != FFE_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
  p->graph = graph;
  e = cudaGraphInstantiate(&p->exec, graph, 0);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
  // locate the two event-record nodes around the k-sum
  size_t n = 0;
  FFE_CU(cudaGraphGetNodes(graph, nullptr, &n), "graph nodes");
  std::vector<cudaGraphNode_t> nodes(n);
  FFE_CU(cudaGraphGetNodes(graph, nodes.data(), &n), "graph nodes");
  for (cudaGraphNode_t node : nodes) {
    cudaGraphNodeType ty;
    FFE_CU(cudaGraphNodeGetType(node, &ty), "node type");
    if (ty != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t ev;
    FFE_CU(cudaGraphEventRecordNodeGetEvent(node, &ev), "node event");
    if (ev == p->ev_cap0) p->node_ev0 = node;
    if (ev == p->ev_cap1) p->node_ev1 = node;
  }
  if (!p->node_ev0 || !p->node_ev1) {
    set_err(ctx, "event nodes not found in the captured graph");
    return FFE_EINTERNAL;
  }
  return FFE_OK;
}

ffe_status plan_run(ffe_context* ctx, ffe_plan* p, cudaStream_t s) {
  {
    const int slot = (int)(p->exec_count % kRing);
    if (!p->ring0[slot]) FFE_CU(cudaEventCreate(&p->ring0[slot]), "event");
    if (!p->ring1[slot]) FFE_CU(cudaEventCreate(&p->ring1[slot]), "event");
  }
  if (p->exec) {
    const int slot = (int)(p->exec_count % kRing);
    FFE_CU(cudaGraphExecEventRecordNodeSetEvent(p->exec, p->node_ev0, p->ring0[slot]), "set event");
    FFE_CU(cudaGraphExecEventRecordNodeSetEvent(p->exec, p->node_ev1, p->ring1[slot]), "set event");
    FFE_CU(cudaGraphLaunch(p->exec, s), "graph launch");
    ++p->exec_count;
    return FFE_OK;
  }
  const int slot = (int)(p->exec_count % kRing);
  ffe_status st = plan_enqueue(ctx, p, s, p->ring0[slot], p->ring1[slot], cudaEventRecordDefault);
  if (st == FFE_OK) ++p->exec_count;
  return st;
}

ffe_status plan_check_status(ffe_context* ctx, ffe_plan* p, cudaStream_t s) {
  int32_t c[8];
  FFE_CU(cudaMemcpyAsync(c, p->d_counters, sizeof c, cudaMemcpyDeviceToHost, s), "status");
  FFE_CU(cudaStreamSynchronize(s), "sync");
  if (c[7] != 0) {
    set_err(ctx, "device status word %d", c[7]);
    return FFE_EINTERNAL;
  }
  return FFE_OK;
}

ffe_plan* plan_new(ffe_context* ctx, int kind) {
  ffe_plan* p = new ffe_plan();
  p->ctx = ctx;
  p->kind = kind;
  p->prec = ctx->model.prec;
  cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
  cudaEventCreate(&p->ev_cap0);
  cudaEventCreate(&p->ev_cap1);  // the timing ring's events are made on first use (plan_run)
  return p;
}

void plan_free(ffe_plan* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->arena) {  // kept by the context for the next plan, or freed
    ffe_context* c = p->ctx;
    if (c && p->arena_bytes <= kSpareMaxBytes && p->arena_bytes > c->spare_bytes) {
      // executions may still run on a caller's stream: wait for the device,
      // as cudaFree would
      cudaDeviceSynchronize();
      if (c->spare) cudaFree(c->spare);
      c->spare = p->arena;
      c->spare_bytes = p->arena_bytes;
    } else {
      cudaFree(p->arena);
    }
  }
  if (p->staging) cudaFreeHost(p->staging);
  if (p->staged_ev) cudaEventDestroy(p->staged_ev);
  if (p->ev_cap0) cudaEventDestroy(p->ev_cap0);
  if (p->ev_cap1) cudaEventDestroy(p->ev_cap1);
  for (int i = 0; i < kRing; ++i) {
    if (p->ring0[i]) cudaEventDestroy(p->ring0[i]);
    if (p->ring1[i]) cudaEventDestroy(p->ring1[i]);
  }
  if (p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

}  // namespace ffe

// ---------------------------------------------------------- plan builders
namespace ffe {

ffe_status check_scan(ffe_context* ctx, const ffe_scan* sc) {
  if (!sc) return set_err(ctx, "scan is NULL"), FFE_EINVAL;
  if (!valid_N(sc->N)) return set_err(ctx, "N=%d must be even in [2, 8192]", sc->N), FFE_EINVAL;
  if (sc->n_q < 1 || sc->n_h < 1 || sc->n_T < 1 || !sc->qx || !sc->qy || !sc->h || !sc->T)
    return set_err(ctx, "scan lists must be non-empty"), FFE_EINVAL;
  if (sc->search != FFE_SEARCH_GRID && sc->search != FFE_SEARCH_GOLDEN)
    return set_err(ctx, "unknown search kind %d", sc->search), FFE_EINVAL;
  if (sc->search == FFE_SEARCH_GRID && (sc->n < 1 || sc->n > 65536))
    return set_err(ctx, "grid points n=%d out of [1, 65536]", sc->n), FFE_EINVAL;
  if (sc->search == FFE_SEARCH_GOLDEN && (sc->n < 1 || sc->n > 200))
    return set_err(ctx, "golden reductions n=%d out of [1, 200]", sc->n), FFE_EINVAL;
  if (!finite(sc->lo) || !finite(sc->hi) || sc->lo > sc->hi || sc->lo != 0.0)
    return set_err(ctx, "Delta range must be finite with lo = 0 <= hi"), FFE_EINVAL;
  for (int i = 0; i < sc->n_q; ++i)
    if (!finite(sc->qx[i]) || !finite(sc->qy[i])) return set_err(ctx, "q not finite"), FFE_EINVAL;
  for (int i = 0; i < sc->n_h; ++i)
    if (!finite(sc->h[i])) return set_err(ctx, "h not finite"), FFE_EINVAL;
  for (int i = 0; i < sc->n_T; ++i)
    if (!(sc->T[i] > 0.0) || !finite(sc->T[i])) return set_err(ctx, "T must be > 0"), FFE_EINVAL;
  const int64_t outs = (int64_t)sc->n_q * sc->n_h * sc->n_T * (int64_t)std::max(1, sc->n);
  if (outs > ((int64_t)1 << 31)) return set_err(ctx, "scan too large"), FFE_EINVAL;
  return FFE_OK;
}

// Labels need the normal state of Q = (0, 0) in the q list.
static bool scan_has_q0(const ffe_scan* sc) {
  for (int i = 0; i < sc->n_q; ++i)
    if (sc->qx[i] == 0.0 && sc->qy[i] == 0.0) return true;
  return false;
}

static bool plan_has_q0(const ffe_plan* p) {
  for (int32_t z : p->q_is_zero)
    if (z) return true;
  return false;
}

// Grid scan: one PRODUCT group per q (outputs = Delta grid x (h,T) points).
static void fill_scan_grid(ffe_plan* p, const ffe_scan* sc) {
  const int n_pts = sc->n_h * sc->n_T;
  p->layout = kLayoutProduct;
  p->n_q = sc->n_q;
  p->n_pts = n_pts;
  p->groups.clear();
  p->delta.clear();
  p->ht.clear();
  p->hlist.clear();
  p->lines.clear();
  p->q_is_zero.assign(sc->n_q, 0);
  std::vector<double> grid(sc->n);
  linspace(sc->lo, sc->hi, sc->n, grid.data());
  int64_t out = 0;
  for (int q = 0; q < sc->n_q; ++q) {
    GroupDesc g;
    std::memset(&g, 0, sizeof g);
    g.N = sc->N;
    g.layout = kLayoutProduct;
    g.n_delta = sc->n;
    g.n_ht = n_pts;
    g.hb = 32;  // apply_tiles sets the batch shape of the kernel variant
    g.n_hblk = (n_pts + 31) / 32;
    g.n_batches = g.n_delta * g.n_hblk;
    g.n_h = sc->n_h;
    g.n_out = sc->n * n_pts;
    g.out_off = out;
    g.delta_off = (int64_t)p->delta.size();
    g.ht_off = (int64_t)p->ht.size();
    g.tab_off = (int64_t)q * 2 * sc->N;
    g.h_off = (int64_t)p->hlist.size();
    g.qx = sc->qx[q];
    g.qy = sc->qy[q];
    p->q_is_zero[q] = (sc->qx[q] == 0.0 && sc->qy[q] == 0.0) ? 1 : 0;
    p->delta.insert(p->delta.end(), grid.begin(), grid.end());
    // (h, T) entries T-major, so that a batch of 32 shares one T where it can
    // (point pt = ih n_T + it is entry it n_h + ih); lines stay in point order
    for (int it = 0; it < sc->n_T; ++it)
      for (int ih = 0; ih < sc->n_h; ++ih) p->ht.push_back(HT{sc->h[ih], sc->T[it], ih, 0});
    p->hlist.insert(p->hlist.end(), sc->h, sc->h + sc->n_h);
    for (int pt = 0; pt < n_pts; ++pt) {
      const int e = (pt % sc->n_T) * sc->n_h + pt / sc->n_T;
      Line L;
      L.out0 = out + e;
      L.stride = n_pts;
      L.count = sc->n;
      L.group = q;
      L.pad = 0;
      L.delta0 = g.delta_off;
      L.ht = g.ht_off + e;
      p->lines.push_back(L);
    }
    out += g.n_out;
    p->groups.push_back(g);
  }
  p->n_out = out;
}

// Golden scan: one LIST group per q whose outputs are the (h, T) points; each
// output carries its own Delta, rewritten on the device after every step.
static void fill_scan_golden(ffe_plan* p, const ffe_scan* sc) {
  const int n_pts = sc->n_h * sc->n_T;
  p->layout = kLayoutList;
  p->n_q = sc->n_q;
  p->n_pts = n_pts;
  p->golden_steps = sc->n;
  p->groups.clear();
  p->delta.clear();
  p->ht.clear();
  p->hlist.clear();
  p->lines.clear();
  p->golden0.clear();
  p->q_is_zero.assign(sc->n_q, 0);
  int64_t out = 0;
  for (int q = 0; q < sc->n_q; ++q) {
    GroupDesc g;
    std::memset(&g, 0, sizeof g);
    g.N = sc->N;
    g.layout = kLayoutList;
    g.n_out = n_pts;
    g.n_delta = n_pts;
    g.n_ht = n_pts;
    g.n_hblk = 1;
    g.n_batches = (n_pts + 31) / 32;
    g.n_h = sc->n_h;
    g.out_off = out;
    g.delta_off = (int64_t)p->delta.size();
    g.ht_off = (int64_t)p->ht.size();
    g.tab_off = (int64_t)q * 2 * sc->N;
    g.h_off = (int64_t)p->hlist.size();
    g.qx = sc->qx[q];
    g.qy = sc->qy[q];
    p->q_is_zero[q] = (sc->qx[q] == 0.0 && sc->qy[q] == 0.0) ? 1 : 0;
    // outputs T-major, so that a batch of 32 shares one T where it can
    // (point pt = ih n_T + it is output it n_h + ih); lines stay in point order
    for (int it = 0; it < sc->n_T; ++it)
      for (int ih = 0; ih < sc->n_h; ++ih) {
        p->ht.push_back(HT{sc->h[ih], sc->T[it], ih, 0});
        p->delta.push_back(sc->lo);
      }
    p->hlist.insert(p->hlist.end(), sc->h, sc->h + sc->n_h);
    for (int pt = 0; pt < n_pts; ++pt) {
      const int e = (pt % sc->n_T) * sc->n_h + pt / sc->n_T;
      Line L;
      L.out0 = out + e;
      L.stride = 1;
      L.count = 1;
      L.group = q;
      L.pad = 0;
      L.delta0 = g.delta_off + e;
      L.ht = g.ht_off + e;
      p->lines.push_back(L);
      GoldenState gs;
      std::memset(&gs, 0, sizeof gs);
      gs.lo = sc->lo;
      gs.hi = sc->hi;
      gs.x0 = sc->lo;
      p->golden0.push_back(gs);
    }
    out += g.n_out;
    p->groups.push_back(g);
  }
  p->n_out = out;
}

void fill_scan(ffe_plan* p, const ffe_scan* sc) {
  if (sc->search == FFE_SEARCH_GOLDEN)
    fill_scan_golden(p, sc);
  else
    fill_scan_grid(p, sc);
}

ffe_status fetch_scan(ffe_context* ctx, ffe_plan* p, ffe_result* per_point, int8_t* labels,
                             int32_t* best_q, cudaStream_t s) {
  ffe_status st = plan_check_status(ctx, p, s);
  if (st != FFE_OK) return st;
  std::vector<LineResult> lr(p->lines.size());
  FFE_CU(cudaMemcpyAsync(lr.data(), p->d_lres, lr.size() * sizeof(LineResult), cudaMemcpyDeviceToHost, s),
         "fetch lines");
  if (labels)
    FFE_CU(cudaMemcpyAsync(labels, p->d_labels, p->n_pts * sizeof(int8_t), cudaMemcpyDeviceToHost, s), "fetch");
  if (best_q)
    FFE_CU(cudaMemcpyAsync(best_q, p->d_bestq, p->n_pts * sizeof(int32_t), cudaMemcpyDeviceToHost, s), "fetch");
  int32_t nreq[2] = {0, 0};
  FFE_CU(cudaMemcpyAsync(nreq, p->d_counters + 3, sizeof nreq, cudaMemcpyDeviceToHost, s), "fetch");
  FFE_CU(cudaStreamSynchronize(s), "sync");
  p->last_rescored[0] = nreq[0];
  p->last_rescored[1] = nreq[1];
  if (nreq[0] > p->cap || nreq[1] > p->cap) {
    set_err(ctx, "FP64 re-evaluation requests (%d, %d) exceeded capacity (%d)", nreq[0], nreq[1], p->cap);
    return FFE_EINTERNAL;
  }
  if (per_point) {
    for (size_t i = 0; i < lr.size(); ++i) {
      ffe_result& r = per_point[i];
      r.delta_star = lr[i].delta_star;
      r.omega_star = lr[i].omega_star;
      r.omega_lo = lr[i].omega_lo;
      r.err_bound = lr[i].eb_star;
      r.idx_star = lr[i].idx_star;
      r.flags = lr[i].flags;
    }
  }
  p->d2h_bytes = lr.size() * sizeof(LineResult) + (labels ? p->n_pts : 0) + (best_q ? 4 * p->n_pts : 0);
  return FFE_OK;
}

}  // namespace ffe

// ------------------------------------------------------------------- C ABI
extern "C" {

const char* ffe_status_string(ffe_status s) {
  switch (s) {
    case FFE_OK: return "ok";
    case FFE_EINVAL: return "invalid argument";
    case FFE_ENOMEM: return "out of memory";
    case FFE_ECUDA: return "CUDA error";
    case FFE_ETIMEOUT: return "device wait timed out";
    case FFE_EUNSUPPORTED: return "unsupported";
    case FFE_EINTERNAL: return "internal error";
  }
  return "unknown status";
}

const char* ffe_last_error(const ffe_context* ctx) { return ctx ? ctx->err.c_str() : ""; }

ffe_status ffe_create(const ffe_model* m, ffe_context** out) {
  if (!out) return FFE_EINVAL;
  *out = nullptr;
  if (!m) return FFE_EINVAL;
  if (m->kind != FFE_MODEL_RAGHU2 && m->kind != FFE_MODEL_DAGHOFER3) return FFE_EUNSUPPORTED;
  if (m->prec != FFE_FP64 && m->prec != FFE_FP32C) return FFE_EINVAL;
  if (!(m->U > 0.0) || !std::isfinite(m->U) || !std::isfinite(m->t1) || !std::isfinite(m->t2) ||
      !std::isfinite(m->t3) || !std::isfinite(m->t4) || !std::isfinite(m->mu) || !std::isfinite(m->eta_amp))
    return FFE_EINVAL;
  if (m->kind == FFE_MODEL_DAGHOFER3) {
    for (double x : {m->t5, m->t6, m->t7, m->t8, m->t9, m->t10, m->t11, m->t12, m->eps0})
      if (!std::isfinite(x)) return FFE_EINVAL;
  }
  const int nb = m->kind == FFE_MODEL_DAGHOFER3 ? 3 : 2;
  for (int b = 0; b < 3; ++b)
    if (!std::isfinite(m->U_band[b]) || m->U_band[b] < 0.0 || (b >= nb && m->U_band[b] != 0.0))
      return FFE_EINVAL;
  ffe_context* ctx = new (std::nothrow) ffe_context();
  if (!ctx) return FFE_ENOMEM;
  ctx->model = *m;
  ModelParams mp;
  std::memset(&mp, 0, sizeof mp);
  mp.t1 = m->t1;
  mp.t2 = m->t2;
  mp.t3 = m->t3;
  mp.t4 = m->t4;
  mp.mu = m->mu;
  mp.U = m->U;
  mp.eta_amp = m->eta_amp;
  mp.kind = m->kind;
  mp.nbands = m->kind == FFE_MODEL_DAGHOFER3 ? 3 : 2;
  if (m->kind == FFE_MODEL_DAGHOFER3) {
    mp.t5 = m->t5;
    mp.t6 = m->t6;
    mp.t7 = m->t7;
    mp.t8 = m->t8;
    mp.t9 = m->t9;
    mp.t10 = m->t10;
    mp.t11 = m->t11;
    mp.t12 = m->t12;
    mp.eps0 = m->eps0;
  }
  for (int b = 0; b < 3; ++b) {
    mp.Ub[b] = m->U_band[b] > 0.0 ? m->U_band[b] : m->U;
    if (b < mp.nbands && mp.Ub[b] != m->U) mp.per_band_u = 1;
  }
  ctx->mp = mp;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) {
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, ctx->device);
    if (e == cudaSuccess) ctx->device_name = prop.name;
  }
  if (e != cudaSuccess) {
    delete ctx;
    return FFE_ECUDA;
  }
  tuning_load(ctx);
  *out = ctx;
  return FFE_OK;
}

void ffe_destroy(ffe_context* ctx) {
  if (!ctx) return;
  for (ffe_plan* p : ctx->plans) plan_free(p);
  for (auto& kv : ctx->cache) plan_free(kv.second);
  if (ctx->spare) cudaFree(ctx->spare);
  if (ctx->direct) cudaFree(ctx->direct);
  delete ctx;
}

ffe_status ffe_plan_phase_scan(ffe_context* ctx, const ffe_scan* scan, void* stream, ffe_plan** out) {
  if (!ctx || !out) return FFE_EINVAL;
  *out = nullptr;
  ffe_status st = check_scan(ctx, scan);
  if (st != FFE_OK) return st;
  ffe_plan* p = plan_new(ctx, scan->search == FFE_SEARCH_GRID ? kPlanScanGrid : kPlanScanGolden);
  fill_scan(p, scan);
  st = plan_configure(ctx, p);
  if (st == FFE_OK) st = plan_finish(ctx, p, true);
  if (st != FFE_OK) {
    plan_free(p);
    return st;
  }
  (void)stream;
  ctx->plans.push_back(p);
  *out = p;
  return FFE_OK;
}

ffe_status ffe_plan_execute(ffe_plan* p, void* stream) {
  if (!p) return FFE_EINVAL;
  return plan_run(p->ctx, p, (cudaStream_t)stream);
}

ffe_status ffe_plan_fetch(ffe_plan* p, ffe_result* per_point, int8_t* labels, int32_t* best_q, void* stream) {
  if (!p) return FFE_EINVAL;
  if ((labels || best_q) && !plan_has_q0(p))
    return set_err(p->ctx, "labels need Q = (0, 0) in the q list"), FFE_EINVAL;
  return fetch_scan(p->ctx, p, per_point, labels, best_q, (cudaStream_t)stream);
}

ffe_status ffe_plan_fetch_grid(ffe_plan* p, double* omega_grid, double* err_grid, void* stream) {
  if (!p || !omega_grid) return FFE_EINVAL;
  ffe_context* ctx = p->ctx;
  if (p->kind != kPlanScanGrid) return set_err(ctx, "ffe_plan_fetch_grid: not a grid phase-scan plan"), FFE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  ffe_status st = plan_check_status(ctx, p, s);
  if (st != FFE_OK) return st;
  std::vector<double> om(p->n_out), eb(err_grid ? p->n_out : 0);
  FFE_CU(cudaMemcpyAsync(om.data(), p->d_omega, p->n_out * sizeof(double), cudaMemcpyDeviceToHost, s), "fetch");
  if (err_grid) FFE_CU(cudaMemcpyAsync(eb.data(), p->d_eb, p->n_out * sizeof(double), cudaMemcpyDeviceToHost, s), "fetch");
  FFE_CU(cudaStreamSynchronize(s), "sync");
  int64_t k = 0;
  for (const Line& L : p->lines)  // lines in the order of ffe_plan_fetch's per_point
    for (int i = 0; i < L.count; ++i, ++k) {
      omega_grid[k] = om[L.out0 + (int64_t)i * L.stride];
      if (err_grid) err_grid[k] = eb[L.out0 + (int64_t)i * L.stride];
    }
  return FFE_OK;
}

ffe_status ffe_plan_stats(const ffe_plan* p, ffe_plan_info* info) {
  if (!p || !info) return FFE_EINVAL;
  std::memset(info, 0, sizeof *info);
  info->k_evals = p->k_evals;
  info->launches = p->launches;
  info->rescored_search = p->last_rescored[0];
  info->rescored_labels = p->last_rescored[1];
  info->kpt = p->kpt;
  info->block = p->block;
  info->grid = p->grid;
  info->work_items = (int32_t)p->items.size();
  info->device_bytes = (double)p->bytes;
  info->k_evals_near = -1.0;
  info->k_evals_single = -1.0;
  info->k_evals_far_closed = -1.0;
  if (p->d_near && p->exec_count > 0) {
    unsigned long long n[3] = {0, 0, 0};
    if (cudaMemcpy(n, p->d_near, sizeof n, cudaMemcpyDeviceToHost) != cudaSuccess) return FFE_ECUDA;
    info->k_evals_near = (double)n[0];
    info->k_evals_single = (double)n[1];
    info->k_evals_far_closed = (double)n[2];
  }
  return FFE_OK;
}

ffe_status ffe_plan_kernel_ms(ffe_plan* p, double* ms, int32_t* count) {
  if (!p) return FFE_EINVAL;
  ffe_context* ctx = p->ctx;
  const int64_t n = std::min<int64_t>(p->exec_count - p->timed_upto, kRing);
  double tot = 0.0;
  for (int64_t i = p->exec_count - n; i < p->exec_count; ++i) {
    const int slot = (int)(i % kRing);
    FFE_CU(cudaEventSynchronize(p->ring1[slot]), "event sync");
    float f = 0.f;
    FFE_CU(cudaEventElapsedTime(&f, p->ring0[slot], p->ring1[slot]), "elapsed");
    tot += f;
  }
  p->timed_upto = p->exec_count;
  if (ms) *ms = n > 0 ? tot / (double)n : 0.0;
  if (count) *count = (int32_t)n;
  return FFE_OK;
}

void ffe_plan_destroy(ffe_plan* p) {
  if (!p) return;
  ffe_context* ctx = p->ctx;
  auto it = std::find(ctx->plans.begin(), ctx->plans.end(), p);
  if (it != ctx->plans.end()) ctx->plans.erase(it);
  plan_free(p);
}

ffe_status ffe_phase_scan_async(ffe_context* ctx, const ffe_scan* scan, ffe_result* per_point, int8_t* labels,
                                int32_t* best_q, void* stream) {
  if (!ctx) return FFE_EINVAL;
  ffe_status st = check_scan(ctx, scan);
  if (st != FFE_OK) return st;
  if ((labels || best_q) && !scan_has_q0(scan))
    return set_err(ctx, "labels need Q = (0, 0) in the q list"), FFE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  char key[160];
  snprintf(key, sizeof key, "ascan:%d:%d:%d:%d:%d:%d:%d", ctx->model.prec, scan->search, scan->N, scan->n_q,
           scan->n_h, scan->n_T, scan->n);
  const int kind = scan->search == FFE_SEARCH_GRID ? kPlanScanGrid : kPlanScanGolden;
  ffe_plan* p = nullptr;
  auto it = ctx->cache.find(key);
  if (it != ctx->cache.end()) {
    p = it->second;
    fill_scan(p, scan);
    const bool ut = ctx->model.prec == FFE_FP32C && kind == kPlanScanGrid && batches_share_T(p);
    if (ut != (p->variant == kLayoutProductUT)) {  // the kernel variant no longer fits: rebuild
      plan_free(p);
      ctx->cache.erase(it);
      p = nullptr;
    } else if ((st = plan_refill(ctx, p, s, true)) != FFE_OK) {
      return st;
    }
  }
  if (!p) {
    p = plan_new(ctx, kind);
    fill_scan(p, scan);
    st = plan_configure(ctx, p);
    if (st == FFE_OK) st = plan_finish(ctx, p, true);
    if (st != FFE_OK) {
      plan_free(p);
      return st;
    }
    ctx->cache[key] = p;
  }
  if ((st = plan_run(ctx, p, s)) != FFE_OK) return st;
  cudaError_t e = cudaSuccess;
  if (per_point) e = results_launch(p->d_lres, (int64_t)p->lines.size(), p->d_counters, p->cap, per_point, s);
  if (e == cudaSuccess && labels)
    e = cudaMemcpyAsync(labels, p->d_labels, p->n_pts * sizeof(int8_t), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && best_q)
    e = cudaMemcpyAsync(best_q, p->d_bestq, p->n_pts * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? FFE_OK : cuda_fail(ctx, e, "ffe_phase_scan_async");
}

ffe_status ffe_phase_scan(ffe_context* ctx, const ffe_scan* scan, ffe_result* per_point, int8_t* labels,
                          int32_t* best_q, void* stream) {
  if (!ctx) return FFE_EINVAL;
  ffe_status st = check_scan(ctx, scan);
  if (st != FFE_OK) return st;
  if ((labels || best_q) && !scan_has_q0(scan))
    return set_err(ctx, "labels need Q = (0, 0) in the q list"), FFE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  char key[160];
  snprintf(key, sizeof key, "scan:%d:%d:%d:%d:%d:%d:%d", ctx->model.prec, scan->search, scan->N, scan->n_q,
           scan->n_h, scan->n_T, scan->n);
  const int kind = scan->search == FFE_SEARCH_GRID ? kPlanScanGrid : kPlanScanGolden;
  ffe_plan* p = nullptr;
  auto it = ctx->cache.find(key);
  if (it != ctx->cache.end()) {
    p = it->second;
    fill_scan(p, scan);
    const bool ut = ctx->model.prec == FFE_FP32C && kind == kPlanScanGrid && batches_share_T(p);
    if (ut != (p->variant == kLayoutProductUT)) {  // the kernel variant no longer fits: rebuild
      plan_free(p);
      ctx->cache.erase(it);
      p = nullptr;
    } else if ((st = plan_refill(ctx, p, s, false)) != FFE_OK) {
      return st;
    }
  }
  if (!p) {
    p = plan_new(ctx, kind);
    fill_scan(p, scan);
    st = plan_configure(ctx, p);
    if (st == FFE_OK) st = plan_finish(ctx, p, true);
    if (st != FFE_OK) {
      plan_free(p);
      return st;
    }
    ctx->cache[key] = p;
  }
  if ((st = plan_run(ctx, p, s)) != FFE_OK) return st;
  return fetch_scan(ctx, p, per_point, labels, best_q, s);
}

}  // extern "C"
