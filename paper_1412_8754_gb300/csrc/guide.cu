// guide.cu -- phase scan guided by the learned surrogate.
//
// A full scan (Alg. 1) searches every (q, h, T) line over the whole Delta
// range.  Guided, the surrogate first predicts the condensation energy of
// every line on a Delta grid (tensor-core inference), and the exact k-sum
// evaluates the lines' normal states (Delta = 0: at a sample of points, and
// at every point where the sample shows the normal states of different q
// to differ by more than a tenth of the margin); per
// (h, T) only q = 0 and the q_keep lines with the lowest predicted minimum
// (exact normal state + predicted condensation energy; with a margin also
// every q predicted to condense by more than the margin within the margin of
// the lowest, and every q whose exact normal state lies more than the margin
// below that of q = 0) are verified by the exact k-sum,
// each on a window of `window` grid points around its predicted
// minimum, with Delta = 0 as the reference (same kernels, same FP64
// re-evaluation of near ties, same label passes as the full scan).  A grid
// scan evaluates the window's grid points; a golden-section scan brackets
// the window and needs fewer reductions for the same final bracket width.
// Where a verified minimum sits on an inner edge of its window (or the
// margin flags a line), the (h, T) point is scanned again with all its
// verified lines over the whole range.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "plan.h"

namespace ffe {

// x[l * n + i] = (q_l, h_l, T_l, grid_i)
__global__ void guide_inputs_kernel(const float4* __restrict__ line_qht, const float* __restrict__ grid, int n_lines,
                                    int n, float4* x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n_lines * n) return;
  const int l = (int)(i / n), j = (int)(i - (int64_t)l * n);
  const float4 p = line_qht[l];
  x[i] = make_float4(p.x, p.y, p.z, grid[j]);
}

// Per line: the grid index of the lowest prediction (ties to the lowest index).
__global__ void guide_argmin_kernel(const float* __restrict__ y, int n_lines, int n, int32_t* idx, float* ymin) {
  const int l = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (l >= n_lines) return;
  float best = INFINITY;
  int bi = 0x7fffffff;
  for (int j = lane; j < n; j += 32) {
    const float v = y[(int64_t)l * n + j];
    if (v < best) {
      best = v;
      bi = j;
    }
  }
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const float ov = __shfl_xor_sync(kFull, best, s);
    const int oi = __shfl_xor_sync(kFull, bi, s);
    if (ov < best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  if (lane == 0) {
    idx[l] = bi == 0x7fffffff ? 0 : bi;
    ymin[l] = best;
  }
}

// Copies the prediction rows of the listed lines next to each other.
__global__ void guide_gather_kernel(const float* __restrict__ y, const int32_t* __restrict__ rows, int n_rows, int n,
                                    float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n_rows * n) return;
  const int r = (int)(i / n), j = (int)(i - (int64_t)r * n);
  out[i] = y[(int64_t)rows[r] * n + j];
}

namespace {

constexpr int kGuideGrid = 256;  // prediction grid of a golden-section scan
constexpr double kGuidePhi = 0.61803398874989484820;

struct LineSpec {
  std::vector<int> grid_idx;    // grid search: grid index of each output, grid_idx[0] == 0
  double wlo = 0.0, whi = 0.0;  // golden search: bracket
  bool alias = false;           // not evaluated: reads the q = 0 line's reference output
};

// A scan-shaped plan over the points `pts` (indices ih * n_T + it of the
// scan) whose lines carry explicit Delta lists (grid) or brackets (golden):
// one LIST group per q, lines q-major (the label passes expect that order),
// spec[q * pts.size() + j].  A group's h list holds only the h values of its
// evaluated lines.  An alias line points at the q = 0 line's first output
// (grid: Delta = 0): its minimum is its lower end, so it never competes for
// a label and costs no k-sum work.
void fill_explicit(ffe_plan* p, const ffe_scan* sc, int q0, const std::vector<int>& pts, int golden_steps,
                   const std::vector<double>& grid, const std::vector<LineSpec>& spec) {
  const int n_sub = (int)pts.size();
  const bool golden = golden_steps > 0;
  p->layout = kLayoutList;
  p->n_q = sc->n_q;
  p->n_pts = n_sub;
  p->golden_steps = golden_steps;
  p->q_is_zero.assign(sc->n_q, 0);
  p->lines.assign((size_t)sc->n_q * n_sub, Line{});
  if (golden) p->golden0.assign((size_t)sc->n_q * n_sub, GoldenState{});
  int64_t out = 0;
  std::vector<int> h_local(sc->n_h);
  for (int q = 0; q < sc->n_q; ++q) {
    GroupDesc g;
    std::memset(&g, 0, sizeof g);
    g.N = sc->N;
    g.layout = kLayoutList;
    g.out_off = out;
    g.delta_off = (int64_t)p->delta.size();
    g.ht_off = (int64_t)p->ht.size();
    g.tab_off = (int64_t)q * 2 * sc->N;
    g.h_off = (int64_t)p->hlist.size();
    g.qx = sc->qx[q];
    g.qy = sc->qy[q];
    p->q_is_zero[q] = (sc->qx[q] == 0.0 && sc->qy[q] == 0.0) ? 1 : 0;
    std::fill(h_local.begin(), h_local.end(), -1);
    int n_hq = 0;
    for (int j = 0; j < n_sub; ++j)
      if (!spec[(size_t)q * n_sub + j].alias) h_local[pts[j] / sc->n_T] = 0;
    for (int ih = 0; ih < sc->n_h; ++ih)
      if (h_local[ih] == 0) {
        h_local[ih] = n_hq++;
        p->hlist.push_back(sc->h[ih]);
      }
    g.n_h = n_hq;
    // Golden: the group's outputs (one per line) ordered by T, then bracket, so
    // that a batch of 32 outputs shares T and, while its lines take the same
    // decisions, Delta -- the shared-T evaluation of the k-sum; the lines keep
    // their order (each points at its own output).
    std::vector<int> order;
    for (int j = 0; j < n_sub; ++j)
      if (!spec[(size_t)q * n_sub + j].alias) order.push_back(j);
    if (golden)
      std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const LineSpec &a = spec[(size_t)q * n_sub + x], &b = spec[(size_t)q * n_sub + y];
        const int tx = pts[x] % sc->n_T, ty = pts[y] % sc->n_T;
        if (tx != ty) return tx < ty;
        if (a.wlo != b.wlo) return a.wlo < b.wlo;
        return a.whi < b.whi;
      });
    int n_out = 0;
    for (const int j : order) {
      const size_t l = (size_t)q * n_sub + j;
      const LineSpec& ls = spec[l];
      const int ih = pts[j] / sc->n_T, it = pts[j] % sc->n_T;
      Line& L = p->lines[l];
      L.out0 = out + n_out;
      L.stride = 1;
      L.count = golden ? 1 : (int32_t)ls.grid_idx.size();
      L.group = q;
      L.pad = 0;
      L.delta0 = g.delta_off + n_out;
      L.ht = g.ht_off + n_out;
      if (golden) {
        p->delta.push_back(sc->lo);
        p->ht.push_back(HT{sc->h[ih], sc->T[it], h_local[ih], 0});
        GoldenState& gs = p->golden0[l];
        gs.lo = ls.wlo;
        gs.hi = ls.whi;
        gs.x0 = sc->lo;
        gs.wide = 1e-2 * (sc->hi - sc->lo);  // basins judged on the whole range, as in the full scan
      } else {
        for (int gi : ls.grid_idx) {
          p->delta.push_back(grid[gi]);
          p->ht.push_back(HT{sc->h[ih], sc->T[it], h_local[ih], 0});
        }
      }
      n_out += L.count;
    }
    g.n_out = n_out;
    g.n_delta = n_out;
    g.n_ht = n_out;
    g.n_hblk = 1;
    g.n_batches = (n_out + 31) / 32;
    p->groups.push_back(g);
    out += n_out;
  }
  for (int q = 0; q < sc->n_q; ++q)
    for (int j = 0; j < n_sub; ++j)
      if (spec[(size_t)q * n_sub + j].alias) {
        Line L = p->lines[(size_t)q0 * n_sub + j];
        L.count = 1;
        L.pad = kLineAlias;
        p->lines[(size_t)q * n_sub + j] = L;
      }
  p->n_out = out;
}

struct PassResult {
  std::vector<ffe_result> res;  // [n_q][pts.size()]
  std::vector<int8_t> labels;
  std::vector<int32_t> best;
  std::vector<double> omega;    // grid search: every output
};

ffe_status run_explicit(ffe_context* ctx, const ffe_scan* sc, int q0, const std::vector<int>& pts, int golden_steps,
                        const std::vector<double>& grid, const std::vector<LineSpec>& spec, cudaStream_t s,
                        PassResult& out, double* k_evals) {
  ffe_plan* p = plan_new(ctx, golden_steps > 0 ? kPlanScanGolden : kPlanScanGrid);
  fill_explicit(p, sc, q0, pts, golden_steps, grid, spec);
  ffe_status st = plan_configure(ctx, p);
  if (st == FFE_OK) st = plan_finish(ctx, p, false);
  if (st == FFE_OK) st = plan_run(ctx, p, s);
  const int n_sub = (int)pts.size();
  out.res.assign((size_t)sc->n_q * n_sub, ffe_result{});
  out.labels.assign(n_sub, 0);
  out.best.assign(n_sub, -1);
  if (st == FFE_OK) st = fetch_scan(ctx, p, out.res.data(), out.labels.data(), out.best.data(), s);
  if (st == FFE_OK && golden_steps == 0) {
    out.omega.resize(p->n_out);
    cudaError_t e = cudaMemcpyAsync(out.omega.data(), p->d_omega, p->n_out * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(ctx, e, "fetch omega");
  }
  if (k_evals) *k_evals += plan_k_evals(p);
  plan_free(p);
  return st;
}

}  // namespace
}  // namespace ffe

using namespace ffe;

extern "C" ffe_status ffe_surrogate_scan(ffe_context* ctx, ffe_surrogate* sur, const ffe_scan* sc,
                                         const ffe_guide* guide, ffe_result* per_point, int8_t* labels_out,
                                         int32_t* best_q_out, ffe_guide_stats* stats, void* stream) {
  if (!ctx || !sur || !sc || !guide) return FFE_EINVAL;
  const bool golden = sc->search == FFE_SEARCH_GOLDEN;
  if (sc->search != FFE_SEARCH_GRID && !golden) return set_err(ctx, "unknown search kind"), FFE_EINVAL;
  if (sc->N < 2 || sc->N > 8192 || sc->N % 2 || sc->n_q < 1 || sc->n_h < 1 || sc->n_T < 1 || !(sc->lo == 0.0) ||
      !(sc->hi > sc->lo) || (!golden && (sc->n < 2 || sc->n > 65536)) || (golden && (sc->n < 1 || sc->n > 200)))
    return set_err(ctx, "guided scan: invalid scan"), FFE_EINVAL;
  // G: points of the prediction grid (the search grid itself for a grid scan)
  const int G = golden ? kGuideGrid : sc->n;
  if (guide->window < 2 || guide->window > G || guide->q_keep < 0)
    return set_err(ctx, "guided scan: window in [2, grid points], q_keep >= 0"), FFE_EINVAL;
  int q0 = -1;
  for (int q = 0; q < sc->n_q; ++q) {
    if (!std::isfinite(sc->qx[q]) || !std::isfinite(sc->qy[q])) return set_err(ctx, "q not finite"), FFE_EINVAL;
    if (q0 < 0 && sc->qx[q] == 0.0 && sc->qy[q] == 0.0) q0 = q;
  }
  if (q0 < 0) return set_err(ctx, "the q list must contain Q = (0, 0)"), FFE_EINVAL;
  for (int i = 0; i < sc->n_T; ++i)
    if (!(sc->T[i] > 0.0)) return set_err(ctx, "T must be > 0"), FFE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int n_pts = sc->n_h * sc->n_T, n_lines = sc->n_q * n_pts;
  std::vector<double> grid(G);
  linspace(sc->lo, sc->hi, G, grid.data());

  // 1. predictions of every line on the grid, and their argmin
  std::vector<float4> qht(n_lines);
  for (int q = 0; q < sc->n_q; ++q)
    for (int pt = 0; pt < n_pts; ++pt)
      qht[(size_t)q * n_pts + pt] = make_float4((float)sc->qx[q], (float)sc->h[pt / sc->n_T],
                                                (float)sc->T[pt % sc->n_T], 0.0f);
  std::vector<float> gridf(grid.begin(), grid.end());
  float4 *d_qht = nullptr, *d_x = nullptr;
  float *d_grid = nullptr, *d_y = nullptr, *d_ymin = nullptr;
  int32_t* d_idx = nullptr;
  const int64_t n_pred = (int64_t)n_lines * G;
  cudaError_t e = cudaMalloc(&d_qht, n_lines * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc(&d_grid, G * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_x, n_pred * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc(&d_y, n_pred * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_ymin, n_lines * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_idx, n_lines * sizeof(int32_t));
  std::vector<int32_t> idx(n_lines);
  std::vector<float> ymin(n_lines);
  ffe_status st = FFE_OK;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_qht, qht.data(), n_lines * sizeof(float4), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_grid, gridf.data(), G * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    guide_inputs_kernel<<<(int)((n_pred + 255) / 256), 256, 0, s>>>(d_qht, d_grid, n_lines, G, d_x);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) st = surrogate_infer_device(sur, reinterpret_cast<const float*>(d_x), n_pred, d_y, s);
  if (e == cudaSuccess && st == FFE_OK) {
    guide_argmin_kernel<<<(int)(((int64_t)n_lines * 32 + 255) / 256), 256, 0, s>>>(d_y, n_lines, G, d_idx, d_ymin);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && st == FFE_OK) e = cudaMemcpyAsync(idx.data(), d_idx, n_lines * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && st == FFE_OK) e = cudaMemcpyAsync(ymin.data(), d_ymin, n_lines * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && st == FFE_OK) e = cudaStreamSynchronize(s);

  // 2. the exact normal state Omega(q, Delta = lo) of the lines.  The
  // surrogate predicts condensation energies, each relative to its own line's
  // normal state, while the labels compare Omega across q, and on a finite
  // lattice the normal states of different q differ; the pruning orders the
  // q by exact normal state + predicted condensation energy.  With a margin,
  // the normal states of every q are first evaluated at a sample of at most
  // 64 (h, T) points spread over the scan; where they differ from those of
  // q = 0 by more than a tenth of the margin somewhere in the sample, every
  // line's normal state is evaluated, otherwise (large lattices, where they
  // agree) the predictions alone order the q.  Without a margin the
  // predictions alone order them.
  double k_evals = 0.0;
  std::vector<double> anchor(n_lines, 0.0);  // per site, relative to q = 0 at the same (h, T)
  const double n2 = (double)sc->N * (double)sc->N;
  bool anchored = false;
  auto normal_states = [&](const std::vector<int>& pts, std::vector<double>& rel) -> ffe_status {
    std::vector<LineSpec> spec0((size_t)sc->n_q * pts.size());
    for (LineSpec& ls : spec0) ls.grid_idx = {0};
    PassResult r0;
    ffe_status st0 = run_explicit(ctx, sc, q0, pts, 0, grid, spec0, s, r0, &k_evals);
    if (st0 != FFE_OK) return st0;
    rel.assign(spec0.size(), 0.0);
    for (int q = 0; q < sc->n_q; ++q)
      for (size_t j = 0; j < pts.size(); ++j)
        rel[(size_t)q * pts.size() + j] =
            (r0.res[(size_t)q * pts.size() + j].omega_lo - r0.res[(size_t)q0 * pts.size() + j].omega_lo) / n2;
    return FFE_OK;
  };
  if (e == cudaSuccess && st == FFE_OK && guide->margin > 0.0 && sc->n_q > 1) {
    std::vector<int> sample;
    const int stride = std::max(1, (n_pts + 63) / 64);
    for (int pt = 0; pt < n_pts; pt += stride) sample.push_back(pt);
    std::vector<double> rel;
    st = normal_states(sample, rel);
    double spread = 0.0;
    for (double v : rel) spread = std::max(spread, std::fabs(v));
    if (st == FFE_OK && spread > 0.1 * guide->margin) {
      std::vector<int> all_pts(n_pts);
      std::iota(all_pts.begin(), all_pts.end(), 0);
      if ((int)sample.size() == n_pts) {
        anchor = rel;
      } else {
        st = normal_states(all_pts, rel);
        if (st == FFE_OK) anchor = rel;
      }
      anchored = st == FFE_OK;
    }
  }

  // 3. which lines to verify, and on which window
  const int w = guide->window;
  std::vector<char> kept(n_lines, 0);
  const float ys = surrogate_y_scale(sur);
  std::vector<int> wstart(n_lines, 0);
  std::vector<int32_t> kept_rows;
  std::vector<int64_t> row_of(n_lines, -1);
  std::vector<float> ypred;  // prediction rows of the kept lines
  if (e == cudaSuccess && st == FFE_OK) {
    std::vector<int> order;
    // predicted minimum per site: exact normal state + predicted condensation
    auto pred_min = [&](int q, int pt) {
      const size_t l = (size_t)q * n_pts + pt;
      return anchor[l] + (double)ymin[l] * ys;
    };
    for (int pt = 0; pt < n_pts; ++pt) {
      order.clear();
      for (int q = 0; q < sc->n_q; ++q)
        if (q != q0) order.push_back(q);
      std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return pred_min(a, pt) < pred_min(b, pt); });
      kept[(size_t)q0 * n_pts + pt] = 1;
      for (int k = 0; k < (int)order.size() && k < guide->q_keep; ++k) kept[(size_t)order[k] * n_pts + pt] = 1;
      // beyond q_keep: every q predicted to condense by more than the margin
      // whose predicted minimum is within the margin of the lowest one (q = 0
      // included): the surrogate cannot order them; and every q whose exact
      // normal state lies more than the margin below that of q = 0: any
      // condensation, even one below the surrogate's resolution, makes it the
      // winner (on a finite lattice the normal states of different q differ)
      if (guide->margin > 0.0 && !order.empty()) {
        const double best = std::min(pred_min(order[0], pt), pred_min(q0, pt));
        for (int k = guide->q_keep; k < (int)order.size(); ++k) {
          const size_t l = (size_t)order[k] * n_pts + pt;
          const bool condenses = (double)ymin[l] * ys < -guide->margin && pred_min(order[k], pt) <= best + guide->margin;
          if (condenses || (anchored && anchor[l] < -guide->margin)) kept[l] = 1;
        }
      }
    }
    for (int l = 0; l < n_lines; ++l)
      if (kept[l]) {
        row_of[l] = (int64_t)kept_rows.size();
        kept_rows.push_back(l);
      }
    // the kept lines' prediction rows, gathered on the device into d_x's storage
    const int n_rows = (int)kept_rows.size();
    int32_t* d_rows = reinterpret_cast<int32_t*>(d_qht);  // n_rows <= n_lines
    float* d_rowsy = reinterpret_cast<float*>(d_x);       // n_rows * G <= n_pred
    ypred.resize((size_t)n_rows * G);
    e = cudaMemcpyAsync(d_rows, kept_rows.data(), n_rows * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      guide_gather_kernel<<<(int)(((int64_t)n_rows * G + 255) / 256), 256, 0, s>>>(d_y, d_rows, n_rows, G, d_rowsy);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ypred.data(), d_rowsy, ypred.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  for (void* ptr : {(void*)d_qht, (void*)d_grid, (void*)d_x, (void*)d_y, (void*)d_ymin, (void*)d_idx})
    if (ptr) cudaFree(ptr);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "surrogate predictions");
  if (st != FFE_OK) return st;

  // golden: a window of w grid points spans (w - 1)/(G - 1) of the range;
  // that many fewer reductions reach the full scan's final bracket width
  int steps_w = 0;
  if (golden) {
    const double ratio = (double)(G - 1) / (double)(w - 1);
    steps_w = std::max(1, (int)std::ceil(sc->n - std::log(ratio) / std::log(1.0 / kGuidePhi) - 1e-9));
  }
  std::vector<LineSpec> spec(n_lines);
  std::vector<char> redo(n_lines, 0);  // searched over the whole range
  // (ys: the surrogate's y scale, |t1| per site per unit of y)
  for (int l = 0; l < n_lines; ++l) {
    if (!kept[l]) {
      spec[l].grid_idx = {0};
      spec[l].alias = true;
      continue;
    }
    const int i0 = std::max(0, std::min(G - w, idx[l] - w / 2));
    wstart[l] = i0;
    if (golden) {
      spec[l].wlo = grid[i0];
      spec[l].whi = grid[i0 + w - 1];
    } else {
      if (i0 > 0) spec[l].grid_idx.push_back(0);
      for (int i = i0; i < i0 + w; ++i) spec[l].grid_idx.push_back(i);
    }
    // a predicted normal state with a second predicted basin close to it
    if (i0 == 0 && guide->margin > 0.0) {
      const float* yrow = ypred.data() + (size_t)row_of[l] * G;
      float y2 = INFINITY;
      for (int j = w; j < G; ++j) y2 = std::min(y2, yrow[j]);
      if ((double)y2 * ys < guide->margin) redo[l] = 1;
    }
  }
  int64_t ambiguous = 0;
  for (int l = 0; l < n_lines; ++l) ambiguous += redo[l];

  // points with a line searched over the whole range go to the second pass
  std::vector<int> pos_in(n_pts, -1), pts1, again;
  auto point_has_redo = [&](int pt) {
    for (int q = 0; q < sc->n_q; ++q)
      if (redo[(size_t)q * n_pts + pt]) return true;
    return false;
  };
  for (int pt = 0; pt < n_pts; ++pt)
    if (!point_has_redo(pt)) {
      pos_in[pt] = (int)pts1.size();
      pts1.push_back(pt);
    }
  const int n1 = (int)pts1.size();
  // whole: every verified line of the points over the whole range (the
  // second pass; a window left there would get no edge check)
  auto sub_spec = [&](const std::vector<int>& pts, bool whole) {
    std::vector<LineSpec> out((size_t)sc->n_q * pts.size());
    for (int q = 0; q < sc->n_q; ++q)
      for (size_t j = 0; j < pts.size(); ++j) {
        const size_t l = (size_t)q * n_pts + pts[j];
        LineSpec ls = spec[l];
        if (whole && !ls.alias) {
          if (golden) {
            ls.wlo = sc->lo;
            ls.whi = sc->hi;
          } else {
            ls.grid_idx.resize(G);
            std::iota(ls.grid_idx.begin(), ls.grid_idx.end(), 0);
          }
        }
        out[(size_t)q * pts.size() + j] = ls;
      }
    return out;
  };

  // 4. exact verification of the windows
  PassResult r1;
  std::vector<LineSpec> spec1;
  if (n1 > 0) {
    spec1 = sub_spec(pts1, false);
    st = run_explicit(ctx, sc, q0, pts1, steps_w, grid, spec1, s, r1, &k_evals);
    if (st != FFE_OK) return st;
  }

  // 5. surrogate error at the verified points; lines whose minimum sits on an inner window edge
  double se = 0.0;
  int64_t n_se = 0, fallbacks = 0, n_kept = 0;
  std::vector<int64_t> off((size_t)sc->n_q * n1 + 1, 0);
  for (size_t m = 0; m < (size_t)sc->n_q * n1; ++m)
    off[m + 1] = off[m] + (spec1[m].alias || golden ? 0 : (int64_t)spec1[m].grid_idx.size());
  for (int l = 0; l < n_lines; ++l) n_kept += kept[l];
  for (int q = 0; q < sc->n_q; ++q)
    for (int j = 0; j < n1; ++j) {
      const size_t l = (size_t)q * n_pts + pts1[j], m = (size_t)q * n1 + j;
      if (!kept[l]) continue;
      const float* yrow = ypred.data() + (size_t)row_of[l] * G;
      bool lower_edge = false, upper_edge = false;
      if (golden) {
        // prediction at Delta*: linear interpolation on the prediction grid
        const ffe_result& r = r1.res[m];
        const double u = (r.delta_star - sc->lo) / (sc->hi - sc->lo) * (G - 1);
        const int i = std::max(0, std::min(G - 2, (int)std::floor(u)));
        const double t = std::min(1.0, std::max(0.0, u - i));
        const double pred = ((1.0 - t) * yrow[i] + t * yrow[i + 1]) * ys;
        const double exact = (r.omega_star - r.omega_lo) / n2;
        se += (exact - pred) * (exact - pred);
        ++n_se;
        lower_edge = (r.flags & kFlagBracketLo) != 0;
        upper_edge = (r.flags & FFE_FLAG_EDGE) && spec[l].whi < sc->hi;
      } else {
        const std::vector<int>& gi = spec[l].grid_idx;
        const double om0 = r1.omega[off[m]];
        int wbest = -1;  // position of the lowest value among the window points
        for (size_t k = (wstart[l] > 0 ? 1 : 0); k < gi.size(); ++k) {
          const double om = r1.omega[off[m] + k];
          const double exact = (om - om0) / n2;
          const double pred = (double)yrow[gi[k]] * ys;
          se += (exact - pred) * (exact - pred);
          ++n_se;
          if (wbest < 0 || om < r1.omega[off[m] + wbest]) wbest = (int)k;
        }
        const int lo_pos = wstart[l] > 0 ? 1 : 0;
        const int hi_pos = (int)gi.size() - 1;
        lower_edge = wbest == lo_pos && gi[lo_pos] > 0;
        upper_edge = wbest == hi_pos && gi[hi_pos] < G - 1;
      }
      if (lower_edge || upper_edge) {
        redo[l] = 1;
        ++fallbacks;
      }
    }

  // 6. the second pass: every point with a line to search over the whole range
  // (an ambiguous line, or one whose minimum sat on an inner window edge) has
  // all its verified lines searched over the whole range
  std::vector<int> pos_in2(n_pts, -1);
  for (int pt = 0; pt < n_pts; ++pt)
    if (point_has_redo(pt)) {
      pos_in2[pt] = (int)again.size();
      again.push_back(pt);
    }
  const int n2p = (int)again.size();
  PassResult r2;
  std::vector<LineSpec> spec2;
  if (n2p > 0) {
    spec2 = sub_spec(again, true);
    st = run_explicit(ctx, sc, q0, again, golden ? sc->n : 0, grid, spec2, s, r2, &k_evals);
    if (st != FFE_OK) return st;
  }

  // 7. results: per line from the pass that scanned its point last; grid indices
  for (int l = 0; l < n_lines; ++l) {
    const int q = l / n_pts, pt = l % n_pts;
    const bool second = pos_in2[pt] >= 0;
    const int j = second ? pos_in2[pt] : pos_in[pt];
    const int nsub = second ? n2p : n1;
    const size_t m = (size_t)q * nsub + j;
    const LineSpec& ls = second ? spec2[m] : spec1[m];
    const PassResult& pr = second ? r2 : r1;
    ffe_result r = pr.res[m];
    if (!kept[l]) {  // the q = 0 line's reference value
      const ffe_result& rn = pr.res[(size_t)q0 * nsub + j];
      r.delta_star = sc->lo;
      r.omega_star = rn.omega_lo;
      r.omega_lo = rn.omega_lo;
      r.err_bound = 0.0;
      r.idx_star = golden ? -1 : 0;
      r.flags = FFE_FLAG_LOWER | FFE_FLAG_PRUNED;
    } else if (golden) {
      const bool at_hi = (r.flags & FFE_FLAG_EDGE) && ls.whi == sc->hi;
      r.flags &= ~(FFE_FLAG_EDGE | kFlagBracketLo);
      if (at_hi) r.flags |= FFE_FLAG_EDGE;
    } else {
      const int loc = r.idx_star;
      r.idx_star = (loc >= 0 && loc < (int)ls.grid_idx.size()) ? ls.grid_idx[loc] : -1;
      r.flags &= ~(FFE_FLAG_EDGE | FFE_FLAG_LOWER);
      if (r.idx_star == 0) r.flags |= FFE_FLAG_LOWER;
      if (r.idx_star == G - 1) r.flags |= FFE_FLAG_EDGE;
    }
    if (per_point) per_point[l] = r;
  }
  for (int pt = 0; pt < n_pts; ++pt) {
    const bool second = pos_in2[pt] >= 0;
    if (labels_out) labels_out[pt] = second ? r2.labels[pos_in2[pt]] : r1.labels[pos_in[pt]];
    if (best_q_out) best_q_out[pt] = second ? r2.best[pos_in2[pt]] : r1.best[pos_in[pt]];
  }
  if (stats) {
    std::memset(stats, 0, sizeof *stats);
    stats->k_evals = k_evals;
    stats->k_evals_full = n2 * (double)n_lines * (golden ? 3.0 + sc->n : (double)sc->n);
    stats->lines_kept = n_kept;
    stats->lines_pruned = n_lines - n_kept;
    stats->fallbacks = fallbacks + ambiguous;
    stats->rms_error = n_se > 0 ? std::sqrt(se / (double)n_se) : 0.0;
    stats->mlp_flops = 2.0 * (double)n_pred * (4.0 * 128 + 2 * 128.0 * 128 + 128.0);
  }
  return FFE_OK;
}
