// guide.cu -- phase scan guided by the learned surrogate.
//
// A grid scan (Alg. 1) evaluates every (q, h, T) line on the whole Delta
// grid.  Guided, the surrogate first predicts the condensation energy of
// every line on the whole grid (tensor-core inference); per (h, T) only
// q = 0 and the q_keep lines with the lowest predicted minimum are verified,
// each on a window of `window` grid points around its predicted minimum plus
// Delta = 0, by the exact k-sum (same kernels, same FP64 re-evaluation of
// near ties, same label passes as the full scan).  A line whose verified
// minimum sits on an inner edge of its window is re-run on the whole grid.
// The exact values on the window points also measure the surrogate's error.
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

namespace {

struct LineSpec {
  std::vector<int> grid_idx;  // grid index of each output, grid_idx[0] == 0 (Delta = 0)
  bool alias = false;         // not evaluated: reads the q = 0 line's Delta = 0 output
};

// A scan-shaped plan whose lines carry explicit grid-index lists: one LIST
// group per q, lines q-major (the label passes expect that order).  A group's
// h list holds only the h values of its evaluated lines.  An alias line is a
// one-point line on the q = 0 line's Delta = 0 output: its minimum is its
// lower end, so it never competes for a label and costs no k-sum work.
void fill_explicit(ffe_plan* p, const ffe_scan* sc, int q0, const std::vector<double>& grid,
                   const std::vector<LineSpec>& spec) {
  const int n_pts = sc->n_h * sc->n_T;
  p->layout = kLayoutList;
  p->n_q = sc->n_q;
  p->n_pts = n_pts;
  p->q_is_zero.assign(sc->n_q, 0);
  p->lines.assign((size_t)sc->n_q * n_pts, Line{});
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
    for (int pt = 0; pt < n_pts; ++pt) {
      const int ih = pt / sc->n_T;
      if (!spec[(size_t)q * n_pts + pt].alias && h_local[ih] < 0) h_local[ih] = 0;
    }
    for (int ih = 0; ih < sc->n_h; ++ih)
      if (h_local[ih] == 0) {
        h_local[ih] = n_hq++;
        p->hlist.push_back(sc->h[ih]);
      }
    g.n_h = n_hq;
    int n_out = 0;
    for (int pt = 0; pt < n_pts; ++pt) {
      const LineSpec& ls = spec[(size_t)q * n_pts + pt];
      if (ls.alias) continue;
      const int ih = pt / sc->n_T, it = pt % sc->n_T;
      Line& L = p->lines[(size_t)q * n_pts + pt];
      L.out0 = out + n_out;
      L.stride = 1;
      L.count = (int32_t)ls.grid_idx.size();
      L.group = q;
      L.pad = 0;
      L.delta0 = g.delta_off + n_out;
      L.ht = g.ht_off + n_out;
      for (int gi : ls.grid_idx) {
        p->delta.push_back(grid[gi]);
        p->ht.push_back(HT{sc->h[ih], sc->T[it], h_local[ih], 0});
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
    for (int pt = 0; pt < n_pts; ++pt)
      if (spec[(size_t)q * n_pts + pt].alias) {
        Line L = p->lines[(size_t)q0 * n_pts + pt];
        L.count = 1;
        p->lines[(size_t)q * n_pts + pt] = L;
      }
  p->n_out = out;
}

ffe_status run_explicit(ffe_context* ctx, const ffe_scan* sc, int q0, const std::vector<double>& grid,
                        const std::vector<LineSpec>& spec, cudaStream_t s, std::vector<ffe_result>& res,
                        std::vector<int8_t>& labels, std::vector<int32_t>& best, std::vector<double>* omega,
                        double* k_evals) {
  ffe_plan* p = plan_new(ctx, kPlanScanGrid);
  fill_explicit(p, sc, q0, grid, spec);
  ffe_status st = plan_configure(ctx, p);
  if (st == FFE_OK) st = plan_finish(ctx, p, false);
  if (st == FFE_OK) st = plan_run(ctx, p, s);
  const int n_pts = sc->n_h * sc->n_T;
  res.assign((size_t)sc->n_q * n_pts, ffe_result{});
  labels.assign(n_pts, 0);
  best.assign(n_pts, -1);
  if (st == FFE_OK) st = fetch_scan(ctx, p, res.data(), labels.data(), best.data(), s);
  if (st == FFE_OK && omega) {
    omega->resize(p->n_out);
    cudaError_t e = cudaMemcpyAsync(omega->data(), p->d_omega, p->n_out * sizeof(double), cudaMemcpyDeviceToHost, s);
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
  if (sc->search != FFE_SEARCH_GRID) return set_err(ctx, "guided scans use the grid search"), FFE_EINVAL;
  if (sc->N < 2 || sc->N > 8192 || sc->N % 2 || sc->n_q < 1 || sc->n_h < 1 || sc->n_T < 1 || sc->n < 2 ||
      sc->n > 65536 || !(sc->lo == 0.0) || !(sc->hi > sc->lo))
    return set_err(ctx, "guided scan: invalid scan"), FFE_EINVAL;
  if (guide->window < 2 || guide->window > sc->n || guide->q_keep < 0)
    return set_err(ctx, "guided scan: window in [2, n], q_keep >= 0"), FFE_EINVAL;
  int q0 = -1;
  for (int q = 0; q < sc->n_q; ++q) {
    if (!std::isfinite(sc->qx[q]) || !std::isfinite(sc->qy[q])) return set_err(ctx, "q not finite"), FFE_EINVAL;
    if (q0 < 0 && sc->qx[q] == 0.0 && sc->qy[q] == 0.0) q0 = q;
  }
  if (q0 < 0) return set_err(ctx, "the q list must contain Q = (0, 0)"), FFE_EINVAL;
  for (int i = 0; i < sc->n_T; ++i)
    if (!(sc->T[i] > 0.0)) return set_err(ctx, "T must be > 0"), FFE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = sc->n, n_pts = sc->n_h * sc->n_T, n_lines = sc->n_q * n_pts;
  std::vector<double> grid(n);
  linspace(sc->lo, sc->hi, n, grid.data());

  // 1. predictions of every line on the whole grid, and their argmin
  std::vector<float4> qht(n_lines);
  for (int q = 0; q < sc->n_q; ++q)
    for (int pt = 0; pt < n_pts; ++pt)
      qht[(size_t)q * n_pts + pt] = make_float4((float)sc->qx[q], (float)sc->h[pt / sc->n_T],
                                                (float)sc->T[pt % sc->n_T], 0.0f);
  std::vector<float> gridf(grid.begin(), grid.end());
  float4 *d_qht = nullptr, *d_x = nullptr;
  float *d_grid = nullptr, *d_y = nullptr, *d_ymin = nullptr;
  int32_t* d_idx = nullptr;
  const int64_t n_pred = (int64_t)n_lines * n;
  cudaError_t e = cudaMalloc(&d_qht, n_lines * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc(&d_grid, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_x, n_pred * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc(&d_y, n_pred * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_ymin, n_lines * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_idx, n_lines * sizeof(int32_t));
  std::vector<int32_t> idx(n_lines);
  std::vector<float> ymin(n_lines), ypred(n_pred);
  ffe_status st = FFE_OK;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_qht, qht.data(), n_lines * sizeof(float4), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_grid, gridf.data(), n * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    guide_inputs_kernel<<<(int)((n_pred + 255) / 256), 256, 0, s>>>(d_qht, d_grid, n_lines, n, d_x);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) st = surrogate_infer_device(sur, reinterpret_cast<const float*>(d_x), n_pred, d_y, s);
  if (e == cudaSuccess && st == FFE_OK) {
    guide_argmin_kernel<<<(int)(((int64_t)n_lines * 32 + 255) / 256), 256, 0, s>>>(d_y, n_lines, n, d_idx, d_ymin);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && st == FFE_OK) e = cudaMemcpyAsync(idx.data(), d_idx, n_lines * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && st == FFE_OK) e = cudaMemcpyAsync(ymin.data(), d_ymin, n_lines * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && st == FFE_OK) e = cudaMemcpyAsync(ypred.data(), d_y, n_pred * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && st == FFE_OK) e = cudaStreamSynchronize(s);
  for (void* ptr : {(void*)d_qht, (void*)d_grid, (void*)d_x, (void*)d_y, (void*)d_ymin, (void*)d_idx})
    if (ptr) cudaFree(ptr);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "surrogate predictions");
  if (st != FFE_OK) return st;

  // 2. which lines to verify, and on which window
  const int w = guide->window;
  std::vector<char> kept(n_lines, 0);
  std::vector<int> wstart(n_lines, 0);
  for (int pt = 0; pt < n_pts; ++pt) {
    std::vector<int> order;
    for (int q = 0; q < sc->n_q; ++q)
      if (q != q0) order.push_back(q);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return ymin[(size_t)a * n_pts + pt] < ymin[(size_t)b * n_pts + pt];
    });
    kept[(size_t)q0 * n_pts + pt] = 1;
    for (int k = 0; k < (int)order.size() && k < guide->q_keep; ++k) kept[(size_t)order[k] * n_pts + pt] = 1;
  }
  std::vector<LineSpec> spec(n_lines);
  for (int l = 0; l < n_lines; ++l) {
    if (!kept[l]) {
      spec[l].grid_idx = {0};
      spec[l].alias = true;
      continue;
    }
    const int i0 = std::max(0, std::min(n - w, idx[l] - w / 2));
    wstart[l] = i0;
    if (i0 > 0) spec[l].grid_idx.push_back(0);
    for (int i = i0; i < i0 + w; ++i) spec[l].grid_idx.push_back(i);
  }

  // 3. exact verification of the windows
  double k_evals = 0.0;
  std::vector<ffe_result> res;
  std::vector<int8_t> labels;
  std::vector<int32_t> best;
  std::vector<double> omega;
  st = run_explicit(ctx, sc, q0, grid, spec, s, res, labels, best, &omega, &k_evals);
  if (st != FFE_OK) return st;

  // 4. surrogate error on the verified points; lines to re-run on the whole grid
  const double n2 = (double)sc->N * (double)sc->N;
  const float ys = surrogate_y_scale(sur);
  double se = 0.0;
  int64_t n_se = 0, fallbacks = 0, n_kept = 0;
  std::vector<int64_t> off(n_lines + 1, 0);
  for (int l = 0; l < n_lines; ++l) off[l + 1] = off[l] + (spec[l].alias ? 0 : (int64_t)spec[l].grid_idx.size());
  std::vector<char> redo(n_lines, 0);
  for (int l = 0; l < n_lines; ++l) {
    if (!kept[l]) continue;
    ++n_kept;
    const std::vector<int>& gi = spec[l].grid_idx;
    const double om0 = omega[off[l]];
    int wbest = -1;  // position of the lowest value among the window points
    for (size_t j = (wstart[l] > 0 ? 1 : 0); j < gi.size(); ++j) {
      const double om = omega[off[l] + j];
      const double exact = (om - om0) / n2;
      const double pred = (double)ypred[(size_t)l * n + gi[j]] * ys;
      se += (exact - pred) * (exact - pred);
      ++n_se;
      if (wbest < 0 || om < omega[off[l] + wbest]) wbest = (int)j;
    }
    const int lo_pos = wstart[l] > 0 ? 1 : 0;
    const int hi_pos = (int)gi.size() - 1;
    const bool lower_edge = wbest == lo_pos && gi[lo_pos] > 0;
    const bool upper_edge = wbest == hi_pos && gi[hi_pos] < n - 1;
    if (lower_edge || upper_edge) {
      redo[l] = 1;
      ++fallbacks;
    }
  }

  // 5. the whole grid for those lines (the others keep Delta = 0 and their minimum)
  if (fallbacks > 0) {
    std::vector<LineSpec> spec2(n_lines);
    for (int l = 0; l < n_lines; ++l) {
      if (redo[l]) {
        spec2[l].grid_idx.resize(n);
        std::iota(spec2[l].grid_idx.begin(), spec2[l].grid_idx.end(), 0);
      } else {
        spec2[l].grid_idx = {0};
        spec2[l].alias = !kept[l];
        const int i = res[l].idx_star;
        if (kept[l] && i > 0) spec2[l].grid_idx.push_back(spec[l].grid_idx[i]);
      }
    }
    spec = spec2;
    st = run_explicit(ctx, sc, q0, grid, spec, s, res, labels, best, nullptr, &k_evals);
    if (st != FFE_OK) return st;
  }

  // 6. results in grid indices
  for (int l = 0; l < n_lines; ++l) {
    ffe_result r = res[l];
    const int loc = r.idx_star;
    r.idx_star = (loc >= 0 && loc < (int)spec[l].grid_idx.size()) ? spec[l].grid_idx[loc] : -1;
    r.flags &= ~(FFE_FLAG_EDGE | FFE_FLAG_LOWER);
    if (r.idx_star == 0) r.flags |= FFE_FLAG_LOWER;
    if (r.idx_star == n - 1) r.flags |= FFE_FLAG_EDGE;
    if (!kept[l]) r.flags |= FFE_FLAG_PRUNED;
    if (per_point) per_point[l] = r;
  }
  if (labels_out) std::memcpy(labels_out, labels.data(), n_pts);
  if (best_q_out) std::memcpy(best_q_out, best.data(), n_pts * sizeof(int32_t));
  if (stats) {
    std::memset(stats, 0, sizeof *stats);
    stats->k_evals = k_evals;
    stats->k_evals_full = n2 * (double)n_lines * (double)n;
    stats->lines_kept = n_kept;
    stats->lines_pruned = n_lines - n_kept;
    stats->fallbacks = fallbacks;
    stats->rms_error = n_se > 0 ? std::sqrt(se / (double)n_se) : 0.0;
    stats->mlp_flops = 2.0 * (double)n_pred * (4.0 * 128 + 2 * 128.0 * 128 + 128.0);
  }
  return FFE_OK;
}
