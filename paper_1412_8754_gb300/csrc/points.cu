// points.cu -- ffe_omega (independent points) and ffe_minimize (independent
// Delta searches, uneven lattices and grid lengths in one persistent launch).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "plan.h"

using namespace ffe;

namespace {

bool valid_N(int32_t N) { return N >= 2 && N <= 8192 && (N % 2) == 0; }

// Points sharing (N, Q) form one LIST group; outputs keep input order inside.
// bands > 0: every group once per band, restricted to it (outputs
// [b n, (b + 1) n) for band b, in the same order).
void fill_points(ffe_plan* p, const ffe_point* pts, int64_t n, int bands = 0) {
  p->layout = kLayoutList;
  std::map<std::tuple<int32_t, double, double>, std::vector<int64_t>> by_key;
  std::vector<std::tuple<int32_t, double, double>> keys;
  for (int64_t i = 0; i < n; ++i) {
    auto k = std::make_tuple(pts[i].N, pts[i].qx, pts[i].qy);
    auto it = by_key.find(k);
    if (it == by_key.end()) {
      keys.push_back(k);
      by_key[k].push_back(i);
    } else {
      it->second.push_back(i);
    }
  }
  int64_t out = 0, tab = 0;
  for (int pass = 0; pass < std::max(1, bands); ++pass)
  for (const auto& k : keys) {
    const std::vector<int64_t>& idx = by_key[k];
    GroupDesc g;
    std::memset(&g, 0, sizeof g);
    g.band_only = bands > 0 ? pass + 1 : 0;
    g.N = std::get<0>(k);
    g.layout = kLayoutList;
    g.n_out = (int32_t)idx.size();
    g.n_delta = g.n_out;
    g.n_ht = g.n_out;
    g.n_hblk = 1;
    g.n_batches = (g.n_out + 31) / 32;
    g.out_off = out;
    g.delta_off = (int64_t)p->delta.size();
    g.ht_off = (int64_t)p->ht.size();
    g.tab_off = tab;
    g.h_off = (int64_t)p->hlist.size();
    g.qx = std::get<1>(k);
    g.qy = std::get<2>(k);
    std::map<double, int> hmap;
    for (int64_t i : idx) {
      const double h = pts[i].h;
      auto it = hmap.find(h);
      int hi;
      if (it == hmap.end()) {
        hi = (int)hmap.size();
        hmap[h] = hi;
        p->hlist.push_back(h);
      } else {
        hi = it->second;
      }
      p->delta.push_back(pts[i].delta);
      p->ht.push_back(HT{h, pts[i].T, hi, 0});
      p->order.push_back(i);
    }
    g.n_h = (int32_t)hmap.size();
    p->groups.push_back(g);
    out += g.n_out;
    tab += 2 * (int64_t)g.N;
  }
  p->n_out = out;
}

// One LIST group per parameter point: outputs = its Delta grid.  bands > 0:
// every point once per band, restricted to it (lines [b n, (b + 1) n)).
void fill_min_grid(ffe_plan* p, const ffe_param* ps, int64_t n, int bands = 0) {
  p->layout = kLayoutList;
  int64_t out = 0, tab = 0;
  std::vector<double> grid;
  for (int64_t li = 0; li < std::max(1, bands) * n; ++li) {
    const int64_t i = li % n;
    const ffe_param& q = ps[i];
    GroupDesc g;
    std::memset(&g, 0, sizeof g);
    g.band_only = bands > 0 ? (int32_t)(li / n) + 1 : 0;
    g.N = q.N;
    g.layout = kLayoutList;
    g.n_out = q.n;
    g.n_delta = q.n;
    g.n_ht = q.n;
    g.n_hblk = 1;
    g.n_batches = (q.n + 31) / 32;
    g.n_h = 1;
    g.out_off = out;
    g.delta_off = (int64_t)p->delta.size();
    g.ht_off = (int64_t)p->ht.size();
    g.tab_off = tab;
    g.h_off = (int64_t)p->hlist.size();
    g.qx = q.qx;
    g.qy = q.qy;
    grid.resize(q.n);
    linspace(q.lo, q.hi, q.n, grid.data());
    p->delta.insert(p->delta.end(), grid.begin(), grid.end());
    for (int j = 0; j < q.n; ++j) p->ht.push_back(HT{q.h, q.T, 0, 0});
    p->hlist.push_back(q.h);
    Line L;
    L.out0 = out;
    L.stride = 1;
    L.count = q.n;
    L.group = (int32_t)li;
    L.pad = 0;
    L.delta0 = g.delta_off;
    L.ht = g.ht_off;
    p->lines.push_back(L);
    p->groups.push_back(g);
    out += q.n;
    tab += 2 * (int64_t)q.N;
  }
  p->n_out = out;
}

// Golden-section searches: parameter points sharing (N, Q) form one LIST
// group (their (h, T) and pending Delta are the outputs); one line per point,
// in input order.  bands > 0: every group once per band, restricted to it
// (lines [b n, (b + 1) n)).
void fill_min_golden(ffe_plan* p, const ffe_param* ps, int64_t n, int bands = 0) {
  p->layout = kLayoutList;
  int steps = 0;
  for (int64_t i = 0; i < n; ++i) steps = std::max(steps, ps[i].n);
  p->golden_steps = steps;
  std::map<std::tuple<int32_t, double, double>, std::vector<int64_t>> by_key;
  std::vector<std::tuple<int32_t, double, double>> keys;
  for (int64_t i = 0; i < n; ++i) {
    auto k = std::make_tuple(ps[i].N, ps[i].qx, ps[i].qy);
    if (by_key.find(k) == by_key.end()) keys.push_back(k);
    by_key[k].push_back(i);
  }
  const int passes = std::max(1, bands);
  p->lines.resize(n * passes);
  p->golden0.resize(n * passes);
  int64_t out = 0, tab = 0;
  for (size_t gp = 0; gp < keys.size() * passes; ++gp) {
    const size_t gi = gp % keys.size();
    const int pass = (int)(gp / keys.size());
    const std::vector<int64_t>& idx = by_key[keys[gi]];
    GroupDesc g;
    std::memset(&g, 0, sizeof g);
    g.band_only = bands > 0 ? pass + 1 : 0;
    g.N = std::get<0>(keys[gi]);
    g.layout = kLayoutList;
    g.n_out = (int32_t)idx.size();
    g.n_delta = g.n_out;
    g.n_ht = g.n_out;
    g.n_hblk = 1;
    g.n_batches = (g.n_out + 31) / 32;
    g.out_off = out;
    g.delta_off = (int64_t)p->delta.size();
    g.ht_off = (int64_t)p->ht.size();
    g.tab_off = tab;
    g.h_off = (int64_t)p->hlist.size();
    g.qx = std::get<1>(keys[gi]);
    g.qy = std::get<2>(keys[gi]);
    std::map<double, int> hmap;
    for (size_t j = 0; j < idx.size(); ++j) {
      const ffe_param& q = ps[idx[j]];
      auto it = hmap.find(q.h);
      int hi;
      if (it == hmap.end()) {
        hi = (int)hmap.size();
        hmap[q.h] = hi;
        p->hlist.push_back(q.h);
      } else {
        hi = it->second;
      }
      p->delta.push_back(q.lo);
      p->ht.push_back(HT{q.h, q.T, hi, 0});
      Line L;
      L.out0 = out + (int64_t)j;
      L.stride = 1;
      L.count = 1;
      L.group = (int32_t)gp;
      L.pad = 0;
      L.delta0 = g.delta_off + (int64_t)j;
      L.ht = g.ht_off + (int64_t)j;
      p->lines[pass * n + idx[j]] = L;
      GoldenState gs;
      std::memset(&gs, 0, sizeof gs);
      gs.lo = q.lo;
      gs.hi = q.hi;
      gs.x0 = q.lo;
      p->golden0[pass * n + idx[j]] = gs;
    }
    g.n_h = (int32_t)hmap.size();
    p->groups.push_back(g);
    out += g.n_out;
    tab += 2 * (int64_t)g.N;
  }
  p->n_out = out;
}


ffe_status check_params(ffe_context* ctx, int32_t search, const ffe_param* ps, int64_t n) {
  if (!ps || n < 1) return set_err(ctx, "empty or NULL parameter list"), FFE_EINVAL;
  if (search != FFE_SEARCH_GRID && search != FFE_SEARCH_GOLDEN)
    return set_err(ctx, "unknown search kind %d", search), FFE_EINVAL;
  int64_t total = 0;
  for (int64_t i = 0; i < n; ++i) {
    const ffe_param& q = ps[i];
    if (!valid_N(q.N)) return set_err(ctx, "param %lld: N=%d must be even in [2, 8192]", (long long)i, q.N), FFE_EINVAL;
    if (!(q.T > 0.0) || !std::isfinite(q.T) || !std::isfinite(q.qx) || !std::isfinite(q.qy) ||
        !std::isfinite(q.h) || !std::isfinite(q.lo) || !std::isfinite(q.hi) || q.lo > q.hi)
      return set_err(ctx, "param %lld: non-finite value, T <= 0 or lo > hi", (long long)i), FFE_EINVAL;
    if (search == FFE_SEARCH_GRID && (q.n < 1 || q.n > 65536))
      return set_err(ctx, "param %lld: grid points n=%d out of [1, 65536]", (long long)i, q.n), FFE_EINVAL;
    if (search == FFE_SEARCH_GOLDEN && (q.n < 1 || q.n > 200))
      return set_err(ctx, "param %lld: golden reductions n=%d out of [1, 200]", (long long)i, q.n), FFE_EINVAL;
    if (search == FFE_SEARCH_GOLDEN && q.n != ps[0].n)
      return set_err(ctx, "param %lld: golden searches of one call share n", (long long)i), FFE_EINVAL;
    total += q.n;
  }
  if (total > ((int64_t)1 << 31)) return set_err(ctx, "too many outputs"), FFE_EINVAL;
  return FFE_OK;
}

ffe_status build_min_plan(ffe_context* ctx, int32_t search, const ffe_param* ps, int64_t n, bool graph,
                          ffe_plan** out, int bands = 0) {
  ffe_plan* p = plan_new(ctx, search == FFE_SEARCH_GRID ? kPlanMinGrid : kPlanMinGolden);
  *out = p;
  if (search == FFE_SEARCH_GRID)
    fill_min_grid(p, ps, n, bands);
  else
    fill_min_golden(p, ps, n, bands);
  ffe_status st = plan_configure(ctx, p);
  if (st == FFE_OK) st = plan_finish(ctx, p, graph);
  return st;
}

ffe_status fetch_min(ffe_context* ctx, ffe_plan* p, ffe_result* out, double* omega_grid, double* err_grid,
                     cudaStream_t s) {
  ffe_status st = plan_check_status(ctx, p, s);
  if (st != FFE_OK) return st;
  std::vector<LineResult> lr(p->lines.size());
  cudaError_t e = cudaMemcpyAsync(lr.data(), p->d_lres, lr.size() * sizeof(LineResult), cudaMemcpyDeviceToHost, s);
  int32_t nreq = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nreq, p->d_counters + 3, sizeof nreq, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && omega_grid)
    e = cudaMemcpyAsync(omega_grid, p->d_omega, p->n_out * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && err_grid)
    e = cudaMemcpyAsync(err_grid, p->d_eb, p->n_out * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fetch results");
  p->last_rescored[0] = nreq;
  if (nreq > p->cap) {
    set_err(ctx, "FP64 re-evaluation requests (%d) exceeded capacity (%d)", nreq, p->cap);
    return FFE_EINTERNAL;
  }
  for (size_t i = 0; i < lr.size(); ++i) {
    out[i].delta_star = lr[i].delta_star;
    out[i].omega_star = lr[i].omega_star;
    out[i].omega_lo = lr[i].omega_lo;
    out[i].err_bound = lr[i].eb_star;
    out[i].idx_star = lr[i].idx_star;
    out[i].flags = lr[i].flags;
  }
  p->d2h_bytes = lr.size() * sizeof(LineResult) + (omega_grid ? p->n_out * 8 : 0) + (err_grid ? p->n_out * 8 : 0);
  return FFE_OK;
}

}  // namespace

extern "C" {

ffe_status ffe_omega(ffe_context* ctx, const ffe_point* pts, int64_t n, double* omega, double* omega_band,
                     void* stream) {
  if (!ctx) return FFE_EINVAL;
  if (!pts || !omega || n < 1) return set_err(ctx, "ffe_omega: empty or NULL arguments"), FFE_EINVAL;
  for (int64_t i = 0; i < n; ++i) {
    const ffe_point& q = pts[i];
    if (!valid_N(q.N)) return set_err(ctx, "point %lld: N=%d must be even in [2, 8192]", (long long)i, q.N), FFE_EINVAL;
    if (q.reserved != 0) return set_err(ctx, "point %lld: reserved must be 0", (long long)i), FFE_EINVAL;
    if (!(q.T > 0.0) || !std::isfinite(q.T) || !std::isfinite(q.qx) || !std::isfinite(q.qy) ||
        !std::isfinite(q.h) || !std::isfinite(q.delta))
      return set_err(ctx, "point %lld: non-finite value or T <= 0", (long long)i), FFE_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  ffe_plan* p = plan_new(ctx, kPlanOmega);
  const int nb = ctx->mp.nbands;
  fill_points(p, pts, n, omega_band ? nb : 0);
  ffe_status st = plan_configure(ctx, p);
  if (st == FFE_OK) st = plan_finish(ctx, p, false);
  if (st == FFE_OK) st = plan_run(ctx, p, s);
  if (st == FFE_OK) st = plan_check_status(ctx, p, s);
  if (st == FFE_OK) {
    std::vector<double> om(p->n_out);
    cudaError_t e = cudaMemcpyAsync(om.data(), p->d_omega, om.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = cuda_fail(ctx, e, "fetch omega");
    } else {
      if (omega_band) {  // outputs [b n, (b + 1) n): band b, same order
        for (int64_t o = 0; o < n; ++o) {
          const int64_t i = p->order[o];
          double tot = 0.0;
          for (int b = 0; b < nb; ++b) {
            omega_band[nb * i + b] = om[b * n + o];
            tot += om[b * n + o];
          }
          omega[i] = tot;
        }
      } else {
        for (int64_t o = 0; o < p->n_out; ++o) omega[p->order[o]] = om[o];
      }
    }
  }
  plan_free(p);
  return st;
}

ffe_status ffe_minimize_bands(ffe_context* ctx, int32_t search, const ffe_param* ps, int64_t n, ffe_result* out,
                              void* stream) {
  if (!ctx) return FFE_EINVAL;
  if (!out) return set_err(ctx, "ffe_minimize_bands: out is NULL"), FFE_EINVAL;
  ffe_status st = check_params(ctx, search, ps, n);
  if (st != FFE_OK) return st;
  if (n > ((int64_t)1 << 30)) return set_err(ctx, "too many parameter points"), FFE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  ffe_plan* p = nullptr;
  const int nb = ctx->mp.nbands;
  st = build_min_plan(ctx, search, ps, n, false, &p, nb);
  std::vector<ffe_result> lines(nb * n);
  if (st == FFE_OK) st = plan_run(ctx, p, s);
  if (st == FFE_OK) st = fetch_min(ctx, p, lines.data(), nullptr, nullptr, s);
  if (st == FFE_OK)
    for (int64_t i = 0; i < n; ++i)
      for (int b = 0; b < nb; ++b) out[nb * i + b] = lines[b * n + i];
  plan_free(p);
  return st;
}

ffe_status ffe_minimize(ffe_context* ctx, int32_t search, const ffe_param* ps, int64_t n, ffe_result* out,
                        double* omega_grid, double* err_grid, void* stream) {
  if (!ctx) return FFE_EINVAL;
  if (!out) return set_err(ctx, "ffe_minimize: out is NULL"), FFE_EINVAL;
  ffe_status st = check_params(ctx, search, ps, n);
  if (st != FFE_OK) return st;
  if (search == FFE_SEARCH_GOLDEN && (omega_grid || err_grid))
    return set_err(ctx, "omega_grid/err_grid apply to grid searches only"), FFE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  ffe_plan* p = nullptr;
  st = build_min_plan(ctx, search, ps, n, false, &p);
  if (st == FFE_OK) st = plan_run(ctx, p, s);
  if (st == FFE_OK) st = fetch_min(ctx, p, out, omega_grid, err_grid, s);
  plan_free(p);
  return st;
}

ffe_status ffe_minimize_async(ffe_context* ctx, int32_t search, const ffe_param* ps, int64_t n, ffe_result* out,
                              double* omega_grid, void* stream) {
  if (!ctx) return FFE_EINVAL;
  if (!out) return set_err(ctx, "ffe_minimize_async: out is NULL"), FFE_EINVAL;
  ffe_status st = check_params(ctx, search, ps, n);
  if (st != FFE_OK) return st;
  if (search == FFE_SEARCH_GOLDEN && omega_grid)
    return set_err(ctx, "omega_grid applies to grid searches only"), FFE_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // plans are cached by shape: the lattices, grid lengths and pair momenta
  // (which decide the groups and work items), not the (h, T, Delta) values
  uint64_t hash = 1469598103934665603ull;
  auto mix = [&](const void* v, size_t bytes) {
    const unsigned char* c = static_cast<const unsigned char*>(v);
    for (size_t i = 0; i < bytes; ++i) hash = (hash ^ c[i]) * 1099511628211ull;
  };
  for (int64_t i = 0; i < n; ++i) {
    mix(&ps[i].N, sizeof ps[i].N);
    mix(&ps[i].n, sizeof ps[i].n);
    mix(&ps[i].qx, sizeof ps[i].qx);
    mix(&ps[i].qy, sizeof ps[i].qy);
  }
  char key[160];
  snprintf(key, sizeof key, "amin:%d:%d:%lld:%016llx", ctx->model.prec, search, (long long)n,
           (unsigned long long)hash);
  ffe_plan* p = nullptr;
  auto it = ctx->cache.find(key);
  if (it != ctx->cache.end()) {
    p = it->second;
    p->groups.clear();
    p->delta.clear();
    p->ht.clear();
    p->hlist.clear();
    p->lines.clear();
    p->golden0.clear();
    if (search == FFE_SEARCH_GRID)
      fill_min_grid(p, ps, n);
    else
      fill_min_golden(p, ps, n);
    if ((st = plan_refill(ctx, p, s, true)) != FFE_OK) return st;
  } else {
    st = build_min_plan(ctx, search, ps, n, true, &p);
    if (st != FFE_OK) {
      plan_free(p);
      return st;
    }
    ctx->cache[key] = p;
  }
  if ((st = plan_run(ctx, p, s)) != FFE_OK) return st;
  cudaError_t e = results_launch(p->d_lres, (int64_t)p->lines.size(), p->d_counters, p->cap, out, s);
  if (e == cudaSuccess && omega_grid)
    e = cudaMemcpyAsync(omega_grid, p->d_omega, p->n_out * sizeof(double), cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? FFE_OK : cuda_fail(ctx, e, "ffe_minimize_async");
}

ffe_status ffe_plan_minimize(ffe_context* ctx, int32_t search, const ffe_param* ps, int64_t n, void* stream,
                             ffe_plan** out) {
  if (!ctx || !out) return FFE_EINVAL;
  *out = nullptr;
  (void)stream;
  ffe_status st = check_params(ctx, search, ps, n);
  if (st != FFE_OK) return st;
  ffe_plan* p = nullptr;
  st = build_min_plan(ctx, search, ps, n, true, &p);
  if (st != FFE_OK) {
    plan_free(p);
    return st;
  }
  ctx->plans.push_back(p);
  *out = p;
  return FFE_OK;
}

ffe_status ffe_plan_fetch_minimize(ffe_plan* p, ffe_result* out, double* omega_grid, double* err_grid,
                                   void* stream) {
  if (!p || !out) return FFE_EINVAL;
  if (p->kind != kPlanMinGrid && p->kind != kPlanMinGolden)
    return set_err(p->ctx, "not a minimisation plan"), FFE_EINVAL;
  if (p->kind == kPlanMinGolden && (omega_grid || err_grid))
    return set_err(p->ctx, "omega_grid/err_grid apply to grid searches only"), FFE_EINVAL;
  return fetch_min(p->ctx, p, out, omega_grid, err_grid, (cudaStream_t)stream);
}

}  // extern "C"
