// search.cu -- Delta search, FP64 re-evaluation of near ties, phase labels.
//
// Alg. 1 keeps, per pair momentum q, the Delta of lowest Omega and then the q
// of lowest Omega.  The paper does the Delta search on the host after copying
// partial sums back (Sec. 3, step 3); here it stays on the device:
//  * argmin_kernel, pass A: per line (one Delta grid of one (q, h, T)) the
//    lowest Omega and every grid point whose FP32 error band overlaps the
//    minimum's band; if there is more than one, those points are queued for
//    FP64 re-evaluation ("run at lower precision, then selectively verify with
//    double precision", Sec. 3, performance evaluation).
//  * rescore_kernel: the k-sum of one (q, h, T, Delta) in FP64, split over
//    k-chunks with a deterministic last-block-done reduction.
//  * argmin_kernel, pass B: the final argmin (ties -> lowest index).
//  * labels_kernel: per (h, T) the normal / BCS / FF label from the per-q
//    minima, FP64 comparisons with a tie band tau = 1e-12 |Omega_N|; values
//    whose FP32 error band could flip a comparison are re-evaluated in FP64
//    (pass 0) before the final labels (pass 1).
#include <cfloat>
#include <climits>

#include "../../include/ffe.h"
#include "ffe_internal.cuh"
#include "ksum.cuh"

namespace ffe {

constexpr double kTauRel = 1e-12;

__device__ __forceinline__ void warp_argmin(double& v, int& i) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const double ov = __shfl_xor_sync(kFull, v, s);
    const int oi = __shfl_xor_sync(kFull, i, s);
    if (ov < v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
}

__device__ __forceinline__ void push_request(Rescore* req, int32_t* n_req, int32_t cap, const Rescore& r) {
  const int pos = atomicAdd(n_req, 1);
  if (pos < cap) req[pos] = r;
}

__global__ void argmin_kernel(const Line* __restrict__ lines, int n_lines, const double* __restrict__ omega,
                              const double* __restrict__ eb, const double* __restrict__ delta,
                              const int32_t* __restrict__ rescored, int mode, Rescore* req, int32_t* n_req,
                              int32_t cap, LineResult* res) {
  const int gw = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (gw >= n_lines) return;
  const Line L = lines[gw];
  double best = DBL_MAX;
  int bi = INT_MAX;
  for (int i = lane; i < L.count; i += 32) {
    const double v = omega[L.out0 + (int64_t)i * L.stride];
    if (v < best) {
      best = v;
      bi = i;
    }
  }
  warp_argmin(best, bi);
  if (bi == INT_MAX) bi = 0;  // all values NaN: keep the index in range
  const int64_t out_b = L.out0 + (int64_t)bi * L.stride;
  if (mode == 0) {
    const double thr = best + eb[out_b];
    int ncand = 0;
    for (int i0 = 0; i0 < L.count; i0 += 32) {
      const int i = i0 + lane;
      bool c = false;
      if (i < L.count) {
        const int64_t o = L.out0 + (int64_t)i * L.stride;
        c = (omega[o] - eb[o] <= thr);
      }
      ncand += __popc(__ballot_sync(kFull, c));
    }
    if (ncand > 1) {
      for (int i = lane; i < L.count; i += 32) {
        const int64_t o = L.out0 + (int64_t)i * L.stride;
        if (omega[o] - eb[o] <= thr && eb[o] > 0.0) {
          Rescore r;
          r.group = L.group;
          r.kind = 0;
          r.dst = o;
          r.ht = L.ht;
          r.delta = delta[L.delta0 + i];
          push_request(req, n_req, cap, r);
        }
      }
    }
  } else if (lane == 0) {
    LineResult r;
    r.idx_star = bi;
    r.out_star = out_b;
    r.delta_star = delta[L.delta0 + bi];
    r.omega_star = best;
    r.eb_star = eb[out_b];
    r.omega_lo = omega[L.out0];
    r.eb_lo = eb[L.out0];
    r.delta_lo = delta[L.delta0];
    int f = 0;
    if (rescored[out_b]) f |= kFlagRescored;
    if (bi == L.count - 1) f |= kFlagEdge;
    if (bi == 0) f |= kFlagLower;
    r.flags = f;
    res[gw] = r;
  }
}

cudaError_t argmin_launch(const Line* lines, int n_lines, const double* omega, const double* ebound,
                          const double* delta, const int32_t* rescored, int mode, Rescore* req,
                          int32_t* n_req, int32_t cap, LineResult* res, cudaStream_t s) {
  if (n_lines <= 0) return cudaSuccess;
  const int threads = 256;
  const int grid = (int)(((int64_t)n_lines * 32 + threads - 1) / threads);
  argmin_kernel<<<grid, threads, 0, s>>>(lines, n_lines, omega, ebound, delta, rescored, mode, req, n_req,
                                         cap, res);
  return cudaGetLastError();
}

// Near-band entries per warp and request in the FP64 re-evaluation: a flush
// takes the top 32, a step of 32 k-points adds at most 32 x (two slots) per
// band pair; the three-band model (two pairs) takes two request slots.
constexpr int kRescoreBufSlot = 32 + 32 * 2;
__host__ __device__ constexpr int rescore_run_max(int nbands) { return nbands == 3 ? kRescoreRun / 2 : kRescoreRun; }

// -T ln(1 + q), q = e1 + e2 + e1 e2, of one near band (y1 = |R - |d|| / T < kExpNegligible,
// y2 = (R + |d|) / T), with band_term_f64's cut-off for e2.
__device__ __forceinline__ double near_log_term(double2 y, double t) {
  const double e1 = exp(-y.x);
  const double e2 = y.y < kExpNegligible ? exp(-y.y) : 0.0;
  return -t * log1p(e1 + e2 + e1 * e2);
}

// Groups the queued requests by group: counts, offsets and a scatter of the
// request indices, then runs of at most rescore_run_max of one group.  Which
// requests share a run does not change any request's sums (each keeps its own
// accumulators and near-band buffer in rescore_kernel).  One block.
__global__ void __launch_bounds__(1024) rescore_sort_kernel(const RescoreArgs a) {
  __shared__ int32_t part[1024];
  __shared__ int32_t rpart[1024];
  const int nreq = min(*a.n_req, a.cap);
  const int ng = a.n_groups;
  const int R = rescore_run_max(a.m.nbands);
  int32_t* cnt = a.gcount;                // [ng + 1]; cnt[ng] = runs in total
  int32_t* off = a.gcount + (ng + 1);     // [ng + 1] request offset per group
  int32_t* roff = a.gcount + 2 * (ng + 1);  // [ng + 1] run offset per group
  int32_t* fill = a.gcount + 3 * (ng + 1);  // [ng + 1]
  const int t = threadIdx.x, nt = blockDim.x;
  for (int g = t; g <= ng; g += nt) {
    cnt[g] = 0;
    fill[g] = 0;
  }
  __syncthreads();
  for (int r = t; r < nreq; r += nt) {
    const int g = a.req[r].group;
    if (g >= 0 && g < ng) atomicAdd(cnt + g, 1);
  }
  __syncthreads();
  // exclusive scans of the request and run counts: contiguous ranges per thread
  const int per = (ng + nt - 1) / nt, g0 = min(ng, t * per), g1 = min(ng, g0 + per);
  int sum = 0, rsum = 0;
  for (int g = g0; g < g1; ++g) {
    sum += cnt[g];
    rsum += (cnt[g] + R - 1) / R;
  }
  part[t] = sum;
  rpart[t] = rsum;
  __syncthreads();
  if (t == 0) {
    int acc = 0, racc = 0;
    for (int i = 0; i < nt; ++i) {
      const int v = part[i], rv = rpart[i];
      part[i] = acc;
      rpart[i] = racc;
      acc += v;
      racc += rv;
    }
    cnt[ng] = racc;
  }
  __syncthreads();
  int acc = part[t], racc = rpart[t];
  for (int g = g0; g < g1; ++g) {
    off[g] = acc;
    roff[g] = racc;
    acc += cnt[g];
    racc += (cnt[g] + R - 1) / R;
  }
  __syncthreads();
  for (int r = t; r < nreq; r += nt) {
    const int g = a.req[r].group;
    if (g >= 0 && g < ng) a.order[off[g] + atomicAdd(fill + g, 1)] = r;
  }
  for (int g = t; g < ng; g += nt)
    for (int i = 0; i * R < cnt[g]; ++i) a.runs[roff[g] + i] = make_int2(off[g] + i * R, min(R, cnt[g] - i * R));
}

// The FP64 k-sums of a run of requests of one group, k-chunk by k-chunk: the
// band energies of each k-point are formed once and serve every request of
// the run.  Per request each warp takes 32 consecutive k-points per step;
// every active band adds its clamp term min(max(|d| - |s|, 0) - a, 0) at
// once, and only a band with |R - |d|| / T < kExpNegligible (near) has
// exponentials that are not 0: such bands are compacted (ballot + prefix
// count) into the request's warp buffer and their -T ln(1 + q) evaluated 32 at
// a time, so the exponentials and the logarithm run on full warps.  Each
// request keeps its own per-thread sums and buffers, so its result has the
// same bits whichever requests share its run.
constexpr int kRescoreThreads = 128;

__global__ void __launch_bounds__(kRescoreThreads) rescore_kernel(const RescoreArgs a) {
  __shared__ double red[kRescoreThreads / 32];
  __shared__ int sh_w, sh_last;
  __shared__ Rescore sh_req[kRescoreRun];
  __shared__ int32_t sh_ri[kRescoreRun];
  __shared__ double acc[kRescoreRun][kRescoreThreads];
  __shared__ double2 near_buf[kRescoreThreads / 32][kRescoreRun * kRescoreBufSlot];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int slot = a.m.nbands == 3 ? 2 * kRescoreBufSlot : kRescoreBufSlot;
  const int n_runs = a.gcount[a.n_groups];
  const int total = n_runs * a.max_chunks;
  for (;;) {
    if (threadIdx.x == 0) sh_w = atomicAdd(a.queue, 1);
    __syncthreads();
    const int w = sh_w;
    if (w >= total) break;
    const int ru = w / a.max_chunks, c = w - ru * a.max_chunks;
    const int2 run = a.runs[ru];
    const int m = run.y;
    if (threadIdx.x < m) {
      const int ri = a.order[run.x + threadIdx.x];
      sh_ri[threadIdx.x] = ri;
      sh_req[threadIdx.x] = a.req[ri];
    }
    for (int j = 0; j < m; ++j) acc[j][threadIdx.x] = 0.0;
    __syncthreads();
    const GroupDesc g = a.groups[sh_req[0].group];
    const int64_t nk = (int64_t)g.N * g.N;
    const int64_t k0 = (int64_t)c * a.chunk_k;
    const int64_t k1 = min(nk, k0 + a.chunk_k);
    int n_near[kRescoreRun];
#pragma unroll
    for (int j = 0; j < kRescoreRun; ++j) n_near[j] = 0;
    for (int64_t kb = k0 + warp * 32; kb < k1; kb += blockDim.x) {
      const int64_t k = kb + lane;
      const bool valid = k < k1;
      const int iy = valid ? (int)(k / g.N) : 0;
      const int ix = valid ? (int)(k - (int64_t)iy * g.N) : 0;
      for (int pair = 0; pair < band_pairs(a.m.nbands); ++pair) {
        KState<double> st;
        if (!valid) {
          kstate_invalid<double>(st);
        } else if (a.m.nbands == 3) {
          const double eta = a.m.eta_amp * a.c0d[g.tab_off + ix] * a.c0d[g.tab_off + g.N + iy];
          kstate_from_table3<double, E3D>(a.m, eta, a.e3d[g.e3_off + k], a.e3d[g.e3_off + nk + k], pair, st);
        } else {
          kstate_make<double, TabRowD>(a.m, a.tabd[g.tab_off + ix], a.tabd[g.tab_off + g.N + iy],
                                       a.c0d[g.tab_off + ix], a.c0d[g.tab_off + g.N + iy], st);
        }
#pragma unroll
        for (int j = 0; j < kRescoreRun; ++j) {
          if (j >= m) break;
          const Rescore q = sh_req[j];
          const HT ht = a.ht[q.ht];
          const double inv_t = 1.0 / ht.T;
          const double D = (q.delta * q.delta) * st.eta2;
          double2* nb = near_buf[warp] + j * slot;
          double sj = 0.0;
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            const bool use = valid && slot_active(a.m.nbands, g.band_only, pair, b);
            double R, A;
            ra_f64(D, st.s2[b], st.as[b], R, A);
            const double ad = fabs(st.d0[b] - ht.h);
            const double y1 = fabs(R - ad) * inv_t;
            if (use) sj += fmin(fmax(ad - st.as[b], 0.0) - A, 0.0);
            const bool near = use && y1 < kExpNegligible;
            const unsigned msk = __ballot_sync(kFull, near);
            if (near) nb[n_near[j] + __popc(msk & lt)] = make_double2(y1, (R + ad) * inv_t);
            n_near[j] += __popc(msk);
          }
          acc[j][threadIdx.x] += sj;
        }
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < kRescoreRun; ++j) {
        if (j >= m) break;
        const double T = a.ht[sh_req[j].ht].T;
        const double2* nb = near_buf[warp] + j * slot;
        while (n_near[j] >= 32) {  // the top 32 entries, one per lane
          n_near[j] -= 32;
          acc[j][threadIdx.x] += near_log_term(nb[n_near[j] + lane], T);
        }
      }
      __syncwarp();
    }
    for (int j = 0; j < m; ++j) {
      const double T = a.ht[sh_req[j].ht].T;
      double s = acc[j][threadIdx.x];
      if (lane < n_near[j]) s += near_log_term(near_buf[warp][j * slot + lane], T);
      __syncwarp();
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
      if (lane == 0) red[warp] = s;
      __syncthreads();
      const int r = sh_ri[j];
      const Rescore q = sh_req[j];
      if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b += red[i];
        a.partials[(int64_t)r * a.max_chunks + c] = b;
        __threadfence();
        sh_last = (atomicAdd(a.counters + r, 1) == a.max_chunks - 1);
      }
      __syncthreads();
      if (sh_last && threadIdx.x == 0) {
        __threadfence();
        const HT ht = a.ht[q.ht];
        double V = 0.0;
        for (int i = 0; i < a.max_chunks; ++i) V += __ldcg(a.partials + (int64_t)r * a.max_chunks + i);
        const double n2 = (double)g.N * (double)g.N;
        const double om = a.M[g.h_off + ht.h_idx] + V + pairing_term(a.m, g.band_only, n2, q.delta);
        if (q.kind == 0) {
          a.omega[q.dst] = om;
          a.ebound[q.dst] = 0.0;
          a.rescored[q.dst] = 1;
        } else if (q.kind == 3) {
          a.golden[q.dst].f1 = om;
          a.golden[q.dst].eb1 = 0.0;
        } else if (q.kind == 4) {
          a.golden[q.dst].f2 = om;
          a.golden[q.dst].eb2 = 0.0;
        } else if (q.kind == 5) {
          a.golden[q.dst].fb = om;
          a.golden[q.dst].ebb = 0.0;
        } else if (q.kind == 6) {
          a.golden[q.dst].flo = om;
          a.golden[q.dst].eblo = 0.0;
        } else {
          // kinds 1 (minimum) and 2 (Delta = lo) name the same value when the
          // minimum is the Delta = lo point: keep both copies identical
          LineResult& L = a.lines[q.dst];
          const bool same = (L.flags & kFlagLower) != 0;
          if (q.kind == 1 || same) {
            L.omega_star = om;
            L.eb_star = 0.0;
            L.flags |= kFlagRescored;
          }
          if (q.kind == 2 || same) {
            L.omega_lo = om;
            L.eb_lo = 0.0;
          }
        }
        a.counters[r] = 0;
      }
      __syncthreads();
    }
  }
}

cudaError_t rescore_occupancy(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, rescore_kernel, kRescoreThreads, 0);
}

cudaError_t rescore_launch(const RescoreArgs& a, int grid, cudaStream_t s) {
  rescore_sort_kernel<<<1, 1024, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  rescore_kernel<<<grid, kRescoreThreads, 0, s>>>(a);
  return cudaGetLastError();
}

// One thread per (h, T) point; lines are q-major: line = q * n_pts + p.
__global__ void labels_kernel(LineResult* res, int n_q, int n_pts, const int32_t* __restrict__ q_is_zero,
                              const Line* __restrict__ lines, const double* __restrict__ delta, int mode,
                              Rescore* req, int32_t* n_req, int32_t cap, int8_t* labels, int32_t* best_q) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pts) return;
  int q0 = -1;
  for (int q = 0; q < n_q; ++q)
    if (q_is_zero[q]) {
      q0 = q;
      break;
    }
  if (q0 < 0) {
    labels[p] = -1;
    best_q[p] = -1;
    return;
  }
  const LineResult rN = res[(int64_t)q0 * n_pts + p];
  const double omega_n = rN.omega_lo;
  const double tau = kTauRel * fabs(omega_n);
  int best = -1;
  double wbest = 0.0;
  for (int q = 0; q < n_q; ++q) {
    const LineResult r = res[(int64_t)q * n_pts + p];
    if (r.omega_star < r.omega_lo - tau && (best < 0 || r.omega_star < wbest)) {
      best = q;
      wbest = r.omega_star;
    }
  }
  if (mode == 0) {
    const double eb_best = best >= 0 ? res[(int64_t)best * n_pts + p].eb_star : 0.0;
    // A line whose minimum is the Delta = lo point compares one value with
    // itself: never a candidate, whatever its error band.
    auto maybe_candidate = [&](const LineResult& r) {
      return !(r.flags & kFlagLower) && r.omega_star < r.omega_lo - tau + r.eb_star + r.eb_lo;
    };
    // a q that may be a candidate and whose minimum is within error of the best one
    auto contests = [&](const LineResult& r, int q) {
      return best >= 0 && q != best && maybe_candidate(r) && fabs(r.omega_star - wbest) <= r.eb_star + eb_best;
    };
    const bool vs_normal = best >= 0 && fabs(omega_n - tau - wbest) <= eb_best + rN.eb_lo;
    bool best_contested = false;
    for (int q = 0; q < n_q && best >= 0; ++q)
      if (contests(res[(int64_t)q * n_pts + p], q)) best_contested = true;
    for (int q = 0; q < n_q; ++q) {
      const int64_t l = (int64_t)q * n_pts + p;
      const LineResult r = res[l];
      // candidate test Omega* < Omega(lo) - tau within error
      bool need_star = !(r.flags & kFlagLower) && fabs(r.omega_lo - tau - r.omega_star) <= r.eb_star + r.eb_lo;
      bool need_lo = need_star;
      if (contests(r, q)) need_star = true;
      if (q == best && (best_contested || vs_normal)) need_star = true;
      if (q == q0 && vs_normal) need_lo = true;
      const Line L = lines[l];
      if (need_star && r.eb_star > 0.0) {
        Rescore rq;
        rq.group = L.group;
        rq.kind = 1;
        rq.dst = l;
        rq.ht = L.ht;
        rq.delta = r.delta_star;
        push_request(req, n_req, cap, rq);
      }
      if (need_lo && r.eb_lo > 0.0) {
        Rescore rq;
        rq.group = L.group;
        rq.kind = 2;
        rq.dst = l;
        rq.ht = L.ht;
        rq.delta = r.delta_lo;
        push_request(req, n_req, cap, rq);
      }
    }
  }
  int label = 0;
  if (best >= 0 && wbest < omega_n - tau) label = q_is_zero[best] ? 1 : 2;
  labels[p] = (int8_t)label;
  best_q[p] = label == 0 ? -1 : best;
}

cudaError_t labels_launch(LineResult* res, int n_q, int n_pts, const int32_t* q_is_zero, const Line* lines,
                          const double* delta, int mode, Rescore* req, int32_t* n_req, int32_t cap,
                          int8_t* labels, int32_t* best_q, cudaStream_t s) {
  if (n_pts <= 0) return cudaSuccess;
  labels_kernel<<<(n_pts + 127) / 128, 128, 0, s>>>(res, n_q, n_pts, q_is_zero, lines, delta, mode, req,
                                                     n_req, cap, labels, best_q);
  return cudaGetLastError();
}

// Line results in the C ABI's layout, written on the device for the
// stream-ordered entry points.  counters: the plan's counter block ([3], [4]
// the FP64 requests of the search and of the labels, [7] the status word); a
// request count above cap or a non-zero status marks every line
// FFE_FLAG_INVALID with NaN values.
__global__ void results_kernel(const LineResult* __restrict__ lr, int64_t n, const int32_t* __restrict__ counters,
                               int32_t cap, ffe_result* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool bad = counters[7] != 0 || counters[3] > cap || counters[4] > cap;
  const LineResult r = lr[i];
  ffe_result o;
  o.delta_star = bad ? NAN : r.delta_star;
  o.omega_star = bad ? NAN : r.omega_star;
  o.omega_lo = bad ? NAN : r.omega_lo;
  o.err_bound = bad ? NAN : r.eb_star;
  o.idx_star = r.idx_star;
  o.flags = bad ? (r.flags | FFE_FLAG_INVALID) : r.flags;
  out[i] = o;
}

cudaError_t results_launch(const LineResult* lr, int64_t n, const int32_t* counters, int32_t cap, void* out,
                           cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  results_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(lr, n, counters, cap, static_cast<ffe_result*>(out));
  return cudaGetLastError();
}

}  // namespace ffe
