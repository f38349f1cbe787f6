// merge.cu -- the outer argmin of Alg. 1 over q lists split across ranks
// (host code; no device work).
//
// A phase scan whose q list is split across ranks gives each rank the Delta
// minima of its own lines only.  Per (h, T) point a rank reduces its lines to
// one candidate -- the lowest Omega* among its lines that condense
// (Omega* < Omega(Delta = lo) - tau), ties to the lowest global q index -- and
// the ranks' candidates are merged with the same rule, then compared with the
// normal state Omega_N = Omega(q = 0, Delta = 0) of the rank that holds
// q = 0: the labels of ffe_phase_scan (tau = 1e-12 |Omega_N|).
#include <cmath>

#include "../../include/ffe.h"

namespace {
constexpr double kTauRel = 1e-12;
}

extern "C" {

ffe_status ffe_label_candidates(const ffe_result* per_point, int32_t n_q, int32_t n_pts, const int32_t* q_global,
                                const double* omega_n, double* best_val, int32_t* best_q) {
  if (!per_point || !q_global || !omega_n || !best_val || !best_q || n_q < 0 || n_pts < 0) return FFE_EINVAL;
  for (int32_t p = 0; p < n_pts; ++p) {
    const double tau = kTauRel * std::fabs(omega_n[p]);
    int32_t bq = -1;
    double bv = INFINITY;
    for (int32_t q = 0; q < n_q; ++q) {
      const ffe_result& r = per_point[(int64_t)q * n_pts + p];
      if (!(r.omega_star < r.omega_lo - tau)) continue;
      if (bq < 0 || r.omega_star < bv || (r.omega_star == bv && q_global[q] < bq)) {
        bv = r.omega_star;
        bq = q_global[q];
      }
    }
    best_val[p] = bv;
    best_q[p] = bq;
  }
  return FFE_OK;
}

ffe_status ffe_merge_candidates(int32_t world, int32_t n_pts, const double* best_val, const int32_t* best_q,
                                const double* omega_n, int32_t zero_q, int8_t* labels, int32_t* best_q_out) {
  if (!best_val || !best_q || !omega_n || !labels || !best_q_out || world < 1 || n_pts < 0) return FFE_EINVAL;
  for (int32_t p = 0; p < n_pts; ++p) {
    const double tau = kTauRel * std::fabs(omega_n[p]);
    int32_t bq = -1;
    double bv = INFINITY;
    for (int32_t r = 0; r < world; ++r) {
      const int64_t i = (int64_t)r * n_pts + p;
      if (best_q[i] < 0) continue;
      if (bq < 0 || best_val[i] < bv || (best_val[i] == bv && best_q[i] < bq)) {
        bv = best_val[i];
        bq = best_q[i];
      }
    }
    const bool win = bq >= 0 && bv < omega_n[p] - tau;
    labels[p] = (int8_t)(win ? (bq == zero_q ? FFE_PHASE_BCS : FFE_PHASE_FFLO) : FFE_PHASE_NORMAL);
    best_q_out[p] = win ? bq : -1;
  }
  return FFE_OK;
}

}  // extern "C"
