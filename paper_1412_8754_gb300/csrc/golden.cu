// golden.cu -- lockstep golden-section search over Delta for every line
// (one (q, h, T) point each) of a plan, on the device.
//
// Alg. 1 scans Delta from 0 to Delta_max; with a smooth Omega(Delta) the
// minimum can be bracketed instead.  Every line keeps a bracket [a, b] with
// interior points x1 = a + (1-phi)(b-a), x2 = a + phi(b-a), phi = (sqrt5-1)/2;
// it keeps [a, x2] when Omega(x1) <= Omega(x2), else [x1, b], and evaluates
// one new interior point per reduction.  A reference point x0 is evaluated
// first: the normal state Delta = lo, or Delta = 0 when the bracket is a
// window [lo, hi] inside the range.  The result is the lowest Omega seen,
// ties to the smaller Delta.  All lines advance together: one k-sum launch evaluates the
// pending Delta of every line.  While the two interior points are far apart
// (more than 1 % of the range), a decision whose two FP32 values lie within
// their error bounds is taken on FP64 re-evaluations instead.
#include "ffe_internal.cuh"
#include "ksum.cuh"

namespace ffe {

constexpr double kPhi = 0.61803398874989484820;
constexpr double kWideRel = 1e-2;

__device__ __forceinline__ void golden_take(GoldenState& s, double x, double f, double eb) {
  if (f < s.fb || (f == s.fb && x < s.xb)) {
    s.xb = x;
    s.fb = f;
    s.ebb = eb;
  }
}

// Interior points a + w (b - a), rounded step by step (no fused multiply-add),
// so that every line's bracket sequence is the one the textbook formula gives
// in IEEE double: the same Delta values as any other plain evaluation of it.
__device__ __forceinline__ double golden_point(double a, double b, double w) {
  return __dadd_rn(a, __dmul_rn(w, __dsub_rn(b, a)));
}

__device__ __forceinline__ void set_delta(double* delta, float* d2f, int64_t e, double x) {
  delta[e] = x;
  d2f[e] = (float)(x * x);
}

__global__ void golden_kernel(int mode, const Line* __restrict__ lines, int n_lines, GoldenState* gs,
                              const double* __restrict__ omega, const double* __restrict__ ebound, double* delta,
                              float* d2f, Rescore* req, int32_t* n_req, int32_t cap, LineResult* res) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= n_lines) return;
  const Line L = lines[l];
  if (L.pad & kLineAlias) {  // no outputs of its own: never a candidate
    if (mode == kGoldenFinish) {
      LineResult r;
      r.delta_star = 0.0;
      r.omega_star = NAN;
      r.eb_star = 0.0;
      r.omega_lo = NAN;
      r.eb_lo = 0.0;
      r.delta_lo = 0.0;
      r.out_star = L.out0;
      r.idx_star = -1;
      r.flags = kFlagLower;
      res[l] = r;
    }
    return;
  }
  const int64_t o = L.out0;
  const int64_t e = L.delta0;
  GoldenState s = gs[l];
  switch (mode) {
    case kGoldenInit:
      s.a = s.lo;
      s.b = s.hi;
      if (!(s.wide > 0.0)) s.wide = kWideRel * (s.hi - s.lo);
      s.x1 = golden_point(s.a, s.b, 1.0 - kPhi);
      s.x2 = golden_point(s.a, s.b, kPhi);
      s.side = 0;
      set_delta(delta, d2f, e, s.x0);
      break;
    case kGoldenLo:
      s.flo = omega[o];
      s.eblo = ebound[o];
      s.xb = s.x0;
      s.fb = s.flo;
      s.ebb = s.eblo;
      set_delta(delta, d2f, e, s.x1);
      break;
    case kGoldenX1:
      s.f1 = omega[o];
      s.eb1 = ebound[o];
      golden_take(s, s.x1, s.f1, s.eb1);
      set_delta(delta, d2f, e, s.x2);
      break;
    case kGoldenX2:
      s.f2 = omega[o];
      s.eb2 = ebound[o];
      golden_take(s, s.x2, s.f2, s.eb2);
      break;
    case kGoldenMark:
      // Only a decision between interior points far apart (possibly different
      // basins) is worth FP64: close points lie in one basin, where either
      // choice keeps the minimum inside the bracket to within the error band.
      if (fabs(s.f1 - s.f2) <= s.eb1 + s.eb2 && (s.x2 - s.x1) > s.wide) {
        Rescore r;
        r.group = L.group;
        r.dst = l;
        r.ht = L.ht;
        if (s.eb1 > 0.0) {
          r.kind = 3;
          r.delta = s.x1;
          const int pos = atomicAdd(n_req, 1);
          if (pos < cap) req[pos] = r;
        }
        if (s.eb2 > 0.0) {
          r.kind = 4;
          r.delta = s.x2;
          const int pos = atomicAdd(n_req, 1);
          if (pos < cap) req[pos] = r;
        }
      }
      return;  // state unchanged (the FP64 values are written by the re-evaluation)
    case kGoldenDecide:
      if (s.f1 <= s.f2) {  // keep [a, x2]
        s.b = s.x2;
        s.x2 = s.x1;
        s.f2 = s.f1;
        s.eb2 = s.eb1;
        s.x1 = golden_point(s.a, s.b, 1.0 - kPhi);
        s.side = 0;
        set_delta(delta, d2f, e, s.x1);
      } else {  // keep [x1, b]
        s.a = s.x1;
        s.x1 = s.x2;
        s.f1 = s.f2;
        s.eb1 = s.eb2;
        s.x2 = golden_point(s.a, s.b, kPhi);
        s.side = 1;
        set_delta(delta, d2f, e, s.x2);
      }
      break;
    case kGoldenRecord:
      if (s.side == 0) {
        s.f1 = omega[o];
        s.eb1 = ebound[o];
        golden_take(s, s.x1, s.f1, s.eb1);
      } else {
        s.f2 = omega[o];
        s.eb2 = ebound[o];
        golden_take(s, s.x2, s.f2, s.eb2);
      }
      break;
    case kGoldenMarkFinal:
      // The best point against the reference x0 (the normal state wins exact
      // ties).  A bracket whose lower end never left lo = x0 has converged
      // onto x0: its best interior point differs from x0 by O(x^2) and x0 is
      // taken directly (kGoldenFinish); otherwise a near tie is settled in FP64.
      if (!(s.a == s.lo && s.lo == s.x0) && s.xb != s.x0 && fabs(s.fb - s.flo) <= s.ebb + s.eblo) {
        Rescore r;
        r.group = L.group;
        r.dst = l;
        r.ht = L.ht;
        if (s.ebb > 0.0) {
          r.kind = 5;
          r.delta = s.xb;
          const int pos = atomicAdd(n_req, 1);
          if (pos < cap) req[pos] = r;
        }
        if (s.eblo > 0.0) {
          r.kind = 6;
          r.delta = s.x0;
          const int pos = atomicAdd(n_req, 1);
          if (pos < cap) req[pos] = r;
        }
      }
      return;
    case kGoldenFinish: {
      const bool onto_lo = s.a == s.lo && s.lo == s.x0 && fabs(s.fb - s.flo) <= s.ebb + s.eblo;
      if (s.xb != s.x0 && (s.flo <= s.fb || onto_lo)) {
        s.xb = s.x0;
        s.fb = s.flo;
        s.ebb = s.eblo;
      }
      LineResult r;
      r.delta_star = s.xb;
      r.omega_star = s.fb;
      r.eb_star = s.ebb;
      r.omega_lo = s.flo;
      r.eb_lo = s.eblo;
      r.delta_lo = s.x0;
      r.out_star = o;
      r.idx_star = -1;
      int f = 0;
      if (s.xb == s.x0) f |= kFlagLower;
      if (s.b == s.hi) f |= kFlagEdge;
      if (s.a == s.lo && s.lo != s.x0) f |= kFlagBracketLo;
      r.flags = f;
      res[l] = r;
      return;
    }
    default:
      return;
  }
  gs[l] = s;
}

cudaError_t golden_launch(int mode, const Line* lines, int n_lines, GoldenState* gs, const double* omega,
                          const double* ebound, double* delta, float* d2f, Rescore* req, int32_t* n_req,
                          int32_t cap, LineResult* res, cudaStream_t s) {
  if (n_lines <= 0) return cudaSuccess;
  golden_kernel<<<(n_lines + 127) / 128, 128, 0, s>>>(mode, lines, n_lines, gs, omega, ebound, delta, d2f, req,
                                                       n_req, cap, res);
  return cudaGetLastError();
}

}  // namespace ffe
