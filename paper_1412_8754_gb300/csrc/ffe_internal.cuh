// ffe_internal.cuh -- device-side data layout and arithmetic of the free-energy
// engine.  Shared by the kernels in this directory; not part of the C ABI.
//
// Reformulation of Eq. freeene used by every kernel.  Per band eps and k, with
//   E_up = E_eps(k+Q/2) - mu - h,  E_dn = E_eps(-k+Q/2) - mu + h   (App. A, Sec. 2)
//   s = (E_up + E_dn)/2,  d = (E_up - E_dn)/2 = d0 - h,
//   R = sqrt(s^2 + Delta^2 eta^2),  E+/- = d +/- R            (Eq. enequasiparticle)
// the k-point term F(E+) + F(E-) + E_dn splits exactly into
//   [min(E_up,0) + min(E_dn,0)]                         (normal ground state, Delta-free)
// + min(0, max(|d|-|s|, 0) - a),  a = R - |s| = Delta^2 eta^2 / (R + |s|)
// - T ln[(1 + e^{-|R-|d||/T}) (1 + e^{-(R+|d|)/T})]
// using F(E) = min(E,0) - T ln(1 + e^{-|E|/T}) and
// min(d+R,0) + min(d-R,0) = d - max(|d|, R).  The first bracket does not depend
// on Delta or T; it is summed once per (Q, h) in FP64 (the "M" sum).  The rest,
// v_k(Delta), is sign-definite (v <= 0) and free of cancellation, so FP32
// evaluation keeps a relative error of a few ulp of |v|.  With the pairing term
//   Omega(Delta) = M + sum_k v_k(Delta) + 2 N^2 Delta^2 / U.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ffe {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kLayoutProduct = 0;  // outputs = Delta-list x (h,T)-list, shared R per Delta
constexpr int kLayoutList = 1;     // outputs = explicit (Delta, h, T) triples
constexpr int kLayoutProductUT = 2;  // kernel variant of PRODUCT: one T per 32-output batch
constexpr int kMaxBatchesPerItem = 16;
constexpr int kFlagRescored = 1;  // values of include/ffe.h FFE_FLAG_*
constexpr int kFlagEdge = 2;
constexpr int kFlagLower = 4;
constexpr int kFlagBracketLo = 16;  // golden, window bracket: lower end never moved (internal)
constexpr int kLineAlias = 1;       // Line::pad bit: line without outputs of its own
constexpr float kLn2f = 0.693147180559945309f;

struct ModelParams {
  double t1, t2, t3, t4, mu, U, eta_amp;
};

// One group of outputs sharing (N, Q): the unit that shares per-k band work.
struct GroupDesc {
  int32_t N;
  int32_t layout;     // kLayoutProduct / kLayoutList
  int32_t n_delta;    // PRODUCT: Delta values; LIST: outputs
  int32_t n_ht;       // PRODUCT: (h,T) pairs; LIST: outputs
  int32_t n_hblk;     // PRODUCT: ceil(n_ht/32); LIST: 1
  int32_t n_batches;  // PRODUCT: n_delta*n_hblk; LIST: ceil(n_out/32)
  int32_t n_h;        // distinct h values of the group (for the M sum)
  int32_t n_out;      // outputs of the group
  int64_t out_off;    // first output in the global output arrays
  int64_t delta_off;  // first Delta entry
  int64_t ht_off;     // first (h,T) entry
  int64_t tab_off;    // first table row: x rows [tab_off, tab_off+N), y rows after
  int64_t h_off;      // first entry of the distinct-h list and of the M sums
  double qx, qy;
  int32_t band_only;  // 0: both bands; 1: the lower band only; 2: the upper band only
  int32_t pad;
};

// (h, T) entry with the index of its h in the group's distinct-h list.
struct HT {
  double h, T;
  int32_t h_idx;
  int32_t pad;
};

// Per-entry FP32 parameters of an (h,T) entry: h, c = 1/(T ln 2), TL = T ln 2.
// Per-entry FP64 parameters: h, 1/T, T.
struct HTf { float h, c, tl, pad; };
struct HTd { double h, inv_t, t, pad; };

// Warp work item of the persistent k-sum: k-sets [kset0, kset1) of one group
// for batches [b0, b1) of its outputs.  A k-set is 32*KPT consecutive k-points.
struct WorkItem {
  int32_t group;
  int32_t seg;
  int32_t chunk;
  int32_t kset0, kset1;
  int32_t b0, b1;
  // FP32 path: every output of the item has h in [far_hlo, far_hhi]; a
  // k-point with min over bands of |s| - max(|d0 - far_hlo|, |d0 - far_hhi|)
  // >= far_tgap is "far" for all of them (see ksum.cu); far_tgap = +inf:
  // no k-point is.
  float far_hlo, far_hhi, far_tgap;
  int32_t pad[3];
};

// A segment = (group, batch range); its chunks partition the k-sets.
struct Segment {
  int32_t group;
  int32_t b0, b1;
  int32_t n_chunks;
  int64_t partial_off;
};

// Table row: cos/sin of k + q/2 and k - q/2 on one axis, and cos k.
struct TabRowF { float cp, sp, cm, sm; };
struct TabRowD { double cp, sp, cm, sm; };
// The FP64 row as unevaluated sums hi + lo of two floats (double-float).
struct TabRowDF { float2 cp, sp, cm, sm; };

// ---------------------------------------------------------------- FP32 MUFU
__device__ __forceinline__ float ex2a(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2a(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqa(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcpa(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// App. A eigenvalues at one momentum from its cos/sin values: lo = E_-, hi = E_+.
template <typename Real>
__device__ __forceinline__ void band_pair(const ModelParams& m, Real cx, Real cy, Real sx,
                                          Real sy, Real& lo, Real& hi) {
  const Real t1 = (Real)m.t1, t2 = (Real)m.t2, t3 = (Real)m.t3, t4 = (Real)m.t4;
  Real mean = -(t1 + t2) * (cx + cy) - (Real)4 * t3 * (cx * cy);  // (T11+T22)/2
  Real half = -(t1 - t2) * (cx - cy);                              // (T11-T22)/2
  Real t12 = -(Real)4 * t4 * (sx * sy);
  Real root = sqrt(half * half + t12 * t12);
  lo = mean - root;
  hi = mean + root;
}

// Per-k state: eta^2 and, per band, |s|, s^2 (floored at 1e-30 so that
// rsqrt stays finite), d0 = (E(k+Q/2) - E(k-Q/2))/2.
template <typename Real>
struct KState {
  Real eta2;
  Real as[2], s2[2], d0[2];
};

template <typename Real>
__device__ __forceinline__ void kstate_invalid(KState<Real>& st) {
  st.eta2 = (Real)0;
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    st.as[b] = (Real)1e15;
    st.s2[b] = (Real)1e30;
    st.d0[b] = (Real)0;
  }
}

template <typename Real, typename Row>
__device__ __forceinline__ void kstate_make(const ModelParams& m, const Row& rx, const Row& ry,
                                            Real c0x, Real c0y, KState<Real>& st) {
  Real eta = (Real)m.eta_amp * c0x * c0y;
  st.eta2 = eta * eta;
  Real ulo, uhi, dlo, dhi;
  band_pair<Real>(m, (Real)rx.cp, (Real)ry.cp, (Real)rx.sp, (Real)ry.sp, ulo, uhi);  // k + Q/2
  band_pair<Real>(m, (Real)rx.cm, (Real)ry.cm, (Real)rx.sm, (Real)ry.sm, dlo, dhi);  // -k + Q/2
  const Real mu = (Real)m.mu;
  Real s0 = (Real)0.5 * (ulo + dlo) - mu, s1 = (Real)0.5 * (uhi + dhi) - mu;
  st.d0[0] = (Real)0.5 * (ulo - dlo);
  st.d0[1] = (Real)0.5 * (uhi - dhi);
  st.as[0] = fabs(s0);
  st.as[1] = fabs(s1);
  st.s2[0] = fmax(s0 * s0, (Real)1e-30);
  st.s2[1] = fmax(s1 * s1, (Real)1e-30);
}

// A group restricted to one band: the other band's state is made inert
// (|s| = 1e15: no log term, a = Delta^2 eta^2 / 2e15 <= 2e-17 per k-point).
template <typename Real>
__device__ __forceinline__ void kstate_band_only(KState<Real>& st, int band_only) {
  if (band_only == 0) return;
  const int off = band_only == 1 ? 1 : 0;
  st.as[off] = (Real)1e15;
  st.s2[off] = (Real)1e30;
  st.d0[off] = (Real)0;
}

// Delta-dependent, (h,T)-independent part for one band: R and a = R - |s|.
__device__ __forceinline__ void ra_f32(float D, float s2, float as, float& R, float& a) {
  float u = D + s2;
  R = u * rsqa(u);
  a = D * rcpa(R + as);
}

// FP32 k-point term in units of T ln 2.  With c = 1/(T ln 2) the term of one
// band is  -T ln2 [ c min(max(R - |d|, 0), a) + log2((1+e1)(1+e2)) ],
// e1 = 2^{-c|R-d|}, e2 = 2^{-c|R+d|} (the pair {|R-d|, |R+d|} equals
// {|R-|d||, R+|d|}), because
//   min(0, max(|d|-|s|, 0) - a) = -min(max(R - |d|, 0), a)     (R = |s| + a)
// and R - |d| = min(R - d, R + d).  The factor -T ln2 is constant over k and
// is applied once per output after the k-sum, so the accumulated quantity
// W = sum_k [...] is non-negative.  The two bands are evaluated as the two
// halves of packed FP32x2 operations.
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Per-k FP32 state with the two bands packed: eta^2, |s|, s^2, d0.
struct KState32 {
  float eta2;
  float2 as, s2, d0;
};

// One k-point, both bands, one (h, c): adds c min(...) of each band to cp2 and
// returns log2 of the product of the four (1 + e) factors.
// Rc = R c and ac = a c per band; nh2 = (-h, -h); c2 = (c, c); nc2 = -c2.
__device__ __forceinline__ float w_term32(const KState32& st, float2 Rc, float2 ac, float2 nh2, float2 c2,
                                          float2 nc2, float2& cp2) {
  const float2 d = __fadd2_rn(st.d0, nh2);  // d = d0 - h
  const float2 y1 = __ffma2_rn(d, nc2, Rc);  // c (R - d)
  const float2 y2 = __ffma2_rn(d, c2, Rc);   // c (R + d)
  const float2 e1 = make_float2(ex2a(-fabsf(y1.x)), ex2a(-fabsf(y1.y)));
  const float2 e2 = make_float2(ex2a(-fabsf(y2.x)), ex2a(-fabsf(y2.y)));
  const float2 o1 = __fadd2_rn(e1, make_float2(1.0f, 1.0f));
  const float2 p = __ffma2_rn(o1, e2, o1);
  const float2 cp = make_float2(fmaxf(min3f(y1.x, y2.x, ac.x), 0.0f), fmaxf(min3f(y1.y, y2.y, ac.y), 0.0f));
  cp2 = __fadd2_rn(cp2, cp);
  return lg2a(p.x * p.y);
}
__device__ __forceinline__ void ra_f64(double D, double s2, double as, double& R, double& a) {
  R = sqrt(D + s2);
  a = D / (R + as);
}

// FP64 band term for one (h,T): q = p - 1 = e1 + e2 + e1 e2 (kept as p - 1
// for log1p) and first = min(0, max(|d|-|s|, 0) - a).
__device__ __forceinline__ void band_term_f64(double R, double a, double as, double d0, double h,
                                              double inv_t, double& q, double& first) {
  double d = d0 - h;
  double ad = fabs(d);
  double x1 = fabs(R - ad);
  double x2 = R + ad;
  double e1 = exp(-x1 * inv_t);
  double e2 = exp(-x2 * inv_t);
  q = e1 + e2 + e1 * e2;
  double g = fmax(ad - as, 0.0);
  first = fmin(g - a, 0.0);
}

// Sum of 32 per-lane values per output index: on return lane l holds the warp
// total of part[l] (butterfly reduce-scatter: 31 shuffles for 32 outputs).
template <typename Real>
__device__ __forceinline__ Real reduce_scatter32(Real (&part)[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      Real send = upper ? part[i] : part[i + s];
      Real keep = upper ? part[i + s] : part[i];
      part[i] = keep + __shfl_xor_sync(kFull, send, s);
    }
  }
  return part[0];
}

}  // namespace ffe
