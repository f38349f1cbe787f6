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
constexpr int kLayoutProductUT = 2;  // kernel variant of PRODUCT: one T per tile of a batch
// Batches (of 32 outputs) per work item, at most: the FP64 accumulator rows a
// warp keeps in shared memory at 16 warps per SM.  FP32 PRODUCT items take 24
// (the per-k-point classification is shared by 768 outputs) and at most
// kMaxTileDeltas Delta rows (the warp's FP64 far sums); FP64 PRODUCT items 16;
// LIST items 8 (their entry buffers and moments take the rest).
constexpr int kMaxBatchesPerItem = 16;
constexpr int kMaxBatchesTile = 24;
constexpr int kMaxTileDeltas = 96;
constexpr int kMaxBatchesList = 8;
__host__ __device__ constexpr int max_batches(int group_layout, bool fp32) {
  return group_layout == kLayoutList ? kMaxBatchesList : (fp32 ? kMaxBatchesTile : kMaxBatchesPerItem);
}
constexpr int kFlagRescored = 1;  // values of include/ffe.h FFE_FLAG_*
constexpr int kFlagEdge = 2;
constexpr int kFlagLower = 4;
constexpr int kFlagBracketLo = 16;  // golden, window bracket: lower end never moved (internal)
constexpr int kLineAlias = 1;       // Line::pad bit: line without outputs of its own
constexpr float kLn2f = 0.693147180559945309f;

struct ModelParams {
  double t1, t2, t3, t4, mu, U, eta_amp;
  int32_t kind;    // FFE_MODEL_RAGHU2 (0) or FFE_MODEL_DAGHOFER3 (1)
  int32_t nbands;  // 2 or 3
  double t5, t6, t7, t8, t9, t10, t11, t12, eps0;  // three-band model only
  // per-band couplings (Sec. 2: V_eps per band); used when per_band_u != 0,
  // else every band has U
  double Ub[3];
  int32_t per_band_u;
  int32_t pad;
};

// The pairing term of Eq. freeene summed over the k-points and over the bands
// of an output (all of them, or band band_only - 1): N^2 Delta^2 sum_b 1/U_b.
__host__ __device__ __forceinline__ double pairing_term(const ModelParams& m, int band_only, double n2, double dl) {
  if (!m.per_band_u) return (band_only ? 1.0 : (double)m.nbands) * n2 * dl * dl / m.U;
  if (band_only) return n2 * dl * dl / m.Ub[band_only - 1];
  double t = 0.0;
  for (int b = 0; b < m.nbands; ++b) t += n2 * dl * dl / m.Ub[b];
  return t;
}

// One group of outputs sharing (N, Q): the unit that shares per-k band work.
struct GroupDesc {
  int32_t N;
  int32_t layout;     // kLayoutProduct / kLayoutList
  int32_t n_delta;    // PRODUCT: Delta values; LIST: outputs
  int32_t n_ht;       // PRODUCT: (h,T) pairs; LIST: outputs
  int32_t n_hblk;     // PRODUCT: ceil(n_ht/hb); LIST: 1
  int32_t n_batches;  // PRODUCT: n_hblk*ceil(n_delta/(32/hb)); LIST: ceil(n_out/32)
  int32_t n_h;        // distinct h values of the group (for the M sum)
  int32_t n_out;      // outputs of the group
  int64_t out_off;    // first output in the global output arrays
  int64_t delta_off;  // first Delta entry
  int64_t ht_off;     // first (h,T) entry
  int64_t tab_off;    // first table row: x rows [tab_off, tab_off+N), y rows after
  int64_t h_off;      // first entry of the distinct-h list and of the M sums
  double qx, qy;
  int32_t band_only;  // 0: every band; b + 1: band b only (bands in ascending order of energy)
  int32_t hb;         // PRODUCT: (h,T) entries per batch (a power of two <= 32; 0 means 32)
  int64_t e3_off;     // three-band model: first entry of the group's band tables
                      // (k + Q/2 at e3_off + k, -k + Q/2 at e3_off + N^2 + k)
  int64_t kst_off;    // FP32 k-state table: entry of (pair, k) at kst_off + pair N^2 + k
};

// PRODUCT batches are tiles of hb (h,T) entries x db = 32/hb Delta values:
// lane l holds Delta dblk db + l / hb and entry hblk hb + l % hb.  Batches run
// h-block-major, b = hblk n_dblk + dblk, so a work item (consecutive batches
// of one h-block) spans the h range of hb entries only.  hb = 32 is the plain
// layout: one Delta and 32 entries per batch.
__host__ __device__ inline int tile_hb(const GroupDesc& g) { return g.hb > 0 ? g.hb : 32; }
__host__ __device__ inline int tile_db(const GroupDesc& g) { return 32 / tile_hb(g); }
__host__ __device__ inline int tile_n_dblk(const GroupDesc& g) {
  const int db = tile_db(g);
  return (g.n_delta + db - 1) / db;
}
// Delta index and (h,T) entry of lane `lane` in PRODUCT batch b (in range or not).
__host__ __device__ inline void tile_pos(const GroupDesc& g, int b, int lane, int& di, int& hi) {
  const int hb = tile_hb(g), nd = tile_n_dblk(g);
  const int hblk = b / nd, dblk = b - hblk * nd;
  di = dblk * (32 / hb) + lane / hb;
  hi = hblk * hb + (lane & (hb - 1));
}
// Outputs of PRODUCT batch b that exist: (Delta rows) x (entries).
__host__ __device__ inline int tile_outputs(const GroupDesc& g, int b) {
  const int hb = tile_hb(g), db = 32 / hb, nd = tile_n_dblk(g);
  const int hblk = b / nd, dblk = b - hblk * nd;
  const int rows = g.n_delta - dblk * db < db ? g.n_delta - dblk * db : db;
  const int cols = g.n_ht - hblk * hb < hb ? g.n_ht - hblk * hb : hb;
  return rows * cols;
}

// Bands are evaluated two at a time, as the two halves of packed operations:
// the two-band model in one pair, the three-band model in two, (0, 1) and
// (2, inert).  Slot s of pair p holds band 2p + s.
__device__ __forceinline__ int band_pairs(int nbands) { return (nbands + 1) / 2; }
__device__ __forceinline__ bool slot_active(int nbands, int band_only, int pair, int slot) {
  const int b = 2 * pair + slot;
  return b < nbands && (band_only == 0 || band_only - 1 == b);
}

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
  // Delta^2 <= far_d2max for every output of the item (the scale of the
  // far-band moments, ksum.cu)
  float far_d2max;
  // Delta^2 >= sgl_d2min for every output; sgl_r = 27 ln2 Tmax (+ rounding
  // margin): a near band with R + |d| >= sgl_r for every output has
  // c (R + |d|) >= 27, so its factor (1 + 2^-c(R+|d|)) is exactly 1 in FP32
  // (see ksum.cu); sgl_r = +inf: no band is tested
  float sgl_d2min, sgl_r;
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
// The three bands of the three-band model at one momentum, ascending (FP64; the
// FP32 copy is a float4 with the same layout).
struct __align__(16) E3D {
  double x, y, z, pad;
};
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

// ---- three-band model (App. B): eigenvalues of its hopping matrix -------
// Its 3x3 hopping matrix has real T11, T22, T33, T12 and purely imaginary
// T13 = i x, T23 = i y; conjugating with diag(1, 1, i) turns it into the real
// symmetric matrix with off-diagonals T12, -x, -y and the same eigenvalues.
// One Jacobi rotation (Jacobi 1846; the rotation of Rutishauser's
// formulation) zeroing a_pq of a symmetric 3x3 matrix; r is the third index.
// The FP32 form (estimates only) takes the approximate divide, reciprocal
// square root and square root (x rsqrt(x)).
template <typename R>
__device__ __forceinline__ void jacobi_rotate(R& app, R& aqq, R& apq, R& arp, R& arq) {
  if (apq == (R)0) return;
  R t, c;
  if constexpr (sizeof(R) == 4) {
    const float theta = __fdividef(aqq - app, 2.0f * apq);
    if (fabsf(theta) > 1e18f) {  // theta^2 would overflow
      t = __fdividef(0.5f, theta);
    } else {
      const float q = theta * theta + 1.0f;
      t = __fdividef(theta >= 0.0f ? 1.0f : -1.0f, fabsf(theta) + q * rsqrtf(q));
    }
    c = rsqrtf(t * t + 1.0f);
  } else {
    const R theta = (aqq - app) / ((R)2 * apq);
    if (fabs(theta) > (R)1e150)  // theta^2 would overflow
      t = (R)0.5 / theta;
    else
      t = (theta >= (R)0 ? (R)1 : (R)-1) / (fabs(theta) + sqrt(theta * theta + (R)1));
    c = (R)1 / sqrt(t * t + (R)1);
  }
  const R s = t * c;
  app -= t * apq;
  aqq += t * apq;
  apq = (R)0;
  const R rp = c * arp - s * arq, rq = s * arp + c * arq;
  arp = rp;
  arq = rq;
}

// Cyclic Jacobi sweeps until the off-diagonal is `tol` of the diagonal
// (quadratic convergence: 3 to 4 sweeps); eigenvalues ascending.
template <typename R>
__device__ __forceinline__ void jacobi3(R a00, R a11, R a22, R a01, R a02, R a12, R tol, R& e0, R& e1, R& e2) {
  for (int sweep = 0; sweep < 8; ++sweep) {
    const R off = fabs(a01) + fabs(a02) + fabs(a12);
    if (off <= tol * (fabs(a00) + fabs(a11) + fabs(a22) + (R)1e-30)) break;
    jacobi_rotate<R>(a00, a11, a01, a02, a12);  // (p, q) = (0, 1), r = 2
    jacobi_rotate<R>(a00, a22, a02, a01, a12);  // (0, 2), r = 1
    jacobi_rotate<R>(a11, a22, a12, a01, a02);  // (1, 2), r = 0
  }
  const R lo = fmin(a00, fmin(a11, a22)), hi = fmax(a00, fmax(a11, a22));
  e0 = lo;
  e2 = hi;
  e1 = a00 + a11 + a22 - lo - hi;
}

// Eigenvalues, ascending, of the three-band matrix at momentum (cos, sin) of
// each axis, in FP64.  FP32 Jacobi gives estimates; two FP64 Newton steps on
// the characteristic polynomial det(A - x) = ((c2 - x) x - c1) x + c0 from
// the outer estimates give the outer eigenvalues and the trace the middle
// one (each step divides by the derivative through an FP32 reciprocal: the
// error still shrinks by a factor of ~1e-7 per step).  Where two estimates are
// closer than 1e-4 of the scale (the polynomial's roots are ill-conditioned
// there) or a Newton step is not small, FP64 Jacobi rotations to 1e-14 of the
// diagonal decide instead.
__device__ __forceinline__ void bands3_at(const ModelParams& m, double cx, double sx, double cy, double sy,
                                          double& e0, double& e1, double& e2) {
  const double c2x = 2.0 * cx * cx - 1.0, c2y = 2.0 * cy * cy - 1.0;
  const double a00 = 2.0 * m.t2 * cx + 2.0 * m.t1 * cy + 4.0 * m.t3 * cx * cy + 2.0 * m.t11 * (c2x - c2y) +
                     4.0 * m.t12 * c2x * c2y;
  const double a11 = 2.0 * m.t1 * cx + 2.0 * m.t2 * cy + 4.0 * m.t3 * cx * cy - 2.0 * m.t11 * (c2x - c2y) +
                     4.0 * m.t12 * c2x * c2y;
  const double a22 = m.eps0 + 2.0 * m.t5 * (cx + cy) + 4.0 * m.t6 * cx * cy + 2.0 * m.t9 * (c2x + c2y) +
                     4.0 * m.t10 * (c2x * cy + cx * c2y);
  const double a01 = 4.0 * m.t4 * sx * sy;
  const double a02 = -(2.0 * m.t7 * sx + 4.0 * m.t8 * sx * cy);
  const double a12 = -(2.0 * m.t7 * sy + 4.0 * m.t8 * sy * cx);
  float f0, f1, f2;
  jacobi3<float>((float)a00, (float)a11, (float)a22, (float)a01, (float)a02, (float)a12, 1e-6f, f0, f1, f2);
  const double scale = fmax(fabs((double)f0), fabs((double)f2)) + 1e-30;
  bool ok = fmin(f1 - f0, f2 - f1) >= 1e-4 * scale;
  if (ok) {
    const double c2 = a00 + a11 + a22;
    const double c1 = a00 * a11 + a00 * a22 + a11 * a22 - a01 * a01 - a02 * a02 - a12 * a12;
    const double c0 = a00 * (a11 * a22 - a12 * a12) - a01 * (a01 * a22 - a12 * a02) + a02 * (a01 * a12 - a11 * a02);
    double x[2] = {(double)f0, (double)f2};
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int it = 0; it < 2; ++it) {
        const double p = ((c2 - x[r]) * x[r] - c1) * x[r] + c0;
        const double dp = (2.0 * c2 - 3.0 * x[r]) * x[r] - c1;
        const double step = p * (double)__frcp_rn((float)dp);
        ok = ok && fabs(step) <= 1e-4 * scale;  // also false for NaN
        x[r] -= step;
      }
    e0 = x[0];
    e2 = x[1];
    e1 = c2 - x[0] - x[1];
  }
  if (!ok) jacobi3<double>(a00, a11, a22, a01, a02, a12, 1e-14, e0, e1, e2);
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

// Per-k state of two bands from their energies at k + Q/2 (u0, u1) and
// -k + Q/2 (d0, d1).
template <typename Real>
__device__ __forceinline__ void kstate_from_bands(const ModelParams& m, Real eta, Real u0, Real u1, Real d0,
                                                  Real d1, KState<Real>& st) {
  st.eta2 = eta * eta;
  const Real mu = (Real)m.mu;
  Real s0 = (Real)0.5 * (u0 + d0) - mu, s1 = (Real)0.5 * (u1 + d1) - mu;
  st.d0[0] = (Real)0.5 * (u0 - d0);
  st.d0[1] = (Real)0.5 * (u1 - d1);
  st.as[0] = fabs(s0);
  st.as[1] = fabs(s1);
  st.s2[0] = fmax(s0 * s0, (Real)1e-30);
  st.s2[1] = fmax(s1 * s1, (Real)1e-30);
}

template <typename Real, typename Row>
__device__ __forceinline__ void kstate_make(const ModelParams& m, const Row& rx, const Row& ry,
                                            Real c0x, Real c0y, KState<Real>& st) {
  Real eta = (Real)m.eta_amp * c0x * c0y;
  Real ulo, uhi, dlo, dhi;
  band_pair<Real>(m, (Real)rx.cp, (Real)ry.cp, (Real)rx.sp, (Real)ry.sp, ulo, uhi);  // k + Q/2
  band_pair<Real>(m, (Real)rx.cm, (Real)ry.cm, (Real)rx.sm, (Real)ry.sm, dlo, dhi);  // -k + Q/2
  kstate_from_bands<Real>(m, eta, ulo, uhi, dlo, dhi, st);
}

// A slot without an active band (one band of a pair selected, or the empty
// second slot of the three-band model's pair (2, -)) is made inert:
// |s| = 1e15, so no log term and a = Delta^2 eta^2 / 2e15 <= 2e-17 per k-point.
template <typename Real>
__device__ __forceinline__ void kstate_mask(KState<Real>& st, int nbands, int band_only, int pair) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
    if (!slot_active(nbands, band_only, pair, s)) {
      st.as[s] = (Real)1e15;
      st.s2[s] = (Real)1e30;
      st.d0[s] = (Real)0;
    }
}

// Band energies of the three-band model at one k: slots of pair p from the
// tables (float4 / double4 rows holding the three bands in ascending order).
template <typename Real, typename Row4>
__device__ __forceinline__ void kstate_from_table3(const ModelParams& m, Real eta, const Row4& eu, const Row4& ed,
                                                   int pair, KState<Real>& st) {
  if (pair == 0)
    kstate_from_bands<Real>(m, eta, (Real)eu.x, (Real)eu.y, (Real)ed.x, (Real)ed.y, st);
  else
    kstate_from_bands<Real>(m, eta, (Real)eu.z, (Real)eu.z, (Real)ed.z, (Real)ed.z, st);
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

// FP32 state of two (k-point, band) entries packed as the halves of float2
// operations: eta^2, |s|, s^2, d0.  Either the two bands of one k-point, or
// the near bands of two k-points.
struct KState32 {
  float2 eta2;
  float2 as, s2, d0;
};

// One float2 slot (two entries), one output, given y1 = c (R - d) and
// y2 = c (R + d) of each entry: adds c min(max(R - |d|, 0), a) of each entry
// to cp2 (R - |d| = min(R - d, R + d)) and multiplies each half of P2 by its
// entry's (1 + 2^-|y1|)(1 + 2^-|y2|), a factor in [1, 4] (the caller takes
// one lg2 of the product over its slots).  ac = a c per entry.
// SINGLE: both entries have c (R + |d|) >= 27, whose factor would leave the
// product unchanged (P + P e with P e below half an ulp of P), so only the
// factor of min(|y1|, |y2|) = c |R - |d|| is formed -- the same bits.
template <bool SINGLE>
__device__ __forceinline__ void w_term32(float2 y1, float2 y2, float2 ac, float2& P2, float2& cp2) {
  if constexpr (SINGLE) {
    const float2 e = make_float2(ex2a(fmaxf(-fabsf(y1.x), -fabsf(y2.x))), ex2a(fmaxf(-fabsf(y1.y), -fabsf(y2.y))));
    P2 = __ffma2_rn(P2, e, P2);
  } else {
    const float2 e1 = make_float2(ex2a(-fabsf(y1.x)), ex2a(-fabsf(y1.y)));
    const float2 e2 = make_float2(ex2a(-fabsf(y2.x)), ex2a(-fabsf(y2.y)));
    P2 = __ffma2_rn(P2, e1, P2);
    P2 = __ffma2_rn(P2, e2, P2);
  }
  const float2 cp = make_float2(fmaxf(min3f(y1.x, y2.x, ac.x), 0.0f), fmaxf(min3f(y1.y, y2.y, ac.y), 0.0f));
  cp2 = __fadd2_rn(cp2, cp);
}
__device__ __forceinline__ void ra_f64(double D, double s2, double as, double& R, double& a) {
  R = sqrt(D + s2);
  a = D / (R + as);
}

// FP64 band term for one (h,T): q = p - 1 = e1 + e2 + e1 e2 (kept as p - 1
// for log1p) and first = min(0, max(|d|-|s|, 0) - a).
// An exponential exp(-y) with y >= kExpNegligible = 40 is taken as 0 without
// evaluating it: e^-40 < 4.3e-18, so the band's -T ln(1 + q) term, which is
// then dropped, is below 3 e^-40 T < 1.3e-17 T, and the free energy per site
// changes by less than 3.9e-17 T (three bands) -- for T <= 1 below a fifth of
// one FP64 ulp of a per-site value of 1, and far below the rounding of the
// k-sum itself (its N^2 terms are added in FP64).
constexpr double kExpNegligible = 40.0;
__device__ __forceinline__ void band_term_f64(double R, double a, double as, double d0, double h,
                                              double inv_t, double& q, double& first) {
  double d = d0 - h;
  double ad = fabs(d);
  double x1 = fabs(R - ad);
  double x2 = R + ad;
  const double y1 = x1 * inv_t, y2 = x2 * inv_t;
  double e1 = 0.0, e2 = 0.0;
  if (y1 < kExpNegligible) e1 = exp(-y1);
  if (y2 < kExpNegligible) e2 = exp(-y2);
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
