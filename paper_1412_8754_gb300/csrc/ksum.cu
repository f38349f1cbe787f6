// ksum.cu -- the k-sum of Eq. freeene (Sec. 2) as one persistent map-reduce.
//
// Each warp repeatedly takes a work item (group, k-set range, output-batch
// range) from a global atomic queue.  For every k-set of 32*KPT lattice points
// it loads the per-k band states (|s|, d0 per band, eta^2) from the FP32
// k-state table that kstate_table_kernel writes once per execution (or, for
// plans too large for the table, builds them from the trig tables: App. A
// band energies at k+Q/2 and -k+Q/2).  FP32: each band is classified against
// the item's window -- far bands (every log factor 1 in FP32) add c a, summed
// per batch; near bands are compacted into a per-warp buffer and, 64*KPT at a
// time, evaluated with the full term for every output of the item.  Per-lane
// sums of a batch's 32 outputs are folded into one value per output through a
// 32 x 36 transpose buffer in shared memory.  The warp keeps FP64
// accumulators per output in shared memory; at the end of the item it writes
// them as one partial per output and the last warp to finish a segment (a
// fixed output range) adds the partials of all its k-chunks in a fixed order
// (deterministic) and writes
//   Omega = M + V + N^2 Delta^2 sum_bands 1/U_band
// together with an error bound for FP32 evaluation.  This replaces the
// paper's per-block partial sums + second reduction kernel + host-side
// remainder (Sec. 3, Alg. 2 and the three steps around it) by one launch.
#include <type_traits>

#include "ffe_internal.cuh"
#include "ksum.cuh"

namespace ffe {

// A warp's (k-point, band) entry buffers: a flush takes 64 KPT entries (two
// per float2 slot) and a k-set adds at most 64 KPT, so 128 KPT entries each.
__host__ __device__ constexpr int kbuf_entries(int kpt) { return 128 * kpt; }

// Batch parameters staged in shared memory, one entry per output of a batch.
struct BParF {  // FP32: Delta^2, h, c = 1/(T ln 2), c h
  float d2, h, c, ch;
};
struct BParD {  // FP64: Delta^2 (LIST only), h, 1/T, T
  double d2, h, inv_t, t;
};

template <typename Real>
using BPar = typename std::conditional<std::is_same<Real, float>::value, BParF, BParD>::type;

template <typename Real>
__device__ __forceinline__ void load_row(const KsumArgs& a, int64_t row, TabRowF& r, float& c0) {
  r = a.tabf[row];
  c0 = a.c0f[row];
}
template <typename Real>
__device__ __forceinline__ void load_row(const KsumArgs& a, int64_t row, TabRowD& r, double& c0) {
  r = a.tabd[row];
  c0 = a.c0d[row];
}

// The state of lattice point kidx = iy N + ix (< N^2 <= 2^26) of group g for band pair `pair`.
template <typename Real>
__device__ __forceinline__ void state_at_xy(const KsumArgs& a, const GroupDesc& g, int ix, int iy, int kidx,
                                            int pair, KState<Real>& st) {
  using Row = typename std::conditional<std::is_same<Real, float>::value, TabRowF, TabRowD>::type;
  Row rx, ry;
  Real c0x, c0y;
  load_row<Real>(a, g.tab_off + ix, rx, c0x);
  load_row<Real>(a, g.tab_off + g.N + iy, ry, c0y);
  if (a.m.nbands == 3) {
    const Real eta = (Real)a.m.eta_amp * c0x * c0y;
    const int64_t nk = (int64_t)g.N * g.N;
    if constexpr (std::is_same<Real, float>::value)
      kstate_from_table3<float, float4>(a.m, eta, a.e3f[g.e3_off + kidx], a.e3f[g.e3_off + nk + kidx], pair, st);
    else
      kstate_from_table3<double, E3D>(a.m, eta, a.e3d[g.e3_off + kidx], a.e3d[g.e3_off + nk + kidx], pair, st);
  } else {
    kstate_make<Real, Row>(a.m, rx, ry, c0x, c0y, st);
  }
  kstate_mask<Real>(st, a.m.nbands, g.band_only, pair);
}

template <typename Real>
__device__ __forceinline__ void state_at(const KsumArgs& a, const GroupDesc& g, int kidx, int pair,
                                         KState<Real>& st) {
  const int iy = kidx / g.N;
  state_at_xy<Real>(a, g, kidx - iy * g.N, iy, kidx, pair, st);
}

// The lane's KPT states of k-set ks: points ks 32 KPT + 32 j + lane; one
// division, then the lattice coordinates advance by 32.
template <typename Real, int KPT>
__device__ __forceinline__ void build_states(const KsumArgs& a, const GroupDesc& g, int ks, int lane, int pair,
                                             KState<Real> (&st)[KPT]) {
  const int nk = g.N * g.N;
  const int k0 = ks * (32 * KPT) + lane;
  int iy = k0 / g.N, ix = k0 - iy * g.N;
#pragma unroll
  for (int j = 0; j < KPT; ++j) {
    const int kidx = k0 + j * 32;
    if (kidx < nk)
      state_at_xy<Real>(a, g, ix, iy, kidx, pair, st[j]);
    else
      kstate_invalid<Real>(st[j]);
    ix += 32;
    while (ix >= g.N) {
      ix -= g.N;
      ++iy;
    }
  }
}

// Stage the parameters of batch b (32 outputs) into this warp's shared slot.
// Returns the number of rows to evaluate: LIST, the valid outputs (a prefix);
// PRODUCT, up to the last valid lane (a lane inside that range whose entry
// lies past n_ht is staged with c = 0 and its row is ignored).  delta_i:
// PRODUCT, the Delta of lane 0 (the batch's Delta when hb = 32).
template <typename Real, int LAYOUT>
__device__ __forceinline__ int stage_batch(const KsumArgs& a, const GroupDesc& g, int b, int lane,
                                           BPar<Real>* bp, int& delta_i) {
  int nvalid;
  bool valid;
  int64_t ht_e, d_e;
  if (LAYOUT == kLayoutProduct) {
    const int hb = tile_hb(g);
    int di, hi, di0, hi0;
    tile_pos(g, b, lane, di, hi);
    tile_pos(g, b, 0, di0, hi0);
    delta_i = di0;
    const int rows = min(32 / hb, g.n_delta - di0), cols = min(hb, g.n_ht - hi0);
    nvalid = (rows - 1) * hb + cols;
    valid = di < g.n_delta && hi < g.n_ht;
    ht_e = g.ht_off + hi;
    d_e = g.delta_off + di;
  } else {
    delta_i = -1;
    const int o0 = b * 32;
    nvalid = min(32, g.n_out - o0);
    valid = lane < nvalid;
    ht_e = g.ht_off + o0 + lane;
    d_e = g.delta_off + o0 + lane;
  }
  __syncwarp();
  BPar<Real> p;
  if (valid) {
    if constexpr (std::is_same<Real, float>::value) {
      const HTf q = a.htf[ht_e];
      p.d2 = a.d2f[d_e];
      p.h = q.h;
      p.c = q.c;
      p.ch = q.c * q.h;
    } else {
      const HTd q = a.htd[ht_e];
      const double dd = a.delta[d_e];
      p.d2 = dd * dd;
      p.h = q.h;
      p.inv_t = q.inv_t;
      p.t = q.t;
    }
  } else {
    p.d2 = 0;
    p.h = 0;
    if constexpr (std::is_same<Real, float>::value) {
      p.c = 0;
      p.ch = 0;
    } else {
      p.inv_t = 0;
      p.t = 0;
    }
  }
  bp[lane] = p;
  __syncwarp();
  return nvalid;
}

// ------------------------------------------------------------ FP32 path
template <int KPT>
__device__ __forceinline__ void build_states32(const KsumArgs& a, const GroupDesc& g, int ks, int lane, int pair,
                                               KState32 (&st)[KPT]) {
  if (a.kst4) {  // from the k-state table (s^2 = |s|^2 exactly, as built)
    const int nk = g.N * g.N;
    const int k0 = ks * (32 * KPT) + lane;
    const int64_t base = g.kst_off + (int64_t)pair * nk;
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
      const int kidx = k0 + j * 32;
      if (kidx < nk) {
        const float4 v = a.kst4[base + kidx];
        const float e = a.kste[base + kidx];
        st[j].eta2 = make_float2(e, e);
        st[j].as = make_float2(v.x, v.y);
        st[j].s2 = make_float2(fmaxf(v.x * v.x, 1e-30f), fmaxf(v.y * v.y, 1e-30f));
        st[j].d0 = make_float2(v.z, v.w);
      } else {
        st[j].eta2 = make_float2(0.0f, 0.0f);
        st[j].as = make_float2(1e15f, 1e15f);
        st[j].s2 = make_float2(1e30f, 1e30f);
        st[j].d0 = make_float2(0.0f, 0.0f);
      }
    }
    return;
  }
  KState<float> s[KPT];
  build_states<float, KPT>(a, g, ks, lane, pair, s);
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    st[k].eta2 = make_float2(s[k].eta2, s[k].eta2);
    st[k].as = make_float2(s[k].as[0], s[k].as[1]);
    st[k].s2 = make_float2(s[k].s2[0], s[k].s2[1]);
    st[k].d0 = make_float2(s[k].d0[0], s[k].d0[1]);
  }
}

// A buffered (k-point, band) entry: lattice index | band pair << kPairBit |
// band slot << kSlotBit (lattice index < 8192^2 = 2^26).
constexpr int kPairBit = 27, kSlotBit = 28;
constexpr int32_t kKidxMask = (1 << 26) - 1;

// One band of one entry: eta^2, |s|, s^2, d0; an inert band past the end.
struct Band32 {
  float eta2, as, s2, d0;
};

__device__ __forceinline__ Band32 band32_at(const KsumArgs& a, const GroupDesc& g, int32_t e) {
  const int b = (e >> kSlotBit) & 1;
  if (a.kst4) {  // from the k-state table
    const int64_t o = g.kst_off + (int64_t)((e >> kPairBit) & 1) * g.N * g.N + (e & kKidxMask);
    const float4 v = a.kst4[o];
    const float as = b ? v.y : v.x;
    return Band32{a.kste[o], as, fmaxf(as * as, 1e-30f), b ? v.w : v.z};
  }
  KState<float> s;
  state_at<float>(a, g, e & kKidxMask, (e >> kPairBit) & 1, s);
  return Band32{s.eta2, s.as[b], s.s2[b], s.d0[b]};
}

__device__ __forceinline__ Band32 band32_inert() { return Band32{0.0f, 1e15f, 1e30f, 0.0f}; }

// Single band: c (R + |d|) >= 27 for every output of the item (R + |d| >=
// sgl_r, from R^2 >= s^2 + Delta_min^2 eta^2 and |d| >= the distance of d0
// from [hlo, hhi]), so its second factor (1 + 2^-c(R + |d|)) is 1 in FP32 and
// one exponential, of min(|y1|, |y2|) = c |R - |d||, gives its term.  The
// inert band counts as single.
__device__ __forceinline__ bool single_band32(const Band32& b, const WorkItem& w) {
  const float t = w.sgl_r - fmaxf(0.0f, fmaxf(w.far_hlo - b.d0, b.d0 - w.far_hhi));
  return t <= 0.0f || fmaf(w.sgl_d2min, b.eta2, b.s2) >= t * t;
}

__device__ __forceinline__ KState32 pack32(const Band32& x, const Band32& y) {
  KState32 t;
  t.eta2 = make_float2(x.eta2, y.eta2);
  t.as = make_float2(x.as, y.as);
  t.s2 = make_float2(x.s2, y.s2);
  t.d0 = make_float2(x.d0, y.d0);
  return t;
}

// Far band (see api.cu, item_far_window): for every output of the item the
// band has c |R -+ d| >= 27, so its W is c a exactly in FP32.
__device__ __forceinline__ bool far_band32(float as, float d0, const WorkItem& w) {
  return as - fmaxf(fabsf(d0 - w.far_hlo), fabsf(d0 - w.far_hhi)) >= w.far_tgap;
}

// Blocked band: for every output of the item |d| - R >= far_tgap, with
// |d| = |d0 - h| >= its distance from [far_hlo, far_hhi] and
// R^2 <= s^2 + far_d2max eta^2.  Then c |R -+ d| >= 27 for both signs, so both
// factors (1 + 2^-c|R -+ d|) leave the FP32 product unchanged, and
// min(c (R - d), c (R + d), c a) = c (R - |d|) < 0 clamps to 0: the band adds
// nothing to W, the same bits as its full term.  (The pair state is
// "blocked": one member below and one above the chemical potential by more
// than the window.)  The squares are compared with a relative margin of
// 2^-20 for their FP32 rounding.
__device__ __forceinline__ bool blocked_band32(float d0, float eta2, float s2, const WorkItem& w) {
  const float m = fmaxf(0.0f, fmaxf(w.far_hlo - d0, d0 - w.far_hhi)) - w.far_tgap;
  return m > 0.0f && m * m >= fmaf(w.far_d2max, eta2, s2) * (1.0f + 0x1p-20f);
}

// R and a = Delta^2 eta^2 / (R + |s|) of both halves at Delta^2 = d2.
__device__ __forceinline__ void ra32(const KState32& st, float d2, float2& R, float2& A) {
  const float2 D2 = __fmul2_rn(make_float2(d2, d2), st.eta2);
  const float2 u = __fadd2_rn(D2, st.s2);
  R = __fmul2_rn(u, make_float2(rsqa(u.x), rsqa(u.y)));
  const float2 den = __fadd2_rn(R, st.as);
  A = __fmul2_rn(D2, make_float2(rcpa(den.x), rcpa(den.y)));
}

// W of one output summed over this lane's KPT slots: the clamp terms plus
// one lg2 of the product of all (1 + e) factors (each half of P2 at most
// 4^KPT, the product at most 16^KPT <= 2^32).  Rc = R c, Ac = a c per slot;
// y1 = c (R - d), y2 = c (R + d) with d = d0 - h.
// SINGLE: only the factor of x = min(y1, y2) = c R - c |d| differs from 1; x is
// formed directly by one fused multiply-add per band (the same rounding as the
// smaller of y1 and y2, so the same bits as the two-sided form) and enters as
// 2^-|x| and max(min(x, c a), 0).
template <int KPT, bool SINGLE>
__device__ __forceinline__ float w_out32(const KState32 (&st)[KPT], const float2 (&Rc)[KPT],
                                         const float2 (&Ac)[KPT], float h, float c) {
  const float2 nh2 = make_float2(-h, -h), c2 = make_float2(c, c), nc2 = make_float2(-c, -c);
  float2 cp2 = make_float2(0.0f, 0.0f), P2 = make_float2(1.0f, 1.0f);
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const float2 d = __fadd2_rn(st[k].d0, nh2);
    if constexpr (SINGLE) {
      const float x0 = fmaf(-c, fabsf(d.x), Rc[k].x), x1 = fmaf(-c, fabsf(d.y), Rc[k].y);
      P2 = __ffma2_rn(P2, make_float2(ex2a(-fabsf(x0)), ex2a(-fabsf(x1))), P2);
      cp2 = __fadd2_rn(cp2, make_float2(fmaxf(fminf(x0, Ac[k].x), 0.0f), fmaxf(fminf(x1, Ac[k].y), 0.0f)));
    } else {
      w_term32<false>(__ffma2_rn(d, nc2, Rc[k]), __ffma2_rn(d, c2, Rc[k]), Ac[k], P2, cp2);
    }
  }
  return (cp2.x + cp2.y) + lg2a(P2.x * P2.y);
}

// The same for one c shared by the batch, from A1 = c (R - d0) and
// A2 = c (R + d0) per slot: y1 = A1 + c h, y2 = A2 - c h.
template <int KPT, bool SINGLE>
__device__ __forceinline__ float w_out32_ut(const float2 (&A1)[KPT], const float2 (&A2)[KPT],
                                            const float2 (&Ac)[KPT], float ch) {
  const float2 ch2 = make_float2(ch, ch), nch2 = make_float2(-ch, -ch);
  float2 cp2 = make_float2(0.0f, 0.0f), P2 = make_float2(1.0f, 1.0f);
#pragma unroll
  for (int k = 0; k < KPT; ++k) w_term32<SINGLE>(__fadd2_rn(A1[k], ch2), __fadd2_rn(A2[k], nch2), Ac[k], P2, cp2);
  return (cp2.x + cp2.y) + lg2a(P2.x * P2.y);
}

// Lane l: the sum of row l of the warp's transpose buffer (0 for l >= nvalid).
__device__ __forceinline__ float transposed_total(float* red, int nvalid, int lane) {
  __syncwarp();
  float tot = 0.0f;
  if (lane < nvalid) {
    const float4* row = reinterpret_cast<const float4*>(red + lane * 36);
    float4 s4 = row[0];
#pragma unroll
    for (int i = 1; i < 8; ++i) {
      const float4 v = row[i];
      s4.x += v.x;
      s4.y += v.y;
      s4.z += v.z;
      s4.w += v.w;
    }
    tot = (s4.x + s4.y) + (s4.z + s4.w);
  }
  __syncwarp();
  return tot;
}

// Far bands with y = Delta_max^2 eta^2 / s^2 <= kSeriesY (Delta_max^2 =
// far_d2max bounds Delta^2 of every output of the item): by the binomial
// series of a = R - |s| = |s| (sqrt(1 + x) - 1), x = Delta^2 eta^2 / s^2 =
// t y with t = Delta^2 / Delta_max^2 <= 1,
//   a = |s| sum_n alpha_n x^n = sum_n alpha_n t^n |s| y^n,
//   alpha = 1/2, -1/8, 1/16, -5/128, 7/256, -21/1024 (n = 1..6; the next term,
// 33/2048 x^7, is below 3.3e-8 of the first for y <= 0.1), so the far sum of
// every output is the same six moments M_n = sum_k |s_k| y_k^n, weighted by
// alpha_n t^n: the k-sum is taken once per item (LIST) or k-set (shared
// Delta), not once per output.
constexpr int kMoments = 6;
constexpr float kSeriesY = 0.1f;
// Kahan's compensated summation: s + x with the rounding error carried in c
// (the sum is s - c); additions only, so nothing is fused or reordered.
__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}
__device__ __forceinline__ void moments_add(float as, float y, float (&pm)[kMoments]) {
  float t = as * y;
#pragma unroll
  for (int n = 0; n < kMoments; ++n) {
    pm[n] += t;
    t *= y;
  }
}
__device__ __forceinline__ double moments_sum(const double (&M)[kMoments], double t) {
  constexpr double alpha[kMoments] = {0.5, -0.125, 0.0625, -5.0 / 128.0, 7.0 / 256.0, -21.0 / 1024.0};
  double r = alpha[kMoments - 1] * M[kMoments - 1];
#pragma unroll
  for (int n = kMoments - 2; n >= 0; --n) r = alpha[n] * M[n] + t * r;
  return t * r;
}

// One batch of up to 32 outputs.  Output j's per-lane sum goes to row j of
// the warp's transpose buffer `red` (row stride 36 floats); lane l then adds
// row l.  The output loop stays rolled (small code); returns in lane l the
// warp total of output l (0 for l >= nvalid).  Shared-T batches (ProductUT)
// are tiles of rows of hb outputs sharing a Delta: R and a once per row.
template <int KPT, int VARIANT, bool SINGLE>
__device__ __forceinline__ float eval_batch32(const KState32 (&st)[KPT], const BParF* bp, int nvalid,
                                              float d2_product, int lane, float* red, int hb = 32) {
  if (VARIANT == kLayoutProductUT) {
    const float c = bp[0].c;
    const float2 c2 = make_float2(c, c), nc2 = make_float2(-c, -c);
    for (int j0 = 0; j0 < nvalid; j0 += hb) {
      const float d2 = bp[j0].d2;
      float2 A1[KPT], A2[KPT], Ac[KPT];
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        float2 R, A;
        ra32(st[k], d2, R, A);
        const float2 Rc = __fmul2_rn(R, c2);
        A1[k] = __ffma2_rn(st[k].d0, nc2, Rc);
        A2[k] = __ffma2_rn(st[k].d0, c2, Rc);
        Ac[k] = __fmul2_rn(A, c2);
      }
      const int j1 = min(nvalid, j0 + hb);
      // four outputs in flight at 2 k-points per thread; two at 4 (registers)
#pragma unroll(KPT <= 2 ? 4 : 2)
      for (int j = j0; j < j1; ++j) red[j * 36 + lane] = w_out32_ut<KPT, SINGLE>(A1, A2, Ac, bp[j].ch);
    }
  } else if (VARIANT == kLayoutProduct) {
    float2 R[KPT], A[KPT];
#pragma unroll
    for (int k = 0; k < KPT; ++k) ra32(st[k], d2_product, R[k], A[k]);
#pragma unroll 2
    for (int j = 0; j < nvalid; ++j) {
      const BParF p = bp[j];
      const float2 c2 = make_float2(p.c, p.c);
      float2 Rc[KPT], Ac[KPT];
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        Rc[k] = __fmul2_rn(R[k], c2);
        Ac[k] = __fmul2_rn(A[k], c2);
      }
      red[j * 36 + lane] = w_out32<KPT, SINGLE>(st, Rc, Ac, p.h, p.c);
    }
  } else {
#pragma unroll 2
    for (int j = 0; j < nvalid; ++j) {
      const BParF p = bp[j];
      const float2 c2 = make_float2(p.c, p.c);
      float2 Rc[KPT], Ac[KPT];
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        float2 R, A;
        ra32(st[k], p.d2, R, A);
        Rc[k] = __fmul2_rn(R, c2);
        Ac[k] = __fmul2_rn(A, c2);
      }
      red[j * 36 + lane] = w_out32<KPT, SINGLE>(st, Rc, Ac, p.h, p.c);
    }
  }
  return transposed_total(red, nvalid, lane);
}

// Far k-points of a LIST batch: W = c (a_0 + a_1) per output and k-point;
// with one Delta for the whole batch (uniform), a once per k-point.
template <int KPT>
__device__ __forceinline__ float eval_far32(const KState32 (&st)[KPT], const BParF* bp, int nvalid, int lane,
                                            float* red, bool uniform) {
  if (uniform) {
    float2 S = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      float2 R, A;
      ra32(st[k], bp[0].d2, R, A);
      S = __fadd2_rn(S, A);
    }
    const float s = S.x + S.y;
#pragma unroll 4
    for (int j = 0; j < nvalid; ++j) red[j * 36 + lane] = bp[j].c * s;
    return transposed_total(red, nvalid, lane);
  }
#pragma unroll 2
  for (int j = 0; j < nvalid; ++j) {
    const BParF p = bp[j];
    float2 S = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      float2 R, A;
      ra32(st[k], p.d2, R, A);
      S = __fadd2_rn(S, A);
    }
    red[j * 36 + lane] = p.c * (S.x + S.y);
  }
  return transposed_total(red, nvalid, lane);
}

// FP64 far band: for every output of the item |R -+ d| / T >= kExpNegligible
// (window as in the FP32 path, threshold kExpNegligible T_max), so both
// exponentials are taken as 0 (band_term_f64) and the band's term is -a.
__device__ __forceinline__ bool far_band64(double as, double d0, const WorkItem& w) {
  return as - fmax(fabs(d0 - (double)w.far_hlo), fabs(d0 - (double)w.far_hhi)) >= (double)w.far_tgap;
}

// FP64 blocked band: |d| - R >= kExpNegligible T_max for every output of the
// item (as blocked_band32), so both exponentials are taken as 0 and the clamp
// term min(max(|d| - |s|, 0) - a, 0) = min(|d| - R, 0) is 0: the band's term
// is exactly 0.
__device__ __forceinline__ bool blocked_band64(double d0, double eta2, double s2, const WorkItem& w) {
  const double m = fmax(0.0, fmax((double)w.far_hlo - d0, d0 - (double)w.far_hhi)) - (double)w.far_tgap;
  return m > 0.0 && m * m >= fma((double)w.far_d2max, eta2, s2) * (1.0 + 0x1p-40);
}

// FP64 near-band entries per warp buffer: a flush takes 64 (two per lane), a
// k-set adds at most 64 KPT, the remainder after flushing is below 64.
__host__ __device__ constexpr int kbuf64_entries(int kpt) { return 64 + 64 * kpt; }

// One buffered near (k-point, band) entry of a lane in FP64: |s|, s^2, d0,
// eta^2 (an empty slot: a band far above every window, which adds nothing).
struct Ent64 {
  double as = 1e15, s2 = 1e30, d0 = 0.0, eta2 = 0.0;
};

// Lane l: the sum of row l (32 doubles, in order) of the warp's FP64 transpose
// buffer (row stride 33), 0 for l >= nrows.
__device__ __forceinline__ double row_total64(const double* red, int nrows, int lane) {
  __syncwarp();
  double t = 0.0;
  if (lane < nrows)
#pragma unroll 8
    for (int i = 0; i < 32; ++i) t += red[lane * 33 + i];
  __syncwarp();
  return t;
}

// Split exponentials.  With P = R - d0 + h and M = R + d0 - h (P + M = 2R >= 0)
// the two arguments of band_term_f64 are {|R - |d||, R + |d|} = {|P|, |M|},
// and for a batch whose outputs share T,
//   e^{-|P|/T} = e^{-alpha} e^{-eta}  (P >= 0),  e^{alpha} e^{eta}  (P < 0),
//   e^{-|M|/T} = e^{-beta} e^{eta}    (M >= 0),  e^{beta} e^{-eta}  (M < 0),
// alpha = (R - d0)/T, beta = (R + d0)/T per entry, eta = h/T per output: four
// exponentials per entry and two per output for the whole batch instead of two
// per (entry, output).  With |eta| <= 600 every factor taken is finite: a
// factor e^{-alpha} is used only where alpha >= -eta >= -600 (the arguments
// are capped at 700, so an unused one never overflows), and one that
// underflows belongs to an argument |P|/T or |M|/T beyond kExpNegligible,
// which is 0 anyway.  Rounding: each factor and the product are within a few
// ulp; the arguments' own rounding (the cancellation in R - d0, scaled by 1/T)
// is of the same size as in the direct form.
__device__ __forceinline__ bool split_exp_batch(const BParD* bp, int nvalid, int lane) {
  const BParD p0 = bp[0];
  const bool ok = lane >= nvalid || (bp[lane].t == p0.t && fabs(bp[lane].h * p0.inv_t) <= 600.0);
  return __all_sync(kFull, ok);
}

// |x| >= kExpNegligible (40) from the high word of x: the order of the bit
// patterns of non-negative doubles is their numeric order.
static_assert(kExpNegligible == 40.0, "beyond_exp40 compares against the high word of 40.0");
__device__ __forceinline__ bool beyond_exp40(double x) {
  return (__double2hiint(x) & 0x7fffffff) >= 0x40440000;  // high word of 40.0 (low word 0)
}

// flush64's band terms of one shared-T batch by split exponentials: the lane's
// two entries (R, A at the batch's Delta) on every output j, their two log
// factors under one log1p (log1p(q0) + log1p(q1) = log1p(q0 + q1 + q0 q1)),
// into red[j][lane].
__device__ __forceinline__ void flush64_split(const BParD* bp, int nvalid, int lane, const bool (&live)[2],
                                              const double (&R)[2], const double (&A)[2], const Ent64 (&en)[2],
                                              double* red) {
  const double it = bp[0].inv_t, t = bp[0].t;
  const double eta_l = lane < nvalid ? bp[lane].h * it : 0.0;
  const double xp_l = exp(eta_l), xm_l = exp(-eta_l);  // this lane's output: e^{eta}, e^{-eta}
  double al[2], be[2], eam[2], eap[2], ebm[2], ebp[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    al[u] = (R[u] - en[u].d0) * it;
    be[u] = (R[u] + en[u].d0) * it;
    eam[u] = exp(fmin(-al[u], 700.0));
    eap[u] = exp(fmin(al[u], 700.0));
    ebm[u] = exp(fmin(-be[u], 700.0));
    ebp[u] = exp(fmin(be[u], 700.0));
  }
  for (int j = 0; j < nvalid; ++j) {
    const double xp = __shfl_sync(kFull, xp_l, j), xm = __shfl_sync(kFull, xm_l, j);
    const double h = bp[j].h;
    const double eta = h * it;  // the same bits as output j's lane computed
    double f = 0.0, q = 0.0;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!live[u]) continue;
      const double ps = al[u] + eta, ms = be[u] - eta;
      double e1 = __double2hiint(ps) >= 0 ? eam[u] * xm : eap[u] * xp;
      double e2 = __double2hiint(ms) >= 0 ? ebm[u] * xp : ebp[u] * xm;
      if (beyond_exp40(ps)) e1 = 0.0;
      if (beyond_exp40(ms)) e2 = 0.0;
      const double qu = e1 + e2 + e1 * e2;
      q = q + qu + q * qu;
      f += fmin(fmax(fabs(en[u].d0 - h) - en[u].as, 0.0) - A[u], 0.0);
    }
    red[j * 33 + lane] = q == 0.0 ? f : f - t * log1p(q);
  }
}

// FP64 evaluation of up to 64 buffered near (k-point, band) entries, entries
// lane and lane + 32 of each lane, on every output of the item (PRODUCT
// batches that share T: by split exponentials, flush64_split):
// v = min(max(|d| - |s|, 0) - a, 0) - T ln(1 + q) per band, q = e1 + e2 + e1 e2;
// the lane's two entries add their logarithms under one log1p.
template <int LAYOUT>
__device__ __forceinline__ void flush64(const KsumArgs& a, const WorkItem& w, const GroupDesc& g, int lane,
                                        const int32_t* buf, int n, double* acc, BParD* bp, double* red) {
  constexpr int kG = (LAYOUT == kLayoutList) ? kLayoutList : kLayoutProduct;
  bool live[2];
  Ent64 en[2];
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int i = lane + 32 * u;
    live[u] = i < n;
    if (live[u]) {
      const int32_t e = buf[i];
      KState<double> st;
      state_at<double>(a, g, e & kKidxMask, (e >> kPairBit) & 1, st);
      const int sl = (e >> kSlotBit) & 1;
      en[u].as = st.as[sl];
      en[u].s2 = st.s2[sl];
      en[u].d0 = st.d0[sl];
      en[u].eta2 = st.eta2;
    }
  }
  for (int b = w.b0; b < w.b1; ++b) {
    int di;
    const int nvalid = stage_batch<double, kG>(a, g, b, lane, bp, di);
    double R[2] = {0.0, 0.0}, A[2] = {0.0, 0.0};
    if (kG == kLayoutProduct) {
      const double dd = a.delta[g.delta_off + di];
#pragma unroll
      for (int u = 0; u < 2; ++u) ra_f64(dd * dd * en[u].eta2, en[u].s2, en[u].as, R[u], A[u]);
      if (split_exp_batch(bp, nvalid, lane)) {
        flush64_split(bp, nvalid, lane, live, R, A, en, red);
        const double t = row_total64(red, nvalid, lane);
        if (lane < nvalid) acc[(b - w.b0) * 32 + lane] += t;
        continue;
      }
    }
    for (int j = 0; j < nvalid; ++j) {
      const BParD p = bp[j];
      double f = 0.0, q = 0.0;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (!live[u]) continue;
        if (kG == kLayoutList) ra_f64(p.d2 * en[u].eta2, en[u].s2, en[u].as, R[u], A[u]);
        double qu, fu;
        band_term_f64(R[u], A[u], en[u].as, en[u].d0, p.h, p.inv_t, qu, fu);
        q = q + qu + q * qu;
        f += fu;
      }
      red[j * 33 + lane] = q == 0.0 ? f : f - p.t * log1p(q);
    }
    const double t = row_total64(red, nvalid, lane);
    if (lane < nvalid) acc[(b - w.b0) * 32 + lane] += t;
  }
}

// One work item in FP64.  Every band of every k-point is classified per lane:
// far (its term is -a exactly, far_band64), blocked (its term is 0,
// blocked_band64) or near.  Far bands form a once per
// (k-point, Delta) -- per batch with a shared Delta (PRODUCT), per output
// (LIST) -- and their warp sums go through the transpose buffer; near bands
// are compacted (ballot + prefix count) into the warp's buffer and evaluated
// in full, 32 at a time, on every output.  Only near bands pay the
// exponentials and the logarithm.
template <int KPT, int LAYOUT>
__device__ __forceinline__ void item64(const KsumArgs& a, const WorkItem& w, const GroupDesc& g, int lane,
                                       double* acc, BParD* bp, double* red, int32_t* nbuf) {
  constexpr int kG = (LAYOUT == kLayoutList) ? kLayoutList : kLayoutProduct;
  const int64_t nk = (int64_t)g.N * g.N;
  const unsigned lt = (1u << lane) - 1u;
  const int nb = w.b1 - w.b0;
  int n_near = 0;
  double far_acc = 0.0;  // PRODUCT: lane b - b0 holds batch b's sum of a over far bands
  for (int ks = w.kset0; ks < w.kset1; ++ks)
  for (int pair = 0; pair < band_pairs(a.m.nbands); ++pair) {
    KState<double> st[KPT];
    build_states<double, KPT>(a, g, ks, lane, pair, st);
    const bool act0 = slot_active(a.m.nbands, g.band_only, pair, 0);
    const bool act1 = slot_active(a.m.nbands, g.band_only, pair, 1);
    bool far[KPT][2], near[KPT][2];
    int32_t kidx[KPT];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      kidx[k] = ks * (32 * KPT) + k * 32 + lane;
      const bool valid = kidx[k] < nk;
#pragma unroll
      for (int sl = 0; sl < 2; ++sl) {
        const bool use = valid && (sl == 0 ? act0 : act1);
        far[k][sl] = use && far_band64(st[k].as[sl], st[k].d0[sl], w);
        near[k][sl] = use && !far[k][sl] && !blocked_band64(st[k].d0[sl], st[k].eta2, st[k].s2[sl], w);
      }
    }
    if (__any_sync(kFull, far[0][0] || far[0][1] || (KPT > 1 && (far[KPT - 1][0] || far[KPT - 1][1])))) {
      if (kG == kLayoutProduct) {
        for (int b = w.b0; b < w.b1; ++b) {
          int di0, hi0;  // hb = 32 in FP64 plans: one Delta per batch
          tile_pos(g, b, 0, di0, hi0);
          const double dd = a.delta[g.delta_off + di0];
          double S = 0.0;
#pragma unroll
          for (int k = 0; k < KPT; ++k)
#pragma unroll
            for (int sl = 0; sl < 2; ++sl)
              if (far[k][sl]) {
                double R, A;
                ra_f64(dd * dd * st[k].eta2, st[k].s2[sl], st[k].as[sl], R, A);
                S += A;
              }
          red[(b - w.b0) * 33 + lane] = S;
        }
        far_acc += row_total64(red, nb, lane);
      } else {
        for (int b = w.b0; b < w.b1; ++b) {
          int di;
          const int nvalid = stage_batch<double, kG>(a, g, b, lane, bp, di);
          for (int j = 0; j < nvalid; ++j) {
            const double d2 = bp[j].d2;
            double S = 0.0;
#pragma unroll
            for (int k = 0; k < KPT; ++k)
#pragma unroll
              for (int sl = 0; sl < 2; ++sl)
                if (far[k][sl]) {
                  double R, A;
                  ra_f64(d2 * st[k].eta2, st[k].s2[sl], st[k].as[sl], R, A);
                  S += A;
                }
            red[j * 33 + lane] = S;
          }
          const double t = row_total64(red, nvalid, lane);
          if (lane < nvalid) acc[(b - w.b0) * 32 + lane] -= t;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < KPT; ++k)
#pragma unroll
      for (int sl = 0; sl < 2; ++sl) {
        const unsigned m = __ballot_sync(kFull, near[k][sl]);
        if (near[k][sl]) nbuf[n_near + __popc(m & lt)] = kidx[k] | (pair << kPairBit) | (sl << kSlotBit);
        n_near += __popc(m);
      }
    __syncwarp();
    int done = 0;
    for (; n_near - done >= 64; done += 64) flush64<LAYOUT>(a, w, g, lane, nbuf + done, 64, acc, bp, red);
    if (done > 0) {
      __syncwarp();
      // fewer than 64 left, moved from [done, ...) to [0, ...): done >= 64, so the ranges do not overlap
      for (int i = lane; i < n_near - done; i += 32) nbuf[i] = nbuf[done + i];
      __syncwarp();
      n_near -= done;
    }
  }
  if (n_near > 0) flush64<LAYOUT>(a, w, g, lane, nbuf, n_near, acc, bp, red);
  if (kG == kLayoutProduct)
    for (int b = w.b0; b < w.b1; ++b) acc[(b - w.b0) * 32 + lane] -= __shfl_sync(kFull, far_acc, b - w.b0);
  __syncwarp();
}

// Output index (within the group) of lane `lane` in batch b, or -1.
__device__ __forceinline__ int batch_output(const GroupDesc& g, int b, int lane, int& delta_i,
                                            int& ht_i) {
  if (g.layout == kLayoutProduct) {
    tile_pos(g, b, lane, delta_i, ht_i);
    if (ht_i >= g.n_ht || delta_i >= g.n_delta) return -1;
    return delta_i * g.n_ht + ht_i;
  }
  const int o = b * 32 + lane;
  if (o >= g.n_out) return -1;
  delta_i = o;
  ht_i = o;
  return o;
}

// Last warp of a segment: add the chunk partials in chunk order and finish.
__device__ void finalize_segment(const KsumArgs& a, const Segment& sg, const GroupDesc& g, int lane) {
  const int nb = sg.b1 - sg.b0;
  const double n2 = (double)g.N * (double)g.N;
  for (int b = sg.b0; b < sg.b1; ++b) {
    int di, hi;
    const int o = batch_output(g, b, lane, di, hi);
    if (o < 0) continue;
    const double* src = a.partials + sg.partial_off + (int64_t)(b - sg.b0) * 32 + lane;
    double V = 0.0;
    for (int c = 0; c < sg.n_chunks; ++c) V += __ldcg(src + (int64_t)c * nb * 32);
    const double dl = a.delta[g.delta_off + di];
    const HT ht = a.ht[g.ht_off + hi];
    if (a.w_scaled) V *= -ht.T * 0.69314718055994530942;  // W -> sum_k v_k
    const double M = a.M[g.h_off + ht.h_idx];
    const int64_t out = g.out_off + o;
    a.V[out] = V;
    a.omega[out] = M + V + pairing_term(a.m, g.band_only, n2, dl);
    a.ebound[out] = a.eb_rel * fabs(V) + a.eb_abs * n2 * ht.T;
  }
}

// Shared-T items (kLayoutProductUT): the item's batch parameters, staged once per
// item in the warp's batch-parameter slot as floats -- c = 1/(T ln 2) (one T for
// the item: its batches are tiles of one h-block), c h of the h-block's hb <= 8
// entries (0 past n_ht) and Delta^2 of its nd_item <= kMaxTileDeltas Delta rows.
constexpr int kUtMaxHb = 8, kUtCh = 1, kUtD2 = 1 + kUtMaxHb;
static_assert(kUtD2 + kMaxTileDeltas <= 32 * (int)(sizeof(BParF) / sizeof(float)),
              "shared-T item parameters exceed the batch-parameter slot");

__device__ __forceinline__ void stage_item_ut(const KsumArgs& a, const GroupDesc& g, const WorkItem& w, int lane,
                                              int dbase, int nd_item, float* ip) {
  const int hb = tile_hb(g);
  const int e0 = (w.b0 / tile_n_dblk(g)) * hb;  // first (h,T) entry of the item's h-block
  const int cols = min(hb, g.n_ht - e0);
  __syncwarp();
  if (lane < hb) {
    float c = 0.0f, ch = 0.0f;
    if (lane < cols) {
      const HTf q = a.htf[g.ht_off + e0 + lane];
      c = q.c;
      ch = q.c * q.h;
    }
    ip[kUtCh + lane] = ch;
    if (lane == 0) ip[0] = c;
  }
  for (int r = lane; r < nd_item; r += 32) ip[kUtD2 + r] = a.d2f[g.delta_off + dbase + r];
  __syncwarp();
}

// W of one output summed over this lane's KPT slots when every band of the warp
// is single (single_band32): the one factor that differs from 1 is
// 1 + 2^-|x| with x = min(y1, y2) = c (R - |d|) (R >= 0 gives
// min(|y1|, |y2|) = |x|), and the clamp term is max(min(x, c a), 0).  From
// Rc = c R, D0c = c d0 and Ac = c a per slot: x = Rc - |D0c - c h|.
template <int KPT>
__device__ __forceinline__ float w_out32_x(const float2 (&Rc)[KPT], const float2 (&D0c)[KPT],
                                           const float2 (&Ac)[KPT], float ch) {
  const float2 nch2 = make_float2(-ch, -ch);
  float2 cp2 = make_float2(0.0f, 0.0f), P2 = make_float2(1.0f, 1.0f);
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const float2 t = __fadd2_rn(D0c[k], nch2);  // c d
    const float x0 = Rc[k].x - fabsf(t.x), x1 = Rc[k].y - fabsf(t.y);
    P2 = __ffma2_rn(P2, make_float2(ex2a(-fabsf(x0)), ex2a(-fabsf(x1))), P2);
    cp2 = __fadd2_rn(cp2, make_float2(fmaxf(fminf(x0, Ac[k].x), 0.0f), fmaxf(fminf(x1, Ac[k].y), 0.0f)));
  }
  return (cp2.x + cp2.y) + lg2a(P2.x * P2.y);
}

// Near entries of a shared-T item on each of its batches: per Delta row R and a
// once per slot, then the hb outputs of the row (single bands: from c R, c d0
// and c a; otherwise from A1 = c (R - d0), A2 = c (R + d0) and c a); the
// batch's per-lane sums go through the transpose buffer into acc.
template <int KPT, bool SINGLE>
__device__ __forceinline__ void flush_batches_ut(const KState32 (&st)[KPT], const WorkItem& w, const GroupDesc& g,
                                                 int lane, const float* ip, int nd_item, double* acc, float* red) {
  const int hb = tile_hb(g), db = 32 / hb;
  const int cols = min(hb, g.n_ht - (w.b0 / tile_n_dblk(g)) * hb);
  const float c = ip[0];
  const float2 c2 = make_float2(c, c), nc2 = make_float2(-c, -c);
  float2 D0c[KPT];
#pragma unroll
  for (int k = 0; k < KPT; ++k) D0c[k] = __fmul2_rn(st[k].d0, c2);
  for (int b = w.b0; b < w.b1; ++b) {
    const int rb = (b - w.b0) * db;  // the batch's first Delta row in the item
    const int rows = min(db, nd_item - rb);
    const int nvalid = (rows - 1) * hb + cols;
    for (int r = 0; r < rows; ++r) {
      const float d2 = ip[kUtD2 + rb + r];
      const int j0 = r * hb, j1 = min(nvalid, j0 + hb);
      if constexpr (SINGLE) {
        float2 Rc[KPT], Ac[KPT];
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
          float2 R, A;
          ra32(st[k], d2, R, A);
          Rc[k] = __fmul2_rn(R, c2);
          Ac[k] = __fmul2_rn(A, c2);
        }
#pragma unroll 2
        for (int j = j0; j < j1; ++j) red[j * 36 + lane] = w_out32_x<KPT>(Rc, D0c, Ac, ip[kUtCh + j - j0]);
      } else {
        float2 A1[KPT], A2[KPT], Ac[KPT];
#pragma unroll
        for (int k = 0; k < KPT; ++k) {
          float2 R, A;
          ra32(st[k], d2, R, A);
          const float2 Rc = __fmul2_rn(R, c2);
          A1[k] = __ffma2_rn(st[k].d0, nc2, Rc);
          A2[k] = __ffma2_rn(st[k].d0, c2, Rc);
          Ac[k] = __fmul2_rn(A, c2);
        }
#pragma unroll(KPT <= 2 ? 4 : 2)
        for (int j = j0; j < j1; ++j) red[j * 36 + lane] = w_out32_ut<KPT, false>(A1, A2, Ac, ip[kUtCh + j - j0]);
      }
    }
    acc[(b - w.b0) * 32 + lane] += (double)transposed_total(red, nvalid, lane);
  }
}

// FP32 evaluation of n buffered (k-point, band) entries on every batch of the
// item, two entries per float2 slot: the full term, or the far form W = c a.
template <int KPT, int LAYOUT, bool FAR>
__device__ __forceinline__ void flush32(const KsumArgs& a, const WorkItem& w, const GroupDesc& g, int lane,
                                        const int32_t* buf, int n, double* acc, BParF* bp, float* red,
                                        int nd_item = 0) {
  constexpr int kG = (LAYOUT == kLayoutList) ? kLayoutList : kLayoutProduct;
  KState32 st[KPT];
  bool sgl = true;  // every entry of this lane single (padding counts as single)
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int i0 = 2 * k * 32 + lane, i1 = i0 + 32;
    const Band32 x = i0 < n ? band32_at(a, g, buf[i0]) : band32_inert();
    const Band32 y = i1 < n ? band32_at(a, g, buf[i1]) : band32_inert();
    if (!FAR) sgl = sgl && single_band32(x, w) && single_band32(y, w);
    st[k] = pack32(x, y);
  }
  const bool single = __all_sync(kFull, sgl);  // warp-uniform: one ex2 per near band
  int64_t outs = 0;
  if constexpr (LAYOUT == kLayoutProductUT && !FAR) {  // parameters staged per item (stage_item_ut)
    const float* ip = reinterpret_cast<const float*>(bp);
    if (single)
      flush_batches_ut<KPT, true>(st, w, g, lane, ip, nd_item, acc, red);
    else
      flush_batches_ut<KPT, false>(st, w, g, lane, ip, nd_item, acc, red);
    if (a.near_evals && lane == 0) {
      for (int b = w.b0; b < w.b1; ++b) outs += tile_outputs(g, b);
      atomicAdd(a.near_evals, (unsigned long long)(n * outs));
      if (single) atomicAdd(a.near_evals + 1, (unsigned long long)(n * outs));
    }
    return;
  }
  const int hb = tile_hb(g);
  for (int b = w.b0; b < w.b1; ++b) {
    int di;
    const int nvalid = stage_batch<float, kG>(a, g, b, lane, bp, di);
    outs += kG == kLayoutList ? nvalid : tile_outputs(g, b);
    float tot;
    // LIST: a batch whose outputs share Delta (a golden-section search whose lines took the same
    // decisions, a reference at Delta = 0) forms R and a once per slot, and with one T too takes
    // the shared-T form of the scans
    bool uni_d = false, uni_c = false;
    if constexpr (kG == kLayoutList) {
      const BParF p0 = bp[0], pl = bp[lane];
      uni_d = __all_sync(kFull, lane >= nvalid || pl.d2 == p0.d2);
      uni_c = __all_sync(kFull, lane >= nvalid || pl.c == p0.c);
    }
    if constexpr (FAR) {
      tot = eval_far32<KPT>(st, bp, nvalid, lane, red, uni_d);
    } else if constexpr (kG == kLayoutList) {
      const float d2u = bp[0].d2;
      if (uni_d && uni_c)
        tot = single ? eval_batch32<KPT, kLayoutProductUT, true>(st, bp, nvalid, d2u, lane, red)
                     : eval_batch32<KPT, kLayoutProductUT, false>(st, bp, nvalid, d2u, lane, red);
      else
        tot = single ? eval_batch32<KPT, LAYOUT, true>(st, bp, nvalid, 0.0f, lane, red)
                     : eval_batch32<KPT, LAYOUT, false>(st, bp, nvalid, 0.0f, lane, red);
    } else {
      const float d2p = a.d2f[g.delta_off + di];  // hb = 32 (plain PRODUCT): the batch's Delta
      tot = single ? eval_batch32<KPT, LAYOUT, true>(st, bp, nvalid, d2p, lane, red, hb)
                   : eval_batch32<KPT, LAYOUT, false>(st, bp, nvalid, d2p, lane, red, hb);
    }
    acc[(b - w.b0) * 32 + lane] += (double)tot;
  }
  if (a.near_evals && lane == 0) {
    if (FAR) {
      atomicAdd(a.near_evals + 2, (unsigned long long)(n * outs));
    } else {
      atomicAdd(a.near_evals, (unsigned long long)(n * outs));
      if (single) atomicAdd(a.near_evals + 1, (unsigned long long)(n * outs));
    }
  }
}

// PRODUCT far bands outside the series range (closed form): n buffered
// entries, two per float2 slot.  For each of the item's Delta values r (the
// Delta rows dbase + r, r < nd_item <= kMaxTileDeltas) the warp's sum of a
// over the entries is added, through the transpose buffer, to fsum[r] (the
// warp's FP64 far sums in shared memory); each output later adds c times its
// Delta's sum.
template <int KPT>
__device__ __forceinline__ void flush_far_product(const KsumArgs& a, const WorkItem& w, const GroupDesc& g, int lane,
                                                  const int32_t* buf, int n, float* red, int dbase, int nd_item,
                                                  double* fsum) {
  KState32 st[KPT];
#pragma unroll
  for (int k = 0; k < KPT; ++k) {
    const int i0 = 2 * k * 32 + lane, i1 = i0 + 32;
    st[k] = pack32(i0 < n ? band32_at(a, g, buf[i0]) : band32_inert(),
                   i1 < n ? band32_at(a, g, buf[i1]) : band32_inert());
  }
  for (int r0 = 0; r0 < nd_item; r0 += 32) {
    const int r1 = min(nd_item, r0 + 32);
#pragma unroll 2
    for (int r = r0; r < r1; ++r) {
      const float d2 = a.d2f[g.delta_off + dbase + r];
      float2 S = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        float2 R, A;
        ra32(st[k], d2, R, A);
        S = __fadd2_rn(S, A);
      }
      red[(r - r0) * 36 + lane] = S.x + S.y;
    }
    const float tot = transposed_total(red, r1 - r0, lane);  // lane r - r0: Delta r
    if (lane < r1 - r0) fsum[r0 + lane] += (double)tot;
  }
  if (a.near_evals && lane == 0) {
    int64_t outs = 0;
    for (int b = w.b0; b < w.b1; ++b) outs += tile_outputs(g, b);
    atomicAdd(a.near_evals + 2, (unsigned long long)((int64_t)n * outs));
  }
}

// Drops the first `done` entries of a warp's buffer of n entries.
__device__ __forceinline__ void buffer_shift(int32_t* buf, int done, int n, int lane) {
  __syncwarp();
  for (int i = lane; i < n - done; i += 32) buf[i] = buf[done + i];  // n - done < done: no overlap
  __syncwarp();
}

// One work item in FP32.  Every band of every k-point of a k-set is "far"
// (far_band32: for all outputs of the item its log terms are 1 in FP32 and
// W = c a), "blocked" (blocked_band32: W = 0, skipped) or "near".  Far bands cost, per batch, their R and a: with a
// shared Delta (PRODUCT layouts) their a is summed over the warp once per
// batch and applied as c (sum) to every output at the end; with a Delta per
// output (LIST) they are buffered and evaluated per output in the far form.
// Near bands are buffered as (k-point, band) entries and, once 64 KPT of
// them are collected, evaluated with the full term for every output, two
// entries per float2 slot -- at a near k-point usually one band is near, so
// this halves the full-term work against evaluating whole k-points.
template <int KPT, int LAYOUT>
__device__ __forceinline__ void item32(const KsumArgs& a, const WorkItem& w, const GroupDesc& g, int lane,
                                       double* acc, BParF* bp, float* red, int32_t* nbuf, int32_t* fbuf,
                                       double* mom) {
  constexpr int kG = (LAYOUT == kLayoutList) ? kLayoutList : kLayoutProduct;
  constexpr int kFlush = 64 * KPT;
  const int64_t nk = (int64_t)g.N * g.N;
  const unsigned lt = (1u << lane) - 1u;
  int n_near = 0, n_far = 0;  // LIST: far entries in closed form (fbuf) or in the moments (mom)
  if constexpr (kG == kLayoutList)
#pragma unroll
    for (int n = 0; n < kMoments; ++n) mom[n * 32 + lane] = 0.0;
  // PRODUCT: the item's Delta values are dbase + r, r < nd_item <=
  // kMaxTileDeltas (one h-block, consecutive Delta rows); fsum[r] (shared
  // memory, per warp) holds the FP64 far sum of Delta r
  double* fsum = mom;
  int dbase = 0, nd_item = 0;
  if constexpr (kG == kLayoutProduct) {
    const int db = tile_db(g);
    dbase = (w.b0 % tile_n_dblk(g)) * db;
    nd_item = min(g.n_delta - dbase, (w.b1 - w.b0) * db);
    for (int r = lane; r < kMaxTileDeltas; r += 32) fsum[r] = 0.0;
    if constexpr (LAYOUT == kLayoutProductUT) stage_item_ut(a, g, w, lane, dbase, nd_item, reinterpret_cast<float*>(bp));
  }
  float msum[kMoments], mcomp[kMoments];  // PRODUCT: this lane's moments (sum, compensation)
#pragma unroll
  for (int n = 0; n < kMoments; ++n) msum[n] = mcomp[n] = 0.0f;
  const int npairs = band_pairs(a.m.nbands);
  for (int ks = w.kset0; ks < w.kset1; ++ks)
  for (int pair = 0; pair < npairs; ++pair) {
    KState32 st[KPT];
    build_states32<KPT>(a, g, ks, lane, pair, st);
    const bool act0 = slot_active(a.m.nbands, g.band_only, pair, 0);
    const bool act1 = slot_active(a.m.nbands, g.band_only, pair, 1);
    float pm[kMoments] = {};  // LIST: this k-set's moments, this lane
    bool any_ser = false;
    bool far0[KPT], far1[KPT], valid[KPT];
    int32_t kidx[KPT];
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
      kidx[k] = ks * (32 * KPT) + k * 32 + lane;
      valid[k] = kidx[k] < nk;
      far0[k] = !act0 || !valid[k] || far_band32(st[k].as.x, st[k].d0.x, w);
      far1[k] = !act1 || !valid[k] || far_band32(st[k].as.y, st[k].d0.y, w);
    }
    if constexpr (kG == kLayoutProduct) {
      // Far bands in the series range (y = Delta_max^2 eta^2 / s^2 <= kSeriesY):
      // this lane's six moments, summed over the item's k-sets with Kahan's
      // compensation and over the warp at the end of the item.  The other far
      // bands go to the closed-form buffer.
      float2 pm2[kMoments];
#pragma unroll
      for (int n = 0; n < kMoments; ++n) pm2[n] = make_float2(0.0f, 0.0f);
      const float2 dmx = make_float2(w.far_d2max, w.far_d2max);
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
        const bool f0 = far0[k] && act0 && valid[k], f1 = far1[k] && act1 && valid[k];
        const bool s0 = f0 && st[k].eta2.x * w.far_d2max <= kSeriesY * st[k].s2.x;
        const bool s1 = f1 && st[k].eta2.y * w.far_d2max <= kSeriesY * st[k].s2.y;
        const float2 y = __fmul2_rn(__fmul2_rn(st[k].eta2, dmx), make_float2(rcpa(st[k].s2.x), rcpa(st[k].s2.y)));
        float2 tt = __fmul2_rn(make_float2(s0 ? st[k].as.x : 0.0f, s1 ? st[k].as.y : 0.0f), y);
#pragma unroll
        for (int n = 0; n < kMoments; ++n) {
          pm2[n] = __fadd2_rn(pm2[n], tt);
          tt = __fmul2_rn(tt, y);
        }
      }
#pragma unroll
      for (int n = 0; n < kMoments; ++n) kahan_add(msum[n], mcomp[n], pm2[n].x + pm2[n].y);
    }
    // near bands and far bands in the closed form are appended to their buffers; most k-sets
    // hold neither (they cluster where the lattice row crosses a Fermi line), and the warp
    // then skips the ballots
    bool nr[KPT][2], cf[KPT][2];
    bool any_buf = false;
#pragma unroll
    for (int k = 0; k < KPT; ++k) {
#pragma unroll
      for (int sl = 0; sl < 2; ++sl) {
        const bool fr = sl == 0 ? far0[k] : far1[k];
        const bool act = sl == 0 ? act0 : act1;
        const float eta2 = sl == 0 ? st[k].eta2.x : st[k].eta2.y;
        const float s2 = sl == 0 ? st[k].s2.x : st[k].s2.y;
        const float d0 = sl == 0 ? st[k].d0.x : st[k].d0.y;
        nr[k][sl] = !fr && !blocked_band32(d0, eta2, s2, w);  // near implies active and valid
        const bool fe = fr && act && valid[k];
        const bool ser = fe && eta2 * w.far_d2max <= kSeriesY * s2;  // into the moments
        cf[k][sl] = fe && !ser;
        any_buf = any_buf || nr[k][sl] || cf[k][sl];
        if constexpr (kG == kLayoutList) {
          if (ser) {
            moments_add(sl == 0 ? st[k].as.x : st[k].as.y, __fdividef(eta2 * w.far_d2max, s2), pm);
            any_ser = true;
          }
        }
      }
    }
    if (__any_sync(kFull, any_buf)) {
#pragma unroll
      for (int k = 0; k < KPT; ++k) {
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
          const int32_t e = kidx[k] | (pair << kPairBit) | (sl << kSlotBit);
          const unsigned m = __ballot_sync(kFull, nr[k][sl]);
          if (nr[k][sl]) nbuf[n_near + __popc(m & lt)] = e;
          n_near += __popc(m);
          const unsigned mf = __ballot_sync(kFull, cf[k][sl]);
          if (cf[k][sl]) fbuf[n_far + __popc(mf & lt)] = e;
          n_far += __popc(mf);
        }
      }
    }
    if constexpr (kG == kLayoutList) {  // FP32 within a k-set, FP64 across k-sets
      if (__any_sync(kFull, any_ser))
#pragma unroll
        for (int n = 0; n < kMoments; ++n) mom[n * 32 + lane] += (double)pm[n];
    }
    __syncwarp();
    if (n_near >= kFlush) {
      flush32<KPT, LAYOUT, false>(a, w, g, lane, nbuf, kFlush, acc, bp, red, nd_item);
      buffer_shift(nbuf, kFlush, n_near, lane);
      n_near -= kFlush;
    }
    if (n_far >= kFlush) {
      if constexpr (kG == kLayoutList)
        flush32<KPT, LAYOUT, true>(a, w, g, lane, fbuf, kFlush, acc, bp, red);
      else
        flush_far_product<KPT>(a, w, g, lane, fbuf, kFlush, red, dbase, nd_item, fsum);
      buffer_shift(fbuf, kFlush, n_far, lane);
      n_far -= kFlush;
    }
  }
  if (n_near > 0) flush32<KPT, LAYOUT, false>(a, w, g, lane, nbuf, n_near, acc, bp, red, nd_item);
  if constexpr (kG == kLayoutProduct) {
    if (n_far > 0) flush_far_product<KPT>(a, w, g, lane, fbuf, n_far, red, dbase, nd_item, fsum);
  }
  if constexpr (kG == kLayoutList) {
    if (n_far > 0) flush32<KPT, LAYOUT, true>(a, w, g, lane, fbuf, n_far, acc, bp, red);
    // the moments' warp totals, then per output c sum_n alpha_n t^n M_n
    double M[kMoments];
    bool any = false;
#pragma unroll
    for (int n = 0; n < kMoments; ++n) {
      double v = mom[n * 32 + lane];
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
      M[n] = v;
      any = any || v != 0.0;
    }
    if (any) {
      const double inv_d2max = 1.0 / (double)w.far_d2max;
      for (int b = w.b0; b < w.b1; ++b) {
        int di;
        stage_batch<float, kG>(a, g, b, lane, bp, di);
        const int o = b * 32 + lane;
        if (o < g.n_out) {
          const double d = a.delta[g.delta_off + o];
          acc[(b - w.b0) * 32 + lane] += (double)bp[lane].c * moments_sum(M, d * d * inv_d2max);
        }
      }
    }
  } else {
    // the moments' warp totals (FP64), then per Delta r of the item
    // fsum[r] += sum_n alpha_n t^n M_n, t = Delta_r^2 / Delta_max^2
    double M[kMoments];
    bool any = false;
#pragma unroll
    for (int n = 0; n < kMoments; ++n) {
      double v = (double)msum[n] - (double)mcomp[n];
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
      M[n] = v;
      any = any || v != 0.0;
    }
    if (any) {
      const double inv_d2max = 1.0 / (double)w.far_d2max;
      for (int r = lane; r < nd_item; r += 32)
        fsum[r] += moments_sum(M, (double)a.d2f[g.delta_off + dbase + r] * inv_d2max);
    }
    const int hb = tile_hb(g), db = 32 / hb;
    __syncwarp();
    for (int b = w.b0; b < w.b1; ++b) {
      int di;
      stage_batch<float, kG>(a, g, b, lane, bp, di);
      const int r = min(kMaxTileDeltas - 1, (b - w.b0) * db + lane / hb);  // this output's Delta in the item
      acc[(b - w.b0) * 32 + lane] += (double)bp[lane].c * fsum[r];  // c = 0 without an output
    }
  }
  __syncwarp();
}

template <typename Real, int KPT, int LAYOUT>
__global__ void __launch_bounds__(256, (sizeof(Real) == 4 ? KPT <= 4 : KPT == 1) ? 2 : 1) ksum_kernel(const KsumArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  constexpr int kGroupLayout = (LAYOUT == kLayoutList) ? kLayoutList : kLayoutProduct;
  constexpr int kMB = max_batches(kGroupLayout, std::is_same<Real, float>::value);
  double* acc = reinterpret_cast<double*>(smem_raw) + (size_t)warp * (kMB * 32);
  unsigned char* after_acc = smem_raw + (size_t)nwarps * kMB * 32 * sizeof(double);
  BPar<Real>* bp = reinterpret_cast<BPar<Real>*>(after_acc) + warp * 32;
  // FP32 only: per-warp 32 x 36 transpose buffer of the output reduction and
  // the entry buffers (near, far closed form), kbuf_entries(KPT) each
  unsigned char* after_bp = after_acc + (size_t)nwarps * 32 * sizeof(BPar<Real>);
  float* red = reinterpret_cast<float*>(after_bp) + warp * 32 * 36;
  constexpr int kBufs = 2;  // near, far closed form
  int32_t* nbuf = reinterpret_cast<int32_t*>(after_bp + (size_t)nwarps * 32 * 36 * sizeof(float)) +
                  (size_t)warp * kBufs * kbuf_entries(KPT);
  int32_t* fbuf = nbuf + (kBufs > 1 ? 1 : 0) * kbuf_entries(KPT);
  // LIST: per-lane FP64 far-band moments, kMoments x 32 per warp; PRODUCT:
  // the FP64 far sums of the item's (at most 64) Delta values
  constexpr int kMomStride = (LAYOUT == kLayoutList) ? kMoments * 32 : kMaxTileDeltas;
  double* mom = reinterpret_cast<double*>(after_bp + (size_t)nwarps * 32 * 36 * sizeof(float) +
                                          (size_t)nwarps * kBufs * kbuf_entries(KPT) * sizeof(int32_t)) +
                (size_t)warp * kMomStride;
  // FP64 only: per-warp 32 x 33 transpose buffer and near-entry buffer
  double* red64 = reinterpret_cast<double*>(after_bp) + (size_t)warp * 32 * 33;
  if constexpr (!std::is_same<Real, float>::value)
    nbuf = reinterpret_cast<int32_t*>(after_bp + (size_t)nwarps * 32 * 33 * sizeof(double)) +
           (size_t)warp * kbuf64_entries(KPT);
  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(a.queue, 1);
    it = __shfl_sync(kFull, it, 0);
    if (it >= a.n_items) break;
    const WorkItem w = a.items[it];
    const GroupDesc g = a.groups[w.group];
    const int nb = w.b1 - w.b0;
    const bool bad_tile = kGroupLayout == kLayoutProduct &&
                          (w.b0 / tile_n_dblk(g) != (w.b1 - 1) / tile_n_dblk(g) ||
                           nb * tile_db(g) > (std::is_same<Real, float>::value ? kMaxTileDeltas : 32) ||
                           (LAYOUT == kLayoutProductUT && tile_hb(g) > kUtMaxHb));
    if (nb > kMB || g.layout != kGroupLayout || bad_tile) {
      if (lane == 0) atomicOr(a.status, 1);
      continue;
    }
    for (int b = 0; b < nb; ++b) acc[b * 32 + lane] = 0.0;
    if constexpr (std::is_same<Real, float>::value)
      item32<KPT, LAYOUT>(a, w, g, lane, acc, bp, red, nbuf, fbuf, mom);
    else
      item64<KPT, LAYOUT>(a, w, g, lane, acc, bp, red64, nbuf);
    const Segment sg = a.segs[w.seg];
    double* dst = a.partials + sg.partial_off + (int64_t)w.chunk * nb * 32;
    for (int b = 0; b < nb; ++b) dst[b * 32 + lane] = acc[b * 32 + lane];
    __threadfence();
    __syncwarp();
    int prev = 0;
    if (lane == 0) prev = atomicAdd(a.seg_count + w.seg, 1);
    prev = __shfl_sync(kFull, prev, 0);
    if (prev == sg.n_chunks - 1) {
      __threadfence();
      finalize_segment(a, sg, g, lane);
      __syncwarp();
      if (lane == 0) a.seg_count[w.seg] = 0;  // ready for the next launch
    }
  }
}

// The FP32 state of every (group, band pair, lattice point) -- the values
// the k-sum would otherwise rebuild in each of its segments -- as |s| and d0
// of both slots (float4) and eta^2.  Grid: (k blocks, group, pair).
__global__ void __launch_bounds__(256) kstate_table_kernel(const KsumArgs a) {
  const GroupDesc g = a.groups[blockIdx.y];
  const int pair = blockIdx.z;
  const int nk = g.N * g.N;
  const int64_t base = g.kst_off + (int64_t)pair * nk;
  for (int k = blockIdx.x * 256 + threadIdx.x; k < nk; k += gridDim.x * 256) {
    KState<float> st;
    state_at<float>(a, g, k, pair, st);
    a.kst4[base + k] = make_float4(st.as[0], st.as[1], st.d0[0], st.d0[1]);
    a.kste[base + k] = st.eta2;
  }
}

cudaError_t kstate_table_launch(const KsumArgs& a, int n_groups, int max_n, cudaStream_t s) {
  if (n_groups < 1 || n_groups > 65535) return cudaErrorInvalidValue;
  const int64_t nk = (int64_t)max_n * max_n;
  const int bx = (int)std::min<int64_t>((nk + 255) / 256, 1024);
  kstate_table_kernel<<<dim3(bx, n_groups, (a.m.nbands + 1) / 2), 256, 0, s>>>(a);
  return cudaGetLastError();
}

size_t ksum_smem_bytes(int prec, int layout, int kpt, int block_threads) {
  const int nw = block_threads / 32;
  const size_t par = (prec == 1) ? sizeof(BParF) : sizeof(BParD);
  const int bufs = 2;
  const size_t mom = (layout == kLayoutList ? (size_t)kMoments * 32 : kMaxTileDeltas) * sizeof(double);
  const size_t red = (prec == 1) ? 32 * 36 * sizeof(float) + (size_t)bufs * kbuf_entries(kpt) * sizeof(int32_t) + mom
                                 : 32 * 33 * sizeof(double) + (size_t)kbuf64_entries(kpt) * sizeof(int32_t);
  const int mb = max_batches(layout == kLayoutList ? kLayoutList : kLayoutProduct, prec == 1);
  return (size_t)nw * (mb * 32 * sizeof(double) + 32 * par + red);
}

template <typename Real, int KPT, int LAYOUT>
static cudaError_t launch_one(const KsumArgs& a, int grid, int block, size_t smem, cudaStream_t s) {
  auto k = ksum_kernel<Real, KPT, LAYOUT>;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  if (cs == cudaStreamCaptureStatusNone) {  // during capture the attribute is already set (occupancy query)
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename Real, int KPT, int LAYOUT>
static cudaError_t occupancy_one(int block, size_t smem, int* blocks_per_sm) {
  auto k = ksum_kernel<Real, KPT, LAYOUT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, block, smem);
}

#define FFE_KSUM_DISPATCH(FN, ...)                                                         \
  do {                                                                                     \
    if (prec == 1) {                                                                       \
      if (layout == kLayoutProductUT) {                                                    \
        if (kpt == 2) return FN<float, 2, kLayoutProductUT>(__VA_ARGS__);                  \
        if (kpt == 4) return FN<float, 4, kLayoutProductUT>(__VA_ARGS__);                  \
        if (kpt == 8) return FN<float, 8, kLayoutProductUT>(__VA_ARGS__);                  \
      } else if (layout == kLayoutProduct) {                                               \
        if (kpt == 2) return FN<float, 2, kLayoutProduct>(__VA_ARGS__);                    \
        if (kpt == 4) return FN<float, 4, kLayoutProduct>(__VA_ARGS__);                    \
        if (kpt == 8) return FN<float, 8, kLayoutProduct>(__VA_ARGS__);                    \
      } else {                                                                             \
        if (kpt == 2) return FN<float, 2, kLayoutList>(__VA_ARGS__);                       \
        if (kpt == 4) return FN<float, 4, kLayoutList>(__VA_ARGS__);                       \
        if (kpt == 8) return FN<float, 8, kLayoutList>(__VA_ARGS__);                       \
      }                                                                                    \
    } else {                                                                               \
      if (layout != kLayoutList) {                                                         \
        if (kpt == 1) return FN<double, 1, kLayoutProduct>(__VA_ARGS__);                   \
        if (kpt == 2) return FN<double, 2, kLayoutProduct>(__VA_ARGS__);                   \
      } else {                                                                             \
        if (kpt == 1) return FN<double, 1, kLayoutList>(__VA_ARGS__);                      \
        if (kpt == 2) return FN<double, 2, kLayoutList>(__VA_ARGS__);                      \
      }                                                                                    \
    }                                                                                      \
    return cudaErrorInvalidValue;                                                          \
  } while (0)

cudaError_t ksum_launch(int prec, int layout, int kpt, const KsumArgs& a, int grid, int block,
                        cudaStream_t s) {
  const size_t smem = ksum_smem_bytes(prec, layout, kpt, block);
  FFE_KSUM_DISPATCH(launch_one, a, grid, block, smem, s);
}

cudaError_t ksum_occupancy(int prec, int layout, int kpt, int block, int* blocks_per_sm) {
  const size_t smem = ksum_smem_bytes(prec, layout, kpt, block);
  FFE_KSUM_DISPATCH(occupancy_one, block, smem, blocks_per_sm);
}

bool ksum_kpt_supported(int prec, int kpt) {
  return prec == 1 ? (kpt == 2 || kpt == 4 || kpt == 8) : (kpt == 1 || kpt == 2);
}

}  // namespace ffe
