// FP32 evaluation of the collocation entries (MIXED precision).
//
// Same rules and singular treatments as the FP64 functions of entry.cuh
// (Sec. 2.3; Duffy for x on the element, CPV and free term for centroid
// rows, rigid-body static diagonal for node rows), with every quadrature
// point in FP32: B300 issues about 2 FP64 FMA per clock per SM against 128
// FP32, and the near/singular rules (64-768 points) are the costliest
// entries.  Accuracy is kept by (i) the series branch up to |s| r / c2 < 2,
// (ii) geometry relative to the collocation point (differences formed once
// per element in FP64, then rounded), (iii) two-level summation: plain FP32
// over at most 16 points, then compensated (Kahan) accumulation.
//
// Every function sums the points q = lane, lane + nl, ... of the entry's
// rules, so that a warp can share one heavy entry (lanes over quadrature
// points, shuffle reduction) while light entries run one per thread
// (lane = 0, nl = 1).  Terms that do not depend on a quadrature point (free
// term, CPV, rigid-body diagonal) are added by lane 0 only.
#pragma once

namespace gcq {

// running sums: block of <= 16 terms in t, then Kahan into (s, c)
template <int N>
struct FAcc {
  float t[N], s[N], c[N];
  int cnt;
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int i = 0; i < N; ++i) t[i] = s[i] = c[i] = 0.f;
    cnt = 0;
  }
  __device__ __forceinline__ void flush() {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const float y = t[i] - c[i];
      const float u = s[i] + y;
      c[i] = (u - s[i]) - y;
      s[i] = u;
      t[i] = 0.f;
    }
    cnt = 0;
  }
  __device__ __forceinline__ void tick() {
    if (++cnt == 16) flush();
  }
  __device__ __forceinline__ void add_const(int i, float x) {
    const float y = x - c[i];
    const float u = s[i] + y;
    c[i] = (u - s[i]) - y;
    s[i] = u;
  }
};

// FP64 rule decision with the tie band (same as the oracle), no square root
__device__ __noinline__ int rule_index2(const ElemGeo& g, const double* x) {
  const double dx = g.c[0] - x[0], dy = g.c[1] - x[1], dz = g.c[2] - x[2];
  const double d2 = dx * dx + dy * dy + dz * dz;
  const double hb = g.h * (1.0 - 1e-12);
  const double h2 = hb * hb;
  if (d2 >= rule_dist(0) * rule_dist(0) * h2) return 0;
  if (d2 >= rule_dist(1) * rule_dist(1) * h2) return 1;
  if (d2 >= rule_dist(2) * rule_dist(2) * h2) return 2;
  return 3;
}

// row point x_i as a float pair (hi, lo): node coordinates or the centroid
template <int ROWS>
__device__ __forceinline__ void row_point_ff(const EntryView& v, int i, float4& hi, float4& lo) {
  const float4* p = (ROWS == BEM_ROWS_NODES ? v.nff : v.cff) + 2 * (int64_t)i;
  hi = p[0];
  lo = p[1];
}

// the same decision as rule_index2 from an FP32 |c - x|^2 (relative error
// below 2^-20): thresholds 16 h^2, 4 h^2, h^2 in FP32 carry a relative error
// below 2^-21, so outside a band of 2^-17 around a threshold both sides of
// the comparison are certain; inside it the FP64 decision is taken
__device__ __forceinline__ int rule_index_f(float d2, float h, int e, const EntryView& v, const double* x) {
  const float h2 = h * h;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float T = (float)(rule_dist(r) * rule_dist(r)) * h2;
    if (d2 >= T * (1.f + 0x1p-17f)) return r;
    if (d2 > T * (1.f - 0x1p-17f)) return rule_index2(v.geo[e], x);
  }
  return 3;
}

// rule of element e for row point x from the float pairs: |D|^2 with
// D = (c_hi - x_hi) + (c_lo - x_lo) per component
__device__ __forceinline__ int rule_ff(const EntryView& v, int e, const float4& xh, const float4& xl, const double* x) {
  const float4 ch = v.cff[2 * (int64_t)e], cl = v.cff[2 * (int64_t)e + 1];
  const float dx = (ch.x - xh.x) + (cl.x - xl.x);
  const float dy = (ch.y - xh.y) + (cl.y - xl.y);
  const float dz = (ch.z - xh.z) + (cl.z - xl.z);
  return rule_index_f(dx * dx + dy * dy + dz * dz, ch.w, e, v, x);
}

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fadd_rn(s, -a);
  e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
}

// CPV int_e rh / r^2 dA in FP32, x inside the flat element (closed form per
// sub-triangle, as cpv_rh_r2); vertices relative to p0, x relative to p0
__device__ void cpv_rh_r2_f(const float* e1, const float* e2, const float* xr, float* G) {
  float P[3][3] = {{0.f, 0.f, 0.f}, {e1[0], e1[1], e1[2]}, {e2[0], e2[1], e2[2]}};
  G[0] = G[1] = G[2] = 0.f;
  for (int a = 0; a < 3; ++a) {
    const float* Pa = P[a];
    const float* Pb = P[(a + 1) % 3];
    float t[3] = {Pb[0] - Pa[0], Pb[1] - Pa[1], Pb[2] - Pa[2]};
    const float tl = sqrtf(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    for (int k = 0; k < 3; ++k) t[k] /= tl;
    const float xa = (xr[0] - Pa[0]) * t[0] + (xr[1] - Pa[1]) * t[1] + (xr[2] - Pa[2]) * t[2];
    float e0[3] = {Pa[0] + xa * t[0] - xr[0], Pa[1] + xa * t[1] - xr[1], Pa[2] + xa * t[2] - xr[2]};
    const float h = sqrtf(e0[0] * e0[0] + e0[1] * e0[1] + e0[2] * e0[2]);
    for (int k = 0; k < 3; ++k) e0[k] /= h;
    const float ta = -xa, tb = tl - xa;   // tangential coordinates of Pa, Pb from the foot
    const float Ra = sqrtf(h * h + ta * ta), Rb = sqrtf(h * h + tb * tb);
    const float p0 = (tb / Rb) * (logf(Rb) + 1.f) - asinhf(tb / h) - ((ta / Ra) * (logf(Ra) + 1.f) - asinhf(ta / h));
    const float p1 = -(h / Rb) * (logf(Rb) + 1.f) + (h / Ra) * (logf(Ra) + 1.f);
    for (int k = 0; k < 3; ++k) G[k] += e0[k] * p0 + t[k] * p1;
  }
}

// element frame in FP32 relative to the collocation point
struct FrameF {
  float d0[3];   // p0 - x
  float e1[3], e2[3], n[3];
  float area2;
};
__device__ __forceinline__ FrameF frame_f(const ElemGeo& g, const double* x) {
  FrameF f;
  for (int k = 0; k < 3; ++k) {
    f.d0[k] = (float)(g.p0[k] - x[k]);
    f.e1[k] = (float)g.e1[k];
    f.e2[k] = (float)g.e2[k];
    f.n[k] = (float)g.n[k];
  }
  f.area2 = (float)g.area2;
  return f;
}

// Duffy sub-triangle (apex at x): edges ba = B - A, cb = C - B, 2 * area
struct SubF {
  float ba[3], cb[3], ar2;
};
__device__ __forceinline__ SubF sub_f(const float* A, const float* B, const float* C) {
  SubF s;
  float ca[3];
  for (int k = 0; k < 3; ++k) {
    s.ba[k] = B[k] - A[k];
    s.cb[k] = C[k] - B[k];
    ca[k] = C[k] - A[k];
  }
  const float c0 = s.ba[1] * ca[2] - s.ba[2] * ca[1], c1 = s.ba[2] * ca[0] - s.ba[0] * ca[2],
              c2 = s.ba[0] * ca[1] - s.ba[1] * ca[0];
  s.ar2 = sqrtf(c0 * c0 + c1 * c1 + c2 * c2);
  return s;
}

// vertices of element e relative to p0 (P0 = 0, P1 = e1, P2 = e2)
__device__ __forceinline__ void vert_f(const FrameF& f, int a, float* P) {
  for (int k = 0; k < 3; ++k) P[k] = a == 0 ? 0.f : (a == 1 ? f.e1[k] : f.e2[k]);
}

// exp(-s r0 / c_a), a = 1, 2, at a reference distance r0 (an FP32 number):
// the phase (Im s / c_a) r0 is formed as a float-float product and reduced
// modulo 2 pi by Cody and Waite's additive reduction (W. J. Cody and
// W. Waite, Software Manual for the Elementary Functions, 1980): 2 pi split
// into a leading part C1 = fl(2 pi) and a correction C2 = 2 pi - C1, the
// product nt C1 subtracted exactly by FMA, then nt C2 added; the magnitude
// exp(-(Re s / c_a) r0) gets the low part of its exponent as a first-order
// factor.  Removes the FP32 error proportional to |s| r / c of
// exp(-s r / c) evaluated at full r.
__device__ __forceinline__ void ref_exp(const EntryView& v, int k, float r0, cx<float>* E0, cx<float>* w) {
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const float4 q = v.sw[2 * k + a];   // (re_hi, re_lo, im_hi, im_lo) of s_k / c_a
    w[a] = {q.x, q.z};
    const float ph = q.z * r0;
    float pe = fmaf(q.z, r0, -ph);
    pe = fmaf(q.w, r0, pe);
    const float nt = rintf(ph * 0.159154943091895336f);
    float t = fmaf(-nt, 6.28318548202514648f, ph);   // Cody-Waite: C1 = fl(2 pi), C2 = 2 pi - C1 = -1.7484556e-7
    t = fmaf(nt, 1.74845553e-07f, t) + pe;
    const float mg = q.x * r0;
    float me = fmaf(q.x, r0, -mg);
    me = fmaf(q.y, r0, me);
    const float mag = expf(-mg) * (1.f - me);
    float sn, cs;
    sincosf(t, &sn, &cs);
    E0[a] = {mag * cs, -mag * sn};
  }
}

// reference data of a regular element integral for row point x: D = c - x
// rounded to FP32, r0 = |D| rounded to FP32, c0 = |c - x|^2 - r0^2 to about
// 2^-40 |D|^2, and the quadrature rule (the FP64 decision).  All in FP32:
// c - x = (c_hi - x_hi) + (c_lo - x_lo) with the first difference split
// exactly (two-sum), |D|^2 - r0^2 from the exact squares (FMA residuals).
struct RefF {
  float D[3], r0, c0;
  int ri;
  bool use;
};
__device__ __forceinline__ RefF ref_f(const EntryView& v, int e, const float4& xh, const float4& xl,
                                      const double* x) {
  RefF R;
  const float4 ch = v.cff[2 * (int64_t)e], cl = v.cff[2 * (int64_t)e + 1];
  const float hc[3] = {ch.x, ch.y, ch.z}, lc[3] = {cl.x, cl.y, cl.z};
  const float hx[3] = {xh.x, xh.y, xh.z}, lx[3] = {xl.x, xl.y, xl.z};
  float Dl[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float a, ea;
    two_sum_f(hc[k], -hx[k], a, ea);
    const float b = __fadd_rn(__fadd_rn(lc[k], -lx[k]), ea);
    two_sum_f(a, b, R.D[k], Dl[k]);
  }
  // |D + Dl|^2 = q0 + q1 + q2 + (f0 + f1 + f2) + 2 D.Dl + |Dl|^2 (last term dropped)
  float q[3], f[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    q[k] = __fmul_rn(R.D[k], R.D[k]);
    f[k] = fmaf(R.D[k], R.D[k], -q[k]);
  }
  float s1, e1, s2, e2;
  two_sum_f(q[0], q[1], s1, e1);
  two_sum_f(s1, q[2], s2, e2);
  R.r0 = sqrtf(s2);
  const float rr = __fmul_rn(R.r0, R.r0), er = fmaf(R.r0, R.r0, -rr);
  const float dot = R.D[0] * Dl[0] + R.D[1] * Dl[1] + R.D[2] * Dl[2];
  const float tail = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(f[0], f[1]), f[2])) - er + 2.f * dot;
  R.c0 = __fadd_rn(s2, -rr) + tail;   // s2 - rr exact (Sterbenz: rr within 2 ulp of s2)
  R.ri = rule_index_f(s2, ch.w, e, v, x);
  R.use = false;
  return R;
}

// geometry of regular point (xi, eta): d = y - x, r = |d|, dr = r - r0
// computed from the small offset dd = y - c without cancellation
__device__ __forceinline__ void ref_point(const RefF& R, const float4& a0, const float4& e1, const float4& e2,
                                          float xi, float et, float* d, float& r, float& dr) {
  const float dd0 = a0.x + xi * e1.x + et * e2.x;
  const float dd1 = a0.y + xi * e1.y + et * e2.y;
  const float dd2 = a0.z + xi * e1.z + et * e2.z;
  d[0] = R.D[0] + dd0;
  d[1] = R.D[1] + dd1;
  d[2] = R.D[2] + dd2;
  r = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  const float num = R.c0 + 2.f * (R.D[0] * dd0 + R.D[1] * dd1 + R.D[2] * dd2) + (dd0 * dd0 + dd1 * dd1 + dd2 * dd2);
  dr = num / (r + R.r0);
}

// exp(-w (r0 + dr)) from the reference exponential E0 = exp(-w r0).  When
// E0 underflowed to zero (Re(w) r0 beyond the FP32 range, elements far
// larger than the decay length exp(-Re(w) r)), the factor exp(-w dr) of a
// point nearer than r0 can overflow and the product would be 0 x inf: the
// value is then evaluated directly at r (where it is at most a few orders
// above the underflow threshold, and its phase error immaterial).
__device__ __forceinline__ cx<float> exp_from_ref(cx<float> E0, cx<float> w, float r, float dr) {
  if (E0.x == 0.f && E0.y == 0.f) return cexp_neg(cx<float>{w.x * r, w.y * r});
  return E0 * cexp_neg(cx<float>{w.x * dr, w.y * dr});
}

// kernel coefficients at a regular point: series for |s| r / c2 < 2, else the
// closed form with exp(-s r / c_a) = E0_a exp(-s dr / c_a) when the reference
// is in use (large |s| r0 / c2), or evaluated directly
template <bool D>
__device__ __forceinline__ void coeffs_ref(const KC<float>& k, float r, float dr, cx<float> s, cx<float> is2,
                                           bool use, const cx<float>* E0, const cx<float>* w, cx<float>& A,
                                           cx<float>& B, cx<float>& dA, cx<float>& dB, cx<float>& S3) {
  const cx<float> ws = {-s.x * r * k.ic2, -s.y * r * k.ic2};
  if (ws.x * ws.x + ws.y * ws.y < 4.f) {
    series_coeffs<float, D, false>(k, r, ws, A, B, dA, dB, S3);
    return;
  }
  const cx<float> kr1 = {w[0].x * r, w[0].y * r}, kr2 = {w[1].x * r, w[1].y * r};
  cx<float> e1, e2;
  if (use) {
    e1 = exp_from_ref(E0[0], w[0], r, dr);
    e2 = exp_from_ref(E0[1], w[1], r, dr);
  } else {
    e1 = cexp_neg(kr1);
    e2 = cexp_neg(kr2);
  }
  closed_coeffs<float, D, false>(k, r, kr1, kr2, e1, e2, is2, A, B, dA, dB, S3);
}

// wave-speed derivative coefficients at a regular point (DC = 1: c1, 2: c2),
// exp(-k_a r) through the reference exponential when it is in use
template <int DC>
__device__ __forceinline__ void dcoeffs_ref(const KC<float>& k, float r, float dr, bool use, const cx<float>* E0,
                                            const cx<float>* w, cx<float>& A, cx<float>& B) {
  const cx<float> wa = w[DC - 1];
  const cx<float> kr = {wa.x * r, wa.y * r};
  const cx<float> e = use ? exp_from_ref(E0[DC - 1], wa, r, dr) : cexp_neg(kr);
  dcoeffs_from<float, DC>(k, r, kr, e, A, B);
}

// ---- single layer: V[i, e] partial sum over points lane, lane + nl, ... -------
// (DC = 1, 2: the wave-speed derivative dV/dc_a)
template <int ROWS, int DC>
__device__ void entry_sl_f(const EntryView& v, int i, int e, cx<float> s, cx<float> is2, int kf, int lane, int nl,
                           float* out18) {
  const ElemGeo& g = v.geo[e];
  const double* x = row_point<ROWS>(v, i);
  const int32_t* t = v.tri + 3 * (int64_t)e;
  int apex = -1;
  if (ROWS == BEM_ROWS_NODES)
    apex = (t[0] == i) ? 0 : (t[1] == i) ? 1 : (t[2] == i) ? 2 : -1;
  else if (e == i)
    apex = 3;
  FAcc<14> acc;   // SA (2) + SB[6] (12)
  acc.init();
  cx<float>* SA = reinterpret_cast<cx<float>*>(acc.t);
  cx<float>* SB = reinterpret_cast<cx<float>*>(acc.t + 2);
  if (apex >= 0) {
    const FrameF f = frame_f(g, x);
    // sub-triangles with apex x, coordinates relative to p0; x - p0 = -d0
    const float xr[3] = {-f.d0[0], -f.d0[1], -f.d0[2]};
    const int nsub = apex == 3 ? 3 : 1;
    for (int q = lane; q < nsub * 256; q += nl) {
      const int sb = q >> 8, a = (q >> 4) & 15, b = q & 15;
      float A[3], Bv[3], Cv[3];
      if (apex == 3) {
        for (int k = 0; k < 3; ++k) A[k] = xr[k];
        vert_f(f, sb, Bv);
        vert_f(f, (sb + 1) % 3, Cv);
      } else {
        vert_f(f, apex, A);
        vert_f(f, (apex + 1) % 3, Bv);
        vert_f(f, (apex + 2) % 3, Cv);
      }
      const SubF st = sub_f(A, Bv, Cv);
      const float u = c_gl16_f[a], wu = c_gl16_f[16 + a];
      const float vv = c_gl16_f[b], wv = c_gl16_f[16 + b];
      // y - x = (A - x) + u (ba + v cb) with A = x
      acc_sl<float, DC>(v.kf, wu * wv * st.ar2 * u, u * (st.ba[0] + vv * st.cb[0]),
                        u * (st.ba[1] + vv * st.cb[1]), u * (st.ba[2] + vv * st.cb[2]), s, is2, *SA, SB);
      acc.tick();
    }
  } else {
    float4 xh, xl;
    row_point_ff<ROWS>(v, i, xh, xl);
    const RefF R = ref_f(v, e, xh, xl, x);
    const int q0 = rule_offset(R.ri), q1 = rule_offset(R.ri + 1);
    const float4 a0 = v.ef[4 * (int64_t)e], fe1 = v.ef[4 * (int64_t)e + 1], fe2 = v.ef[4 * (int64_t)e + 2];
    cx<float> E0[2], w[2];
    const bool use = kf >= 0 && (s.x * s.x + s.y * s.y) * R.r0 * R.r0 * v.kf.ic2s > 16.f;   // |s| r0 / c2 > 4
    if (use) ref_exp(v, kf, R.r0, E0, w);
    else w[0] = s * v.kf.ic1, w[1] = s * v.kf.ic2;
    for (int q = q0 + lane; q < q1; q += nl) {
      const float xi = c_rule_f[3 * q], et = c_rule_f[3 * q + 1];
      const float wq = c_rule_f[3 * q + 2] * a0.w;
      float d[3], r, dr;
      ref_point(R, a0, fe1, fe2, xi, et, d, r, dr);
      const float ir = 1.f / r;
      const float hh[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
      cx<float> A, Bc;
      if constexpr (DC == 0) {
        cx<float> dA, dB, S3;
        coeffs_ref<false>(v.kf, r, dr, s, is2, use, E0, w, A, Bc, dA, dB, S3);
      } else {
        dcoeffs_ref<DC>(v.kf, r, dr, use, E0, w, A, Bc);
      }
      acc_U_from<float>(wq, hh, A, Bc, *SA, SB);
      acc.tick();
    }
  }
  acc.flush();
  const float c = v.kf.inv4pirho;
  const cx<float> sa = {acc.s[0], acc.s[1]};
  cx<float> sbv[6];
  for (int k = 0; k < 6; ++k) sbv[k] = {acc.s[2 + 2 * k], acc.s[3 + 2 * k]};
  const cx<float> o[9] = {c * (sa + sbv[0]), c * sbv[1], c * sbv[2], c * sbv[1], c * (sa + sbv[3]),
                          c * sbv[4], c * sbv[2], c * sbv[4], c * (sa + sbv[5])};
  for (int k = 0; k < 9; ++k) {
    out18[2 * k] = o[k].x;
    out18[2 * k + 1] = o[k].y;
  }
}

// ---- double layer (C + K)[i, j] partial sum ---------------------------------
// (DC = 1, 2: the wave-speed derivative d(C + K)/dc_a)
template <int ROWS, int DC>
__device__ void entry_dl_f(const EntryView& v, int i, int j, cx<float> s, cx<float> is2, int kf, int lane, int nl,
                           float* out18) {
  const double* x = row_point<ROWS>(v, i);
  float4 xh, xl;
  row_point_ff<ROWS>(v, i, xh, xl);
  FAcc<18> acc;
  acc.init();
  cx<float>* A9 = reinterpret_cast<cx<float>*>(acc.t);
  float st0[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // static parts (point-independent or T0)
  const float nu = (float)v.nu;
  const int p0 = v.ne_ptr[j], p1 = v.ne_ptr[j + 1];
  for (int p = p0; p < p1; ++p) {
    const int e = v.ne_elem[p];
    const int a = v.ne_loc[p];   // local vertex of column node j in e
    const ElemGeo& g = v.geo[e];
    const int32_t* t = v.tri + 3 * (int64_t)e;
    int apex = -1;
    if (ROWS == BEM_ROWS_NODES)
      apex = (t[0] == i) ? 0 : (t[1] == i) ? 1 : (t[2] == i) ? 2 : -1;
    else if (e == i)
      apex = 3;
    if (apex < 0) {
      const RefF R = ref_f(v, e, xh, xl, x);
      const int q0 = rule_offset(R.ri), q1 = rule_offset(R.ri + 1);
      const float4 a0 = v.ef[4 * (int64_t)e], fe1 = v.ef[4 * (int64_t)e + 1], fe2 = v.ef[4 * (int64_t)e + 2];
      const float4 fn = v.ef[4 * (int64_t)e + 3];
      const float nf[3] = {fn.x, fn.y, fn.z};
      cx<float> E0[2], w[2];
      const bool use = kf >= 0 && (s.x * s.x + s.y * s.y) * R.r0 * R.r0 * v.kf.ic2s > 16.f;
      if (use) ref_exp(v, kf, R.r0, E0, w);
      else w[0] = s * v.kf.ic1, w[1] = s * v.kf.ic2;
      for (int q = q0 + lane; q < q1; q += nl) {
        const float xi = c_rule_f[3 * q], et = c_rule_f[3 * q + 1];
        const float phi = a == 0 ? 1.f - xi - et : (a == 1 ? xi : et);
        const float wq = c_rule_f[3 * q + 2] * a0.w * phi;
        float d[3], r, dr;
        ref_point(R, a0, fe1, fe2, xi, et, d, r, dr);
        const float ir = 1.f / r;
        const float hh[3] = {d[0] * ir, d[1] * ir, d[2] * ir};
        cx<float> A, Bc, dA, dB, S3;
        coeffs_ref<true>(v.kf, r, dr, s, is2, use, E0, w, A, Bc, dA, dB, S3);
        if constexpr (DC == 0) {
          acc_TT_from<float>(v.kf, wq, r, hh, nf, A, Bc, dA, dB, S3, A9);
        } else {
          const cx<float> wa = w[DC - 1];
          const cx<float> xr = {wa.x * r, wa.y * r};
          const cx<float> ea = use ? exp_from_ref(E0[DC - 1], wa, r, dr) : cexp_neg(xr);
          cx<float> DA, DB, DAp, DBp, DS3;
          dcoeffs2_from<float, DC>(v.kf, r, xr, ea, ea, DA, DB, DAp, DBp, DS3);
          acc_dTT_from<float, DC>(v.kf, wq, r, hh, nf, Bc, dA, dB, S3, DB, DAp, DBp, DS3, A9);
        }
        acc.tick();
      }
      continue;
    }
    const FrameF f = frame_f(g, x);
    const float xr[3] = {-f.d0[0], -f.d0[1], -f.d0[2]};
    const int nsub = apex == 3 ? 3 : 1;
    for (int q = lane; q < nsub * 256; q += nl) {
      const int sb = q >> 8, qa = (q >> 4) & 15, qb = q & 15;
      float A[3], Bv[3], Cv[3];
      int lb, lc;
      if (apex == 3) {
        lb = sb;
        lc = (sb + 1) % 3;
        for (int k = 0; k < 3; ++k) A[k] = xr[k];
      } else {
        lb = (apex + 1) % 3;
        lc = (apex + 2) % 3;
        vert_f(f, apex, A);
      }
      vert_f(f, lb, Bv);
      vert_f(f, lc, Cv);
      const SubF sbf = sub_f(A, Bv, Cv);
      const float u = c_gl16_f[qa], wu = c_gl16_f[16 + qa];
      const float vv = c_gl16_f[qb], wv = c_gl16_f[16 + qb];
      const float d0 = u * (sbf.ba[0] + vv * sbf.cb[0]);
      const float d1 = u * (sbf.ba[1] + vv * sbf.cb[1]);
      const float d2 = u * (sbf.ba[2] + vv * sbf.cb[2]);
      const float wq = wu * wv * sbf.ar2 * u;
      const float lam_b = u * (1.f - vv), lam_c = u * vv;
      float phi;
      if (apex == 3)
        phi = (1.f - u) * (1.f / 3.f) + (a == lb ? lam_b : 0.f) + (a == lc ? lam_c : 0.f);
      else
        phi = (a == apex) ? 1.f - u : (a == lb ? lam_b : lam_c);
      if (apex == 3) {
        acc_dl<float, true, DC>(v.kf, wq * phi, d0, d1, d2, f.n, s, is2, A9);
        acc_dl0<float, DC>(v.kf, nu, wq * (phi - 1.f / 3.f), d0, d1, d2, f.n, st0);
      } else if (a == apex) {
        acc_dl<float, true, DC>(v.kf, wq * phi, d0, d1, d2, f.n, s, is2, A9);
      } else {
        acc_dl<float, false, DC>(v.kf, wq * phi, d0, d1, d2, f.n, s, is2, A9);
      }
      acc.tick();
    }
    if (apex == 3 && lane == 0) {
      float G[3];
      cpv_rh_r2_f(f.e1, f.e2, xr, G);
      // (DC: d/dnu of -(1-2nu)/(1-nu) is 1/(1-nu)^2; the free term is fixed)
      const float fc = DC == 0 ? -(1.f - 2.f * nu) / (8.f * (float)M_PI * (1.f - nu)) / 3.f
                               : (DC == 1 ? v.kf.dnu1 : v.kf.dnu2) / (8.f * (float)M_PI * (1.f - nu) * (1.f - nu)) / 3.f;
      const float fr = DC == 0 ? 1.f / 6.f : 0.f;
      for (int aa = 0; aa < 3; ++aa)
        for (int bb = 0; bb < 3; ++bb)
          st0[3 * aa + bb] += fc * (G[bb] * f.n[aa] - f.n[bb] * G[aa]) + (aa == bb ? fr : 0.f);
    }
  }
  acc.flush();
  if (ROWS == BEM_ROWS_NODES && j == i && lane == 0) {
    if (DC == 0 && v.rb) {
      for (int c = 0; c < 9; ++c) st0[c] += (float)v.rb[9 * (int64_t)i + c];
    } else if (DC != 0 && v.rb_dnu) {
      const double dn = DC == 1 ? v.kd.dnu1 : v.kd.dnu2;
      for (int c = 0; c < 9; ++c) st0[c] += (float)(dn * v.rb_dnu[9 * (int64_t)i + c]);
    }
  }
  for (int c = 0; c < 9; ++c) {
    acc.add_const(2 * c, st0[c]);
    out18[2 * c] = acc.s[2 * c];
    out18[2 * c + 1] = acc.s[2 * c + 1];
  }
}

// does the entry use a rule of 64 or more points (near or singular)?
template <int KERN, int ROWS>
__device__ __forceinline__ bool entry_heavy(const EntryView& v, int i, int j) {
  const double* x = row_point<ROWS>(v, i);
  float4 xh, xl;
  row_point_ff<ROWS>(v, i, xh, xl);
  if constexpr (kern_sl(KERN)) {
    const int32_t* t = v.tri + 3 * (int64_t)j;
    if (ROWS == BEM_ROWS_NODES ? (t[0] == i || t[1] == i || t[2] == i) : j == i) return true;
    return rule_ff(v, j, xh, xl, x) >= 2;
  } else {
    for (int p = v.ne_ptr[j]; p < v.ne_ptr[j + 1]; ++p) {
      const int e = v.ne_elem[p];
      const int32_t* t = v.tri + 3 * (int64_t)e;
      if (ROWS == BEM_ROWS_NODES ? (t[0] == i || t[1] == i || t[2] == i) : e == i) return true;
      if (rule_ff(v, e, xh, xl, x) >= 2) return true;
    }
    return false;
  }
}

template <int KERN, int ROWS>
__device__ __forceinline__ void entry_f(const EntryView& v, int i, int j, cx<float> s, cx<float> is2, int kf,
                                        int lane, int nl, float* out18) {
  if constexpr (kern_sl(KERN))
    entry_sl_f<ROWS, kern_dc(KERN)>(v, i, j, s, is2, kf, lane, nl, out18);
  else
    entry_dl_f<ROWS, kern_dc(KERN)>(v, i, j, s, is2, kf, lane, nl, out18);
}

// warp-cooperative evaluation: every lane of the warp calls this with the
// same (i, j, s); the sum over all points is returned in all lanes
template <int KERN, int ROWS>
__device__ __forceinline__ void entry_f_warp(const EntryView& v, int i, int j, cx<float> s, cx<float> is2, int kf,
                                             float* out18) {
  const int lane = threadIdx.x & 31;
  entry_f<KERN, ROWS>(v, i, j, s, is2, kf, lane, 32, out18);
#pragma unroll
  for (int c = 0; c < 18; ++c)
    for (int o = 16; o > 0; o >>= 1) out18[c] += __shfl_xor_sync(0xffffffffu, out18[c], o);
}

// entry in the precision of the context: FP64 (entry.cuh) or FP32 (above,
// one thread for all points); result in double
template <typename R, int KERN, int ROWS>
__device__ __forceinline__ void entry(const EntryView& v, int i, int j, int kf, cx<double> s, cx<double> is2,
                                      cx<double>* out) {
  if constexpr (sizeof(R) == sizeof(float)) {
    float o[18];
    entry_f<KERN, ROWS>(v, i, j, cx<float>{(float)s.x, (float)s.y}, cx<float>{(float)is2.x, (float)is2.y}, kf, 0, 1,
                        o);
    for (int c = 0; c < 9; ++c) out[c] = {(double)o[2 * c], (double)o[2 * c + 1]};
  } else {
    if constexpr (kern_sl(KERN))
      entry_sl<double, ROWS, kern_dc(KERN)>(v, i, j, s, is2, out);
    else
      entry_dl<double, ROWS, kern_dc(KERN)>(v, i, j, s, is2, out);
  }
}

}  // namespace gcq
