// Laplace-domain elastodynamic kernels and collocation matrix entries on the
// device (Sec. 2.3-2.4; kernels written from the Laplace-transformed Navier
// equation, Eq. (2.1a), traction operator Eq. (2.4), stress Eq. (2.5)).
//
//   U_ab = [A d_ab + B rh_a rh_b] / (4 pi rho),  r = y - x
//   A = h2/c2^2 + (P2 - P1)/s^2,  B = (Q1 - Q2)/s^2,   h_a = e^{-k_a r}/r,
//   P_a = (k_a r + 1) e^{-k_a r}/r^3,  Q_a = (k_a^2 r^2 + 3 k_a r + 3) e^{-k_a r}/r^3,
//   A' = -r P2/c2^2 + B/r,  B' = (R1 - R2)/s^2,
//   R_a = -(k^3 r^3 + 4 k^2 r^2 + 9 k r + 9) e^{-k r}/r^4,   k_a = s / c_a,
//   4 pi T_ab = f1 (rn d_ab + rh_a n_b) + f2 rn rh_a rh_b + f3 n_a rh_b,
//   f1 = c2^2 (A' + B/r), f2 = 2 c2^2 (B' - 2B/r),
//   f3 = (c1^2 - 2 c2^2)(A' + B' + 2B/r) + 2 c2^2 B/r.
// For |s| r / c2 < 1 the closed form cancels and the exact Taylor series in
// w = -s r / c2 is used (coefficients from the host, Material::ta/tb).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace gcq {

// ---------------------------------------------------------------------------
// constant tables: collapsed rules n = 3, 5, 8, 16 (xi, eta, w) and the
// 16-point Gauss-Legendre rule on [0, 1] for the Duffy map
// ---------------------------------------------------------------------------
__constant__ double c_rule[3 * 354];
__constant__ double c_gl16[32];
__constant__ float c_rule_f[3 * 354];   // FP32 copies for the MIXED path
__constant__ float c_gl16_f[32];

template <typename R>
struct cx {
  R x, y;
};

template <typename R>
__device__ __forceinline__ cx<R> mk(R a, R b) {
  return cx<R>{a, b};
}
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) {
  return {a.x - b.x, a.y - b.y};
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(R a, cx<R> b) {
  return {a * b.x, a * b.y};
}
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> b, R a) {
  return {a * b.x, a * b.y};
}
template <typename R>
__device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> b, cx<R> c) {  // a*b + c
  return {fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y))};
}
template <typename R>
__device__ __forceinline__ cx<R> conj(cx<R> a) {
  return {a.x, -a.y};
}
__device__ __forceinline__ cx<double> cexp_neg(cx<double> z) {  // exp(-z)
  double sn, cs;
  sincos(z.y, &sn, &cs);
  double m = exp(-z.x);
  return {m * cs, -m * sn};
}
__device__ __forceinline__ cx<float> cexp_neg(cx<float> z) {
  float sn, cs;
  sincosf(z.y, &sn, &cs);
  float m = expf(-z.x);
  return {m * cs, -m * sn};
}
// exp(-z) - 1 without cancellation at small |z|:
// re = expm1(-x) cos y - 2 sin^2(y / 2), im = -exp(-x) sin y
__device__ __forceinline__ cx<double> cexpm1_neg(cx<double> z) {
  double sn, cs, sh, ch;
  sincos(z.y, &sn, &cs);
  sincos(0.5 * z.y, &sh, &ch);
  return {expm1(-z.x) * cs - 2.0 * sh * sh, -exp(-z.x) * sn};
}
__device__ __forceinline__ cx<float> cexpm1_neg(cx<float> z) {
  float sn, cs, sh, ch;
  sincosf(z.y, &sn, &cs);
  sincosf(0.5f * z.y, &sh, &ch);
  return {expm1f(-z.x) * cs - 2.f * sh * sh, -expf(-z.x) * sn};
}

// kernel constants in the compute type
template <typename R>
struct KC {
  R c1, c2, c1s, c2s, ic1, ic2, ic2s, inv4pirho, inv4pi, alpha, beta;
  R ic1c, ic2c;   // 1 / c1^3, 1 / c2^3 (wave-speed derivatives)
  R dnu1, dnu2;   // d nu / d c1, d nu / d c2 at fixed rho
  R ta[kSeriesTerms], tb[kSeriesTerms];
};

template <typename R>
KC<R> make_kc(const Material& m) {
  KC<R> k;
  k.c1 = (R)m.c1;
  k.c2 = (R)m.c2;
  k.c1s = (R)(m.c1 * m.c1);
  k.c2s = (R)(m.c2 * m.c2);
  k.ic1 = (R)(1.0 / m.c1);
  k.ic2 = (R)(1.0 / m.c2);
  k.ic2s = (R)(1.0 / (m.c2 * m.c2));
  k.inv4pirho = (R)(1.0 / (4.0 * M_PI * m.rho));
  k.inv4pi = (R)(1.0 / (4.0 * M_PI));
  k.alpha = (R)(0.5 * (1.0 / (m.c1 * m.c1) + 1.0 / (m.c2 * m.c2)));
  k.beta = (R)(0.5 * (1.0 / (m.c2 * m.c2) - 1.0 / (m.c1 * m.c1)));
  k.ic1c = (R)(1.0 / (m.c1 * m.c1 * m.c1));
  k.ic2c = (R)(1.0 / (m.c2 * m.c2 * m.c2));
  // nu = (c1^2 - 2 c2^2) / (2 (c1^2 - c2^2))
  const double dd = (m.c1 * m.c1 - m.c2 * m.c2) * (m.c1 * m.c1 - m.c2 * m.c2);
  k.dnu1 = (R)(m.c1 * m.c2 * m.c2 / dd);
  k.dnu2 = (R)(-m.c1 * m.c1 * m.c2 / dd);
  for (int i = 0; i < kSeriesTerms; ++i) {
    k.ta[i] = (R)m.ta[i];
    k.tb[i] = (R)m.tb[i];
  }
  return k;
}

// Series branch per compute type: FP64 uses it for |w| < 1 (22 terms, tail
// < 1/22!); FP32 for |w| < 2 (18 terms, tail < 2^18/18! ~ 4e-11): in FP32 the
// closed form loses ~1/|w|^2 of its digits to cancellation (2.5e-6 block-
// relative error of the traction kernel at |w| = 1), while the alternating
// series stays accurate up to |w| ~ 2 (largest term 2^m/m! <= 2).
template <typename R>
struct SeriesLen;
template <>
struct SeriesLen<double> {
  static constexpr int n = 22;
  static constexpr double z = 1.0;
};
template <>
struct SeriesLen<float> {
  static constexpr int n = 18;
  static constexpr double z = 2.0;
};

// Series branch: A, B (and A', B' if D) from the Taylor series in
// w = -s r / c2; DYN drops the m = 0 (static) term.
template <typename R, bool D, bool DYN>
__device__ __forceinline__ void series_coeffs(const KC<R>& k, R r, cx<R> w, cx<R>& A, cx<R>& B, cx<R>& dA,
                                              cx<R>& dB, cx<R>& S3) {
  const R ir = R(1) / r;
  constexpr int M = SeriesLen<R>::n;
  const int m0 = DYN ? 1 : 0;
  cx<R> pa = mk<R>(k.ta[M - 1], R(0)), pb = mk<R>(k.tb[M - 1], R(0));
  cx<R> qa = mk<R>(R(M - 2) * k.ta[M - 1], R(0)), qb = mk<R>(R(M - 2) * k.tb[M - 1], R(0));
#pragma unroll
  for (int m = M - 2; m >= m0; --m) {
    pa = cfma(pa, w, mk<R>(k.ta[m], R(0)));
    pb = cfma(pb, w, mk<R>(k.tb[m], R(0)));
    if (D) {
      qa = cfma(qa, w, mk<R>(R(m - 1) * k.ta[m], R(0)));
      qb = cfma(qb, w, mk<R>(R(m - 1) * k.tb[m], R(0)));
    }
  }
  if (DYN) {  // the polynomials above started at m = 1: multiply by w
    pa = pa * w;
    pb = pb * w;
    qa = qa * w;
    qb = qb * w;
  }
  const R f = k.ic2s * ir;
  A = f * pa;
  B = f * pb;
  if (D) {
    dA = (f * ir) * qa;
    dB = (f * ir) * qb;
    S3 = dA + dB + (R(2) * ir) * B;
  }
}

// Closed form with given k_a r (kr1, kr2) and exponentials e_a = exp(-k_a r).
// S3 = A' + B' + 2 B / r, the combination of the traction kernel's n_i rh_j
// term: in closed form the c2-wave parts cancel exactly and
//   S3 = -(k1 r + 1) exp(-k1 r) / (c1^2 r^2),
// which is evaluated directly (no cancellation).
template <typename R, bool D, bool DYN>
__device__ __forceinline__ void closed_coeffs(const KC<R>& k, R r, cx<R> kr1, cx<R> kr2, cx<R> e1, cx<R> e2,
                                              cx<R> is2, cx<R>& A, cx<R>& B, cx<R>& dA, cx<R>& dB, cx<R>& S3) {
  const R ir = R(1) / r;
  const R ir2 = ir * ir, ir3 = ir2 * ir;
  cx<R> kk1 = kr1 * kr1, kk2 = kr2 * kr2;
  cx<R> P1 = (ir3 * e1) * (kr1 + mk<R>(R(1), R(0)));
  cx<R> P2 = (ir3 * e2) * (kr2 + mk<R>(R(1), R(0)));
  cx<R> Q1 = (ir3 * e1) * (kk1 + R(3) * kr1 + mk<R>(R(3), R(0)));
  cx<R> Q2 = (ir3 * e2) * (kk2 + R(3) * kr2 + mk<R>(R(3), R(0)));
  A = (ir * k.ic2s) * e2 + (P2 - P1) * is2;
  B = (Q1 - Q2) * is2;
  if (D) {
    cx<R> R1 = (-ir3 * ir * e1) * (kk1 * kr1 + R(4) * kk1 + R(9) * kr1 + mk<R>(R(9), R(0)));
    cx<R> R2 = (-ir3 * ir * e2) * (kk2 * kr2 + R(4) * kk2 + R(9) * kr2 + mk<R>(R(9), R(0)));
    dA = (-r * k.ic2s) * P2 + ir * B;
    dB = (R1 - R2) * is2;
    S3 = (-ir2 * k.ic1 * k.ic1) * (e1 * (kr1 + mk<R>(R(1), R(0))));
  }
  if (DYN) {
    A.x -= k.alpha * ir;
    B.x -= k.beta * ir;
    if (D) {
      dA.x += k.alpha * ir2;
      dB.x += k.beta * ir2;
      // static S3 = (beta - alpha) / r^2 = -1 / (c1^2 r^2)
      S3.x += k.ic1 * k.ic1 * ir2;
    }
  }
}

// A, B (and A', B' if D) at distance r and frequency s; DYN subtracts the
// static (s = 0) values (bounded remainder next to a singular point).
template <typename R, bool D, bool DYN>
__device__ __forceinline__ void kernel_coeffs(const KC<R>& k, R r, cx<R> s, cx<R> is2, cx<R>& A, cx<R>& B,
                                              cx<R>& dA, cx<R>& dB, cx<R>& S3) {
  cx<R> w = mk<R>(-s.x * r * k.ic2, -s.y * r * k.ic2);
  if (w.x * w.x + w.y * w.y < R(SeriesLen<R>::z * SeriesLen<R>::z)) {
    series_coeffs<R, D, DYN>(k, r, w, A, B, dA, dB, S3);
    return;
  }
  cx<R> kr1 = mk<R>(s.x * r * k.ic1, s.y * r * k.ic1);
  cx<R> kr2 = mk<R>(s.x * r * k.ic2, s.y * r * k.ic2);
  closed_coeffs<R, D, DYN>(k, r, kr1, kr2, cexp_neg(kr1), cexp_neg(kr2), is2, A, B, dA, dB, S3);
}

// wave-speed derivatives of A, B at fixed rho (DC = 1: c1, DC = 2: c2),
// from kr = k_a r and e = exp(-k_a r) of that wave:
//   dA/dc1 = -e1 / (r c1^3),            dB/dc1 = (1 + k1 r) e1 / (r c1^3)
//   dA/dc2 = (k2 r - 1) e2 / (r c2^3),  dB/dc2 = -(1 + k2 r) e2 / (r c2^3)
// (the 1 / s^2 of A and B cancels against k_a^2 = s^2 / c_a^2: no series)
template <typename R, int DC>
__device__ __forceinline__ void dcoeffs_from(const KC<R>& k, R r, cx<R> kr, cx<R> e, cx<R>& A, cx<R>& B) {
  const cx<R> f = ((DC == 1 ? k.ic1c : k.ic2c) / r) * e;
  const cx<R> g = f * (kr + mk<R>(R(1), R(0)));
  if (DC == 1) {
    A = mk<R>(-f.x, -f.y);
    B = g;
  } else {
    A = f * (kr - mk<R>(R(1), R(0)));
    B = mk<R>(-g.x, -g.y);
  }
}

// accumulate w dU/dc_a(d) into (SA, SB[6])
template <typename R, int DC>
__device__ __forceinline__ void acc_dU(const KC<R>& k, R wq, R dx, R dy, R dz, cx<R> s, cx<R>& SA, cx<R>* SB) {
  R r = sqrt(dx * dx + dy * dy + dz * dz);
  R ir = R(1) / r;
  R h[3] = {dx * ir, dy * ir, dz * ir};
  const R ic = DC == 1 ? k.ic1 : k.ic2;
  const cx<R> kr = mk<R>(s.x * r * ic, s.y * r * ic);
  cx<R> A, B;
  dcoeffs_from<R, DC>(k, r, kr, cexp_neg(kr), A, B);
  SA = SA + wq * A;
  cx<R> wb = wq * B;
  SB[0] = SB[0] + (h[0] * h[0]) * wb;
  SB[1] = SB[1] + (h[0] * h[1]) * wb;
  SB[2] = SB[2] + (h[0] * h[2]) * wb;
  SB[3] = SB[3] + (h[1] * h[1]) * wb;
  SB[4] = SB[4] + (h[1] * h[2]) * wb;
  SB[5] = SB[5] + (h[2] * h[2]) * wb;
}

// c_a-derivatives of A, B, A', B' and S3 = A' + B' + 2B/r (traction kernel),
// x = k_a r, e = exp(-x), em = e (DYN: e - 1, the static parts removed):
//   c1: A = -em/(r c^3), B = (em + x e)/(r c^3), A' = (em + x e)/(r^2 c^3),
//       B' = -(em + (x + x^2) e)/(r^2 c^3), S3 = (2 em + (2x - x^2) e)/(r^2 c^3)
//   c2: A = (x e - em)/(r c^3), B = -(em + x e)/(r c^3),
//       A' = (em + (x - x^2) e)/(r^2 c^3), B' = (em + (x + x^2) e)/(r^2 c^3), S3 = 0
template <typename R, int DC>
__device__ __forceinline__ void dcoeffs2_from(const KC<R>& k, R r, cx<R> x, cx<R> e, cx<R> em, cx<R>& A, cx<R>& B,
                                              cx<R>& Ap, cx<R>& Bp, cx<R>& S3) {
  const R f1 = (DC == 1 ? k.ic1c : k.ic2c) / r, f2 = f1 / r;
  const cx<R> xe = x * e, x2e = x * xe;
  if (DC == 1) {
    A = mk<R>(-f1 * em.x, -f1 * em.y);
    B = f1 * (em + xe);
    Ap = f2 * (em + xe);
    const cx<R> t = em + xe + x2e;
    Bp = mk<R>(-f2 * t.x, -f2 * t.y);
    S3 = f2 * (R(2) * em + R(2) * xe - x2e);
  } else {
    A = f1 * (xe - em);
    const cx<R> t = em + xe;
    B = mk<R>(-f1 * t.x, -f1 * t.y);
    Ap = f2 * (em + xe - x2e);
    Bp = f2 * (em + xe + x2e);
    S3 = mk<R>(R(0), R(0));
  }
}

// T^T accumulation from the three coefficient functions (already weighted):
// [a*3+b] = T_ba = f1 (rn d_ab + h_b n_a) + f2 rn h_a h_b + f3 n_b h_a
template <typename R>
__device__ __forceinline__ void acc_T_tensor(const R* h, const R* n, cx<R> f1, cx<R> f2, cx<R> f3, cx<R>* acc) {
  R rn = h[0] * n[0] + h[1] * n[1] + h[2] * n[2];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      R c1v = (a == b ? rn : R(0)) + h[b] * n[a];
      R c2v = rn * h[a] * h[b];
      R c3v = n[b] * h[a];
      acc[3 * a + b] = acc[3 * a + b] + c1v * f1 + c2v * f2 + c3v * f3;
    }
}

// w dT^T/dc_a: product rule on f1 = c2^2 (A' + B/r), f2 = 2 c2^2 (B' - 2B/r),
// f3 = (c1^2 - 2 c2^2) S3 + 2 c2^2 B/r (B, dA, dB, S3: T's coefficients;
// DB, DAp, DBp, DS3: their c_a-derivatives)
template <typename R, int DC>
__device__ __forceinline__ void acc_dTT_from(const KC<R>& k, R wq, R r, const R* h, const R* n, cx<R> B, cx<R> dA,
                                             cx<R> dB, cx<R> S3, cx<R> DB, cx<R> DAp, cx<R> DBp, cx<R> DS3,
                                             cx<R>* acc) {
  const R ir = R(1) / r, w = wq * k.inv4pi;
  const R d1s = DC == 1 ? R(2) * k.c1 : R(0), d2s = DC == 2 ? R(2) * k.c2 : R(0);
  const cx<R> Bir = ir * B, DBir = ir * DB;
  const cx<R> f1 = w * (d2s * (dA + Bir) + k.c2s * (DAp + DBir));
  const cx<R> f2 = (R(2) * w) * (d2s * (dB - R(2) * Bir) + k.c2s * (DBp - R(2) * DBir));
  const cx<R> f3 = w * ((d1s - R(2) * d2s) * S3 + (k.c1s - R(2) * k.c2s) * DS3 + (R(2) * d2s) * Bir +
                        (R(2) * k.c2s) * DBir);
  acc_T_tensor<R>(h, n, f1, f2, f3, acc);
}

// accumulate w dT^T/dc_a(d, n); DYN: of T - T0
template <typename R, bool DYN, int DC>
__device__ __forceinline__ void acc_dTT(const KC<R>& k, R wq, R dx, R dy, R dz, const R* n, cx<R> s, cx<R> is2,
                                        cx<R>* acc) {
  R r = sqrt(dx * dx + dy * dy + dz * dz);
  R ir = R(1) / r;
  R h[3] = {dx * ir, dy * ir, dz * ir};
  cx<R> A, B, dA, dB, S3;
  kernel_coeffs<R, true, DYN>(k, r, s, is2, A, B, dA, dB, S3);
  const R ic = DC == 1 ? k.ic1 : k.ic2;
  const cx<R> x = mk<R>(s.x * r * ic, s.y * r * ic);
  const cx<R> e = cexp_neg(x);
  cx<R> DA, DB, DAp, DBp, DS3;
  dcoeffs2_from<R, DC>(k, r, x, e, DYN ? cexpm1_neg(x) : e, DA, DB, DAp, DBp, DS3);
  acc_dTT_from<R, DC>(k, wq, r, h, n, B, dA, dB, S3, DB, DAp, DBp, DS3, acc);
}

// w dT0^T/dnu (real): dT0/dnu = -[Q - P] / (8 pi (1-nu)^2 r^2) with
// P = rn I + rh n^T - n rh^T, Q = 3 rn rh rh^T; [a*3+b] = (dT0/dnu)_ba
template <typename R>
__device__ __forceinline__ void acc_dT0T_dnu(R nu, R wq, R dx, R dy, R dz, const R* n, R* acc) {
  R r2 = dx * dx + dy * dy + dz * dz;
  R ir = R(1) / sqrt(r2);
  R h[3] = {dx * ir, dy * ir, dz * ir};
  R rn = h[0] * n[0] + h[1] * n[1] + h[2] * n[2];
  R f = -wq / (R(8.0 * M_PI) * (R(1) - nu) * (R(1) - nu) * r2);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      R v = R(3) * rn * h[a] * h[b] - ((a == b ? rn : R(0)) + h[b] * n[a] - n[b] * h[a]);
      acc[3 * a + b] += f * v;
    }
}

// the double-layer integrand T^T (DC = 0) or dT^T/dc_a (DC = 1, 2)
template <typename R, bool DYN, int DC>
__device__ __forceinline__ void acc_dl(const KC<R>& k, R wq, R dx, R dy, R dz, const R* n, cx<R> s, cx<R> is2,
                                       cx<R>* acc);

// its static part T0^T (DC = 0) or dT0^T/dc_a = (dnu/dc_a) dT0^T/dnu
template <typename R, int DC>
__device__ __forceinline__ void acc_dl0(const KC<R>& k, R nu, R wq, R dx, R dy, R dz, const R* n, R* acc);

// the single-layer integrand: U (DC = 0) or dU/dc_a (DC = 1, 2)
template <typename R, int DC>
__device__ __forceinline__ void acc_sl(const KC<R>& k, R wq, R dx, R dy, R dz, cx<R> s, cx<R> is2, cx<R>& SA,
                                       cx<R>* SB);

// accumulate w U into (SA, SB[6]) from the coefficients, unit vector h
template <typename R>
__device__ __forceinline__ void acc_U_from(R wq, const R* h, cx<R> A, cx<R> B, cx<R>& SA, cx<R>* SB) {
  SA = SA + wq * A;
  cx<R> wb = wq * B;
  SB[0] = SB[0] + (h[0] * h[0]) * wb;
  SB[1] = SB[1] + (h[0] * h[1]) * wb;
  SB[2] = SB[2] + (h[0] * h[2]) * wb;
  SB[3] = SB[3] + (h[1] * h[1]) * wb;
  SB[4] = SB[4] + (h[1] * h[2]) * wb;
  SB[5] = SB[5] + (h[2] * h[2]) * wb;
}

// accumulate w T^T (double-layer integrand) from the coefficients
template <typename R>
__device__ __forceinline__ void acc_TT_from(const KC<R>& k, R wq, R r, const R* h, const R* n, cx<R> A, cx<R> B,
                                            cx<R> dA, cx<R> dB, cx<R> S3, cx<R>* acc) {
  (void)A;
  const R ir = R(1) / r;
  cx<R> Bir = ir * B;
  cx<R> f1 = (wq * k.c2s * k.inv4pi) * (dA + Bir);
  cx<R> f2 = (wq * R(2) * k.c2s * k.inv4pi) * (dB - R(2) * Bir);
  cx<R> f3 = (wq * k.inv4pi) * ((k.c1s - R(2) * k.c2s) * S3 + (R(2) * k.c2s) * Bir);
  R rn = h[0] * n[0] + h[1] * n[1] + h[2] * n[2];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      R c1v = (a == b ? rn : R(0)) + h[b] * n[a];
      R c2v = rn * h[a] * h[b];
      R c3v = n[b] * h[a];
      acc[3 * a + b] = acc[3 * a + b] + c1v * f1 + c2v * f2 + c3v * f3;
    }
}

// accumulate w U(d) into (SA, SB[6]): U = (SA I + SB) / (4 pi rho)
template <typename R>
__device__ __forceinline__ void acc_U(const KC<R>& k, R wq, R dx, R dy, R dz, cx<R> s, cx<R> is2, cx<R>& SA,
                                      cx<R>* SB) {
  R r = sqrt(dx * dx + dy * dy + dz * dz);
  R ir = R(1) / r;
  R h[3] = {dx * ir, dy * ir, dz * ir};
  cx<R> A, B, dA, dB, S3;
  kernel_coeffs<R, false, false>(k, r, s, is2, A, B, dA, dB, S3);
  SA = SA + wq * A;
  cx<R> wb = wq * B;
  SB[0] = SB[0] + (h[0] * h[0]) * wb;
  SB[1] = SB[1] + (h[0] * h[1]) * wb;
  SB[2] = SB[2] + (h[0] * h[2]) * wb;
  SB[3] = SB[3] + (h[1] * h[1]) * wb;
  SB[4] = SB[4] + (h[1] * h[2]) * wb;
  SB[5] = SB[5] + (h[2] * h[2]) * wb;
}

template <typename R, int DC>
__device__ __forceinline__ void acc_sl(const KC<R>& k, R wq, R dx, R dy, R dz, cx<R> s, cx<R> is2, cx<R>& SA,
                                       cx<R>* SB) {
  if constexpr (DC == 0)
    acc_U<R>(k, wq, dx, dy, dz, s, is2, SA, SB);
  else
    acc_dU<R, DC>(k, wq, dx, dy, dz, s, SA, SB);
}

// accumulate w T^T(d, n) (double-layer integrand, 9 entries [a*3+b] = T_ba)

template <typename R, bool DYN>
__device__ __forceinline__ void acc_TT(const KC<R>& k, R wq, R dx, R dy, R dz, const R* n, cx<R> s, cx<R> is2,
                                       cx<R>* acc) {
  R r = sqrt(dx * dx + dy * dy + dz * dz);
  R ir = R(1) / r;
  R h[3] = {dx * ir, dy * ir, dz * ir};
  cx<R> A, B, dA, dB, S3;
  kernel_coeffs<R, true, DYN>(k, r, s, is2, A, B, dA, dB, S3);
  acc_TT_from<R>(k, wq, r, h, n, A, B, dA, dB, S3, acc);
}

template <typename R, bool DYN, int DC>
__device__ __forceinline__ void acc_dl(const KC<R>& k, R wq, R dx, R dy, R dz, const R* n, cx<R> s, cx<R> is2,
                                       cx<R>* acc) {
  if constexpr (DC == 0)
    acc_TT<R, DYN>(k, wq, dx, dy, dz, n, s, is2, acc);
  else
    acc_dTT<R, DYN, DC>(k, wq, dx, dy, dz, n, s, is2, acc);
}

// static Kelvin T0^T (real), [a*3+b] = T0_ba
template <typename R>
__device__ __forceinline__ void acc_T0T(R nu, R wq, R dx, R dy, R dz, const R* n, R* acc) {
  R r2 = dx * dx + dy * dy + dz * dz;
  R ir = R(1) / sqrt(r2);
  R h[3] = {dx * ir, dy * ir, dz * ir};
  R rn = h[0] * n[0] + h[1] * n[1] + h[2] * n[2];
  R a12 = R(1) - R(2) * nu;
  R f = -wq / (R(8.0 * M_PI) * (R(1) - nu) * r2);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // T0_ba = -[rn((1-2nu) d + 3 h_b h_a) + (1-2nu)(h_b n_a - n_b h_a)] / (8 pi (1-nu) r^2)
      R v = rn * ((a == b ? a12 : R(0)) + R(3) * h[a] * h[b]) + a12 * (h[b] * n[a] - n[b] * h[a]);
      acc[3 * a + b] += f * v;
    }
}

template <typename R, int DC>
__device__ __forceinline__ void acc_dl0(const KC<R>& k, R nu, R wq, R dx, R dy, R dz, const R* n, R* acc) {
  if constexpr (DC == 0)
    acc_T0T<R>(nu, wq, dx, dy, dz, n, acc);
  else
    acc_dT0T_dnu<R>(nu, wq * (DC == 1 ? k.dnu1 : k.dnu2), dx, dy, dz, n, acc);
}

__device__ __forceinline__ int rule_index(double dist, double h) {
  const double hb = h * (1.0 - 1e-12);
  if (dist >= rule_dist(0) * hb) return 0;
  if (dist >= rule_dist(1) * hb) return 1;
  if (dist >= rule_dist(2) * hb) return 2;
  return 3;
}

// device view of a mesh + material for entry evaluation
struct EntryView {
  const ElemGeo* geo;
  const int32_t* tri;
  const double* nodes;
  const double* cent;
  const int32_t* ne_ptr;
  const int32_t* ne_elem;
  const int32_t* ne_loc;
  const double* rb;          // n_nodes x 9 (node rows, double layer) or null
  const double* rb_dnu;      // its derivative in nu (wave-speed derivative operators) or null
  const double2* s;          // K
  const double2* inv_s2;     // K
  const float4* sw;          // [K][2] s_k / c_a float-float (MIXED path)
  const float4* ef;          // [n_tris][4] FP32 element frames (MIXED path)
  const float4* cff;         // [n_tris][2] centroid (hi, h), (lo, 0) (MIXED path)
  const float4* nff;         // [n_nodes][2] node (hi, 0), (lo, 0) (MIXED path)
  int64_t n_nodes, n_tris;
  int32_t K;
  double nu;
  KC<double> kd;
  KC<float> kf;
};

template <int ROWS>
__device__ __forceinline__ const double* row_point(const EntryView& v, int i) {
  return ROWS == BEM_ROWS_NODES ? v.nodes + 3 * (int64_t)i : v.cent + 3 * (int64_t)i;
}

// ---- single layer -----------------------------------------------------------
// V[i, e](s) = int_e U(y - x_i, s) dy; R = compute type of regular far rules;
// DC = 1, 2: the wave-speed derivative dV/dc_a (integrand dU/dc_a)
template <typename R, int ROWS, int DC>
__device__ void entry_sl(const EntryView& v, int i, int e, cx<double> s, cx<double> is2, cx<double>* out) {
  const ElemGeo& g = v.geo[e];
  const double* x = row_point<ROWS>(v, i);
  const int32_t* t = v.tri + 3 * (int64_t)e;
  int apex = -1;  // singular: local vertex == node row, or 3 for own centroid
  if (ROWS == BEM_ROWS_NODES) {
    apex = (t[0] == i) ? 0 : (t[1] == i) ? 1 : (t[2] == i) ? 2 : -1;
  } else if (e == i) {
    apex = 3;
  }
  cx<double> SA = {0, 0}, SB[6] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
  if (apex >= 0) {
    double P[3][3];
    for (int k = 0; k < 3; ++k) {
      P[0][k] = g.p0[k];
      P[1][k] = g.p0[k] + g.e1[k];
      P[2][k] = g.p0[k] + g.e2[k];
    }
    const int nsub = apex == 3 ? 3 : 1;
    for (int sub = 0; sub < nsub; ++sub) {
      double A[3], Bv[3], Cv[3];
      for (int k = 0; k < 3; ++k) {
        if (apex == 3) {
          A[k] = x[k];
          Bv[k] = P[sub][k];
          Cv[k] = P[(sub + 1) % 3][k];
        } else {
          A[k] = P[apex][k];
          Bv[k] = P[(apex + 1) % 3][k];
          Cv[k] = P[(apex + 2) % 3][k];
        }
      }
      double ba[3] = {Bv[0] - A[0], Bv[1] - A[1], Bv[2] - A[2]};
      double cb[3] = {Cv[0] - Bv[0], Cv[1] - Bv[1], Cv[2] - Bv[2]};
      double ca[3] = {Cv[0] - A[0], Cv[1] - A[1], Cv[2] - A[2]};
      double cr0 = ba[1] * ca[2] - ba[2] * ca[1], cr1 = ba[2] * ca[0] - ba[0] * ca[2],
             cr2 = ba[0] * ca[1] - ba[1] * ca[0];
      double ar2 = sqrt(cr0 * cr0 + cr1 * cr1 + cr2 * cr2);
      double ax[3] = {A[0] - x[0], A[1] - x[1], A[2] - x[2]};
      for (int a = 0; a < kSingN; ++a) {
        double u = c_gl16[a], wu = c_gl16[16 + a];
        for (int b = 0; b < kSingN; ++b) {
          double vv = c_gl16[b], wv = c_gl16[16 + b];
          double d0 = ax[0] + u * (ba[0] + vv * cb[0]);
          double d1 = ax[1] + u * (ba[1] + vv * cb[1]);
          double d2 = ax[2] + u * (ba[2] + vv * cb[2]);
          acc_sl<double, DC>(v.kd, wu * wv * ar2 * u, d0, d1, d2, s, is2, SA, SB);
        }
      }
    }
  } else {
    double dc[3] = {g.c[0] - x[0], g.c[1] - x[1], g.c[2] - x[2]};
    double dist = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
    int ri = rule_index(dist, g.h);
    const int q0 = rule_offset(ri), q1 = rule_offset(ri + 1);
    double d0[3] = {g.p0[0] - x[0], g.p0[1] - x[1], g.p0[2] - x[2]};
    if (sizeof(R) == sizeof(float) && ri < 2) {
      // regular far rule in FP32: geometry relative to x, then all FP32
      cx<float> SAf = {0, 0}, SBf[6] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}};
      float f0[3] = {(float)d0[0], (float)d0[1], (float)d0[2]};
      float f1[3] = {(float)g.e1[0], (float)g.e1[1], (float)g.e1[2]};
      float f2[3] = {(float)g.e2[0], (float)g.e2[1], (float)g.e2[2]};
      cx<float> sf = {(float)s.x, (float)s.y}, isf = {(float)is2.x, (float)is2.y};
      float ar = (float)g.area2;
      for (int q = q0; q < q1; ++q) {
        float xi = (float)c_rule[3 * q], et = (float)c_rule[3 * q + 1], wq = (float)c_rule[3 * q + 2] * ar;
        acc_sl<float, DC>(v.kf, wq, f0[0] + xi * f1[0] + et * f2[0], f0[1] + xi * f1[1] + et * f2[1],
                          f0[2] + xi * f1[2] + et * f2[2], sf, isf, SAf, SBf);
      }
      SA = {SAf.x, SAf.y};
      for (int c = 0; c < 6; ++c) SB[c] = {SBf[c].x, SBf[c].y};
    } else {
      for (int q = q0; q < q1; ++q) {
        double xi = c_rule[3 * q], et = c_rule[3 * q + 1], wq = c_rule[3 * q + 2] * g.area2;
        acc_sl<double, DC>(v.kd, wq, d0[0] + xi * g.e1[0] + et * g.e2[0], d0[1] + xi * g.e1[1] + et * g.e2[1],
                           d0[2] + xi * g.e1[2] + et * g.e2[2], s, is2, SA, SB);
      }
    }
  }
  // U = (SA I + SB) / (4 pi rho)
  const double c = v.kd.inv4pirho;
  out[0] = c * (SA + SB[0]);
  out[1] = c * SB[1];
  out[2] = c * SB[2];
  out[3] = c * SB[1];
  out[4] = c * (SA + SB[3]);
  out[5] = c * SB[4];
  out[6] = c * SB[2];
  out[7] = c * SB[4];
  out[8] = c * (SA + SB[5]);
}

// CPV int_e rh / r^2 dA for x inside the flat element (closed form per
// sub-triangle (x; P_a, P_b) in polar coordinates about x).
__device__ void cpv_rh_r2(const ElemGeo& g, const double* x, double* G) {
  double P[3][3];
  for (int k = 0; k < 3; ++k) {
    P[0][k] = g.p0[k];
    P[1][k] = g.p0[k] + g.e1[k];
    P[2][k] = g.p0[k] + g.e2[k];
  }
  G[0] = G[1] = G[2] = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double* Pa = P[a];
    const double* Pb = P[(a + 1) % 3];
    double t[3] = {Pb[0] - Pa[0], Pb[1] - Pa[1], Pb[2] - Pa[2]};
    double tl = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    for (int k = 0; k < 3; ++k) t[k] /= tl;
    double xa = (x[0] - Pa[0]) * t[0] + (x[1] - Pa[1]) * t[1] + (x[2] - Pa[2]) * t[2];
    double F[3] = {Pa[0] + xa * t[0], Pa[1] + xa * t[1], Pa[2] + xa * t[2]};
    double e0[3] = {F[0] - x[0], F[1] - x[1], F[2] - x[2]};
    double h = sqrt(e0[0] * e0[0] + e0[1] * e0[1] + e0[2] * e0[2]);
    for (int k = 0; k < 3; ++k) e0[k] /= h;
    double ta = (Pa[0] - F[0]) * t[0] + (Pa[1] - F[1]) * t[1] + (Pa[2] - F[2]) * t[2];
    double tb = (Pb[0] - F[0]) * t[0] + (Pb[1] - F[1]) * t[1] + (Pb[2] - F[2]) * t[2];
    double Ra = sqrt(h * h + ta * ta), Rb = sqrt(h * h + tb * tb);
    // int cos(phi) ln(h/cos phi) = sin(phi)(ln R + 1) - asinh(tan phi)
    double p0 = (tb / Rb) * (log(Rb) + 1.0) - asinh(tb / h) - ((ta / Ra) * (log(Ra) + 1.0) - asinh(ta / h));
    // int sin(phi) ln(h/cos phi) = -cos(phi)(ln R + 1)
    double p1 = -(h / Rb) * (log(Rb) + 1.0) + (h / Ra) * (log(Ra) + 1.0);
    for (int k = 0; k < 3; ++k) G[k] += e0[k] * p0 + t[k] * p1;
  }
}

// ---- double layer (C + K) -----------------------------------------------------
// (C+K)[i, j](s) = sum_{e ni j} int_e T^T(x_i, y, s) phi_j(y) dy with the
// singular treatments (node rows: Duffy + rigid-body static diagonal;
// centroid rows: free term I/6, CPV of the static part, Duffy remainders).
// DC = 1, 2: the wave-speed derivative d(C + K)/dc_a (integrands dT/dc_a and
// dT0/dc_a, CPV coefficient through nu, no free term, rigid-body diagonal
// of dT0/dnu times dnu/dc_a).
template <typename R, int ROWS, int DC>
__device__ void entry_dl(const EntryView& v, int i, int j, cx<double> s, cx<double> is2, cx<double>* out) {
  const double* x = row_point<ROWS>(v, i);
  cx<double> acc[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) acc[c] = {0, 0};
  double acc0[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};   // static parts (real)
  const int p0 = v.ne_ptr[j], p1 = v.ne_ptr[j + 1];
  for (int p = p0; p < p1; ++p) {
    const int e = v.ne_elem[p];
    const int a = v.ne_loc[p];   // local vertex of column node j in e
    const ElemGeo& g = v.geo[e];
    const int32_t* t = v.tri + 3 * (int64_t)e;
    int apex = -1;
    if (ROWS == BEM_ROWS_NODES) {
      apex = (t[0] == i) ? 0 : (t[1] == i) ? 1 : (t[2] == i) ? 2 : -1;
    } else if (e == i) {
      apex = 3;
    }
    const double n[3] = {g.n[0], g.n[1], g.n[2]};
    if (apex < 0) {
      double dc[3] = {g.c[0] - x[0], g.c[1] - x[1], g.c[2] - x[2]};
      double dist = sqrt(dc[0] * dc[0] + dc[1] * dc[1] + dc[2] * dc[2]);
      int ri = rule_index(dist, g.h);
      const int q0 = rule_offset(ri), q1 = rule_offset(ri + 1);
      double d0[3] = {g.p0[0] - x[0], g.p0[1] - x[1], g.p0[2] - x[2]};
      if (sizeof(R) == sizeof(float) && ri < 2) {
        cx<float> af[9];
#pragma unroll
        for (int c = 0; c < 9; ++c) af[c] = {0.f, 0.f};
        float f0[3] = {(float)d0[0], (float)d0[1], (float)d0[2]};
        float f1[3] = {(float)g.e1[0], (float)g.e1[1], (float)g.e1[2]};
        float f2[3] = {(float)g.e2[0], (float)g.e2[1], (float)g.e2[2]};
        float nf[3] = {(float)n[0], (float)n[1], (float)n[2]};
        cx<float> sf = {(float)s.x, (float)s.y}, isf = {(float)is2.x, (float)is2.y};
        float ar = (float)g.area2;
        for (int q = q0; q < q1; ++q) {
          float xi = (float)c_rule[3 * q], et = (float)c_rule[3 * q + 1];
          float phi = a == 0 ? 1.f - xi - et : (a == 1 ? xi : et);
          float wq = (float)c_rule[3 * q + 2] * ar * phi;
          acc_dl<float, false, DC>(v.kf, wq, f0[0] + xi * f1[0] + et * f2[0], f0[1] + xi * f1[1] + et * f2[1],
                                   f0[2] + xi * f1[2] + et * f2[2], nf, sf, isf, af);
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) acc[c] = acc[c] + mk<double>(af[c].x, af[c].y);
      } else {
        for (int q = q0; q < q1; ++q) {
          double xi = c_rule[3 * q], et = c_rule[3 * q + 1];
          double phi = a == 0 ? 1.0 - xi - et : (a == 1 ? xi : et);
          double wq = c_rule[3 * q + 2] * g.area2 * phi;
          acc_dl<double, false, DC>(v.kd, wq, d0[0] + xi * g.e1[0] + et * g.e2[0],
                                    d0[1] + xi * g.e1[1] + et * g.e2[1], d0[2] + xi * g.e1[2] + et * g.e2[2], n, s,
                                    is2, acc);
        }
      }
      continue;
    }
    // singular element: Duffy sub-triangles with apex at x_i
    double P[3][3];
    for (int k = 0; k < 3; ++k) {
      P[0][k] = g.p0[k];
      P[1][k] = g.p0[k] + g.e1[k];
      P[2][k] = g.p0[k] + g.e2[k];
    }
    const int nsub = apex == 3 ? 3 : 1;
    for (int sub = 0; sub < nsub; ++sub) {
      double A[3], Bv[3], Cv[3];
      int lb, lc;  // local vertices of B and C
      if (apex == 3) {
        lb = sub;
        lc = (sub + 1) % 3;
        for (int k = 0; k < 3; ++k) A[k] = x[k];
      } else {
        lb = (apex + 1) % 3;
        lc = (apex + 2) % 3;
        for (int k = 0; k < 3; ++k) A[k] = P[apex][k];
      }
      for (int k = 0; k < 3; ++k) {
        Bv[k] = P[lb][k];
        Cv[k] = P[lc][k];
      }
      double ba[3] = {Bv[0] - A[0], Bv[1] - A[1], Bv[2] - A[2]};
      double cb[3] = {Cv[0] - Bv[0], Cv[1] - Bv[1], Cv[2] - Bv[2]};
      double ca[3] = {Cv[0] - A[0], Cv[1] - A[1], Cv[2] - A[2]};
      double cr0 = ba[1] * ca[2] - ba[2] * ca[1], cr1 = ba[2] * ca[0] - ba[0] * ca[2],
             cr2 = ba[0] * ca[1] - ba[1] * ca[0];
      double ar2 = sqrt(cr0 * cr0 + cr1 * cr1 + cr2 * cr2);
      double ax[3] = {A[0] - x[0], A[1] - x[1], A[2] - x[2]};
      for (int qa = 0; qa < kSingN; ++qa) {
        double u = c_gl16[qa], wu = c_gl16[16 + qa];
        for (int qb = 0; qb < kSingN; ++qb) {
          double vv = c_gl16[qb], wv = c_gl16[16 + qb];
          double d0 = ax[0] + u * (ba[0] + vv * cb[0]);
          double d1 = ax[1] + u * (ba[1] + vv * cb[1]);
          double d2 = ax[2] + u * (ba[2] + vv * cb[2]);
          double wq = wu * wv * ar2 * u;
          // barycentric coordinate of local vertex a at the Duffy point
          double lam_b = u * (1.0 - vv), lam_c = u * vv;
          double phi;
          if (apex == 3) {
            phi = (1.0 - u) / 3.0 + (a == lb ? lam_b : 0.0) + (a == lc ? lam_c : 0.0);
          } else {
            phi = (a == apex) ? 1.0 - u : (a == lb ? lam_b : lam_c);
          }
          if (apex == 3) {
            acc_dl<double, true, DC>(v.kd, wq * phi, d0, d1, d2, n, s, is2, acc);
            acc_dl0<double, DC>(v.kd, v.nu, wq * (phi - 1.0 / 3.0), d0, d1, d2, n, acc0);
          } else if (a == apex) {
            acc_dl<double, true, DC>(v.kd, wq * phi, d0, d1, d2, n, s, is2, acc);
          } else {
            acc_dl<double, false, DC>(v.kd, wq * phi, d0, d1, d2, n, s, is2, acc);
          }
        }
      }
    }
    if (apex == 3) {
      // free term C = I/2 at the centroid: I/6 per vertex; CPV of T0^T / 3:
      // CPV T0^T_ab = -(1-2nu)(G_b n_a - n_b G_a) / (8 pi (1-nu))
      // (DC: d/dnu of -(1-2nu)/(1-nu) is 1/(1-nu)^2; the free term is fixed)
      double G[3];
      cpv_rh_r2(g, x, G);
      const double f = DC == 0 ? -(1.0 - 2.0 * v.nu) / (8.0 * M_PI * (1.0 - v.nu)) / 3.0
                               : (DC == 1 ? v.kd.dnu1 : v.kd.dnu2) / (8.0 * M_PI * (1.0 - v.nu) * (1.0 - v.nu)) / 3.0;
      const double fr = DC == 0 ? 1.0 / 6.0 : 0.0;
      for (int aa = 0; aa < 3; ++aa)
        for (int bb = 0; bb < 3; ++bb) acc0[3 * aa + bb] += f * (G[bb] * n[aa] - n[bb] * G[aa]) + (aa == bb ? fr : 0.0);
    }
  }
  if (ROWS == BEM_ROWS_NODES && j == i) {
    if (DC == 0 && v.rb) {
      for (int c = 0; c < 9; ++c) acc0[c] += v.rb[9 * (int64_t)i + c];
    } else if (DC != 0 && v.rb_dnu) {
      const double dn = DC == 1 ? v.kd.dnu1 : v.kd.dnu2;
      for (int c = 0; c < 9; ++c) acc0[c] += dn * v.rb_dnu[9 * (int64_t)i + c];
    }
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) out[c] = {acc[c].x + acc0[c], acc[c].y};
}

// launch with compile-time (kernel, rows): LAUNCH may use KK and RR
#define GCQ_DISPATCH_ROWS(KIND, rows, LAUNCH)                                                   \
  do {                                                                                           \
    if ((rows) == BEM_ROWS_NODES) {                                                              \
      constexpr int KK = KIND, RR = BEM_ROWS_NODES;                                              \
      LAUNCH;                                                                                    \
    } else {                                                                                     \
      constexpr int KK = KIND, RR = BEM_ROWS_CENTROIDS;                                          \
      LAUNCH;                                                                                    \
    }                                                                                            \
  } while (0)
#define GCQ_DISPATCH(kernel, rows, LAUNCH)                                                       \
  do {                                                                                           \
    if ((kernel) == BEM_SL)                                                                      \
      GCQ_DISPATCH_ROWS(BEM_SL, rows, LAUNCH);                                                   \
    else if ((kernel) == BEM_DL)                                                                 \
      GCQ_DISPATCH_ROWS(BEM_DL, rows, LAUNCH);                                                   \
    else if ((kernel) == BEM_SL_DCP)                                                             \
      GCQ_DISPATCH_ROWS(BEM_SL_DCP, rows, LAUNCH);                                               \
    else if ((kernel) == BEM_SL_DCS)                                                             \
      GCQ_DISPATCH_ROWS(BEM_SL_DCS, rows, LAUNCH);                                               \
    else if ((kernel) == BEM_DL_DCP)                                                             \
      GCQ_DISPATCH_ROWS(BEM_DL_DCP, rows, LAUNCH);                                               \
    else                                                                                         \
      GCQ_DISPATCH_ROWS(BEM_DL_DCS, rows, LAUNCH);                                               \
  } while (0)

}  // namespace gcq
