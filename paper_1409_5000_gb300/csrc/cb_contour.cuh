// FP64 building blocks for functions of the small Lanczos tridiagonal T.
//
//  * lambda_max: the largest eigenvalue of T by Laguerre's iteration on
//    det(xI - T), started above the Gershgorin bound.  For a polynomial
//    with only real roots, Laguerre's method started above the largest root
//    decreases monotonically to it and converges cubically.  f'/f and f''/f
//    come from the ratio form of the three-term determinant recurrence
//    (r_k = p_k / p_{k-1}), which cannot overflow.
//  * contour nodes: exp(x) on (-inf, 0] as the trapezoid rule for the
//    Cauchy integral over the cotangent contour of Trefethen, Weideman &
//    Schmelzer ("Talbot quadratures and rational approximations", BIT 46,
//    2006): z(t) = N (a t cot(b t) - c + i d t), N = 24, error ~2e-14.
//    Nodes come in conjugate pairs; only the 12 in the upper half plane are
//    evaluated and the real result is 2 Re of their sum.
//  * thomas_e1: (z I - (T - theta I))^{-1} e1 for complex z (Thomas
//    algorithm; z I - S is complex symmetric tridiagonal).
#pragma once

#include "cb_internal.cuh"

namespace cb {
namespace contour {

constexpr int kNodes = 24;
constexpr int kHalf = kNodes / 2;
constexpr double kA = 0.5017, kB = 0.6407, kC = 0.6122, kD = 0.2645;
constexpr double kPi = 3.14159265358979323846;

struct cplx {
  double re, im;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ cplx cinv(cplx a) {
  const double d = 1.0 / (a.re * a.re + a.im * a.im);
  return {a.re * d, -a.im * d};
}

// f'/f and (f'/f)^2 - f''/f of f(x) = det(xI - T) via the ratios
// r_k = p_k / p_{k-1} of the leading principal minors and their derivatives
// (one reciprocal per k).  Returns false if some r_k <= 0, i.e. x is not
// above every eigenvalue of every leading block.  R is float or double.
template <typename R>
__device__ inline bool laguerre_terms(const double *al, const double *be, int M, R x, R *G,
                                      R *H) {
  R r = x - (R)al[0], rd = R(1), rdd = R(0);
  if (!(r > R(0))) return false;
  R ir = R(1) / r;
  R g = rd * ir;
  R h = g * g - rdd * ir;
  for (int k = 1; k < M; ++k) {
    const R b2 = (R)be[k - 1] * (R)be[k - 1];
    const R q = b2 * ir;
    const R nr = (x - (R)al[k]) - q;
    const R nrd = R(1) + q * ir * rd;
    const R nrdd = q * ir * (rdd - R(2) * rd * rd * ir);
    r = nr;
    rd = nrd;
    rdd = nrdd;
    if (!(r > R(0))) return false;
    ir = R(1) / r;
    const R gk = rd * ir;
    g += gk;
    h += gk * gk - rdd * ir;
  }
  *G = g;
  *H = h;
  return true;
}

// One Laguerre step from x (above the largest root); false when x is not
// above the spectrum or the step is not finite.
template <typename R>
__device__ inline bool laguerre_step(const double *al, const double *be, int M, R x, R *step) {
  R G, H;
  if (!laguerre_terms<R>(al, be, M, x, &G, &H)) return false;
  const R disc = (R)(M - 1) * ((R)M * H - G * G);
  const R den = G + sqrt(disc > R(0) ? disc : R(0));
  if (!(den > R(0))) return false;
  *step = (R)M / den;
  return true;
}

// Largest eigenvalue of tridiag(be, al, be) (be[0..M-2] used).  Laguerre's
// iteration from above the Gershgorin bound runs in FP32 until its step is
// below 1e-6 relative (FP64 arithmetic is scarce on GB300), then two FP64
// steps polish the result: the convergence is cubic, so the FP32 estimate
// turns into an FP64-accurate one.  theta only has to lie within rounding
// of lambda_max for the contour rule to keep its accuracy.
__device__ inline double lambda_max(const double *al, const double *be, int M) {
  if (M == 1) return al[0];
  double x0 = -1e300;
  for (int i = 0; i < M; ++i) {
    const double lo = i > 0 ? fabs(be[i - 1]) : 0.0;
    const double hi = i < M - 1 ? fabs(be[i]) : 0.0;
    x0 = fmax(x0, al[i] + lo + hi);
  }
  x0 += 1e-3 * (fabs(x0) + 1.0);  // strictly above the spectrum, also in FP32
  float xf = (float)x0;
  if ((double)xf < x0) xf = nextafterf(xf, 3.0e38f);
  float st;
  if (laguerre_step<float>(al, be, M, xf, &st)) {
    for (int it = 0; it < 40; ++it) {
      const float nx = xf - st;
      float st2;
      if (!laguerre_step<float>(al, be, M, nx, &st2)) break;  // nx not above: keep xf
      xf = nx;
      st = st2;
      if (st <= 1e-6f * (fabsf(xf) + 1.0f)) break;
    }
  }
  double x = xf;
  for (int it = 0; it < 2; ++it) {  // FP64 polish (a failed step leaves x above the root)
    double sd;
    if (!laguerre_step<double>(al, be, M, x, &sd)) break;
    x -= sd;
  }
  return x;
}

// Node z and weight w = e^z z'(t) / (i N) of upper-half node q (0..kHalf-1).
__device__ inline void node(int q, cplx *z, cplx *w) {
  const int k = kHalf + q;
  const double t = -kPi + (k + 0.5) * (2.0 * kPi / kNodes);
  double sn, cs;
  sincos(kB * t, &sn, &cs);
  const double cot = cs / sn;
  *z = {kNodes * (kA * t * cot - kC), kNodes * kD * t};
  const cplx dz = {kNodes * (kA * cot - kA * kB * t / (sn * sn)), kNodes * kD};
  double es, ec;
  sincos(z->im, &es, &ec);
  const double ez = exp(z->re);
  const cplx ezdz = cmul({ez * ec, ez * es}, dz);
  *w = {ezdz.im / kNodes, -ezdz.re / kNodes};
}

// x = (z I - (T - theta I))^{-1} e1; diag z - (al_i - theta), off-diagonal -be_i.
// cp is scratch of length M.
__device__ inline void thomas_e1(const double *al, const double *be, int M, double theta, cplx z,
                                 cplx *cp, cplx *x) {
  cplx den = {z.re - (al[0] - theta), z.im};
  cplx inv = cinv(den);
  const double b0 = M > 1 ? be[0] : 0.0;
  cp[0] = {-b0 * inv.re, -b0 * inv.im};
  x[0] = inv;
  for (int i = 1; i < M; ++i) {
    const double b = be[i - 1];
    den = {z.re - (al[i] - theta) + b * cp[i - 1].re, z.im + b * cp[i - 1].im};
    inv = cinv(den);
    const double bn = (i < M - 1) ? be[i] : 0.0;
    cp[i] = {-bn * inv.re, -bn * inv.im};
    x[i] = cmul({b * x[i - 1].re, b * x[i - 1].im}, inv);
  }
  for (int i = M - 2; i >= 0; --i) {
    const cplx t2 = cmul(cp[i], x[i + 1]);
    x[i] = {x[i].re - t2.re, x[i].im - t2.im};
  }
}

}  // namespace contour
}  // namespace cb
