// FP64 tridiagonal step of the Krylov approximation: (theta, c) with
// theta = lambda_max(T) and c = exp(T - theta I) e1, one warp per
// realisation.
//
// The Lanczos approximation of e^A 1 (paper, "Identification algorithm")
// projects A onto K_m(A, 1); what remains is the small matrix function
// exp(T_m) e1.  GB300 executes FP64 at a small fraction of its FP32 rate,
// so the solve is organised to use few FP64 operations and to run the
// independent parts in parallel lanes:
//
//  1. theta = lambda_max(T) by Laguerre's iteration on det(xI - T), started
//     above the Gershgorin bound.  For a polynomial with only real roots,
//     Laguerre's method started above the largest root decreases
//     monotonically to it and converges cubically.  f'/f and f''/f come
//     from the ratio form of the three-term determinant recurrence, which
//     cannot overflow.
//  2. exp(S) e1 with S = T - theta I <= 0 by the rational approximation
//     that the trapezoid rule gives for the Cauchy integral of e^z over a
//     Hankel contour (Trefethen, Weideman & Schmelzer, "Talbot quadratures
//     and rational approximations", BIT 46 (2006)), with their cotangent
//     contour z(t) = N (a t cot(b t) - c + i d t), N = 24 nodes:
//         exp(S) e1 ~= sum_k w_k (z_k I - S)^{-1} e1,
//         w_k = e^{z_k} z'(t_k) / (i N).
//     Its error is about 2e-14 uniformly on (-inf, 0].  The nodes come in
//     conjugate pairs, so 12 complex tridiagonal solves (Thomas algorithm,
//     one per lane) give the real result as 2 Re(sum over the upper half).
//  3. gamma_j = beta0 * c_j * scale_j, the weight of the stored basis vector
//     W_j in the combine step.
#include "cb_internal.cuh"

namespace cb {

namespace {

constexpr int kNodes = 24;  // contour nodes (12 solves)
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

// f'/f and (f'/f)^2 - f''/f of f(x) = det(xI - T) at x, via the ratios
// r_k = p_k / p_{k-1} of the leading principal minors.  Returns false if
// some r_k <= 0 (x is not above every eigenvalue of every leading block).
__device__ bool laguerre_terms(const double *al, const double *be, int M, double x, double *G,
                               double *H) {
  double r = x - al[0], rd = 1.0, rdd = 0.0;  // r_1 and its x-derivatives
  if (!(r > 0.0)) return false;
  double g = rd / r;
  double h = g * g - rdd / r;
  for (int k = 1; k < M; ++k) {
    const double b2 = be[k - 1] * be[k - 1];
    const double ir = 1.0 / r;
    const double q = b2 * ir;
    const double nr = (x - al[k]) - q;
    const double nrd = 1.0 + q * ir * rd;
    const double nrdd = b2 * ir * ir * (rdd - 2.0 * rd * rd * ir);
    r = nr;
    rd = nrd;
    rdd = nrdd;
    if (!(r > 0.0)) return false;
    const double gk = rd / r;
    g += gk;
    h += gk * gk - rdd / r;
  }
  *G = g;
  *H = h;
  return true;
}

__device__ double lambda_max(const double *al, const double *be, int M) {
  if (M == 1) return al[0];
  double x = -1e300;
  for (int i = 0; i < M; ++i) {
    const double lo = i > 0 ? fabs(be[i - 1]) : 0.0;
    const double hi = i < M - 1 ? fabs(be[i]) : 0.0;
    x = fmax(x, al[i] + lo + hi);
  }
  x += 1e-6 * (fabs(x) + 1.0);  // strictly above the spectrum
  for (int it = 0; it < 64; ++it) {
    double G, H;
    if (!laguerre_terms(al, be, M, x, &G, &H)) break;  // stepped below: keep x
    const double disc = fmax((M - 1.0) * (M * H - G * G), 0.0);
    const double den = G + sqrt(disc);
    if (!(den > 0.0)) break;
    const double step = M / den;
    const double nx = x - step;
    double G2, H2;
    if (!laguerre_terms(al, be, M, nx, &G2, &H2)) {
      // rounding put nx at or below the root: x is within one step of it
      x = nx;
      break;
    }
    x = nx;
    if (step <= 1e-15 * fabs(x) + 1e-300) break;
  }
  return x;
}

}  // namespace

__global__ void __launch_bounds__(32) tridiag_kernel(Scalars sc, const InstDesc *inst,
                                                     uint32_t r0) {
  __shared__ double s_al[CB_MAX_M], s_be[CB_MAX_M];
  __shared__ double s_c[12][CB_MAX_M];
  __shared__ double s_theta;
  const uint32_t r = r0 + blockIdx.x;
  const uint32_t lane = threadIdx.x;
  const uint32_t ms = sc.ms;
  const int M = (int)sc.meff[r];
  if (sc.status[r] != CB_OK || M < 1) {
    if (lane == 0) sc.theta[r] = 0.0;
    return;
  }
  for (int i = lane; i < M; i += 32) {
    s_al[i] = sc.alpha[r * ms + i];
    s_be[i] = sc.beta[r * ms + i];
  }
  __syncwarp();
  if (lane == 0) s_theta = lambda_max(s_al, s_be, M);
  __syncwarp();
  const double theta = s_theta;

  if (lane < kNodes / 2) {
    // node in the upper half plane: t_k = -pi + (k + 1/2) 2 pi / N, k >= N/2
    const int k = kNodes / 2 + (int)lane;
    const double t = -kPi + (k + 0.5) * (2.0 * kPi / kNodes);
    double sn, cs;
    sincos(kB * t, &sn, &cs);
    const double cot = cs / sn;
    const cplx z = {kNodes * (kA * t * cot - kC), kNodes * kD * t};
    const cplx dz = {kNodes * (kA * cot - kA * kB * t / (sn * sn)), kNodes * kD};
    double es, ec;
    sincos(z.im, &es, &ec);
    const double ez = exp(z.re);
    // w = e^z z' / (i N) = -i e^z z' / N
    const cplx ezdz = cmul({ez * ec, ez * es}, dz);
    const cplx w = {ezdz.im / kNodes, -ezdz.re / kNodes};
    // Thomas algorithm for (z I - S) x = e1, S = T - theta I.
    // diag d_i = z - (alpha_i - theta); off-diagonal -beta_i.
    cplx cp[CB_MAX_M], xp[CB_MAX_M];
    cplx den = {z.re - (s_al[0] - theta), z.im};
    cplx inv = cinv(den);
    cp[0] = {-s_be[0] * inv.re, -s_be[0] * inv.im};
    xp[0] = inv;
    for (int i = 1; i < M; ++i) {
      const double b = s_be[i - 1];
      den = {z.re - (s_al[i] - theta) + b * cp[i - 1].re, z.im + b * cp[i - 1].im};
      inv = cinv(den);
      const double bn = (i < M - 1) ? s_be[i] : 0.0;
      cp[i] = {-bn * inv.re, -bn * inv.im};
      const cplx num = {b * xp[i - 1].re, b * xp[i - 1].im};
      xp[i] = cmul(num, inv);
    }
    cplx xn = xp[M - 1];
    s_c[lane][M - 1] = 2.0 * (w.re * xn.re - w.im * xn.im);
    for (int i = M - 2; i >= 0; --i) {
      const cplx t2 = cmul(cp[i], xn);
      xn = {xp[i].re - t2.re, xp[i].im - t2.im};
      s_c[lane][i] = 2.0 * (w.re * xn.re - w.im * xn.im);
    }
  }
  __syncwarp();
  const double beta0 = sqrt((double)inst[r].n);
  for (int i = lane; i < M; i += 32) {
    double c = 0.0;
    for (int q = 0; q < kNodes / 2; ++q) c += s_c[q][i];
    sc.gamma[r * ms + i] = beta0 * c * sc.scale[r * ms + i];
  }
  if (lane == 0) sc.theta[r] = theta;
}

int tridiag_run(cb_graph *h, uint32_t r0, uint32_t r1, int /*prec*/, cudaStream_t s) {
  const int tok = prof_begin(CB_K_TRIDIAG, s);
  tridiag_kernel<<<r1 - r0, 32, 0, s>>>(h->ws.sc, h->d_inst, r0);
  prof_end(tok, s);
  return cuda_error(cudaGetLastError(), "tridiag launch");
}

}  // namespace cb
