// Restarted Lanczos for e^A 1, batched over the realisations of a handle
// (the restarted Krylov method of the paper's ref [10], Afanasjew, Eiermann,
// Ernst & Guettel 2008).
//
// Cycle k runs m Lanczos steps from the last basis vector of cycle k-1 (the
// first cycle from 1), so the m + 1 basis vectors of the workspace serve any
// total depth.  After k cycles the approximation is
//     f_k = beta0 [V_1 ... V_k] exp(H_k) e1,
// with H_k block lower bidiagonal: T_1..T_k on the diagonal and the residual
// norm b_i of cycle i coupling the first row of block i+1 to the last column
// of block i.  H_k is block lower triangular, so the blocks of exp(H_k) e1
// that belong to earlier cycles do not change when a cycle is added; only
// the new block is computed.  With the contour rule
//     exp(S) ~= 2 Re sum_q w_q (z_q I - S)^{-1}        (cb_contour.cuh)
// block forward substitution gives, per contour node q,
//     block k of (z_q I - (H_k - theta I))^{-1} e1 = p_q^(k) x_q^(k),
//     x_q^(k) = (z_q I - (T_k - theta I))^{-1} e1,
//     p_q^(1) = 1,   p_q^(k+1) = p_q^(k) b_k [x_q^(k)]_m,
// and cycle k adds beta0 V_k 2 Re sum_q w_q p_q^(k) x_q^(k) to the result:
// the partial-fraction form of the restart in ref [10].
//
// The shift theta has to lie on or above the spectrum of H_k (the contour
// rule loses accuracy quickly to the right of 0: about 1e-9 relative at
// +0.5).  Cycle 1 takes lambda_max(T_1).  A later cycle whose
// lambda_max(T_k) is larger raises theta, rescales the accumulated result by
// exp(theta_old - theta_new) and recomputes the products p_q at the new
// shift from the stored T_i; this is exact, because
// exp(H - theta I) = exp(theta' - theta) exp(H - theta' I).
//
// Per cycle: the m Lanczos steps (cb_lanczos.cu, unchanged), one warp per
// realisation for the FP64 part (restart_tridiag_kernel), and one
// bandwidth-bound pass Y = rho Y + sum_j gamma_j W_j into an FP64
// accumulator (restart_combine_kernel).  The ensemble sum (eq. 5) runs once,
// after the last cycle.
#include <vector>

#include "cb_contour.cuh"

namespace cb {
namespace {

struct RState {
  double *hal, *hbe;  // [N][cmax][m] T of every finished cycle (recomputing p_q)
  double *couple;     // [N][cmax]    residual norm b_k of every finished cycle
  double *p;          // [N][kHalf][2] running products p_q (complex)
  double *theta;      // [N] current shift
  double *rho;        // [N] factor on the accumulated Y in this cycle
  double *rscale;     // [N] scale of W_0 in the next cycle; 0: finished
  double *blast;      // [N] last residual norm computed
  uint32_t *steps;    // [N] Lanczos steps over all cycles
  int32_t *status;    // [N] first failure, CB_OK otherwise
  uint32_t cmax, m;
};

// [(z I - (T - theta I))^{-1} e1]_M, the last entry: the forward sweep of the
// Thomas algorithm alone (back substitution leaves the last entry as is).
__device__ inline contour::cplx thomas_last(const double *al, const double *be, int M,
                                            double theta, contour::cplx z) {
  using namespace contour;
  cplx inv = cinv({z.re - (al[0] - theta), z.im});
  cplx cp = {-(M > 1 ? be[0] : 0.0) * inv.re, -(M > 1 ? be[0] : 0.0) * inv.im};
  cplx x = inv;
  for (int i = 1; i < M; ++i) {
    const double b = be[i - 1];
    inv = cinv({z.re - (al[i] - theta) + b * cp.re, z.im + b * cp.im});
    const double bn = (i < M - 1) ? be[i] : 0.0;
    x = cmul({b * x.re, b * x.im}, inv);
    cp = {-bn * inv.re, -bn * inv.im};
  }
  return x;
}

// One warp per realisation: the shift, the combine weights gamma_j of the
// current cycle's basis, and the state the next cycle starts from.
__global__ void __launch_bounds__(32) restart_tridiag_kernel(Scalars sc, RState rs,
                                                             const InstDesc *inst, uint32_t c) {
  using namespace contour;
  __shared__ double s_al[CB_MAX_M], s_be[CB_MAX_M];
  __shared__ double s_c[kHalf][CB_MAX_M];
  __shared__ double s_theta;
  __shared__ int s_recompute;
  const uint32_t r = blockIdx.x, lane = threadIdx.x, ms = sc.ms, m = rs.m;
  const bool active = c == 0 || rs.rscale[r] > 0.0;
  const int M = (int)sc.meff[r];
  if (!active || sc.status[r] != CB_OK || M < 1) {
    if (lane == 0) {
      if (sc.status[r] != CB_OK && rs.status[r] == CB_OK) rs.status[r] = sc.status[r];
      rs.rho[r] = 1.0;  // the accumulated result stays as it is
      rs.rscale[r] = 0.0;
    }
    return;
  }
  for (int i = lane; i < M; i += 32) {
    s_al[i] = sc.alpha[r * ms + i];
    s_be[i] = sc.beta[r * ms + i];
  }
  __syncwarp();
  if (lane == 0) {
    const double tk = lambda_max(s_al, s_be, M);
    const double told = rs.theta[r];
    const double tn = c == 0 ? tk : fmax(told, tk);
    rs.rho[r] = c == 0 ? 0.0 : exp(told - tn);
    rs.theta[r] = tn;
    s_theta = tn;
    s_recompute = c > 0 && tn > told;
  }
  __syncwarp();
  const double theta = s_theta;
  const bool more = M == (int)m && sc.scale[r * ms + m] > 0.0 && c + 1 < rs.cmax;
  if (lane < kHalf) {
    double *pq = rs.p + ((size_t)r * kHalf + lane) * 2;
    cplx z, w;
    node((int)lane, &z, &w);
    cplx p = {1.0, 0.0};
    if (s_recompute) {  // the shift moved: the products again from cycle 1
      for (uint32_t i = 0; i < c; ++i) {
        const size_t o = ((size_t)r * rs.cmax + i) * m;
        const cplx xl = thomas_last(rs.hal + o, rs.hbe + o, (int)m, theta, z);
        const double b = rs.couple[(size_t)r * rs.cmax + i];
        p = cmul(p, {b * xl.re, b * xl.im});
      }
    } else if (c > 0) {
      p = {pq[0], pq[1]};
    }
    cplx cp[CB_MAX_M], x[CB_MAX_M];
    thomas_e1(s_al, s_be, M, theta, z, cp, x);
    const cplx wp = cmul(w, p);
    for (int i = 0; i < M; ++i) s_c[lane][i] = 2.0 * (wp.re * x[i].re - wp.im * x[i].im);
    if (more) {
      const double b = sc.beta[r * ms + m - 1];
      const cplx np = cmul(p, {b * x[m - 1].re, b * x[m - 1].im});
      pq[0] = np.re;
      pq[1] = np.im;
    }
  }
  __syncwarp();
  const double beta0 = sqrt((double)inst[r].n);
  for (int i = lane; i < M; i += 32) {
    double cc = 0.0;
    for (int q = 0; q < kHalf; ++q) cc += s_c[q][i];
    sc.gamma[r * ms + i] = beta0 * cc * sc.scale[r * ms + i];
    if (more) {
      const size_t o = ((size_t)r * rs.cmax + c) * m + i;
      rs.hal[o] = s_al[i];
      rs.hbe[o] = s_be[i];
    }
  }
  if (lane == 0) {
    rs.steps[r] += (uint32_t)M;
    rs.blast[r] = sc.beta[r * ms + M - 1];
    if (more) rs.couple[(size_t)r * rs.cmax + c] = sc.beta[r * ms + m - 1];
    rs.rscale[r] = more ? sc.scale[r * ms + m] : 0.0;  // 1 / b_k: W_m becomes W_0
  }
}

// Y(i) = rho_r Y(i) + sum_j gamma_j W_j(i) over one finalize tile (kFinRows
// nodes of realisation r), 8 consecutive nodes per thread.  The first cycle
// writes Y; realisations with nothing to add leave it untouched.
template <typename T>
__global__ void __launch_bounds__(256) restart_combine_kernel(const T *V, uint64_t vs, Scalars sc,
                                                              const double *rho,
                                                              const InstDesc *inst,
                                                              const uint32_t *fin_inst, double *Y,
                                                              bool first) {
  __shared__ T s_g[CB_MAX_M];
  const uint32_t t = blockIdx.x;
  const uint32_t r = fin_inst[t];
  const InstDesc I = inst[r];
  const uint32_t ms = sc.ms;
  const uint32_t M = sc.status[r] == CB_OK ? sc.meff[r] : 0u;
  if (M == 0 && !first) return;
  for (uint32_t j = threadIdx.x; j < M; j += blockDim.x) s_g[j] = (T)sc.gamma[r * ms + j];
  __syncthreads();
  const uint32_t i0 = (t - I.fin_base) * kFinRows + 8 * threadIdx.x;
  if (i0 >= I.n) return;
  const uint32_t cnt = min(8u, I.n - i0);
  T acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = T(0);
  const T *w = V + I.node_base + i0;
  if (cnt == 8) {
    for (uint32_t j = 0; j < M; ++j) {
      T x[8];
      Vec8<T>::load(w + (uint64_t)j * vs, x);
      const T g = s_g[j];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] += g * x[q];
    }
  } else {
    for (uint32_t j = 0; j < M; ++j) {
      const T g = s_g[j];
      const T *wj = w + (uint64_t)j * vs;
#pragma unroll
      for (uint32_t q = 0; q < 8; ++q)
        if (q < cnt) acc[q] += g * wj[q];
    }
  }
  double *y = Y + I.node_base + i0;
  const double f = rho[r];
#pragma unroll
  for (uint32_t q = 0; q < 8; ++q)
    if (q < cnt) y[q] = first ? (double)acc[q] : f * y[q] + (double)acc[q];
}

// The shifts and sticky statuses go where the ensemble sum reads them.
__global__ void restart_finish_kernel(Scalars sc, RState rs, uint32_t n_inst) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_inst) return;
  sc.theta[r] = rs.theta[r];
  sc.status[r] = rs.status[r];
}

template <typename T>
int cycles_run(cb_graph *h, const RState &rs, double *Y, uint32_t m, uint32_t cycles, int prec,
               cudaStream_t s) {
  Workspace &W = h->ws;
  T *V = reinterpret_cast<T *>(W.V);
  prefer_shared(restart_tridiag_kernel);
  prefer_shared(restart_combine_kernel<T>);
  int rc = CB_OK;
  for (uint32_t c = 0; c < cycles && rc == CB_OK; ++c) {
    if (c > 0) {  // the last vector of the previous cycle starts this one
      const cudaError_t e = cudaMemcpyAsync(V, V + (uint64_t)m * W.vec_stride,
                                            W.vec_stride * sizeof(T), cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return cuda_error(e, "restart: basis copy");
    }
    rc = lanczos_run(h, W, 0, h->n_inst, m, prec, s, nullptr, 0, false, c ? rs.rscale : nullptr);
    if (rc != CB_OK) break;
    int tok = prof_begin(CB_K_TRIDIAG, s);
    restart_tridiag_kernel<<<h->n_inst, 32, 0, s>>>(W.sc, rs, h->d_inst, c);
    prof_end(tok, s);
    tok = prof_begin(CB_K_COMBINE, s);
    if (h->total_fin)
      restart_combine_kernel<T><<<h->total_fin, 256, 0, s>>>(V, W.vec_stride, W.sc, rs.rho,
                                                            h->d_inst, h->d_fin_inst, Y, c == 0);
    prof_end(tok, s);
    rc = cuda_error(cudaGetLastError(), "restart launch");
  }
  return rc;
}

}  // namespace
}  // namespace cb

using namespace cb;

CB_API int cb_ensemble_scores_restarted(cb_graph *h, uint32_t m, uint32_t cycles, int prec,
                                        uint32_t n_out, double *S, double *log_scale,
                                        cb_inst_report *rep, void *stream) {
  NvtxRange nvtx_range("cb_ensemble_scores_restarted");
  if (!h || !S || !log_scale) return set_error(CB_ERR_ARG, "cb_ensemble_scores_restarted: null argument");
  if (m < 1 || m > CB_MAX_M)
    return set_error(CB_ERR_ARG, "cb_ensemble_scores_restarted: need 1 <= m <= CB_MAX_M");
  if (cycles < 1 || cycles > CB_MAX_CYCLES)
    return set_error(CB_ERR_ARG, "cb_ensemble_scores_restarted: need 1 <= cycles <= CB_MAX_CYCLES");
  const bool reorth = split_prec(prec);
  if (prec != CB_FP32 && prec != CB_FP64)
    return set_error(CB_ERR_ARG, "cb_ensemble_scores_restarted: bad precision");
  h->reorth = reorth;  // within each cycle
  if (n_out < h->n_max) return set_error(CB_ERR_ARG, "cb_ensemble_scores_restarted: n_out < largest n");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = ensure_workspace(h, h->ws, m, prec, s);
  if (rc != CB_OK) return rc;
  h->basis_m = 0;  // the workspace no longer holds the basis of K_m(A, 1)
  const uint32_t N = h->n_inst;
  const size_t hist = (size_t)N * cycles * m;
  const size_t nd = 2 * hist + (size_t)N * cycles + (size_t)N * contour::kHalf * 2 + 4 * (size_t)N;
  const size_t bytes = nd * sizeof(double) + 2 * (size_t)N * sizeof(uint32_t);
  void *blob = nullptr;
  double *Y = nullptr;
  cudaError_t e = dev_alloc(&blob, bytes);
  if (e == cudaSuccess) e = dev_alloc_n(&Y, h->ws.vec_stride);
  if (e == cudaSuccess) e = cudaMemsetAsync(blob, 0, bytes, s);
  if (e != cudaSuccess) {
    dev_free(blob);
    dev_free(Y);
    return cuda_error(e, "cb_ensemble_scores_restarted: state");
  }
  RState rs;
  double *d = reinterpret_cast<double *>(blob);
  rs.hal = d; d += hist;
  rs.hbe = d; d += hist;
  rs.couple = d; d += (size_t)N * cycles;
  rs.p = d; d += (size_t)N * contour::kHalf * 2;
  rs.theta = d; d += N;
  rs.rho = d; d += N;
  rs.rscale = d; d += N;
  rs.blast = d; d += N;
  rs.steps = reinterpret_cast<uint32_t *>(d);
  rs.status = reinterpret_cast<int32_t *>(rs.steps + N);
  rs.cmax = cycles;
  rs.m = m;
  rc = prec == CB_FP64 ? cycles_run<double>(h, rs, Y, m, cycles, prec, s)
                       : cycles_run<float>(h, rs, Y, m, cycles, prec, s);
  if (rc == CB_OK) {
    restart_finish_kernel<<<(N + 255) / 256, 256, 0, s>>>(h->ws.sc, rs, N);
    rc = cuda_error(cudaGetLastError(), "restart finish launch");
  }
  if (rc == CB_OK) rc = combine_sum_f64(h, Y, n_out, S, log_scale, s);
  if (rc == CB_OK) rc = cuda_error(cudaStreamSynchronize(s), "cb_ensemble_scores_restarted");
  if (rc == CB_OK && rep) {
    std::vector<uint32_t> steps(N);
    std::vector<int32_t> st(N);
    std::vector<double> th(N), bl(N);
    e = cudaMemcpy(steps.data(), rs.steps, N * 4ull, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(st.data(), rs.status, N * 4ull, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(th.data(), rs.theta, N * 8ull, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(bl.data(), rs.blast, N * 8ull, cudaMemcpyDeviceToHost);
    rc = cuda_error(e, "cb_ensemble_scores_restarted: report");
    for (uint32_t r = 0; r < N && rc == CB_OK; ++r) {
      rep[r].m_eff = steps[r];
      rep[r].status = st[r];
      rep[r].theta = th[r];
      rep[r].beta_last = bl[r];
      rep[r].beta0 = std::sqrt((double)h->inst[r].n);
    }
    for (uint32_t r = 0; r < N && rc == CB_OK; ++r)
      if (st[r] != CB_OK) rc = status_error(st[r]);
  }
  dev_free(blob);
  dev_free(Y);
  return rc;
}
