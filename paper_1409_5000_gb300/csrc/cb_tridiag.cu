// FP64 tridiagonal step of the Krylov approximation: (theta, c) with
// theta = lambda_max(T) and c = exp(T - theta I) e1, one warp per
// realisation.
//
// The Lanczos approximation of e^A 1 (paper, "Identification algorithm")
// projects A onto K_m(A, 1); what remains is the small matrix function
// exp(T_m) e1.  GB300 executes FP64 at a small fraction of its FP32 rate,
// so the solve is organised to use few FP64 operations and to run the
// independent parts in parallel lanes (cb_contour.cuh):
//  1. theta = lambda_max(T) by Laguerre's iteration (lane 0);
//  2. exp(S) e1, S = T - theta I <= 0, as 2 Re sum_k w_k (z_k I - S)^{-1} e1
//     over the 12 upper-half contour nodes, one complex Thomas solve per lane;
//  3. gamma_j = beta0 * c_j * scale_j, the weight of the stored basis vector
//     W_j in the combine step.
#include "cb_contour.cuh"

namespace cb {

__global__ void __launch_bounds__(32) tridiag_kernel(Scalars sc, const InstDesc *inst,
                                                     uint32_t r0) {
  using namespace contour;
  __shared__ double s_al[CB_MAX_M], s_be[CB_MAX_M];
  __shared__ double s_c[kHalf][CB_MAX_M];
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
  if (lane < kHalf) {
    cplx z, w;
    node((int)lane, &z, &w);
    cplx cp[CB_MAX_M], x[CB_MAX_M];
    thomas_e1(s_al, s_be, M, theta, z, cp, x);
    for (int i = 0; i < M; ++i) s_c[lane][i] = 2.0 * (w.re * x[i].re - w.im * x[i].im);
  }
  __syncwarp();
  const double beta0 = sqrt((double)inst[r].n);
  for (int i = lane; i < M; i += 32) {
    double c = 0.0;
    for (int q = 0; q < kHalf; ++q) c += s_c[q][i];
    sc.gamma[r * ms + i] = beta0 * c * sc.scale[r * ms + i];
  }
  if (lane == 0) sc.theta[r] = theta;
}

int tridiag_run(cb_graph *h, uint32_t r0, uint32_t r1, int /*prec*/, cudaStream_t s) {
  NvtxRange nvtx_range("tridiagonal exp");
  prefer_shared(tridiag_kernel);
  const int tok = prof_begin(CB_K_TRIDIAG, s);
  tridiag_kernel<<<r1 - r0, 32, 0, s>>>(h->ws.sc, h->d_inst, r0);
  prof_end(tok, s);
  return cuda_error(cudaGetLastError(), "tridiag launch");
}

}  // namespace cb
