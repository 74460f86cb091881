// Sub-graph centrality SC(i) = (e^A)_ii (eq. 3) of a set of nodes of one
// realisation, by Gauss quadrature.
//
// e_i^T e^A e_i is the integral of exp against the spectral measure of A
// seen from e_i; m Lanczos steps from e_i (beta0 = ||e_i|| = 1) give the
// m-point Gauss rule e1^T exp(T_m) e1 (Golub & Meurant, "Matrices, Moments
// and Quadrature with Applications", 2010).  Every derivative of exp is
// positive, so the rule is a lower bound that increases with m, exact once
// the Krylov space is invariant.  The paper calls SC expensive for large
// graphs ("Identification algorithm"); restricted to candidate nodes it
// costs one Lanczos run per node, all run together here.
//
// The k start nodes become k realisations of a temporary handle that holds
// k copies of the graph (device-to-device copies through cb_graph_upload),
// so every Lanczos kernel runs unchanged with one start node per
// realisation.  Only e1^T exp(T - theta) e1 is needed: no basis combine.
#include "cb_contour.cuh"

namespace cb {
namespace {

// One warp per start node: theta_q = lambda_max(T), c0_q = [exp(T - theta) e1]_0
// via the contour rule (theta in sc.theta[q], c0 in sc.gamma[q * ms]).
__global__ void __launch_bounds__(32) sc_tridiag_kernel(Scalars sc) {
  using namespace contour;
  __shared__ double s_al[CB_MAX_M], s_be[CB_MAX_M];
  __shared__ double s_c0[kHalf];
  __shared__ double s_theta;
  const uint32_t q = blockIdx.x, lane = threadIdx.x, ms = sc.ms;
  const int M = (int)sc.meff[q];
  if (sc.status[q] != CB_OK || M < 1) {
    if (lane == 0) {
      sc.theta[q] = 0.0;
      sc.gamma[q * ms] = M < 1 && sc.status[q] == CB_OK ? 0.0 : __longlong_as_double(0x7ff8000000000000ll);
    }
    return;
  }
  for (int i = lane; i < M; i += 32) {
    s_al[i] = sc.alpha[q * ms + i];
    s_be[i] = sc.beta[q * ms + i];
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
    s_c0[lane] = 2.0 * (w.re * x[0].re - w.im * x[0].im);
  }
  __syncwarp();
  if (lane == 0) {
    double c0 = 0.0;
    for (int t = 0; t < kHalf; ++t) c0 += s_c0[t];
    sc.theta[q] = theta;
    sc.gamma[q * ms] = c0;
  }
}

// Common shift theta* = max_q theta_q; out[q] = exp(theta_q - theta*) c0_q.
__global__ void __launch_bounds__(256) sc_finish_kernel(Scalars sc, uint32_t k, double *out,
                                                        double *log_scale) {
  __shared__ double s_max[8];
  double tm = -1e308;
  for (uint32_t q = threadIdx.x; q < k; q += blockDim.x)
    if (sc.status[q] == CB_OK) tm = fmax(tm, sc.theta[q]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tm = fmax(tm, __shfl_xor_sync(0xffffffffu, tm, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = tm;
  __syncthreads();
  double tmax = s_max[0];
  for (int w = 1; w < 8; ++w) tmax = fmax(tmax, s_max[w]);
  if (tmax < -1e307) tmax = 0.0;
  for (uint32_t q = threadIdx.x; q < k; q += blockDim.x)
    out[q] = sc.status[q] == CB_OK ? exp(sc.theta[q] - tmax) * sc.gamma[q * sc.ms]
                                   : __longlong_as_double(0x7ff8000000000000ll);
  if (threadIdx.x == 0) *log_scale = tmax;
}

}  // namespace
}  // namespace cb

using namespace cb;

CB_API int cb_subgraph_centrality(cb_graph *h, uint32_t inst, uint32_t m, int prec, uint32_t k,
                                  const uint32_t *nodes, double *sc_scaled, double *log_scale,
                                  void *stream) {
  NvtxRange nvtx_range("cb_subgraph_centrality");
  if (!h || !nodes || !sc_scaled || !log_scale)
    return set_error(CB_ERR_ARG, "cb_subgraph_centrality: null argument");
  if (inst >= h->n_inst) return set_error(CB_ERR_ARG, "cb_subgraph_centrality: realisation out of range");
  if (m < 1 || m > CB_MAX_M) return set_error(CB_ERR_ARG, "cb_subgraph_centrality: need 1 <= m <= CB_MAX_M");
  const bool reorth = split_prec(prec);
  if (prec != CB_FP32 && prec != CB_FP64) return set_error(CB_ERR_ARG, "cb_subgraph_centrality: bad precision");
  if (k < 1 || k > CB_MAX_SC_NODES)
    return set_error(CB_ERR_ARG, "cb_subgraph_centrality: need 1 <= k <= CB_MAX_SC_NODES");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const InstDesc I = h->inst[inst];
  // the node indices are read back once to reject out-of-range entries
  std::vector<uint32_t> hn(k);
  cudaError_t e = cudaMemcpyAsync(hn.data(), nodes, k * 4ull, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_error(e, "cb_subgraph_centrality: read nodes");
  for (uint32_t q = 0; q < k; ++q)
    if (hn[q] >= I.n) return set_error(CB_ERR_ARG, "cb_subgraph_centrality: node index >= n");
  const uint64_t nnz = (inst + 1 < h->n_inst ? h->inst[inst + 1].edge_base : h->total_nnz) - I.edge_base;
  // k copies of realisation inst, one per start node
  std::vector<uint32_t> vn(k, I.n);
  std::vector<uint64_t> vnnz(k, nnz);
  std::vector<const uint32_t *> vrp(k, h->row_ptr + I.rp_base), vcol(k, h->col + I.edge_base);
  cb_graph *v = nullptr;
  int rc = cb_graph_upload(k, vn.data(), vnnz.data(), vrp.data(), vcol.data(), CB_DEVICE_PTRS,
                           stream, &v);
  if (rc != CB_OK) return rc;
  const uint32_t *d_nodes = nodes;
  uint32_t *tmp = nullptr;
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, nodes) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
    cudaGetLastError();  // host pointer: stage the indices on the device
    e = dev_alloc_n(&tmp, k);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, hn.data(), k * 4ull, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      dev_free(tmp);
      cb_graph_free(v);
      return cuda_error(e, "cb_subgraph_centrality: stage nodes");
    }
    d_nodes = tmp;
  }
  v->reorth = reorth;
  rc = ensure_workspace(v, v->ws, m, prec, s);
  if (rc == CB_OK) rc = lanczos_run(v, v->ws, 0, k, m, prec, s, d_nodes, k, true);
  if (rc == CB_OK) {
    sc_tridiag_kernel<<<k, 32, 0, s>>>(v->ws.sc);
    sc_finish_kernel<<<1, 256, 0, s>>>(v->ws.sc, k, sc_scaled, log_scale);
    rc = cuda_error(cudaGetLastError(), "cb_subgraph_centrality: launch");
  }
  if (rc == CB_OK) rc = cuda_error(cudaStreamSynchronize(s), "cb_subgraph_centrality");
  dev_free(tmp);
  const int rf = cb_graph_free(v);
  return rc != CB_OK ? rc : rf;
}
