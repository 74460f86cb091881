// Adjoint: edge gradient of the summed top-k total communicability.
//
// The paper has no gradient; this differentiates its score.  With w the
// indicator of a fixed node set S (the recovered top-k of eq. 5), the loss is
//     L = sum_r sum_{i in S, i < n_r} (e^{A_r} 1)_i = sum_r w_r^T e^{A_r} 1,
// and for the undirected weight a_ij = a_ji of an existing edge of A_r
//     dL/da_ij = G_ij + G_ji,   G = int_0^1 e^{sA} w 1^T e^{(1-s)A} ds
// (the Frechet derivative of e^A, contracted with w and 1).
//
// Krylov form.  With Lanczos bases V_w (from w) and V_1 (from 1) and their
// tridiagonals T_w, T_1, e^{sA} w ~ ||w|| V_w e^{s T_w} e1 and
// e^{(1-s)A} 1 ~ sqrt(n) V_1 e^{(1-s) T_1} e1, so G ~ V_w M V_1^T with
//     M = ||w|| sqrt(n) int_0^1 (e^{s T_w} e1)(e^{(1-s) T_1} e1)^T ds.
// M is the upper-right block of exp([[T_w, e1 e1^T], [0, T_1]]) (Van Loan's
// block formula).  The resolvent of that block-triangular matrix has
// upper-right block R_w(z) e1 e1^T R_1(z), so the contour rule of the
// forward step (cb_contour.cuh) gives, with the shift theta,
//     M = ||w|| sqrt(n) 2 Re sum_k w_k x_k y_k^T,
//     x_k = (z_k I - (T_w - theta))^{-1} e1,  y_k = (z_k I - (T_1 - theta))^{-1} e1:
// 24 complex tridiagonal solves and 12 rank-1 terms, no eigendecomposition.
//
// Then P = V_w M and U = V_1 are written node-major (m contiguous values per
// node) and every CSR entry (i, j) gets g = P_i . U_j + P_j . U_i, computed
// in the basis precision (FP32 or FP64).  Realisations share one shift theta* =
// max_r theta_r; dL/da_e = exp(theta*) * grad[e].
#include <algorithm>
#include <cstdlib>

#include "cb_contour.cuh"
#include "cb_reduce.cuh"

namespace cb {

CB_DEBUG_STATE()

constexpr uint32_t kMaxAdjM = 64;  // adjoint depth limit (shared-memory staging)

void free_backwork(BackWork &B) {
  dev_free(B.P);
  dev_free(B.U);
  dev_free(B.blob);
  B = BackWork{};
}

static int ensure_backwork(cb_graph *h, uint32_t m, int prec, cudaStream_t s) {
  BackWork &B = h->bw;
  if (B.P && B.prec == prec && B.m == m) return CB_OK;
  free_backwork(B);
  const uint32_t mpad = (m + 3) / 4 * 4;
  const size_t esz = prec == CB_FP64 ? sizeof(double) : sizeof(float);
  const size_t vb = h->total_nodes_padded * mpad * esz + 16;
  cudaError_t e = dev_alloc(&B.P, vb);
  if (e == cudaSuccess) e = dev_alloc(&B.U, vb);
  const uint32_t N = h->n_inst;
  const size_t bytes = ((size_t)N * m * m + N) * sizeof(double) + (size_t)N * sizeof(uint32_t) + 64;
  if (e == cudaSuccess) e = dev_alloc(&B.blob, bytes);
  if (e != cudaSuccess) {
    free_backwork(B);
    return cuda_error(e, "adjoint workspace");
  }
  B.K = reinterpret_cast<double *>(B.blob);
  B.theta = B.K + (size_t)N * m * m;
  B.cnt = reinterpret_cast<uint32_t *>(B.theta + N);
  B.prec = prec;
  B.m = m;
  B.mpad = mpad;
  return cuda_error(cudaMemsetAsync(B.blob, 0, bytes, s), "adjoint workspace clear");
}

// One warp per realisation: theta_r and the coefficient matrix K_r = M_r.
__global__ void __launch_bounds__(32) bw_tridiag_kernel(Scalars s1, Scalars sw,
                                                        const InstDesc *inst, double *K,
                                                        uint32_t kdim, double *theta_out,
                                                        uint32_t *cnt_out) {
  using namespace contour;
  __shared__ double s_a1[kMaxAdjM], s_b1[kMaxAdjM], s_aw[kMaxAdjM], s_bw[kMaxAdjM];
  __shared__ cplx s_x[kHalf][kMaxAdjM], s_y[kHalf][kMaxAdjM];
  __shared__ double s_th[2];
  const uint32_t r = blockIdx.x, lane = threadIdx.x;
  const int M1 = (int)s1.meff[r], Mw = (int)sw.meff[r];
  const bool ok = M1 > 0 && Mw > 0 && s1.status[r] == CB_OK && sw.status[r] == CB_OK;
  if (!ok) {
    if (lane == 0) {
      theta_out[r] = -1e308;
      cnt_out[r] = 0;
    }
    return;
  }
  for (int i = lane; i < M1; i += 32) {
    s_a1[i] = s1.alpha[r * s1.ms + i];
    s_b1[i] = s1.beta[r * s1.ms + i];
  }
  for (int i = lane; i < Mw; i += 32) {
    s_aw[i] = sw.alpha[r * sw.ms + i];
    s_bw[i] = sw.beta[r * sw.ms + i];
  }
  __syncwarp();
  if (lane == 0) s_th[0] = lambda_max(s_a1, s_b1, M1);
  if (lane == 1) s_th[1] = lambda_max(s_aw, s_bw, Mw);
  __syncwarp();
  const double theta = fmax(s_th[0], s_th[1]);
  if (lane < kHalf) {
    cplx z, w;
    node((int)lane, &z, &w);
    cplx cp[kMaxAdjM], x[kMaxAdjM];
    thomas_e1(s_aw, s_bw, Mw, theta, z, cp, x);
    for (int i = 0; i < Mw; ++i) s_x[lane][i] = cmul(w, x[i]);
    thomas_e1(s_a1, s_b1, M1, theta, z, cp, x);
    for (int i = 0; i < M1; ++i) s_y[lane][i] = x[i];
  }
  __syncwarp();
  // ||w|| = 1 / scale_w[0], sqrt(n) = 1 / scale_1[0]
  const double c = 1.0 / (sw.scale[r * sw.ms] * s1.scale[r * s1.ms]);
  double *Kr = K + (size_t)r * kdim * kdim;
  for (int q = lane; q < Mw * M1; q += 32) {
    const int a = q / M1, b = q % M1;
    double acc = 0.0;
    for (int k = 0; k < kHalf; ++k) {
      const cplx xa = s_x[k][a], yb = s_y[k][b];
      acc += xa.re * yb.re - xa.im * yb.im;
    }
    Kr[a * kdim + b] = 2.0 * c * acc;
  }
  if (lane == 0) {
    theta_out[r] = theta;
    const double sw0 = sw.scale[r * sw.ms];
    cnt_out[r] = (uint32_t)llrint(1.0 / (sw0 * sw0));
  }
}

// Node-major P = exp(theta_r - theta*) V_w K_r and U = V_1 (scales applied).
// One CTA per finalize tile (kFinRows nodes of one realisation), 4 warps;
// each warp stages 32 nodes' basis values in shared memory and writes the
// node-major rows with lanes over the row index (coalesced).  All per-node
// arithmetic runs in T: the FP64 scalars are converted once per CTA (FP64
// instructions are scarce on GB300).
template <typename T>
__global__ void __launch_bounds__(128) bw_node_kernel(const T *V1, const T *Vw, uint64_t vs,
                                                      Scalars s1, Scalars sw,
                                                      const InstDesc *inst, const uint32_t *fin_inst,
                                                      uint32_t n_inst, const double *K,
                                                      uint32_t kdim, const double *theta_in,
                                                      uint32_t mpad, T *P, T *U,
                                                      double *log_scale) {
  extern __shared__ unsigned char s_raw[];
  T *sK = reinterpret_cast<T *>(s_raw);              // kdim * kdim
  T *sV = sK + kdim * kdim;                          // 4 warps x kdim x 32 (V_w values)
  T *sW = sV + 4 * kdim * 32;                        // 4 warps x kdim x 32 (V_1 values)
  __shared__ T s_sc1[kMaxAdjM], s_scw[kMaxAdjM];
  __shared__ double s_wmax[4];
  const uint32_t t = blockIdx.x;
  const uint32_t r = fin_inst[t];
  const InstDesc I = inst[r];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double tm = -1e308;
  for (uint32_t q = threadIdx.x; q < n_inst; q += blockDim.x) tm = fmax(tm, theta_in[q]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tm = fmax(tm, __shfl_xor_sync(0xffffffffu, tm, o));
  if (lane == 0) s_wmax[warp] = tm;
  const double th = theta_in[r];
  const bool active = th > -1e307;
  const int M1 = active ? (int)s1.meff[r] : 0, Mw = active ? (int)sw.meff[r] : 0;
  for (int q = threadIdx.x; q < M1; q += blockDim.x) s_sc1[q] = (T)s1.scale[r * s1.ms + q];
  for (int q = threadIdx.x; q < Mw; q += blockDim.x) s_scw[q] = (T)sw.scale[r * sw.ms + q];
  __syncthreads();
  const double tmax = fmax(fmax(s_wmax[0], s_wmax[1]), fmax(s_wmax[2], s_wmax[3]));
  if (t == 0 && threadIdx.x == 0) *log_scale = tmax > -1e307 ? tmax : 0.0;
  const double f = active ? exp(th - tmax) : 0.0;
  for (uint32_t q = threadIdx.x; q < (uint32_t)(Mw * M1); q += blockDim.x) {
    const uint32_t a = q / M1, b = q % M1;
    sK[a * kdim + b] = (T)(f * K[(size_t)r * kdim * kdim + a * kdim + b]);
  }
  __syncthreads();
  T *myV = sV + warp * kdim * 32, *myW = sW + warp * kdim * 32;
  const uint32_t i0 = (t - I.fin_base) * kFinRows, i1 = min(i0 + kFinRows, I.n);
  for (uint32_t base = i0 + warp * 32; base < i1; base += 4 * 32) {
    const uint32_t i = base + lane;
    const bool valid = i < i1;
    for (int a = 0; a < Mw; ++a)
      myV[a * 32 + lane] = valid ? s_scw[a] * Vw[(uint64_t)a * vs + I.node_base + i] : T(0);
    for (int b = 0; b < M1; ++b)
      myW[b * 32 + lane] = valid ? s_sc1[b] * V1[(uint64_t)b * vs + I.node_base + i] : T(0);
    __syncwarp();
    const uint32_t nn = min(32u, i1 - base);
    for (uint32_t q = 0; q < nn; ++q) {
      const uint64_t row = (I.node_base + base + q) * (uint64_t)mpad;
      for (uint32_t b = lane; b < mpad; b += 32) {
        T p = T(0), u = T(0);
        if ((int)b < M1) {
          for (int a = 0; a < Mw; ++a) p += myV[a * 32 + q] * sK[a * kdim + b];
          u = myW[b * 32 + q];
        }
        P[row + b] = p;
        U[row + b] = u;
      }
    }
    __syncwarp();
  }
}

// dot of 4 consecutive values of a with 4 of b (16- or 32-byte aligned)
__device__ __forceinline__ float dot4(const float *a, const float *b) {
  const float4 x = *reinterpret_cast<const float4 *>(a), y = *reinterpret_cast<const float4 *>(b);
  return x.x * y.x + x.y * y.y + x.z * y.z + x.w * y.w;
}
__device__ __forceinline__ double dot4(const double *a, const double *b) {
  const double2 x0 = *reinterpret_cast<const double2 *>(a);
  const double2 x1 = *reinterpret_cast<const double2 *>(a + 2);
  const double2 y0 = *reinterpret_cast<const double2 *>(b);
  const double2 y1 = *reinterpret_cast<const double2 *>(b + 2);
  return x0.x * y0.x + x0.y * y0.y + x1.x * y1.x + x1.y * y1.y;
}

// mirror[e] for every CSR entry e = (i, j) of one SpMV tile: the position of
// (j, i) in row j (rows are sorted; binary search).  An entry without a
// mirror (asymmetric input) points at itself.
__global__ void __launch_bounds__(256) bw_mirror_kernel(const InstDesc *inst,
                                                        const uint32_t *tile_inst,
                                                        const uint2 *tile_rows,
                                                        const uint32_t *row_ptr, const uint32_t *col,
                                                        uint32_t *mirror) {
  __shared__ uint32_t s_rp[kTileRows + 1];
  const uint32_t t = blockIdx.x;
  const InstDesc I = inst[tile_inst[t]];
  const uint32_t *rp = row_ptr + I.rp_base;
  const uint32_t *cl = col + I.edge_base;
  const uint2 tr = tile_rows[t];
  const uint32_t row0 = tr.x, nrows = tr.y - tr.x;
  for (uint32_t q = threadIdx.x; q <= nrows; q += blockDim.x) s_rp[q] = rp[row0 + q];
  __syncthreads();
  for (uint32_t e = s_rp[0] + threadIdx.x; e < s_rp[nrows]; e += blockDim.x) {
    uint32_t lo = 0, hi = nrows;  // last lr with s_rp[lr] <= e
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_rp[mid] <= e) lo = mid; else hi = mid;
    }
    const uint32_t i = row0 + lo, j = __ldg(cl + e);
    if (!CB_DCHECK(j < I.n, kDbgAdjointCol, j)) {
      mirror[I.edge_base + e] = e;
      continue;
    }
    uint32_t a = rp[j], b = rp[j + 1];  // first position in row j with col >= i
    while (a < b) {
      const uint32_t mid = (a + b) >> 1;
      if (__ldg(cl + mid) < i) a = mid + 1; else b = mid;
    }
    mirror[I.edge_base + e] = (a < rp[j + 1] && __ldg(cl + a) == i) ? a : e;
  }
}

// The gradient is symmetric: g(i, j) = P_i . U_j + P_j . U_i = g(j, i).  Each
// undirected edge is computed once, from its upper entry (j >= i, a suffix
// of the sorted row i), and written to both CSR entries (the lower one
// through mirror).  A group of kEdgeLanes lanes shares an edge: lane c takes
// the 4-value chunks c, c + kEdgeLanes, ... of the four node-major rows, so
// each row is read as whole 128-byte lines; the partials are summed across
// the group with a shuffle tree.  Arithmetic in T (FP32 in CB_FP32 mode):
// FP64 instructions are scarce on GB300 and would bound this kernel.
constexpr uint32_t kEdgeLanes = 8;
template <typename T>
__global__ void __launch_bounds__(256) bw_edge_kernel(const T *P, const T *U, uint32_t mpad,
                                                      const InstDesc *inst,
                                                      const uint32_t *tile_inst,
                                                      const uint2 *tile_rows,
                                                      const uint32_t *row_ptr, const uint32_t *col,
                                                      const uint32_t *mirror,
                                                      const double *theta_in, float *grad) {
  __shared__ uint32_t s_rp[kTileRows + 1];
  __shared__ uint32_t s_first[kTileRows];   // first upper entry of each row
  __shared__ uint32_t s_up[kTileRows + 1];  // prefix of upper-entry counts
  const uint32_t t = blockIdx.x;
  const uint32_t r = tile_inst[t];
  const InstDesc I = inst[r];
  const uint32_t *rp = row_ptr + I.rp_base;
  const uint32_t *cl = col + I.edge_base;
  const uint2 tr = tile_rows[t];
  const uint32_t row0 = tr.x;
  const uint32_t nrows = tr.y - tr.x;
  for (uint32_t q = threadIdx.x; q <= nrows; q += blockDim.x) s_rp[q] = rp[row0 + q];
  __syncthreads();
  for (uint32_t lr = threadIdx.x; lr < nrows; lr += blockDim.x) {
    uint32_t a = s_rp[lr], b = s_rp[lr + 1];
    const uint32_t row = row0 + lr;
    while (a < b) {
      const uint32_t mid = (a + b) >> 1;
      if (__ldg(cl + mid) < row) a = mid + 1; else b = mid;
    }
    s_first[lr] = a;
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // warp 0: prefix over up to 32 x 8 rows
    constexpr uint32_t kPer = kTileRows / 32;
    const uint32_t lane = threadIdx.x, base = lane * kPer;
    uint32_t c[kPer], sum = 0;
#pragma unroll
    for (uint32_t q = 0; q < kPer; ++q) {
      const uint32_t lr = base + q;
      c[q] = lr < nrows ? s_rp[lr + 1] - s_first[lr] : 0u;
      sum += c[q];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)lane >= o) incl += y;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (uint32_t q = 0; q < kPer; ++q) {
      if (base + q <= nrows) s_up[base + q] = run;
      run += c[q];
    }
    if (lane == 31 && nrows == kTileRows) s_up[kTileRows] = run;
  }
  __syncthreads();
  const uint32_t nup = s_up[nrows];
  const bool active = theta_in[r] > -1e307;
  const uint32_t nv = mpad / 4;
  const uint32_t c0 = threadIdx.x % kEdgeLanes;
  constexpr uint32_t kGroups = 256 / kEdgeLanes;
  // the loop bound is uniform across each group, so the shuffles see all lanes
  for (uint32_t ub = 0; ub < nup; ub += kGroups) {
    const uint32_t u = ub + threadIdx.x / kEdgeLanes;
    T g = T(0);
    uint32_t e = 0;
    if (u < nup) {
      uint32_t lo = 0, hi = nrows;  // s_up[lo] <= u < s_up[hi]
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_up[mid] <= u) lo = mid; else hi = mid;
      }
      e = s_first[lo] + (u - s_up[lo]);
      if (active && CB_DCHECK(__ldg(cl + e) < I.n, kDbgAdjointCol, __ldg(cl + e))) {
        const uint64_t i = I.node_base + row0 + lo;
        const uint64_t j = I.node_base + __ldg(cl + e);
        const T *Pi = P + i * mpad, *Ui = U + i * mpad, *Pj = P + j * mpad, *Uj = U + j * mpad;
        for (uint32_t c = c0; c < nv; c += kEdgeLanes)
          g += dot4(Pi + 4 * c, Uj + 4 * c) + dot4(Pj + 4 * c, Ui + 4 * c);
      }
    }
    for (uint32_t off = kEdgeLanes / 2; off > 0; off >>= 1)
      g += __shfl_xor_sync(0xffffffffu, g, off, kEdgeLanes);
    if (c0 == 0 && u < nup) {
      grad[I.edge_base + e] = (float)g;
      grad[I.edge_base + mirror[I.edge_base + e]] = (float)g;
    }
  }
}

template <typename T>
static int backward_t(cb_graph *h, uint32_t m, const uint32_t *idx, uint32_t k, float *grad,
                      double *log_scale, cudaStream_t s) {
  BackWork &B = h->bw;
  const uint32_t N = h->n_inst;
  prefer_shared(bw_tridiag_kernel);
  prefer_shared(bw_node_kernel<T>);
  prefer_shared(bw_edge_kernel<T>);
  const int tok = prof_begin(CB_K_BACKWARD, s);
  bw_tridiag_kernel<<<N, 32, 0, s>>>(h->ws.sc, h->ws2.sc, h->d_inst, B.K, m, B.theta, B.cnt);
  const size_t shm = (size_t)(m * m + 8 * m * 32) * sizeof(T);
  auto nk = bw_node_kernel<T>;
  if (shm > 48 * 1024) cudaFuncSetAttribute(nk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  nk<<<h->total_fin, 128, shm, s>>>((const T *)h->ws.V, (const T *)h->ws2.V, h->ws.vec_stride,
                                    h->ws.sc, h->ws2.sc, h->d_inst, h->d_fin_inst, N, B.K, m,
                                    B.theta, B.mpad, (T *)B.P, (T *)B.U, log_scale);
  bw_edge_kernel<T><<<h->total_tiles, 256, 0, s>>>((const T *)B.P, (const T *)B.U, B.mpad,
                                                   h->d_inst, h->d_tile_inst, h->d_tile_rows,
                                                   h->row_ptr, h->col, h->d_mirror,
                                                   B.theta, grad);
  prof_end(tok, s);
  (void)idx;
  (void)k;
  return cuda_error(cudaGetLastError(), "adjoint launch");
}

CB_DEBUG_READER(adjoint)

}  // namespace cb

using namespace cb;

CB_API int cb_scores_backward(cb_graph *h, uint32_t m, int prec, const uint32_t *topk_idx,
                              uint32_t k, float *grad, double *log_scale, void *stream) {
  NvtxRange nvtx_range("cb_scores_backward");
  if (!h || !topk_idx || !grad || !log_scale)
    return set_error(CB_ERR_ARG, "cb_scores_backward: null argument");
  if (m < 1 || m > kMaxAdjM)
    return set_error(CB_ERR_ARG, "cb_scores_backward: need 1 <= m <= 64");
  if (k < 1 || k > CB_MAX_TOPK)
    return set_error(CB_ERR_ARG, "cb_scores_backward: need 1 <= k <= CB_MAX_TOPK");
  const bool reorth = split_prec(prec);
  if (prec != CB_FP32 && prec != CB_FP64)
    return set_error(CB_ERR_ARG, "cb_scores_backward: bad precision");
  h->reorth = reorth;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = ensure_workspace(h, h->ws, m, prec, s);
  if (rc == CB_OK) rc = ensure_workspace(h, h->ws2, m, prec, s);
  if (rc == CB_OK) rc = ensure_backwork(h, m, prec, s);
  if (rc == CB_OK && !h->d_mirror) {  // once per handle: the position of each entry's mirror
    cudaError_t e = dev_alloc_n(&h->d_mirror, std::max<uint64_t>(h->total_nnz, 1));
    if (e == cudaSuccess && h->total_tiles) {
      bw_mirror_kernel<<<h->total_tiles, 256, 0, s>>>(h->d_inst, h->d_tile_inst, h->d_tile_rows,
                                                      h->row_ptr, h->col, h->d_mirror);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      dev_free(h->d_mirror);
      h->d_mirror = nullptr;
      rc = cuda_error(e, "adjoint: mirror index");
    }
  }
  // the basis from 1 is the forward pass's when an ensemble pass at this m
  // and precision ran last on the handle (same stream order assumed)
  const bool reuse = rc == CB_OK && h->basis_m == m && h->basis_prec == prec &&
                     h->basis_reorth == reorth && h->basis_gen == h->ws.gen;
  if (rc == CB_OK && !reuse) {
    h->basis_m = 0;
    rc = lanczos_run(h, h->ws, 0, h->n_inst, m, prec, s);
    if (rc == CB_OK) {
      h->basis_m = m;
      h->basis_prec = prec;
      h->basis_reorth = reorth;
      h->basis_gen = h->ws.gen;
    }
  }
  if (rc == CB_OK) rc = lanczos_run(h, h->ws2, 0, h->n_inst, m, prec, s, topk_idx, k);
  if (rc == CB_OK)
    rc = prec == CB_FP64 ? backward_t<double>(h, m, topk_idx, k, grad, log_scale, s)
                         : backward_t<float>(h, m, topk_idx, k, grad, log_scale, s);
  return rc;
}

namespace cb {
namespace {

// loss = sum over q of S[nodes[q]] for the nodes inside [0, n), FP64: lane l
// sums q = l, l + 32, ... in order, then a fixed shuffle tree (deterministic).
__global__ void __launch_bounds__(32) score_sum_kernel(const double *S, uint32_t n,
                                                       const uint32_t *nodes, uint32_t k,
                                                       double *out) {
  double acc = 0.0;
  for (uint32_t q = threadIdx.x; q < k; q += 32) {
    const uint32_t i = nodes[q];
    if (i < n) acc += S[i];
  }
  acc = warp_sum_d(acc);
  if (threadIdx.x == 0) *out = acc;
}

// grad *= exp(ls_grad - ls_ref) * (grad_out ? *grad_out : 1), the factor
// formed once in FP64 and applied in FP32.
__global__ void __launch_bounds__(256) grad_rescale_kernel(float *g, uint64_t n,
                                                           const double *ls_grad,
                                                           const double *ls_ref,
                                                           const double *grad_out) {
  const double f64 = exp(*ls_grad - *ls_ref) * (grad_out ? *grad_out : 1.0);
  const float f = (float)f64;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    g[i] *= f;
}

__global__ void scale_grad_kernel(float *g, uint64_t n, const double *ls_group,
                                  const double *ls_all) {
  const float f = (float)exp(*ls_group - *ls_all);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    g[i] *= f;
}

__global__ void max_shift_kernel(const double *ls, uint32_t n, double *out) {
  if (threadIdx.x == 0) {
    double t = ls[0];
    for (uint32_t q = 1; q < n; ++q) t = fmax(t, ls[q]);
    *out = t;
  }
}

}  // namespace
}  // namespace cb

// Working set of the adjoint for realisation r: two (m + 1)-vector bases and
// the node-major P and U, plus the copy of its graph and format in a group
// handle (about 12 bytes per CSR entry).
static uint64_t adjoint_bytes(const cb::InstDesc &I, uint64_t nnz, uint32_t m, int prec) {
  const uint64_t esz = prec == CB_FP64 ? 8 : 4;
  const uint64_t npad = (I.n + cb::kNodeAlign - 1) / cb::kNodeAlign * cb::kNodeAlign;
  const uint64_t mpad = (m + 3) / 4 * 4;
  return esz * npad * (2 * (uint64_t)(m + 1) + 2 * mpad) + 12 * nnz + 8ull * I.n;
}

CB_API int cb_scores_backward_budget(cb_graph *h, uint32_t m, int prec, const uint32_t *topk_idx,
                                     uint32_t k, float *grad, double *log_scale,
                                     size_t mem_budget, void *stream) {
  NvtxRange nvtx_range("cb_scores_backward_budget");
  if (!h || !topk_idx || !grad || !log_scale)
    return set_error(CB_ERR_ARG, "cb_scores_backward_budget: null argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const uint32_t N = h->n_inst;
  std::vector<uint64_t> nnz(N), need(N);
  uint64_t total = 0;
  for (uint32_t r = 0; r < N; ++r) {
    nnz[r] = (r + 1 < N ? h->inst[r + 1].edge_base : h->total_nnz) - h->inst[r].edge_base;
    need[r] = adjoint_bytes(h->inst[r], nnz[r], m, prec & ~CB_REORTH);
    total += need[r];
  }
  if (total <= mem_budget || N == 1)
    return cb_scores_backward(h, m, prec, topk_idx, k, grad, log_scale, stream);
  // groups of consecutive realisations whose working set fits (at least one each)
  std::vector<uint32_t> starts;
  uint64_t acc = 0;
  for (uint32_t r = 0; r < N; ++r) {
    if (starts.empty() || acc + need[r] > mem_budget) {
      starts.push_back(r);
      acc = 0;
    }
    acc += need[r];
  }
  starts.push_back(N);
  const uint32_t G = (uint32_t)starts.size() - 1;
  double *d_ls = nullptr;  // per-group shift, then the common one
  cudaError_t e = dev_alloc_n(&d_ls, G + 1);
  if (e != cudaSuccess) return cuda_error(e, "cb_scores_backward_budget: allocate");
  int rc = CB_OK;
  for (uint32_t g = 0; g < G && rc == CB_OK; ++g) {
    const uint32_t r0 = starts[g], r1 = starts[g + 1];
    std::vector<uint32_t> vn(r1 - r0);
    std::vector<const uint32_t *> vrp(r1 - r0), vcol(r1 - r0);
    for (uint32_t r = r0; r < r1; ++r) {
      vn[r - r0] = h->inst[r].n;
      vrp[r - r0] = h->row_ptr + h->inst[r].rp_base;
      vcol[r - r0] = h->col + h->inst[r].edge_base;
    }
    cb_graph *v = nullptr;
    rc = cb_graph_upload(r1 - r0, vn.data(), nnz.data() + r0, vrp.data(), vcol.data(),
                         CB_DEVICE_PTRS, stream, &v);
    if (rc != CB_OK) break;
    rc = cb_scores_backward(v, m, prec, topk_idx, k, grad + h->inst[r0].edge_base, d_ls + g, stream);
    if (rc == CB_OK) rc = cuda_error(cudaStreamSynchronize(s), "cb_scores_backward_budget");
    const int rf = cb_graph_free(v);
    if (rc == CB_OK) rc = rf;
  }
  if (rc == CB_OK) {
    max_shift_kernel<<<1, 32, 0, s>>>(d_ls, G, d_ls + G);
    for (uint32_t g = 0; g < G; ++g) {
      const uint64_t e0 = h->inst[starts[g]].edge_base;
      const uint64_t e1 = starts[g + 1] < N ? h->inst[starts[g + 1]].edge_base : h->total_nnz;
      if (e1 > e0)
        scale_grad_kernel<<<(uint32_t)std::min<uint64_t>((e1 - e0 + 255) / 256, 152 * 8), 256, 0, s>>>(
            grad + e0, e1 - e0, d_ls + g, d_ls + G);
    }
    e = cudaMemcpyAsync(log_scale, d_ls + G, 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    rc = cuda_error(e, "cb_scores_backward_budget: combine");
  }
  dev_free(d_ls);
  return rc;
}

CB_API int cb_score_sum(const double *S, uint32_t n, const uint32_t *nodes, uint32_t k,
                        double *loss, void *stream) {
  NvtxRange nvtx_range("cb_score_sum");
  if (!S || !nodes || !loss) return set_error(CB_ERR_ARG, "cb_score_sum: null argument");
  if (k < 1 || k > CB_MAX_TOPK)
    return set_error(CB_ERR_ARG, "cb_score_sum: need 1 <= k <= CB_MAX_TOPK");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  score_sum_kernel<<<1, 32, 0, s>>>(S, n, nodes, k, loss);
  return cuda_error(cudaGetLastError(), "cb_score_sum");
}

CB_API int cb_grad_rescale(float *grad, uint64_t count, const double *log_scale_grad,
                           const double *log_scale_ref, const double *grad_out, void *stream) {
  NvtxRange nvtx_range("cb_grad_rescale");
  if (!grad || !log_scale_grad || !log_scale_ref)
    return set_error(CB_ERR_ARG, "cb_grad_rescale: null argument");
  if (count == 0) return CB_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const uint64_t blocks = std::min<uint64_t>((count + 255) / 256, 152ull * 8);
  grad_rescale_kernel<<<(uint32_t)blocks, 256, 0, s>>>(grad, count, log_scale_grad, log_scale_ref,
                                                       grad_out);
  return cuda_error(cudaGetLastError(), "cb_grad_rescale");
}
