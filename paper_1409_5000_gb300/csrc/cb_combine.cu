// Combine step: scores from the Krylov basis, and the ensemble sum (eq. 5).
//
//   y_r(i) = beta0 (V_m c)_i = sum_j gamma_{r,j} W_{r,j}(i)        (eq. 4)
//   S(i)   = sum_r [i < n_r] exp(theta_r - theta*) y_r(i)           (eq. 5)
//   theta* = max_r theta_r
//
// The sum over j runs in the basis precision (FP32 in CB_FP32 mode, FP64 in
// CB_FP64 mode); the sum over realisations r always runs in FP64 and in
// realisation order, so it is deterministic.  Reads of W are coalesced
// (consecutive nodes are consecutive addresses in every basis vector).
#include "cb_internal.cuh"

namespace cb {

template <typename T>
__global__ void __launch_bounds__(256) combine_single_kernel(const T *V, uint64_t vs, Scalars sc,
                                                             const InstDesc *inst, uint32_t r,
                                                             double *y, double *log_scale) {
  const InstDesc I = inst[r];
  const uint32_t ms = sc.ms;
  const uint32_t M = sc.meff[r];
  const bool ok = sc.status[r] == CB_OK;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *log_scale = ok ? sc.theta[r] : __longlong_as_double(0x7ff8000000000000ll);
  if (i >= I.n) return;
  T acc = T(0);
  const T *w = V + I.node_base + i;
  for (uint32_t j = 0; j < M; ++j) acc += (T)sc.gamma[r * ms + j] * w[(uint64_t)j * vs];
  y[i] = ok ? (double)acc : __longlong_as_double(0x7ff8000000000000ll);
}

template <typename T>
__global__ void __launch_bounds__(256) combine_ensemble_kernel(const T *V, uint64_t vs,
                                                               Scalars sc, const InstDesc *inst,
                                                               uint32_t n_inst, uint32_t n_out,
                                                               double *S, double *log_scale) {
  // per-realisation tables staged in shared memory
  extern __shared__ unsigned char s_raw[];
  double *s_wt = reinterpret_cast<double *>(s_raw);             // exp(theta_r - theta*)
  uint64_t *s_base = reinterpret_cast<uint64_t *>(s_wt + n_inst); // node_base
  uint32_t *s_n = reinterpret_cast<uint32_t *>(s_base + n_inst);  // n_r
  uint32_t *s_m = s_n + n_inst;                                   // m_eff
  __shared__ double s_max[8];
  __shared__ int s_badw[8];
  double t = -1e308;
  int bad = 0;
  for (uint32_t r = threadIdx.x; r < n_inst; r += blockDim.x) {
    t = fmax(t, sc.theta[r]);
    bad |= (sc.status[r] != CB_OK);
    s_base[r] = inst[r].node_base;
    s_n[r] = inst[r].n;
    s_m[r] = sc.meff[r];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) { s_max[threadIdx.x >> 5] = t; s_badw[threadIdx.x >> 5] = bad; }
  __syncthreads();
  double tmax = s_max[0];
  int any_bad = s_badw[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { tmax = fmax(tmax, s_max[w]); any_bad |= s_badw[w]; }
  for (uint32_t r = threadIdx.x; r < n_inst; r += blockDim.x) s_wt[r] = exp(sc.theta[r] - tmax);
  __syncthreads();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  if (i == 0) *log_scale = any_bad ? qnan : tmax;
  if (i >= n_out) return;
  const uint32_t ms = sc.ms;
  double sum = 0.0;
  for (uint32_t r = 0; r < n_inst; ++r) {
    if (i >= s_n[r]) continue;
    const uint32_t M = s_m[r];
    const T *w = V + s_base[r] + i;
    const double *g = sc.gamma + (uint64_t)r * ms;
    T acc = T(0);
    for (uint32_t j = 0; j < M; ++j) acc += (T)__ldg(g + j) * w[(uint64_t)j * vs];
    sum += s_wt[r] * (double)acc;
  }
  S[i] = any_bad ? qnan : sum;
}

int combine_single(cb_graph *h, uint32_t r, int prec, double *y, double *log_scale,
                   cudaStream_t s) {
  const uint32_t n = h->inst[r].n;
  const uint32_t grid = (n + 255) / 256;
  const int tok = prof_begin(CB_K_COMBINE, s);
  if (prec == CB_FP64)
    combine_single_kernel<double><<<grid, 256, 0, s>>>((const double *)h->ws.V, h->ws.vec_stride,
                                                       h->ws.sc, h->d_inst, r, y, log_scale);
  else
    combine_single_kernel<float><<<grid, 256, 0, s>>>((const float *)h->ws.V, h->ws.vec_stride,
                                                      h->ws.sc, h->d_inst, r, y, log_scale);
  prof_end(tok, s);
  return cuda_error(cudaGetLastError(), "combine launch");
}

int combine_ensemble(cb_graph *h, int prec, uint32_t n_out, double *S, double *log_scale,
                     cudaStream_t s) {
  const uint32_t grid = (n_out + 255) / 256;
  const size_t shm = (sizeof(double) + sizeof(uint64_t) + 2 * sizeof(uint32_t)) * h->n_inst;
  if (shm > 200 * 1024) return set_error(CB_ERR_ARG, "too many realisations for one combine");
  const int tok = prof_begin(CB_K_COMBINE, s);
  if (prec == CB_FP64) {
    auto k = combine_ensemble_kernel<double>;
    if (shm > 48 * 1024)
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    k<<<grid, 256, shm, s>>>((const double *)h->ws.V, h->ws.vec_stride, h->ws.sc, h->d_inst,
                             h->n_inst, n_out, S, log_scale);
  } else {
    auto k = combine_ensemble_kernel<float>;
    if (shm > 48 * 1024)
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    k<<<grid, 256, shm, s>>>((const float *)h->ws.V, h->ws.vec_stride, h->ws.sc, h->d_inst,
                             h->n_inst, n_out, S, log_scale);
  }
  prof_end(tok, s);
  return cuda_error(cudaGetLastError(), "combine launch");
}

}  // namespace cb
