// Combine step: scores from the Krylov basis, and the ensemble sum (eq. 5).
//
// Two phases for the ensemble: every realisation's y_r over all its nodes in
// parallel (combine_y_kernel, bandwidth-bound reads of the basis), then the
// ordered FP64 sum over realisations per node (combine_sum_kernel).
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

__global__ void log_scale_kernel(Scalars sc, uint32_t r, double *log_scale) {
  if (threadIdx.x == 0)
    *log_scale = sc.status[r] == CB_OK ? sc.theta[r] : __longlong_as_double(0x7ff8000000000000ll);
}

// y(i) = sum_j gamma_{r,j} W_j(i) over one finalize tile (kFinRows nodes of
// realisation r), 8 consecutive nodes per thread: the M loads of a thread
// are independent, so they are all in flight together.  OutT is double for
// the single-realisation result and T for the ensemble's per-realisation
// terms (written into basis slot `out_slot`).
template <typename T, typename OutT>
__global__ void __launch_bounds__(256) combine_y_kernel(const T *V, uint64_t vs, Scalars sc,
                                                        const InstDesc *inst,
                                                        const uint32_t *fin_inst, uint32_t fin_off,
                                                        OutT *out, bool out_is_basis) {
  __shared__ T s_g[CB_MAX_M + 1];
  const uint32_t t = fin_off + blockIdx.x;
  const uint32_t r = fin_inst[t];
  const InstDesc I = inst[r];
  const uint32_t ms = sc.ms;
  const uint32_t M = sc.status[r] == CB_OK ? sc.meff[r] : 0u;
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
    // full group: vector loads (node_base is a multiple of 32 elements), four
    // basis vectors per iteration so that 8 vector loads are in flight
    uint32_t j = 0;
    for (; j + 4 <= M; j += 4) {
      T x[4][8];
#pragma unroll
      for (int u = 0; u < 4; ++u) Vec8<T>::load(w + (uint64_t)(j + u) * vs, x[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const T g = s_g[j + u];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] += g * x[u][q];
      }
    }
    for (; j < M; ++j) {
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
      for (int q = 0; q < 8; ++q)
        if ((uint32_t)q < cnt) acc[q] += g * wj[q];
    }
  }
  OutT *o = out_is_basis ? out + I.node_base + i0 : out + i0;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if ((uint32_t)q < cnt) o[q] = (OutT)acc[q];
}

// S(i) = sum_r [i < n_r] exp(theta_r - theta*) y_r(i), in realisation order,
// FP64; y_r was written into basis slot `yslot` by combine_y_kernel.
template <typename T>
__global__ void __launch_bounds__(256) combine_sum_kernel(const T *Y, Scalars sc,
                                                          const InstDesc *inst, uint32_t n_inst,
                                                          uint32_t n_out, double *S,
                                                          double *log_scale) {
  extern __shared__ unsigned char s_raw[];
  double *s_wt = reinterpret_cast<double *>(s_raw);                // exp(theta_r - theta*)
  uint64_t *s_base = reinterpret_cast<uint64_t *>(s_wt + n_inst);  // node_base
  uint32_t *s_n = reinterpret_cast<uint32_t *>(s_base + n_inst);   // n_r
  __shared__ double s_max[8];
  __shared__ int s_badw[8];
  double tm = -1e308;
  int bad = 0;
  for (uint32_t r = threadIdx.x; r < n_inst; r += blockDim.x) {
    tm = fmax(tm, sc.theta[r]);
    bad |= (sc.status[r] != CB_OK);
    s_base[r] = inst[r].node_base;
    s_n[r] = inst[r].n;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tm = fmax(tm, __shfl_xor_sync(0xffffffffu, tm, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) { s_max[threadIdx.x >> 5] = tm; s_badw[threadIdx.x >> 5] = bad; }
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
  // 8 realisations' loads in flight, then their terms in realisation order;
  // realisations with n_r <= i are skipped (warp-uniform except at n_r), so
  // the scarce FP64 pipe only sees real terms
  constexpr uint32_t kB = 8;
  double sum = 0.0;
  for (uint32_t r0 = 0; r0 < n_inst; r0 += kB) {
    T y[kB];
    bool in[kB];
#pragma unroll
    for (uint32_t u = 0; u < kB; ++u) {
      const uint32_t r = r0 + u;
      in[u] = r < n_inst && i < s_n[r];
      y[u] = in[u] ? Y[s_base[r] + i] : T(0);
    }
#pragma unroll
    for (uint32_t u = 0; u < kB; ++u)
      if (in[u]) sum += s_wt[r0 + u] * (double)y[u];
  }
  S[i] = any_bad ? qnan : sum;
}

int combine_single(cb_graph *h, uint32_t r, int prec, double *y, double *log_scale,
                   cudaStream_t s) {
  const InstDesc &I = h->inst[r];
  prefer_shared(combine_y_kernel<double, double>);
  prefer_shared(combine_y_kernel<float, double>);
  prefer_shared(log_scale_kernel);
  const int tok = prof_begin(CB_K_COMBINE, s);
  if (I.n_fin) {
    if (prec == CB_FP64)
      combine_y_kernel<double, double><<<I.n_fin, 256, 0, s>>>(
          (const double *)h->ws.V, h->ws.vec_stride, h->ws.sc, h->d_inst, h->d_fin_inst,
          I.fin_base, y, false);
    else
      combine_y_kernel<float, double><<<I.n_fin, 256, 0, s>>>(
          (const float *)h->ws.V, h->ws.vec_stride, h->ws.sc, h->d_inst, h->d_fin_inst,
          I.fin_base, y, false);
  }
  log_scale_kernel<<<1, 32, 0, s>>>(h->ws.sc, r, log_scale);
  prof_end(tok, s);
  return cuda_error(cudaGetLastError(), "combine launch");
}

int combine_ensemble(cb_graph *h, int prec, uint32_t n_out, double *S, double *log_scale,
                     cudaStream_t s) {
  NvtxRange nvtx_range("ensemble combine");
  const size_t shm = (sizeof(double) + sizeof(uint64_t) + sizeof(uint32_t)) * h->n_inst;
  if (shm > 200 * 1024) return set_error(CB_ERR_ARG, "too many realisations for one combine");
  const uint32_t grid = (n_out + 255) / 256;
  prefer_shared(combine_y_kernel<double, double>);
  prefer_shared(combine_y_kernel<float, float>);
  prefer_shared(combine_sum_kernel<double>);
  prefer_shared(combine_sum_kernel<float>);
  const int tok = prof_begin(CB_K_COMBINE, s);
  // per-realisation terms go into the last basis slot, which the combine never reads
  const uint64_t yoff = (uint64_t)h->ws.m * h->ws.vec_stride;
  if (prec == CB_FP64) {
    double *Y = (double *)h->ws.V + yoff;
    combine_y_kernel<double, double><<<h->total_fin, 256, 0, s>>>(
        (const double *)h->ws.V, h->ws.vec_stride, h->ws.sc, h->d_inst, h->d_fin_inst, 0, Y, true);
    auto k = combine_sum_kernel<double>;
    if (shm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    k<<<grid, 256, shm, s>>>(Y, h->ws.sc, h->d_inst, h->n_inst, n_out, S, log_scale);
  } else {
    float *Y = (float *)h->ws.V + yoff;
    combine_y_kernel<float, float><<<h->total_fin, 256, 0, s>>>(
        (const float *)h->ws.V, h->ws.vec_stride, h->ws.sc, h->d_inst, h->d_fin_inst, 0, Y, true);
    auto k = combine_sum_kernel<float>;
    if (shm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    k<<<grid, 256, shm, s>>>(Y, h->ws.sc, h->d_inst, h->n_inst, n_out, S, log_scale);
  }
  prof_end(tok, s);
  return cuda_error(cudaGetLastError(), "combine launch");
}

int combine_sum_f64(cb_graph *h, const double *Y, uint32_t n_out, double *S, double *log_scale,
                    cudaStream_t s) {
  const size_t shm = (sizeof(double) + sizeof(uint64_t) + sizeof(uint32_t)) * h->n_inst;
  if (shm > 200 * 1024) return set_error(CB_ERR_ARG, "too many realisations for one combine");
  auto k = combine_sum_kernel<double>;
  prefer_shared(k);
  if (shm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  const int tok = prof_begin(CB_K_COMBINE, s);
  k<<<(n_out + 255) / 256, 256, shm, s>>>(Y, h->ws.sc, h->d_inst, h->n_inst, n_out, S, log_scale);
  prof_end(tok, s);
  return cuda_error(cudaGetLastError(), "combine launch");
}

}  // namespace cb
