// Deterministic CTA / grid reductions used by the Lanczos kernels.
//
// Grid-wide sums follow the "last CTA to arrive" pattern: every CTA writes
// its partial to a slot, fences, and bumps its group's arrival counter; the
// CTA that completes a group sums that group's slots in a fixed order, and
// the CTA that completes the last group of a realisation sums the group
// partials in a fixed order.  Nothing ever waits on another CTA, so there is
// no spin loop, and the summation order does not depend on scheduling.  The
// finalize step's norm uses the same slots and groups but no counters: its
// CTAs only write their partials, and a following kernel (one CTA per
// realisation) forms the group and realisation sums in the same order.
#pragma once

#include "cb_internal.cuh"

namespace cb {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v);
template <>
__device__ __forceinline__ float warp_sum<float>(float v) { return warp_sum_f(v); }
template <>
__device__ __forceinline__ double warp_sum<double>(double v) { return warp_sum_d(v); }

// Sum over a group of G consecutive lanes (G a power of two <= 32); every
// lane of the group gets the sum.
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of a per-thread value: warp sums in T, then the per-warp sums
// are added in FP64 in warp order.  Result valid in thread 0.
template <typename T>
__device__ __forceinline__ double block_sum_to_double(T v, double *sh /* >= 32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum<T>(v);
  if (lane == 0) sh[warp] = (double)v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) r += sh[w];
  }
  __syncthreads();
  return r;
}

struct RedBufs {
  double *part;
  double *gpart;
  uint32_t *gcnt;
  uint32_t *icnt;
};

// All threads of the CTA must call this.  `val` is read from thread 0.
// Returns true in thread 0 of the single CTA that completes the
// realisation; `*total` then holds the realisation's sum.
__device__ __forceinline__ bool arrive_and_reduce(const RedPlan &P, uint32_t slot_local,
                                                  uint32_t inst, double val, const RedBufs &B,
                                                  double *total) {
  __shared__ int s_flag;
  __shared__ double s_red[32];
  const uint32_t g = slot_local / kGroup;
  const uint32_t gsize = min((uint32_t)kGroup, P.n_slots - g * kGroup);
  if (threadIdx.x == 0) {
    B.part[P.slot_base + slot_local] = val;
    __threadfence();
    const uint32_t prev = atomicAdd(&B.gcnt[P.group_base + g], 1u);
    s_flag = (prev == gsize - 1);
  }
  __syncthreads();
  if (!s_flag) return false;
  __threadfence();
  if (threadIdx.x < 32) {
    const uint32_t l = threadIdx.x;
    double v = (l < gsize) ? __ldcg(&B.part[P.slot_base + g * kGroup + l]) : 0.0;
    v = warp_sum_d(v);
    if (l == 0) {
      B.gpart[P.group_base + g] = v;
      B.gcnt[P.group_base + g] = 0u;
      __threadfence();
      const uint32_t prev = atomicAdd(&B.icnt[inst], 1u);
      s_flag = (prev == P.n_groups - 1);
    }
  }
  __syncthreads();
  if (!s_flag) return false;
  __threadfence();
  double acc = 0.0;
  for (uint32_t q = threadIdx.x; q < P.n_groups; q += blockDim.x)
    acc += __ldcg(&B.gpart[P.group_base + q]);
  acc = warp_sum_d(acc);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += s_red[w];
    *total = t;
    B.icnt[inst] = 0u;
    return true;
  }
  return false;
}

// arrive_and_reduce run by one full warp (the other warps of the CTA may
// have exited): the same slots, groups and counters, the group sum over its
// kGroup slots by the warp's lanes, the realisation sum over the groups by
// lane-strided partial sums and a shuffle tree.  Returns true (in every
// lane) in the warp that completes the realisation; *total then holds its
// sum.
__device__ __forceinline__ bool warp_arrive_and_reduce(const RedPlan &P, uint32_t slot_local,
                                                       uint32_t inst, double val, const RedBufs &B,
                                                       double *total) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t g = slot_local / kGroup;
  const uint32_t gsize = min((uint32_t)kGroup, P.n_slots - g * kGroup);
  uint32_t last = 0;
  if (lane == 0) {
    B.part[P.slot_base + slot_local] = val;
    __threadfence();
    last = atomicAdd(&B.gcnt[P.group_base + g], 1u) == gsize - 1;
  }
  if (!__shfl_sync(0xffffffffu, last, 0)) return false;
  __threadfence();
  double v = lane < gsize ? __ldcg(&B.part[P.slot_base + g * kGroup + lane]) : 0.0;
  v = warp_sum_d(v);
  if (lane == 0) {
    B.gpart[P.group_base + g] = v;
    B.gcnt[P.group_base + g] = 0u;
    __threadfence();
    last = atomicAdd(&B.icnt[inst], 1u) == P.n_groups - 1;
  }
  if (!__shfl_sync(0xffffffffu, last, 0)) return false;
  __threadfence();
  double acc = 0.0;
  for (uint32_t q = lane; q < P.n_groups; q += 32) acc += __ldcg(&B.gpart[P.group_base + q]);
  acc = warp_sum_d(acc);
  if (lane == 0) B.icnt[inst] = 0u;
  *total = acc;
  return true;
}

}  // namespace cb
