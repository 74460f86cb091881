// Device-side pieces shared by the Lanczos step kernels (cb_lanczos.cu and
// cb_twophase.cu): the launch arguments, the row epilogue of the SpMV step,
// the completion of alpha_j, and the mbarrier / bulk-copy helpers.
#pragma once

#include "cb_internal.cuh"
#include "cb_reduce.cuh"

namespace cb {

// debug-build violation record of the translation unit (see cb_internal.cuh)
CB_DEBUG_STATE()

struct LArgs {
  const InstDesc *inst;
  const uint32_t *tile_inst;
  const uint2 *tile_rows;
  const HeavyRow *heavy;
  const uint32_t *chunk_heavy;
  const uint32_t *fin_inst;
  const uint32_t *row_ptr;
  const uint32_t *col;
  void *V;
  uint64_t vs;  // vector stride (elements)
  Scalars sc;
  RedBufs red;
  double *cpart;   // per heavy-row chunk partial sums
  uint32_t *hcnt;  // per heavy row arrival counters
  double tau;      // breakdown tolerance
  // column-blocked format (FP32 path)
  const uint32_t *btile_inst;
  const uint64_t *bseg_base, *bwstart;
  const uint32_t *bwlen;
  const uint32_t *belem;
  const uint32_t *blong_ptr, *blong_rows;
  uint32_t skip_blocked;  // the tiled-CSR kernel leaves blocked realisations alone
  uint32_t stall_btile;   // test hook: this tile's first column block is never copied
  // two-phase format (FP32 path)
  const PBin *pbin;
  const uint64_t *ptbase;
  const uint32_t *ptile_inst;
  const uint64_t *pxbase;
  const uint16_t *psrc;
  const uint32_t *pgdst;
  float *pX;
  const uint16_t *psl;      // phase-2 plans (sliced rows)
  const P2Desc *pdesc;      // per bin: its phase-2 copies
  uint64_t pgroups;  // groups of the value array (bounds of the debug build)
  uint32_t skip_pb;  // the tiled-CSR kernel leaves two-phase realisations alone
};

// Column indices are read once per step: streaming (evict-first) load.
__device__ __forceinline__ uint32_t ld_stream(const uint32_t *p) { return __ldcs(p); }

template <typename T>
__device__ __forceinline__ T ld_vec(const T *p) {
  return __ldg(p);
}

// Row epilogue: u = sj*sum - bp*W_{j-1}[row]; store; return W_j[row]*u.
template <typename T>
__device__ __forceinline__ T row_epilogue(T sum, uint32_t row, const T *x, const T *xp, T *out,
                                          T sj, T bp, bool has_prev) {
  T u = sj * sum;
  if (has_prev) u -= bp * xp[row];
  out[row] = u;
  return x[row] * u;
}

template <typename T>
__device__ __forceinline__ void finish_alpha(const LArgs &a, uint32_t r, uint32_t j, double total) {
  const uint32_t ms = a.sc.ms;
  const double alpha = a.sc.scale[r * ms + j] * total;
  a.sc.alpha[r * ms + j] = alpha;
  if (!isfinite(alpha)) {
    if (a.sc.status[r] == CB_OK) a.sc.status[r] = CB_ERR_NONFINITE;
    a.sc.meff[r] = j;  // stop; this realisation is reported as failed
  }
}

// One chunk of kChunk entries of a heavy row (degree > kHeavyDeg), summed by
// the whole CTA (any width) with global gathers; the last chunk of the row to
// finish sums the chunk partials in chunk order, applies the row epilogue and
// enters the row's alpha term as slot `slot` of `plan` -- by the CTA
// (arrive_and_reduce) or, with WarpArrive, by its first warp
// (warp_arrive_and_reduce), whichever the plan's other slots use, so that
// the realisation's sum takes one order whichever CTA arrives last.
template <typename T, bool WarpArrive = false>
__device__ __forceinline__ void heavy_chunk(const LArgs &a, uint32_t j, uint32_t cidx, uint32_t hid,
                                            uint32_t r, const RedPlan &plan, uint32_t slot) {
  __shared__ double s_hred[32];
  __shared__ int s_hlast;
  const InstDesc &I = a.inst[r];
  const uint32_t ms = a.sc.ms;
  const uint32_t *rp = a.row_ptr + I.rp_base;
  const uint32_t *col = a.col + I.edge_base;
  T *Vb = reinterpret_cast<T *>(a.V);
  const T *x = Vb + (uint64_t)j * a.vs + I.node_base;
  const bool has_prev = j > 0;
  const T *xp = has_prev ? Vb + (uint64_t)(j - 1) * a.vs + I.node_base : x;
  T *out = Vb + (uint64_t)(j + 1) * a.vs + I.node_base;
  const T sj = (T)a.sc.scale[r * ms + j];
  const T bp = has_prev ? (T)(a.sc.beta[r * ms + j - 1] * a.sc.scale[r * ms + j - 1]) : T(0);
  const HeavyRow H = a.heavy[hid];
  const uint32_t c = cidx - H.chunk_base;
  const uint32_t e0 = rp[H.row] + c * kChunk;
  const uint32_t e1 = min(e0 + kChunk, rp[H.row + 1]);
  T s = T(0);
  for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const uint32_t cl = ld_stream(col + e);
    if (CB_DCHECK(cl < I.n, kDbgCsrCol, cl)) s += ld_vec(x + cl);
  }
  const double part = block_sum_to_double<T>(s, s_hred);
  if (threadIdx.x == 0) {
    a.cpart[cidx] = part;
    __threadfence();
    const uint32_t prev = atomicAdd(&a.hcnt[hid], 1u);
    s_hlast = (prev == H.n_chunks - 1);
  }
  __syncthreads();
  if (!s_hlast) return;
  __threadfence();
  double dot = 0.0;
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (uint32_t q = 0; q < H.n_chunks; ++q) tot += __ldcg(&a.cpart[H.chunk_base + q]);
    a.hcnt[hid] = 0u;
    dot = (double)row_epilogue<T>((T)tot, H.row, x, xp, out, sj, bp, has_prev);
  }
  double total;
  if (WarpArrive) {
    if (threadIdx.x < 32) {
      dot = __shfl_sync(0xffffffffu, dot, 0);
      if (warp_arrive_and_reduce(plan, slot, r, dot, a.red, &total) && threadIdx.x == 0)
        finish_alpha<T>(a, r, j, total);
    }
  } else if (arrive_and_reduce(plan, slot, r, dot, a.red, &total)) {
    finish_alpha<T>(a, r, j, total);
  }
}

// mbarrier and bulk-copy helpers (shared-window addresses).
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase of `parity` to complete: false after 1 s of
// global time or kSpinLimit polls, whichever comes first.
constexpr uint32_t kSpinLimit = 1u << 26;
constexpr uint64_t kWaitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1; it < kSpinLimit; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 15u) == 0 && global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}
// Bounded wait as mbar_wait, but each poll may suspend the thread until the
// phase completes (up to 0.1 ms), so a waiting warp takes almost no issue
// slots from the warps that compute.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait_sleep(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1; it < kSpinLimit; ++it) {
    if (mbar_try_wait_sleep(bar, parity)) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}
// One bulk copy global -> shared whose bytes complete on `bar` (16-byte
// aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Prefetch of a global range into L2 (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void l2_prefetch(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned);
// cp_async_wait_all waits for every copy the thread has issued.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Two-phase SpMV step of the realisations in the given ranges (cb_twophase.cu):
// phase 1 over the streams of source tiles [tile_lo, tile_hi) (groups
// [g_lo, g_hi)), then phase 2 over heavy-row chunks [chunk_off, +n_chunks)
// (those of two-phase realisations) and bins [bin_off, +n_bins).
void launch_twophase(const LArgs &a, int lanes, uint32_t j, uint32_t tile_lo, uint32_t tile_hi,
                     uint64_t g_lo, uint64_t g_hi, uint32_t chunk_off, uint32_t n_chunks,
                     uint32_t bin_off, uint32_t n_bins, cudaStream_t s);

}  // namespace cb
