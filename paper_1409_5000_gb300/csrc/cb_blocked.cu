// Builder of the column-blocked adjacency format used by the FP32 SpMV.
//
// On GB300 a random 4-byte gather from L2 costs one 32-byte sector request
// (about one per clock per SM), while a shared-memory gather is ~6x cheaper.
// The format lets the SpMV stage a block of kBCol entries of v_j in shared
// memory and gather only from there:
//   * rows are tiled by kBTileRows; thread i of a tile owns rows
//     i + kBThreads * k, k = 0..kBRowsPerThread-1 (row slot k), and its row
//     sums sit in shared memory at k * kBThreads + i, so the sums of one
//     warp's rows fall in bank (i mod 32) of the owning lane;
//   * a tile's edges are grouped by column block b = col >> kBColBits into
//     one segment per (tile, b), and within it per warp: the elements of the
//     warp's 512 rows, taken lane by lane (each lane's rows in slot order,
//     each row's columns in order), are dealt round-robin over the T steps
//     of the warp's stream: element j goes to step j mod T, lane j / T.
//     With T >= the elements / 32, >= half the elements of any one lane and
//     >= the elements of any one row, a step holds at most 32 elements, never
//     two of one row (no two lanes add into the same sum at once) and at
//     most two of one lane's rows (at most two-way bank conflicts on the
//     sums), while the padding stays a few percent instead of the spread
//     between the warp's fullest and emptiest lane;
//   * an element is one u32: the local column (col & (kBCol-1)) and, above
//     it, the offset of its row sum from the warp's base (k * kBThreads +
//     owner lane); steps are stored in pairs, [step / 2][lane][2], so a lane
//     reads two elements per 8-byte load and a warp 256 contiguous bytes;
//   * padding elements read column 0 into the executing lane's spare sum
//     (slot kBRowsPerThread), which the epilogue never reads.
// Rows with more than kBLongDeg entries stay out of the streams; the SpMV
// sums them from the CSR with whole-CTA global gathers.  Built on the device
// from the CSR (one count pass per group of realisations as its copies land,
// a device prefix over the step counts, one fill pass), once per upload.
#include <algorithm>
#include <cstdlib>

#include "cb_internal.cuh"

namespace cb {

CB_DEBUG_STATE()

namespace {

constexpr uint32_t kFillThreads = 128;  // lanes of a tile per count / fill CTA
constexpr uint32_t kFillBatch = 4;      // column loads a lane keeps in flight

// Entry ranges of a lane's kBRowsPerThread rows (first row `row`, stride
// kBThreads), all loaded before the walk; rows past n and rows longer than
// kBLongDeg (summed by the SpMV from the CSR) get an empty range.
__device__ __forceinline__ void row_ranges(const uint32_t *rp, uint32_t row, uint32_t n,
                                           uint32_t (&e0)[kBRowsPerThread],
                                           uint32_t (&e1)[kBRowsPerThread]) {
#pragma unroll
  for (int k = 0; k < kBRowsPerThread; ++k) {
    const uint32_t r = row + kBThreads * k;
    e0[k] = e1[k] = 0;
    if (r < n) {
      e0[k] = rp[r];
      e1[k] = rp[r + 1];
    }
  }
#pragma unroll
  for (int k = 0; k < kBRowsPerThread; ++k)
    if (e1[k] - e0[k] > kBLongDeg) e1[k] = e0[k];
}

// Columns e .. e + kFillBatch - 1 of a row ending at e1, issued together
// (entries past e1 are not read).
__device__ __forceinline__ void load_batch(const uint32_t *cl, uint32_t e, uint32_t e1,
                                           uint32_t (&cv)[kFillBatch]) {
#pragma unroll
  for (uint32_t u = 0; u < kFillBatch; ++u) cv[u] = e + u < e1 ? __ldg(cl + e + u) : 0u;
}

// Per (segment, warp): the stream's step count T, the smallest even T with
// 32 T >= the warp's elements in the column block, 2 T >= the most elements
// of one lane, and T >= the most elements of one row (see the layout in the
// header), and each lane's element count per block, kept for the fill.
// CTAs of kFillThreads lanes of a tile; per-(block, lane) counters in shared
// memory.  Columns of a row are sorted, so a row's elements in one block are
// one run of its walk.
__global__ void __launch_bounds__(kFillThreads) bcount_kernel(const InstDesc *inst,
                                                              const uint32_t *btile_inst,
                                                              const uint64_t *bseg_base,
                                                              const uint32_t *row_ptr,
                                                              const uint32_t *col, uint32_t *bwlen,
                                                              uint16_t *bcnt, uint32_t *unsorted,
                                                              uint32_t t_off) {
  __shared__ uint16_t s_cnt[kBMaxBlocks][kFillThreads];  // elements of the lane in block b
  __shared__ uint16_t s_run[kBMaxBlocks][kFillThreads];  // its longest row in block b
  const uint32_t t = t_off + blockIdx.x;
  const InstDesc I = inst[btile_inst[t]];
  const uint32_t *rp = row_ptr + I.rp_base;
  const uint32_t *cl = col + I.edge_base;
  const uint32_t row0 = (t - I.btile_base) * kBTileRows;
  const uint32_t tid = threadIdx.x;
  const uint32_t v = blockIdx.y * kFillThreads + tid;
  const uint32_t nb = I.nb;
  for (uint32_t b = 0; b < nb; ++b) {
    s_cnt[b][tid] = 0;
    s_run[b][tid] = 0;
  }
  bool bad = false;
  uint32_t re0[kBRowsPerThread], re1[kBRowsPerThread];
  row_ranges(rp, row0 + v, I.n, re0, re1);
#pragma unroll
  for (int k = 0; k < kBRowsPerThread; ++k) {
    const uint32_t e0 = re0[k], e1 = re1[k];
    uint32_t prev = 0, cur_b = kBMaxBlocks, run = 0;
    for (uint32_t e = e0; e < e1; e += kFillBatch) {
      uint32_t cv[kFillBatch];
      load_batch(cl, e, e1, cv);
#pragma unroll
      for (uint32_t u = 0; u < kFillBatch; ++u) {
        if (e + u >= e1) break;
        const uint32_t c = cv[u];
        const uint32_t b = c >> kBColBits;
        bad |= e + u > e0 && c < prev;  // the format needs sorted rows
        prev = c;
        if (b >= nb) continue;          // columns >= n are invalid input: skipped
        s_cnt[b][tid]++;
        if (b == cur_b) {
          ++run;
        } else {
          if (cur_b < nb) s_run[cur_b][tid] = (uint16_t)max((uint32_t)s_run[cur_b][tid], run);
          cur_b = b;
          run = 1;
        }
      }
    }
    if (cur_b < nb) s_run[cur_b][tid] = (uint16_t)max((uint32_t)s_run[cur_b][tid], run);
  }
  if (bad) *unsorted = 1u;
  for (uint32_t b = 0; b < nb; ++b) {
    const uint32_t c = s_cnt[b][tid];
    const uint32_t tot = __reduce_add_sync(0xffffffffu, c);
    const uint32_t most = __reduce_max_sync(0xffffffffu, c);
    const uint32_t row = __reduce_max_sync(0xffffffffu, (uint32_t)s_run[b][tid]);
    const uint32_t T = max(max((tot + 31) / 32, (most + 1) / 2), row);
    if ((tid & 31) == 0) bwlen[(bseg_base[t] + b) * 32 + (v >> 5)] = (T + 1) & ~1u;
    bcnt[(bseg_base[t] + b) * kBThreads + v] = (uint16_t)c;  // the fill's lane offsets
  }
}

// Fill the streams.  The count pass left each lane's elements per block; a
// warp prefix over the lanes gives each lane the first index j of its
// elements in the warp's sequence (lanes in order, each lane's in walk order:
// rows in slot order, columns in input order).  Element j belongs at
// step j mod T, lane j / T, and the positions past the warp's last element
// (j from its count to 32 T) take the lane's padding element.  The streams
// are then written a batch of blocks at a time: each warp assembles its
// streams of the batch in shared memory (one walk over the rows, each row
// resumed where the previous batch stopped -- the columns of a row are
// sorted) and copies them out with coalesced 16-byte stores.  A block whose stream does not fit the
// staging area is written element by element.
constexpr uint32_t kStageWords = 2048;  // staging u32 words per warp

__global__ void __launch_bounds__(kFillThreads) bfill_kernel(const InstDesc *inst,
                                                             const uint32_t *btile_inst,
                                                             const uint64_t *bseg_base,
                                                             const uint64_t *bwstart,
                                                             const uint32_t *bwlen,
                                                             const uint16_t *bcnt,
                                                             const uint32_t *row_ptr,
                                                             const uint32_t *col, uint32_t *belem,
                                                             uint32_t nbmax) {
  // dynamic shared memory: the staging areas [4][kStageWords] u32, then per
  // (block, warp of the CTA) the stream start (u64), step count and element
  // count (u32), then the next index [nbmax][kFillThreads] u32
  extern __shared__ uint4 s_dyn4[];
  uint32_t *s_stage = reinterpret_cast<uint32_t *>(s_dyn4);
  uint64_t *s_start = reinterpret_cast<uint64_t *>(s_stage + (kFillThreads / 32) * kStageWords);
  uint32_t *s_T = reinterpret_cast<uint32_t *>(s_start + nbmax * (kFillThreads / 32));
  uint32_t *s_tot = s_T + nbmax * (kFillThreads / 32);
  uint32_t *s_sb = s_tot + nbmax * (kFillThreads / 32);  // staging offset of block b's stream
  uint32_t *s_next = s_sb + nbmax * (kFillThreads / 32);
  uint32_t *s_ecur = s_next + nbmax * kFillThreads;  // [k][lane]: next entry of row slot k
  uint32_t *s_re1 = s_ecur + kBRowsPerThread * kFillThreads;  // [k][lane]: end of row slot k
  const uint32_t t = blockIdx.x;
  const InstDesc I = inst[btile_inst[t]];
  const uint32_t *rp = row_ptr + I.rp_base;
  const uint32_t *cl = col + I.edge_base;
  const uint32_t row0 = (t - I.btile_base) * kBTileRows;
  const uint32_t tid = threadIdx.x;
  const uint32_t v = blockIdx.y * kFillThreads + tid;  // lane index within the tile (SpMV thread)
  const uint32_t lane = v & 31, wl = tid >> 5;          // wl: warp within this CTA
  const uint32_t nb = I.nb;
  constexpr uint32_t W = kFillThreads / 32;
  uint32_t *stage = s_stage + wl * kStageWords;  // this warp's staging area
  for (uint32_t q = tid; q < nb * W; q += kFillThreads) {
    const uint32_t b = q / W, w = q % W;
    const uint64_t wi = (bseg_base[t] + b) * 32 + blockIdx.y * W + w;
    s_start[q] = bwstart[wi];
    s_T[q] = bwlen[wi];
  }
  __syncthreads();
  {
    uint32_t re0[kBRowsPerThread], re1[kBRowsPerThread];
    row_ranges(rp, row0 + v, I.n, re0, re1);
#pragma unroll
    for (int k = 0; k < kBRowsPerThread; ++k) {
      s_ecur[k * kFillThreads + tid] = re0[k];
      s_re1[k * kFillThreads + tid] = re1[k];
    }
  }
  // the walk loops over the row slots without unrolling (the kernel stays
  // small enough for the instruction cache); the row cursors live in shared
  // memory.
  // The lane's elements per block come from the count pass; their exclusive
  // prefix over the warp's lanes gives each lane its first position (step s,
  // lane l), kept as l << 16 | s and advanced per element
  for (uint32_t b = 0; b < nb; ++b) {
    const uint32_t c = bcnt[(bseg_base[t] + b) * kBThreads + v];
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    const uint32_t j0 = incl - c, T = s_T[b * W + wl];
    s_next[b * kFillThreads + tid] = T ? ((j0 / T) << 16) | (j0 % T) : 0u;
    if (lane == 31) s_tot[b * W + wl] = incl;
  }
  __syncwarp();
  // second walk, a batch of blocks [b0, b1) at a time; the batch ends before
  // the block that would overflow the staging area of this warp
  uint32_t b0 = 0;
  while (b0 < nb) {
    uint32_t b1 = b0, used = 0;
    while (b1 < nb && (used + 32 * s_T[b1 * W + wl] <= kStageWords || b1 == b0)) {
      if (lane == 0) s_sb[b1 * W + wl] = used;
      used += 32 * s_T[b1 * W + wl];
      ++b1;
    }
    __syncwarp();
    const bool staged = used <= kStageWords;  // false: one block too large, written directly
    // the padding of the batch's streams
    for (uint32_t b = b0; b < b1; ++b) {
      const uint32_t T = s_T[b * W + wl], base = s_sb[b * W + wl];
      const uint64_t st = s_start[b * W + wl];
      for (uint32_t j = s_tot[b * W + wl] + lane; j < 32 * T; j += 32) {
        const uint32_t s = j % T, l = j / T;
        const uint32_t q = 64 * (s >> 1) + 2 * l + (s & 1);
        const uint32_t el = kBPadOff(l) << kBColBits;
        if (staged) stage[base + q] = el; else belem[st + q] = el;
      }
    }
    // the elements of blocks [b0, b1), resuming each row where the last batch stopped
#pragma unroll 1
    for (int k = 0; k < kBRowsPerThread; ++k) {
      const uint32_t e1 = s_re1[k * kFillThreads + tid];
      const uint32_t off = (uint32_t)k * kBThreads + lane;  // row sum of (slot k, lane)
      uint32_t e = s_ecur[k * kFillThreads + tid];
      bool more = e < e1;
      while (more) {  // kFillBatch columns per round of loads
        uint32_t cv[kFillBatch];
        load_batch(cl, e, e1, cv);
        uint32_t taken = kFillBatch;
#pragma unroll
        for (uint32_t u = 0; u < kFillBatch; ++u) {
          if (e + u >= e1 || (cv[u] >> kBColBits) >= b1) {  // the row is done for this batch
            taken = u;
            break;
          }
          const uint32_t c = cv[u];
          const uint32_t b = c >> kBColBits;  // b0 <= b < b1 (columns >= n end the row's walk)
          const uint32_t T = s_T[b * W + wl];
          uint32_t p = s_next[b * kFillThreads + tid];
          const uint32_t s = p & 0xffffu, l = p >> 16;
          p = s + 1 == T ? p + (1u << 16) - s : p + 1;
          s_next[b * kFillThreads + tid] = p;
          if (!CB_DCHECK(l < 32u && s < T, kDbgBlockedFill, p)) continue;
          const uint32_t q = 64 * (s >> 1) + 2 * l + (s & 1);
          const uint32_t el = (c & (kBCol - 1)) | (off << kBColBits);
          if (staged) stage[s_sb[b * W + wl] + q] = el; else belem[s_start[b * W + wl] + q] = el;
        }
        e += taken;
        more = taken == kFillBatch && e < e1;
      }
      s_ecur[k * kFillThreads + tid] = e;
    }
    __syncwarp();
    if (staged) {  // the batch's streams, 16 bytes per lane per store
      for (uint32_t b = b0; b < b1; ++b) {
        const uint32_t words = 32 * s_T[b * W + wl];
        uint4 *dst = reinterpret_cast<uint4 *>(belem + s_start[b * W + wl]);
        const uint4 *src = reinterpret_cast<const uint4 *>(stage + s_sb[b * W + wl]);
        for (uint32_t q = lane; q < words / 4; q += 32) dst[q] = src[q];
      }
    }
    __syncwarp();
    b0 = b1;
  }
}

size_t fill_smem_bytes(uint32_t nbmax) {
  return (size_t)(kFillThreads / 32) * kStageWords * 4 +
         (size_t)nbmax * ((kFillThreads / 32) * (8 + 4 + 4 + 4) + kFillThreads * 4) +
         2 * kBRowsPerThread * kFillThreads * 4;
}

// x[i] *= 32: stream offsets in elements from the prefix of per-lane lengths
__global__ void times32_kernel(uint64_t *x, uint64_t n) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] *= 32;
}

template <typename P>
cudaError_t dalloc(P **p, size_t count) {
  return dev_alloc_n(p, count);
}

}  // namespace

void free_blocked(cb_graph *h) {
  dev_free(h->d_btile_inst);
  dev_free(h->d_bseg_base);
  dev_free(h->d_bwstart);
  dev_free(h->d_bwlen);
  dev_free(h->d_bcnt);
  h->d_bcnt = nullptr;
  dev_free(h->d_bwscan);
  dev_free(h->d_belem);
  dev_free(h->d_blong_ptr);
  dev_free(h->d_blong_rows);
  h->d_btile_inst = nullptr;
  h->d_bseg_base = h->d_bwstart = h->d_bwscan = nullptr;
  h->d_bwlen = nullptr;
  h->d_belem = nullptr;
  h->d_blong_ptr = h->d_blong_rows = nullptr;
  h->total_btiles = 0;
  h->total_bseg = 0;
}

int blocked_count(cb_graph *h, cudaStream_t s, const std::vector<CopyGroup> &groups,
                  BlockedBuild &bb) {
  NvtxRange nvtx_range("column-blocked format: count");
  if (h->csr_only) return CB_OK;
  // which realisations, their tiles, segments and reduction plans (sizes only)
  uint32_t nbt = 0, slot = 0, group = 0;
  uint64_t nseg = 0;
  std::vector<uint32_t> btile_inst;
  std::vector<uint64_t> bseg_base;
  for (uint32_t r = 0; r < h->n_inst; ++r) {
    InstDesc &I = h->inst[r];
    I.blocked = !h->force_pb && I.n <= kBMaxBlocks * kBCol ? 1u : 0u;
    I.nb = I.blocked ? (I.n + kBCol - 1) / kBCol : 0u;
    I.btile_base = nbt;
    I.n_btiles = I.blocked ? (I.n + kBTileRows - 1) / kBTileRows : 0u;
    I.bspmv = RedPlan{slot, I.n_btiles, group, (I.n_btiles + kGroup - 1) / kGroup};
    slot += I.bspmv.n_slots;
    group += I.bspmv.n_groups;
    for (uint32_t q = 0; q < I.n_btiles; ++q) {
      btile_inst.push_back(r);
      bseg_base.push_back(nseg);
      nseg += I.nb;
    }
    nbt += I.n_btiles;
  }
  h->total_btiles = nbt;
  h->total_bseg = nseg;
  h->total_slots = std::max(h->total_slots, slot);
  h->total_groups = std::max(h->total_groups, group);
  if (!nbt) return CB_OK;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  const uint64_t nw = nseg * 32;
  chk(dalloc(&h->d_btile_inst, nbt));
  chk(dalloc(&h->d_bseg_base, nbt));
  chk(dalloc(&h->d_bwstart, nw + 1));
  chk(dalloc(&h->d_bwlen, nw + 1));  // + the sortedness flag of the count pass
  chk(dalloc(&h->d_bcnt, nseg * kBThreads));
  chk(dalloc(&h->d_bwscan, nw / 4096 + 2));  // prefix scratch
  bb.result = reinterpret_cast<uint64_t *>(stage_reserve(16));
  if (e == cudaSuccess && !bb.result) e = cudaErrorMemoryAllocation;
  if (e != cudaSuccess) {
    free_blocked(h);
    return cuda_error(e, "blocked format: allocate");
  }
  chk(stage_h2d(h->d_btile_inst, btile_inst.data(), nbt * 4, s));
  chk(stage_h2d(h->d_bseg_base, bseg_base.data(), nbt * 8, s));
  chk(stage_h2d(h->d_inst, h->inst.data(), h->n_inst * sizeof(InstDesc), s));
  // no temporary allocation here: a free synchronises the device, which
  // would stall an upload behind another thread's kernels
  uint32_t *d_unsorted = h->d_bwlen + nw;
  if (e == cudaSuccess) chk(cudaMemsetAsync(d_unsorted, 0, 4, s));
  // count each group of realisations as soon as its columns are on the device
  uint32_t r_begin = 0;
  for (const CopyGroup &g : groups) {
    chk(cudaStreamWaitEvent(s, g.ev, 0));
    const uint32_t t0 = h->inst[r_begin].btile_base;
    const uint32_t t1 = h->inst[g.r_end - 1].btile_base + h->inst[g.r_end - 1].n_btiles;
    if (t1 > t0 && e == cudaSuccess)
      bcount_kernel<<<dim3(t1 - t0, kBThreads / kFillThreads), kFillThreads, 0, s>>>(
          h->d_inst, h->d_btile_inst, h->d_bseg_base, h->row_ptr, h->col, h->d_bwlen, h->d_bcnt,
          d_unsorted, t0);
    r_begin = g.r_end;
  }
  chk(cudaGetLastError());
  // stream offsets on the device: bwstart = 32 x the exclusive prefix of
  // the lengths; only the total and the sortedness flag come back
  if (e == cudaSuccess) chk(exclusive_scan(h->d_bwlen, nw, h->d_bwstart, h->d_bwscan, s));
  if (e == cudaSuccess)
    times32_kernel<<<(uint32_t)((nw + 1 + 255) / 256), 256, 0, s>>>(h->d_bwstart, nw + 1);
  bb.result[0] = 0;
  bb.result[1] = 0;
  chk(cudaMemcpyAsync(bb.result, h->d_bwstart + nw, 8, cudaMemcpyDeviceToHost, s));
  chk(cudaMemcpyAsync(bb.result + 1, d_unsorted, 4, cudaMemcpyDeviceToHost, s));
  chk(cudaEventCreateWithFlags(&bb.ev, cudaEventDisableTiming));
  if (e == cudaSuccess) chk(cudaEventRecord(bb.ev, s));
  if (e != cudaSuccess) {
    cudaStreamSynchronize(s);
    free_blocked(h);
    return cuda_error(e, "blocked format: count");
  }
  return CB_OK;
}

int blocked_fill(cb_graph *h, cudaStream_t s, BlockedBuild &bb) {
  NvtxRange nvtx_range("column-blocked format: fill");
  if (h->csr_only || !h->total_btiles) return CB_OK;
  cudaError_t e = cudaEventSynchronize(bb.ev);
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  if (e == cudaSuccess && bb.result[1]) {
    free_blocked(h);
    return set_error(CB_ERR_ARG, "cb_graph_upload: column indices of every row must be sorted ascending");
  }
  const uint64_t alloc = bb.result[0] + 16;
  chk(dalloc(&h->d_belem, alloc));
  if (e == cudaSuccess) {
    uint32_t nbmax = 1;
    for (uint32_t r = 0; r < h->n_inst; ++r) nbmax = std::max(nbmax, h->inst[r].nb);
    const size_t shm = fill_smem_bytes(nbmax);
    if (shm > 48 * 1024)
      chk(cudaFuncSetAttribute(bfill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    if (e == cudaSuccess)
      bfill_kernel<<<dim3(h->total_btiles, kBThreads / kFillThreads), kFillThreads, shm, s>>>(
          h->d_inst, h->d_btile_inst, h->d_bseg_base, h->d_bwstart, h->d_bwlen, h->d_bcnt,
          h->row_ptr, h->col, h->d_belem, nbmax);
    chk(cudaGetLastError());
  }
  if (e != cudaSuccess) {
    cudaStreamSynchronize(s);
    free_blocked(h);
    return cuda_error(e, "blocked format: fill");
  }
  return CB_OK;
}

int blocked_long_rows(cb_graph *h, const std::vector<const uint32_t *> &rp_host, cudaStream_t s) {
  NvtxRange nvtx_range("column-blocked format: long rows");
  if (h->csr_only || !h->total_btiles) return CB_OK;
  // long rows per tile (tile-local indices), scanned in parallel over realisations
  std::vector<std::vector<uint32_t>> lrows(h->n_inst), lcount(h->n_inst);
  parallel_for(h->n_inst, [&](uint32_t r) {
    const InstDesc &I = h->inst[r];
    const uint32_t *rp = rp_host[r];
    for (uint32_t q = 0; q < I.n_btiles; ++q) {
      const uint32_t row0 = q * kBTileRows, row1 = std::min<uint32_t>(row0 + kBTileRows, I.n);
      uint32_t c = 0;
      for (uint32_t row = row0; row < row1; ++row)
        if (rp[row + 1] - rp[row] > kBLongDeg) {
          lrows[r].push_back(row - row0);
          ++c;
        }
      lcount[r].push_back(c);
    }
  });
  std::vector<uint32_t> long_ptr(1, 0), long_rows;
  for (uint32_t r = 0; r < h->n_inst; ++r) {
    for (uint32_t c : lcount[r]) long_ptr.push_back(long_ptr.back() + c);
    long_rows.insert(long_rows.end(), lrows[r].begin(), lrows[r].end());
  }
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  chk(dalloc(&h->d_blong_ptr, long_ptr.size()));
  chk(dalloc(&h->d_blong_rows, std::max<size_t>(long_rows.size(), 1)));
  chk(stage_h2d(h->d_blong_ptr, long_ptr.data(), long_ptr.size() * 4, s));
  if (!long_rows.empty()) chk(stage_h2d(h->d_blong_rows, long_rows.data(), long_rows.size() * 4, s));
  if (e != cudaSuccess) {
    cudaStreamSynchronize(s);
    free_blocked(h);
    return cuda_error(e, "blocked format: long rows");
  }
  return CB_OK;
}

CB_DEBUG_READER(blocked)

}  // namespace cb
