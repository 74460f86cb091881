// Builder of the column-blocked adjacency format used by the FP32 SpMV.
//
// On GB300 a random 4-byte gather from L2 costs one 32-byte sector request
// (about one per clock per SM), while a shared-memory gather is ~6x cheaper.
// The format lets the SpMV stage a block of kBCol entries of v_j in shared
// memory and gather only from there:
//   * rows are tiled by kBTileRows; thread i of a tile owns rows
//     i + kBThreads * k, k = 0..kBRowsPerThread-1 (row slot k), so even a
//     partly filled tile spreads its rows over all warps;
//   * a tile's edges are grouped by column block b = col >> kBColBits into
//     one segment per (tile, b); thread i's edges of a segment (its rows in
//     order, each row's columns in order) form its stream;
//   * the 32 streams of a warp are interleaved in stripes of 4: element q of
//     lane l sits at start(segment, warp) + 128 (q / 4) + 4 l + q % 4, and
//     every stream is padded to the warp's longest, rounded up to a multiple
//     of 4 (len(segment, warp)).  A lane reads 4 columns (8 bytes) and 4
//     slots (4 bytes) per stripe; a warp's stripe is 384 contiguous bytes, so
//     the loads are coalesced and need no per-element range checks;
//   * each element stores the local column (u16, col & (kBCol-1)) and the row
//     slot of the owning lane (u8, 0..kBRowsPerThread-1); padding elements
//     carry column kBPadCol (a zero word after the staged block) and slot 0,
//     so they add +0.
// Rows with more than kBLongDeg entries stay out of the streams; the SpMV
// sums them from the CSR with whole-CTA global gathers.  Built on the device
// from the CSR (one count pass per group of realisations as its copies land,
// a device prefix over segment lengths, one fill pass), once per upload.
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

// Per (segment, warp) stream length: the largest per-lane element count of the
// warp in that column block, rounded up to a multiple of 4.  CTAs of
// kFillThreads lanes of a tile; per-(block, lane) counters in shared memory.
__global__ void __launch_bounds__(kFillThreads) bcount_kernel(const InstDesc *inst,
                                                              const uint32_t *btile_inst,
                                                              const uint64_t *bseg_base,
                                                              const uint32_t *row_ptr,
                                                              const uint32_t *col, uint32_t *bwlen,
                                                              uint32_t *unsorted, uint32_t t_off) {
  __shared__ uint16_t s_cnt[kBMaxBlocks][kFillThreads];
  const uint32_t t = t_off + blockIdx.x;
  const InstDesc I = inst[btile_inst[t]];
  const uint32_t *rp = row_ptr + I.rp_base;
  const uint32_t *cl = col + I.edge_base;
  const uint32_t row0 = (t - I.btile_base) * kBTileRows;
  const uint32_t tid = threadIdx.x;
  const uint32_t v = blockIdx.y * kFillThreads + tid;
  const uint32_t nb = I.nb;
  for (uint32_t b = 0; b < nb; ++b) s_cnt[b][tid] = 0;
  bool bad = false;
  uint32_t re0[kBRowsPerThread], re1[kBRowsPerThread];
  row_ranges(rp, row0 + v, I.n, re0, re1);
#pragma unroll
  for (int k = 0; k < kBRowsPerThread; ++k) {
    const uint32_t e0 = re0[k], e1 = re1[k];
    uint32_t prev = 0;
    for (uint32_t e = e0; e < e1; e += kFillBatch) {
      uint32_t cv[kFillBatch];
      load_batch(cl, e, e1, cv);
#pragma unroll
      for (uint32_t u = 0; u < kFillBatch; ++u) {
        if (e + u >= e1) break;
        const uint32_t c = cv[u];
        const uint32_t b = c >> kBColBits;
        if (b < nb) s_cnt[b][tid]++;    // columns >= n are invalid input: skipped
        bad |= e + u > e0 && c < prev;  // the format needs sorted rows
        prev = c;
      }
    }
  }
  if (bad) *unsorted = 1u;
  for (uint32_t b = 0; b < nb; ++b) {
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, (uint32_t)s_cnt[b][tid]);
    if ((tid & 31) == 0)
      bwlen[(bseg_base[t] + b) * 32 + (v >> 5)] = (wmax + 3) & ~3u;
  }
}

// Fill the streams in one pass over the CSR.  A CTA takes kFillThreads of the
// tile's kBThreads lanes ("virtual threads" v); each walks its rows in slot
// order and each row's columns once, appending every element to the stream
// of its column block.  Per (block, lane), the 4 elements of the open stripe
// wait in shared memory and go out as one 8-byte and one 4-byte store when
// the stripe is full; partial stripes are written at the end (their unfilled
// positions keep the padding values).  The element order within a stream is
// the lane's rows in slot order, each row's columns in input order.
__global__ void __launch_bounds__(kFillThreads) bfill_kernel(const InstDesc *inst,
                                                             const uint32_t *btile_inst,
                                                             const uint64_t *bseg_base,
                                                             const uint64_t *bwstart,
                                                             const uint32_t *row_ptr,
                                                             const uint32_t *col, uint16_t *bcol,
                                                             uint8_t *bslot, uint32_t nbmax) {
  // dynamic shared memory, nbmax column blocks:
  //   start[nbmax][4] u64, col[nbmax][4][128] u16, q[nbmax][128] u16, slot[nbmax][4][128] u8
  extern __shared__ uint64_t s_dyn[];
  uint64_t *s_start = s_dyn;
  uint16_t *s_col = reinterpret_cast<uint16_t *>(s_start + nbmax * (kFillThreads / 32));
  uint16_t *s_q = s_col + nbmax * 4 * kFillThreads;
  uint8_t *s_slot = reinterpret_cast<uint8_t *>(s_q + nbmax * kFillThreads);
  const uint32_t t = blockIdx.x;
  const InstDesc I = inst[btile_inst[t]];
  const uint32_t *rp = row_ptr + I.rp_base;
  const uint32_t *cl = col + I.edge_base;
  const uint32_t row0 = (t - I.btile_base) * kBTileRows;
  const uint32_t tid = threadIdx.x;
  const uint32_t v = blockIdx.y * kFillThreads + tid;  // lane index within the tile
  const uint32_t lane = v & 31, wl = tid >> 5;          // wl: warp within this CTA
  const uint32_t nb = I.nb;
  // element (b, p) of this thread's open stripes
#define COL(b, p) s_col[((b) * 4 + (p)) * kFillThreads + tid]
#define SLOT(b, p) s_slot[((b) * 4 + (p)) * kFillThreads + tid]
  for (uint32_t b = 0; b < nb; ++b) s_q[b * kFillThreads + tid] = 0;
  for (uint32_t q = tid; q < nb * (kFillThreads / 32); q += kFillThreads) {
    const uint32_t b = q / (kFillThreads / 32), w = q % (kFillThreads / 32);
    s_start[q] = bwstart[(bseg_base[t] + b) * 32 + blockIdx.y * (kFillThreads / 32) + w];
  }
  __syncthreads();
  auto flush = [&](uint32_t b, uint32_t stripe) {
    uint2 cv;
    cv.x = (uint32_t)COL(b, 0) | ((uint32_t)COL(b, 1) << 16);
    cv.y = (uint32_t)COL(b, 2) | ((uint32_t)COL(b, 3) << 16);
    const uint32_t sv = (uint32_t)SLOT(b, 0) | ((uint32_t)SLOT(b, 1) << 8) |
                        ((uint32_t)SLOT(b, 2) << 16) | ((uint32_t)SLOT(b, 3) << 24);
    const uint64_t st = s_start[b * (kFillThreads / 32) + wl];
#ifdef CB_DEBUG
    // the stripe lies inside this (segment, warp) stream: before the next one starts
    const uint64_t wi = (bseg_base[t] + b) * 32 + blockIdx.y * (kFillThreads / 32) + wl;
    if (!CB_DCHECK(st + 128ull * stripe + 4 * lane + 3 < bwstart[wi + 1], kDbgBlockedFill,
                   st + 128ull * stripe + 4 * lane))
      return;
#endif
    reinterpret_cast<uint2 *>(bcol + st)[32 * stripe + lane] = cv;
    reinterpret_cast<uint32_t *>(bslot + st)[32 * stripe + lane] = sv;
  };
  uint32_t re0[kBRowsPerThread], re1[kBRowsPerThread];
  row_ranges(rp, row0 + v, I.n, re0, re1);
#pragma unroll
  for (int k = 0; k < kBRowsPerThread; ++k) {
    const uint32_t e1 = re1[k];
    for (uint32_t e = re0[k]; e < e1; e += kFillBatch) {
      uint32_t cv[kFillBatch];
      load_batch(cl, e, e1, cv);
#pragma unroll
      for (uint32_t u = 0; u < kFillBatch; ++u) {
        if (e + u >= e1) break;
        const uint32_t c = cv[u];
        const uint32_t b = c >> kBColBits;
        if (b >= nb) continue;  // columns >= n are invalid input: skipped
        const uint32_t q = s_q[b * kFillThreads + tid];
        const uint32_t p = q & 3;
        COL(b, p) = (uint16_t)(c & (kBCol - 1));
        SLOT(b, p) = (uint8_t)k;
        s_q[b * kFillThreads + tid] = (uint16_t)(q + 1);
        if (p == 3) flush(b, q >> 2);
      }
    }
  }
  for (uint32_t b = 0; b < nb; ++b) {
    const uint32_t q = s_q[b * kFillThreads + tid];
    if (q & 3) {
      for (uint32_t p = q & 3; p < 4; ++p) {
        COL(b, p) = (uint16_t)kBPadCol;
        SLOT(b, p) = 0;
      }
      flush(b, q >> 2);
    }
  }
#undef COL
#undef SLOT
}

size_t fill_smem_bytes(uint32_t nbmax) {
  return (size_t)nbmax * ((kFillThreads / 32) * 8 + kFillThreads * (4 * 2 + 2 + 4));
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
  dev_free(h->d_bwscan);
  dev_free(h->d_bcol);
  dev_free(h->d_bslot);
  dev_free(h->d_blong_ptr);
  dev_free(h->d_blong_rows);
  h->d_btile_inst = nullptr;
  h->d_bseg_base = h->d_bwstart = h->d_bwscan = nullptr;
  h->d_bwlen = nullptr;
  h->d_bcol = nullptr;
  h->d_bslot = nullptr;
  h->d_blong_ptr = h->d_blong_rows = nullptr;
  h->total_btiles = 0;
  h->total_bseg = 0;
}

int build_blocked(cb_graph *h, const std::vector<const uint32_t *> &rp_host, cudaStream_t s,
                  const std::vector<CopyGroup> &groups) {
  NvtxRange nvtx_range("column-blocked format");
  if (h->csr_only) return CB_OK;
  // which realisations, their tiles, segments and reduction plans
  uint32_t nbt = 0, slot = 0, group = 0;
  uint64_t nseg = 0;
  std::vector<uint32_t> btile_inst;
  std::vector<uint64_t> bseg_base;
  std::vector<uint32_t> long_ptr(1, 0), long_rows;
  // long rows per tile, scanned in parallel over realisations
  std::vector<std::vector<uint32_t>> lrows(h->n_inst), lcount(h->n_inst);
  parallel_for(h->n_inst, [&](uint32_t r) {
    const InstDesc &I = h->inst[r];
    if (h->force_pb || I.n > kBMaxBlocks * kBCol) return;
    const uint32_t *rp = rp_host[r];
    const uint32_t ntile = (I.n + kBTileRows - 1) / kBTileRows;
    for (uint32_t q = 0; q < ntile; ++q) {
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
      long_ptr.push_back(long_ptr.back() + lcount[r][q]);
    }
    long_rows.insert(long_rows.end(), lrows[r].begin(), lrows[r].end());
    nbt += I.n_btiles;
  }
  h->total_btiles = nbt;
  h->total_bseg = nseg;
  h->total_slots = std::max(h->total_slots, slot);
  h->total_groups = std::max(h->total_groups, group);
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  if (nbt) {
    const uint64_t nw = nseg * 32;
    chk(dalloc(&h->d_btile_inst, nbt));
    chk(dalloc(&h->d_bseg_base, nbt));
    chk(dalloc(&h->d_bwstart, nw + 1));
    chk(dalloc(&h->d_bwlen, nw + 1));  // + the sortedness flag of the count pass
    chk(dalloc(&h->d_bwscan, nw / 4096 + 2));  // prefix scratch
    chk(dalloc(&h->d_blong_ptr, long_ptr.size()));
    chk(dalloc(&h->d_blong_rows, std::max<size_t>(long_rows.size(), 1)));
    if (e != cudaSuccess) {
      free_blocked(h);
      return cuda_error(e, "blocked format: allocate");
    }
    chk(stage_h2d(h->d_btile_inst, btile_inst.data(), nbt * 4, s));
    chk(stage_h2d(h->d_bseg_base, bseg_base.data(), nbt * 8, s));
    chk(stage_h2d(h->d_blong_ptr, long_ptr.data(), long_ptr.size() * 4, s));
    if (!long_rows.empty()) chk(stage_h2d(h->d_blong_rows, long_rows.data(), long_rows.size() * 4, s));
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
            h->d_inst, h->d_btile_inst, h->d_bseg_base, h->row_ptr, h->col, h->d_bwlen, d_unsorted, t0);
      r_begin = g.r_end;
    }
    chk(cudaGetLastError());
    // stream offsets on the device: bwstart = 32 x the exclusive prefix of
    // the lengths; only the total and the sortedness flag come back
    if (e == cudaSuccess) chk(exclusive_scan(h->d_bwlen, nw, h->d_bwstart, h->d_bwscan, s));
    if (e == cudaSuccess)
      times32_kernel<<<(uint32_t)((nw + 1 + 255) / 256), 256, 0, s>>>(h->d_bwstart, nw + 1);
    uint64_t tot = 0;
    uint32_t unsorted = 0;
    chk(cudaMemcpyAsync(&tot, h->d_bwstart + nw, 8, cudaMemcpyDeviceToHost, s));
    chk(cudaMemcpyAsync(&unsorted, d_unsorted, 4, cudaMemcpyDeviceToHost, s));
    chk(cudaStreamSynchronize(s));
    if (e == cudaSuccess && unsorted) {
      free_blocked(h);
      return set_error(CB_ERR_ARG, "cb_graph_upload: column indices of every row must be sorted ascending");
    }
    const uint64_t alloc = tot + 16;
    chk(dalloc(&h->d_bcol, alloc));
    chk(dalloc(&h->d_bslot, alloc));
    if (e == cudaSuccess) {
      static_assert((kBPadCol >> 8) == (kBPadCol & 0xff), "padding column must be a repeated byte");
      chk(cudaMemsetAsync(h->d_bcol, (int)(kBPadCol & 0xff), alloc * 2, s));  // padding: zero word
      chk(cudaMemsetAsync(h->d_bslot, 0, alloc, s));                          // into slot 0
      uint32_t nbmax = 1;
      for (uint32_t r = 0; r < h->n_inst; ++r) nbmax = std::max(nbmax, h->inst[r].nb);
      const size_t shm = fill_smem_bytes(nbmax);
      if (shm > 48 * 1024)
        chk(cudaFuncSetAttribute(bfill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      bfill_kernel<<<dim3(nbt, kBThreads / kFillThreads), kFillThreads, shm, s>>>(
          h->d_inst, h->d_btile_inst, h->d_bseg_base, h->d_bwstart, h->row_ptr, h->col, h->d_bcol,
          h->d_bslot, nbmax);
      chk(cudaGetLastError());
      chk(cudaStreamSynchronize(s));
    }
  } else {
    chk(stage_h2d(h->d_inst, h->inst.data(), h->n_inst * sizeof(InstDesc), s));
    chk(cudaStreamSynchronize(s));
  }
  if (e != cudaSuccess) {
    free_blocked(h);
    return cuda_error(e, "blocked format: build");
  }
  return CB_OK;
}

CB_DEBUG_READER(blocked)

}  // namespace cb
