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
// from the CSR (one count pass, a host prefix over segment lengths, one
// fill pass), once per upload.
#include <algorithm>
#include <cstdlib>

#include "cb_internal.cuh"

namespace cb {

namespace {

__global__ void __launch_bounds__(kBThreads) bcount_kernel(const InstDesc *inst,
                                                           const uint32_t *btile_inst,
                                                           const uint64_t *bseg_base,
                                                           const uint32_t *row_ptr,
                                                           const uint32_t *col, uint32_t *bwlen,
                                                           uint32_t *unsorted) {
  const uint32_t t = blockIdx.x;
  const InstDesc I = inst[btile_inst[t]];
  const uint32_t *rp = row_ptr + I.rp_base;
  const uint32_t *cl = col + I.edge_base;
  const uint32_t row0 = (t - I.btile_base) * kBTileRows;
  uint32_t len[kBMaxBlocks];
  for (uint32_t b = 0; b < kBMaxBlocks; ++b) len[b] = 0;
  for (int k = 0; k < kBRowsPerThread; ++k) {
    const uint32_t row = row0 + threadIdx.x + kBThreads * k;
    if (row >= I.n) break;
    const uint32_t e0 = rp[row], e1 = rp[row + 1];
    if (e1 - e0 > kBLongDeg) continue;
    for (uint32_t e = e0; e < e1; ++e) {
      const uint32_t b = cl[e] >> kBColBits;
      if (b < I.nb) len[b]++;  // columns >= n are invalid input: skipped
      if (e > e0 && cl[e] < cl[e - 1]) *unsorted = 1u;  // the fill needs sorted rows
    }
  }
  for (uint32_t b = 0; b < I.nb; ++b) {
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, len[b]);
    if ((threadIdx.x & 31) == 0)
      bwlen[(bseg_base[t] + b) * 32 + (threadIdx.x >> 5)] = (wmax + 3) & ~3u;
  }
}

// Fill the streams one column block at a time: each row keeps a cursor into
// its (column-sorted) CSR row, so block b's edges of a row are the ones
// under the cursor, and all writes of block b land in this warp's region.
__global__ void __launch_bounds__(kBThreads) bfill_kernel(const InstDesc *inst,
                                                          const uint32_t *btile_inst,
                                                          const uint64_t *bseg_base,
                                                          const uint64_t *bwstart,
                                                          const uint32_t *row_ptr,
                                                          const uint32_t *col, uint16_t *bcol,
                                                          uint8_t *bslot) {
  const uint32_t t = blockIdx.x;
  const InstDesc I = inst[btile_inst[t]];
  const uint32_t *rp = row_ptr + I.rp_base;
  const uint32_t *cl = col + I.edge_base;
  const uint32_t row0 = (t - I.btile_base) * kBTileRows;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t cur[kBRowsPerThread], end[kBRowsPerThread];
#pragma unroll
  for (int k = 0; k < kBRowsPerThread; ++k) {
    const uint32_t row = row0 + threadIdx.x + kBThreads * k;
    cur[k] = end[k] = 0;
    if (row < I.n) {
      const uint32_t e0 = rp[row], e1 = rp[row + 1];
      if (e1 - e0 <= kBLongDeg) {
        cur[k] = e0;
        end[k] = e1;
      }
    }
  }
  // Elements are collected 4 at a time in registers (the lane's stripe) and
  // written with one 8-byte and one 4-byte store; unfilled positions of the
  // last stripe keep the padding values.
  constexpr uint32_t kPad2 = kBPadCol | (kBPadCol << 16);
  for (uint32_t b = 0; b < I.nb; ++b) {
    const uint64_t start = bwstart[(bseg_base[t] + b) * 32 + warp];
    uint2 *dc = reinterpret_cast<uint2 *>(bcol + start) + lane;  // stripe s at dc[32 s]
    uint32_t *dk = reinterpret_cast<uint32_t *>(bslot + start) + lane;
    uint32_t q = 0;
    uint2 cv = make_uint2(kPad2, kPad2);
    uint32_t sv = 0;
#pragma unroll
    for (int k = 0; k < kBRowsPerThread; ++k) {
      while (cur[k] < end[k]) {
        const uint32_t c = __ldg(cl + cur[k]);
        const uint32_t cb = c >> kBColBits;
        if (cb > b) break;  // the row's next edges belong to a later block
        if (cb == b) {
          const uint32_t p = q & 3, sh = 16 * (p & 1);
          const uint32_t v = c & (kBCol - 1);
          if (p < 2) cv.x = (cv.x & ~(0xffffu << sh)) | (v << sh);
          else cv.y = (cv.y & ~(0xffffu << sh)) | (v << sh);
          sv |= (uint32_t)k << (8 * p);
          if (p == 3) {
            dc[32 * (q >> 2)] = cv;
            dk[32 * (q >> 2)] = sv;
            cv = make_uint2(kPad2, kPad2);
            sv = 0;
          }
          ++q;
        }
        ++cur[k];
      }
    }
    if (q & 3) {
      dc[32 * (q >> 2)] = cv;
      dk[32 * (q >> 2)] = sv;
    }
  }
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
  dev_free(h->d_bcol);
  dev_free(h->d_bslot);
  dev_free(h->d_blong_ptr);
  dev_free(h->d_blong_rows);
  h->d_btile_inst = nullptr;
  h->d_bseg_base = h->d_bwstart = nullptr;
  h->d_bwlen = nullptr;
  h->d_bcol = nullptr;
  h->d_bslot = nullptr;
  h->d_blong_ptr = h->d_blong_rows = nullptr;
  h->total_btiles = 0;
  h->total_bseg = 0;
}

int build_blocked(cb_graph *h, const std::vector<const uint32_t *> &rp_host, cudaStream_t s) {
  if (std::getenv("CB_NO_BLOCKED")) return CB_OK;
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
    if (I.n > kBMaxBlocks * kBCol) return;
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
    I.blocked = I.n <= kBMaxBlocks * kBCol ? 1u : 0u;
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
    chk(dalloc(&h->d_bwstart, nw));
    chk(dalloc(&h->d_bwlen, nw));
    chk(dalloc(&h->d_blong_ptr, long_ptr.size()));
    chk(dalloc(&h->d_blong_rows, std::max<size_t>(long_rows.size(), 1)));
    if (e != cudaSuccess) {
      free_blocked(h);
      return cuda_error(e, "blocked format: allocate");
    }
    chk(cudaMemcpyAsync(h->d_btile_inst, btile_inst.data(), nbt * 4, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(h->d_bseg_base, bseg_base.data(), nbt * 8, cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(h->d_blong_ptr, long_ptr.data(), long_ptr.size() * 4, cudaMemcpyHostToDevice, s));
    if (!long_rows.empty())
      chk(cudaMemcpyAsync(h->d_blong_rows, long_rows.data(), long_rows.size() * 4,
                          cudaMemcpyHostToDevice, s));
    chk(cudaMemcpyAsync(h->d_inst, h->inst.data(), h->n_inst * sizeof(InstDesc),
                        cudaMemcpyHostToDevice, s));
    uint32_t *d_unsorted = nullptr;
    chk(dalloc(&d_unsorted, 1));
    if (e == cudaSuccess) chk(cudaMemsetAsync(d_unsorted, 0, 4, s));
    bcount_kernel<<<nbt, kBThreads, 0, s>>>(h->d_inst, h->d_btile_inst, h->d_bseg_base, h->row_ptr,
                                            h->col, h->d_bwlen, d_unsorted);
    chk(cudaGetLastError());
    std::vector<uint32_t> len(nw);
    uint32_t unsorted = 0;
    chk(cudaMemcpyAsync(len.data(), h->d_bwlen, nw * 4, cudaMemcpyDeviceToHost, s));
    chk(cudaMemcpyAsync(&unsorted, d_unsorted, 4, cudaMemcpyDeviceToHost, s));
    chk(cudaStreamSynchronize(s));
    dev_free(d_unsorted);
    if (e == cudaSuccess && unsorted) {
      free_blocked(h);
      return set_error(CB_ERR_ARG, "cb_graph_upload: column indices of every row must be sorted ascending");
    }
    std::vector<uint64_t> start(nw);
    uint64_t tot = 0;
    for (uint64_t q = 0; q < nw; ++q) {
      start[q] = tot;
      tot += 32ull * len[q];
    }
    const uint64_t alloc = tot + 16;
    chk(dalloc(&h->d_bcol, alloc));
    chk(dalloc(&h->d_bslot, alloc));
    if (e == cudaSuccess) {
      static_assert((kBPadCol >> 8) == (kBPadCol & 0xff), "padding column must be a repeated byte");
      chk(cudaMemsetAsync(h->d_bcol, (int)(kBPadCol & 0xff), alloc * 2, s));  // padding: zero word
      chk(cudaMemsetAsync(h->d_bslot, 0, alloc, s));                          // into slot 0
      chk(cudaMemcpyAsync(h->d_bwstart, start.data(), nw * 8, cudaMemcpyHostToDevice, s));
      bfill_kernel<<<nbt, kBThreads, 0, s>>>(h->d_inst, h->d_btile_inst, h->d_bseg_base,
                                             h->d_bwstart, h->row_ptr, h->col, h->d_bcol,
                                             h->d_bslot);
      chk(cudaGetLastError());
      chk(cudaStreamSynchronize(s));
    }
  } else {
    chk(cudaMemcpyAsync(h->d_inst, h->inst.data(), h->n_inst * sizeof(InstDesc),
                        cudaMemcpyHostToDevice, s));
    chk(cudaStreamSynchronize(s));
  }
  if (e != cudaSuccess) {
    free_blocked(h);
    return cuda_error(e, "blocked format: build");
  }
  return CB_OK;
}

}  // namespace cb
