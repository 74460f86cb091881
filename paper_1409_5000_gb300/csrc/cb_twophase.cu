// Two-phase (propagation-blocked) Lanczos SpMV step for large graphs (FP32).
//
// The Krylov evaluation of e^A 1 (section "Identification algorithm") costs
// one product u = A v_j per Lanczos step.  When a realisation's vector is
// too long for the column-blocked kernel (n > 32 column blocks of 16384),
// every gather of v_j from the CSR is a random 4-byte load from L2: one
// 32-byte sector request each, about one per clock per SM.  This step moves
// every random access into shared memory, at the price of one extra pass of
// edge values through memory (propagation blocking):
//
//   * columns are cut into source tiles of kPSrc nodes, rows into bins: runs
//     of rows whose entries, with chunk padding, fit a region of kPRegion
//     slots; rows heavier than kHeavyDeg stay out of the bins;
//   * the value array X holds one region per bin, in bin order; region t is
//     the chunks (s, t), s = 0..S-1, each holding the entries of bin t whose
//     column lies in tile s, padded to whole groups of kPGroup slots (one
//     32-byte sector);
//   * phase 1 (pscatter_kernel) stages tile s of W_j in shared memory with
//     one bulk copy, then walks the tile's stream -- its chunks for all bins,
//     in bin order -- a group at a time: 8 u16 source offsets and the
//     group's place in X in, 8 gathers from shared memory, and two float4
//     stores that fill one sector of X exactly;
//   * phase 2 (pgather_kernel, one bin per CTA) brings its bin's region and
//     the head of the bin's plan into shared memory with two bulk copies and
//     sums the rows from there: rows are cut into pieces of at most kPPiece
//     entries, the pieces sorted by length and dealt 32 at a time (one per
//     lane) into slices, so a lane walks its piece's region slots with no
//     branch and no search; each row then adds its pieces in order and takes
//     the same row epilogue and alpha partial as the other kernels.  Heavy
//     rows are summed in chunks from the CSR as in the tiled-CSR kernel.
//
// DRAM bytes per entry: 2 (source offset) + 0.5 (group place) + 4 (value
// write) in phase 1, 4 (value read) + ~2.1 (slot, with the slices' padding)
// in phase 2, plus the chunk padding, against the 4 of one u32 column index;
// in exchange every access is sequential or a whole sector, and every random
// one hits shared memory.
//
// The format is built on the device at upload: a count pass per bin (chunk
// sizes, region offsets), a prefix over the bins' region sizes, a pass per
// source tile (chunk offsets within the tile's stream), a fill pass per bin
// that gives every entry a slot and every stream group its place, and a pass
// per bin that builds its phase-2 plan.  The slot of an entry inside its
// chunk comes from a shared-memory atomic, so the layout may differ between
// uploads, but the sums cannot: phase 2 adds each piece's entries in CSR
// order and each row's pieces in order, wherever the entries sit.
#include <algorithm>

#include "cb_internal.cuh"
#include "cb_reduce.cuh"
#include "cb_step.cuh"

namespace cb {

namespace {

constexpr int kBuildThreads = 512;

// Exclusive prefix of v over the CTA (threads in order); *total gets the
// sum.  s_w holds >= 33 words.  All threads must call it.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_w, uint32_t *total) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t nw = (blockDim.x + 31) >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (uint32_t)o) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < nw ? s_w[lane] : 0u;
    uint32_t y = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= (uint32_t)o) y += z;
    }
    s_w[lane] = y - w;
    if (lane == 31) s_w[32] = y;
  }
  __syncthreads();
  const uint32_t r = s_w[warp] + x - v;
  *total = s_w[32];
  __syncthreads();
  return r;
}

// Per bin: the chunk sizes by source tile (shared-memory histogram), padded
// to whole groups, and their exclusive prefix over s: roff[bin][s] is the
// group offset of chunk (s, bin) in the bin's region, roff[bin][S] and
// rtot[bin] the region's groups.  A column >= n sets *bad (the upload then
// fails).
__global__ void __launch_bounds__(kBuildThreads) pcount_kernel(const InstDesc *inst, const PBin *bins,
                                                               const uint32_t *row_ptr,
                                                               const uint32_t *col, uint32_t *roff,
                                                               uint32_t *rtot, uint32_t *bad) {
  extern __shared__ uint32_t s_hist[];  // pns_max
  __shared__ uint32_t s_w[33];
  const PBin B = bins[blockIdx.x];
  const InstDesc I = inst[B.inst];
  const uint32_t S = I.pns;
  for (uint32_t q = threadIdx.x; q < S; q += blockDim.x) s_hist[q] = 0u;
  __syncthreads();
  const uint32_t *rp = row_ptr + I.rp_base;
  const uint32_t *cl = col + I.edge_base;
  const uint32_t e0 = rp[B.row0], e1 = rp[B.row1];
  bool oob = false;
  for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const uint32_t c = cl[e];
    if (c >= I.n) {
      oob = true;
      continue;
    }
    atomicAdd(&s_hist[c >> kPSrcBits], 1u);
  }
  if (oob) *bad = 1u;
  __syncthreads();
  // each thread owns a contiguous range of source tiles
  const uint32_t per = (S + blockDim.x - 1) / blockDim.x;
  const uint32_t s0 = min(S, threadIdx.x * per), s1 = min(S, s0 + per);
  uint32_t mine = 0;
  for (uint32_t q = s0; q < s1; ++q) mine += (s_hist[q] + kPGroup - 1) / kPGroup;
  uint32_t total;
  uint32_t run = block_excl_scan(mine, s_w, &total);
  uint32_t *ro = roff + I.pmat_base + (uint64_t)(blockIdx.x - I.pbin_base) * (S + 1);
  for (uint32_t q = s0; q < s1; ++q) {
    ro[q] = run;
    run += (s_hist[q] + kPGroup - 1) / kPGroup;
  }
  if (threadIdx.x == 0) {
    ro[S] = total;
    rtot[blockIdx.x] = total;
  }
}

// Per source tile s: cstart[bin][s], the group offset of chunk (s, bin) in
// the tile's stream (exclusive prefix over the realisation's bins), and the
// tile's total groups.
__global__ void __launch_bounds__(kBuildThreads) pcolscan_kernel(const InstDesc *inst,
                                                                 const uint32_t *ptile_inst,
                                                                 const uint32_t *roff,
                                                                 uint32_t *cstart, uint32_t *ptotal) {
  __shared__ uint32_t s_w[33];
  const uint32_t g = blockIdx.x;
  const InstDesc I = inst[ptile_inst[g]];
  const uint32_t S = I.pns, s = g - I.ptile_base;
  const uint32_t *ro = roff + I.pmat_base;
  uint32_t *cs = cstart + I.pmat_base;
  uint32_t carry = 0;
  for (uint32_t t0 = 0; t0 < I.n_pbin; t0 += blockDim.x) {
    const uint32_t t = t0 + threadIdx.x;
    uint32_t v = 0;
    if (t < I.n_pbin) v = ro[(uint64_t)t * (S + 1) + s + 1] - ro[(uint64_t)t * (S + 1) + s];
    uint32_t total;
    const uint32_t ex = block_excl_scan(v, s_w, &total);
    if (t < I.n_pbin) cs[(uint64_t)t * (S + 1) + s] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) ptotal[g] = carry;
}

// Per bin: every entry gets the next free slot of its chunk (a shared-memory
// counter per source tile): pos[e] is the slot's place in the bin region and
// psrc[stream slot] the entry's column within its tile; every stream group of
// the bin's chunks gets its group in the value array (gdst).
__global__ void __launch_bounds__(kBuildThreads) pfill_kernel(const InstDesc *inst, const PBin *bins,
                                                              const uint32_t *row_ptr,
                                                              const uint32_t *col,
                                                              const uint32_t *roff,
                                                              const uint32_t *cstart,
                                                              const uint64_t *ptbase,
                                                              const uint64_t *pxbase, uint16_t *ppos,
                                                              uint16_t *psrc, uint32_t *pgdst) {
  extern __shared__ uint64_t s_q[];  // pns_max stream group bases, then region group bases, counters
  const PBin B = bins[blockIdx.x];
  const InstDesc I = inst[B.inst];
  const uint32_t S = I.pns;
  uint32_t *s_r = reinterpret_cast<uint32_t *>(s_q + S);
  uint32_t *s_c = s_r + S;
  const uint64_t mrow = I.pmat_base + (uint64_t)(blockIdx.x - I.pbin_base) * (S + 1);
  const uint64_t xb = pxbase[blockIdx.x];
  for (uint32_t q = threadIdx.x; q < S; q += blockDim.x) {
    const uint64_t g0 = ptbase[I.ptile_base + q] + cstart[mrow + q];
    const uint32_t r0 = roff[mrow + q], ng = roff[mrow + q + 1] - r0;
    s_q[q] = g0;
    s_r[q] = r0;
    s_c[q] = 0u;
    for (uint32_t k = 0; k < ng; ++k) pgdst[g0 + k] = (uint32_t)(xb + r0 + k);
  }
  __syncthreads();
  const uint32_t *rp = row_ptr + I.rp_base;
  const uint32_t *cl = col + I.edge_base;
  uint16_t *pos = ppos + I.edge_base;
  const uint32_t e0 = rp[B.row0], e1 = rp[B.row1];
  for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const uint32_t c = cl[e];
    if (c >= I.n) continue;  // rejected by the count pass
    const uint32_t s = c >> kPSrcBits;
    const uint32_t k = atomicAdd(&s_c[s], 1u);
    pos[e] = (uint16_t)(kPGroup * s_r[s] + k);
    psrc[kPGroup * s_q[s] + k] = (uint16_t)(c & (kPSrc - 1));
  }
}

// Per bin: the phase-2 plan (sliced rows).  Every row of the bin is cut into
// pieces of at most kPPiece entries, in entry order; the pieces, sorted by
// length (longest first, ties in piece order), are dealt 32 at a time into
// slices, one piece per lane; a slice runs as many steps as its first piece
// is long, rounded up to an even number, and a lane past its piece's end
// reads the region's zero slot.  The slices go to the warps longest first,
// each to the warp with the least work so far (ties: the lower warp).  The
// plan (u16 words, every part a multiple of 8 words) is:
//   [0, 17)      ws: warp w runs slices [ws[w], ws[w+1]) (warp-major order)
//   [24, 58)     wo: the slot-array offset of warp w's first slice (u32 as
//                two words, low first); wo[16] is the array's length
//   [64, ...)    slen[ns]: steps of each slice
//                pid[ns][32]: the piece of each lane (0xffff: none)
//                slots: per slice, [step / 2][lane] pairs of u16 region slots
//                pf[nrows + 1]: first piece of each row (pf[nrows] = pieces)
// Phase 2 copies everything before pf to shared memory; this kernel also
// writes the bin's P2Desc.  The host sized each plan from the same piece
// lengths (slice_plan_words); a size that disagrees fails the upload.
__global__ void __launch_bounds__(kP2Threads) pslice_kernel(const InstDesc *inst, const PBin *bins,
                                                            const uint32_t *row_ptr,
                                                            const uint16_t *ppos,
                                                            const uint64_t *psloff,
                                                            const uint64_t *pxbase, uint16_t *psl,
                                                            P2Desc *pdesc, uint32_t *bad) {
  constexpr uint32_t W = kP2Threads / 32;
  __shared__ uint32_t s_rp[kPBinRows + 1];           // bin-relative row offsets
  __shared__ uint16_t s_pf[kPBinRows + 2];           // first piece of each row
  __shared__ uint16_t s_prow[kPMaxPieces];           // row of each piece
  __shared__ uint8_t s_plen[kPMaxPieces];            // entries of each piece
  __shared__ uint16_t s_order[kPMaxPieces];          // sorted position -> piece
  __shared__ uint32_t s_base[kPPiece + 1], s_carry[kPPiece + 1];
  __shared__ uint32_t s_wc[W][kPPiece + 1];
  __shared__ uint16_t s_perm[kPMaxSlices], s_ulen[kPMaxSlices];
  __shared__ uint32_t s_uoff[kPMaxSlices + 1];
  __shared__ uint32_t s_ws[W + 1], s_wo[W + 1];
  __shared__ uint32_t s_w[33];
  const PBin B = bins[blockIdx.x];
  const InstDesc I = inst[B.inst];
  const uint32_t *rp = row_ptr + I.rp_base + B.row0;
  const uint32_t nrows = B.row1 - B.row0;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (uint32_t q = tid; q <= nrows; q += blockDim.x) s_rp[q] = rp[q] - rp[0];
  if (tid <= kPPiece) s_base[tid] = 0u;
  __syncthreads();
  // pieces per row and their prefix (each thread two consecutive rows)
  auto npieces = [&](uint32_t q) -> uint32_t {
    return q < nrows ? (s_rp[q + 1] - s_rp[q] + kPPiece - 1) / kPPiece : 0u;
  };
  const uint32_t n0 = npieces(2 * tid), n1 = npieces(2 * tid + 1);
  uint32_t NP;
  const uint32_t ex = block_excl_scan(n0 + n1, s_w, &NP);
  if (NP > kPMaxPieces) {  // cannot happen within the bin limits; fails the upload
    if (tid == 0) atomicExch(bad, 1u);
    return;
  }
  if (2 * tid < nrows) s_pf[2 * tid] = (uint16_t)ex;
  if (2 * tid + 1 < nrows) s_pf[2 * tid + 1] = (uint16_t)(ex + n0);
  if (tid == 0) s_pf[nrows] = (uint16_t)NP;
  __syncthreads();
  // each piece's row and length; the length histogram (key = kPPiece - len)
  for (uint32_t p = tid; p < NP; p += blockDim.x) {
    uint32_t lo = 0, hi = nrows;  // s_pf[lo] <= p < s_pf[hi]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_pf[mid] <= p) lo = mid; else hi = mid;
    }
    const uint32_t k = p - s_pf[lo], deg = s_rp[lo + 1] - s_rp[lo];
    const uint32_t len = min(kPPiece, deg - k * kPPiece);
    s_prow[p] = (uint16_t)lo;
    s_plen[p] = (uint8_t)len;
    atomicAdd(&s_base[kPPiece - len], 1u);
  }
  __syncthreads();
  if (tid == 0) {
    uint32_t run = 0;
    for (uint32_t key = 0; key <= kPPiece; ++key) {
      const uint32_t c = s_base[key];
      s_base[key] = run;
      s_carry[key] = 0u;
      run += c;
    }
  }
  // stable placement, 512 pieces at a time: the rank of a piece among the
  // equal keys of its warp, after those of the lower warps and earlier chunks
  for (uint32_t c0 = 0; c0 < NP; c0 += blockDim.x) {
    for (uint32_t q = tid; q < W * (kPPiece + 1); q += blockDim.x) (&s_wc[0][0])[q] = 0u;
    __syncthreads();
    const uint32_t p = c0 + tid;
    const uint32_t key = p < NP ? kPPiece - s_plen[p] : kPPiece;  // kPPiece: no piece
    const uint32_t peers = __match_any_sync(0xffffffffu, key);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (rank == 0) s_wc[warp][key] = __popc(peers);
    __syncthreads();
    if (p < NP) {
      uint32_t at = s_base[key] + s_carry[key] + rank;
      for (uint32_t w = 0; w < warp; ++w) at += s_wc[w][key];
      s_order[at] = (uint16_t)p;
    }
    __syncthreads();
    if (tid < kPPiece) {
      uint32_t t = 0;
      for (uint32_t w = 0; w < W; ++w) t += s_wc[w][tid];
      s_carry[tid] += t;
    }
    __syncthreads();
  }
  // slices, longest first, to the least-loaded warp; warp-major order
  const uint32_t ns = (NP + 31) / 32;
  if (tid == 0) {
    uint32_t load[W], owner[kPMaxSlices];
    for (uint32_t w = 0; w < W; ++w) load[w] = 0u;
    for (uint32_t s = 0; s < ns; ++s) {
      const uint32_t L = (s_plen[s_order[32 * s]] + 1u) & ~1u;
      uint32_t best = 0;
      for (uint32_t w = 1; w < W; ++w)
        if (load[w] < load[best]) best = w;
      owner[s] = best;
      load[best] += L;
    }
    uint32_t u = 0, off = 0;
    for (uint32_t w = 0; w < W; ++w) {
      s_ws[w] = u;
      s_wo[w] = off;
      for (uint32_t s = 0; s < ns; ++s) {
        if (owner[s] != w) continue;
        const uint32_t L = (s_plen[s_order[32 * s]] + 1u) & ~1u;
        s_perm[u] = (uint16_t)s;
        s_ulen[u] = (uint16_t)L;
        s_uoff[u] = off;
        off += 32 * L;
        ++u;
      }
    }
    s_ws[W] = u;
    s_wo[W] = off;
    s_uoff[u] = off;
  }
  __syncthreads();
  const uint32_t ns8 = (ns + 7) & ~7u, nr8 = (nrows + 1 + 7) & ~7u;
  const uint32_t head = 64 + ns8 + 32 * ns + s_wo[W];  // words copied by phase 2
  if (head + nr8 != psloff[blockIdx.x + 1] - psloff[blockIdx.x] || s_wo[W] > kPSlotsMax) {
    if (tid == 0) atomicExch(bad, 1u);
    return;
  }
  uint16_t *out = psl + psloff[blockIdx.x];
  if (tid == 0) {
    P2Desc d;
    d.xg0 = pxbase[blockIdx.x];
    d.plan = psloff[blockIdx.x];
    d.node = I.node_base + B.row0;
    d.reg_bytes = (uint32_t)(pxbase[blockIdx.x + 1] - d.xg0) * kPGroup * 4u;
    d.head_bytes = head * 2u;
    d.pf = head;
    d.inst = B.inst;
    d.nrows = nrows;
    d.slot = blockIdx.x - I.pbin_base;
    pdesc[blockIdx.x] = d;
  }
  if (tid < 64) {
    uint16_t v = 0;
    if (tid <= W) v = (uint16_t)s_ws[tid];
    else if (tid >= 24 && tid < 24 + 2 * (W + 1)) {
      const uint32_t o = s_wo[(tid - 24) >> 1];
      v = (uint16_t)((tid & 1) ? o >> 16 : o & 0xffffu);
    }
    out[tid] = v;
  }
  uint16_t *slen = out + 64, *pid = slen + ns8, *slots = pid + 32 * ns, *pf = slots + s_wo[W];
  for (uint32_t q = tid; q < ns8; q += blockDim.x) slen[q] = q < ns ? s_ulen[q] : (uint16_t)0;
  for (uint32_t q = tid; q < 32 * ns; q += blockDim.x) {
    const uint32_t at = 32 * s_perm[q >> 5] + (q & 31);
    pid[q] = at < NP ? s_order[at] : (uint16_t)0xffffu;
  }
  for (uint32_t q = tid; q < nr8; q += blockDim.x) pf[q] = q <= nrows ? s_pf[q] : (uint16_t)0;
  const uint16_t *pos = ppos + I.edge_base + rp[0];  // pos of the bin's first entry
  const uint32_t total = s_wo[W];
  for (uint32_t q = tid; q < total; q += blockDim.x) {
    uint32_t lo = 0, hi = s_ws[W];  // the slice holding word q: s_uoff[lo] <= q < s_uoff[hi]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_uoff[mid] <= q) lo = mid; else hi = mid;
    }
    const uint32_t local = q - s_uoff[lo];
    const uint32_t l = (local >> 1) & 31u, t = 2 * (local >> 6) + (local & 1u);
    const uint32_t at = 32 * s_perm[lo] + l;
    uint16_t v = (uint16_t)kPRegion;  // the zero slot
    if (at < NP) {
      const uint32_t p = s_order[at];
      if (t < s_plen[p]) {
        const uint32_t row = s_prow[p];
        v = pos[s_rp[row] + (p - s_pf[row]) * kPPiece + t];
      }
    }
    slots[q] = v;
  }
}

// ---------------------------------------------------------------------------
// Phase 1: persistent CTAs (one per SM), each an equal share of the stream's
// groups.  The source tile is restaged only where the share crosses into the
// next tile's stream; the share's source offsets and group places stream
// through shared memory in blocks of kP1Block groups (bulk copies into
// kP1Bufs buffers).  There is no CTA barrier per block: each warp waits for
// the block it needs on that buffer's mbarrier, and the last warp done with
// a buffer refills it, so warps drift apart by up to kP1Bufs - 1 blocks.
// The threads' only global accesses are the sector-filling value stores.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t umin64(uint64_t x, uint64_t y) { return x < y ? x : y; }

constexpr uint32_t kP1Block = 1024;  // groups per streamed block (32 per warp)
constexpr uint32_t kP1Bufs = 3;
constexpr uint32_t kP1Warps = kP1Threads / 32;
static_assert(kP1Block == 32 * kP1Warps, "32 groups per warp per block");
constexpr size_t kP1TileBytes = (size_t)kPSrc * sizeof(float);
constexpr size_t kP1SrcBytes = (size_t)kP1Block * 16;  // 8 u16 per group
constexpr size_t kP1DstBytes = (size_t)kP1Block * 4;   // one u32 per group
constexpr size_t kP1SmemBytes = kP1TileBytes + kP1Bufs * (kP1SrcBytes + kP1DstBytes);

__global__ void __launch_bounds__(kP1Threads, 1) pscatter_kernel(LArgs a, uint32_t j, uint32_t tile_lo,
                                                                 uint32_t tile_hi, uint64_t g_lo,
                                                                 uint64_t g_hi) {
  extern __shared__ float4 s_dyn4[];
  float *vt = reinterpret_cast<float *>(s_dyn4);  // the current source tile of W_j
  uint4 *sbuf = reinterpret_cast<uint4 *>(vt + kPSrc);                       // [kP1Bufs][kP1Block]
  uint32_t *dbuf = reinterpret_cast<uint32_t *>(sbuf + kP1Bufs * kP1Block);  // [kP1Bufs][kP1Block]
  __shared__ __align__(8) uint64_t s_tbar, s_bbar[kP1Bufs];
  __shared__ uint32_t s_tile, s_issued[kP1Bufs], s_used[kP1Bufs];
  __shared__ int s_go, s_fail;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t span = g_hi - g_lo;
  uint64_t gb = g_lo + span * blockIdx.x / gridDim.x;
  const uint64_t ge = g_lo + span * (blockIdx.x + 1) / gridDim.x;
  if (gb >= ge) return;
  if (tid == 0) {
    // the tile whose stream holds group gb: the last t with ptbase[t] <= gb
    uint32_t lo = tile_lo, hi = tile_hi;  // ptbase[lo] <= gb < ptbase[hi]
    while (hi - lo > 1) {
      const uint32_t mid = lo + (hi - lo) / 2;
      if (a.ptbase[mid] <= gb) lo = mid; else hi = mid;
    }
    s_tile = lo;
    s_fail = 0;
    mbar_init(&s_tbar, 1);
    for (uint32_t q = 0; q < kP1Bufs; ++q) {
      mbar_init(&s_bbar[q], 1);
      s_issued[q] = 0;
      s_used[q] = 0;
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t t = s_tile, tpar = 0, blk = 0;  // blk: blocks streamed before this segment
  bool staged = false;                      // a tile copy was issued (its phase: tpar ^ 1)
  float4 *X = reinterpret_cast<float4 *>(a.pX);  // 2 float4 per group
  // block q (absolute block number bq) of a segment: groups [w, w + len)
  auto issue = [&](uint64_t w, uint32_t len, uint32_t bq) {
    const uint32_t b = bq % kP1Bufs;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&s_bbar[b], len * 20u);
    bulk_g2s(sbuf + b * kP1Block, a.psrc + kPGroup * w, len * 16u, &s_bbar[b]);
    bulk_g2s(dbuf + b * kP1Block, a.pgdst + w, len * 4u, &s_bbar[b]);
    s_issued[b] += 1;
  };
  while (gb < ge) {
    const uint64_t se = umin64(ge, a.ptbase[t + 1]);
    if (se > gb) {
      const uint32_t r = a.ptile_inst[t];
      const InstDesc &I = a.inst[r];
      // blocks start at a multiple of 4 groups (16-byte aligned places) and
      // cover whole multiples of 4; groups outside [gb, se) are skipped
      const uint64_t w0 = gb & ~3ull, wend = (se + 3) & ~3ull;
      const uint32_t nblk = (uint32_t)((wend - w0 + kP1Block - 1) / kP1Block);
      if (tid == 0) {
        s_go = j < a.sc.meff[r];  // the realisation is still running (one reading for the CTA)
        if (s_go) {
          const float *x = reinterpret_cast<const float *>(a.V) + (uint64_t)j * a.vs + I.node_base;
          const uint32_t node0 = (t - I.ptile_base) << kPSrcBits;
          const uint32_t nn = min(kPSrc, I.n - node0);
          // whole 16-byte units: up to 3 floats past node n-1, inside the padded vector
          const uint32_t bytes = ((nn + 3u) & ~3u) * 4u;
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          mbar_expect_tx(&s_tbar, bytes);
          bulk_g2s(vt, x + node0, bytes, &s_tbar);
          for (uint32_t q = 0; q < kP1Bufs && q < nblk; ++q)
            issue(w0 + (uint64_t)q * kP1Block, (uint32_t)umin64(kP1Block, wend - w0 - (uint64_t)q * kP1Block),
                  blk + q);
        }
      }
      __syncthreads();
      const bool go = s_go != 0;
      __syncthreads();  // s_go is rewritten for the next segment
      if (go) {
        bool fail = !__all_sync(0xffffffffu, mbar_wait(&s_tbar, tpar));
        tpar ^= 1u;
        staged = true;
        for (uint32_t q = 0; q < nblk && !fail; ++q) {
          const uint32_t bq = blk + q, b = bq % kP1Bufs;
          if (!__all_sync(0xffffffffu, mbar_wait(&s_bbar[b], (bq / kP1Bufs) & 1u))) {
            fail = true;
            break;
          }
          const uint64_t wq = w0 + (uint64_t)q * kP1Block;
          // this warp's 32 groups, two lanes per group, one half (4 slots,
          // 16 bytes) each: a store instruction fills 16 groups' sectors,
          // contiguous within a chunk
          const uint2 *sb2 = reinterpret_cast<const uint2 *>(sbuf + b * kP1Block);
#pragma unroll
          for (uint32_t h = 0; h < 2; ++h) {
            const uint32_t gi = warp * 32 + h * 16 + (lane >> 1), half = lane & 1u;
            const uint64_t g = wq + gi;
            if (g >= gb && g < se) {
              const uint2 sv = sb2[2 * gi + half];
              const uint32_t d = dbuf[b * kP1Block + gi];
#ifdef CB_DEBUG
              const uint32_t nn = min(kPSrc, I.n - ((t - I.ptile_base) << kPSrcBits));
              const uint32_t smax = max(max(sv.x & 0xffffu, sv.x >> 16), max(sv.y & 0xffffu, sv.y >> 16));
              if (!CB_DCHECK(smax < nn, kDbgTwoPhaseSrc, smax) ||
                  !CB_DCHECK(d < a.pgroups, kDbgTwoPhaseDst, d))
                continue;
#endif
              float4 o;
              o.x = vt[sv.x & 0xffffu];
              o.y = vt[sv.x >> 16];
              o.z = vt[sv.y & 0xffffu];
              o.w = vt[sv.y >> 16];
              __stcs(X + 2ull * d + half, o);  // read back by phase 2 only, much later
            }
          }
          // this warp is done with buffer b; the last warp refills it
          __syncwarp();
          if (lane == 0) {
            __threadfence_block();
            if (atomicAdd(&s_used[b], 1u) == kP1Warps - 1) {
              s_used[b] = 0;
              if (q + kP1Bufs < nblk) {
                __threadfence_block();
                const uint64_t wn = w0 + (uint64_t)(q + kP1Bufs) * kP1Block;
                issue(wn, (uint32_t)umin64(kP1Block, wend - wn), bq + kP1Bufs);
              }
            }
          }
        }
        if (fail && lane == 0) s_fail = 1;
        blk += nblk;
        __syncthreads();  // every warp is done with this tile before the next copy
        if (s_fail) break;
      }
    }
    gb = se;
    ++t;
  }
  __syncthreads();
  if (tid == 0) {
    if (s_fail) {  // a copy never landed: this step of the realisation fails
      const uint32_t r = a.ptile_inst[min(t, tile_hi - 1)];
      a.sc.status[r] = CB_ERR_TIMEOUT;
      a.sc.meff[r] = j;
    }
    // every copy issued has landed before the CTA ends (bounded)
    for (uint32_t q = 0; q < kP1Bufs; ++q)
      if (s_issued[q]) mbar_wait(&s_bbar[q], (s_issued[q] - 1) & 1u);
    if (staged) mbar_wait(&s_tbar, tpar ^ 1u);
  }
}

// ---------------------------------------------------------------------------
// Phase 2: one bin per CTA, after the heavy-row chunk CTAs; two CTAs per SM,
// so one CTA's copies overlap the other's sums.  Everything the CTA needs
// to start comes from the bin's P2Desc (one load): thread 0 issues the bulk
// copies of the region and of the head of the plan on one mbarrier, and
// every thread loads its rows' epilogue operands while they are in flight.
// Each warp then runs its slices (see pslice_kernel): a lane sums its
// piece's entries in entry order from the region, gathering at the slots the
// plan lists, and stores the piece sum; after a CTA barrier each thread adds
// its rows' pieces in order and applies the row epilogue (coalesced stores),
// and the last warp to finish adds the warp partials in warp order and
// enters the bin's alpha term.
// ---------------------------------------------------------------------------
constexpr uint32_t kP2Warps = kP2Threads / 32;
// the region (+ 4 floats: the zero slot), the copied head of the plan
// (header, slice lengths, lane pieces, slots) and the piece sums, each a
// whole number of 16-byte units (the first two are bulk-copy targets)
constexpr uint32_t kP2RegionWords = kPRegion + 4;
constexpr uint32_t kP2PlanWords = 64 + 64 + 32 * kPMaxSlices + kPSlotsMax;
static_assert((kP2RegionWords * 4) % 16 == 0 && (kP2PlanWords * 2) % 16 == 0 &&
                  (kPMaxPieces * 4) % 16 == 0 && kPMaxSlices <= 64,
              "phase-2 shared-memory buffers must keep 16-byte alignment");
constexpr size_t kP2SmemBytes = (size_t)kP2RegionWords * sizeof(float) + kP2PlanWords * sizeof(uint16_t) +
                                kPMaxPieces * sizeof(float);
// two CTAs per SM: 228 KB per SM, 1 KB reserved per CTA, < 640 B of static
// shared memory (ptxas -v reports it)
static_assert(2 * (kP2SmemBytes + 1024 + 640) <= 228 * 1024, "two phase-2 CTAs per SM");
static_assert(kPBinRows <= 2 * kP2Threads, "each phase-2 thread owns at most two rows");

__global__ void __launch_bounds__(kP2Threads, 2) pgather_kernel(LArgs a, uint32_t j, uint32_t chunk_off,
                                                                uint32_t n_chunks, uint32_t bin_off,
                                                                uint32_t n_bins, uint32_t ahead) {
  extern __shared__ float4 s_dyn4[];
  float *reg = reinterpret_cast<float *>(s_dyn4);                         // the bin region
  uint16_t *s_plan = reinterpret_cast<uint16_t *>(reg + kP2RegionWords);  // the plan's head
  float *s_psum = reinterpret_cast<float *>(s_plan + kP2PlanWords);       // piece sums
  __shared__ double s_wpart[kP2Warps];
  __shared__ __align__(8) uint64_t s_full;
  __shared__ uint32_t s_done;
  __shared__ int s_fail;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (blockIdx.x < n_chunks) {  // one chunk of a heavy row of a two-phase realisation
    const uint32_t cidx = chunk_off + blockIdx.x;
    const uint32_t hid = a.chunk_heavy[cidx];
    const uint32_t r = a.heavy[hid].inst;
    if (j >= a.sc.meff[r] || !a.inst[r].pb) return;
    const InstDesc &I = a.inst[r];
    heavy_chunk<float, true>(a, j, cidx, hid, r, I.pspmv, I.n_pbin + (hid - I.heavy_base));
    return;
  }
  const uint32_t bin = bin_off + (blockIdx.x - n_chunks);
  const P2Desc D = a.pdesc[bin];
  const uint32_t r = D.inst, nrows = D.nrows;
  if (j >= a.sc.meff[r]) return;  // realisation stopped (uniform per CTA)
  if (tid == 0) {
    s_done = 0;
    s_fail = 0;
    reg[kPRegion] = 0.f;  // the zero slot (outside the copied region)
    mbar_init(&s_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (D.reg_bytes <= kPRegion * 4u && D.head_bytes <= kP2PlanWords * 2u) {
      mbar_expect_tx(&s_full, D.reg_bytes + D.head_bytes);
      if (D.reg_bytes) bulk_g2s(reg, a.pX + D.xg0 * kPGroup, D.reg_bytes, &s_full);
      bulk_g2s(s_plan, a.psl + D.plan, D.head_bytes, &s_full);
    } else {  // cannot happen with a plan the upload built: no copy, the step fails
      s_fail = 1;
      mbar_expect_tx(&s_full, 0);
    }
    // the bin `ahead` places on (about one wave of CTAs later) into L2, so
    // that DRAM keeps streaming while the resident CTAs sum
    const uint32_t nb = bin + ahead;
    if (nb < bin_off + n_bins) {
      const P2Desc N = a.pdesc[nb];
      if (N.reg_bytes <= kPRegion * 4u && N.head_bytes <= kP2PlanWords * 2u) {
        if (N.reg_bytes) l2_prefetch(a.pX + N.xg0 * kPGroup, N.reg_bytes);
        l2_prefetch(a.psl + N.plan, N.head_bytes);
      }
    }
  }
  // this thread's rows' epilogue operands, while the copies are in flight
  float *Vb = reinterpret_cast<float *>(a.V);
  const bool has_prev = j > 0;
  const float *x = Vb + (uint64_t)j * a.vs + D.node;  // W_j of the bin's rows
  const uint16_t *pf = a.psl + D.plan + D.pf;         // first piece of each row
  const uint32_t ms = a.sc.ms;
  const float sj = (float)a.sc.scale[r * ms + j];
  const float bp = has_prev ? (float)(a.sc.beta[r * ms + j - 1] * a.sc.scale[r * ms + j - 1]) : 0.f;
  float xv[2] = {0.f, 0.f}, xpv[2] = {0.f, 0.f};
  uint32_t pb[2] = {0u, 0u}, pe[2] = {0u, 0u};
#pragma unroll
  for (uint32_t h = 0; h < 2; ++h) {
    const uint32_t lr = tid + h * kP2Threads;
    if (lr < nrows) {
      xv[h] = x[lr];
      if (has_prev) xpv[h] = (x - a.vs)[lr];
      pb[h] = pf[lr];
      pe[h] = pf[lr + 1];
    }
  }
  if (tid == 0 && (!mbar_wait(&s_full, 0) || s_fail)) s_fail = 1;
  __syncthreads();  // the bin has landed (or the wait gave up)
  const bool ok = s_fail == 0;
  double wpart = 0.0;
  if (ok) {
    const uint32_t ns = s_plan[kP2Warps];
    const uint32_t u0 = s_plan[warp], u1 = s_plan[warp + 1];
    uint32_t soff = ((uint32_t)s_plan[24 + 2 * warp] | ((uint32_t)s_plan[25 + 2 * warp] << 16)) >> 1;
    const uint16_t *slen = s_plan + 64;
    const uint16_t *pid = slen + ((ns + 7) & ~7u);
    const uint32_t *slots = reinterpret_cast<const uint32_t *>(pid + 32 * ns);  // slot pairs
#ifdef CB_DEBUG
    const uint32_t rslots = D.reg_bytes / 4u;
    const uint32_t npieces = pf[nrows];
#endif
    for (uint32_t u = u0; u < u1; ++u) {
      const uint32_t L = slen[u];  // steps of the slice: even, at most kPPiece
      const uint32_t p = pid[32 * u + lane];
      const uint32_t *sp = slots + soff + lane;
      float acc = 0.f;
#pragma unroll
      for (uint32_t k = 0; k < kPPiece / 2; ++k) {
        if (2 * k < L) {  // uniform over the warp
          const uint32_t q = sp[32 * k];
#ifdef CB_DEBUG
          const uint32_t lo = q & 0xffffu, hi = q >> 16;
          if (!CB_DCHECK((lo < rslots || lo == kPRegion) && (hi < rslots || hi == kPRegion),
                         kDbgTwoPhasePos, max(lo, hi)))
            continue;
#endif
          acc += reg[q & 0xffffu];
          acc += reg[q >> 16];
        }
      }
      if (p != 0xffffu && CB_DCHECK(p < npieces, kDbgTwoPhasePos, p)) s_psum[p] = acc;
      soff += 16 * L;
    }
  }
  __syncthreads();  // every piece sum is in shared memory
  if (ok) {
    // rows: the sum of their pieces in order; u = sj * sum - bp * W_{j-1}[row]
    // (coalesced store), and the alpha partial W_j[row] * u
    float *out = Vb + (uint64_t)(j + 1) * a.vs + D.node;
    float acc = 0.f;
#pragma unroll
    for (uint32_t h = 0; h < 2; ++h) {
      const uint32_t lr = tid + h * kP2Threads;
      if (lr < nrows) {
        float sum = 0.f;
        for (uint32_t p = pb[h]; p < pe[h]; ++p) sum += s_psum[p];
        float v = sj * sum;
        if (has_prev) v -= bp * xpv[h];
        out[lr] = v;
        acc += xv[h] * v;
      }
    }
    wpart = (double)warp_sum<float>(acc);
  }
  // the last warp to finish sums the warp partials in warp order
  uint32_t last = 0;
  if (lane == 0) {
    s_wpart[warp] = wpart;
    __threadfence_block();
    last = atomicAdd(&s_done, 1u) == kP2Warps - 1;
  }
  if (!__shfl_sync(0xffffffffu, last, 0)) return;
  __threadfence_block();
  double part = 0.0;
  if (lane == 0) {
    for (uint32_t w = 0; w < kP2Warps; ++w) part += s_wpart[w];
    if (!ok) {  // the bin never landed: this step of the realisation fails
      a.sc.status[r] = CB_ERR_TIMEOUT;
      part = __longlong_as_double(0x7ff8000000000000ll);
      mbar_wait(&s_full, 0);  // the copies in flight complete (bounded) before the CTA ends
    }
  }
  part = __shfl_sync(0xffffffffu, part, 0);
  double total;
  if (warp_arrive_and_reduce(a.inst[r].pspmv, D.slot, r, part, a.red, &total) && lane == 0)
    finish_alpha<float>(a, r, j, total);
}

void launch_p2(const LArgs &a, uint32_t j, uint32_t chunk_off, uint32_t n_chunks, uint32_t bin_off,
               uint32_t n_bins, int n_sm, cudaStream_t s) {
  static bool attr = false;  // opt-in to > 48 KB of shared memory
  if (!attr) {
    cudaFuncSetAttribute(pgather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kP2SmemBytes);
    cudaFuncSetAttribute(pgather_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    attr = true;
  }
  // prefetch distance: the CTAs resident at once (two per SM)
  pgather_kernel<<<n_chunks + n_bins, kP2Threads, kP2SmemBytes, s>>>(a, j, chunk_off, n_chunks, bin_off,
                                                                     n_bins, 2u * (uint32_t)n_sm);
}

template <typename P>
cudaError_t dalloc(P **p, size_t count) {
  return dev_alloc_n(p, count);
}

}  // namespace

void launch_twophase(const LArgs &a, int lanes, uint32_t j, uint32_t tile_lo, uint32_t tile_hi,
                     uint64_t g_lo, uint64_t g_hi, uint32_t chunk_off, uint32_t n_chunks,
                     uint32_t bin_off, uint32_t n_bins, cudaStream_t s) {
  static int n_sm = 0;
  if (!n_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (n_sm <= 0) n_sm = 1;
    cudaFuncSetAttribute(pscatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kP1SmemBytes);
    cudaFuncSetAttribute(pscatter_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
  }
  if (g_hi > g_lo) {
    // one CTA per SM, each at least 1024 groups
    const uint64_t want = (g_hi - g_lo + 1023) / 1024;
    const uint32_t grid = (uint32_t)std::min<uint64_t>((uint64_t)n_sm, want);
    pscatter_kernel<<<grid, kP1Threads, kP1SmemBytes, s>>>(a, j, tile_lo, tile_hi, g_lo, g_hi);
  }
  if (n_chunks + n_bins) launch_p2(a, j, chunk_off, n_chunks, bin_off, n_bins, n_sm, s);
  (void)lanes;  // the sliced rows of phase 2 need no group width
}

void free_twophase(cb_graph *h) {
  dev_free(h->d_pbin);
  dev_free(h->d_ptbase);
  dev_free(h->d_ptotal);
  dev_free(h->d_ptile_inst);
  dev_free(h->d_proff);
  dev_free(h->d_pcstart);
  dev_free(h->d_prtot);
  dev_free(h->d_pxbase);
  dev_free(h->d_pxscan);
  dev_free(h->d_ppos);
  dev_free(h->d_psrc);
  dev_free(h->d_pgdst);
  dev_free(h->d_pX);
  dev_free(h->d_psl);
  dev_free(h->d_psloff);
  dev_free(h->d_pdesc);
  h->d_psl = nullptr;
  h->d_psloff = nullptr;
  h->d_pdesc = nullptr;
  h->d_pbin = nullptr;
  h->d_ptbase = h->d_pxbase = h->d_pxscan = nullptr;
  h->d_ptotal = h->d_ptile_inst = h->d_proff = h->d_pcstart = h->d_prtot = h->d_pgdst = nullptr;
  h->d_ppos = h->d_psrc = nullptr;
  h->d_pX = nullptr;
  h->total_ptiles = h->total_pbins = 0;
  h->ptbase.clear();
  h->total_pgroups = 0;
  h->pns_max = 0;
  for (cb::InstDesc &I : h->inst) I.pb = 0;
}

// u16 words of a bin's phase-2 plan, as pslice_kernel lays it out: slice s
// runs the length (rounded up to even) of the piece at rank 32 s when the
// pieces are sorted longest first
uint64_t slice_plan_words(const uint32_t *rp, const PBin &b) {
  uint32_t hist[kPPiece + 1] = {};
  uint32_t np = 0;
  for (uint32_t i = b.row0; i < b.row1; ++i) {
    const uint32_t d = rp[i + 1] - rp[i];
    hist[kPPiece] += d / kPPiece;
    if (d % kPPiece) hist[d % kPPiece] += 1;
    np += (d + kPPiece - 1) / kPPiece;
  }
  const uint32_t ns = (np + 31) / 32;
  uint64_t steps = 0;
  uint32_t len = kPPiece, seen = 0;  // seen: pieces longer than len
  for (uint32_t s = 0; s < ns; ++s) {
    while (seen + hist[len] <= 32 * s) seen += hist[len--];
    steps += (len + 1) & ~1u;
  }
  return 64 + ((ns + 7) & ~7u) + 32ull * ns + ((b.row1 - b.row0 + 1 + 7) & ~7u) + 32 * steps;
}

int build_twophase(cb_graph *h, const std::vector<const uint32_t *> &rp_host, cudaStream_t s,
                   const std::vector<CopyGroup> &groups, bool force) {
  NvtxRange nvtx_range("two-phase format");
  if (h->csr_only) return CB_OK;
  const uint32_t N = h->n_inst;
  // which realisations, their bins (host, from row_ptr), in parallel
  std::vector<std::vector<PBin>> rbins(N);
  std::vector<std::vector<uint64_t>> rsize(N);  // u16 words of each bin's phase-2 plan
  std::vector<uint8_t> want(N, 0);
  for (uint32_t r = 0; r < N; ++r) {
    const InstDesc &I = h->inst[r];
    const bool big = I.n > kBMaxBlocks * kBCol;
    // every row of at most kHeavyDeg entries must fit a bin with the
    // worst-case chunk padding: (kPGroup - 1) S + kHeavyDeg <= kPRegion, so
    // n <= 1170 tiles (about 3.8e7 nodes); larger ones keep the tiled CSR
    const uint32_t S = (I.n + kPSrc - 1) / kPSrc;
    const bool fits = I.n <= kPSrc * kPMaxSrc && (kPGroup - 1) * S + kHeavyDeg <= kPRegion;
    want[r] = (force || big) && fits && !I.blocked ? 1 : 0;
  }
  parallel_for(N, [&](uint32_t r) {
    if (!want[r]) return;
    const InstDesc &I = h->inst[r];
    const uint32_t *rp = rp_host[r];
    const uint32_t S = (I.n + kPSrc - 1) / kPSrc;
    // worst-case padding: kPGroup - 1 slots per chunk, one chunk per source tile
    const uint32_t cap = kPRegion - (kPGroup - 1) * S;
    // the phase-2 slot array: at most 32 kPPiece + sum(deg + (deg & 1)) words
    const uint32_t scap = kPSlotsMax - 32 * kPPiece;
    uint32_t row0 = 0, acc = 0, sacc = 0;
    bool open = false;
    for (uint32_t i = 0; i < I.n; ++i) {
      const uint32_t deg = rp[i + 1] - rp[i];
      const bool heavy = deg > kHeavyDeg;
      if (open && (heavy || i - row0 == kPBinRows || acc + deg > cap || sacc + deg + (deg & 1u) > scap)) {
        rbins[r].push_back(PBin{r, row0, i, 0});
        open = false;
      }
      if (heavy) continue;
      if (!open) {
        row0 = i;
        acc = 0;
        sacc = 0;
        open = true;
      }
      acc += deg;
      sacc += deg + (deg & 1u);
    }
    if (open) rbins[r].push_back(PBin{r, row0, I.n, 0});
    for (const PBin &b : rbins[r]) rsize[r].push_back(slice_plan_words(rp, b));
  });
  uint32_t tiles = 0, nbins = 0, slot = 0, group = 0, pns_max = 0;
  uint64_t mat = 0;
  std::vector<PBin> bins;
  std::vector<uint32_t> tile_inst;
  std::vector<uint64_t> psloff;
  uint64_t plan_words = 0;
  for (uint32_t r = 0; r < N; ++r) {
    InstDesc &I = h->inst[r];
    I.pb = want[r];
    I.pns = I.pb ? (I.n + kPSrc - 1) / kPSrc : 0u;
    I.ptile_base = tiles;
    I.pbin_base = nbins;
    I.n_pbin = I.pb ? (uint32_t)rbins[r].size() : 0u;
    I.pmat_base = mat;
    I.pspmv = RedPlan{slot, 0, group, 0};
    if (!I.pb) continue;
    tiles += I.pns;
    nbins += I.n_pbin;
    mat += (uint64_t)I.n_pbin * (I.pns + 1);
    I.pspmv.n_slots = I.n_pbin + I.n_heavy;
    I.pspmv.n_groups = (I.pspmv.n_slots + kGroup - 1) / kGroup;
    slot += I.pspmv.n_slots;
    group += I.pspmv.n_groups;
    pns_max = std::max(pns_max, I.pns);
    bins.insert(bins.end(), rbins[r].begin(), rbins[r].end());
    for (uint64_t w : rsize[r]) {
      psloff.push_back(plan_words);
      plan_words += w;
    }
    tile_inst.insert(tile_inst.end(), I.pns, r);
  }
  if (tiles == 0) return CB_OK;
  h->total_ptiles = tiles;
  h->total_pbins = nbins;
  h->pns_max = pns_max;
  h->total_slots = std::max(h->total_slots, slot);
  h->total_groups = std::max(h->total_groups, group);

  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  auto fail = [&](int code, const char *msg) {
    free_twophase(h);
    return code == CB_ERR_ARG ? set_error(code, msg) : cuda_error(e, msg);
  };
  // nothing here is freed before the handle is: a free would synchronise the
  // device (and stall an upload behind another thread's kernels)
  chk(dalloc(&h->d_pbin, std::max<uint32_t>(nbins, 1)));
  chk(dalloc(&h->d_ptbase, tiles + 1));
  chk(dalloc(&h->d_ptotal, tiles + 1));  // + the invalid-column flag
  chk(dalloc(&h->d_ptile_inst, tiles));
  chk(dalloc(&h->d_proff, std::max<uint64_t>(mat, 1)));
  chk(dalloc(&h->d_pcstart, std::max<uint64_t>(mat, 1)));
  chk(dalloc(&h->d_prtot, std::max<uint32_t>(nbins, 1)));
  chk(dalloc(&h->d_pxbase, (uint64_t)nbins + 1));
  chk(dalloc(&h->d_pxscan, (uint64_t)nbins / 4096 + 2));
  chk(dalloc(&h->d_ppos, h->total_nnz + 8));
  chk(dalloc(&h->d_psloff, (uint64_t)nbins + 1));
  chk(dalloc(&h->d_pdesc, std::max<uint32_t>(nbins, 1)));
  chk(dalloc(&h->d_psl, plan_words + 8));
  if (e != cudaSuccess) return fail(CB_ERR_OOM, "two-phase format: allocate");
  uint32_t *d_bad = h->d_ptotal + tiles;
  // every copy of the upload has landed on `s` before the format reads it
  for (const CopyGroup &g : groups) chk(cudaStreamWaitEvent(s, g.ev, 0));
  psloff.push_back(plan_words);
  if (nbins) chk(stage_h2d(h->d_pbin, bins.data(), nbins * sizeof(PBin), s));
  chk(stage_h2d(h->d_psloff, psloff.data(), (nbins + 1) * 8, s));
  chk(stage_h2d(h->d_ptile_inst, tile_inst.data(), tiles * 4, s));
  chk(stage_h2d(h->d_inst, h->inst.data(), N * sizeof(InstDesc), s));
  chk(cudaMemsetAsync(d_bad, 0, 4, s));
  const size_t shm_count = (size_t)pns_max * 4;
  const size_t shm_fill = (size_t)pns_max * 16;
  if (e == cudaSuccess && shm_fill > 48 * 1024)
    chk(cudaFuncSetAttribute(pfill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_fill));
  if (e == cudaSuccess && nbins) {
    pcount_kernel<<<nbins, kBuildThreads, shm_count, s>>>(h->d_inst, h->d_pbin, h->row_ptr, h->col,
                                                          h->d_proff, h->d_prtot, d_bad);
    chk(exclusive_scan(h->d_prtot, nbins, h->d_pxbase, h->d_pxscan, s));
  }
  if (e == cudaSuccess)
    pcolscan_kernel<<<tiles, kBuildThreads, 0, s>>>(h->d_inst, h->d_ptile_inst, h->d_proff,
                                                    h->d_pcstart, h->d_ptotal);
  chk(cudaGetLastError());
  std::vector<uint32_t> tot(tiles + 1);
  chk(cudaMemcpyAsync(tot.data(), h->d_ptotal, (tiles + 1) * 4, cudaMemcpyDeviceToHost, s));
  chk(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return fail(CB_ERR_CUDA, "two-phase format: count");
  if (tot[tiles]) return fail(CB_ERR_ARG, "cb_graph_upload: a column index is >= n");
  // stream bases per source tile (host copy kept for the launch ranges)
  std::vector<uint64_t> tbase(tiles + 1);
  uint64_t gsum = 0;
  for (uint32_t g = 0; g < tiles; ++g) {
    tbase[g] = gsum;
    gsum += tot[g];
  }
  tbase[tiles] = gsum;
  if (gsum >= (1ull << 32)) return fail(CB_ERR_ARG, "cb_graph_upload: two-phase format too large");
  h->total_pgroups = gsum;
  // + 4 groups: the streamed windows of phase 1 end on a multiple of 4 groups
  chk(dalloc(&h->d_psrc, kPGroup * (gsum + 4)));
  chk(dalloc(&h->d_pgdst, gsum + 4));
  chk(dalloc(&h->d_pX, kPGroup * gsum + kPGroup));
  if (e != cudaSuccess) return fail(CB_ERR_OOM, "two-phase format: allocate stream");
  chk(stage_h2d(h->d_ptbase, tbase.data(), (tiles + 1) * 8, s));
  h->ptbase = std::move(tbase);
  chk(stage_h2d(h->d_inst, h->inst.data(), N * sizeof(InstDesc), s));
  // padding slots read node 0 of their tile: harmless, never summed
  chk(cudaMemsetAsync(h->d_psrc, 0, kPGroup * (gsum + 4) * 2, s));
  chk(cudaMemsetAsync(h->d_pgdst, 0, (gsum + 4) * 4, s));
  if (e == cudaSuccess && nbins)
    pfill_kernel<<<nbins, kBuildThreads, shm_fill, s>>>(h->d_inst, h->d_pbin, h->row_ptr, h->col,
                                                        h->d_proff, h->d_pcstart, h->d_ptbase,
                                                        h->d_pxbase, h->d_ppos, h->d_psrc,
                                                        h->d_pgdst);
  // the phase-2 plans, from the slots the fill gave the entries
  chk(cudaMemsetAsync(d_bad, 0, 4, s));
  if (e == cudaSuccess && nbins)
    pslice_kernel<<<nbins, kP2Threads, 0, s>>>(h->d_inst, h->d_pbin, h->row_ptr, h->d_ppos,
                                               h->d_psloff, h->d_pxbase, h->d_psl, h->d_pdesc,
                                               d_bad);
  chk(cudaGetLastError());
  uint32_t bad = 0;
  chk(cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, s));
  chk(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return fail(CB_ERR_CUDA, "two-phase format: fill");
  if (bad) {  // internal consistency: the host and device plan sizes disagree
    free_twophase(h);
    return set_error(CB_ERR_STATE, "two-phase format: phase-2 plan size");
  }
  return CB_OK;
}

CB_DEBUG_READER(twophase)

}  // namespace cb
