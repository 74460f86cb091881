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
//   * phase 2 (pgather_kernel) brings its bin's region, the entries' region
//     slots (pos: u16 per CSR entry) and the row offsets into shared memory
//     with three bulk copies, then sums each row as the tiled-CSR kernel does
//     -- G-lane groups for short rows, a warp for medium ones, the CTA for
//     long ones -- gathering region[pos[e]] instead of W_j[col[e]], and
//     applies the same row epilogue and alpha partial.  Heavy rows are summed
//     in chunks from the CSR as in the tiled-CSR kernel.
//
// DRAM bytes per entry: 2 (source offset) + 0.5 (group place) + 4 (value
// write) in phase 1, 4 (value read) + 2 (pos) in phase 2, plus the chunk
// padding, against the 4 of one u32 column index; in exchange every access
// is sequential or a whole sector, and every random one hits shared memory.
//
// The format is built on the device at upload: a count pass per bin (chunk
// sizes, region offsets), a prefix over the bins' region sizes, a pass per
// source tile (chunk offsets within the tile's stream), and a fill pass per
// bin that gives every entry a slot and every stream group its place.  The
// slot of an entry inside its chunk comes from a shared-memory atomic, so
// the layout may differ between uploads, but the sums cannot: phase 2 adds
// each row's entries in CSR order wherever they sit.
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

// Per bin: the phase-2 work plan.  The bin's rows are split among the
// kP2Threads / 32 warps by entry count (warp w owns the rows that start in
// [E w / W, E (w + 1) / W)), and each lane of a warp gets an equal share of
// the warp's merge path -- the merged sequence of its entries and row ends --
// whose start (row, entry), both bin-relative, is stored as row | entry << 16;
// plan_end[bin] = nrows | E << 16 ends the last lane's share.
__global__ void __launch_bounds__(kP2Threads) pplan_kernel(const InstDesc *inst, const PBin *bins,
                                                           const uint32_t *row_ptr, uint32_t *plan,
                                                           uint32_t *plan_end) {
  constexpr uint32_t W = kP2Threads / 32;
  __shared__ uint32_t s_rp[kPBinRows + 1];
  __shared__ uint32_t s_wrow[W + 1];
  const PBin B = bins[blockIdx.x];
  const InstDesc I = inst[B.inst];
  const uint32_t *rp = row_ptr + I.rp_base + B.row0;
  const uint32_t nrows = B.row1 - B.row0;
  const uint32_t tid = threadIdx.x;
  for (uint32_t q = tid; q <= nrows; q += blockDim.x) s_rp[q] = rp[q] - rp[0];
  __syncthreads();
  const uint32_t E = s_rp[nrows];
  auto lower_bound = [&](uint32_t t) -> uint32_t {  // least lr with s_rp[lr] >= t
    uint32_t lo = 0, hi = nrows;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_rp[mid] < t) lo = mid + 1; else hi = mid;
    }
    return lo;
  };
  if (tid < W) s_wrow[tid] = lower_bound((uint32_t)((uint64_t)E * tid / W));
  if (tid == 0) s_wrow[W] = nrows;
  __syncthreads();
  const uint32_t w = tid >> 5, l = tid & 31;
  const uint32_t rb = s_wrow[w], re = s_wrow[w + 1];
  const uint32_t k0 = s_rp[rb], nr = re - rb, ne = s_rp[re] - k0;
  const uint32_t d0 = (uint32_t)((uint64_t)(nr + ne) * l / 32);
  // rows of the warp completed before step d0: row i ends at step
  // (s_rp[rb + i + 1] - k0) + i
  uint32_t lo = 0, hi = nr;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (s_rp[rb + mid + 1] - k0 + mid < d0) lo = mid + 1; else hi = mid;
  }
  plan[(uint64_t)blockIdx.x * kP2Threads + tid] = (rb + lo) | ((k0 + d0 - lo) << 16);
  if (tid == 0) plan_end[blockIdx.x] = nrows | (E << 16);
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
              X[2ull * d + half] = o;
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
// Phase 2: one bin per CTA (blocks after the heavy-row chunk CTAs), two CTAs
// per SM, so one CTA's copies overlap the other's sums.  The bin's region,
// its entries' pos, its row offsets and its rows of W_j and W_{j-1} arrive
// by bulk copies on one mbarrier (one thread polls it while the others
// sleep in the CTA barrier; nothing waits on the CTA after that).  The rows
// are split among the warps by entry count (a warp owns the rows that start
// in its share); within a warp each lane takes an equal share of the merged
// sequence of the warp's entries and row ends (merge path, Merrill &
// Garland 2016), sums its entries in order -- the gathers issued four
// entries ahead -- and writes every row it completes to shared memory; a
// row that spans lanes is completed by the lane that reaches its end, after
// a segmented scan of the lanes' carries in lane order.  The warp then
// applies the row epilogue to its rows (coalesced stores), and the last warp
// to finish adds the warp partials in warp order and enters the bin's alpha
// term.  The row searches are warp-cooperative (ballots over 32 candidate
// rows at a time) instead of per-lane binary searches.
// ---------------------------------------------------------------------------
constexpr uint32_t kP2Warps = kP2Threads / 32;
// every part a whole number of 16-byte units (each but the row sums is the
// destination of a bulk copy): the region, the bin's pos entries (+ 8 for
// the 16-byte alignment of the copy), its row offsets (+ 4), its rows of
// W_j and W_{j-1} (+ 4 each) for the epilogue, and the row sums
constexpr uint32_t kP2PosElems = kPRegion + 8;
constexpr uint32_t kP2RpWords = kPBinRows + 4;
constexpr uint32_t kP2XWords = kPBinRows + 4;
static_assert((kPRegion * 4) % 16 == 0 && (kP2PosElems * 2) % 16 == 0 && (kP2RpWords * 4) % 16 == 0 &&
                  (kP2XWords * 4) % 16 == 0,
              "phase-2 shared-memory buffers must keep 16-byte alignment");
constexpr size_t kP2SmemBytes = (size_t)kPRegion * sizeof(float) + kP2PosElems * sizeof(uint16_t) +
                                kP2RpWords * sizeof(uint32_t) + 2 * kP2XWords * sizeof(float) +
                                kPBinRows * sizeof(float);
// two CTAs per SM: 228 KB per SM, 1 KB reserved per CTA, < 640 B of static
// shared memory (ptxas -v reports it)
static_assert(2 * (kP2SmemBytes + 1024 + 640) <= 228 * 1024, "two phase-2 CTAs per SM");

__global__ void __launch_bounds__(kP2Threads, 2) pgather_kernel(LArgs a, uint32_t j, uint32_t chunk_off,
                                                                uint32_t n_chunks, uint32_t bin_off) {
  extern __shared__ float4 s_dyn4[];
  float *reg = reinterpret_cast<float *>(s_dyn4);                       // the bin region
  uint16_t *s_pos = reinterpret_cast<uint16_t *>(reg + kPRegion);       // pos of the bin's entries
  uint32_t *s_rpw = reinterpret_cast<uint32_t *>(s_pos + kP2PosElems);  // row offsets
  float *s_xw = reinterpret_cast<float *>(s_rpw + kP2RpWords);          // the bin's rows of W_j
  float *s_xpw = s_xw + kP2XWords;                                      // and of W_{j-1}
  float *s_sum = s_xpw + kP2XWords;                                     // row sums
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
  const PBin B = a.pbin[bin];
  const uint32_t r = B.inst;
  if (j >= a.sc.meff[r]) return;  // realisation stopped (uniform per CTA)
  const InstDesc &I = a.inst[r];
  const uint32_t row0 = B.row0, nrows = B.row1 - B.row0;
  float *Vb = reinterpret_cast<float *>(a.V);
  const float *x = Vb + (uint64_t)j * a.vs + I.node_base;
  const bool has_prev = j > 0;
  const uint32_t *rpg = a.row_ptr + I.rp_base + row0;
  const uint32_t rp_lead = (uint32_t)((reinterpret_cast<uintptr_t>(rpg) >> 2) & 3u);
  // node_base is a multiple of 32 elements: the rows' window starts 16-byte
  // aligned at row0 - (row0 & 3) and ends at most 3 floats past row n - 1
  const uint32_t x_lead = row0 & 3u;
  if (tid == 0) {
    s_done = 0;
    s_fail = 0;
    mbar_init(&s_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const uint32_t rp_words = (rp_lead + nrows + 1 + 3u) & ~3u;
    const uint32_t e_first = rpg[0], e_last = rpg[nrows];  // the bin's CSR entry range
    const uint16_t *pg = a.ppos + I.edge_base + e_first;
    const uint32_t pos_lead = (uint32_t)((reinterpret_cast<uintptr_t>(pg) >> 1) & 7u);
    const uint32_t pos_elems = (pos_lead + (e_last - e_first) + 7u) & ~7u;
    const uint64_t xg0 = a.pxbase[bin], xg1 = a.pxbase[bin + 1];
    const uint32_t reg_bytes = (uint32_t)(xg1 - xg0) * kPGroup * 4u;
    const uint32_t xb = ((x_lead + nrows + 3u) & ~3u) * 4u;
    mbar_expect_tx(&s_full, reg_bytes + pos_elems * 2u + rp_words * 4u + (has_prev ? 2u : 1u) * xb);
    if (reg_bytes) bulk_g2s(reg, a.pX + xg0 * kPGroup, reg_bytes, &s_full);
    if (pos_elems) bulk_g2s(s_pos, pg - pos_lead, pos_elems * 2u, &s_full);
    bulk_g2s(s_rpw, rpg - rp_lead, rp_words * 4u, &s_full);
    bulk_g2s(s_xw, x + row0 - x_lead, xb, &s_full);
    if (has_prev) bulk_g2s(s_xpw, x - a.vs + row0 - x_lead, xb, &s_full);
    if (!mbar_wait(&s_full, 0)) s_fail = 1;
  }
  const uint32_t ms = a.sc.ms;
  const float sj = (float)a.sc.scale[r * ms + j];
  const float bp = has_prev ? (float)(a.sc.beta[r * ms + j - 1] * a.sc.scale[r * ms + j - 1]) : 0.f;
  float *out = Vb + (uint64_t)(j + 1) * a.vs + I.node_base + row0;
  // this lane's merge-path start and end, from the plan built at upload
  const uint32_t *plan = a.pplan + (uint64_t)bin * kP2Threads;
  const uint32_t ps = __ldg(plan + tid);
  const uint32_t pe = tid + 1 < (uint32_t)kP2Threads ? __ldg(plan + tid + 1) : a.pplan_end[bin];
  __syncthreads();  // the bin has landed (or the wait gave up); no CTA barrier below
  const bool ok = s_fail == 0;
  double wpart = 0.0;
  if (ok) {
    const uint32_t *s_rp = s_rpw + rp_lead;  // s_rp[q] = row_ptr[row0 + q]
    const uint32_t e_first = s_rp[0], E = s_rp[nrows] - e_first;
    const uint16_t *pos =
        s_pos + ((uint32_t)((reinterpret_cast<uintptr_t>(a.ppos + I.edge_base + e_first) >> 1) & 7u));
    // this lane's share of the warp's merge path: from (row, entry) =
    // plan[t] to plan[t + 1] (the last lane's end is the bin's end), both
    // bin-relative; a warp's first lane starts at its first row's start
    const uint32_t sp = ps, ep = pe;
    const uint32_t lr0 = sp & 0xffffu, kk0 = sp >> 16, lr1 = ep & 0xffffu, kk1 = ep >> 16;
    const uint32_t rb = __shfl_sync(0xffffffffu, lr0, 0), re = __shfl_sync(0xffffffffu, lr1, 31);
    uint32_t ri = lr0, k = kk0;
    const uint32_t nsteps = (lr1 + kk1) - (lr0 + kk0);
    const uint32_t i_first = ri;
    uint32_t re_i = ri < nrows ? s_rp[ri + 1] - e_first : E;  // end of row ri (bin-relative entries)
    float sum = 0.f, head = 0.f;
    bool head_done = false;
    // one step per iteration, without divergence: every step gathers (entry
    // k, clamped to the bin; its slot clamped to the region), and a row end
    // only selects what it keeps, so the lanes of a warp never run two paths
    const uint32_t elast = E ? E - 1 : 0;
#ifdef CB_DEBUG
    const uint32_t rslots = (uint32_t)(a.pxbase[bin + 1] - a.pxbase[bin]) * kPGroup;
#endif
    for (uint32_t d = 0; d < nsteps; ++d) {
      const bool ent = k < re_i;  // the next entry of row ri, or row ri ends
      // the slot clamped to the region: a bin without entries copies no pos,
      // and the value of a row-end step is never added
      const float v = reg[min((uint32_t)pos[min(k, elast)], kPRegion - 1)];
#ifdef CB_DEBUG
      // an entry's slot lies inside the bin's region (the clamp above only
      // guards the look of a row-end step)
      CB_DCHECK(!ent || pos[min(k, elast)] < rslots, kDbgTwoPhasePos, pos[min(k, elast)]);
#endif
      const bool first = !ent && ri == i_first;
      if (!ent && !first) s_sum[ri] = sum;
      head = first ? sum : head;  // may continue an earlier lane's row: completed below
      head_done = head_done || first;
      sum = ent ? sum + v : 0.f;
      k += ent ? 1u : 0u;
      const uint32_t rn = ri + 1;
      const uint32_t ren = rn < nrows ? s_rp[min(rn + 1, nrows)] - e_first : E;
      re_i = ent ? re_i : ren;
      ri = ent ? ri : rn;
    }
    // carries: the lane's unfinished row and its partial sum; an inclusive
    // segmented scan (rows are non-decreasing over lanes) in lane order
    uint32_t crow = ri;
    float csum = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float up = __shfl_up_sync(0xffffffffu, csum, o);
      const uint32_t urow = __shfl_up_sync(0xffffffffu, crow, o);
      if (lane >= (uint32_t)o && urow == crow) csum = up + csum;
    }
    const float prev = __shfl_up_sync(0xffffffffu, csum, 1);
    const uint32_t prow = __shfl_up_sync(0xffffffffu, crow, 1);
    if (head_done) s_sum[i_first] = (lane > 0 && prow == i_first) ? prev + head : head;
    __syncwarp();
    // the row epilogue of the warp's rows: u = sj * sum - bp * W_{j-1}[row],
    // stored (coalesced); the alpha partial gathers W_j[row] * u
    const float *sx = s_xw + x_lead, *sxp = s_xpw + x_lead;  // sx[q] = W_j[row0 + q]
    float acc = 0.f;
    for (uint32_t lr = rb + lane; lr < re; lr += 32) {
      float u = sj * s_sum[lr];
      if (has_prev) u -= bp * sxp[lr];
      out[lr] = u;
      acc += sx[lr] * u;
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
  if (warp_arrive_and_reduce(I.pspmv, bin - I.pbin_base, r, part, a.red, &total) && lane == 0)
    finish_alpha<float>(a, r, j, total);
}

void launch_p2(const LArgs &a, uint32_t j, uint32_t chunk_off, uint32_t n_chunks, uint32_t bin_off,
               uint32_t n_bins, cudaStream_t s) {
  static bool attr = false;  // opt-in to > 48 KB of shared memory
  if (!attr) {
    cudaFuncSetAttribute(pgather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kP2SmemBytes);
    cudaFuncSetAttribute(pgather_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    attr = true;
  }
  pgather_kernel<<<n_chunks + n_bins, kP2Threads, kP2SmemBytes, s>>>(a, j, chunk_off, n_chunks, bin_off);
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
  if (n_chunks + n_bins) launch_p2(a, j, chunk_off, n_chunks, bin_off, n_bins, s);
  (void)lanes;  // the merge-path walk of phase 2 needs no group width
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
  dev_free(h->d_pplan);
  dev_free(h->d_pplan_end);
  h->d_pplan = h->d_pplan_end = nullptr;
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

int build_twophase(cb_graph *h, const std::vector<const uint32_t *> &rp_host, cudaStream_t s,
                   const std::vector<CopyGroup> &groups, bool force) {
  NvtxRange nvtx_range("two-phase format");
  if (h->csr_only) return CB_OK;
  const uint32_t N = h->n_inst;
  // which realisations, their bins (host, from row_ptr), in parallel
  std::vector<std::vector<PBin>> rbins(N);
  std::vector<uint8_t> want(N, 0);
  for (uint32_t r = 0; r < N; ++r) {
    const InstDesc &I = h->inst[r];
    const bool big = I.n > kBMaxBlocks * kBCol;
    want[r] = (force || big) && I.n <= kPSrc * kPMaxSrc && !I.blocked ? 1 : 0;
  }
  parallel_for(N, [&](uint32_t r) {
    if (!want[r]) return;
    const InstDesc &I = h->inst[r];
    const uint32_t *rp = rp_host[r];
    const uint32_t S = (I.n + kPSrc - 1) / kPSrc;
    // worst-case padding: kPGroup - 1 slots per chunk, one chunk per source tile
    const uint32_t cap = kPRegion - (kPGroup - 1) * S;
    uint32_t row0 = 0, acc = 0;
    bool open = false;
    for (uint32_t i = 0; i < I.n; ++i) {
      const uint32_t deg = rp[i + 1] - rp[i];
      const bool heavy = deg > kHeavyDeg;
      if (open && (heavy || i - row0 == kPBinRows || acc + deg > cap)) {
        rbins[r].push_back(PBin{r, row0, i, 0});
        open = false;
      }
      if (heavy) continue;
      if (!open) {
        row0 = i;
        acc = 0;
        open = true;
      }
      acc += deg;
    }
    if (open) rbins[r].push_back(PBin{r, row0, I.n, 0});
  });
  uint32_t tiles = 0, nbins = 0, slot = 0, group = 0, pns_max = 0;
  uint64_t mat = 0;
  std::vector<PBin> bins;
  std::vector<uint32_t> tile_inst;
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
  chk(dalloc(&h->d_pplan, (uint64_t)std::max<uint32_t>(nbins, 1) * kP2Threads));
  chk(dalloc(&h->d_pplan_end, std::max<uint32_t>(nbins, 1)));
  if (e != cudaSuccess) return fail(CB_ERR_OOM, "two-phase format: allocate");
  uint32_t *d_bad = h->d_ptotal + tiles;
  // every copy of the upload has landed on `s` before the format reads it
  for (const CopyGroup &g : groups) chk(cudaStreamWaitEvent(s, g.ev, 0));
  if (nbins) chk(stage_h2d(h->d_pbin, bins.data(), nbins * sizeof(PBin), s));
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
    pplan_kernel<<<nbins, kP2Threads, 0, s>>>(h->d_inst, h->d_pbin, h->row_ptr, h->d_pplan,
                                              h->d_pplan_end);
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
  chk(cudaGetLastError());
  chk(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return fail(CB_ERR_CUDA, "two-phase format: fill");
  return CB_OK;
}

CB_DEBUG_READER(twophase)

}  // namespace cb
