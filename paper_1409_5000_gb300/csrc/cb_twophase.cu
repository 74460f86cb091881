// Two-phase (propagation-blocked) Lanczos SpMV step for large graphs (FP32).
//
// The Krylov evaluation of e^A 1 (section "Identification algorithm") costs
// one product u = A v_j per Lanczos step.  When a realisation's vector is
// too long for the column-blocked kernel (n > 32 column blocks of 16384),
// every gather of v_j from the CSR is a random 4-byte load from L2: one
// 32-byte sector request each, about one per clock per SM.  This step moves
// every random access into shared memory, at the price of one extra stream
// of edge values through memory (propagation blocking):
//
//   * columns are cut into source tiles of kPSrc nodes, rows into bins: runs
//     of rows whose entries, with chunk padding, fit a region of kPRegion
//     values; rows heavier than kHeavyDeg stay out of the bins;
//   * the stream has one slot per entry of a bin row, ordered by (source tile
//     s, bin t): chunk (s, t) holds the entries of bin t whose column lies in
//     tile s, padded to a multiple of 4 slots (16 bytes);
//   * phase 1 (pscatter_kernel) stages tile s of W_j in shared memory with
//     one bulk copy and writes every slot of the tile's stream:
//     X[q] = W_j[node of q], reading 4 u16 source offsets and writing one
//     float4 per 4 slots (coalesced, sequential);
//   * phase 2 (pgather_kernel) copies the chunks (s, t), s = 0..S-1, of its
//     bin into a shared-memory region (cp.async, 16-byte units), then sums
//     each row as the tiled-CSR kernel does -- G-lane groups for short rows,
//     a warp for medium ones, the CTA for long ones -- but gathering
//     region[pos[e]] (pos: u16 per CSR entry) instead of W_j[col[e]], and
//     applies the same row epilogue and alpha partial.  Heavy rows are summed
//     in chunks from the CSR as in the tiled-CSR kernel.
//
// DRAM bytes per entry: 2 (source offset) + 4 (stream write) in phase 1,
// 4 (stream read) + 2 (pos) in phase 2, plus padding, against the 4 of one
// u32 column index; in exchange no access is a random L2 sector request.
//
// The format is built on the device at upload: a count pass per bin (chunk
// sizes, region offsets), a pass per source tile (chunk offsets within the
// tile's stream), and a fill pass per bin that gives every entry a slot.
// The slot of an entry inside its chunk comes from a shared-memory atomic, so
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
// to whole 4-slot units, and their exclusive prefix over s: roff[bin][s] is
// the unit offset of chunk (s, bin) in the bin's region, roff[bin][S] the
// region's units.  A column >= n sets *bad (the upload then fails).
__global__ void __launch_bounds__(kBuildThreads) pcount_kernel(const InstDesc *inst, const PBin *bins,
                                                               const uint32_t *row_ptr,
                                                               const uint32_t *col, uint32_t *roff,
                                                               uint32_t *bad) {
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
  for (uint32_t q = s0; q < s1; ++q) mine += (s_hist[q] + 3u) >> 2;
  uint32_t total;
  uint32_t run = block_excl_scan(mine, s_w, &total);
  uint32_t *ro = roff + I.pmat_base + (uint64_t)(blockIdx.x - I.pbin_base) * (S + 1);
  for (uint32_t q = s0; q < s1; ++q) {
    ro[q] = run;
    run += (s_hist[q] + 3u) >> 2;
  }
  if (threadIdx.x == 0) ro[S] = total;
}

// Per source tile s: cstart[bin][s], the unit offset of chunk (s, bin) in the
// tile's stream (exclusive prefix over the realisation's bins of the padded
// chunk units), and the tile's total units.
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
// counter per source tile); pos[e] is that slot's place in the bin region
// and psrc[slot] the entry's column within its tile.
__global__ void __launch_bounds__(kBuildThreads) pfill_kernel(const InstDesc *inst, const PBin *bins,
                                                              const uint32_t *row_ptr,
                                                              const uint32_t *col,
                                                              const uint32_t *roff,
                                                              const uint32_t *cstart,
                                                              const uint64_t *ptbase, uint16_t *ppos,
                                                              uint16_t *psrc) {
  extern __shared__ uint64_t s_q[];  // pns_max stream slot bases, then pns_max region bases and counters
  const PBin B = bins[blockIdx.x];
  const InstDesc I = inst[B.inst];
  const uint32_t S = I.pns;
  uint32_t *s_r = reinterpret_cast<uint32_t *>(s_q + S);
  uint32_t *s_c = s_r + S;
  const uint64_t mrow = I.pmat_base + (uint64_t)(blockIdx.x - I.pbin_base) * (S + 1);
  for (uint32_t q = threadIdx.x; q < S; q += blockDim.x) {
    s_q[q] = 4ull * (ptbase[I.ptile_base + q] + cstart[mrow + q]);
    s_r[q] = 4u * roff[mrow + q];
    s_c[q] = 0u;
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
    pos[e] = (uint16_t)(s_r[s] + k);
    psrc[s_q[s] + k] = (uint16_t)(c & (kPSrc - 1));
  }
}

// ---------------------------------------------------------------------------
// Phase 1: stream slots of one piece of a source tile's stream.
// ---------------------------------------------------------------------------
constexpr int kP1Unroll = 8;
constexpr size_t kP1SmemBytes = (size_t)kPSrc * sizeof(float);

__global__ void __launch_bounds__(kP1Threads, 1) pscatter_kernel(LArgs a, uint32_t j,
                                                                 uint32_t piece_off) {
  extern __shared__ float4 s_dyn4[];
  float *vt = reinterpret_cast<float *>(s_dyn4);  // the source tile of W_j
  __shared__ __align__(8) uint64_t s_full;
  const PPiece P = a.ppiece[piece_off + blockIdx.x];
  const uint32_t r = P.inst;
  if (j >= a.sc.meff[r]) return;  // realisation stopped (uniform per CTA)
  const InstDesc &I = a.inst[r];
  const float *x = reinterpret_cast<const float *>(a.V) + (uint64_t)j * a.vs + I.node_base;
  const uint32_t node0 = P.tile << kPSrcBits;
  const uint32_t nn = min(kPSrc, I.n - node0);
  // whole 16-byte units: up to 3 floats past node n-1, inside the padded vector
  const uint32_t bytes = ((nn + 3u) & ~3u) * 4u;
  const uint32_t tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&s_full, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    mbar_expect_tx(&s_full, bytes);
    bulk_g2s(vt, x + node0, bytes, &s_full);
  }
  const uint2 *src = reinterpret_cast<const uint2 *>(a.psrc) + P.u0;
  float4 *X = reinterpret_cast<float4 *>(a.pX) + P.u0;
  const uint32_t nu = P.nu;
  uint2 sv[kP1Unroll];
#pragma unroll
  for (int u = 0; u < kP1Unroll; ++u) {
    const uint32_t i = tid + u * kP1Threads;
    if (i < nu) sv[u] = __ldcs(src + i);
  }
  if (!mbar_wait(&s_full, 0)) {
    // the tile never landed: this step of the realisation fails; the copy
    // still in flight completes (bounded) before the CTA ends
    if (tid == 0) {
      a.sc.status[r] = CB_ERR_TIMEOUT;
      a.sc.meff[r] = j;
      mbar_wait(&s_full, 0);
    }
    return;
  }
  for (uint32_t b = tid; b < nu; b += kP1Unroll * kP1Threads) {
    uint2 nx[kP1Unroll];
    const uint32_t b1 = b + kP1Unroll * kP1Threads;
#pragma unroll
    for (int u = 0; u < kP1Unroll; ++u) {
      const uint32_t i = b1 + u * kP1Threads;
      if (i < nu) nx[u] = __ldcs(src + i);
    }
#pragma unroll
    for (int u = 0; u < kP1Unroll; ++u) {
      const uint32_t i = b + u * kP1Threads;
      if (i < nu) {
        float4 o;
        o.x = vt[sv[u].x & 0xffffu];
        o.y = vt[sv[u].x >> 16];
        o.z = vt[sv[u].y & 0xffffu];
        o.w = vt[sv[u].y >> 16];
        X[i] = o;
      }
    }
#pragma unroll
    for (int u = 0; u < kP1Unroll; ++u) sv[u] = nx[u];
  }
}

// ---------------------------------------------------------------------------
// Phase 2: one bin per CTA (blocks after the heavy-row chunks).
// ---------------------------------------------------------------------------
constexpr uint32_t kP2Short = 8;  // short rows: at most 8 entries per lane of a G-lane group

inline size_t p2_smem_bytes(uint32_t pns_max) {
  return (size_t)kPRegion * sizeof(float) + (size_t)pns_max * sizeof(uint4) +
         (size_t)(kPBinRows + 1) * sizeof(uint32_t);
}

template <int G>
__global__ void __launch_bounds__(kP2Threads, 2) pgather_kernel(LArgs a, uint32_t j, uint32_t chunk_off,
                                                                uint32_t n_chunks, uint32_t bin_off,
                                                                uint32_t pns_max) {
  extern __shared__ float4 s_dyn4[];
  float *reg = reinterpret_cast<float *>(s_dyn4);                 // the bin region
  uint4 *s_desc = reinterpret_cast<uint4 *>(reg + kPRegion);      // per chunk: region unit, units, stream unit
  uint32_t *s_rp = reinterpret_cast<uint32_t *>(s_desc + pns_max);  // the bin's row offsets
  __shared__ double s_red[32];
  __shared__ uint16_t s_med[kP2Threads], s_long[kP2Threads];
  __shared__ uint32_t s_wcnt[kP2Threads / 32][2];
  __shared__ uint32_t s_nmed, s_nlong;
  __shared__ float s_rowsum[32];
  constexpr uint32_t T = kP2Threads;
  const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (blockIdx.x < n_chunks) {  // one chunk of a heavy row of a two-phase realisation
    const uint32_t cidx = chunk_off + blockIdx.x;
    const uint32_t hid = a.chunk_heavy[cidx];
    const uint32_t r = a.heavy[hid].inst;
    if (j >= a.sc.meff[r] || !a.inst[r].pb) return;
    const InstDesc &I = a.inst[r];
    heavy_chunk<float>(a, j, cidx, hid, r, I.pspmv, I.n_pbin + (hid - I.heavy_base));
    return;
  }
  const uint32_t bidx = bin_off + (blockIdx.x - n_chunks);
  const PBin B = a.pbin[bidx];
  const uint32_t r = B.inst;
  if (j >= a.sc.meff[r]) return;
  const InstDesc &I = a.inst[r];
  const uint32_t S = I.pns;
  const uint32_t tb = bidx - I.pbin_base;
  const uint64_t mrow = I.pmat_base + (uint64_t)tb * (S + 1);
  for (uint32_t s = tid; s < S; s += T) {
    const uint32_t r0 = a.proff[mrow + s], r1 = a.proff[mrow + s + 1];
    const uint64_t q = a.ptbase[I.ptile_base + s] + a.pcstart[mrow + s];
    s_desc[s] = make_uint4(r0, r1 - r0, (uint32_t)q, (uint32_t)(q >> 32));
  }
  const uint32_t row0 = B.row0, nrows = B.row1 - B.row0;
  const uint32_t *rp = a.row_ptr + I.rp_base;
  for (uint32_t q = tid; q <= nrows; q += T) s_rp[q] = rp[row0 + q];
  __syncthreads();
  const uint16_t *pos = a.ppos + I.edge_base;
  if (tid == 0) {  // the bin's pos entries into L2 while the region is copied
    const uintptr_t p0 = reinterpret_cast<uintptr_t>(pos + s_rp[0]) & ~uintptr_t(15);
    const uintptr_t p1 = (reinterpret_cast<uintptr_t>(pos + s_rp[nrows]) + 15) & ~uintptr_t(15);
    if (p1 > p0) l2_prefetch(reinterpret_cast<const void *>(p0), (uint32_t)(p1 - p0));
  }
  // the bin's chunks of the stream into the region: a warp per chunk
  const float4 *X4 = reinterpret_cast<const float4 *>(a.pX);
  for (uint32_t s = warp; s < S; s += T / 32) {
    const uint4 d = s_desc[s];
    const uint64_t q = (uint64_t)d.z | ((uint64_t)d.w << 32);
    for (uint32_t u = lane; u < d.y; u += 32) cp_async16(reg + 4 * (d.x + u), X4 + q + u);
  }
  cp_async_wait_all();
  __syncthreads();

  const uint32_t ms = a.sc.ms;
  float *Vb = reinterpret_cast<float *>(a.V);
  const float *x = Vb + (uint64_t)j * a.vs + I.node_base;
  const bool has_prev = j > 0;
  const float *xp = has_prev ? Vb + (uint64_t)(j - 1) * a.vs + I.node_base : x;
  float *out = Vb + (uint64_t)(j + 1) * a.vs + I.node_base;
  const float sj = (float)a.sc.scale[r * ms + j];
  const float bp = has_prev ? (float)(a.sc.beta[r * ms + j - 1] * a.sc.scale[r * ms + j - 1]) : 0.f;

  float acc = 0.f;
  const uint32_t lane_g = tid % G, grp = tid / G;
  constexpr uint32_t kGroups = T / G;
  constexpr uint32_t kShort = kP2Short * G;
  for (uint32_t p0 = 0; p0 < nrows; p0 += T) {
    const uint32_t np = min(T, nrows - p0);
    // short rows: G lanes per row, a fixed predicated trip count (all of a
    // lane's pos loads, then all of its gathers, in flight together); the
    // trip count depends only on the bin, so the group shuffles converge
    for (uint32_t base = 0; base < np; base += kGroups) {
      const uint32_t lr = p0 + base + grp;
      const bool valid = base + grp < np;
      uint32_t e0 = 0, e1 = 0;
      if (valid) {
        e0 = s_rp[lr];
        e1 = s_rp[lr + 1];
      }
      const bool is_short = valid && (e1 - e0) <= kShort;
      float sum = 0.f;
      if (is_short) {
        const uint32_t len = e1 - e0;
#pragma unroll
        for (uint32_t i = 0; i < kP2Short; ++i) {
          const uint32_t t = lane_g + i * G;
          if (t < len) sum += reg[__ldcs(pos + e0 + t)];
        }
      }
      sum = group_sum<G, float>(sum);
      if (is_short && lane_g == 0) acc += row_epilogue<float>(sum, row0 + lr, x, xp, out, sj, bp, has_prev);
    }
    // medium (kShort < deg <= kLongDeg) and long (kLongDeg < deg) rows of
    // this pass: lists in row order from one ballot per warp
    {
      const uint32_t q = tid;
      uint32_t deg = 0;
      if (q < np) deg = s_rp[p0 + q + 1] - s_rp[p0 + q];
      const bool med = deg > kShort && deg <= kLongDeg;
      const bool lng = deg > kLongDeg;
      const uint32_t bm = __ballot_sync(0xffffffffu, med), bl = __ballot_sync(0xffffffffu, lng);
      if (lane == 0) {
        s_wcnt[warp][0] = __popc(bm);
        s_wcnt[warp][1] = __popc(bl);
      }
      __syncthreads();
      uint32_t om = 0, ol = 0, nm = 0, nl = 0;
      for (uint32_t w = 0; w < T / 32; ++w) {
        if (w < warp) {
          om += s_wcnt[w][0];
          ol += s_wcnt[w][1];
        }
        nm += s_wcnt[w][0];
        nl += s_wcnt[w][1];
      }
      const uint32_t below = (1u << lane) - 1u;
      if (med) s_med[om + __popc(bm & below)] = (uint16_t)q;
      if (lng) s_long[ol + __popc(bl & below)] = (uint16_t)q;
      if (tid == 0) {
        s_nmed = nm;
        s_nlong = nl;
      }
    }
    __syncthreads();
    {  // medium rows: a warp each
      const uint32_t nmed = s_nmed;
      for (uint32_t q = warp; q < nmed; q += T / 32) {
        const uint32_t lr = p0 + s_med[q];
        const uint32_t e0 = s_rp[lr], e1 = s_rp[lr + 1];
        float sum = 0.f;
#pragma unroll 4
        for (uint32_t e = e0 + lane; e < e1; e += 32) sum += reg[__ldcs(pos + e)];
        sum = warp_sum<float>(sum);
        if (lane == 0) acc += row_epilogue<float>(sum, row0 + lr, x, xp, out, sj, bp, has_prev);
      }
    }
    const uint32_t nlong = s_nlong;
    for (uint32_t q = 0; q < nlong; ++q) {  // long rows: the whole CTA, in row order
      const uint32_t lr = p0 + s_long[q];
      const uint32_t e0 = s_rp[lr], e1 = s_rp[lr + 1];
      float sum = 0.f;
#pragma unroll 4
      for (uint32_t e = e0 + tid; e < e1; e += T) sum += reg[__ldcs(pos + e)];
      sum = warp_sum<float>(sum);
      if (lane == 0) s_rowsum[warp] = sum;
      __syncthreads();
      if (tid == 0) {
        float tot = 0.f;
        for (uint32_t w = 0; w < T / 32; ++w) tot += s_rowsum[w];
        acc += row_epilogue<float>(tot, row0 + lr, x, xp, out, sj, bp, has_prev);
      }
      __syncthreads();
    }
    __syncthreads();  // the lists are rebuilt by the next pass
  }
  const double part = block_sum_to_double<float>(acc, s_red);
  double total;
  if (arrive_and_reduce(I.pspmv, tb, r, part, a.red, &total)) finish_alpha<float>(a, r, j, total);
}

template <int G>
void launch_p2(const LArgs &a, uint32_t j, uint32_t chunk_off, uint32_t n_chunks, uint32_t bin_off,
               uint32_t n_bins, uint32_t pns_max, cudaStream_t s) {
  const size_t shm = p2_smem_bytes(pns_max);
  static size_t attr = 0;  // opt-in to > 48 KB of shared memory, per instantiation
  if (shm > attr) {
    cudaFuncSetAttribute(pgather_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    cudaFuncSetAttribute(pgather_kernel<G>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    attr = shm;
  }
  pgather_kernel<G><<<n_chunks + n_bins, kP2Threads, shm, s>>>(a, j, chunk_off, n_chunks, bin_off,
                                                               pns_max);
}

template <typename P>
cudaError_t dalloc(P **p, size_t count) {
  return dev_alloc_n(p, count);
}

}  // namespace

void launch_twophase(const LArgs &a, int lanes, uint32_t j, uint32_t piece_off, uint32_t n_pieces,
                     uint32_t chunk_off, uint32_t n_chunks, uint32_t bin_off, uint32_t n_bins,
                     uint32_t pns_max, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(pscatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kP1SmemBytes);
    cudaFuncSetAttribute(pscatter_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    attr = true;
  }
  if (n_pieces) pscatter_kernel<<<n_pieces, kP1Threads, kP1SmemBytes, s>>>(a, j, piece_off);
  if (n_chunks + n_bins == 0) return;
  switch (lanes) {
    case 1: launch_p2<1>(a, j, chunk_off, n_chunks, bin_off, n_bins, pns_max, s); break;
    case 2: launch_p2<2>(a, j, chunk_off, n_chunks, bin_off, n_bins, pns_max, s); break;
    case 4: launch_p2<4>(a, j, chunk_off, n_chunks, bin_off, n_bins, pns_max, s); break;
    case 8: launch_p2<8>(a, j, chunk_off, n_chunks, bin_off, n_bins, pns_max, s); break;
    case 16: launch_p2<16>(a, j, chunk_off, n_chunks, bin_off, n_bins, pns_max, s); break;
    default: launch_p2<32>(a, j, chunk_off, n_chunks, bin_off, n_bins, pns_max, s); break;
  }
}

void free_twophase(cb_graph *h) {
  dev_free(h->d_pbin);
  dev_free(h->d_ppiece);
  dev_free(h->d_ptbase);
  dev_free(h->d_ptotal);
  dev_free(h->d_proff);
  dev_free(h->d_pcstart);
  dev_free(h->d_ppos);
  dev_free(h->d_psrc);
  dev_free(h->d_pX);
  dev_free(h->d_ptile_inst);
  h->d_ptile_inst = nullptr;
  h->d_pbin = nullptr;
  h->d_ppiece = nullptr;
  h->d_ptbase = nullptr;
  h->d_ptotal = nullptr;
  h->d_proff = h->d_pcstart = nullptr;
  h->d_ppos = h->d_psrc = nullptr;
  h->d_pX = nullptr;
  h->total_ptiles = h->total_pbins = h->total_ppieces = 0;
  h->total_punits = 0;
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
    // worst-case padding: 3 slots per chunk, one chunk per source tile
    const uint32_t cap = kPRegion - 3 * S;
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
  for (uint32_t r = 0; r < N; ++r) {  // piece ranges are set below; keep them contiguous
    h->inst[r].ppiece_base = 0;
    h->inst[r].n_ppiece = 0;
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
  uint32_t *d_bad = nullptr;
  chk(dalloc(&h->d_pbin, std::max<uint32_t>(nbins, 1)));
  chk(dalloc(&h->d_ptbase, tiles + 1));
  chk(dalloc(&h->d_ptotal, tiles + 2));  // + the invalid-column flag, + the tile -> realisation map below
  chk(dalloc(&h->d_proff, std::max<uint64_t>(mat, 1)));
  chk(dalloc(&h->d_pcstart, std::max<uint64_t>(mat, 1)));
  chk(dalloc(&h->d_ppos, h->total_nnz + 8));
  // kept with the handle: a free here would synchronise the device
  chk(dalloc(&h->d_ptile_inst, tiles));
  uint32_t *d_tile_inst = h->d_ptile_inst;
  if (e != cudaSuccess) return fail(CB_ERR_OOM, "two-phase format: allocate");
  d_bad = h->d_ptotal + tiles;
  // every copy of the upload has landed on `s` before the format reads it
  for (const CopyGroup &g : groups) chk(cudaStreamWaitEvent(s, g.ev, 0));
  if (nbins) chk(stage_h2d(h->d_pbin, bins.data(), nbins * sizeof(PBin), s));
  chk(stage_h2d(d_tile_inst, tile_inst.data(), tiles * 4, s));
  chk(stage_h2d(h->d_inst, h->inst.data(), N * sizeof(InstDesc), s));
  chk(cudaMemsetAsync(d_bad, 0, 4, s));
  const size_t shm_count = (size_t)pns_max * 4;
  const size_t shm_fill = (size_t)pns_max * 16;
  if (e == cudaSuccess && shm_fill > 48 * 1024)
    chk(cudaFuncSetAttribute(pfill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_fill));
  if (e == cudaSuccess && nbins)
    pcount_kernel<<<nbins, kBuildThreads, shm_count, s>>>(h->d_inst, h->d_pbin, h->row_ptr, h->col,
                                                          h->d_proff, d_bad);
  if (e == cudaSuccess)
    pcolscan_kernel<<<tiles, kBuildThreads, 0, s>>>(h->d_inst, d_tile_inst, h->d_proff,
                                                    h->d_pcstart, h->d_ptotal);
  chk(cudaGetLastError());
  std::vector<uint32_t> tot(tiles + 1);
  chk(cudaMemcpyAsync(tot.data(), h->d_ptotal, (tiles + 1) * 4, cudaMemcpyDeviceToHost, s));
  chk(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return fail(CB_ERR_CUDA, "two-phase format: count");
  if (tot[tiles]) return fail(CB_ERR_ARG, "cb_graph_upload: a column index is >= n");
  // stream bases per source tile and the phase-1 pieces
  std::vector<uint64_t> tbase(tiles + 1);
  std::vector<PPiece> pieces;
  uint64_t u = 0;
  uint32_t g = 0;
  for (uint32_t r = 0; r < N; ++r) {
    InstDesc &I = h->inst[r];
    I.ppiece_base = (uint32_t)pieces.size();
    for (uint32_t t = 0; I.pb && t < I.pns; ++t, ++g) {
      tbase[g] = u;
      for (uint32_t p = 0; p < tot[g]; p += kPPieceUnits)
        pieces.push_back(PPiece{u + p, std::min(kPPieceUnits, tot[g] - p), r, t, 0});
      u += tot[g];
    }
    I.n_ppiece = (uint32_t)pieces.size() - I.ppiece_base;
  }
  tbase[tiles] = u;
  h->total_punits = u;
  h->total_ppieces = (uint32_t)pieces.size();
  chk(dalloc(&h->d_ppiece, std::max<size_t>(pieces.size(), 1)));
  chk(dalloc(&h->d_psrc, 4 * u + 8));
  chk(dalloc(&h->d_pX, 4 * u + 8));
  if (e != cudaSuccess) return fail(CB_ERR_OOM, "two-phase format: allocate stream");
  chk(stage_h2d(h->d_ptbase, tbase.data(), (tiles + 1) * 8, s));
  if (!pieces.empty()) chk(stage_h2d(h->d_ppiece, pieces.data(), pieces.size() * sizeof(PPiece), s));
  chk(stage_h2d(h->d_inst, h->inst.data(), N * sizeof(InstDesc), s));
  // padding slots read node 0 of their tile: harmless, never summed
  chk(cudaMemsetAsync(h->d_psrc, 0, (4 * u + 8) * 2, s));
  if (e == cudaSuccess && nbins)
    pfill_kernel<<<nbins, kBuildThreads, shm_fill, s>>>(h->d_inst, h->d_pbin, h->row_ptr, h->col,
                                                        h->d_proff, h->d_pcstart, h->d_ptbase,
                                                        h->d_ppos, h->d_psrc);
  chk(cudaGetLastError());
  chk(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return fail(CB_ERR_CUDA, "two-phase format: fill");
  return CB_OK;
}

}  // namespace cb
