// On-device generation of the background realisations, each with one
// embedded target: the N graphs that eq. 5 sums over (paper, "Multiple
// backgrounds scenario"), built straight into a handle so that they never
// cross the host-device link.  Three models, each a reading of the paper's
// ER / small-world / scale-free backgrounds in which every decision is
// integer arithmetic on one counter-based generator, so that a CPU statement
// of the same definition can be compared bit for bit.
//
// Generator: SplitMix64 in counter form, output(c) = mix(seed + (c + 1) G)
// with G = 0x9E3779B97F4A7C15 and mix the generator's output function
// (Steele, Lea & Flood, OOPSLA 2014).  Realisation r makes draws
// t = 0 .. D_r - 1 with counter c = r * 2^32 + t; z is the output.
//  * ER (a fixed-draw G(n, M) reading): D_r = M_r; draw t is the pair
//    u = (hi32(z) n_r) >> 32, v = (lo32(z) n_r) >> 32.
//  * WS (Watts & Strogatz): D_r = n_r k/2; draw t = i k/2 + (d - 1) is the
//    ring edge (i, (i + d) mod n_r), d = 1..k/2, rewired to
//    v = (lo32(z) n_r) >> 32 when hi32(z) < floor(p 2^32).
//  * BA (Barabasi & Albert, by the endpoint list of Batagelj & Brandes):
//    nodes 0..m-1 are seeds; draw t is edge t of new node m + t/m; the first
//    new node links to the m seeds, and a later one to the endpoint at a
//    uniform position of the list of all earlier new nodes' edge endpoints,
//    a degree-proportional pick (see ba_target).
// In every model self-loops are dropped, repeated pairs collapse (so a WS
// rewiring onto an existing edge, or a BA node drawing one target twice,
// leaves fewer edges), the target's edges are OR-ed into every realisation
// (those with an endpoint >= n_r are skipped), and rows come out sorted: a
// simple undirected graph as a symmetric CSR pattern.
//
// Construction: count the entries of every row (atomics), prefix, scatter
// (atomic cursors), sort and de-duplicate each row, prefix again, compact.
// The atomics only decide where an entry lands before its row is sorted, so
// the result does not depend on their order.  The handle is then built by
// cb_graph_upload from the device arrays.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "cb_internal.cuh"

namespace cb {
namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr uint32_t kGenThreads = 256;
constexpr uint32_t kScanItems = 4;                       // per thread
constexpr uint32_t kScanBlock = 1024 * kScanItems;       // elements per scan CTA

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

enum GenKind : int { kGenER = 0, kGenWS = 1, kGenBA = 2 };

struct GenArgs {
  uint32_t n_inst;
  const uint32_t *n;         // [N] nodes per realisation
  const uint64_t *node_off;  // [N + 1] prefix of n
  const uint64_t *draw_off;  // [N + 1] prefix of the draws
  uint64_t seed;
  const uint32_t *tedges;    // [E][2] target edges
  uint32_t n_tedges;
  uint64_t items;            // draws + N * E
  int kind;
  uint32_t k_half;           // WS: ring neighbours per side
  uint64_t p32;              // WS: rewire when hi32(z) < p32 = floor(p 2^32)
  uint32_t m_ba;             // BA: edges per new node (and seeds)
};

__device__ __forceinline__ uint64_t gen_z(const GenArgs &a, uint32_t r, uint64_t t) {
  return sm64_mix(a.seed + ((((uint64_t)r << 32) + t) + 1) * kGolden);
}

// BA target of edge t of realisation r: edge t belongs to new node
// m + t / m and points at the endpoint at a uniform position of the
// endpoint list of the edges of all earlier new nodes (positions
// [0, 2 m T), T = t / m; even position 2e' holds the new node of edge e',
// odd position 2e' + 1 its target).  The first new node (T = 0) links to the
// m seeds.  An odd position is resolved through edge e', an earlier edge, so
// the walk ends; it takes about two steps on average.
__device__ __forceinline__ uint32_t ba_target(const GenArgs &a, uint32_t r, uint64_t t) {
  const uint64_t m = a.m_ba;
  for (;;) {
    const uint64_t T = t / m;
    if (T == 0) return (uint32_t)t;  // seed t
    const uint64_t z = gen_z(a, r, t);
    const uint64_t pos = ((z & 0xffffffffull) * (2 * m * T)) >> 32;
    if (!(pos & 1)) return (uint32_t)(m + (pos >> 1) / m);
    t = pos >> 1;
  }
}

// Realisation of draw g (g < D): draw_off[r] <= g < draw_off[r + 1].
__device__ __forceinline__ uint32_t draw_owner(const GenArgs &a, uint64_t g) {
  uint32_t lo = 0, hi = a.n_inst;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a.draw_off[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

// Realisation of row i: node_off[r] <= i < node_off[r + 1].
__device__ __forceinline__ uint32_t node_owner(const GenArgs &a, uint64_t i) {
  uint32_t lo = 0, hi = a.n_inst;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a.node_off[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// Work item g -> realisation r and pair (u, v); false when it makes no edge.
// A draw (g < D) comes in with r already its owner; a target-edge item
// (g >= D) sets r here.
__device__ __forceinline__ bool gen_item(const GenArgs &a, uint64_t g, uint64_t D, uint32_t &r,
                                         uint32_t &u, uint32_t &v) {
  if (g < D) {
    const uint64_t t = g - a.draw_off[r];
    const uint64_t nr = a.n[r];
    if (a.kind == kGenER) {
      const uint64_t z = gen_z(a, r, t);
      u = (uint32_t)(((z >> 32) * nr) >> 32);
      v = (uint32_t)(((z & 0xffffffffull) * nr) >> 32);
    } else if (a.kind == kGenWS) {
      const uint64_t i = t / a.k_half, d = t % a.k_half + 1;
      const uint64_t z = gen_z(a, r, t);
      u = (uint32_t)i;
      v = (uint32_t)((i + d) % nr);
      if ((z >> 32) < a.p32) v = (uint32_t)(((z & 0xffffffffull) * nr) >> 32);  // rewired
    } else {
      u = (uint32_t)(a.m_ba + t / a.m_ba);
      v = ba_target(a, r, t);
    }
  } else {
    const uint64_t q = g - D;
    r = (uint32_t)(q / a.n_tedges);
    const uint32_t e = (uint32_t)(q % a.n_tedges);
    u = a.tedges[2 * e];
    v = a.tedges[2 * e + 1];
    if (u >= a.n[r] || v >= a.n[r]) return false;
  }
  return u != v;
}

// The count and fill kernels give each CTA one chunk of kGenChunk
// consecutive work items (thread t takes items base + j * kGenThreads + t).
// CTAs are dispatched in order, so the items in flight belong to one or two
// realisations and the rows they touch (the realisation's degree or cursor
// array and its entry range) stay in L2 while they are written.  The owner
// of a thread's first draw is found by bisection; later items move it on.
constexpr uint32_t kGenItems = 8;
constexpr uint32_t kGenChunk = kGenThreads * kGenItems;

__device__ __forceinline__ void advance_owner(const GenArgs &a, uint64_t g, uint64_t D,
                                              uint32_t &r) {
  if (g < D)
    while (a.draw_off[r + 1] <= g) ++r;
}

__global__ void __launch_bounds__(kGenThreads) gen_count_kernel(GenArgs a, uint32_t *deg) {
  const uint64_t D = a.draw_off[a.n_inst];
  const uint64_t g0 = blockIdx.x * (uint64_t)kGenChunk + threadIdx.x;
  uint32_t r0 = g0 < D ? draw_owner(a, g0) : 0;
#pragma unroll
  for (uint32_t j = 0; j < kGenItems; ++j) {
    const uint64_t g = g0 + (uint64_t)j * kGenThreads;
    if (g >= a.items) break;
    advance_owner(a, g, D, r0);
    uint32_t r = r0, u, v;
    if (!gen_item(a, g, D, r, u, v)) continue;
    atomicAdd(deg + a.node_off[r] + u, 1u);
    atomicAdd(deg + a.node_off[r] + v, 1u);
  }
}

// cursor[row] counts from the realisation's first entry (32-bit atomics).
// All of a thread's cursor increments are issued before its first store, so
// up to 2 kGenItems returning atomics are in flight per thread.
__global__ void __launch_bounds__(kGenThreads) gen_fill_kernel(GenArgs a,
                                                               const uint64_t *__restrict__ ebase,
                                                               uint32_t *__restrict__ cursor,
                                                               uint32_t *__restrict__ raw) {
  const uint64_t D = a.draw_off[a.n_inst];
  const uint64_t g0 = blockIdx.x * (uint64_t)kGenChunk + threadIdx.x;
  uint32_t r0 = g0 < D ? draw_owner(a, g0) : 0;
  uint32_t rr[kGenItems], uu[kGenItems], vv[kGenItems], pu[kGenItems], pv[kGenItems];
  uint32_t live = 0;
#pragma unroll
  for (uint32_t j = 0; j < kGenItems; ++j) {
    const uint64_t g = g0 + (uint64_t)j * kGenThreads;
    rr[j] = uu[j] = vv[j] = 0;
    if (g >= a.items) continue;
    advance_owner(a, g, D, r0);
    rr[j] = r0;
    if (gen_item(a, g, D, rr[j], uu[j], vv[j])) live |= 1u << j;
  }
#pragma unroll
  for (uint32_t j = 0; j < kGenItems; ++j) {
    pu[j] = pv[j] = 0;
    if (!(live >> j & 1u)) continue;
    const uint64_t row0 = a.node_off[rr[j]];
    pu[j] = atomicAdd(cursor + row0 + uu[j], 1u);
    pv[j] = atomicAdd(cursor + row0 + vv[j], 1u);
  }
#pragma unroll
  for (uint32_t j = 0; j < kGenItems; ++j) {
    if (!(live >> j & 1u)) continue;
    const uint64_t eb = ebase[rr[j]];
    raw[eb + pu[j]] = vv[j];
    raw[eb + pv[j]] = uu[j];
  }
}

__global__ void __launch_bounds__(kGenThreads) gen_cursor_kernel(GenArgs a, const uint64_t *off,
                                                                 const uint64_t *ebase,
                                                                 uint32_t *cursor, uint64_t rows) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < rows;
       i += (uint64_t)gridDim.x * blockDim.x)
    cursor[i] = (uint32_t)(off[i] - ebase[node_owner(a, i)]);
}

// Sort each row ascending and drop repeats; deg[i] becomes the number of
// distinct columns.  A warp takes kRowChunk consecutive rows, whose entries
// are one contiguous range of raw.  When that range fits kSortStage words
// the warp copies it into shared memory and each lane sorts its own row of
// up to 32 entries in registers (a fixed bitonic network, padded with
// UINT32_MAX), writes the distinct values to the front of the row's segment
// and the warp copies the range back; entries after a row's distinct count
// are left as they were (only deg[i] of them are read later).  Longer rows,
// and every row of a chunk that does not fit, take the warp path below.
constexpr uint32_t kRowChunk = 32;
constexpr uint32_t kSortStage = 1024;  // words of shared memory per warp

__device__ __forceinline__ void bitonic32_regs(uint32_t (&v)[32]) {
#pragma unroll
  for (uint32_t k = 2; k <= 32; k <<= 1)
#pragma unroll
    for (uint32_t j = k >> 1; j > 0; j >>= 1)
#pragma unroll
      for (uint32_t i = 0; i < 32; ++i) {
        const uint32_t l = i ^ j;
        if (l > i) {
          const uint32_t lo = min(v[i], v[l]), hi = max(v[i], v[l]);
          const bool up = (i & k) == 0;
          v[i] = up ? lo : hi;
          v[l] = up ? hi : lo;
        }
      }
}

__device__ __forceinline__ uint32_t bitonic_cx(uint32_t x, uint32_t y, bool keep_min) {
  return keep_min ? min(x, y) : max(x, y);
}

// Rows of more than 64 raw entries are sorted by whole CTAs in shared memory
// (gen_sort_block_kernel): up to kSortMid entries by small CTAs, up to
// kSortBig by large ones; their rows are listed from the two ends of one
// array.  Rows beyond kSortBig (a degree above 32768 before de-duplication)
// keep a serial insertion sort.
constexpr uint32_t kSortMid = 1024, kSortBig = 32768;

// The warp path for row i (entries p[0, d)): up to 64 entries are sorted
// across the warp by a bitonic network over shuffles (entry e in lane
// e % 32, register e / 32), as wide as the next power of two of d.  Returns
// the row's degree to record (its raw length when a CTA sorts it later).
__device__ uint32_t sort_row_warp(uint32_t *p, uint32_t d, uint64_t i, uint64_t rows,
                                  uint32_t *long_rows, uint32_t *long_cnt, uint32_t lane) {
  if (d > 64 && d <= kSortBig) {  // a CTA sorts it and sets its degree
    if (lane == 0) {
      if (d <= kSortMid)
        long_rows[atomicAdd(&long_cnt[0], 1u)] = (uint32_t)i;
      else
        long_rows[rows - 1 - atomicAdd(&long_cnt[1], 1u)] = (uint32_t)i;
    }
    return d;
  }
  if (d > 64) {
    uint32_t w = 0;
    if (lane == 0) {
      for (uint32_t q = 1; q < d; ++q) {
        const uint32_t x = p[q];
        uint32_t s = q;
        while (s > 0 && p[s - 1] > x) {
          p[s] = p[s - 1];
          --s;
        }
        p[s] = x;
      }
      for (uint32_t q = 0; q < d; ++q)
        if (w == 0 || p[q] != p[w - 1]) p[w++] = p[q];
    }
    return __shfl_sync(0xffffffffu, w, 0);
  }
  uint32_t x0 = lane < d ? p[lane] : 0xffffffffu;
  uint32_t x1 = lane + 32 < d ? p[lane + 32] : 0xffffffffu;
  uint32_t kmax = 2;
  while (kmax < d) kmax <<= 1;
  for (uint32_t kk = 2; kk <= kmax; kk <<= 1) {
    for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
      if (j == 32) {  // partner is the other register of the same lane (kk = 64)
        const uint32_t lo = min(x0, x1), hi = max(x0, x1);
        x0 = lo;
        x1 = hi;
        continue;
      }
      const bool lower = (lane & j) == 0;
      const uint32_t y0 = __shfl_xor_sync(0xffffffffu, x0, j);
      x0 = bitonic_cx(x0, y0, lower == ((lane & kk) == 0));
      if (kmax == 64) {
        const uint32_t y1 = __shfl_xor_sync(0xffffffffu, x1, j);
        x1 = bitonic_cx(x1, y1, lower == (((lane + 32) & kk) == 0));
      }
    }
  }
  // distinct values: keep an entry unless it equals its predecessor
  const uint32_t pr0 = __shfl_up_sync(0xffffffffu, x0, 1);
  const uint32_t pr1 = __shfl_up_sync(0xffffffffu, x1, 1);
  const uint32_t last0 = __shfl_sync(0xffffffffu, x0, 31);
  const bool k0 = lane < d && (lane == 0 || x0 != pr0);
  const bool k1 = lane + 32 < d && (lane == 0 ? x1 != last0 : x1 != pr1);
  const uint32_t b0 = __ballot_sync(0xffffffffu, k0), b1 = __ballot_sync(0xffffffffu, k1);
  const uint32_t lt = (1u << lane) - 1u;
  __syncwarp();  // every lane has read its entries before any is overwritten
  if (k0) p[__popc(b0 & lt)] = x0;
  if (k1) p[__popc(b0) + __popc(b1 & lt)] = x1;
  return __popc(b0) + __popc(b1);
}

__global__ void __launch_bounds__(kGenThreads) gen_sort_kernel(const uint64_t *__restrict__ off,
                                                               uint32_t *__restrict__ raw,
                                                               uint32_t *__restrict__ deg,
                                                               uint64_t rows,
                                                               uint32_t *__restrict__ long_rows,
                                                               uint32_t *__restrict__ long_cnt) {
  __shared__ uint32_t s_stage[kGenThreads / 32][kSortStage];
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t i0 =
      (blockIdx.x * (uint64_t)(kGenThreads / 32) + (threadIdx.x >> 5)) * kRowChunk;
  if (i0 >= rows) return;
  const uint32_t nr = (uint32_t)(rows - i0 < kRowChunk ? rows - i0 : kRowChunk);
  const uint64_t o_lane = lane < nr ? off[i0 + lane] : 0, o_end = off[i0 + nr];
  const uint64_t o_next = __shfl_sync(0xffffffffu, o_lane, (lane + 1) & 31);
  const uint32_t d_lane = lane < nr ? (uint32_t)((lane + 1 < nr ? o_next : o_end) - o_lane) : 0;
  const uint64_t base = __shfl_sync(0xffffffffu, o_lane, 0);
  const uint64_t total = o_end - base;
  uint32_t my_deg = d_lane;
  uint32_t warp_rows;  // rows left to the warp path
  if (total <= kSortStage) {
    uint32_t *sw = s_stage[threadIdx.x >> 5];
    for (uint32_t q = lane; q < total; q += 32) sw[q] = raw[base + q];
    __syncwarp();
    if (d_lane <= 32 && lane < nr) {
      uint32_t *seg = sw + (o_lane - base);
      uint32_t v[32];
#pragma unroll
      for (uint32_t q = 0; q < 32; ++q) v[q] = q < d_lane ? seg[q] : 0xffffffffu;
      bitonic32_regs(v);
      uint32_t w = 0;
#pragma unroll
      for (uint32_t q = 0; q < 32; ++q)
        if (v[q] != 0xffffffffu && (q == 0 || v[q] != v[q - 1])) seg[w++] = v[q];
      my_deg = w;
    }
    __syncwarp();
    for (uint32_t q = lane; q < total; q += 32) raw[base + q] = sw[q];
    __syncwarp();  // the copy-back is visible to the warp path's loads
    warp_rows = __ballot_sync(0xffffffffu, d_lane > 32);
  } else {
    warp_rows = __ballot_sync(0xffffffffu, lane < nr);
  }
  while (warp_rows) {
    const uint32_t k = __ffs(warp_rows) - 1;
    warp_rows &= warp_rows - 1;
    const uint64_t st = __shfl_sync(0xffffffffu, o_lane, k);
    const uint32_t d = __shfl_sync(0xffffffffu, d_lane, k);
    const uint32_t w = sort_row_warp(raw + st, d, i0 + k, rows, long_rows, long_cnt, lane);
    if (lane == k) my_deg = w;
  }
  if (lane < nr) deg[i0 + lane] = my_deg;
}

// Compact the distinct columns into the concatenated CSR and write each
// realisation's local row_ptr (n_r + 1 entries at node_off[r] + r).  A warp
// takes kRowChunk consecutive rows; lane j reads the offsets of row i0 + j
// and writes its row_ptr entry, then the rows are copied four at a time
// (all four rows' loads before their stores).
__global__ void __launch_bounds__(kGenThreads) gen_compact_kernel(
    GenArgs a, const uint64_t *__restrict__ off, const uint32_t *__restrict__ raw,
    const uint64_t *__restrict__ off2, uint32_t *__restrict__ col, uint32_t *__restrict__ rp,
    uint64_t rows) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t i0 =
      (blockIdx.x * (uint64_t)(kGenThreads / 32) + (threadIdx.x >> 5)) * kRowChunk;
  if (i0 >= rows) return;
  const uint32_t nr = (uint32_t)(rows - i0 < kRowChunk ? rows - i0 : kRowChunk);
  uint64_t src = 0, dst = 0;
  uint32_t d = 0;
  if (lane < nr) {
    const uint64_t i = i0 + lane;
    src = off[i];
    dst = off2[i];
    const uint64_t dst_end = off2[i + 1];
    d = (uint32_t)(dst_end - dst);
    const uint32_t r = node_owner(a, i);
    const uint64_t row0 = a.node_off[r], base = off2[row0];
    rp[row0 + r + (i - row0)] = (uint32_t)(dst - base);
    if (i + 1 == a.node_off[r + 1]) rp[row0 + r + (i - row0) + 1] = (uint32_t)(dst_end - base);
  }
  for (uint32_t k = 0; k < nr; k += 4) {
    uint64_t sk[4], dk[4];
    uint32_t nk[4], val[4];
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      sk[q] = __shfl_sync(0xffffffffu, src, k + q);
      dk[q] = __shfl_sync(0xffffffffu, dst, k + q);
      nk[q] = __shfl_sync(0xffffffffu, d, k + q);  // 0 for rows past nr
      val[q] = lane < nk[q] ? raw[sk[q] + lane] : 0u;
    }
#pragma unroll
    for (uint32_t q = 0; q < 4; ++q) {
      if (lane < nk[q]) col[dk[q] + lane] = val[q];
      for (uint32_t t = lane + 32; t < nk[q]; t += 32) col[dk[q] + t] = raw[sk[q] + t];
    }
  }
}

// Exclusive prefix of u32 counts into u64 offsets: out[0..n], out[n] = total.
// Level 1: each CTA scans kScanBlock elements and leaves its total;
// level 2: one CTA scans the totals; level 3: offsets are added back.
__global__ void __launch_bounds__(1024) scan_block_kernel(const uint32_t *in, uint64_t n,
                                                          uint64_t *out, uint64_t *bsum) {
  __shared__ uint64_t s_warp[32];
  const uint64_t base = (uint64_t)blockIdx.x * kScanBlock + (uint64_t)threadIdx.x * kScanItems;
  uint64_t v[kScanItems], t = 0;
#pragma unroll
  for (uint32_t q = 0; q < kScanItems; ++q) {
    v[q] = base + q < n ? in[base + q] : 0u;
    t += v[q];
  }
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t incl = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = s_warp[lane], wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if ((int)lane >= o) wi += y;
    }
    s_warp[lane] = wi - w;  // exclusive over warps
    if (lane == 31) bsum[blockIdx.x] = wi;
  }
  __syncthreads();
  uint64_t run = s_warp[warp] + incl - t;
#pragma unroll
  for (uint32_t q = 0; q < kScanItems; ++q) {
    if (base + q < n) out[base + q] = run;
    run += v[q];
  }
}

__global__ void __launch_bounds__(1024) scan_sums_kernel(uint64_t *bsum, uint64_t nb,
                                                         uint64_t *total) {
  __shared__ uint64_t s_warp[32];
  __shared__ uint64_t s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t c = 0; c < nb; c += 1024) {
    const uint64_t i = c + threadIdx.x;
    const uint64_t x = i < nb ? bsum[i] : 0;
    uint64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint64_t w = s_warp[lane], wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, wi, o);
        if ((int)lane >= o) wi += y;
      }
      s_warp[lane] = wi - w;
    }
    __syncthreads();
    const uint64_t carry = s_carry;
    if (i < nb) bsum[i] = carry + s_warp[warp] + incl - x;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = carry + s_warp[warp] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = s_carry;
}

__global__ void scan_add_kernel(uint64_t *out, uint64_t n, const uint64_t *bsum,
                                const uint64_t *total) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] += bsum[i / kScanBlock];
  if (i == 0) out[n] = *total;
}

}  // namespace

cudaError_t exclusive_scan(const uint32_t *in, uint64_t n, uint64_t *out, uint64_t *bsum,
                           cudaStream_t s) {
  const uint64_t nb = std::max<uint64_t>((n + kScanBlock - 1) / kScanBlock, 1);
  scan_block_kernel<<<(uint32_t)nb, 1024, 0, s>>>(in, n, out, bsum);
  scan_sums_kernel<<<1, 1024, 0, s>>>(bsum, nb, bsum + nb);
  scan_add_kernel<<<(uint32_t)((n + 256) / 256), 256, 0, s>>>(out, n, bsum, bsum + nb);
  return cudaGetLastError();
}

namespace {

__global__ void gather_bounds_kernel(const uint64_t *off2, const uint64_t *node_off,
                                     uint32_t n_inst, uint64_t *bound) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r <= n_inst) bound[r] = off2[node_off[r]];
}

uint32_t grid_for(uint64_t work) {
  const uint64_t g = (work + kGenThreads - 1) / kGenThreads;
  return (uint32_t)std::min<uint64_t>(std::max<uint64_t>(g, 1), 152ull * 16);
}

// one CTA per `per_cta` units of work (the chunked kernels; no grid-stride loop)
uint64_t chunk_grid(uint64_t work, uint64_t per_cta) {
  return std::max<uint64_t>((work + per_cta - 1) / per_cta, 1);
}
constexpr uint64_t kRowsPerCta = kRowChunk * (kGenThreads / 32);

// One CTA per listed row: bitonic sort of the row (padded with UINT32_MAX
// to a power of two) in shared memory, then thread 0 writes the distinct
// values back and sets the row's degree.  rows_from_end: the row list is
// read from the end of the array (the large rows).
template <uint32_t CAP>
__global__ void gen_sort_block_kernel(const uint64_t *off, uint32_t *raw, uint32_t *deg,
                                      const uint32_t *long_rows, uint64_t rows,
                                      bool rows_from_end) {
  extern __shared__ uint32_t s_row[];
  const uint32_t i = rows_from_end ? long_rows[rows - 1 - blockIdx.x] : long_rows[blockIdx.x];
  uint32_t *p = raw + off[i];
  const uint32_t d = (uint32_t)(off[i + 1] - off[i]);
  uint32_t P = 1;
  while (P < d) P <<= 1;
  for (uint32_t q = threadIdx.x; q < P; q += blockDim.x) s_row[q] = q < d ? p[q] : 0xffffffffu;
  __syncthreads();
  for (uint32_t k = 2; k <= P; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t t = threadIdx.x; t < P; t += blockDim.x) {
        const uint32_t u = t ^ j;
        if (u > t) {
          const uint32_t a = s_row[t], b = s_row[u];
          const bool asc = (t & k) == 0;
          if ((a > b) == asc) {
            s_row[t] = b;
            s_row[u] = a;
          }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x == 0) {
    uint32_t w = 0;
    for (uint32_t q = 0; q < d; ++q)
      if (q == 0 || s_row[q] != s_row[q - 1]) p[w++] = s_row[q];
    deg[i] = w;
  }
}

// device buffers of one generation call, freed on every exit path
struct GenBuffers {
  std::vector<void *> ptrs;
  template <typename P>
  cudaError_t alloc(P **p, size_t count) {
    cudaError_t e = dev_alloc_n(p, count);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  void release(void *p) {  // p now belongs to someone else
    ptrs.erase(std::remove(ptrs.begin(), ptrs.end(), p), ptrs.end());
  }
  ~GenBuffers() {
    for (void *p : ptrs) dev_free(p);
  }
};

}  // namespace
}  // namespace cb

using namespace cb;

// The construction shared by the three models: per-realisation draw counts
// in `draws`; the model's parameters in `kp` (kind, k_half, p32, m_ba).
static int generate(const GenArgs &kp, const char *who, uint32_t n_inst, const uint32_t *n,
                    const std::vector<uint64_t> &draws, uint64_t seed, uint32_t n_tedges,
                    const uint32_t *tedges, void *stream, cb_graph **out) {
  auto fail = [&](const char *what) { return set_error(CB_ERR_ARG, std::string(who) + ": " + what); };
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<uint64_t> node_off(n_inst + 1, 0), draw_off(n_inst + 1, 0);
  for (uint32_t r = 0; r < n_inst; ++r) {
    if (draws[r] + n_tedges >= (1ull << 31))  // 2 entries per draw, 32-bit cursors
      return fail("need draws + n_tedges < 2^31 per realisation");
    node_off[r + 1] = node_off[r] + n[r];
    draw_off[r + 1] = draw_off[r] + draws[r];
  }
  for (uint32_t e = 0; e < 2 * n_tedges; ++e)
    if (tedges[e] >= (1u << 31)) return fail("target edge endpoint out of range");
  const uint64_t rows = node_off[n_inst];
  if (rows >= 0xffffffffull) return fail("need fewer than 2^32 nodes over all realisations");
  const uint64_t items = draw_off[n_inst] + (uint64_t)n_inst * n_tedges;
  if (chunk_grid(items, kGenChunk) >= (1ull << 31)) return fail("too many draws");

  GenBuffers B;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  uint32_t *d_n = nullptr, *d_tedges = nullptr, *deg = nullptr, *raw = nullptr, *col = nullptr,
           *rp = nullptr;
  uint64_t *d_node_off = nullptr, *d_draw_off = nullptr, *off = nullptr, *off2 = nullptr,
           *bsum = nullptr, *bound = nullptr;
  uint32_t *cursor = nullptr;
  uint64_t *ebase = nullptr;
  chk(B.alloc(&d_n, n_inst));
  chk(B.alloc(&d_node_off, n_inst + 1));
  chk(B.alloc(&d_draw_off, n_inst + 1));
  chk(B.alloc(&d_tedges, std::max<size_t>(2 * (size_t)n_tedges, 1)));
  chk(B.alloc(&deg, rows));
  chk(B.alloc(&off, rows + 1));
  chk(B.alloc(&off2, rows + 1));
  chk(B.alloc(&cursor, rows));
  chk(B.alloc(&bsum, (rows + kScanBlock - 1) / kScanBlock + 2));
  chk(B.alloc(&bound, n_inst + 1));
  chk(B.alloc(&ebase, n_inst + 1));
  uint32_t *long_rows = nullptr, *long_cnt = nullptr;
  chk(B.alloc(&long_rows, std::max<uint64_t>(rows, 1)));
  chk(B.alloc(&long_cnt, 2));
  if (e != cudaSuccess) return cuda_error(e, (std::string(who) + ": allocate").c_str());
  chk(cudaMemcpyAsync(d_n, n, n_inst * 4, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(d_node_off, node_off.data(), (n_inst + 1) * 8, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(d_draw_off, draw_off.data(), (n_inst + 1) * 8, cudaMemcpyHostToDevice, s));
  if (n_tedges) chk(cudaMemcpyAsync(d_tedges, tedges, 8ull * n_tedges, cudaMemcpyHostToDevice, s));
  chk(cudaMemsetAsync(deg, 0, rows * 4, s));
  GenArgs a = kp;
  a.n_inst = n_inst;
  a.n = d_n;
  a.node_off = d_node_off;
  a.draw_off = d_draw_off;
  a.seed = seed;
  a.tedges = d_tedges;
  a.n_tedges = n_tedges;
  a.items = items;
  if (e == cudaSuccess) {
    gen_count_kernel<<<(uint32_t)chunk_grid(items, kGenChunk), kGenThreads, 0, s>>>(a, deg);
    chk(cudaGetLastError());
    chk(exclusive_scan(deg, rows, off, bsum, s));
  }
  uint64_t entries = 0;
  chk(cudaMemcpyAsync(&entries, off + rows, 8, cudaMemcpyDeviceToHost, s));
  chk(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return cuda_error(e, (std::string(who) + ": count").c_str());
  chk(B.alloc(&raw, std::max<uint64_t>(entries, 1)));
  if (e != cudaSuccess) return cuda_error(e, (std::string(who) + ": allocate entries").c_str());
  if (e == cudaSuccess) {
    gather_bounds_kernel<<<(n_inst + 256) / 256, 256, 0, s>>>(off, d_node_off, n_inst, ebase);
    gen_cursor_kernel<<<grid_for(rows), kGenThreads, 0, s>>>(a, off, ebase, cursor, rows);
    gen_fill_kernel<<<(uint32_t)chunk_grid(items, kGenChunk), kGenThreads, 0, s>>>(a, ebase, cursor,
                                                                                raw);
    chk(cudaMemsetAsync(long_cnt, 0, 8, s));
    gen_sort_kernel<<<(uint32_t)chunk_grid(rows, kRowsPerCta), kGenThreads, 0, s>>>(
        off, raw, deg, rows, long_rows, long_cnt);
    chk(cudaGetLastError());
    uint32_t nl[2] = {0, 0};
    chk(cudaMemcpyAsync(nl, long_cnt, 8, cudaMemcpyDeviceToHost, s));
    chk(cudaStreamSynchronize(s));
    if (e == cudaSuccess && nl[0])
      gen_sort_block_kernel<kSortMid><<<nl[0], 256, kSortMid * 4, s>>>(off, raw, deg, long_rows,
                                                                      rows, false);
    if (e == cudaSuccess && nl[1]) {
      chk(cudaFuncSetAttribute(gen_sort_block_kernel<kSortBig>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kSortBig * 4)));
      gen_sort_block_kernel<kSortBig><<<nl[1], 1024, kSortBig * 4, s>>>(off, raw, deg, long_rows,
                                                                       rows, true);
    }
    chk(cudaGetLastError());
    chk(exclusive_scan(deg, rows, off2, bsum, s));
    gather_bounds_kernel<<<(n_inst + 256) / 256, 256, 0, s>>>(off2, d_node_off, n_inst, bound);
    chk(cudaGetLastError());
  }
  std::vector<uint64_t> hb(n_inst + 1, 0);
  chk(cudaMemcpyAsync(hb.data(), bound, (n_inst + 1) * 8, cudaMemcpyDeviceToHost, s));
  chk(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return cuda_error(e, (std::string(who) + ": build rows").c_str());
  std::vector<uint64_t> nnz(n_inst);
  for (uint32_t r = 0; r < n_inst; ++r) {
    nnz[r] = hb[r + 1] - hb[r];
    if (nnz[r] >= 0xffffffffull)
      return fail("a realisation has >= 2^32 entries");
  }
  chk(B.alloc(&col, hb[n_inst] + 4));  // + the 16 zero bytes the handle keeps after the columns
  chk(B.alloc(&rp, rows + n_inst));
  if (e != cudaSuccess) return cuda_error(e, (std::string(who) + ": allocate CSR").c_str());
  gen_compact_kernel<<<(uint32_t)chunk_grid(rows, kRowsPerCta), kGenThreads, 0, s>>>(
      a, off, raw, off2, col, rp, rows);
  chk(cudaGetLastError());
  chk(cudaStreamSynchronize(s));  // the upload reads row_ptr back with a plain copy
  if (e != cudaSuccess) return cuda_error(e, (std::string(who) + ": compact").c_str());
  std::vector<const uint32_t *> rpp(n_inst), colp(n_inst);
  for (uint32_t r = 0; r < n_inst; ++r) {
    rpp[r] = rp + node_off[r] + r;
    colp[r] = col + hb[r];
  }
  // the handle takes col and rp over (they are laid out as its own arrays)
  // and builds its tables; the temporaries are freed when B goes out of scope
  const int rc = upload_adopt(n_inst, n, nnz.data(), rpp.data(), colp.data(), col, rp, stream, out);
  if (rc == CB_OK) {
    B.release(col);
    B.release(rp);
  }
  return rc;
}

static int check_common(const char *who, uint32_t n_inst, const uint32_t *n, uint32_t n_tedges,
                        const uint32_t *tedges, cb_graph **out) {
  if (!out) return set_error(CB_ERR_ARG, std::string(who) + ": out is null");
  *out = nullptr;
  if (n_inst == 0 || !n || (n_tedges && !tedges))
    return set_error(CB_ERR_ARG, std::string(who) + ": empty input or null array");
  for (uint32_t r = 0; r < n_inst; ++r)
    if (n[r] == 0) return set_error(CB_ERR_ARG, std::string(who) + ": realisation with n = 0");
  return CB_OK;
}

CB_API int cb_graph_generate_er(uint32_t n_inst, const uint32_t *n, const uint64_t *m_draws,
                                uint64_t seed, uint32_t n_tedges, const uint32_t *tedges,
                                void *stream, cb_graph **out) {
  NvtxRange nvtx_range("cb_graph_generate_er");
  const char *who = "cb_graph_generate_er";
  int rc = check_common(who, n_inst, n, n_tedges, tedges, out);
  if (rc != CB_OK) return rc;
  if (!m_draws) return set_error(CB_ERR_ARG, "cb_graph_generate_er: empty input or null array");
  GenArgs kp{};
  kp.kind = kGenER;
  return generate(kp, who, n_inst, n, std::vector<uint64_t>(m_draws, m_draws + n_inst), seed,
                  n_tedges, tedges, stream, out);
}

CB_API int cb_graph_generate_ws(uint32_t n_inst, const uint32_t *n, uint32_t k, double p,
                                uint64_t seed, uint32_t n_tedges, const uint32_t *tedges,
                                void *stream, cb_graph **out) {
  NvtxRange nvtx_range("cb_graph_generate_ws");
  const char *who = "cb_graph_generate_ws";
  int rc = check_common(who, n_inst, n, n_tedges, tedges, out);
  if (rc != CB_OK) return rc;
  if (k < 2 || (k & 1)) return set_error(CB_ERR_ARG, "cb_graph_generate_ws: k must be even and >= 2");
  if (!(p >= 0.0 && p <= 1.0)) return set_error(CB_ERR_ARG, "cb_graph_generate_ws: need 0 <= p <= 1");
  std::vector<uint64_t> draws(n_inst);
  for (uint32_t r = 0; r < n_inst; ++r) {
    if (k >= n[r]) return set_error(CB_ERR_ARG, "cb_graph_generate_ws: need k < n");
    draws[r] = (uint64_t)n[r] * (k / 2);
  }
  GenArgs kp{};
  kp.kind = kGenWS;
  kp.k_half = k / 2;
  kp.p32 = (uint64_t)std::floor(p * 4294967296.0);  // 2^32 at p = 1: every edge rewired
  return generate(kp, who, n_inst, n, draws, seed, n_tedges, tedges, stream, out);
}

CB_API int cb_graph_generate_ba(uint32_t n_inst, const uint32_t *n, uint32_t m, uint64_t seed,
                                uint32_t n_tedges, const uint32_t *tedges, void *stream,
                                cb_graph **out) {
  NvtxRange nvtx_range("cb_graph_generate_ba");
  const char *who = "cb_graph_generate_ba";
  int rc = check_common(who, n_inst, n, n_tedges, tedges, out);
  if (rc != CB_OK) return rc;
  if (m < 1) return set_error(CB_ERR_ARG, "cb_graph_generate_ba: need m >= 1");
  std::vector<uint64_t> draws(n_inst);
  for (uint32_t r = 0; r < n_inst; ++r) {
    if (n[r] <= m) return set_error(CB_ERR_ARG, "cb_graph_generate_ba: need n > m");
    draws[r] = (uint64_t)m * (n[r] - m);
  }
  GenArgs kp{};
  kp.kind = kGenBA;
  kp.m_ba = m;
  return generate(kp, who, n_inst, n, draws, seed, n_tedges, tedges, stream, out);
}
