// On-device generation of Erdos-Renyi backgrounds with one embedded target:
// the N realisations that eq. 5 sums over (paper, "Multiple backgrounds
// scenario"), built straight into a handle so that they never cross the
// host-device link.
//
// Model (a fixed-draw G(n, M) reading of the paper's ER backgrounds).
// SplitMix64 in counter form, output(c) = mix(seed + (c + 1) G) with
// G = 0x9E3779B97F4A7C15 and mix the generator's output function (Steele,
// Lea & Flood, OOPSLA 2014).  Realisation r takes draws t = 0 .. M_r - 1 with
// counter c = r * 2^32 + t; draw t is the pair u = (hi32(z) n_r) >> 32,
// v = (lo32(z) n_r) >> 32.  Draws with u == v are dropped, repeated pairs
// collapse, the target's edges are OR-ed into every realisation (those with
// an endpoint >= n_r are skipped), and rows come out sorted: a simple
// undirected graph as a symmetric CSR pattern.
//
// Construction: count the entries of every row (atomics), prefix, scatter
// (atomic cursors), sort and de-duplicate each row, prefix again, compact.
// The atomics only decide where an entry lands before its row is sorted, so
// the result does not depend on their order.  The handle is then built by
// cb_graph_upload from the device arrays.
#include <algorithm>
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

struct GenArgs {
  uint32_t n_inst;
  const uint32_t *n;         // [N] nodes per realisation
  const uint64_t *node_off;  // [N + 1] prefix of n
  const uint64_t *draw_off;  // [N + 1] prefix of M
  uint64_t seed;
  const uint32_t *tedges;    // [E][2] target edges
  uint32_t n_tedges;
  uint64_t items;            // draws + N * E
};

// Work item g -> realisation r and pair (u, v); false when it makes no edge.
__device__ __forceinline__ bool gen_item(const GenArgs &a, uint64_t g, uint32_t &r, uint32_t &u,
                                         uint32_t &v) {
  const uint64_t D = a.draw_off[a.n_inst];
  if (g < D) {
    uint32_t lo = 0, hi = a.n_inst;  // draw_off[lo] <= g < draw_off[hi]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (a.draw_off[mid] <= g) lo = mid; else hi = mid;
    }
    r = lo;
    const uint64_t t = g - a.draw_off[r];
    const uint64_t z = sm64_mix(a.seed + ((((uint64_t)r << 32) + t) + 1) * kGolden);
    const uint64_t nr = a.n[r];
    u = (uint32_t)(((z >> 32) * nr) >> 32);
    v = (uint32_t)(((z & 0xffffffffull) * nr) >> 32);
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

__global__ void __launch_bounds__(kGenThreads) gen_count_kernel(GenArgs a, uint32_t *deg) {
  for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < a.items;
       g += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t r, u, v;
    if (!gen_item(a, g, r, u, v)) continue;
    atomicAdd(deg + a.node_off[r] + u, 1u);
    atomicAdd(deg + a.node_off[r] + v, 1u);
  }
}

// cursor[row] counts from the realisation's first entry (32-bit atomics)
__global__ void __launch_bounds__(kGenThreads) gen_fill_kernel(GenArgs a, const uint64_t *ebase,
                                                               uint32_t *cursor, uint32_t *raw) {
  for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < a.items;
       g += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t r, u, v;
    if (!gen_item(a, g, r, u, v)) continue;
    const uint64_t eb = ebase[r];
    raw[eb + atomicAdd(cursor + a.node_off[r] + u, 1u)] = v;
    raw[eb + atomicAdd(cursor + a.node_off[r] + v, 1u)] = u;
  }
}

__global__ void __launch_bounds__(kGenThreads) gen_cursor_kernel(GenArgs a, const uint64_t *off,
                                                                 const uint64_t *ebase,
                                                                 uint32_t *cursor, uint64_t rows) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < rows;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = a.n_inst;  // node_off[lo] <= i < node_off[hi]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (a.node_off[mid] <= i) lo = mid; else hi = mid;
    }
    cursor[i] = (uint32_t)(off[i] - ebase[lo]);
  }
}

// Sort each row ascending and drop repeats, one warp per row; deg[i] becomes
// the number of distinct columns.  Rows of up to 64 entries are sorted in
// registers by a bitonic network over shuffles (entry e of the row sits in
// lane e % 32, register e / 32; unused slots hold UINT32_MAX); longer rows
// (rare: degrees are ~Poisson) fall back to an insertion sort by lane 0.
__device__ __forceinline__ uint32_t bitonic_cx(uint32_t x, uint32_t y, bool keep_min) {
  return keep_min ? min(x, y) : max(x, y);
}

__global__ void __launch_bounds__(kGenThreads) gen_sort_kernel(const uint64_t *off, uint32_t *raw,
                                                               uint32_t *deg, uint64_t rows) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t i = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < rows;
       i += warps) {
    uint32_t *p = raw + off[i];
    const uint32_t d = (uint32_t)(off[i + 1] - off[i]);
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
        deg[i] = w;
      }
      __syncwarp();
      continue;
    }
    uint32_t x0 = lane < d ? p[lane] : 0xffffffffu;
    uint32_t x1 = lane + 32 < d ? p[lane + 32] : 0xffffffffu;
    const uint32_t kmax = d > 32 ? 64u : 32u;
    for (uint32_t k = 2; k <= kmax; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        if (j == 32) {  // partner is the other register of the same lane (k = 64)
          const uint32_t lo = min(x0, x1), hi = max(x0, x1);
          x0 = lo;
          x1 = hi;
          continue;
        }
        const bool lower = (lane & j) == 0;
        const uint32_t y0 = __shfl_xor_sync(0xffffffffu, x0, j);
        x0 = bitonic_cx(x0, y0, lower == ((lane & k) == 0));
        if (kmax == 64) {
          const uint32_t y1 = __shfl_xor_sync(0xffffffffu, x1, j);
          x1 = bitonic_cx(x1, y1, lower == (((lane + 32) & k) == 0));
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
    if (lane == 0) deg[i] = __popc(b0) + __popc(b1);
  }
}

// Compact the distinct columns into the concatenated CSR and write each
// realisation's local row_ptr (n_r + 1 entries at node_off[r] + r).
__global__ void __launch_bounds__(kGenThreads) gen_compact_kernel(GenArgs a, const uint64_t *off,
                                                                  const uint32_t *raw,
                                                                  const uint64_t *off2,
                                                                  uint32_t *col, uint32_t *rp,
                                                                  uint64_t rows) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t i = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < rows;
       i += warps) {
    uint32_t lo = 0, hi = a.n_inst;  // node_off[lo] <= i < node_off[hi]
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (a.node_off[mid] <= i) lo = mid; else hi = mid;
    }
    const uint32_t r = lo;
    const uint64_t base = off2[a.node_off[r]];
    const uint64_t d = off2[i + 1] - off2[i];
    const uint32_t *src = raw + off[i];
    uint32_t *dst = col + off2[i];
    for (uint64_t q = lane; q < d; q += 32) dst[q] = src[q];
    if (lane == 0) {
      const uint64_t local = i - a.node_off[r];
      rp[a.node_off[r] + r + local] = (uint32_t)(off2[i] - base);
      if (i + 1 == a.node_off[r + 1])
        rp[a.node_off[r] + r + local + 1] = (uint32_t)(off2[i + 1] - base);
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

// device buffers of one generation call, freed on every exit path
struct GenBuffers {
  std::vector<void *> ptrs;
  template <typename P>
  cudaError_t alloc(P **p, size_t count) {
    cudaError_t e = dev_alloc_n(p, count);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  ~GenBuffers() {
    for (void *p : ptrs) dev_free(p);
  }
};

}  // namespace
}  // namespace cb

using namespace cb;

CB_API int cb_graph_generate_er(uint32_t n_inst, const uint32_t *n, const uint64_t *m_draws,
                                uint64_t seed, uint32_t n_tedges, const uint32_t *tedges,
                                void *stream, cb_graph **out) {
  NvtxRange nvtx_range("cb_graph_generate_er");
  if (!out) return set_error(CB_ERR_ARG, "cb_graph_generate_er: out is null");
  *out = nullptr;
  if (n_inst == 0 || !n || !m_draws || (n_tedges && !tedges))
    return set_error(CB_ERR_ARG, "cb_graph_generate_er: empty input or null array");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<uint64_t> node_off(n_inst + 1, 0), draw_off(n_inst + 1, 0);
  for (uint32_t r = 0; r < n_inst; ++r) {
    if (n[r] == 0) return set_error(CB_ERR_ARG, "cb_graph_generate_er: realisation with n = 0");
    if (m_draws[r] + n_tedges >= (1ull << 31))  // 2 entries per draw, 32-bit cursors
      return set_error(CB_ERR_ARG, "cb_graph_generate_er: need m_draws + n_tedges < 2^31 per realisation");
    node_off[r + 1] = node_off[r] + n[r];
    draw_off[r + 1] = draw_off[r] + m_draws[r];
  }
  for (uint32_t e = 0; e < 2 * n_tedges; ++e)
    if (tedges[e] >= (1u << 31))
      return set_error(CB_ERR_ARG, "cb_graph_generate_er: target edge endpoint out of range");
  const uint64_t rows = node_off[n_inst];
  const uint64_t items = draw_off[n_inst] + (uint64_t)n_inst * n_tedges;

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
  if (e != cudaSuccess) return cuda_error(e, "cb_graph_generate_er: allocate");
  chk(cudaMemcpyAsync(d_n, n, n_inst * 4, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(d_node_off, node_off.data(), (n_inst + 1) * 8, cudaMemcpyHostToDevice, s));
  chk(cudaMemcpyAsync(d_draw_off, draw_off.data(), (n_inst + 1) * 8, cudaMemcpyHostToDevice, s));
  if (n_tedges) chk(cudaMemcpyAsync(d_tedges, tedges, 8ull * n_tedges, cudaMemcpyHostToDevice, s));
  chk(cudaMemsetAsync(deg, 0, rows * 4, s));
  GenArgs a{n_inst, d_n, d_node_off, d_draw_off, seed, d_tedges, n_tedges, items};
  if (e == cudaSuccess) {
    gen_count_kernel<<<grid_for(items), kGenThreads, 0, s>>>(a, deg);
    chk(cudaGetLastError());
    chk(exclusive_scan(deg, rows, off, bsum, s));
  }
  uint64_t entries = 0;
  chk(cudaMemcpyAsync(&entries, off + rows, 8, cudaMemcpyDeviceToHost, s));
  chk(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return cuda_error(e, "cb_graph_generate_er: count");
  chk(B.alloc(&raw, std::max<uint64_t>(entries, 1)));
  if (e != cudaSuccess) return cuda_error(e, "cb_graph_generate_er: allocate entries");
  if (e == cudaSuccess) {
    gather_bounds_kernel<<<(n_inst + 256) / 256, 256, 0, s>>>(off, d_node_off, n_inst, ebase);
    gen_cursor_kernel<<<grid_for(rows), kGenThreads, 0, s>>>(a, off, ebase, cursor, rows);
    gen_fill_kernel<<<grid_for(items), kGenThreads, 0, s>>>(a, ebase, cursor, raw);
    gen_sort_kernel<<<grid_for(rows * 32), kGenThreads, 0, s>>>(off, raw, deg, rows);
    chk(cudaGetLastError());
    chk(exclusive_scan(deg, rows, off2, bsum, s));
    gather_bounds_kernel<<<(n_inst + 256) / 256, 256, 0, s>>>(off2, d_node_off, n_inst, bound);
    chk(cudaGetLastError());
  }
  std::vector<uint64_t> hb(n_inst + 1, 0);
  chk(cudaMemcpyAsync(hb.data(), bound, (n_inst + 1) * 8, cudaMemcpyDeviceToHost, s));
  chk(cudaStreamSynchronize(s));
  if (e != cudaSuccess) return cuda_error(e, "cb_graph_generate_er: build rows");
  std::vector<uint64_t> nnz(n_inst);
  for (uint32_t r = 0; r < n_inst; ++r) {
    nnz[r] = hb[r + 1] - hb[r];
    if (nnz[r] >= 0xffffffffull)
      return set_error(CB_ERR_ARG, "cb_graph_generate_er: a realisation has >= 2^32 entries");
  }
  chk(B.alloc(&col, std::max<uint64_t>(hb[n_inst], 1)));
  chk(B.alloc(&rp, rows + n_inst));
  if (e != cudaSuccess) return cuda_error(e, "cb_graph_generate_er: allocate CSR");
  gen_compact_kernel<<<grid_for(rows * 32), kGenThreads, 0, s>>>(a, off, raw, off2, col, rp, rows);
  chk(cudaGetLastError());
  chk(cudaStreamSynchronize(s));  // the upload reads row_ptr back with a plain copy
  if (e != cudaSuccess) return cuda_error(e, "cb_graph_generate_er: compact");
  std::vector<const uint32_t *> rpp(n_inst), colp(n_inst);
  for (uint32_t r = 0; r < n_inst; ++r) {
    rpp[r] = rp + node_off[r] + r;
    colp[r] = col + hb[r];
  }
  // the upload copies the arrays (device to device) and builds the tables;
  // the temporaries are freed when B goes out of scope
  return cb_graph_upload(n_inst, n, nnz.data(), rpp.data(), colp.data(), CB_DEVICE_PTRS, stream,
                         out);
}
