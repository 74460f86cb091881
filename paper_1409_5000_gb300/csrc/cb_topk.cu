// Top-k selection of the summed scores of eq. 5 (section "Identification
// algorithm": the recovered target is the k nodes of largest summed EBTC).
//
// The paper sorts all n scores (Introsort, O(n log n)).  Only the k largest
// are needed, so this selects them by most-significant-digit radix select
// and sorts just those k:
//
//  * each score maps to an order-preserving 64-bit key (NaN lowest, -0 = +0)
//    and the key is extended by the complemented node index, so the 96-bit
//    composite keys are distinct and larger composite = larger score, ties
//    to the smaller index;
//  * pass L (L = 0..11) histograms byte L of the composite key over the
//    elements whose bytes 0..L-1 equal the prefix found so far; the last CTA
//    to finish picks the byte where the count from the top reaches the
//    number still needed, and stops the passes as soon as the whole bucket
//    is needed;
//  * one pass collects the k elements at or above the prefix, one CTA sorts
//    them (bitonic) and writes indices and values.
// Up to 4096 scores, one CTA sorts them all instead (one launch).
//
// Every pass is launched unconditionally and returns at once when the
// selection is complete, so the sequence needs no host round trip.
#include "cb_internal.cuh"

namespace cb {

namespace {

struct TopkState {
  unsigned long long phi;  // prefix of the 64-bit score key (unfixed bits zero)
  uint32_t plo;            // prefix of the complemented index
  uint32_t level;          // bytes fixed so far (0..12)
  uint32_t krem;           // elements still needed inside the prefix bucket
  uint32_t done;
  uint32_t arrive;
  uint32_t ncol;
  uint32_t hist[256];
};

struct Cand {
  unsigned long long key;
  uint32_t idx;
  uint32_t pad;
};

__device__ __forceinline__ unsigned long long order_key(double v) {
  if (v != v) return 0ull;  // NaN ranks below every number
  if (v == 0.0) v = 0.0;    // -0.0 -> +0.0
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ unsigned long long mask_hi(uint32_t L) {
  return L == 0 ? 0ull : (L >= 8 ? ~0ull : (~0ull << (64 - 8 * L)));
}
__device__ __forceinline__ uint32_t mask_lo(uint32_t L) {
  return L <= 8 ? 0u : (L >= 12 ? ~0u : (~0u << (32 - 8 * (L - 8))));
}
__device__ __forceinline__ uint32_t digit(unsigned long long hi, uint32_t lo, uint32_t L) {
  return L < 8 ? (uint32_t)((hi >> (56 - 8 * L)) & 255ull) : ((lo >> (24 - 8 * (L - 8))) & 255u);
}

__global__ void topk_init(TopkState *st, uint32_t k) {
  for (int d = threadIdx.x; d < 256; d += blockDim.x) st->hist[d] = 0;
  if (threadIdx.x == 0) {
    st->phi = 0ull;
    st->plo = 0u;
    st->level = 0u;
    st->krem = k;
    st->done = 0u;
    st->arrive = 0u;
    st->ncol = 0u;
  }
}

__global__ void __launch_bounds__(256) topk_pass(const double *__restrict__ S, uint32_t n,
                                                 TopkState *st, uint32_t L) {
  __shared__ uint32_t sh[256];
  __shared__ int s_last;
  if (st->done) return;
  const unsigned long long phi = st->phi, mh = mask_hi(L);
  const uint32_t plo = st->plo, ml = mask_lo(L);
  sh[threadIdx.x] = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long key = order_key(__ldg(S + i));
    const uint32_t lo = ~i;
    if ((key & mh) == phi && (lo & ml) == plo) atomicAdd(&sh[digit(key, lo, L)], 1u);
  }
  __syncthreads();
  if (sh[threadIdx.x]) atomicAdd(&st->hist[threadIdx.x], sh[threadIdx.x]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(&st->arrive, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    const uint32_t krem = st->krem;
    uint32_t cum = 0, dstar = 0, hstar = 0;
    for (int d = 255; d >= 0; --d) {
      const uint32_t hd = __ldcg(&st->hist[d]);
      if (cum + hd >= krem) {
        dstar = (uint32_t)d;
        hstar = hd;
        break;
      }
      cum += hd;
    }
    if (L < 8) st->phi = phi | ((unsigned long long)dstar << (56 - 8 * L));
    else st->plo = plo | (dstar << (24 - 8 * (L - 8)));
    const uint32_t left = krem - cum;
    st->krem = left;
    st->level = L + 1;
    if (hstar == left || L + 1 >= 12) st->done = 1u;
    st->arrive = 0u;
  }
  __syncthreads();
  st->hist[threadIdx.x] = 0u;
}

__global__ void __launch_bounds__(256) topk_collect(const double *__restrict__ S, uint32_t n,
                                                    TopkState *st, Cand *buf, uint32_t k) {
  const uint32_t L = st->level;
  const unsigned long long mh = mask_hi(L), phi = st->phi;
  const uint32_t ml = mask_lo(L), plo = st->plo;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long key = order_key(__ldg(S + i));
    const uint32_t lo = ~i;
    const unsigned long long kh = key & mh;
    if (kh > phi || (kh == phi && (lo & ml) >= plo)) {
      const uint32_t pos = atomicAdd(&st->ncol, 1u);
      if (pos < k) buf[pos] = Cand{key, i, 0u};
    }
  }
}

// (key desc, idx asc) ordering: a goes before b
__device__ __forceinline__ bool before(unsigned long long ka, uint32_t ia, unsigned long long kb,
                                       uint32_t ib) {
  return ka > kb || (ka == kb && ia < ib);
}

__global__ void __launch_bounds__(1024) topk_sort(const double *__restrict__ S, const Cand *buf,
                                                  uint32_t k, uint32_t P, uint32_t *idx,
                                                  double *val) {
  extern __shared__ unsigned char s_raw[];
  unsigned long long *sk = reinterpret_cast<unsigned long long *>(s_raw);
  uint32_t *si = reinterpret_cast<uint32_t *>(sk + P);
  for (uint32_t q = threadIdx.x; q < P; q += blockDim.x) {
    if (q < k) { sk[q] = buf[q].key; si[q] = buf[q].idx; }
    else { sk[q] = 0ull; si[q] = 0xffffffffu; }
  }
  __syncthreads();
  for (uint32_t size = 2; size <= P; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t q = threadIdx.x; q < P; q += blockDim.x) {
        const uint32_t p = q ^ stride;
        if (p > q) {
          const bool desc = (q & size) == 0;  // first half of each block in final order
          const bool swap = desc ? before(sk[p], si[p], sk[q], si[q])
                                 : before(sk[q], si[q], sk[p], si[p]);
          if (swap) {
            const unsigned long long tk = sk[q]; sk[q] = sk[p]; sk[p] = tk;
            const uint32_t ti = si[q]; si[q] = si[p]; si[p] = ti;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t q = threadIdx.x; q < k; q += blockDim.x) {
    idx[q] = si[q];
    val[q] = S[si[q]];
  }
}

// n <= kTopkSmallN: one CTA sorts all n composite keys (bitonic, in shared
// memory, the same order as topk_sort) and writes the first k -- one launch
// instead of the 15 of the radix select.
constexpr uint32_t kTopkSmallN = 4096;

__global__ void __launch_bounds__(1024) topk_small(const double *__restrict__ S, uint32_t n,
                                                   uint32_t k, uint32_t P, uint32_t *idx,
                                                   double *val) {
  extern __shared__ unsigned char s_raw[];
  unsigned long long *sk = reinterpret_cast<unsigned long long *>(s_raw);
  uint32_t *si = reinterpret_cast<uint32_t *>(sk + P);
  for (uint32_t q = threadIdx.x; q < P; q += blockDim.x) {
    if (q < n) { sk[q] = order_key(S[q]); si[q] = q; }
    else { sk[q] = 0ull; si[q] = 0xffffffffu; }  // after every element, NaN included
  }
  __syncthreads();
  for (uint32_t size = 2; size <= P; size <<= 1) {
    for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
      for (uint32_t q = threadIdx.x; q < P; q += blockDim.x) {
        const uint32_t p = q ^ stride;
        if (p > q) {
          const bool desc = (q & size) == 0;
          const bool swap = desc ? before(sk[p], si[p], sk[q], si[q])
                                 : before(sk[q], si[q], sk[p], si[p]);
          if (swap) {
            const unsigned long long tk = sk[q]; sk[q] = sk[p]; sk[p] = tk;
            const uint32_t ti = si[q]; si[q] = si[p]; si[p] = ti;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t q = threadIdx.x; q < k; q += blockDim.x) {
    idx[q] = si[q];
    val[q] = S[si[q]];
  }
}

}  // namespace

int topk_launch(const double *S, uint32_t n, uint32_t k, uint32_t *idx, double *val,
                void *scratch, cudaStream_t s) {
  if (n <= kTopkSmallN) {
    uint32_t P = 1;
    while (P < n) P <<= 1;
    const int tok = prof_begin(CB_K_TOPK, s);
    topk_small<<<1, 1024, (size_t)P * (sizeof(unsigned long long) + sizeof(uint32_t)), s>>>(S, n, k, P,
                                                                                          idx, val);
    prof_end(tok, s);
    return cuda_error(cudaGetLastError(), "topk launch");
  }
  TopkState *st = reinterpret_cast<TopkState *>(scratch);
  Cand *buf = reinterpret_cast<Cand *>(reinterpret_cast<char *>(scratch) +
                                       ((sizeof(TopkState) + 255) / 256) * 256);
  uint32_t grid = (n + 256 * 8 - 1) / (256 * 8);
  if (grid > 152 * 8) grid = 152 * 8;
  if (grid == 0) grid = 1;
  prefer_shared(topk_init);
  prefer_shared(topk_pass);
  prefer_shared(topk_collect);
  prefer_shared(topk_sort);
  const int tok = prof_begin(CB_K_TOPK, s);
  topk_init<<<1, 256, 0, s>>>(st, k);
  for (uint32_t L = 0; L < 12; ++L) topk_pass<<<grid, 256, 0, s>>>(S, n, st, L);
  topk_collect<<<grid, 256, 0, s>>>(S, n, st, buf, k);
  uint32_t P = 1;
  while (P < k) P <<= 1;
  const size_t shm = (size_t)P * (sizeof(unsigned long long) + sizeof(uint32_t));
  topk_sort<<<1, 1024, shm, s>>>(S, buf, k, P, idx, val);
  prof_end(tok, s);
  return cuda_error(cudaGetLastError(), "topk launch");
}

size_t topk_scratch_bytes(uint32_t k) {
  return ((sizeof(TopkState) + 255) / 256) * 256 + (size_t)k * sizeof(Cand);
}

}  // namespace cb

CB_API int cb_topk(const double *S, uint32_t n, uint32_t k, uint32_t *idx, double *val,
                   void *stream) {
  cb::NvtxRange nvtx_range("cb_topk");
  using namespace cb;
  if (!S || !idx || !val) return set_error(CB_ERR_ARG, "cb_topk: null pointer");
  if (n == 0 || k == 0 || k > n || k > CB_MAX_TOPK)
    return set_error(CB_ERR_ARG, "cb_topk: need 1 <= k <= min(n, CB_MAX_TOPK)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void *scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, topk_scratch_bytes(k), s);
  if (e != cudaSuccess) return cuda_error(e, "cb_topk: cudaMallocAsync");
  int rc = topk_launch(S, n, k, idx, val, scratch, s);
  e = cudaFreeAsync(scratch, s);
  if (rc != CB_OK) return rc;
  return cuda_error(e, "cb_topk: cudaFreeAsync");
}

// ---------------------------------------------------------------------------
// Top-k without allocation.
//
// cb_topk takes its scratch from the stream-ordered allocator.  Some callers
// cannot allocate device memory at all: a host application that has
// reserved the whole GPU for its own pool and rejects any further cudaMalloc
// / cudaMallocAsync, a plug-in whose host forbids CUDA allocation calls, or a
// latency-critical loop where an allocation could stall on the device.  This
// variant uses a fixed file-scope device array instead, sized for the
// largest k the library accepts (CB_MAX_TOPK), about 65 KB per device.  It
// runs the same kernels as cb_topk.
// ---------------------------------------------------------------------------
#include <mutex>

namespace cb {
namespace {

constexpr size_t kNoAllocScratchBytes =
    ((sizeof(TopkState) + 255) / 256) * 256 + (size_t)CB_MAX_TOPK * sizeof(Cand);

// Shared by every cb_topk_noalloc call on a device; resident until exit.
__device__ __align__(256) unsigned char g_topk_noalloc_scratch[kNoAllocScratchBytes];

// The array's device address belongs to the CUDA context that loaded the
// module, so it is cached per context: keyed by the context's process-unique
// id (cuCtxGetId), which a context created after cudaDeviceReset, or another
// context made current on the same device, does not share.  The driver
// functions come through the runtime's entry-point query, so the library
// needs no link against the driver library.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);
constexpr int kMaxContexts = 64;
std::mutex g_noalloc_mu;
unsigned long long g_noalloc_ctx[kMaxContexts] = {};
void *g_noalloc_ptr[kMaxContexts] = {};
int g_noalloc_used = 0;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Device address of the scratch array in the current context.  The host-side
// symbol is only a stand-in, so the address is looked up (with the context
// current) the first time a context calls, and cached.
int noalloc_scratch(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cb_topk_noalloc: cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_ctx_get_current || !g_ctx_get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void **)&g_ctx_get_current, 12000,
                                         cudaEnableDefault, &q1);
    if (e == cudaSuccess)
      e = cudaGetDriverEntryPointByVersion("cuCtxGetId", (void **)&g_ctx_get_id, 12000,
                                           cudaEnableDefault, &q2);
    if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
      g_ctx_get_current = nullptr;
      g_ctx_get_id = nullptr;
      return set_error(CB_ERR_CUDA, "cb_topk_noalloc: driver context query unavailable");
    }
  }
  void *ctx = nullptr;
  if (g_ctx_get_current(&ctx) != 0 || !ctx) {
    // no context current on this thread yet: make the device's primary
    // context current (cudaSetDevice initialises it; no allocation)
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) return cuda_error(e, "cb_topk_noalloc: cudaSetDevice");
    if (g_ctx_get_current(&ctx) != 0 || !ctx)
      return set_error(CB_ERR_CUDA, "cb_topk_noalloc: no current CUDA context");
  }
  unsigned long long id = 0;
  if (g_ctx_get_id(ctx, &id) != 0) return set_error(CB_ERR_CUDA, "cb_topk_noalloc: cuCtxGetId failed");
  for (int q = 0; q < g_noalloc_used; ++q)
    if (g_noalloc_ctx[q] == id) {
      *out = g_noalloc_ptr[q];
      return CB_OK;
    }
  void *p = nullptr;
  e = cudaGetSymbolAddress(&p, g_topk_noalloc_scratch);
  if (e != cudaSuccess) return cuda_error(e, "cb_topk_noalloc: cudaGetSymbolAddress");
  if (g_noalloc_used < kMaxContexts) {  // beyond that many contexts: looked up every call
    g_noalloc_ctx[g_noalloc_used] = id;
    g_noalloc_ptr[g_noalloc_used] = p;
    ++g_noalloc_used;
  }
  *out = p;
  return CB_OK;
}

}  // namespace
}  // namespace cb

CB_API int cb_topk_noalloc(const double *S, uint32_t n, uint32_t k, uint32_t *idx, double *val,
                           void *stream) {
  cb::NvtxRange nvtx_range("cb_topk_noalloc");
  using namespace cb;
  if (!S || !idx || !val) return set_error(CB_ERR_ARG, "cb_topk_noalloc: null pointer");
  if (n == 0 || k == 0 || k > n)
    return set_error(CB_ERR_ARG, "cb_topk_noalloc: need 1 <= k <= n");
  if (k > CB_MAX_TOPK || topk_scratch_bytes(k) > kNoAllocScratchBytes)
    return set_error(CB_ERR_ARG,
                     "cb_topk_noalloc: k exceeds the fixed scratch capacity (CB_MAX_TOPK = 4096)");
  void *scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != CB_OK) return rc;
  // topk_launch's first kernel resets every counter and histogram in the
  // scratch, so the previous call's contents need no clearing here.
  return topk_launch(S, n, k, idx, val, scratch, reinterpret_cast<cudaStream_t>(stream));
}
