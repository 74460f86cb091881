// C ABI entry points: graph upload / free, per-call dispatch, errors.
//
// Upload builds the pattern-only CSR store of the adjacency matrices (paper,
// "Signal processing on graphs": symmetric 0/1 A) for N realisations and
// the static launch tables of the Lanczos kernels:
//   * every realisation's node range is padded to kNodeAlign elements in the
//     Krylov vectors, so vector tiles start aligned;
//   * SpMV tiles of at most kTileRows rows and about kTileNnz entries; rows
//     with more than kHeavyDeg entries are
//     listed as heavy rows and cut into kChunk-edge chunks;
//   * finalize tiles of kFinRows nodes;
//   * one reduction plan (slots and groups) per realisation and kernel kind.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "cb_internal.cuh"

namespace cb {

static thread_local std::string g_err;

// Pinned staging of an upload's small host tables (stage_h2d).  Chunks are
// kept for the next upload; an upload holds the lock from start to end, and
// the buffer is recycled once its copies are done.
struct PinnedArena {
  std::vector<std::pair<char *, size_t>> chunks;
  size_t ci = 0, off = 0;
};
static std::recursive_mutex g_stage_mu;
static PinnedArena g_stage;

int set_error(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

int cuda_error(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return CB_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return set_error(CB_ERR_OOM, std::string(what) + ": out of device memory");
  }
  return set_error(CB_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---- optional launch timing -------------------------------------------
struct ProfRec {
  int kernel;
  cudaEvent_t a, b;
};
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_event_pool;

static cudaEvent_t take_event() {
  if (!g_event_pool.empty()) {
    cudaEvent_t e = g_event_pool.back();
    g_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int prof_begin(int kernel, cudaStream_t s) {
  if (!g_prof_on) return -1;
  ProfRec r{kernel, take_event(), take_event()};
  cudaEventRecord(r.a, s);
  g_prof.push_back(r);
  return (int)g_prof.size() - 1;
}

void prof_end(int token, cudaStream_t s) {
  if (token >= 0) cudaEventRecord(g_prof[token].b, s);
}

static void prof_clear() {
  for (auto &r : g_prof) {
    g_event_pool.push_back(r.a);
    g_event_pool.push_back(r.b);
  }
  g_prof.clear();
}

void parallel_for(uint32_t n, const std::function<void(uint32_t)> &fn) {
  unsigned hw = std::thread::hardware_concurrency();
  const uint32_t nt = std::min<uint32_t>(n, hw ? std::min(hw, 32u) : 1u);
  if (nt <= 1) {
    for (uint32_t i = 0; i < n; ++i) fn(i);
    return;
  }
  std::vector<std::thread> th;
  for (uint32_t t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      for (uint32_t i = t; i < n; i += nt) fn(i);
    });
  for (auto &x : th) x.join();
}

void prefer_shared_impl(const void *kernel) {
  static std::mutex mu;
  static std::vector<const void *> done;
  std::lock_guard<std::mutex> lk(mu);
  for (const void *k : done)
    if (k == kernel) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  done.push_back(kernel);
}

static int pick_lanes(double avg_deg) {
  if (avg_deg < 3) return 1;
  if (avg_deg < 6) return 2;
  if (avg_deg < 24) return 4;
  if (avg_deg < 64) return 8;
  if (avg_deg < 128) return 16;
  return 32;
}

static std::mutex g_pool_mu;
static std::vector<cudaMemPool_t> g_pools;        // per device, created on first use
static std::vector<cudaStream_t> g_alloc_streams;  // per device, non-blocking

static bool use_pool() {
  static const bool on = std::getenv("CB_NO_POOL") == nullptr;
  return on;
}

static cudaError_t device_pool(cudaMemPool_t *pool, cudaStream_t *stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if ((int)g_pools.size() <= dev) {
    g_pools.resize(dev + 1, nullptr);
    g_alloc_streams.resize(dev + 1, nullptr);
  }
  if (!g_alloc_streams[dev]) {
    e = cudaStreamCreateWithFlags(&g_alloc_streams[dev], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      g_alloc_streams[dev] = nullptr;
      return e;
    }
  }
  if (!g_pools[dev]) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    e = cudaMemPoolCreate(&p, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = ~0ull;  // never hand memory back on synchronisation
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = p;
  }
  *pool = g_pools[dev];
  *stream = g_alloc_streams[dev];
  return cudaSuccess;
}

// Pool allocations are ordered on a library stream of their own
// (non-blocking, so they wait for no caller's work) and completed before
// returning, so the memory is usable from any stream.  An upload on one host
// thread therefore proceeds while another thread's kernels run.
// Live bytes of the library's device allocations and the optional cap
// (cb_set_memory_limit); sizes are kept per pointer for dev_free.
static std::mutex g_alloc_mu;
static std::unordered_map<void *, size_t> g_alloc_size;
static size_t g_alloc_live = 0, g_alloc_limit = 0;

cudaError_t dev_alloc(void **p, size_t bytes) {
  *p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_alloc_limit && g_alloc_live + bytes > g_alloc_limit) return cudaErrorMemoryAllocation;
  }
  cudaError_t e;
  if (!use_pool()) {
    e = cudaMalloc(p, bytes);
  } else {
    cudaMemPool_t pool;
    cudaStream_t as = nullptr;
    e = device_pool(&pool, &as);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(p, bytes, pool, as);
    if (e == cudaSuccess) e = cudaStreamSynchronize(as);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc_size[*p] = bytes;
  g_alloc_live += bytes;
  return e;
}

void dev_free(void *p) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    auto it = g_alloc_size.find(p);
    if (it != g_alloc_size.end()) {
      g_alloc_live -= it->second;
      g_alloc_size.erase(it);
    }
  }
  if (!use_pool()) {
    cudaFree(p);
    return;
  }
  cudaMemPool_t pool;
  cudaStream_t as = nullptr;
  cudaDeviceSynchronize();  // no kernel may still use it
  if (device_pool(&pool, &as) == cudaSuccess) cudaFreeAsync(p, as);
}

template <typename P>
static cudaError_t dalloc(P **p, size_t count) {
  return dev_alloc_n(p, count);
}

void free_workspace(Workspace &W) {
  dev_free(W.V);
  dev_free(W.blob);
  W = Workspace{};
}

static void free_graph_arrays(cb_graph *h) {
  if (h->owns_csr) {
    dev_free(h->col);
    dev_free(h->row_ptr);
  }
  dev_free(h->d_inst);
  dev_free(h->d_tile_inst);
  dev_free(h->d_tile_rows);
  dev_free(h->d_heavy);
  dev_free(h->d_chunk_heavy);
  dev_free(h->d_fin_inst);
  dev_free(h->d_mirror);
  h->d_mirror = nullptr;
  h->col = nullptr;
  h->row_ptr = nullptr;
  h->d_inst = nullptr;
  h->d_tile_inst = nullptr;
  h->d_tile_rows = nullptr;
  h->d_heavy = nullptr;
  h->d_chunk_heavy = nullptr;
  h->d_fin_inst = nullptr;
}

// Workspace for depth m in precision prec; reused when large enough.
int ensure_workspace(cb_graph *h, Workspace &W, uint32_t m, int prec, cudaStream_t s) {
  if (W.V && W.prec == prec && W.m >= m) return CB_OK;
  free_workspace(W);
  const size_t esz = prec == CB_FP64 ? sizeof(double) : sizeof(float);
  W.vec_stride = h->total_nodes_padded;
  const size_t vbytes = (size_t)(m + 1) * W.vec_stride * esz;
  cudaError_t e = dev_alloc(&W.V, vbytes ? vbytes : 16);
  if (e != cudaSuccess) {
    W.V = nullptr;
    return cuda_error(e, "workspace: Krylov basis");
  }
  const uint32_t N = h->n_inst, ms = m + 1;
  const size_t nslots = std::max<size_t>(h->total_slots, 1);
  const size_t ngroups = std::max<size_t>(h->total_groups, 1);
  const size_t nchunks = std::max<size_t>(h->total_chunks, 1);
  const size_t nheavy = std::max<size_t>(h->total_heavy, 1);
  // doubles first, then 32-bit words
  const size_t nfin = std::max<size_t>(h->total_fin, 1);
  const size_t nd = 4 * (size_t)N * ms + N + nslots + ngroups + nchunks + nfin * ms + (size_t)N * ms;
  const size_t nw = 2 * (size_t)N + ngroups + N + nheavy;
  const size_t bytes = nd * sizeof(double) + nw * sizeof(uint32_t) + 256;
  e = dev_alloc(&W.blob, bytes);
  if (e != cudaSuccess) {
    W.blob = nullptr;
    free_workspace(W);
    return cuda_error(e, "workspace: scalars");
  }
  double *d = reinterpret_cast<double *>(W.blob);
  W.sc.alpha = d; d += (size_t)N * ms;
  W.sc.beta = d; d += (size_t)N * ms;
  W.sc.scale = d; d += (size_t)N * ms;
  W.sc.gamma = d; d += (size_t)N * ms;
  W.sc.theta = d; d += N;
  W.part = d; d += nslots;
  W.gpart = d; d += ngroups;
  W.cpart = d; d += nchunks;
  W.rpart = d; d += nfin * ms;
  W.rh = d; d += (size_t)N * ms;
  uint32_t *w = reinterpret_cast<uint32_t *>(d);
  W.sc.meff = w; w += N;
  W.sc.status = reinterpret_cast<int32_t *>(w); w += N;
  W.gcnt = w; w += ngroups;
  W.icnt = w; w += N;
  W.hcnt = w; w += nheavy;
  W.sc.ms = ms;
  W.blob_bytes = bytes;
  W.m = m;
  W.prec = prec;
  static std::atomic<uint64_t> generation{0};
  W.gen = ++generation;
  e = cudaMemsetAsync(W.blob, 0, bytes, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_workspace(W);
    return cuda_error(e, "workspace: clear");
  }
  return CB_OK;
}

static int validate_host(uint32_t n, uint64_t nnz, const uint32_t *rp, const uint32_t *col,
                         uint32_t r) {
  char buf[256];
  if (rp[0] != 0 || rp[n] != nnz) {
    snprintf(buf, sizeof buf, "realisation %u: row_ptr[0] must be 0 and row_ptr[n] = nnz", r);
    return set_error(CB_ERR_ARG, buf);
  }
  for (uint32_t i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) {
      snprintf(buf, sizeof buf, "realisation %u: row_ptr decreases at row %u", r, i);
      return set_error(CB_ERR_ARG, buf);
    }
    for (uint32_t e = rp[i]; e < rp[i + 1]; ++e) {
      const uint32_t c = col[e];
      if (e > rp[i] && c <= col[e - 1]) {
        snprintf(buf, sizeof buf, "realisation %u: row %u not sorted ascending (or duplicate)", r, i);
        return set_error(CB_ERR_ARG, buf);
      }
      if (c >= n || c == i) {
        snprintf(buf, sizeof buf, "realisation %u: bad column %u in row %u", r, c, i);
        return set_error(CB_ERR_ARG, buf);
      }
      // symmetric: i must appear in row c (rows need not be sorted)
      bool found = false;
      for (uint32_t f = rp[c]; f < rp[c + 1] && !found; ++f) found = (col[f] == i);
      if (!found) {
        snprintf(buf, sizeof buf, "realisation %u: pattern not symmetric at (%u,%u)", r, i, c);
        return set_error(CB_ERR_ARG, buf);
      }
    }
  }
  return CB_OK;
}

}  // namespace cb

using namespace cb;

CB_API const char *cb_last_error(void) { return g_err.c_str(); }

CB_API int cb_graph_read(const cb_graph *h, uint32_t r, uint32_t *row_ptr, uint32_t *col,
                         void *stream) {
  if (!h || !row_ptr || !col) return set_error(CB_ERR_ARG, "cb_graph_read: null argument");
  if (r >= h->n_inst) return set_error(CB_ERR_ARG, "cb_graph_read: realisation index out of range");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const InstDesc &I = h->inst[r];
  const uint64_t end = r + 1 < h->n_inst ? h->inst[r + 1].edge_base : h->total_nnz;
  cudaError_t e = cudaMemcpyAsync(row_ptr, h->row_ptr + I.rp_base, ((size_t)I.n + 1) * 4,
                                  cudaMemcpyDefault, s);
  if (e == cudaSuccess && end > I.edge_base)
    e = cudaMemcpyAsync(col, h->col + I.edge_base, (end - I.edge_base) * 4, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_error(e, "cb_graph_read");
}

CB_API uint64_t cb_graph_num_entries(const cb_graph *h, uint32_t r) {
  if (!h || r >= h->n_inst) return 0;
  const uint64_t end = r + 1 < h->n_inst ? h->inst[r + 1].edge_base : h->total_nnz;
  return end - h->inst[r].edge_base;
}

static void drop_graphs(cb_graph *h);

CB_API int cb_set_memory_limit(size_t bytes) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc_limit = bytes;
  return CB_OK;
}

CB_API size_t cb_memory_in_use(void) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  return g_alloc_live;
}

CB_API int cb_debug_stall_tile(cb_graph *h, uint32_t btile) {
  if (!h) return set_error(CB_ERR_ARG, "cb_debug_stall_tile: null handle");
  if (btile != UINT32_MAX && btile >= h->total_btiles)
    return set_error(CB_ERR_ARG, "cb_debug_stall_tile: no such column-blocked tile");
  h->stall_btile = btile;
  drop_graphs(h);  // captured launches hold the previous setting
  return CB_OK;
}

CB_API int cb_release_cached_memory(void) {
  {
    std::lock_guard<std::recursive_mutex> lk(g_stage_mu);
    for (auto &c : g_stage.chunks) cudaFreeHost(c.first);
    g_stage.chunks.clear();
    g_stage.ci = g_stage.off = 0;
  }
  cudaError_t e = cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (cudaMemPool_t p : g_pools)
    if (p) {
      const cudaError_t x = cudaMemPoolTrimTo(p, 0);
      if (e == cudaSuccess) e = x;
    }
  return cuda_error(e, "cb_release_cached_memory");
}

CB_API int cb_profile_enable(int on) {
  prof_clear();
  g_prof_on = on != 0;
  return CB_OK;
}

CB_API int cb_profile_read(int kernel, double *total_ms, uint64_t *launches) {
  if (!total_ms || !launches || kernel < 0 || kernel >= CB_K_COUNT)
    return set_error(CB_ERR_ARG, "cb_profile_read: bad argument");
  double t = 0.0;
  uint64_t c = 0;
  for (auto &r : g_prof) {
    if (r.kernel != kernel) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) return cuda_error(e, "cb_profile_read");
    t += ms;
    ++c;
  }
  *total_ms = t;
  *launches = c;
  return CB_OK;
}
CB_API uint32_t cb_version(void) { return (1u << 16) | 1u; }

CB_API uint32_t cb_debug_build(void) {
#ifdef CB_DEBUG
  return 1u;
#else
  return 0u;
#endif
}

CB_API int cb_debug_violations(uint32_t *count, uint64_t *first, int reset) {
  if (!count || !first) return set_error(CB_ERR_ARG, "cb_debug_violations: null argument");
  *count = 0;
  *first = 0;
  if (cb_debug_build() && cudaDeviceSynchronize() != cudaSuccess)
    return set_error(CB_ERR_CUDA, "cb_debug_violations: device synchronize");
  int (*readers[4])(uint32_t *, uint64_t *, bool) = {dbg_read_lanczos, dbg_read_blocked,
                                                     dbg_read_twophase, dbg_read_adjoint};
  for (auto rd : readers) {
    uint32_t c = 0;
    uint64_t f = 0;
    if (rd(&c, &f, reset != 0) != 0) return set_error(CB_ERR_CUDA, "cb_debug_violations: read");
    if (c && !*count) *first = f;
    *count += c;
  }
  return CB_OK;
}

CB_API uint32_t cb_graph_num_instances(const cb_graph *h) { return h ? h->n_inst : 0; }
CB_API uint32_t cb_graph_num_nodes(const cb_graph *h, uint32_t r) {
  return (h && r < h->n_inst) ? h->inst[r].n : 0;
}
CB_API uint32_t cb_graph_max_nodes(const cb_graph *h) { return h ? h->n_max : 0; }

// The copy stream and the per-group events of one upload.  finish() waits
// for the copies and releases both.
namespace {
constexpr uint64_t kCopyGroups = 8;
struct StageScope {
  std::unique_lock<std::recursive_mutex> lk{g_stage_mu};
  cudaStream_t s;
  explicit StageScope(cudaStream_t st) : s(st) {}
  ~StageScope() {
    cudaStreamSynchronize(s);  // every staged copy has been read
    g_stage.ci = 0;
    g_stage.off = 0;
  }
};

struct UploadCopies {
  cudaStream_t stream = nullptr;
  std::vector<CopyGroup> groups;
  cudaError_t start(cudaStream_t caller) {
    cudaError_t e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      stream = nullptr;
      return e;
    }
    // inputs may come from work still queued on the caller's stream
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(ev, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ev, 0);
    cudaEventDestroy(ev);
    return e;
  }
  cudaError_t mark(uint32_t r_end) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    groups.push_back({r_end, ev});
    return cudaEventRecord(ev, stream);
  }
  void finish() {
    if (stream) cudaStreamSynchronize(stream);
    for (const CopyGroup &g : groups) cudaEventDestroy(g.ev);
    groups.clear();
    if (stream) cudaStreamDestroy(stream);
    stream = nullptr;
  }
  ~UploadCopies() { finish(); }
};
}  // namespace

char *cb::stage_reserve(size_t bytes) {
  std::lock_guard<std::recursive_mutex> lk(g_stage_mu);
  const size_t need = (bytes + 255) & ~(size_t)255;
  while (g_stage.ci < g_stage.chunks.size() && g_stage.off + need > g_stage.chunks[g_stage.ci].second) {
    ++g_stage.ci;
    g_stage.off = 0;
  }
  if (g_stage.ci == g_stage.chunks.size()) {
    const size_t sz = std::max<size_t>(need, (size_t)16 << 20);
    char *p = nullptr;
    if (cudaMallocHost(reinterpret_cast<void **>(&p), sz) != cudaSuccess) return nullptr;
    g_stage.chunks.push_back({p, sz});
    g_stage.off = 0;
  }
  char *p = g_stage.chunks[g_stage.ci].first + g_stage.off;
  g_stage.off += need;
  return p;
}

cudaError_t cb::stage_h2d(void *dst, const void *src, size_t bytes, cudaStream_t s) {
  if (!bytes) return cudaSuccess;
  std::lock_guard<std::recursive_mutex> lk(g_stage_mu);
  char *p = stage_reserve(bytes);
  if (!p) return cudaErrorMemoryAllocation;
  std::memcpy(p, src, bytes);
  return cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, s);
}

// own_col / own_rp: device arrays taken over instead of copied (upload_adopt)
static int upload_impl(uint32_t n_inst, const uint32_t *n, const uint64_t *nnz,
                       const uint32_t *const *row_ptr, const uint32_t *const *col,
                       uint32_t flags, void *stream, cb_graph **out, uint32_t *own_col,
                       uint32_t *own_rp) {
  if (!out) return set_error(CB_ERR_ARG, "cb_graph_upload: out is null");
  *out = nullptr;
  if (n_inst == 0 || !n || !nnz || !row_ptr || !col)
    return set_error(CB_ERR_ARG, "cb_graph_upload: empty input or null array");
  if (flags & ~(CB_VALIDATE | CB_DEVICE_PTRS | CB_CSR_ONLY | CB_TWO_PHASE))
    return set_error(CB_ERR_ARG, "cb_graph_upload: unknown flag");
  if ((flags & CB_CSR_ONLY) && (flags & CB_TWO_PHASE))
    return set_error(CB_ERR_ARG, "cb_graph_upload: CB_CSR_ONLY and CB_TWO_PHASE exclude each other");
  const bool dev = (flags & CB_DEVICE_PTRS) != 0;
  if (dev && (flags & CB_VALIDATE))
    return set_error(CB_ERR_ARG, "cb_graph_upload: CB_VALIDATE needs host arrays");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  StageScope stage(s);

  cb_graph *h = new cb_graph();
  cudaGetDevice(&h->device);
  h->csr_only = (flags & CB_CSR_ONLY) != 0;
  h->force_pb = (flags & CB_TWO_PHASE) != 0;
  h->n_inst = n_inst;
  h->inst.resize(n_inst);

  // host views of row_ptr: device uploads read all of them back into one
  // pinned block (one copy per realisation, one wait) for the tables
  std::vector<const uint32_t *> rp_view(row_ptr, row_ptr + n_inst);
  if (dev) {
    uint64_t words = 0;
    for (uint32_t r = 0; r < n_inst; ++r) {
      if (n[r] == 0 || !row_ptr[r]) {
        delete h;
        return set_error(CB_ERR_ARG, "cb_graph_upload: realisation with n = 0 or null array");
      }
      words += (uint64_t)n[r] + 1;
    }
    uint32_t *hb = reinterpret_cast<uint32_t *>(stage_reserve(words * 4));
    if (!hb) {
      delete h;
      return set_error(CB_ERR_OOM, "cb_graph_upload: no pinned host memory to read row_ptr into");
    }
    cudaError_t e = cudaSuccess;
    uint64_t o = 0;
    for (uint32_t r = 0; r < n_inst && e == cudaSuccess; o += (uint64_t)n[r] + 1, ++r) {
      rp_view[r] = hb + o;
      e = cudaMemcpyAsync(hb + o, row_ptr[r], ((size_t)n[r] + 1) * 4, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      delete h;
      return cuda_error(e, "cb_graph_upload: read row_ptr");
    }
  }
  auto rp_of = [&](uint32_t r) -> const uint32_t * { return rp_view[r]; };

  uint64_t node_off = 0, edge_off = 0, rp_off = 0;
  uint32_t tile_off = 0, fin_off = 0, slot_off = 0, group_off = 0;
  for (uint32_t r = 0; r < n_inst; ++r) {
    if (n[r] == 0 || !row_ptr[r] || (nnz[r] && !col[r])) {
      delete h;
      return set_error(CB_ERR_ARG, "cb_graph_upload: realisation with n = 0 or null array");
    }
    if (nnz[r] >= 0xffffffffull) {
      delete h;
      return set_error(CB_ERR_ARG, "cb_graph_upload: nnz of one realisation must be < 2^32");
    }
    const uint32_t *rp = rp_of(r);
    if (rp[0] != 0 || rp[n[r]] != nnz[r]) {
      delete h;
      return set_error(CB_ERR_ARG, "cb_graph_upload: row_ptr[0] must be 0 and row_ptr[n] = nnz");
    }
    if (flags & CB_VALIDATE) {
      int rc = validate_host(n[r], nnz[r], rp, col[r], r);
      if (rc != CB_OK) {
        delete h;
        return rc;
      }
    }
    InstDesc &I = h->inst[r];
    std::memset(&I, 0, sizeof I);
    I.n = n[r];
    I.nnz = (uint32_t)nnz[r];
    I.node_base = node_off;
    I.edge_base = edge_off;
    I.rp_base = rp_off;
    node_off += ((uint64_t)n[r] + kNodeAlign - 1) / kNodeAlign * kNodeAlign;
    edge_off += nnz[r];
    rp_off += (uint64_t)n[r] + 1;
    I.fin_base = fin_off;
    I.n_fin = (n[r] + kFinRows - 1) / kFinRows;
    fin_off += I.n_fin;
    h->n_max = std::max(h->n_max, n[r]);
  }
  if (node_off >= (1ull << 40) || tile_off >= 0x7fffffffu) {
    delete h;
    return set_error(CB_ERR_ARG, "cb_graph_upload: input too large");
  }
  // The bulk copies go first, on a stream of their own and in groups of
  // realisations: the host builds the launch tables, and the count kernel of
  // the blocked format runs on a group, while later groups are in flight.
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  const bool adopt = own_col != nullptr;
  if (adopt) {  // the arrays are the handle's layout already: no copy
    for (uint32_t r = 0; r < n_inst; ++r)
      if (row_ptr[r] != own_rp + h->inst[r].rp_base || (nnz[r] && col[r] != own_col + h->inst[r].edge_base)) {
        delete h;
        return set_error(CB_ERR_ARG, "cb_graph_upload: adopted arrays are not concatenated in order");
      }
    h->col = own_col;
    h->row_ptr = own_rp;
    h->owns_csr = false;
  } else {
    chk(dalloc(&h->col, edge_off + 4));
    chk(dalloc(&h->row_ptr, rp_off));
  }
  chk(dalloc(&h->d_inst, n_inst));
  UploadCopies cp;
  chk(cp.start(s));
  if (e == cudaSuccess && adopt) {
    chk(cudaMemsetAsync(h->col + edge_off, 0, 16, cp.stream));
    chk(cp.mark(n_inst));
  } else if (e == cudaSuccess) {
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    chk(cudaMemsetAsync(h->col + edge_off, 0, 16, cp.stream));
    const uint64_t per_group = edge_off / kCopyGroups + 1;
    uint64_t acc = 0;
    for (uint32_t r = 0; r < n_inst && e == cudaSuccess; ++r) {
      const InstDesc &I = h->inst[r];
      if (nnz[r]) chk(cudaMemcpyAsync(h->col + I.edge_base, col[r], nnz[r] * 4, kind, cp.stream));
      chk(cudaMemcpyAsync(h->row_ptr + I.rp_base, row_ptr[r], ((size_t)I.n + 1) * 4, kind, cp.stream));
      acc += nnz[r];
      if (r + 1 == n_inst || acc >= per_group * (cp.groups.size() + 1)) chk(cp.mark(r + 1));
    }
  }
  if (e != cudaSuccess) {
    cp.finish();
    free_graph_arrays(h);
    delete h;
    return cuda_error(e, "cb_graph_upload: allocate / copy");
  }
  // The column-blocked format needs only the sizes and the device arrays:
  // its count and fill passes are queued first, and the host's scans of
  // row_ptr below run while the device builds it.
  BlockedBuild bb;
  int rc = blocked_count(h, s, cp.groups, bb);
  if (rc == CB_OK) rc = blocked_fill(h, s, bb);
  if (rc != CB_OK) {
    cp.finish();
    free_blocked(h);
    free_graph_arrays(h);
    delete h;
    return rc;
  }
  // heavy rows (degree > kHeavyDeg), in realisation and row order; the row
  // scans run in parallel over realisations
  // SpMV tiles are balanced by entries: a tile closes at kTileRows rows or
  // before it would exceed kTileNnz entries (heavy rows count as empty here:
  // their chunks run in CTAs of their own), so hub-heavy regions of a graph
  // get short tiles and no CTA becomes a straggler.
  std::vector<std::vector<uint32_t>> heavy_rows(n_inst), tile_starts(n_inst);
  parallel_for(n_inst, [&](uint32_t r) {
    const uint32_t *rp = rp_of(r);
    uint32_t rows = 0, acc = 0;
    for (uint32_t i = 0; i < h->inst[r].n; ++i) {
      const uint32_t deg = rp[i + 1] - rp[i];
      if (deg > kHeavyDeg) heavy_rows[r].push_back(i);
      const uint32_t w = deg > kHeavyDeg ? 0u : deg;
      if (rows == 0 || rows == (uint32_t)kTileRows || (acc > 0 && acc + w > kTileNnz)) {
        tile_starts[r].push_back(i);
        rows = 0;
        acc = 0;
      }
      ++rows;
      acc += w;
    }
  });
  for (uint32_t r = 0; r < n_inst; ++r) {
    h->inst[r].tile_base = tile_off;
    h->inst[r].n_tiles = (uint32_t)tile_starts[r].size();
    tile_off += h->inst[r].n_tiles;
  }
  uint32_t chunk_off = 0;
  for (uint32_t r = 0; r < n_inst; ++r) {
    InstDesc &I = h->inst[r];
    const uint32_t *rp = rp_of(r);
    I.heavy_base = (uint32_t)h->heavy.size();
    I.chunk_base = chunk_off;
    for (uint32_t i : heavy_rows[r]) {
      const uint32_t nc = (rp[i + 1] - rp[i] + kChunk - 1) / kChunk;
      h->heavy.push_back(HeavyRow{r, i, chunk_off, nc});
      chunk_off += nc;
    }
    I.n_heavy = (uint32_t)h->heavy.size() - I.heavy_base;
    I.n_chunks = chunk_off - I.chunk_base;
    I.spmv.slot_base = slot_off;
    I.spmv.n_slots = I.n_tiles + I.n_heavy;
    I.spmv.group_base = group_off;
    I.spmv.n_groups = (I.spmv.n_slots + kGroup - 1) / kGroup;
    slot_off += I.spmv.n_slots;
    group_off += I.spmv.n_groups;
  }
  // finalize reductions reuse the same buffers (never concurrent with SpMV)
  uint32_t fslot = 0, fgroup = 0;
  for (uint32_t r = 0; r < n_inst; ++r) {
    InstDesc &I = h->inst[r];
    I.fin.slot_base = fslot;
    I.fin.n_slots = I.n_fin;
    I.fin.group_base = fgroup;
    I.fin.n_groups = (I.n_fin + kGroup - 1) / kGroup;
    fslot += I.fin.n_slots;
    fgroup += I.fin.n_groups;
  }
  h->total_nodes_padded = node_off;
  h->total_nnz = edge_off;
  h->total_tiles = tile_off;
  h->total_fin = fin_off;
  h->total_heavy = (uint32_t)h->heavy.size();
  h->total_chunks = chunk_off;
  h->total_slots = std::max({h->total_slots, slot_off, fslot});  // the blocked plans are counted in
  h->total_groups = std::max({h->total_groups, group_off, fgroup});
  uint64_t nsum = 0;
  for (uint32_t r = 0; r < n_inst; ++r) nsum += n[r];
  h->lanes = pick_lanes((double)edge_off / (double)nsum);
  {
    int sm = 0;
    if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, h->device) == cudaSuccess && sm > 0)
      h->n_sm = (uint32_t)sm;
  }

  // per-tile instance tables
  std::vector<uint32_t> tile_inst(std::max<uint32_t>(tile_off, 1)), fin_inst(std::max<uint32_t>(fin_off, 1));
  std::vector<uint2> tile_rows(std::max<uint32_t>(tile_off, 1));
  for (uint32_t r = 0; r < n_inst; ++r) {
    const auto &ts = tile_starts[r];
    for (size_t q = 0; q < ts.size(); ++q)
      tile_rows[h->inst[r].tile_base + q] = make_uint2(ts[q], q + 1 < ts.size() ? ts[q + 1] : h->inst[r].n);
  }
  std::vector<uint32_t> chunk_heavy(std::max<uint32_t>(chunk_off, 1));
  for (uint32_t r = 0; r < n_inst; ++r) {
    const InstDesc &I = h->inst[r];
    std::fill(tile_inst.begin() + I.tile_base, tile_inst.begin() + I.tile_base + I.n_tiles, r);
    std::fill(fin_inst.begin() + I.fin_base, fin_inst.begin() + I.fin_base + I.n_fin, r);
  }
  for (uint32_t q = 0; q < h->total_heavy; ++q)
    for (uint32_t c = 0; c < h->heavy[q].n_chunks; ++c) chunk_heavy[h->heavy[q].chunk_base + c] = q;

  chk(dalloc(&h->d_tile_inst, tile_inst.size()));
  chk(dalloc(&h->d_tile_rows, tile_rows.size()));
  chk(dalloc(&h->d_fin_inst, fin_inst.size()));
  chk(dalloc(&h->d_heavy, std::max<size_t>(h->heavy.size(), 1)));
  chk(dalloc(&h->d_chunk_heavy, chunk_heavy.size()));
  if (e != cudaSuccess) {
    cp.finish();
    free_blocked(h);
    free_graph_arrays(h);
    delete h;
    return cuda_error(e, "cb_graph_upload: allocate");
  }
  chk(stage_h2d(h->d_inst, h->inst.data(), n_inst * sizeof(InstDesc), s));
  chk(stage_h2d(h->d_tile_inst, tile_inst.data(), tile_inst.size() * 4, s));
  chk(stage_h2d(h->d_tile_rows, tile_rows.data(), tile_rows.size() * sizeof(uint2), s));
  chk(stage_h2d(h->d_fin_inst, fin_inst.data(), fin_inst.size() * 4, s));
  if (!h->heavy.empty()) chk(stage_h2d(h->d_heavy, h->heavy.data(), h->heavy.size() * sizeof(HeavyRow), s));
  chk(stage_h2d(h->d_chunk_heavy, chunk_heavy.data(), chunk_heavy.size() * 4, s));
  if (e != cudaSuccess) {
    cp.finish();
    free_blocked(h);
    free_graph_arrays(h);
    delete h;
    return cuda_error(e, "cb_graph_upload: copy");
  }
  std::vector<const uint32_t *> rpv(n_inst);
  for (uint32_t r = 0; r < n_inst; ++r) rpv[r] = rp_of(r);
  rc = blocked_long_rows(h, rpv, s);
  if (rc == CB_OK) rc = build_twophase(h, rpv, s, cp.groups, h->force_pb);
  if (rc == CB_OK) {  // every copy has landed before the handle is returned
    for (const CopyGroup &g : cp.groups) chk(cudaStreamWaitEvent(s, g.ev, 0));
    chk(cudaStreamSynchronize(s));
    if (e != cudaSuccess) rc = cuda_error(e, "cb_graph_upload: copy");
  }
  cp.finish();
  if (rc != CB_OK) {
    free_twophase(h);
    free_blocked(h);
    free_graph_arrays(h);
    delete h;
    return rc;
  }
  h->owns_csr = true;
  *out = h;
  return CB_OK;
}

CB_API int cb_graph_upload(uint32_t n_inst, const uint32_t *n, const uint64_t *nnz,
                           const uint32_t *const *row_ptr, const uint32_t *const *col,
                           uint32_t flags, void *stream, cb_graph **out) {
  NvtxRange nvtx_range("cb_graph_upload");
  return upload_impl(n_inst, n, nnz, row_ptr, col, flags, stream, out, nullptr, nullptr);
}

int cb::upload_adopt(uint32_t n_inst, const uint32_t *n, const uint64_t *nnz,
                     const uint32_t *const *row_ptr, const uint32_t *const *col,
                     uint32_t *col_all, uint32_t *rp_all, void *stream, cb_graph **out) {
  NvtxRange nvtx_range("cb_graph_upload (adopted arrays)");
  if (!col_all || !rp_all) return set_error(CB_ERR_ARG, "cb_graph_upload: null adopted array");
  return upload_impl(n_inst, n, nnz, row_ptr, col, CB_DEVICE_PTRS, stream, out, col_all, rp_all);
}

static void drop_graphs(cb_graph *h) {
  for (auto &g : h->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  h->graphs.clear();
}

static bool valid_lanes(uint32_t g) {
  return g == 1 || g == 2 || g == 4 || g == 8 || g == 16 || g == 32;
}

CB_API int cb_graph_set_lanes(cb_graph *h, uint32_t lanes) {
  if (!h) return set_error(CB_ERR_ARG, "cb_graph_set_lanes: null handle");
  if (!valid_lanes(lanes)) return set_error(CB_ERR_ARG, "cb_graph_set_lanes: lanes must be 1, 2, 4, 8, 16 or 32");
  if (h->lanes != (int)lanes) {
    h->lanes = (int)lanes;
    drop_graphs(h);  // captured passes hold the old kernel choice
  }
  return CB_OK;
}

CB_API uint32_t cb_graph_lanes(const cb_graph *h) { return h ? (uint32_t)h->lanes : 0u; }

CB_API int cb_graph_set_path(cb_graph *h, int path) {
  if (!h) return set_error(CB_ERR_ARG, "cb_graph_set_path: null handle");
  if (path != CB_PATH_AUTO && path != CB_PATH_FORMATS && path != CB_PATH_CSR)
    return set_error(CB_ERR_ARG, "cb_graph_set_path: unknown path");
  if (h->path != path) {
    h->path = path;
    drop_graphs(h);  // captured passes hold the old kernel choice
  }
  return CB_OK;
}

CB_API int cb_graph_path(const cb_graph *h) { return h ? h->path : -1; }

// Times a short Lanczos run (kProbe steps over all realisations, twice, on a
// workspace of its own) for every group width of the tiled-CSR SpMV and keeps
// the fastest.  Realisations on the column-blocked kernel are timed too but
// do not depend on the width.
CB_API int cb_graph_tune(cb_graph *h, int prec, uint32_t *lanes_out, double *ms_out, void *stream) {
  NvtxRange nvtx_range("cb_graph_tune");
  if (!h) return set_error(CB_ERR_ARG, "cb_graph_tune: null handle");
  split_prec(prec);  // reorthogonalisation does not change the SpMV being tuned
  h->reorth = false;
  if (prec != CB_FP32 && prec != CB_FP64) return set_error(CB_ERR_ARG, "cb_graph_tune: bad precision");
  static const uint32_t kCand[6] = {1, 2, 4, 8, 16, 32};
  for (int c = 0; ms_out && c < 8; ++c) ms_out[c] = -1.0;
  // the format path is a candidate in FP32 when a format was built; the
  // single launch of all steps (the automatic path) when every realisation is
  // small enough for it
  const bool formats = prec == CB_FP32 && (h->total_btiles > 0 || h->total_ptiles > 0);
  bool small = true;
  for (uint32_t r = 0; r < h->n_inst && small; ++r)
    small = h->inst[r].n <= kSmallN && h->inst[r].nnz <= kSmallNnz;
  constexpr uint32_t kProbe = 3;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Workspace W;
  int rc = ensure_workspace(h, W, kProbe, prec, s);
  if (rc != CB_OK) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int keep_lanes = h->lanes, keep_path = h->path;
  int best_lanes = keep_lanes, best_path = keep_path;
  double best_ms = 1e300;
  auto time_one = [&](int lanes, int path, int slot) {
    h->lanes = lanes;
    h->path = path;
    rc = lanczos_run(h, W, 0, h->n_inst, kProbe, prec, s);  // warm-up
    if (rc == CB_OK) e = cudaEventRecord(e0, s);
    for (int rep = 0; rep < 2 && rc == CB_OK && e == cudaSuccess; ++rep)
      rc = lanczos_run(h, W, 0, h->n_inst, kProbe, prec, s);
    if (rc == CB_OK && e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (rc == CB_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (rc == CB_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rc == CB_OK && e == cudaSuccess) {
      if (ms_out) ms_out[slot] = ms / 2.0;
      if (ms < best_ms) {
        best_ms = ms;
        best_lanes = lanes;
        best_path = path;
      }
    }
  };
  for (int c = 0; c < 6 && e == cudaSuccess && rc == CB_OK; ++c) time_one((int)kCand[c], CB_PATH_CSR, c);
  // the format path, with the best width for any tiled-CSR realisations left
  if (formats && e == cudaSuccess && rc == CB_OK) time_one(best_lanes, CB_PATH_FORMATS, 6);
  if (small && e == cudaSuccess && rc == CB_OK) time_one(best_lanes, CB_PATH_AUTO, 7);
  // FP64 depends on the path only through the single launch of small handles
  if (prec == CB_FP64 && !small) best_path = keep_path;
  h->lanes = best_lanes;
  h->path = best_path;
  if (best_lanes != keep_lanes || best_path != keep_path) drop_graphs(h);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  free_workspace(W);
  if (rc != CB_OK || e != cudaSuccess) {
    h->lanes = keep_lanes;
    h->path = keep_path;
    return rc != CB_OK ? rc : cuda_error(e, "cb_graph_tune");
  }
  if (lanes_out) *lanes_out = (uint32_t)best_lanes;
  return CB_OK;
}

CB_API int cb_graph_free(cb_graph *h) {
  NvtxRange nvtx_range("cb_graph_free");
  if (!h) return set_error(CB_ERR_ARG, "cb_graph_free: null handle");
  cudaError_t e = cudaDeviceSynchronize();
  drop_graphs(h);
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  free_workspace(h->ws);
  free_workspace(h->ws2);
  free_backwork(h->bw);
  free_twophase(h);
  free_blocked(h);
  free_graph_arrays(h);
  delete h;
  return cuda_error(e, "cb_graph_free");
}

int cb::status_error(int32_t st) {
  if (st == CB_ERR_TIMEOUT)
    return set_error(CB_ERR_TIMEOUT, "a bounded device-side wait gave up (column-blocked SpMV)");
  return set_error(CB_ERR_NONFINITE, "a recurrence scalar became non-finite");
}

static int fill_report(cb_graph *h, uint32_t r0, uint32_t r1, cb_inst_report *rep, cudaStream_t s) {
  const uint32_t N = r1 - r0, ms = h->ws.sc.ms;
  std::vector<uint32_t> meff(N);
  std::vector<int32_t> st(N);
  std::vector<double> th(N), be((size_t)N * ms);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(meff.data(), h->ws.sc.meff + r0, N * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(st.data(), h->ws.sc.status + r0, N * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(th.data(), h->ws.sc.theta + r0, N * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(be.data(), h->ws.sc.beta + (size_t)r0 * ms, (size_t)N * ms * 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_error(e, "report");
  int rc = CB_OK;
  for (uint32_t q = 0; q < N; ++q) {
    rep[q].m_eff = meff[q];
    rep[q].status = st[q];
    rep[q].theta = th[q];
    rep[q].beta_last = meff[q] ? be[(size_t)q * ms + meff[q] - 1] : 0.0;
    rep[q].beta0 = std::sqrt((double)h->inst[r0 + q].n);
    if (st[q] != CB_OK && rc == CB_OK) rc = status_error(st[q]);
  }
  return rc;
}

CB_API int cb_communicability(cb_graph *h, uint32_t inst, uint32_t m, int prec, double *y_scaled,
                              double *log_scale, cb_inst_report *rep, void *stream) {
  NvtxRange nvtx_range("cb_communicability");
  if (!h || !y_scaled || !log_scale) return set_error(CB_ERR_ARG, "cb_communicability: null argument");
  if (inst >= h->n_inst) return set_error(CB_ERR_ARG, "cb_communicability: realisation index out of range");
  if (m < 1 || m > CB_MAX_M) return set_error(CB_ERR_ARG, "cb_communicability: need 1 <= m <= CB_MAX_M");
  const bool reorth = split_prec(prec);
  if (prec != CB_FP32 && prec != CB_FP64) return set_error(CB_ERR_ARG, "cb_communicability: bad precision");
  h->reorth = reorth;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = ensure_workspace(h, h->ws, m, prec, s);
  h->basis_m = 0;  // overwrites part of the ensemble basis
  if (rc == CB_OK) rc = lanczos_run(h, h->ws, inst, inst + 1, m, prec, s);
  if (rc == CB_OK) rc = tridiag_run(h, inst, inst + 1, prec, s);
  if (rc == CB_OK) rc = combine_single(h, inst, prec, y_scaled, log_scale, s);
  if (rc == CB_OK && rep) rc = fill_report(h, inst, inst + 1, rep, s);
  return rc;
}

// A repeated ensemble pass is launched as one CUDA graph: captured once per
// (m, precision, n_out, output pointers, workspace allocation) on a private
// stream, then replayed on the caller's stream.  The reduction counters are
// returned to zero by the kernels themselves, so a replay needs no reset.
// Direct launches are used for the first call of a shape, while kernel timing
// is on, for report calls, and when CB_NO_GRAPH is set.
static int ensemble_enqueue(cb_graph *h, uint32_t m, int prec, uint32_t n_out, double *S,
                            double *log_scale, cudaStream_t s) {
  int rc = lanczos_run(h, h->ws, 0, h->n_inst, m, prec, s);
  if (rc == CB_OK) rc = tridiag_run(h, 0, h->n_inst, prec, s);
  if (rc == CB_OK) rc = combine_ensemble(h, prec, n_out, S, log_scale, s);
  return rc;
}

static int ensemble_graph(cb_graph *h, uint32_t m, int prec, uint32_t n_out, double *S,
                          double *log_scale, cudaStream_t s) {
  cb_graph::GraphEntry *hit = nullptr;
  for (auto &g : h->graphs)
    if (g.m == m && g.prec == prec && g.reorth == h->reorth && g.n_out == n_out && g.S == S &&
        g.log_scale == log_scale &&
        g.ws_gen == h->ws.gen)
      hit = &g;
  if (hit && hit->exec) return cuda_error(cudaGraphLaunch(hit->exec, s), "cb_ensemble_scores: graph launch");
  if (!hit) {  // first call with this shape: launch directly, capture on a repeat
    if (h->graphs.size() >= 8) {
      if (h->graphs.front().exec) cudaGraphExecDestroy(h->graphs.front().exec);
      h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back({m, prec, n_out, S, log_scale, h->ws.gen, h->reorth, nullptr});
    return ensemble_enqueue(h, m, prec, n_out, S, log_scale, s);
  }
  cudaError_t e = cudaSuccess;
  if (!h->capture_stream) e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_error(e, "cb_ensemble_scores: capture stream");
  // the capture stream itself runs nothing; the caller's pending work is ordered
  // before the replay by launching the graph on the caller's stream
  e = cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return cuda_error(e, "cb_ensemble_scores: begin capture");
  int rc = ensemble_enqueue(h, m, prec, n_out, S, log_scale, h->capture_stream);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(h->capture_stream, &graph);
  if (rc != CB_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_error(e, "cb_ensemble_scores: end capture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_error(e, "cb_ensemble_scores: instantiate");
  hit->exec = exec;
  return cuda_error(cudaGraphLaunch(exec, s), "cb_ensemble_scores: graph launch");
}

CB_API int cb_ensemble_scores(cb_graph *h, uint32_t m, int prec, uint32_t n_out, double *S,
                              double *log_scale, cb_inst_report *rep, void *stream) {
  NvtxRange nvtx_range("cb_ensemble_scores");
  if (!h || !S || !log_scale) return set_error(CB_ERR_ARG, "cb_ensemble_scores: null argument");
  if (m < 1 || m > CB_MAX_M) return set_error(CB_ERR_ARG, "cb_ensemble_scores: need 1 <= m <= CB_MAX_M");
  const bool reorth = split_prec(prec);
  if (prec != CB_FP32 && prec != CB_FP64) return set_error(CB_ERR_ARG, "cb_ensemble_scores: bad precision");
  h->reorth = reorth;
  if (n_out < h->n_max) return set_error(CB_ERR_ARG, "cb_ensemble_scores: n_out < largest n");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = ensure_workspace(h, h->ws, m, prec, s);
  if (rc != CB_OK) return rc;
  const bool use_graph = !g_prof_on && !rep && !std::getenv("CB_NO_GRAPH");
  h->basis_m = 0;
  rc = use_graph ? ensemble_graph(h, m, prec, n_out, S, log_scale, s)
                 : ensemble_enqueue(h, m, prec, n_out, S, log_scale, s);
  if (rc == CB_OK) {  // ws now holds the basis from 1 of every realisation
    h->basis_m = m;
    h->basis_prec = prec;
    h->basis_reorth = h->reorth;
    h->basis_gen = h->ws.gen;
  }
  if (rc == CB_OK && rep) rc = fill_report(h, 0, h->n_inst, rep, s);
  return rc;
}
