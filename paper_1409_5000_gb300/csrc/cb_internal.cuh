// Internal declarations shared by the CUDA translation units of libcb.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cb.h"

#define CB_API extern "C" __attribute__((visibility("default")))

namespace cb {

// ---------------------------------------------------------------------------
// Layout constants
// ---------------------------------------------------------------------------
constexpr int kThreads = 256;        // threads per CTA in the SpMV / finalize kernels
constexpr int kTileRows = 256;       // most rows per SpMV tile
constexpr uint32_t kTileNnz = 6144;  // a tile closes before it exceeds this many entries
constexpr int kFinRows = 2048;       // nodes per finalize tile (256 threads x 8)
constexpr int kGroup = 32;           // reduction slots per last-arriver group
constexpr uint32_t kHeavyDeg = 8192; // rows above this degree are split across CTAs
constexpr uint32_t kChunk = 4096;    // edges per heavy-row chunk
constexpr uint32_t kLongDeg = 1024;  // rows above this (<= kHeavyDeg) use the whole CTA
constexpr int kNodeAlign = 32;       // per-instance node offset alignment (elements)
// Realisations of at most kSmallN nodes and kSmallNnz entries can run all
// their Lanczos steps in one launch, one CTA each (lanczos_small_kernel).
constexpr uint32_t kSmallN = 8192;
constexpr uint32_t kSmallNnz = 1u << 20;

// Column-blocked SpMV (FP32): a CTA of kBThreads owns kBTileRows rows,
// kBRowsPerThread rows per thread (strided by kBThreads); the columns are cut into
// blocks of kBCol that are staged in shared memory, so every gather of v_j
// is a shared-memory load.
constexpr int kBThreads = 1024;
constexpr int kBRowsPerThread = 16;
constexpr int kBTileRows = kBThreads * kBRowsPerThread;  // 16384
constexpr uint32_t kBColBits = 14;
constexpr uint32_t kBCol = 1u << kBColBits;              // 16384 floats = 64 KB per buffer
constexpr uint32_t kBBuf = kBCol + 4;                    // floats per staging buffer (16-byte multiple)
// A padding element of lane l adds into the lane's spare row sum (slot
// kBRowsPerThread), which no row reads.
__host__ __device__ constexpr uint32_t kBPadOff(uint32_t l) { return kBRowsPerThread * kBThreads + l; }
constexpr uint32_t kBMaxBlocks = 32;                     // blocked when n <= 32 * kBCol
constexpr uint32_t kBLongDeg = 512;                      // longer rows: whole-CTA global gathers

// Two-phase (propagation-blocked) SpMV (FP32), for realisations too large
// for the column-blocked kernel.  Columns are cut into source tiles of kPSrc
// nodes and rows into bins whose entries fit a shared-memory region.
// Phase 1 stages a source tile of W_j in shared memory and writes, for every
// entry, the gathered value into its bin's region of a value array; phase 2
// copies a bin's region into shared memory and sums each row from there.
// Both phases gather from shared memory only.
constexpr uint32_t kPSrcBits = 15;
constexpr uint32_t kPSrc = 1u << kPSrcBits;  // nodes per source tile (128 KB of W_j)
constexpr uint32_t kPMaxSrc = 4096;          // source tiles per realisation (n <= 2^27)
constexpr uint32_t kPGroup = 8;              // slots per group: one 32-byte sector of values
constexpr uint32_t kPRegion = 16384;         // slots per bin region (64 KB)
constexpr uint32_t kPBinRows = 1024;         // most rows per bin
constexpr int kP1Threads = 1024;             // phase-1 CTA (one per SM: 128 KB tile)
constexpr int kP2Threads = 512;              // phase-2 CTA (two per SM: ~111 KB each)
// Phase 2 sums rows in pieces of at most kPPiece entries, 32 pieces (one per
// lane) at a time; a bin has at most kPMaxPieces pieces, and bins are closed
// so that their slot array (the pieces' region slots, padded) stays within
// kPSlotsMax u16 words: 32 kPPiece + the sum over rows of deg + (deg & 1)
// bounds it.
constexpr uint32_t kPPiece = 16;
constexpr uint32_t kPMaxPieces = kPBinRows + kPRegion / kPPiece;
constexpr uint32_t kPMaxSlices = kPMaxPieces / 32;
constexpr uint32_t kPSlotsMax = 17408;

// A bin: consecutive rows [row0, row1) of realisation inst, none heavier
// than kHeavyDeg, whose entries (with chunk padding) fit kPRegion slots.
struct PBin {
  uint32_t inst, row0, row1, pad;
};

// What a phase-2 CTA needs to start on a bin: its region (first group of the
// value array, bytes), its plan (first u16 word, bytes of the part copied to
// shared memory, word offset of the rows' piece offsets), its rows (vector
// offset of the first, count), its realisation and its alpha-term slot.
struct P2Desc {
  uint64_t xg0, plan, node;
  uint32_t reg_bytes, head_bytes, pf, inst, nrows, slot;
};
static_assert(sizeof(P2Desc) == 48, "P2Desc is three 16-byte units");

// Two-level deterministic reduction plan of one instance for one kernel kind:
// one partial per slot, slots grouped by kGroup; the last CTA to arrive in a
// group sums the group, the last group of the instance sums the groups.
struct RedPlan {
  uint32_t slot_base, n_slots, group_base, n_groups;
};

// Per-realisation descriptor (device copy and host copy).
struct InstDesc {
  uint64_t node_base;  // offset of node 0 in every Krylov vector
  uint64_t edge_base;  // offset of the first column index in col[]
  uint64_t rp_base;    // offset of row_ptr[0] in the row_ptr array
  uint32_t n;
  uint32_t nnz;        // CSR entries of the realisation (< 2^32)
  uint32_t tile_base, n_tiles;    // SpMV tiles (<= kTileRows rows, ~kTileNnz entries)
  uint32_t heavy_base, n_heavy;   // heavy rows
  uint32_t chunk_base, n_chunks;  // heavy-row chunks
  uint32_t fin_base, n_fin;       // finalize tiles (kFinRows nodes each)
  RedPlan spmv;                   // slots: n_tiles normal tiles, then n_heavy rows
  RedPlan fin;                    // slots: n_fin tiles
  uint32_t blocked, nb;           // column-blocked FP32 SpMV? number of column blocks
  uint32_t btile_base, n_btiles;  // blocked tiles (kBTileRows rows each)
  RedPlan bspmv;                  // slots: n_btiles
  uint32_t pb, pns;               // two-phase FP32 SpMV? number of source tiles
  uint32_t ptile_base;            // first source tile (handle-wide index)
  uint32_t pbin_base, n_pbin;     // bins
  uint32_t pad_p[3];
  uint64_t pmat_base;             // offset of the [bin][pns + 1] chunk tables
  RedPlan pspmv;                  // slots: n_pbin bins, then n_heavy rows
};

struct HeavyRow {
  uint32_t inst, row, chunk_base, n_chunks;
};

// Per-instance Krylov scalars, FP64.  Index j is the 0-based Lanczos step.
struct Scalars {
  double *alpha;  // [n_inst * ms]
  double *beta;   // [n_inst * ms]   beta[j] = ||w_{j+1}||
  double *scale;  // [n_inst * ms]   v_j = scale[j] * W_j
  double *gamma;  // [n_inst * ms]   combine weights beta0 c_j scale_j
  double *theta;  // [n_inst]
  uint32_t *meff; // [n_inst]        steps kept; m until a breakdown
  int32_t *status;// [n_inst]
  uint32_t ms;    // stride (>= m + 1)
};

// Device workspace for one (m, precision) pair.
struct Workspace {
  int prec = -1;
  uint32_t m = 0;
  void *V = nullptr;       // (m + 1) vectors of vec_stride elements
  uint64_t vec_stride = 0; // elements per Krylov vector (all instances)
  Scalars sc{};
  double *part = nullptr;  // reduction partials per slot
  double *gpart = nullptr; // reduction partials per group
  uint32_t *gcnt = nullptr;// arrival counters per group
  uint32_t *icnt = nullptr;// arrival counters per instance
  double *cpart = nullptr; // heavy-row chunk partials
  double *rpart = nullptr; // reorthogonalisation: per finalize tile, ms dot partials
  double *rh = nullptr;    // reorthogonalisation: per realisation, ms coefficients
  uint32_t *hcnt = nullptr;// heavy-row arrival counters
  size_t blob_bytes = 0;
  void *blob = nullptr;    // single allocation backing sc/part/gpart/cnt
  uint64_t gen = 0;        // allocation generation (process-wide unique)
};

// Buffers of the adjoint (cb_scores_backward).
struct BackWork {
  int prec = -1;
  uint32_t m = 0, mpad = 0;  // node-major row length (m rounded up to 4)
  void *P = nullptr;         // node-major P = V_w K   [total_nodes_padded x mpad]
  void *U = nullptr;         // node-major U = V_1     [total_nodes_padded x mpad]
  double *K = nullptr;       // per realisation coefficient matrix [n_inst x ms x ms]
  double *theta = nullptr;   // per realisation shift
  uint32_t *cnt = nullptr;   // per realisation |top-k within [0, n_r)|
  void *blob = nullptr;
};

}  // namespace cb

struct cb_graph {
  int device = 0;
  bool csr_only = false;  // CB_CSR_ONLY: no column-blocked format
  bool force_pb = false;  // CB_TWO_PHASE: the two-phase format for every realisation
  uint32_t n_inst = 0;
  uint32_t n_max = 0;
  uint64_t total_nodes_padded = 0;  // sum of padded node ranges
  uint64_t total_nnz = 0;
  uint32_t total_tiles = 0, total_heavy = 0, total_chunks = 0, total_fin = 0;
  uint32_t total_slots = 0, total_groups = 0;
  int lanes = 8;  // lanes per row for short rows (1, 2, 4, 8, 16, 32)
  int path = CB_PATH_AUTO;  // FP32 SpMV path (cb_graph_set_path)
  uint32_t n_sm = 1;        // SMs of the handle's device
  bool owns_csr = true;     // false while an upload holds CSR arrays its caller still owns
  std::vector<cb::InstDesc> inst;        // host copy
  std::vector<cb::HeavyRow> heavy;       // host copy
  // device arrays
  uint32_t *col = nullptr;
  uint32_t *row_ptr = nullptr;
  cb::InstDesc *d_inst = nullptr;
  uint32_t *d_tile_inst = nullptr;       // instance of each normal tile
  uint2 *d_tile_rows = nullptr;          // [first, last) local row of each normal tile
  cb::HeavyRow *d_heavy = nullptr;
  uint32_t *d_chunk_heavy = nullptr;     // heavy-row index of each chunk
  uint32_t *d_fin_inst = nullptr;        // instance of each finalize tile
  uint32_t *d_mirror = nullptr;          // per CSR entry (i, j): position of (j, i) in its
                                         // realisation (built by the first adjoint call)
  // column-blocked format (FP32 SpMV), for realisations with blocked = 1
  uint32_t total_btiles = 0;
  uint64_t total_bseg = 0;               // (tile, column block) segments
  uint32_t *d_btile_inst = nullptr;      // realisation of each blocked tile
  uint64_t *d_bseg_base = nullptr;       // first (tile, column block) segment of each tile
  uint64_t *d_bwstart = nullptr;         // per (segment, warp): first element of its region
  uint64_t *d_bwscan = nullptr;          // scratch of the prefix that makes d_bwstart
  uint32_t *d_bwlen = nullptr;           // per (segment, warp): steps T of its stream (even)
  uint16_t *d_bcnt = nullptr;            // per (segment, lane): its elements (format build)
  uint32_t *d_belem = nullptr;           // stream elements: local column | row-sum offset << kBColBits
  uint32_t *d_blong_ptr = nullptr;       // per blocked tile: range in d_blong_rows
  uint32_t *d_blong_rows = nullptr;      // local rows with degree > kBLongDeg, in row order
  // two-phase format (FP32 SpMV), for realisations with pb = 1
  uint32_t total_ptiles = 0, total_pbins = 0;
  uint32_t pns_max = 0;                  // most source tiles of one realisation
  uint64_t total_pgroups = 0;            // groups of kPGroup slots (stream and value array)
  cb::PBin *d_pbin = nullptr;
  std::vector<uint64_t> ptbase;          // host copy of d_ptbase
  uint64_t *d_ptbase = nullptr;          // per source tile: first group of its stream (+ total)
  uint32_t *d_ptotal = nullptr;          // per source tile: groups of its stream (build)
  uint32_t *d_ptile_inst = nullptr;      // per source tile: its realisation
  uint32_t *d_proff = nullptr;           // [bin][s]: group offset of chunk (s, bin) in the
                                         //   bin region ([bin][pns]: groups of the region)
  uint32_t *d_pcstart = nullptr;         // [bin][s]: group offset of chunk (s, bin) in
                                         //   tile s's stream
  uint32_t *d_prtot = nullptr;           // per bin: groups of its region (build)
  uint64_t *d_pxbase = nullptr;          // per bin: first group of its region (+ total)
  uint64_t *d_pxscan = nullptr;          // scratch of the prefix that makes d_pxbase
  uint16_t *d_ppos = nullptr;            // per CSR entry of a bin row: its slot in the region
  uint16_t *d_psrc = nullptr;            // per stream slot: source node within its tile
  uint32_t *d_pgdst = nullptr;           // per stream group: its group in the value array
  float *d_pX = nullptr;                 // value array: bin regions, phase 1 writes them
  uint16_t *d_psl = nullptr;             // per bin: the phase-2 plan (sliced rows), u16 words
  uint64_t *d_psloff = nullptr;          // per bin: first word of its plan (+ total)
  cb::P2Desc *d_pdesc = nullptr;         // per bin: its phase-2 copies
  // captured ensemble pass (one CUDA graph per m / precision / outputs)
  struct GraphEntry {
    uint32_t m;
    int prec;
    uint32_t n_out;
    double *S, *log_scale;
    uint64_t ws_gen;  // workspace allocation the graph was captured against
    bool reorth;      // captured with reorthogonalisation
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t capture_stream = nullptr;
  // ws holds the Lanczos basis from 1 of every realisation at this depth and
  // precision (an ensemble pass or an adjoint ran last); 0 = not valid
  uint32_t basis_m = 0;
  int basis_prec = -1;
  bool basis_reorth = false;
  // the current call's CB_REORTH flag (set by every entry point that runs
  // the Lanczos recurrence; read by lanczos_run)
  bool reorth = false;
  uint64_t basis_gen = 0;
  // test hook (cb_debug_stall_tile): this column-blocked tile's first column
  // block is expected but never copied, so its bounded wait runs out
  uint32_t stall_btile = UINT32_MAX;
  cb::Workspace ws;   // Krylov basis from 1 (forward)
  cb::Workspace ws2;  // Krylov basis from the top-k indicator (adjoint)
  cb::BackWork bw;    // adjoint buffers
};

namespace cb {
// ---------------------------------------------------------------------------
// Bounds checks of the debug build (compiled with -DCB_DEBUG; nothing in the
// release build).  A failed check counts a violation, records the site and
// index of the first one, and the caller skips the access: no check traps or
// faults.  Each translation unit keeps its own record (device variables are
// per unit without relocatable device code) and exports a reader that
// cb_debug_violations sums.
// ---------------------------------------------------------------------------
enum DebugSite : uint32_t {
  kDbgBlockedElem = 1,   // column-blocked SpMV: stream element (column, row slot)
  kDbgBlockedFill = 2,   // column-blocked format: stream write position
  kDbgCsrCol = 3,        // CSR gathers of the SpMV kernels: column index
  kDbgTwoPhaseSrc = 4,   // two-phase phase 1: source offset within the tile
  kDbgTwoPhaseDst = 5,   // two-phase phase 1: group place in the value array
  kDbgTwoPhasePos = 6,   // two-phase phase 2: slot in the bin region
  kDbgAdjointCol = 7,    // adjoint mirror and edge kernels: column index
};
#ifdef CB_DEBUG
#define CB_DEBUG_STATE()                                                                    \
  static __device__ unsigned int g_dbg_count = 0;                                          \
  static __device__ unsigned long long g_dbg_first = 0;                                    \
  static __device__ __forceinline__ bool dbg_ok(bool ok, uint32_t site, uint64_t idx) {    \
    if (!ok && atomicAdd(&g_dbg_count, 1u) == 0)                                            \
      g_dbg_first = ((unsigned long long)site << 48) | (idx & 0xffffffffffffull);           \
    return ok;                                                                              \
  }
#define CB_DEBUG_READER(name)                                                               \
  int dbg_read_##name(uint32_t *count, uint64_t *first, bool reset) {                       \
    unsigned int c = 0;                                                                     \
    unsigned long long f = 0;                                                               \
    cudaError_t e = cudaMemcpyFromSymbol(&c, g_dbg_count, sizeof c);                        \
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&f, g_dbg_first, sizeof f);              \
    if (e == cudaSuccess && reset) {                                                        \
      const unsigned int z = 0;                                                             \
      const unsigned long long zf = 0;                                                      \
      e = cudaMemcpyToSymbol(g_dbg_count, &z, sizeof z);                                    \
      if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_dbg_first, &zf, sizeof zf);            \
    }                                                                                       \
    *count = c;                                                                             \
    *first = f;                                                                             \
    return e == cudaSuccess ? 0 : 1;                                                        \
  }
#define CB_DCHECK(cond, site, idx) dbg_ok((cond), (site), (idx))
#else
#define CB_DEBUG_STATE()
#define CB_DEBUG_READER(name)                                                               \
  int dbg_read_##name(uint32_t *count, uint64_t *first, bool) {                             \
    *count = 0;                                                                             \
    *first = 0;                                                                             \
    return 0;                                                                               \
  }
#define CB_DCHECK(cond, site, idx) true
#endif
int dbg_read_lanczos(uint32_t *count, uint64_t *first, bool reset);
int dbg_read_blocked(uint32_t *count, uint64_t *first, bool reset);
int dbg_read_twophase(uint32_t *count, uint64_t *first, bool reset);
int dbg_read_adjoint(uint32_t *count, uint64_t *first, bool reset);

// fn(i) for i in [0, n) on the host, spread over the hardware threads
void parallel_for(uint32_t n, const std::function<void(uint32_t)> &fn);

// Host-to-device copy of a small host table during an upload, staged through
// a library-owned pinned buffer so that it is truly asynchronous: a copy from
// pageable memory would wait for the copy engine, which the upload's bulk
// copies keep busy for the whole transfer, and hold the host thread with it.
// The staging buffer is recycled when the upload returns (cb_api.cu).
cudaError_t stage_h2d(void *dst, const void *src, size_t bytes, cudaStream_t s);
// A pinned host block of `bytes` from the same staging arena, valid until
// the upload returns (nullptr if pinned memory cannot be had).
char *stage_reserve(size_t bytes);

// error plumbing (cb_api.cu)
// Device memory of handles and workspaces.  By default it comes from a
// library-owned stream-ordered pool per device that keeps freed memory for
// the next upload (cudaFree of multi-GB arrays costs ~1 ms per GB);
// cb_release_cached_memory trims it, CB_NO_POOL selects plain cudaMalloc.
// dev_free synchronises the device first, like cudaFree.
cudaError_t dev_alloc(void **p, size_t bytes);
void dev_free(void *p);
template <typename P>
inline cudaError_t dev_alloc_n(P **p, size_t count) {
  return dev_alloc(reinterpret_cast<void **>(p), count * sizeof(P) + 64);
}

// A named NVTX range on the calling host thread for the lifetime of the
// object: library calls and their phases show up by name in Nsight
// timelines.  Without an attached tool it costs a check of one pointer.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

int set_error(int code, const std::string &msg);
// Splits a prec argument into the precision (returned in prec) and the
// CB_REORTH flag (returned).
inline bool split_prec(int &prec) {
  const bool r = (prec & CB_REORTH) != 0;
  prec &= ~CB_REORTH;
  return r;
}
// host error for a failed realisation's device status (CB_ERR_TIMEOUT or CB_ERR_NONFINITE)
int status_error(int32_t st);
int cuda_error(cudaError_t e, const char *what);

// One-time hint that a kernel should run with the shared-memory-heavy L1 /
// shared split that the column-blocked SpMV needs, so that consecutive
// launches of the library's kernels do not reconfigure the SM (cb_api.cu).
void prefer_shared_impl(const void *kernel);
template <typename K>
inline void prefer_shared(K *kernel) {
  prefer_shared_impl(reinterpret_cast<const void *>(kernel));
}

// optional per-launch event timing (cb_api.cu); no-ops unless enabled
int prof_begin(int kernel, cudaStream_t s);
void prof_end(int token, cudaStream_t s);

// column-blocked format builder (cb_blocked.cu); host row_ptr views per realisation
// Upload copies run in groups of realisations on a stream of their own; the
// event of a group fires when realisations [previous end, r_end) are on the
// device.
struct CopyGroup {
  uint32_t r_end;
  cudaEvent_t ev;
};
// Exclusive prefix of u32 counts into u64 offsets (cb_generate.cu):
// out[0..n], out[n] = total; bsum holds n / 4096 + 2 u64 of scratch.
cudaError_t exclusive_scan(const uint32_t *in, uint64_t n, uint64_t *out, uint64_t *bsum,
                           cudaStream_t s);
// Column-blocked format builder (cb_blocked.cu), in three calls so that an
// upload's host work runs while the device builds the format:
//   blocked_count -- layout from the realisation sizes, the count pass (per
//     copy group, as its columns land) and the stream prefix, all queued;
//   blocked_fill  -- waits for the stream total, allocates the streams and
//     queues the fill pass (no wait for it);
//   blocked_long_rows -- the rows summed from the CSR, from host row_ptr.
// h->d_inst must be allocated before blocked_count; the caller synchronises
// the stream before the handle is used.
struct BlockedBuild {
  uint64_t *result = nullptr;  // pinned: stream total, then the sortedness flag
  cudaEvent_t ev = nullptr;    // recorded after the count pass and its prefix
  ~BlockedBuild() {
    if (ev) cudaEventDestroy(ev);
  }
};
int blocked_count(cb_graph *h, cudaStream_t s, const std::vector<CopyGroup> &groups,
                  BlockedBuild &bb);
int blocked_fill(cb_graph *h, cudaStream_t s, BlockedBuild &bb);
int blocked_long_rows(cb_graph *h, const std::vector<const uint32_t *> &rp_host, cudaStream_t s);
void free_blocked(cb_graph *h);
// two-phase format builder (cb_twophase.cu); force: every realisation, else
// those above the column-blocked size limit
// cb_graph_upload from device arrays that the handle takes over instead of
// copying (cb_api.cu): col_all holds the realisations' columns concatenated
// (sum of nnz + 4 entries), rp_all their row_ptr arrays concatenated (sum of
// n + 1 entries), and row_ptr[r] / col[r] point into them at those offsets.
// On success the handle owns both; on failure the caller still does.
int upload_adopt(uint32_t n_inst, const uint32_t *n, const uint64_t *nnz,
                 const uint32_t *const *row_ptr, const uint32_t *const *col, uint32_t *col_all,
                 uint32_t *rp_all, void *stream, cb_graph **out);
int build_twophase(cb_graph *h, const std::vector<const uint32_t *> &rp_host, cudaStream_t s,
                   const std::vector<CopyGroup> &groups, bool force);
void free_twophase(cb_graph *h);

// workspace for depth m in precision prec (cb_api.cu)
int ensure_workspace(cb_graph *h, Workspace &W, uint32_t m, int prec, cudaStream_t s);
void free_workspace(Workspace &W);
void free_backwork(BackWork &B);  // cb_adjoint.cu

// kernel launchers (cb_lanczos.cu).  Range of realisations [r0, r1).  The
// start vector is 1, or, with start_idx, the indicator of the k distinct
// node indices start_idx[0..k) (device array) restricted to [0, n_r).
// start_idx: none (start vector 1), an index set shared by all realisations
// (k entries), or with per_inst one start node per realisation (e_idx[r-r0]).
// restart_scale (device, double[N]): a restarted cycle; W_0 already holds
// the start vector with scale restart_scale[r] (0: nothing to do).
int lanczos_run(cb_graph *h, Workspace &W, uint32_t r0, uint32_t r1, uint32_t m, int prec,
                cudaStream_t s, const uint32_t *start_idx = nullptr, uint32_t k = 0,
                bool per_inst = false, const double *restart_scale = nullptr);
// tridiagonal exp (cb_tridiag.cu)
int tridiag_run(cb_graph *h, uint32_t r0, uint32_t r1, int prec, cudaStream_t s);
// combine (cb_combine.cu)
int combine_single(cb_graph *h, uint32_t r, int prec, double *y, double *log_scale,
                   cudaStream_t s);
int combine_ensemble(cb_graph *h, int prec, uint32_t n_out, double *S, double *log_scale,
                     cudaStream_t s);
// eq. 5 sum of FP64 per-realisation terms Y (node_base layout), shifts in h->ws.sc.theta
int combine_sum_f64(cb_graph *h, const double *Y, uint32_t n_out, double *S, double *log_scale,
                    cudaStream_t s);
// 8 consecutive elements (16- or 32-byte aligned) as one or two vector accesses.
template <typename T>
struct Vec8;
template <>
struct Vec8<float> {
  static __device__ __forceinline__ void load(const float *p, float (&v)[8]) {
    const float4 a = *reinterpret_cast<const float4 *>(p), b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  }
  static __device__ __forceinline__ void store(float *p, const float (&v)[8]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4 *>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
  }
};
template <>
struct Vec8<double> {
  static __device__ __forceinline__ void load(const double *p, double (&v)[8]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double2 a = *reinterpret_cast<const double2 *>(p + 2 * q);
      v[2 * q] = a.x;
      v[2 * q + 1] = a.y;
    }
  }
  static __device__ __forceinline__ void store(double *p, const double (&v)[8]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) *reinterpret_cast<double2 *>(p + 2 * q) = make_double2(v[2 * q], v[2 * q + 1]);
  }
};

}  // namespace cb
