/*
 * cb.h -- C ABI of the GB300 (sm_103a) summed-communicability library.
 *
 * Method (Fioriti & Chinnici, arXiv 1409.5000):
 *   - A is the symmetric 0/1 adjacency matrix of a simple undirected graph
 *     (section "Signal processing on graphs").
 *   - Every node i is scored by its Estrada-Benzi total communicability
 *     EBTC_i = (e^A 1)_i, the row sums of e^A (eq. 4).
 *   - e^A 1 is evaluated with a Krylov (Lanczos) approximation
 *     ("Identification algorithm": the row sums come directly from e^A 1
 *     at linear cost).
 *   - Scores are summed over N background realisations that carry the same
 *     embedded target (eq. 5).
 *   - The k largest summed scores are the recovered target
 *     ("Identification algorithm", k = the target size).
 *
 * Conventions shared by every call:
 *   - Return value: CB_OK (0) or one of the CB_ERR_* codes below.  On error
 *     cb_last_error() returns a message for the calling host thread.
 *   - Streams: `stream` is a cudaStream_t passed as void*; NULL means the
 *     legacy default stream.  Unless a call says otherwise it is
 *     asynchronous: it enqueues work on `stream` and returns.  Device
 *     buffers passed in must stay valid until that work completes.
 *   - Pointers: "device" means a CUDA device pointer on the current device
 *     (for example torch tensor storage); "host" means ordinary or pinned
 *     host memory.
 *   - Scores may exceed the FP64 range (e^lambda_max for large graphs).
 *     They are therefore returned as a scaled vector y plus one log scale:
 *     score_i = exp(log_scale) * y_i.
 *   - Precision: CB_FP32 keeps Krylov vectors and SpMV sums in FP32, and the
 *     recurrence scalars, tridiagonal solve and cross-realisation sums in
 *     FP64.  CB_FP64 computes everything in FP64.
 */
#ifndef CB_H_
#define CB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CB_OK 0
#define CB_ERR_ARG 1       /* invalid argument (null pointer, size, index) */
#define CB_ERR_CUDA 2      /* a CUDA runtime call failed */
#define CB_ERR_OOM 3       /* device allocation failed */
#define CB_ERR_TIMEOUT 4   /* a bounded device-side wait gave up */
#define CB_ERR_NONFINITE 5 /* a recurrence scalar became NaN or Inf */
#define CB_ERR_STATE 6     /* call not valid in the current state */

/* precision modes */
#define CB_FP32 0
#define CB_FP64 1
/* OR-ed into a prec argument: full reorthogonalisation.  Each new Lanczos
 * vector is orthogonalised against every previous one by two passes of
 * classical Gram-Schmidt (the scheme of the FP64 oracle), before its norm
 * beta_j is taken.  Step j then reads about 4 (j + 2) extra vectors.  The
 * paper does not fix this; without it the approximation of e^A 1 stays
 * accurate in finite precision (Greenbaum 1989; Musco, Musco & Sidford 2018),
 * so it is off by default. */
#define CB_REORTH 0x100

/* cb_graph_upload flags */
#define CB_VALIDATE 1u    /* check CSR invariants on the host before upload */
#define CB_DEVICE_PTRS 2u /* row_ptr[r] / col[r] are device pointers */
#define CB_CSR_ONLY 4u    /* no column-blocked format: every FP32 SpMV gathers from the CSR */
#define CB_TWO_PHASE 8u   /* the two-phase format for every realisation (default: n > 2^19 only) */

/* FP32 SpMV path of a handle (cb_graph_set_path) */
#define CB_PATH_AUTO 0    /* one launch of all m steps (one CTA per realisation) when every
                             realisation of the call has n <= 8192 and <= 2^20 entries and no
                             reorthogonalisation is asked; otherwise, per step, the
                             column-blocked kernel when the handle has >= one blocked tile per
                             SM, two-phase kernels where built, else tiled CSR */
#define CB_PATH_FORMATS 1 /* column-blocked and two-phase kernels wherever their format was built */
#define CB_PATH_CSR 2     /* the tiled-CSR kernel for every realisation */

/* largest Krylov depth accepted by the compute calls */
#define CB_MAX_M 128
/* largest k accepted by cb_topk */
#define CB_MAX_TOPK 4096
#define CB_MAX_SC_NODES 1024
#define CB_MAX_CYCLES 1024 /* restart cycles of cb_ensemble_scores_restarted */

typedef struct cb_graph cb_graph;

/* Per-realisation report, filled when a compute call is given a non-NULL
 * report array (the call then synchronises `stream` before returning). */
typedef struct {
  uint32_t m_eff;   /* Lanczos steps kept (< m after an exact breakdown) */
  int32_t status;   /* CB_OK or CB_ERR_NONFINITE for this realisation */
  double theta;     /* lambda_max(T_m_eff): this realisation's log scale */
  double beta_last; /* last residual norm beta_m (0 after breakdown) */
  double beta0;     /* ||1|| = sqrt(n_r) */
} cb_inst_report;

/*
 * cb_graph_upload -- store N graphs (one per background realisation) on the
 * current device as pattern-only CSR.
 *   n_inst     number of realisations N (>= 1).
 *   n[r]       node count of realisation r (>= 1).  Host array.
 *   nnz[r]     directed CSR entries of realisation r (2|E_r|, < 2^32).
 *              Host array.
 *   row_ptr[r] uint32[n[r]+1] row offsets (row_ptr[r][0] = 0).  Host
 *              pointers unless CB_DEVICE_PTRS is set.
 *   col[r]     uint32[nnz[r]] column indices, each row sorted ascending
 *              without duplicates.  Host pointers unless CB_DEVICE_PTRS is set.
 *   flags      CB_VALIDATE: check that row_ptr is monotone, rows are sorted
 *              without duplicates, cols are in range, there are no
 *              self-loops and the pattern is symmetric (host arrays only;
 *              O(nnz * degree) host time).  Without it, unsorted rows are
 *              still detected on the device (CB_ERR_ARG).
 *              CB_DEVICE_PTRS: row_ptr[r] and col[r] are device pointers.
 *              CB_CSR_ONLY: skip the column-blocked format that FP32 calls
 *              use for realisations with n <= 32 * 16384, and the two-phase
 *              format of larger ones; they then run the tiled-CSR SpMV (same
 *              recurrence, FP32 rounding differs), the upload is shorter and
 *              the handle ~3 B per entry smaller.
 *              CB_TWO_PHASE: build the two-phase format (FP32 SpMV in two
 *              passes over a stream of edge values, both gathering from
 *              shared memory) for every realisation instead of only those
 *              with n > 32 * 16384; about 11 B per entry on the device.
 *              Realisations with n > 1170 * 32768 (about 3.8e7) run the
 *              tiled-CSR SpMV: a bin must hold any row of up to 8192
 *              entries beside the worst-case padding of its chunks.
 *              CB_CSR_ONLY with CB_TWO_PHASE, or other bits: CB_ERR_ARG.
 *              A column index >= n fails the two-phase build (CB_ERR_ARG).
 *   stream     used for the copies.  The call synchronises `stream` before
 *              returning, so the input arrays may be freed afterwards.
 *   out        receives the handle.
 * The pattern must be symmetric (A = A^T, paper section "Signal processing
 * on graphs"); duplicates and self-loops are the caller's responsibility.
 * The library owns all device memory of the handle until cb_graph_free().
 * Realisations may have different n; realisation r then contributes 0 to
 * nodes i >= n[r] in the ensemble sum.
 */
int cb_graph_upload(uint32_t n_inst, const uint32_t *n, const uint64_t *nnz,
                    const uint32_t *const *row_ptr, const uint32_t *const *col,
                    uint32_t flags, void *stream, cb_graph **out);

/*
 * cb_graph_generate_er -- N Erdos-Renyi backgrounds with one embedded
 * target, generated on the device into a new handle (paper, "Multiple
 * backgrounds scenario": the N realisations summed by eq. 5, all sharing the
 * target sub-graph; the backgrounds never cross the host-device link).
 * Model: a fixed-draw G(n, M) reading of the paper's ER graphs.  With
 * SplitMix64 in counter form, output(c) = mix(seed + (c + 1) * G),
 * G = 0x9E3779B97F4A7C15 (Steele, Lea & Flood, OOPSLA 2014), realisation r
 * makes draws t = 0 .. m_draws[r]-1 with c = r * 2^32 + t, and draw t is the
 * pair u = (hi32(z) * n[r]) >> 32, v = (lo32(z) * n[r]) >> 32.  Draws with
 * u == v are dropped, repeated pairs collapse, the target edges are added to
 * every realisation (an edge with an endpoint >= n[r] is skipped there), and
 * each row is sorted: a simple undirected graph as a symmetric CSR pattern.
 * m_draws = dbar * n / 2 gives mean degree ~dbar.
 *   n_inst     N >= 1.
 *   n          host uint32[N], nodes per realisation, each >= 1.
 *   m_draws    host uint64[N], draws per realisation; m_draws[r] + n_tedges < 2^31.
 *   seed       generator seed.
 *   n_tedges   number of target edges (0 for none).
 *   tedges     host uint32[2 * n_tedges], pairs (u, v); read during the call.
 *   stream     stream for the work; the call synchronises it.
 *   out        receives the handle (as from cb_graph_upload).
 * Errors: CB_ERR_ARG (null arrays, n = 0, too many draws, endpoints
 * >= 2^31, >= 2^32 entries in one realisation), CB_ERR_CUDA.  Device
 * temporaries (about 3x the final CSR) are released before returning.
 */
int cb_graph_generate_er(uint32_t n_inst, const uint32_t *n, const uint64_t *m_draws,
                         uint64_t seed, uint32_t n_tedges, const uint32_t *tedges, void *stream,
                         cb_graph **out);

/*
 * cb_graph_generate_ws -- N Watts-Strogatz small-world backgrounds with one
 * embedded target, generated on the device into a new handle (the paper's
 * small-world backgrounds, Table 2 and the single-background scenario).
 * Model: the ring lattice in which node i links to i + 1 .. i + k/2 (mod n),
 * every ring edge rewired with probability p to a uniform node.  With the
 * counter generator of cb_graph_generate_er, realisation r makes draws
 * t = 0 .. n[r] k/2 - 1, c = r * 2^32 + t; draw t = i k/2 + (d - 1) is the
 * edge (i, (i + d) mod n[r]), whose second end becomes
 * (lo32(z) * n[r]) >> 32 when hi32(z) < floor(p * 2^32) (as 64-bit values,
 * so p = 1 rewires every edge).  Self-loops are dropped and repeated pairs
 * collapse; the target edges and the output are as cb_graph_generate_er.
 *   k          even, 2 <= k < n[r] for every r.  p: 0 <= p <= 1.
 *   other arguments as cb_graph_generate_er; need n[r] k/2 + n_tedges < 2^31.
 */
int cb_graph_generate_ws(uint32_t n_inst, const uint32_t *n, uint32_t k, double p, uint64_t seed,
                         uint32_t n_tedges, const uint32_t *tedges, void *stream, cb_graph **out);

/*
 * cb_graph_generate_ba -- N Barabasi-Albert scale-free backgrounds with one
 * embedded target, generated on the device into a new handle (the paper's
 * scale-free backgrounds, single-background scenario).  Model: preferential
 * attachment by the endpoint list of Batagelj & Brandes (Phys. Rev. E 71,
 * 036113, 2005).  Nodes 0..m-1 are seeds; new node m + T (T = 0 .. n-m-1)
 * adds m edges, edge t = T m + q.  The first new node links to the m seeds.
 * Edge t of a later node links to the endpoint at position
 * pos = (lo32(z_t) * 2 m T) >> 32 of the list of all earlier new nodes' edge
 * endpoints (position 2e holds edge e's new node m + e/m, position 2e + 1
 * its target), z_t the counter generator's output for c = r * 2^32 + t: a
 * degree-proportional pick.  An odd position is resolved through the
 * earlier edge e = pos >> 1 in the same way.  Repeated pairs collapse (a
 * node that draws one target twice keeps one edge); the target edges and
 * the output are as cb_graph_generate_er.
 *   m          m >= 1 and n[r] > m for every r.
 *   other arguments as cb_graph_generate_er; need m (n[r] - m) + n_tedges < 2^31.
 */
int cb_graph_generate_ba(uint32_t n_inst, const uint32_t *n, uint32_t m, uint64_t seed,
                         uint32_t n_tedges, const uint32_t *tedges, void *stream, cb_graph **out);

/* Number of CSR entries (2 x undirected edges) of realisation r; 0 when r is
 * out of range or h is null. */
uint64_t cb_graph_num_entries(const cb_graph *h, uint32_t r);

/*
 * cb_graph_read -- copy realisation r's CSR pattern out of the handle (for
 * inspection, e.g. of a generated ensemble).
 *   row_ptr    uint32[n[r] + 1], host or device (any pointer CUDA can copy to).
 *   col        uint32[cb_graph_num_entries(h, r)], host or device.
 *   stream     the copies are queued on it; the call synchronises it.
 * Errors: CB_ERR_ARG (null handle or array, r out of range), CB_ERR_CUDA.
 */
int cb_graph_read(const cb_graph *h, uint32_t r, uint32_t *row_ptr, uint32_t *col, void *stream);

/*
 * cb_subgraph_centrality -- Estrada's sub-graph centrality SC(i) = (e^A)_ii
 * (eq. 3) for k nodes of realisation inst, by Gauss quadrature: m Lanczos
 * steps started at e_i give the m-point Gauss rule e1^T exp(T_m) e1 for
 * e_i^T e^A e_i (Golub & Meurant, "Matrices, Moments and Quadrature with
 * Applications", 2010).  For exp the rule is a lower bound that increases
 * with m; it is exact once the Krylov space from e_i is invariant.  The
 * paper calls SC expensive at scale; per node it costs one m-step Lanczos
 * run over the whole realisation, and the k runs go together.
 *   h, inst    handle and realisation index (< N).
 *   m          Krylov depth, 1 <= m <= CB_MAX_M.
 *   prec       CB_FP32 or CB_FP64 (vectors; scalars and the quadrature FP64).
 *   k          number of nodes, 1 <= k <= CB_MAX_SC_NODES.
 *   nodes      uint32[k] node indices (< n[inst]), host or device.
 *   sc_scaled  device double[k], written: SC(nodes[q]) = exp(*log_scale) * sc_scaled[q].
 *   log_scale  device double[1], written: max over q of lambda_max(T_m) from e_q.
 * The call builds a temporary handle with k copies of the realisation
 * (k * (nnz + n) * 4 bytes plus their formats and a (m+1) * k * n basis),
 * synchronises `stream` and frees it before returning.
 * Errors: CB_ERR_ARG (null arguments, ranges), CB_ERR_CUDA.
 */
int cb_subgraph_centrality(cb_graph *h, uint32_t inst, uint32_t m, int prec, uint32_t k,
                           const uint32_t *nodes, double *sc_scaled, double *log_scale,
                           void *stream);

/*
 * cb_graph_tune -- pick, by measurement, the SpMV configuration of this
 * handle at precision `prec`: the group width of the tiled-CSR SpMV (rows of
 * up to 8 * lanes entries share `lanes` lanes of a warp; longer rows go to a
 * warp, a CTA, or several CTAs) and, in FP32, the path -- the specialised
 * formats built at upload (column-blocked kernel for n <= 32 * 16384,
 * two-phase kernels above) or the tiled-CSR kernel for every realisation.
 * Candidates: the six widths 1, 2, 4, 8, 16, 32 on the tiled-CSR path, then
 * (FP32, when the handle has a blocked or two-phase format) the format path,
 * then (when every realisation has n <= 8192 and <= 2^20 entries) the
 * automatic path, which runs all steps of such a handle in one launch.
 * Each is timed on a 3-step Lanczos run over all realisations (CUDA events,
 * two repetitions after a warm-up, on a workspace of its own); the fastest
 * is kept (cb_graph_set_lanes / cb_graph_set_path).  FP64 always runs the
 * tiled-CSR kernel (or the single launch of a small handle), so only the
 * width, and for a small handle the single launch, is tuned there.  Results do not depend
 * on the choice beyond FP summation order.  Synchronises `stream`.
 *   lanes_out  optional host uint32[1]: the width kept.
 *   ms_out     optional host double[8]: ms per run for each width, then for
 *              the format path, then for the single launch (-1 when not
 *              timed).
 *   The path kept is read back with cb_graph_path.
 */
int cb_graph_tune(cb_graph *h, int prec, uint32_t *lanes_out, double *ms_out, void *stream);

/* Set / read the FP32 SpMV path (CB_PATH_AUTO, CB_PATH_FORMATS, CB_PATH_CSR),
 * e.g. from a cached tuning result.  A path whose format was not built
 * (CB_CSR_ONLY, or no realisation in its size range) falls back to the
 * tiled-CSR kernel.  Setting drops the handle's captured passes. */
int cb_graph_set_path(cb_graph *h, int path);
int cb_graph_path(const cb_graph *h);

/* Set / read the tiled-CSR group width (1, 2, 4, 8, 16 or 32), e.g. from a
 * cached tuning result.  Setting drops the handle's captured passes. */
int cb_graph_set_lanes(cb_graph *h, uint32_t lanes);
uint32_t cb_graph_lanes(const cb_graph *h);

/* Release a handle and its device memory (synchronises the device).  The
 * memory goes back to the library's per-device pool (see below), not to the
 * driver. */
int cb_graph_free(cb_graph *h);

/*
 * cb_release_cached_memory -- hand the device memory that the library's
 * pools keep for reuse back to the driver.  Handles, their workspaces and the
 * adjoint buffers are allocated from a stream-ordered pool per device that
 * keeps freed memory, because a cudaFree of multi-GB arrays costs about a
 * millisecond per GB and a following upload reuses the memory at no cost.
 * Memory held by live handles is not affected.  Synchronises the current
 * device.  With the environment variable CB_NO_POOL set (read once, at the
 * first allocation) the library uses cudaMalloc / cudaFree and this call
 * does nothing.  The paper has no counterpart; this is a library service.
 */
int cb_release_cached_memory(void);

/*
 * cb_set_memory_limit -- cap the device memory the library holds in live
 * allocations (handles, workspaces, adjoint and restart buffers; not the
 * top-k scratch).  An allocation that would exceed the cap fails with
 * CB_ERR_OOM as if the device were full, and the call that made it frees
 * what it had taken.  0 (the default) means no cap.  Process-wide.
 * cb_memory_in_use returns the bytes currently held.
 */
int cb_set_memory_limit(size_t bytes);
size_t cb_memory_in_use(void);

/*
 * cb_debug_stall_tile -- test hook for the bounded waits.  The column-
 * blocked SpMV (FP32) stages column blocks of the Krylov vector into shared
 * memory with bulk copies and waits for each on an mbarrier, for at most
 * 1 s of global time.  After this call, tile `btile` (0 <= btile <
 * number of column-blocked tiles, in realisation order) expects its first
 * column block but never copies it: its wait runs out, the step of that
 * realisation records CB_ERR_TIMEOUT (its scores become NaN, a report names
 * it and the call returns CB_ERR_TIMEOUT) and the other realisations are
 * unaffected.  No copy is left in flight and the context stays usable.
 * UINT32_MAX switches the hook off.  Drops the handle's captured passes.
 */
int cb_debug_stall_tile(cb_graph *h, uint32_t btile);

/* Number of realisations / node count of realisation r / largest n. */
uint32_t cb_graph_num_instances(const cb_graph *h);
uint32_t cb_graph_num_nodes(const cb_graph *h, uint32_t r);
uint32_t cb_graph_max_nodes(const cb_graph *h);

/*
 * cb_communicability -- total communicability of one realisation,
 * EBTC = e^A 1 (eq. 4), by the m-step Lanczos approximation
 *   e^A 1 ~= beta0 V_m exp(T_m) e1,  beta0 = sqrt(n),
 * returned as y_scaled[i] * exp(*log_scale), log_scale = lambda_max(T_m).
 *   h, inst    handle and realisation index (< N).
 *   m          Krylov depth, 1 <= m <= CB_MAX_M.  The recurrence stops
 *              early at an exact breakdown (invariant Krylov subspace).
 *   prec       CB_FP32 or CB_FP64.
 *   y_scaled   device, double[n[inst]], written.
 *   log_scale  device, double[1], written.
 *   rep        optional host cb_inst_report[1] (forces a synchronise).
 * This is the plain per-graph path: one realisation per call.
 */
int cb_communicability(cb_graph *h, uint32_t inst, uint32_t m, int prec, double *y_scaled,
                       double *log_scale, cb_inst_report *rep, void *stream);

/*
 * cb_ensemble_scores -- the summed score of eq. 5 over all N realisations
 * of the handle, all computed in one batched pass:
 *   EBTC(i) = sum_r EBTC_r(i) = exp(*log_scale) * S[i],
 *   log_scale = max_r theta_r, each term weighted by exp(theta_r - log_scale)
 *   and summed in realisation order in FP64.
 *   m, prec    as cb_communicability.
 *   n_out      length of S; n_out >= max_r n[r].  Entries >= max n are 0.
 *   S          device, double[n_out], written.
 *   log_scale  device, double[1], written.
 *   rep        optional host cb_inst_report[N] (forces a synchronise).
 * The second call with the same (m, prec, n_out, S, log_scale) on a handle
 * captures the pass into a CUDA graph (on a private stream; nothing runs
 * there) and later calls replay it on `stream`: one launch per call instead
 * of 2m + 5.  A handle keeps up to 8 such graphs; growing the workspace
 * (a larger m, another precision) retires them.  The environment variable
 * CB_NO_GRAPH (any value) forces direct launches; so do cb_profile_enable(1)
 * and a non-null rep.  Results are bit-identical either way.
 */
int cb_ensemble_scores(cb_graph *h, uint32_t m, int prec, uint32_t n_out, double *S,
                       double *log_scale, cb_inst_report *rep, void *stream);

/*
 * cb_ensemble_scores_restarted -- eq. 5, with every realisation's e^A 1
 * evaluated by the restarted Lanczos method of the paper's Krylov reference
 * ([10], Afanasjew, Eiermann, Ernst & Guettel 2008): `cycles` cycles of m
 * steps, each started from the last Lanczos vector of the one before, so
 * that the basis held on the device is m + 1 vectors for any total depth
 * cycles * m.  After k cycles the approximation is
 *   e^A 1 ~= beta0 [V_1 ... V_k] exp(H_k) e1,
 * H_k block lower bidiagonal: the cycles' tridiagonal matrices T_i on the
 * diagonal, the residual norm of cycle i coupling the first row of block
 * i + 1 to the last column of block i.  exp(H_k) e1 is evaluated block by
 * block with the contour rule of cb_communicability (partial fractions).
 *   m          1 <= m <= CB_MAX_M, the cycle length.
 *   cycles     1 <= cycles <= CB_MAX_CYCLES.  A realisation whose cycle
 *              breaks down (invariant Krylov subspace) stops there; its
 *              result is then exact.  cycles = 1 is cb_ensemble_scores.
 *   prec, n_out, S, log_scale   as cb_ensemble_scores; log_scale is the
 *              largest shift, each realisation's shift being the largest
 *              lambda_max(T_i) of its cycles.
 *   rep        optional host cb_inst_report[N]: m_eff = Lanczos steps over
 *              all cycles, beta_last = the last residual norm computed.
 * Accuracy: very short cycles (m <= 2) over many cycles amplify the contour
 * rule's error (H_k is far from normal); m >= 4 keeps FP64 results within
 * about 1e-12 of the exact block form.
 * Synchronous.  Temporary device memory: 8 bytes per node (padded) plus
 * 16 (cycles m + 14) bytes per realisation; the call overwrites the
 * handle's forward basis (cb_scores_backward recomputes it).
 */
int cb_ensemble_scores_restarted(cb_graph *h, uint32_t m, uint32_t cycles, int prec,
                                 uint32_t n_out, double *S, double *log_scale,
                                 cb_inst_report *rep, void *stream);

/*
 * cb_topk -- indices and values of the k largest entries of S (the
 * recovered target of the "Identification algorithm" section; the paper
 * sorts all scores, this selects by radix).
 *   S    device, double[n], read.
 *   n    1 <= n < 2^32.  k: 1 <= k <= min(n, CB_MAX_TOPK).
 *   idx  device, uint32[k], written; val device, double[k], written.
 * Order: value descending, ties to the smaller index; -0.0 equals +0.0;
 * NaN ranks below every number (so it is returned only if k exceeds the
 * count of non-NaN entries).
 * Asynchronous.  Device scratch (about 3 KB + 16 k bytes) comes from the
 * stream-ordered allocator (cudaMallocAsync) and is freed on `stream`.
 */
int cb_topk(const double *S, uint32_t n, uint32_t k, uint32_t *idx, double *val, void *stream);

/*
 * cb_topk_noalloc -- the same selection as cb_topk, without any device
 * allocation.  (The paper has no counterpart: this is a library service.)
 * For callers that cannot allocate device memory: an application that has
 * reserved the whole GPU for its own memory pool and rejects further
 * cudaMalloc / cudaMallocAsync calls, a plug-in whose host forbids CUDA
 * allocation, or a latency-critical loop where an allocation might stall.
 *   Arguments, order and tie rule as cb_topk.  k <= CB_MAX_TOPK (4096);
 *   a larger k is rejected with CB_ERR_ARG and a message naming the limit.
 *   Scratch: one fixed array of about 65 KB in device memory per GPU that
 *   loads the library, held until the process exits.  The first call in a
 *   CUDA context looks up that array's device address in the context
 *   (cudaGetSymbolAddress) and caches it under the context's unique id, so
 *   make the first call on each device before any stream capture.  A
 *   context created later (after cudaDeviceReset, or another context made
 *   current) gets its own lookup on its first call.
 *   Every call on a device shares the one array: calls whose work overlaps
 *   on the GPU (different streams, no ordering between them) race and may
 *   return wrong results.  Calls ordered on one stream are safe; each call
 *   resets the scratch state it needs before using it.
 *   Asynchronous; calls no allocating routine.
 */
int cb_topk_noalloc(const double *S, uint32_t n, uint32_t k, uint32_t *idx, double *val,
                    void *stream);

/*
 * Kernel timing for measurement tools.  While enabled, every launch of the
 * kernel families below is bracketed by a CUDA event pair recorded on the
 * stream it is launched on; cb_profile_read() synchronises those events and
 * returns the summed duration (ms) and the launch count of one family.
 * cb_profile_enable(1) also clears earlier records.  Off by default; not
 * thread-safe; it adds two event records per launch while on.
 */
#define CB_K_SPMV 0     /* Lanczos SpMV step (dominant kernel) */
#define CB_K_FINALIZE 1 /* Lanczos finalize (axpy + norm) */
#define CB_K_TRIDIAG 2  /* FP64 tridiagonal exp */
#define CB_K_COMBINE 3  /* basis combine / ensemble sum */
#define CB_K_TOPK 4     /* top-k selection (all its passes) */
#define CB_K_INIT 5     /* basis / scalar initialisation */
#define CB_K_BACKWARD 6 /* adjoint kernels (tridiagonal, node, edge) */
#define CB_K_COUNT 7
int cb_profile_enable(int on);
int cb_profile_read(int kernel, double *total_ms, uint64_t *launches);

/*
 * cb_scores_backward -- edge gradient of the summed top-k score.  This is an
 * extension: the paper has no gradient.  It differentiates eq. 5 restricted
 * to a fixed node set S (normally the recovered top-k):
 *   L = sum_r sum_{i in S, i < n_r} EBTC_r(i) = sum_r w_r^T e^{A_r} 1,
 *   dL/da_ij = G_ij + G_ji,  G = int_0^1 e^{sA} w 1^T e^{(1-s)A} ds,
 * for the undirected weight a_ij = a_ji of every existing edge (the
 * Frechet derivative of e^A, at unit weights).  It is evaluated in m-step
 * Krylov form from two Lanczos bases (from w and from 1).
 *   h, m, prec  handle, Krylov depth 1 <= m <= 64, CB_FP32 or CB_FP64.
 *   topk_idx    device, uint32[k], DISTINCT node indices of S (1 <= k <=
 *               CB_MAX_TOPK).  Realisation r uses those < n_r; a realisation
 *               without any contributes 0.
 *   grad        device, float[sum_r nnz_r], written in CSR entry order of the
 *               realisations concatenated in handle order.  The entries
 *               (i,j) and (j,i) of one edge get the same value.
 *   log_scale   device, double[1], written:
 *               dL/da_e = exp(*log_scale) * grad[e].
 * Asynchronous.  It overwrites the handle's forward workspace, so it must
 * not run concurrently with other calls on the same handle.  The device
 * memory it uses grows by one more Krylov basis and two node-major
 * n x m arrays.
 */
int cb_scores_backward(cb_graph *h, uint32_t m, int prec, const uint32_t *topk_idx, uint32_t k,
                       float *grad, double *log_scale, void *stream);

/*
 * cb_scores_backward_budget -- cb_scores_backward under a device-memory
 * budget.  The adjoint keeps, per realisation, two Krylov bases and the
 * node-major P and U: about esz * n * (2 (m + 1) + 2 * roundup4(m)) bytes,
 * esz = 4 (FP32) or 8 (FP64).  When the sum over realisations (plus ~12
 * bytes per CSR entry) exceeds mem_budget bytes, consecutive realisations
 * are processed in groups that fit (a single realisation always runs): each
 * group is copied device-to-device into a temporary handle, its basis from 1
 * is recomputed there (the forward pass's basis is not reused), and every
 * group's gradient is rescaled to the common shift max_r theta_r.  The
 * result equals cb_scores_backward's up to FP32 rounding of that rescaling.
 * Arguments as cb_scores_backward; synchronises `stream`.
 */
int cb_scores_backward_budget(cb_graph *h, uint32_t m, int prec, const uint32_t *topk_idx,
                              uint32_t k, float *grad, double *log_scale, size_t mem_budget,
                              void *stream);

/*
 * cb_score_sum -- the summed score of a node set, eq. 5 restricted to it:
 *   *loss = sum_{q < k, nodes[q] < n} S[nodes[q]]   (FP64, in q order).
 * With S from cb_ensemble_scores this is the loss that cb_scores_backward
 * differentiates, in units of exp(log_scale) of that call.
 *   S      device, double[n], read.   nodes: device, uint32[k], read;
 *          entries >= n are skipped, a repeated index counts once per entry.
 *   k      1 <= k <= CB_MAX_TOPK.     loss: device, double[1], written.
 * Asynchronous; deterministic (one warp, fixed summation order).
 */
int cb_score_sum(const double *S, uint32_t n, const uint32_t *nodes, uint32_t k, double *loss,
                 void *stream);

/*
 * cb_grad_rescale -- brings a gradient from cb_scores_backward to the units
 * of another log scale and applies an upstream factor (the vector-Jacobian
 * product of an autograd backward):
 *   grad[e] *= exp(*log_scale_grad - *log_scale_ref) * (grad_out ? *grad_out : 1)
 * for e < count.  The factor is formed once in FP64, applied in FP32.
 *   grad            device, float[count], read and written.
 *   log_scale_grad  device, double[1]: the log scale cb_scores_backward wrote.
 *   log_scale_ref   device, double[1]: the target units (for example the
 *                   log scale of the cb_ensemble_scores call whose summed
 *                   scores formed the loss).
 *   grad_out        device, double[1], or NULL for 1.
 * Asynchronous.  The paper has no gradient; this serves the adjoint.
 */
int cb_grad_rescale(float *grad, uint64_t count, const double *log_scale_grad,
                    const double *log_scale_ref, const double *grad_out, void *stream);

/*
 * Bounds-checked debug build.  A library compiled with -DCB_DEBUG
 * (libcb_debug.so, built beside libcb.so) checks, on the device, every
 * column-blocked stream element (its row-sum offset names one of the warp's
 * rows or the executing lane's spare sum) and stream write position (inside
 * the warp's stream), every CSR column the SpMV kernels gather through
 * (< n), the two-phase kernels' source offsets (< the tile's nodes), group
 * places (< the value array), region slots (< the bin's region or the zero
 * slot) and piece numbers (< the bin's pieces), and the adjoint's edge
 * columns (< n).  A failed check counts a
 * violation, records the first one as (site << 48) | index (sites 1-7 in the
 * order above: blocked element, blocked fill, CSR column, two-phase source,
 * two-phase place, two-phase slot, adjoint column) and skips the access;
 * nothing traps.
 * cb_debug_build: 1 in the debug build, 0 in the release build.
 * cb_debug_violations: the count since the last reset and the first record
 *   (host outputs; both 0 in the release build); reset != 0 clears them.
 *   The debug build synchronizes the device first; the release build
 *   touches no device.  Library service; no counterpart in
 *   the paper.
 */
uint32_t cb_debug_build(void);
int cb_debug_violations(uint32_t *count, uint64_t *first, int reset);

/* Message describing the last error on this host thread ("" if none). */
const char *cb_last_error(void);

/* Library ABI version (major << 16 | minor). */
uint32_t cb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CB_H_ */
