/*
 * contour.h -- C ABI of libcontour.so, a GB300 (sm_103a) connected-components
 * library built around the minimum-mapping operator of the Contour algorithm
 * (Du, Alvarado Rodriguez, Li, Dindoost, Bader: "Contour Algorithm for
 * Connectivity", arXiv 2311.02811).
 *
 * Problem (Section II-A): an undirected graph with vertex ids 0..n-1 and m
 * edges <w, v>.  Every entry point that returns labels returns, for each
 * vertex v, the smallest vertex id of v's connected component.  That value is
 * the unique fixed point reached by Alg. 1 and by its asynchronous variant
 * (Section III-B1): labels only ever decrease to values taken from the same
 * component, and a state in which no edge can lower a label consists of stars
 * whose roots are component minima (Section II-A).
 *
 * Conventions shared by every call:
 *   - No call throws; each returns a cc_status.  cc_last_error() gives a
 *     human-readable detail string for the calling host thread.
 *   - "Device" pointers are CUDA device (or managed) pointers of the current
 *     device; "host" pointers may be pageable or pinned.
 *   - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as
 *     void*; NULL means the legacy default stream).  Calls that return labels
 *     to the host, or that report a status computed on the device, synchronise
 *     that stream before returning.
 *   - A cc_graph handle may be used by one host thread at a time.
 *   - id_bits selects the vertex-id type: CC_ID32 (int32_t, n < 2^31) or
 *     CC_ID64 (int64_t).  Edge counts and offsets are always int64_t.
 */
#ifndef CONTOUR_H
#define CONTOUR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cc_graph cc_graph; /* opaque; owned by the library */

typedef enum {
    CC_OK = 0,
    CC_EINVAL = 1,        /* bad argument (NULL pointer, n < 0, bad enum, bad snapshot) */
    CC_EIDRANGE = 2,      /* an edge endpoint lies outside [0, n) */
    CC_ENOMEM = 3,        /* device or pinned-host allocation failed */
    CC_ECUDA = 4,         /* a CUDA runtime call failed (detail in cc_last_error) */
    CC_ENOTCONVERGED = 5, /* max_sweeps reached; labels are a valid partial state */
    CC_ETIMEOUT = 6       /* a bounded device-side wait gave up (batched launch) */
} cc_status;

enum { CC_ID32 = 32, CC_ID64 = 64 };
enum { CC_COO = 0, CC_CSR = 1, CC_CSR_NATIVE = 2, CC_CSR_NATIVE_SYM = 3 };
/* CC_ASYNC_COMPACT: asynchronous full-chain sweeps (order CC_ORDER_FULL only,
 * check interval 1) that drop every edge whose two chain walks ended at the
 * same root and pass the others to the next sweep, so later sweeps read only
 * the edges that still merge trees.  Dropping is a heuristic (an asynchronous
 * write that read a stale chain can still move a vertex to another tree), so
 * convergence is decided as for CC_ASYNC (Section III-B2) over every edge:
 * once a compacting sweep sees no violation, the next sweeps are ordinary
 * full-chain sweeps over all edges until one sees none.  Labels are those of
 * CC_ASYNC.  int32 edge lists only (no native CSR, no hub layout); the handle
 * allocates two more edge lists of its size on first use.  No counterpart in
 * the paper. */
enum { CC_SYNC = 0, CC_ASYNC = 1, CC_ASYNC_COMPACT = 2 };
/* Operator order: h >= 1 is MM^h of Def. 3; CC_ORDER_FULL follows each label
 * chain to its root (at most 1024 hops, the "C-m" variant with m = 1024 of
 * Section III-B4); CC_ORDER_AUTO lets the learned scheduler choose. */
enum { CC_ORDER_FULL = 0, CC_ORDER_AUTO = -1 };
/* Per-iteration order schedules (Section III-B4), cc_run only, check interval 1:
 * CC_ORDER_11MM ("C-11mm") uses order 1 for the first two sweeps and the full
 * chain afterwards; CC_ORDER_1M1M ("C-1m1m") alternates order 1 and the full
 * chain, starting with order 1. */
enum { CC_ORDER_11MM = -2, CC_ORDER_1M1M = -3 };
enum { CC_MAX_ORDER = 1024 };

typedef struct {
    int32_t sweeps;         /* edge sweeps executed (whole check blocks)            */
    int32_t order;          /* operator order used (CC_ORDER_FULL for full chain)   */
    int32_t mode;           /* CC_SYNC or CC_ASYNC                                  */
    int32_t check_interval; /* sweeps per convergence check                         */
    double solve_ms;        /* device time from label init to final compress        */
    double edges_per_s;     /* m / solve time                                       */
    double alg_bytes;       /* algorithmic bytes moved by all sweeps (see below)    */
    double loop_ms;         /* device time of the sweep loop alone: every sweep, the */
                            /* L = L_u copies and the one-thread check per block    */
} cc_stats;

/*
 * cc_init -- build a graph handle.
 *
 * Section II-A: vertex ids are 0..n-1; the graph is given either as
 *   layout == CC_COO: a = src[m], b = dst[m], m = m_or_nnz undirected edges
 *                     <src[e], dst[e]> (self-loops and repeats allowed), or
 *   layout == CC_CSR: a = int64_t offsets[n+1], b = cols[nnz], nnz = m_or_nnz;
 *                     every stored entry (r, cols[k]) becomes one edge.  A
 *                     symmetric CSR therefore yields every edge twice.  The
 *                     rows are expanded on the device into an edge list.
 *   layout == CC_CSR_NATIVE: the same input, kept as CSR: each sweep walks the
 *                     rows directly (no per-entry row array is built; the
 *                     handle adds one int32 row index per 4 entries).  Every
 *                     entry (r, cols[k]) is one edge <r, cols[k]>.
 *   layout == CC_CSR_NATIVE_SYM: a symmetric CSR (each undirected edge stored
 *                     in both rows) kept as CSR; a sweep applies the operator
 *                     only to the entries with cols[k] < r, i.e. once per
 *                     undirected edge.  Self-loops are dropped (they never
 *                     change a label).  The input is not checked for
 *                     symmetry: an edge stored only as (r, c) with c > r is
 *                     never applied.
 *   The native CSR layouts take int32 ids only (CC_EINVAL otherwise), do not
 *   support cc_graph_reorder (CC_EINVAL), and count m = nnz stored entries
 *   in cc_graph_info and cc_stats.edges_per_s.
 * Ids have the type chosen by id_bits.
 *
 * on_device == 0: a and b are host arrays; they are copied to the device and
 *                 may be freed after the call returns.
 * on_device == 1: a and b are device arrays.  A COO pair whose pointers are
 *                 16-byte aligned is borrowed (no copy) and must stay alive
 *                 and unchanged until cc_free; otherwise it is copied.  For
 *                 the native CSR layouts the offsets (8-byte aligned) and the
 *                 columns (16-byte aligned) are borrowed under the same rule.
 *
 * Every id is checked on the device: CC_EIDRANGE if any endpoint lies
 * outside [0, n) (CSR: also CC_EINVAL for offsets that are not a
 * non-decreasing sequence from 0 to nnz).  n == 0 and m == 0 are valid.
 * On success *g owns its device buffers until cc_free(*g).
 */
cc_status cc_init(cc_graph **g, int64_t n, int id_bits, int layout, const void *a,
                  const void *b, int64_t m_or_nnz, int on_device, void *cuda_stream);

/*
 * cc_run -- label every vertex with the smallest id of its component.
 *
 * Runs the Contour iteration of Alg. 1 on the device: labels L[i] = i
 * (Alg. 1 initialisation) or a resume snapshot, then repeated sweeps in
 * which every edge <w, v> applies the order-h minimum-mapping operator of
 * Def. 3: z = min(L^h[w], L^h[v]) and every chain entry L[w], L[L[w]], ...,
 * L[L^{h-1}[w]] (and the same for v) that is larger than z is set to z
 * (conditional assignment, Def. 1).
 *
 *   order           h >= 1, CC_ORDER_FULL, or CC_ORDER_AUTO (learned scheduler;
 *                   the plain order-2 synchronous schedule when no weights are
 *                   loaded).  h is at most CC_MAX_ORDER.
 *   mode            CC_SYNC: Alg. 1 literally -- reads from L, atomic-min
 *                   writes into the update array L_u (Eq. "cas"), then L = L_u;
 *                   every sweep is deterministic.  CC_ASYNC: in-place plain
 *                   stores into L (Section III-B1 and III-B3).
 *                   CC_ASYNC_COMPACT: CC_ASYNC with edge compaction (above).
 *   check_interval  c >= 1: the convergence flag of Section III-B2 is taken
 *                   from the last sweep of every block of c sweeps; the run
 *                   stops after the first block whose last sweep saw no edge
 *                   whose chain could lower a label.  With CC_ORDER_AUTO a
 *                   value of 0 lets the scheduler choose c as well.
 *   max_sweeps      >= 1; the run stops after this many sweeps (rounded up to
 *                   whole blocks) and returns CC_ENOTCONVERGED, leaving a
 *                   valid partial state in labels_out that a later call can
 *                   resume from.
 *   init_labels     NULL, or n ids to start from (a snapshot of an earlier
 *                   run).  Each entry must satisfy 0 <= init[x] <= x, else
 *                   CC_EINVAL.  Same memory space as labels_out.
 *   labels_out      n ids (id_bits wide), caller-allocated; device memory when
 *                   out_on_device != 0, else host memory.
 *   stats           NULL or filled on return (also on CC_ENOTCONVERGED).
 *
 * After a converged loop a compress pass sets L[x] to the root of its chain
 * and counts the labels it moves: the result is a set of stars (Section II-A)
 * and at a true fixed point nothing moves (a moved label is reported as
 * CC_ECUDA, an internal error).  A run that stops at max_sweeps is returned
 * exactly as its last sweep left it.  Work is enqueued on the handle's stream (cc_init's stream, or the
 * one set by cc_graph_set_stream), which cc_run synchronises before returning.
 *
 * Algorithmic bytes per sweep (stats.alg_bytes): async 2*B*m + B*n, sync adds
 * 3*B*n (L_u writes and the L = L_u copy), B = id_bits / 8.
 */
cc_status cc_run(cc_graph *g, int order, int mode, int check_interval, int32_t max_sweeps,
                 const void *init_labels, void *labels_out, int out_on_device, cc_stats *stats);

/*
 * cc_solve_host -- one solve of an edge list held in HOST memory: cc_init,
 * cc_run and cc_free in one call, with the upload overlapped with sweeps.
 *
 * The edges cross the host link in chunks of 2^24 edges on a copy stream of
 * their own.  Each chunk is checked (ids in [0, n)) as soon as it has landed,
 * stored as (smaller id, larger id) and, on graphs of average degree 8 or more
 * (m >= 4n), sorted by the smaller id into its place in the edge arrays (the
 * operator is symmetric in w and v, and edge order never changes the result);
 * the chunks after the bulk halve in size, so little is left to do once the
 * last copy lands.  In CC_ASYNC mode the order-h operator
 * of Def. 3 is applied once to each of its edges, in place, while the later
 * chunks are still in flight: in the asynchronous iteration (Section III-B1)
 * an edge may be applied at any time, so sweeping the landed part early is one
 * more legal order of applications.  That streamed pass counts as the first
 * sweep.  Once the whole list is
 * resident the solve continues exactly as cc_run on a handle of the same
 * edges, from the streamed labels: checked sweeps (Section III-B2) to the
 * fixed point, then the compress.  CC_SYNC solves with check_interval 1
 * stream Alg. 1's first iteration instead, which reads no label (each edge
 * lowers L_u[max(w, v)] to min(w, v), and these minima commute), and the loop
 * continues from its result; with a larger interval the chunks are only
 * checked.  Either way every synchronous state and sweep count equals
 * cc_run's.  Labels equal cc_run's in both modes (the unique result of the
 * fixed point).
 *
 *   n, src, dst, m  int32 COO edges in host memory (pinned memory lets the
 *                   copies run asynchronously and overlap; pageable memory
 *                   works, without overlap).  Read only; not kept.
 *   order           h >= 1 or CC_ORDER_FULL (no CC_ORDER_AUTO or schedules).
 *   mode            CC_SYNC or CC_ASYNC.
 *   check_interval, max_sweeps, labels_out, out_on_device  as for cc_run
 *                   (CC_ASYNC: max_sweeps >= 2, the streamed pass included).
 *   stats           as for cc_run; solve_ms covers the whole call on the
 *                   device from the first copy to the compress, and sweeps
 *                   and alg_bytes include the streamed pass or iteration.
 *   cuda_stream     the stream the sweeps run on (synchronised before
 *                   returning); the copies use a stream of their own.
 * Errors: CC_EIDRANGE if an id lies outside [0, n) (such an edge is never
 * used by a gather), otherwise as for cc_init and cc_run.  Device memory
 * (the edge arrays, two staging pairs of 2^24 edges and the sort's scratch
 * on dense graphs, the labels) comes from the library's stream-ordered pool
 * and is handed back to it, in stream order, before the call returns.
 */
cc_status cc_solve_host(int64_t n, const int32_t *src, const int32_t *dst, int64_t m, int order, int mode,
                        int check_interval, int32_t max_sweeps, void *labels_out, int out_on_device,
                        cc_stats *stats, void *cuda_stream);

/*
 * cc_run_noalloc -- the same computation as cc_run, for callers that cannot
 * allocate device memory.  The paper has no counterpart to this entry point.
 *
 * Who needs it: code whose device memory belongs to someone else -- a plugin
 * or serving loop inside a framework that owns a pre-reserved memory pool and
 * forbids cudaMalloc during a step, or a latency-critical loop that cannot
 * afford cudaMalloc/cudaFree, which may synchronise the whole device.  Such a
 * caller passes only its own inputs and outputs; no handle is created.
 *
 * Memory: the control words and, for CC_SYNC, the update array L_u live in
 * one fixed device array inside libcontour.so (4 * CC_NOALLOC_MAX_N bytes plus
 * 256), held by every GPU that loads it until the process exits.  No call to
 * cudaMalloc, cudaFree, graph instantiation or any other allocating routine is
 * made; the convergence flag is read back by the host after every check block.
 *
 *   n, src, dst, m  int32 COO edges on the device (ids in [0, n), checked:
 *                   CC_EIDRANGE); src, dst and labels_out must be 16-byte
 *                   aligned memory of the current device (device or managed
 *                   allocations; host memory gives CC_EINVAL before any
 *                   launch) and are never copied.
 *   order, mode, check_interval, max_sweeps  as for cc_run (no CC_ORDER_AUTO).
 *   labels_out      n int32 device labels; also the working label array.
 *   sweeps_out      NULL or the number of sweeps executed.
 *   cuda_stream     stream to run on; synchronised before returning.
 *
 * Limits: CC_SYNC requires n <= CC_NOALLOC_MAX_N (CC_EINVAL beyond it, before
 * any device work); CC_ASYNC needs no L_u and accepts any n < 2^31.
 * Every call looks up the array's address on the current device
 * (cudaGetSymbolAddress, which allocates nothing); the first call on a device
 * also loads the library's device code there, so make that first call before
 * any stream capture.
 * Every call in the process shares the one array and clears the words it
 * needs at the start: calls that may overlap on the GPU (different streams or
 * threads) race and must be serialised by the caller.
 */
enum { CC_NOALLOC_MAX_N = 4194304 };
cc_status cc_run_noalloc(int64_t n, const int32_t *src, const int32_t *dst, int64_t m, int order,
                         int mode, int check_interval, int32_t max_sweeps, int32_t *labels_out,
                         int32_t *sweeps_out, void *cuda_stream);

/*
 * Batched solve: many independent graphs in one CUDA-graph launch.
 *
 * The graphs are concatenated: graph g owns vertices [vtx_off[g], vtx_off[g+1])
 * and edges [edge_off[g], edge_off[g+1]) of src/dst, and its edge ids are
 * LOCAL (0 .. n_g-1).  Each graph runs its own Contour iteration -- Alg. 1 or
 * the asynchronous variant of Section III-B, with its own convergence flag
 * (Section III-B2) and sweep count -- so every label is the smallest LOCAL id
 * of the vertex's component within its own graph.
 *
 * Small graphs (labels fit the shared-memory budget) are solved whole by one
 * CTA each with their labels in shared memory; large graphs advance one sweep
 * per round, all active large graphs together, until each has converged.  An
 * autotuner chooses the shared-memory budget, CTA size and edges per thread
 * of the small-graph kernel by timing candidates on the batch itself and
 * caches the choice per size histogram.
 *
 * cc_batch_init   vtx_off, edge_off: HOST int64 arrays of n_graphs+1 entries
 *                 (non-decreasing, starting at 0); src, dst: DEVICE int32
 *                 arrays of edge_off[n_graphs] local ids, borrowed (must stay
 *                 alive and unchanged until cc_batch_free).  Every id is
 *                 checked on the device (CC_EIDRANGE).  autotune: 0 = defaults,
 *                 1 = tune (or reuse a cached tuning), 2 = always re-tune.
 * cc_batch_run    one schedule for every graph (order, mode, check_interval as
 *                 for cc_run), or order == CC_ORDER_AUTO for a per-graph
 *                 schedule chosen by the learned scheduler (the plain order-2
 *                 synchronous schedule without loaded weights; with AUTO and
 *                 check_interval 0 every graph is checked after every sweep,
 *                 since a batch shares its convergence checks).  labels_out:
 *                 DEVICE int32[vtx_off[n_graphs]]; sweeps_out: HOST int32
 *                 [n_graphs] or NULL; solve_ms: NULL or the device time.
 *                 CC_ENOTCONVERGED if a graph reached max_sweeps.
 *                 Synchronises the plan's stream.
 * cc_batch_set_schedule / cc_batch_run_scheduled   an explicit per-graph
 *                 schedule (HOST arrays of n_graphs entries).
 * cc_batch        one-shot init + run + free (no autotuning; sweeps_out HOST).
 */
typedef struct cc_batch_plan cc_batch_plan;

cc_status cc_batch_init(cc_batch_plan **b, int32_t n_graphs, const int64_t *vtx_off,
                        const int64_t *edge_off, const int32_t *src, const int32_t *dst, int autotune,
                        void *cuda_stream);
cc_status cc_batch_run(cc_batch_plan *b, int order, int mode, int check_interval, int32_t max_sweeps,
                       int32_t *labels_out, int32_t *sweeps_out, double *solve_ms);
cc_status cc_batch_set_schedule(cc_batch_plan *b, const int32_t *order, const int32_t *mode,
                                const int32_t *check_interval);
cc_status cc_batch_run_scheduled(cc_batch_plan *b, int32_t max_sweeps, int32_t *labels_out,
                                 int32_t *sweeps_out, double *solve_ms);
cc_status cc_batch_tuning(const cc_batch_plan *b, int32_t *smem_budget, int32_t *threads,
                          int32_t *edges_per_thread);
/* Override the small-graph kernel's tuning: smem_budget bytes of shared
 * memory per CTA (graphs whose labels do not fit take the large-graph path;
 * 0 sends every non-empty graph there), threads in {256, 512, 1024}, edges
 * per thread 1..4. */
cc_status cc_batch_set_tuning(cc_batch_plan *b, int32_t smem_budget, int32_t threads,
                              int32_t edges_per_thread);
/* One-time layout step for a plan (see cc_graph_reorder): within every graph,
 * edges are oriented from their lower-degree endpoint and grouped by it.  Each
 * graph keeps its own edge range and its labels are unchanged.  The plan then
 * owns the reordered copy (the borrowed arrays are no longer referenced).
 * Batches of at most 2^32 - 1 vertices.  Synchronises the plan's stream. */
cc_status cc_batch_reorder(cc_batch_plan *b);
/* Device pointers of the plan's edge arrays (borrowed, or its own reordered
 * copy); valid until cc_batch_free or the next cc_batch_reorder. */
cc_status cc_batch_edges(const cc_batch_plan *b, const int32_t **src, const int32_t **dst);
void cc_batch_free(cc_batch_plan *b);
cc_status cc_batch(int32_t n_graphs, const int64_t *vtx_off, const int64_t *edge_off,
                   const int32_t *src, const int32_t *dst, int order, int mode, int check_interval,
                   int32_t *labels_out, int32_t *sweeps_out, void *cuda_stream);

/*
 * Learned schedule selection (CC_ORDER_AUTO).
 *
 * The paper chooses operators by hand from graph size and diameter (Section
 * IV-E: C-1 for small low-diameter graphs, C-m for large or long-diameter
 * ones, C-2 as the stable default).  Here a small MLP learns the choice from
 * measured solve times.  All schedules return identical labels.
 *
 * Features (CC_SCHED_FEATURES floats per graph, each log2(1 + x)): n, m, the
 * degree variance and maximum degree estimated on an edge sample (all edges
 * when m <= 16384, else the 16384 edges at positions floor(j*m/16384),
 * counts scaled by m/16384), and the eccentricities of 8 sources in the
 * sampled graph (the src endpoints of sample positions floor((2i+1)*S/16)),
 * by breadth-first search capped at 16 levels.
 * Model: 12 -> 64 -> 64 -> 64 -> CC_SCHED_CLASSES, ReLU, standardised inputs;
 * BF16 weights, FP32 biases and accumulation.  Class k decodes to
 * order {2, 4, CC_ORDER_FULL}[k/6], mode (k/3)%2 (0 sync, 1 async) and check
 * interval {1, 2, 4}[k%3].
 *
 * A handle computes its features and schedule once per loaded model (its
 * edges cannot change).  Its first CC_ORDER_AUTO call does not wait for them:
 * it enqueues the feature pass and the inference on a stream of the handle's
 * own (ordered after the work already on the handle's stream) and solves with
 * the paper's default C-2 (order 2, asynchronous, the caller's check
 * interval or 1); later calls use the predicted schedule.  A plan computes
 * the features of all its graphs on its first CC_ORDER_AUTO call, before the
 * solve.  Every schedule returns the same labels.
 *
 * cc_sched_load        install a weight blob (cc_sched_blob_bytes() bytes, format
 *                      "CCMLP01": header with feature mean/std, then per layer
 *                      BF16 weights [out][in] and FP32 biases); NULL unloads and
 *                      restores the plain order-2 synchronous fallback.  The model
 *                      is process-wide.
 * cc_sched_load_batch  install the weights that batched solves use (same format;
 *                      trained on the sweep counts graphs take inside a batch,
 *                      where a round lasts as long as its slowest graph); NULL
 *                      unloads them, and batches then use cc_sched_load's model.
 * cc_graph_features / cc_batch_features   features of a graph / every graph of
 *                      a plan (int32 ids), written to HOST memory.
 * cc_sched_predict     classes (and optionally CC_SCHED_CLASSES logits) for
 *                      count HOST feature rows; CC_EINVAL without weights.
 *                      cc_sched_predict_batch: the same with the batch model.
 * cc_sched_train       train the MLP on the GPU (mini-batch Adam, softmax cross-
 *                      entropy) on N HOST rows with labels in [0, 18); inputs are
 *                      standardised with their own mean/std; parameters start at
 *                      init_params (cc_sched_param_count() FP32 values, per layer
 *                      weights [out][in] then biases) or, if NULL, at a He-uniform
 *                      draw from SplitMix64(seed).  Writes a blob to blob_out.
 * cc_sched_train_step  one Adam step (t = 1, zero moments, lr) on B standardised
 *                      rows, updating params_inout in place; for testing.
 */
enum { CC_SCHED_FEATURES = 12, CC_SCHED_CLASSES = 18 };
cc_status cc_sched_load(const void *weights, size_t bytes);
cc_status cc_sched_load_batch(const void *weights, size_t bytes);
size_t cc_sched_blob_bytes(void);
int32_t cc_sched_param_count(void);
cc_status cc_sched_decode(int32_t cls, int *order, int *mode, int *check_interval);
cc_status cc_graph_features(cc_graph *g, float *features_out);
cc_status cc_batch_features(cc_batch_plan *b, float *features_out);
cc_status cc_sched_predict(const float *features, int32_t count, int32_t *cls_out, float *logits_out);
cc_status cc_sched_predict_batch(const float *features, int32_t count, int32_t *cls_out, float *logits_out);
cc_status cc_sched_train(const float *features, const int32_t *labels, int32_t N,
                         const float *init_params, int32_t epochs, int32_t batch, float lr,
                         uint64_t seed, void *blob_out, float *final_loss);
cc_status cc_sched_train_step(const float *features_norm, const int32_t *labels, int32_t B,
                              float *params_inout, float lr, float *loss_out);

/*
 * cc_graph_reorder -- one-time layout step: reorder the handle's edge list so
 * that consecutive edges share an endpoint.  The paper's edge loop (Alg. 1)
 * visits edges in any order, so every later cc_run returns the same labels;
 * sweeps become faster because the label gathers of one warp fall into few
 * cache lines.  The handle then owns a reordered copy (a borrowed input is no
 * longer referenced).  int32 ids only.  Synchronises the handle's stream.
 *   CC_REORDER_SRC     sort the (src, dst) pairs by src
 *   CC_REORDER_LOWDEG  orient each edge from its lower-degree endpoint (ties:
 *                      smaller id) and sort by that endpoint
 *   CC_REORDER_HUB     CC_REORDER_LOWDEG, then the vertices of highest degree
 *                      (at most 24,576, each of degree >= 16) become hubs
 *                      whose labels every sweep reads from a shared-memory
 *                      table: in the stored dst array, an entry d < 0 stands
 *                      for vertex hubs[~d] (cc_graph_hubs).  A graph without
 *                      such vertices keeps plain ids.  A hub-encoded handle
 *                      cannot be reordered again (CC_EINVAL).
 *   CC_REORDER_DEGREE  renumber the vertices in order of decreasing degree
 *                      (ties: smaller id first; vertex x becomes perm[x],
 *                      cc_graph_perm), store every edge from its larger new
 *                      id to its smaller and sort by the larger.  The labels
 *                      of the first new ids (at most 24,576, each of degree
 *                      >= 16) are read from a shared-memory copy.  The hot
 *                      labels of a skewed graph then share
 *                      few cache lines and stay in L2 even when the whole
 *                      label array does not.  Sweeps run Alg. 1 / Section
 *                      III-B on the renumbered graph; cc_run returns labels
 *                      in the caller's ids, each tree of the final state
 *                      labelled by its smallest caller id.  At convergence
 *                      that is exactly the result of every other layout; a
 *                      run stopped at max_sweeps returns a valid resume
 *                      snapshot (not Alg. 1's state of the same sweep in the
 *                      caller's ids), and init_labels are mapped in the same
 *                      way.  The handle then holds two more n-entry id maps
 *                      and two n-entry work arrays.  Renumbered handles take
 *                      neither CC_ASYNC_COMPACT nor another reorder
 *                      (CC_EINVAL).
 * CC_EINVAL for native CSR handles.
 */
enum { CC_REORDER_SRC = 1, CC_REORDER_LOWDEG = 2, CC_REORDER_HUB = 3, CC_REORDER_DEGREE = 4 };
cc_status cc_graph_reorder(cc_graph *g, int method);

/* The hub table of a CC_REORDER_HUB handle: *hubs (device, *k int32 ids) is
 * NULL and *k is 0 when the edges carry no hub entries.  For a
 * CC_REORDER_DEGREE handle *hubs is NULL and *k is the number of new ids read
 * from shared memory.  Valid until cc_free or the next cc_graph_reorder. */
cc_status cc_graph_hubs(const cc_graph *g, const int32_t **hubs, int32_t *k);

/* The id maps of a CC_REORDER_DEGREE handle (device, n int32 each): perm[x]
 * is the new id of vertex x, inv the inverse.  Both NULL for other handles.
 * Valid until cc_free. */
cc_status cc_graph_perm(const cc_graph *g, const int32_t **perm, const int32_t **inv);

/* How cc_run drives the sweep loop.  CC_LAUNCH_GRAPH (default): one CUDA
 * graph whose conditional WHILE node repeats the check blocks on the device,
 * with no host round trip.  CC_LAUNCH_HOST: the host enqueues one check block
 * at a time and reads the convergence flag after each; slower (a stream
 * synchronisation per block), but every kernel is an ordinary launch, for
 * profilers and debuggers that do not follow conditional graph nodes.  Both
 * give identical labels and sweep counts.  (The paper's loop is a host
 * do-while, Alg. 1; no counterpart for the graph form.) */
enum { CC_LAUNCH_GRAPH = 0, CC_LAUNCH_HOST = 1 };
cc_status cc_graph_set_launch(cc_graph *g, int launch);

/* Make later cc_run calls on g enqueue on another stream (default: the stream
 * passed to cc_init). */
cc_status cc_graph_set_stream(cc_graph *g, void *cuda_stream);

/* Number of vertices and stored edges of a handle (either may be NULL). */
cc_status cc_graph_info(const cc_graph *g, int64_t *n, int64_t *m);

/* Device pointers of the handle's edge arrays (the borrowed input, or the
 * handle's own copy after cc_init copied or cc_graph_reorder reordered it);
 * valid until cc_free or the next cc_graph_reorder.  For the native CSR
 * layouts *src receives the int64 offsets and *dst the columns; after
 * CC_REORDER_HUB the dst array holds hub entries ~s (see cc_graph_hubs), and
 * after CC_REORDER_DEGREE both arrays hold new ids (see cc_graph_perm). */
cc_status cc_graph_edges(const cc_graph *g, const void **src, const void **dst);

/* Release a handle and every device buffer it owns.  NULL is ignored.  The
 * release is enqueued on the handle's stream, which must still exist. */
void cc_free(cc_graph *g);

/* Device memory of graph handles comes from a per-device stream-ordered pool
 * that keeps released memory for the next handle (repeated cc_init / cc_free
 * cycles then cost no cudaMalloc/cudaFree).  This call waits for the device
 * and returns all unused pool memory to it. */
cc_status cc_release_memory(void);

/* Static description of a status code. */
const char *cc_strerror(cc_status s);

/* Detail message of the last failing call on this host thread ("" if none). */
const char *cc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CONTOUR_H */
