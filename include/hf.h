/*
 * hf.h -- C ABI of the GB300 Hilbert-forest library (libhf.so).
 *
 * The library implements the data-parallel path of the Hilbert forest
 * (Imamura et al., "Hilbert Forest in the SISAP 2025 Indexing Challenge",
 * arXiv 2508.21682): for each of T trees a seeded permutation and reflection
 * of the coordinate axes, b-bit quantization, the Hilbert key of every point,
 * a sort by that key, squared distances between points within w positions of
 * each other in the order, and a per-point top-k merge that yields an
 * approximate kNN graph; queries are located in the same orders by binary
 * search and answered from the windows around their positions.
 *
 * Conventions (the paper fixes none of these):
 *   - curve: Skilling's transposed Hilbert index (AIP Conf. Proc. 707, 2004);
 *     key bit l*d+i, counted from the most significant end, is bit (b-1-l) of
 *     the transformed coordinate i; keys are W = ceil(d*b/64) 64-bit words,
 *     word 0 most significant, zero-padded at the low end;
 *   - quantization: per-axis lo = min, hi = max of the data;
 *     scale = (float)(2^b / (double)(float)(hi - lo)) (0 for a flat axis);
 *     code = clamp(floor(fl32(fl32(x - lo) * scale)), 0, 2^b - 1);
 *   - tree t: splitmix64 from state seed + (t+1)*0x9E3779B97F4A7C15; a
 *     Fisher-Yates shuffle (j = d-1 .. 1, m = next() % (j+1)) gives pi, then
 *     r[j] = next() >> 63; permuted coordinate j is code[pi[j]], replaced by
 *     2^b - 1 - code when r[j] = 1;
 *   - order: ascending (full key, point index);
 *   - graph window: positions p +- delta, 1 <= delta <= w, clipped, no wrap;
 *   - search window: positions [p - w, p + w) around the query's lower-bound
 *     position p, clipped;
 *   - distance: squared Euclidean in float32 with exact coordinate
 *     differences; lists ascending by (distance, index); candidate sets are
 *     sets (a point appears once per list, never in its own list); unfilled
 *     slots are (index -1, distance +inf).
 *
 * Memory: every pointer argument may be device memory or host memory; the
 * library checks with cudaPointerGetAttributes. Host inputs are copied to the
 * device inside the call and host outputs are copied back before it returns,
 * on the given stream. Device inputs are read in place.
 *
 * Synchronisation: every call that takes a stream enqueues its work on that
 * stream (NULL = the legacy default stream), then synchronises the stream,
 * reads the library's device error word and returns a status. No call aborts
 * the process or traps on the device.
 *
 * Errors: HF_EINVAL for bad arguments (checked before any work), HF_ENOMEM
 * when a device allocation fails, HF_ECUDA for any other CUDA error,
 * HF_ENONFINITE when the data or a query holds NaN or +-inf, HF_ETIMEOUT when
 * a bounded inter-block wait inside the sort gave up, HF_ESTATE when a call
 * needs state the forest does not hold. On error, outputs are unspecified.
 */
#ifndef HF_H
#define HF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hf_forest hf_forest; /* opaque; owned by the library */

enum {
  HF_OK = 0,
  HF_EINVAL = -1,
  HF_ENOMEM = -2,
  HF_ECUDA = -3,
  HF_ENONFINITE = -4,
  HF_ETIMEOUT = -5,
  HF_ESTATE = -6,
  HF_ENOTIMPL = -7
};

/* Limits checked by every entry point. */
#define HF_MAX_D 4096
#define HF_MAX_BITS 8
#define HF_MAX_K 64
#define HF_MAX_K2 1024 /* sketch_k2 limit of the sketch-form search */
#define HF_MAX_N (((int64_t)1 << 30) - 1)
/* Widest window of the plain float32 graph form (hf_set_option mode=0). */
#define HF_PLAIN_MAX_W 704

/*
 * hf_build -- preprocessing and the per-tree orders.
 * Paper: Algorithm 2 (every sort shuffles the coordinate axes, then orders
 * all points along the curve); Algorithm 1 (the search's trees are built on
 * shuffled axis orders); Section 2 (Hilbert sort, and the Hilbert tree as the
 * sorted sequence that binary search runs on).
 *
 * points : n x d float32, row-major (point i at points + i*d). Borrowed when
 *          it is device memory: it is never written and must stay valid and
 *          unchanged until hf_free, because hf_knn_graph and hf_search read it.
 *          When it is host memory the forest keeps its own device copy.
 * n      : number of points, 2 <= n <= HF_MAX_N.
 * d      : dimension, 1 <= d <= HF_MAX_D.
 * T      : number of trees (sorts), T >= 1.
 * bits   : bits per coordinate for the key, 1 <= bits <= HF_MAX_BITS.
 * seed   : seed of the per-tree axis permutations and reflections.
 * stream : cudaStream_t (as void*), or NULL.
 * out    : receives the new forest; set to NULL on error.
 * The forest keeps, per tree, the order (sigma: position -> point) and the
 * sorted key prefixes, so that hf_search can run later.
 */
int hf_build(const float* points, int64_t n, int32_t d, int32_t T, int32_t bits,
             uint64_t seed, void* stream, hf_forest** out);

/*
 * hf_build_opts -- hf_build with build options, a comma-separated list of
 * key=value pairs (NULL or "" = defaults):
 *   prefix_words=K   64-bit key words sorted by radix (1..W, default min(2, W));
 *                    runs of equal prefixes are then ordered by the full key;
 *   sort_batch=B     at most B trees keyed and sorted together (default: as
 *                    many as fit in half of the free device memory, 16 GiB
 *                    at most); the result does not depend on B;
 *   spin_limit_us=U  bound of each inter-block wait in the sort (default 2e6);
 *   test_stall=1     test hook: one block of the first sort pass waits on a
 *                    status word that nothing writes, so the bounded wait runs
 *                    out and the call returns HF_ETIMEOUT.
 * Unknown keys give HF_EINVAL.
 */
int hf_build_opts(const float* points, int64_t n, int32_t d, int32_t T, int32_t bits,
                  uint64_t seed, const char* options, void* stream, hf_forest** out);

/*
 * hf_knn_graph -- approximate kNN graph (Algorithm 2; its second stage, the
 * sketch filter, runs in mode 3 only).
 * For every point, the candidates are the points within w positions of it in
 * any tree's order; the result is the k nearest candidates by float32 squared
 * distance, ascending by (distance, index). Every form ends with one re-rank
 * of each point's kept candidates: the returned distances are float32 exact-
 * difference sums whose lane partials are added by a butterfly (relative
 * error below (4 ceil(d / 128) + 7) 2^-24, 1.1e-6 at d = 384).
 * k        : 1 <= k <= HF_MAX_K.
 * w        : window half-width, w >= 1.
 * out_idx  : n x k int32 (row i = neighbours of point i); -1 in unfilled slots.
 * out_dist : n x k float32 squared distances; +inf in unfilled slots.
 */
int hf_knn_graph(hf_forest* f, int32_t k, int32_t w, int32_t* out_idx, float* out_dist,
                 void* stream);

/*
 * hf_search -- batched query search (Algorithm 1 first stage and final
 * selection; Section 2: binary search locates a point in a Hilbert order).
 * Queries are quantized with the data's lo/scale (clamped); in each tree the
 * query's position p is the lower bound of its full key among the data keys;
 * the candidates are the points at positions [p - w, p + w); the result is the
 * k nearest of their union by float32 squared distance.
 * queries  : nq x d float32, row-major; nq >= 0 (0 returns HF_OK at once).
 * out_idx  : nq x k int32; out_dist : nq x k float32.
 */
int hf_search(hf_forest* f, const float* queries, int64_t nq, int32_t k, int32_t w,
              int32_t* out_idx, float* out_dist, void* stream);

/*
 * hf_search_static -- hf_search without any device allocation, for callers
 * that may not allocate device memory while they run (a serving process with
 * a memory budget fixed up front, a runtime whose pool owns all device
 * memory, a latency path that must not take the allocator's locks). The paper
 * has no counterpart: this is an interface variant of hf_search with the same
 * results.
 *
 * The queries' quantized codes go to a fixed scratch array inside the
 * library's device image (HF_STATIC_QUERY_BYTES, held by every GPU that loads
 * the library until the process exits) instead of a per-call allocation.
 * Limits and rules:
 *   - nq * d must not exceed HF_STATIC_QUERY_BYTES, else HF_EINVAL;
 *   - queries, out_idx and out_dist must be device memory (host buffers would
 *     need staging copies), else HF_EINVAL;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture;
 *   - every call uses the same array, overwriting it completely: calls that
 *     overlap on the GPU (other streams, other threads, other forests on the
 *     same device) race on it and must be serialised by the caller.
 * Results, status codes and synchronisation are those of hf_search in modes
 * 0..2; the sketch form (mode 3) is not run here (HF_ENOTIMPL).
 */
#define HF_STATIC_QUERY_BYTES (4u << 20)
int hf_search_static(hf_forest* f, const float* queries, int64_t nq, int32_t k, int32_t w,
                     int32_t* out_idx, float* out_dist, void* stream);

/* ---- batched form: many independent point sets -----------------------------
 * Many small independent problems (point sets of uneven size) are built and
 * graphed together so that every kernel launch covers all of them: the paper
 * treats one dataset at a time; this is an interface and scheduling extension
 * with the same per-set results.
 *
 * hf_build_segmented -- one forest over nsets independent sets stacked in one
 * row-major matrix: rows offsets[s] .. offsets[s+1]-1 form set s (offsets: host,
 * nsets + 1 values, offsets[0] = 0, every set at least 2 rows, nsets <=
 * HF_MAX_SETS). Each set is quantized with its own per-axis range; all sets
 * share the T per-tree permutations and reflections of `seed`; every order
 * lists set 0's points first (in their own Hilbert order), then set 1's, ...
 * hf_knn_graph then gives, for every row, exactly the lists hf_build +
 * hf_knn_graph give on that set alone (plain and sketch forms), with row
 * indices of the stacked matrix (subtract offsets[s]). Tensor forms, the
 * budgeted graph and search return HF_ENOTIMPL on a segmented forest.
 */
#define HF_MAX_SETS 256
int hf_build_segmented(const float* points, const int64_t* offsets, int32_t nsets, int32_t d, int32_t T,
                       int32_t bits, uint64_t seed, const char* options, void* stream, hf_forest** out);

/*
 * Enqueue-only graph, for CUDA-graph capture (plain or Gram form: the forest's
 * mode 0, 1 or 2 when hf_graph_plan runs; a window the form cannot run is
 * HF_ENOTIMPL, never a change of form). hf_graph_plan keeps per-point lists
 * (and, for the Gram forms, the operand copies) in the forest for (k, w) and
 * the plain window kernel's block size `threads` (0: chosen per band, else
 * 256 or 512). hf_knn_graph_enqueue then enqueues the whole graph on
 * `stream` into DEVICE outputs (n x k) without allocating or synchronising,
 * so it can be captured; errors surface through hf_status, which synchronises
 * `stream` and reads and clears the device error word.
 */
int hf_graph_plan(hf_forest* f, int32_t k, int32_t w, int32_t threads, void* stream);
int hf_knn_graph_enqueue(hf_forest* f, int32_t* out_idx, float* out_dist, void* stream);
int hf_status(hf_forest* f, void* stream);

/*
 * CUDA graphs of enqueue-only work: hf_capture_begin starts a (relaxed)
 * capture on `stream` (not the legacy default stream), hf_capture_end ends it
 * and instantiates the graph into *exec; hf_graph_launch replays it on
 * `stream`; hf_graph_destroy frees it.
 */
int hf_capture_begin(void* stream);
int hf_capture_end(void* stream, void** exec);
int hf_graph_launch(void* exec, void* stream);
int hf_graph_destroy(void* exec);

/*
 * hf_exact_knn_rows -- exact k nearest neighbours (float32 exact differences,
 * ties by index, the row itself excluded) of the given rows (host int64) among
 * the points of their own set; out_idx / out_dist nrows x k, host or device.
 * The ground truth of recall estimates (autotuner, tests).
 */
int hf_exact_knn_rows(hf_forest* f, const int64_t* rows, int32_t nrows, int32_t k, int32_t* out_idx,
                      float* out_dist, void* stream);

/*
 * hf_autotune -- picks the graph plan for (k, target recall): for each form
 * in the mask `forms` (bit 0 plain float32, bit 1 BF16 Gram, bit 2 FP8 Gram),
 * the smallest window w of a fixed ladder (2 .. w_max, within the form's
 * limits) whose graph reaches target_recall on `sample` evenly spread rows
 * (recall against hf_exact_knn_rows; it grows with w because the candidate
 * sets grow), found by bisection, and at that w the faster block size of
 * the plain window kernel (256 or 512 threads; the Gram kernel is
 * persistent; the Gram forms are tried with 16 and with 32 list slots per
 * point, i.e. tensor_slack 16 - k and 32 - k, where they hold k + 1); then
 * the fastest variant that reaches the target (CUDA-event time of the whole
 * graph), else the one with the highest recall. Leaves that form
 * (hf_set_option mode, tensor_slack) and plan (hf_graph_plan) in the forest
 * and reports them with the sample recall and the graph's time; *out_form
 * is the mode plus 256 x the list slots for a Gram form.
 */
int hf_autotune(hf_forest* f, int32_t k, double target_recall, int32_t sample, int32_t w_max, int32_t forms,
                int32_t* out_form, int32_t* out_w, int32_t* out_threads, double* out_recall, float* out_ms,
                void* stream);

/* ---- second stage: binary sketches ----------------------------------------
 * The paper filters the forest's candidates by the Hamming distance of 384-bit
 * sketches before the final vector distances (Section 3 index structure;
 * Algorithm 1 and Algorithm 2, second-stage filtering). It does not say how
 * the sketches are made; here bit j of point i is (<x_i, r_j> > 0) for the
 * rows r_j of a caller-supplied projection matrix R (sign random projection),
 * computed from the BF16-rounded x and R with FP32 accumulation on the tensor
 * cores. With hf_set_option mode=3 ("sketch form") hf_knn_graph keeps, per
 * point, the sketch_k2 candidates of smallest Hamming distance (ties by
 * index) over all trees' windows, then the k nearest of those by exact
 * float32 distance (w <= HF_PLAIN_MAX_W, sketch_k2 <= HF_MAX_K, else
 * HF_ENOTIMPL). hf_search in mode 3 follows Algorithm 1 with both filters:
 * each query's sketch (from the same R) against its window candidates of
 * every tree, the sketch_k2 (<= HF_MAX_K2) of smallest (Hamming distance,
 * index) survive, each brings the expand_h points on either side of it in the
 * master order (order 0), and the k nearest of that set by float32 distance
 * are returned. The first such search keeps a master-ordered copy of the
 * points (n x d float32) and the inverse of the master order (n x uint32)
 * until hf_free. hf_search_static does not run the sketch form (HF_ENOTIMPL
 * in mode 3). hf_set_sketch keeps the BF16 copy of R (bits x 64-padded d)
 * for the query sketches.
 */

/*
 * hf_set_sketch -- sketches of all points: R is bits x d float32 row-major
 * (host or device), bits a multiple of 64 in [64, 1024]. Replaces earlier
 * sketches. HF_EINVAL on bad arguments.
 */
int hf_set_sketch(hf_forest* f, const float* R, int32_t bits, void* stream);

/* hf_debug_sketch -- the sketches, n x bits/64 uint64 (bit j of point i is
 * bit j % 64 of word j / 64); HF_ESTATE before hf_set_sketch. */
int hf_debug_sketch(hf_forest* f, uint64_t* out, void* stream);

/* ---- learned per-point budget ---------------------------------------------
 * The paper spends one budget -- the number of sorts T and the window k1
 * around each position (Algorithm 2; Table 2 trades recall against it) -- on
 * every point. These calls learn a budget per point from its coordinates and
 * apply it. They are an extension of the method, not part of the paper.
 */

/*
 * hf_budget_labels -- training targets from a built forest: for each point i,
 * the cheapest cell (T, w) of the grid t_grid x w_grid (cost T * (128 + 2 w))
 * at which at least min_hits of its exact neighbours knn[i][0..k) lie within
 * w positions of i in one of the first T orders (Algorithm 2's candidate
 * rule); the largest cell when none does.
 * knn         : device, n x k int32 exact neighbours of every point (-1 =
 *               none), e.g. from hf_knn_graph with w >= n - 1 (every pair);
 * t_grid      : host, nt ascending tree counts in [1, forest T], nt <= 16;
 * w_grid      : host, nw ascending windows >= 1, nw <= 16;
 * out_targets : device, n x 2 float: (log2 w, log2 T) of the cell;
 * out_cell    : device, n int32: cell index a * nw + b (t_grid[a], w_grid[b]).
 */
int hf_budget_labels(hf_forest* f, const int32_t* knn, int32_t k, const int32_t* t_grid, int32_t nt,
                     const int32_t* w_grid, int32_t nw, int32_t min_hits, float* out_targets, int32_t* out_cell,
                     void* stream);

/*
 * hf_knn_graph_budget -- hf_knn_graph with a budget per point: point i takes
 * part in trees t < T_pt[i] with window w_pt[i] (its candidates are the
 * points within w_pt[i] positions of it in those orders; 0 trees or a 0
 * window leave it out); the band kernel works on each 128-position tile up
 * to the tile's largest window and skips tiles with none. Tensor forms only
 * (hf_set_option mode 1 or 2; HF_ENOTIMPL otherwise).
 * w_pt, T_pt : device, n int32 each;
 * w_max      : the largest w_pt (1 .. 65535; larger entries are cut to it);
 * T_max      : the largest T_pt (1 .. forest T; trees past it are not used).
 * Outputs as hf_knn_graph.
 */
int hf_knn_graph_budget(hf_forest* f, int32_t k, const int32_t* w_pt, const int32_t* T_pt, int32_t w_max,
                        int32_t T_max, int32_t* out_idx, float* out_dist, void* stream);

/*
 * The budget model: an MLP d -> 256 -> 256 -> 2 with GELU activations
 * (GELU(z) = z Phi(z)), predicting (log2 w, log2 T). Weights, inputs and
 * activations are stored in BF16, every product is accumulated in FP32 on the
 * tensor cores (tcgen05); the fp32 master weights are updated by Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8). The loss of a batch of B rows is
 * L = 1/(2B) sum over rows and both outputs of (y - target)^2.
 * Parameters in packed order (floats): W1 [256][d], b1 [256], W2 [256][256],
 * b2 [256], W3 [2][256], b3 [2]; layer l computes z = W h + b.
 */
typedef struct hf_mlp hf_mlp; /* opaque; owned by the library */

/* hf_mlp_create -- a model for d inputs on the current device, weights
 * uniform in +-1/sqrt(fan_in) from splitmix64(seed), biases 0. */
int hf_mlp_create(int32_t d, uint64_t seed, hf_mlp** out);
/* hf_mlp_free -- releases the model (NULL is a no-op). */
int hf_mlp_free(hf_mlp* m);
/* hf_mlp_param_count -- number of floats in the packed parameter order. */
int hf_mlp_param_count(const hf_mlp* m, int64_t* out);
/* hf_mlp_get_params / hf_mlp_set_params -- the fp32 master weights in packed
 * order (host floats); set_params also refreshes the BF16 copies. */
int hf_mlp_get_params(const hf_mlp* m, float* out);
int hf_mlp_set_params(hf_mlp* m, const float* params);
/*
 * hf_mlp_predict -- outputs of n rows: x device n x d float32, out n x 2
 * float32 (device or host).
 */
int hf_mlp_predict(hf_mlp* m, const float* x, int64_t n, float* out, void* stream);
/*
 * hf_mlp_grads -- loss and gradients (packed order, host floats) of one batch
 * of B rows (128 <= B <= 8192, a multiple of 128): x device B x d, targets
 * B x 2 (device or host). Weights unchanged.
 */
int hf_mlp_grads(hf_mlp* m, const float* x, const float* targets, int32_t B, float* out_grads, float* out_loss,
                 void* stream);
/*
 * hf_mlp_train -- `steps` Adam steps with learning rate lr on consecutive
 * batches of B rows (wrapping around) of the device-resident training set
 * x (n x d) and targets (n x 2); *out_loss gets the mean batch loss of the
 * last min(steps, 50) steps.
 */
int hf_mlp_train(hf_mlp* m, const float* x, const float* targets, int64_t n, int32_t B, int32_t steps, float lr,
                 float* out_loss, void* stream);

/* hf_free -- releases the forest and everything it owns (NULL is a no-op). */
int hf_free(hf_forest* f);

/*
 * hf_trim_pool -- device memory of the library (forests and per-call
 * scratch) comes from a library-owned, stream-ordered pool on each device, so
 * that memory freed by one call is reused by the next without a device-wide
 * synchronisation. Up to a quarter of the device's memory (64 GiB at most)
 * stays cached in the pool after it is freed. hf_trim_pool waits for the
 * current device and returns that device's cached memory to the driver, for
 * callers that share the GPU with other allocators. Not part of the paper's
 * method. Returns HF_OK or HF_ECUDA.
 */
int hf_trim_pool(void);

/* hf_status_string -- static text for a status code (never NULL). */
const char* hf_status_string(int status);

/*
 * hf_set_option -- per-forest run-time options for later calls:
 *   mode=0  plain float32 window distances (default), each point keeping its
 *           best window_list_pitch(k) candidates by their sequential-sum
 *           distance before the re-rank; w <= HF_PLAIN_MAX_W (HF_ENOTIMPL
 *           beyond);
 *   mode=1  tensor-core window distances: BF16 Gram bands (tcgen05, FP32
 *           accumulation) estimate every candidate's distance, each point
 *           keeps its best k + slack (rounded up to 16 or 32; see
 *           tensor_slack) by that estimate, and those are re-ranked by
 *           float32 exact-difference distance, so returned distances are
 *           exact float32 values; any w >= 1;
 *   mode=2  as mode 1 with FP8 e4m3 operands and one scale per vector
 *           (s = max|x| / 448; tcgen05 kind::f8f6f4, FP32 accumulation);
 *   modes 1 and 2 fall back to mode 0 when the Gram kernel's shared-memory
 *   layout does not fit: for w > 64 a tile's 128 own rows stay resident next
 *   to two or more stages of 256 rows, which holds up to d = 512 in mode 1
 *   and d = 896 in mode 2 (hf_get_timings slot 8 reports the form that
 *   ran); they return HF_ENOTIMPL when k + slack > 32;
 *   mode=3  sketch form: Hamming screen of binary sketches (hf_set_sketch
 *           first, HF_ESTATE otherwise), then the exact float32 re-rank;
 *   tensor_slack=S  in modes 1 and 2, keep k + S candidates per point for
 *           the re-rank (rounded up to 16 or 32; default S = 1);
 *   sketch_k2=K2  in mode 3, candidates kept by Hamming distance
 *           (1..HF_MAX_K2, default 60; the graph takes at most HF_MAX_K and
 *           keeps at least k);
 *   expand_h=H  in mode 3, master-order neighbours taken on either side of
 *           each search survivor (default 2);
 *   timing=1  record per-phase CUDA-event timings (default 1).
 * Unknown keys or values give HF_EINVAL.
 */
int hf_set_option(hf_forest* f, const char* key, int64_t value);

/*
 * hf_get_timings -- milliseconds of the last calls' phases, in this order:
 * [0] quantize, [1] keys, [2] sort (with the small-run fix-up), [3] big-run
 * fix-up, [4] window distances + merge (all trees; the Gram kernels in mode
 * 1), [5] search, [6] number of kernel launches of the last build (as a
 * float), [7] re-rank (every form), [8] the form the last hf_knn_graph ran
 * (0 = plain float32 window kernel, 1 = BF16 tensor-core Gram bands, 2 = FP8
 * e4m3 Gram bands, 3 = sketch form), so a caller that asked for a tensor form can see whether
 * it fell back, [9] the time spent gathering each tree's rows into its
 * order (tensor forms; on a second stream, overlapping the previous tree's
 * Gram band, so it is not a part of [4]), [10] the Gram band launches alone
 * (tensor forms), [11] reserved (0). Writes min(cap, 12).
 */
int hf_get_timings(const hf_forest* f, float* out_ms, int32_t cap);

/* hf_info -- n, d, T, bits, W (key words), K (prefix words the sort orders
 * by), K2 (key words the prefix kernels form per point, K <= K2 <= W), L (top
 * bit levels those words come from) into out[0..7]; the first `cap` only. */
int hf_info(const hf_forest* f, int64_t* out, int32_t cap);

/*
 * hf_launch_count -- number of CUDA kernels this library has launched in this
 * process so far (all forests, all threads). A diagnostic counter: read it
 * before and after a region to count that region's launches.
 */
uint64_t hf_launch_count(void);

/*
 * hf_tree_params -- host-only: the axis permutation pi[d] and reflection bits
 * r[d] of tree `tree` for `seed` (conventions above). Host pointers only.
 */
int hf_tree_params(uint64_t seed, int32_t tree, int32_t d, int32_t* pi, uint8_t* r);

/* ---- inspection exports (tests and tools) -------------------------------- */

/* Quantized codes, n x d uint8, point order. */
int hf_debug_codes(hf_forest* f, uint8_t* out_codes, void* stream);

/* Full keys of tree t, n x W uint64 (row i = point i, word 0 first). */
int hf_debug_keys(hf_forest* f, int32_t tree, uint64_t* out_keys, void* stream);

/* The first K2 key words of tree t as the build's prefix kernels form them
 * (hf_info's K2; the sort orders by the first K, the rest settle ties),
 * K2 x n uint64 WORD-major: word w of point i at out_words[w * n + i]. They
 * equal the first K2 words of hf_debug_keys; this export checks the prefix
 * kernels (bit-sliced top level, bit-sliced L levels) on their own. */
int hf_debug_prefix(hf_forest* f, int32_t tree, uint64_t* out_words, void* stream);

/* Order of tree t: sigma[p] = point at position p, n uint32. */
int hf_debug_order(hf_forest* f, int32_t tree, uint32_t* out_sigma, void* stream);

/* Lower-bound positions of nq queries in tree t, nq int64. */
int hf_debug_locate(hf_forest* f, int32_t tree, const float* queries, int64_t nq,
                    int64_t* out_pos, void* stream);

/*
 * Full keys of raw codes with the identity permutation and no reflection:
 * codes n x d uint8 (values < 2^bits), out n x W uint64. n >= 1.
 */
int hf_debug_keys_from_codes(const uint8_t* codes, int64_t n, int32_t d, int32_t bits,
                             uint64_t* out_keys, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HF_H */
