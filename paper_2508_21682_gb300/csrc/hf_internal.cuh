// Internal declarations shared by the CUDA translation units of libhf.so.
#pragma once

#include <cuda_runtime.h>

#include <vector>
#include <stdint.h>

#include <string>

#include "../../include/hf.h"

// ---------------------------------------------------------------------------
// Device error word: bit flags OR-ed in by kernels, read by the host at the
// end of every call.
// ---------------------------------------------------------------------------
enum : int {
  HF_ERRBIT_TIMEOUT = 1,    // a bounded inter-block wait gave up
  HF_ERRBIT_NONFINITE = 2,  // NaN or inf in points or queries
};

__device__ __forceinline__ void hf_raise(int* err, int bit) { atomicOr(err, bit); }

// Slots of hf_get_timings (phase milliseconds and a few per-call figures).
constexpr int HF_NTIMINGS = 12;

// ---------------------------------------------------------------------------
// The forest handle.
// ---------------------------------------------------------------------------
struct SortScratch {  // for a batch of TB trees
  uint64_t* keys_a = nullptr;  // [TB][n]
  uint64_t* keys_b = nullptr;  // [TB][n]
  uint32_t* vals_a = nullptr;  // [TB][n]
  uint32_t* vals_b = nullptr;  // [TB][n]
  uint32_t* status = nullptr;  // [passes]([TB][tiles + 1][256] look-back words, ticket)
  uint32_t* hist = nullptr;    // [TB][K*8][256] digit counts -> exclusive offsets
};

struct TieScratch {
  uint32_t* counters = nullptr;  // [0] runs, [1] big runs, [2] big elements
  uint2* runs = nullptr;         // (start, len) of runs, capacity n/2 + 1
  uint2* big_runs = nullptr;     // per tree: runs longer than the small cap
  int64_t big_cap = 0;           // entries per tree in big_runs
  uint64_t* fk = nullptr;        // full-key scratch of the small-run fix-up
};

struct hf_forest {
  int device = 0;
  int64_t n = 0;
  int d = 0, T = 0, bits = 0, W = 0, K = 0, L = 0, W32 = 0;
  int K2 = 0;  // key words computed per point (K sorted + up to 4 tie-breakers)
  uint64_t seed = 0;

  const float* x = nullptr;  // n x d float32, device
  float* x_owned = nullptr;  // device copy when the caller passed host memory

  float* lo = nullptr;        // [nseg][d]
  float* scale = nullptr;     // [nseg][d]
  uint32_t* planes = nullptr; // [bits][n][W32]; plane 0 = most significant bit

  int32_t* pi = nullptr;      // [T][d]
  uint32_t* rbits = nullptr;  // [T][W32]; bit j of word m: reflection of permuted axis 32m+j
  uint64_t* prefix = nullptr; // [T][K][n] key prefixes in sorted order
  uint32_t* sigma = nullptr;  // [T][n] position -> point

  int* err = nullptr;         // device error word

  // tensor mode: operand copy of the points (BF16 or e4m3 rows, pitch
  // gram_row_bytes) and per point (squared norm, scale), made on first use
  void* xb = nullptr;
  float2* xmeta = nullptr;
  int xform = 0;  // form of xb: 0 none, 1 BF16, 2 FP8
  // second stage: binary sketches (n x sketch_bits / 64 words)
  uint64_t* sketch = nullptr;
  int sketch_bits = 0;
  void* sketch_r = nullptr;   // BF16 projection (bits x dp) for query sketches
  float* xm = nullptr;        // master-ordered points (n x d), built on demand
  uint32_t* posm = nullptr;   // inverse of the master order

  // segmented forest: rows seg_off[s] .. seg_off[s+1]-1 are independent set
  // s (own range, own windows); every order lists set 0's points first, then
  // set 1's, ... (each set in its own Hilbert order)
  int nseg = 1;
  int64_t* seg_off = nullptr;  // [nseg + 1], device
  uint32_t* seg = nullptr;     // [n] set of each row, device
  std::vector<int64_t> seg_off_h;

  uint64_t* pk = nullptr;     // [TB][K2][n] key words in point order (scratch)
  uint32_t* p0t = nullptr;    // [ceil(n/32)][d] bit-sliced plane 0 (scratch, top-level prefix path)
  int TB = 1;                 // trees keyed and sorted together
  SortScratch sort;
  TieScratch tie;

  // options
  int64_t spin_limit_us = 2000000;
  int test_stall = 0;
  int sort_batch_max = 0;  // cap on trees per sort batch (0: by memory)
  int mode = 0;
  int tensor_slack = -1;  // extra list slots kept for the re-rank (-1: k)
  // enqueue-only graph plan (hf_graph_plan / hf_autotune)
  uint32_t* plan_li = nullptr;
  float* plan_ld = nullptr;
  void* plan_xs = nullptr;     // tensor forms: operand rows in tree order
  float2* plan_ms = nullptr;
  int plan_k = 0, plan_w = 0, plan_kp = 0, plan_nt = 0, plan_form = 0;
  int sketch_k2 = 60;     // candidates kept by Hamming distance (mode 3)
  int expand_h = 2;       // master-order neighbours per survivor (mode 3 search)
  int timing = 1;
  cudaStream_t side = nullptr;  // second stream of the tensor forms' row gathers

  float timings[HF_NTIMINGS] = {0};
};

// ---------------------------------------------------------------------------
// Launchers (each enqueues on `s`; errors surface through cudaGetLastError)
// ---------------------------------------------------------------------------
// quantize.cu
void launch_range(const float* x, int64_t n, int d, float* lo, float* scale, int bits,
                  int* err, void* scratch, size_t scratch_bytes, cudaStream_t s);
size_t range_scratch_bytes(int64_t n, int d);
// segmented matrix (rows off[s] .. off[s+1]-1 form set s): per-set range
// (lo / scale: nseg x d) and the set of every row
void launch_seg_range(const float* x, int d, const int64_t* off, int nseg, int bits, float* lo, float* scale, int* err,
                      cudaStream_t s);
void launch_seg_of_row(const int64_t* off, int nseg, int64_t n, uint32_t* seg, uint64_t* seg64, cudaStream_t s);
void launch_quantize_planes(const float* x, int64_t n, int d, const float* lo, const float* scale,
                            int bits, uint32_t* planes, int* err, cudaStream_t s, const uint32_t* seg = nullptr);
void launch_quantize_codes(const float* x, int64_t n, int d, const float* lo, const float* scale,
                           int bits, uint8_t* codes, int* err, cudaStream_t s);
void launch_planes_to_codes(const uint32_t* planes, int64_t n, int d, int bits, uint8_t* codes,
                            cudaStream_t s);

// keys.cu
bool prefix_top_path(int d, int K, int L);  // prefix words from plane 0 alone
// plane 0 in bit-sliced form: p0t[g][c] bit j = top bit of coordinate c of point 32g + j
void launch_plane0_slice(const uint32_t* planes, int64_t n, int d, uint32_t* p0t, cudaStream_t s);
// p0t: the bit-sliced plane 0 (used on the top-level path), or null
void launch_prefix_keys(const uint32_t* planes, const uint32_t* p0t, int64_t n, int d, int bits, int K, int L,
                        const int32_t* pi, const uint32_t* rbits, uint64_t* pk, cudaStream_t s);
void launch_full_keys_planes(const uint32_t* planes, int64_t n, int d, int bits, int W,
                             const int32_t* pi, const uint32_t* rbits, uint64_t* out,
                             cudaStream_t s);
void launch_full_keys_codes(const uint8_t* codes, int64_t n, int d, int bits, int W,
                            const int32_t* pi, const uint32_t* rbits, uint64_t* out,
                            cudaStream_t s);

// sort.cu
int sort_batch(hf_forest* f, int t0, int tb, cudaStream_t s);  // keys of trees t0.. -> sigma, prefix
// segmented forest: stable partition of every tree's order by the set of its
// point (seg64: the set of each point as a 64-bit key), after the fix-ups
int segment_pass(hf_forest* f, const uint64_t* seg64, cudaStream_t s);
int tie_fixup_big(hf_forest* f, int tree, uint32_t big_runs, cudaStream_t s);

// window.cu
int window_list_pitch(int k);  // list slots per point kept by the window kernel (>= k)
int launch_window_graph(const float* x, int64_t n, int d, const uint32_t* sigma, int w, int kp,
                        uint32_t* list_idx, float* list_dist, cudaStream_t s,
                        const uint32_t* segr = nullptr, const int64_t* segoff = nullptr, int nt = 0);
void launch_list_init(uint32_t* idx, float* dist, int64_t count, cudaStream_t s);
// the same over binary sketches (words 32-bit words per point), Hamming distance
int launch_window_hamming(const uint32_t* sketch, int64_t n, int words, const uint32_t* sigma, int w, int kp,
                          uint32_t* list_idx, float* list_dist, cudaStream_t s,
                          const uint32_t* segr = nullptr, const int64_t* segoff = nullptr);

// gram.cu -- tensor-core window distances. form 1: BF16 operands; form 2:
// FP8 e4m3 operands with one scale per vector.
int gram_supported(int d, int w, int form);
size_t gram_row_bytes(int d, int form);  // operand row pitch in bytes
// operand rows (n x gram_row_bytes) and per point (squared norm, scale)
void launch_prepare_operands(const float* x, int64_t n, int d, int form, void* xq, float2* meta, cudaStream_t s);
// one tree: tile_w (per tile of 128 positions, this tree's window) and pw
// (per point window) may be null, then every point uses w
// one tree's operand rows and (norm, scale) in its position order:
// xs[p] = xq[sigma[p]] (n x gram_row_bytes), ms[p] = meta[sigma[p]]
void launch_gather_rows(const void* xq, const float2* meta, int form, int64_t n, int d, const uint32_t* sigma,
                        void* xs, float2* ms, cudaStream_t s);
// one tree from its gathered rows; tile_w (per tile of 128 positions, this
// tree's window; 0 skips the tile) and pw (per point window) may be null,
// then every point uses w
int launch_gram_window(int form, int64_t n, int d, const uint32_t* sigma, int w, const int32_t* tile_w,
                       const uint16_t* pw, int kp, uint32_t* li, float* ld, int* err, const void* xs, const float2* ms,
                       cudaStream_t s,
                       const uint32_t* segr = nullptr, const int64_t* segoff = nullptr);
// exact float32 re-rank of the first kc slots of each KP-slot list
int launch_rerank(const float* x, int64_t n, int d, const uint32_t* order, int kp, int kc, uint32_t* li, float* ld,
                  cudaStream_t s);

// budget.cu
// labels from the inverse orders of the first T trees (pos: T x n scratch)
int launch_budget_labels(const uint32_t* sigma, int T, int64_t n, const int32_t* knn, int k, const int32_t* tg,
                         int ntg, const int32_t* wg, int nwg, int min_hits, float* out, int32_t* cell, int32_t* pos,
                         cudaStream_t s);
// tree t's per-point windows pw (0: the point sits this tree out) and per-tile
// largest windows tile_w from per-point (w, T) budgets
void launch_tree_budget(const uint32_t* sigma, int64_t n, int t, const int32_t* wpt, const int32_t* tpt, uint16_t* pw,
                        int32_t* tile_w, cudaStream_t s);

// sketches (budget.cu): bit j of point i = (<x_i, r_j> > 0); xb and rb BF16
// with row pitch dp (a multiple of 64); sketch n x bits/64 words
int launch_sketch(const void* xb, int64_t n, int dp, const void* rb, int bits, uint64_t* sketch, int* err,
                  cudaStream_t s);
// rows x cols float32 (pitch cols) -> rows x ld BF16 (zero padded)
void launch_f32_to_bf16(const float* x, int64_t rows, int cols, int ld, void* out, cudaStream_t s);

// search.cu
int launch_search(const hf_forest* f, const float* q, const uint8_t* qcodes, int64_t nq, int k,
                  int w, uint32_t* out_idx, float* out_dist, int64_t* out_pos, int only_tree,
                  cudaStream_t s);
// sketch form of the search: positions of every tree (pos, T x nq) and query
// sketches (qsk) first; needs f->sketch, f->xm and f->posm
int launch_sketch_search(const hf_forest* f, const float* q, int64_t nq, const int64_t* pos, const uint64_t* qsk,
                         int k, int w, int k2, int h, uint32_t* out_idx, float* out_dist, cudaStream_t s);
void launch_master_layout(const float* x, int64_t n, int d, const uint32_t* sig0, float* xm, uint32_t* posm,
                          cudaStream_t s);
// exact k nearest of given rows (device int64) among their own set's points
int launch_exact_rows(const hf_forest* f, const int64_t* rows, int nrows, int k, uint32_t* out_idx, float* out_dist,
                      cudaStream_t s);
void launch_gather_list_rows(const uint32_t* lists, int kp, const int64_t* rows, int nrows, int k, uint32_t* out,
                             cudaStream_t s);

// host helpers (api.cu)
void hf_tree_params_host(uint64_t seed, int tree, int d, int32_t* pi, uint8_t* r);
// Device memory from the library's stream-ordered pool (allocated and freed
// in order on s).
cudaError_t hf_dalloc_bytes(void** p, size_t bytes, cudaStream_t s);
void hf_dfree_bytes(void* p, cudaStream_t s);
// Synchronises s, reads and clears the forest's error word and maps it (and
// any CUDA error) to a status code; every entry point ends with it.
int hf_finish(hf_forest* f, cudaStream_t s);

// With HF_DEBUG=1 in the environment: synchronise `s` after a launch and print
// the kernel's name and any CUDA error to stderr (a no-op otherwise).
void hf_after_launch(const char* what, cudaStream_t s);

static inline unsigned hf_blocks(int64_t work, int per_block, int64_t cap = (1 << 30)) {
  int64_t b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}
