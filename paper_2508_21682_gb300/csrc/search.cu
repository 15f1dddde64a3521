// Batched query search.
//
// Paper, Section 2: since the Hilbert order is a total order, binary search
// locates an arbitrary point in a sorted set; Algorithm 1 then takes the
// candidates near each query's position in every tree and keeps the top k by
// vector distance. The paper simulates a collective Hilbert sort of all queries
// on the CPU; here every query is located independently, which parallelises
// trivially.
//
// One warp per query, looping over the trees; the query's top-k list lives in
// registers across the warp (entry e in lane e % 32, slot e / 32).
//  * Key prefix: when the first K key words lie in the top bit level (d >=
//    64K) the warp forms them with ballots (running XOR of the permuted,
//    reflected top bits); otherwise lane 0 runs the transform.
//  * Locate: 32-way probing rounds find the lower bound among the sorted
//    prefixes; only when the prefix at that position equals the query's does
//    a second search find the end of the equal run, inside which lane 0
//    refines the position by full keys (computed on demand from the planes).
//  * Score: the window's candidates go 32 at a time. Every lane reads its 4
//    coordinates of each candidate row (a row is read by the warp in 512-byte
//    coalesced pieces) and keeps one partial sum per candidate; a transposing
//    butterfly (31 shuffles) leaves candidate j's distance in lane j. The
//    butterfly adds lane partials in the same tree for every candidate, so a
//    (query, point) pair gets the same value in every tree.
//  * Merge: the 32 scored candidates are sorted across the warp and inserted
//    in ascending order until the first one that cannot enter.
#include <cuda_runtime.h>
#include <math.h>

#include "hf_internal.cuh"
#include "hilbert_device.cuh"

namespace {

constexpr int SWARPS = 4;
constexpr unsigned FULL = 0xffffffffu;

// Shared bytes per warp: query prefix (K words), candidate ids (32 words),
// two coordinate scratch rows (d bytes each), rounded to 16.
__host__ __device__ __forceinline__ size_t search_per_warp(int K, int d) {
  return ((size_t)K * 8 + 32 * 4 + 2 * (size_t)d + 15) & ~(size_t)15;
}

__device__ __forceinline__ bool lessp(float da, uint32_t ia, float db, uint32_t ib) {
  return da < db || (da == db && ia < ib);
}

// -1 / 0 / +1 comparing the sorted prefix at position m with the query prefix.
__device__ __forceinline__ int cmp_prefix(const uint64_t* __restrict__ pre, int64_t n, int K, int64_t m,
                                          const uint64_t* qp) {
  for (int w = 0; w < K; ++w) {
    const uint64_t a = __ldg(pre + (size_t)w * n + m);
    if (a != qp[w]) return a < qp[w] ? -1 : 1;
  }
  return 0;
}

// Full-key comparison: is the key of transformed Yd smaller than that of Yq?
__device__ __forceinline__ bool full_key_less(const uint8_t* Yd, const uint8_t* Yq, int d, int bits, int W) {
  for (int w = 0; w < W; ++w) {
    const uint64_t a = hf_pack_word(Yd, d, bits, w), b = hf_pack_word(Yq, d, bits, w);
    if (a != b) return a < b;
  }
  return false;
}

// Running XOR from the most significant bit down: bit j of the result is the
// XOR of bits 31..j of v.
__device__ __forceinline__ uint32_t xor_scan_msb(uint32_t v) {
  v ^= v >> 1;
  v ^= v >> 2;
  v ^= v >> 4;
  v ^= v >> 8;
  v ^= v >> 16;
  return v;
}

struct SearchArgs {
  const float* x;
  int64_t n;
  int d, bits, K, L, W, W32, T;
  const uint32_t* planes;
  const int32_t* pi;
  const uint32_t* rbits;
  const uint64_t* prefix;
  const uint32_t* sigma;
  const float* q;
  const uint8_t* qcodes;
  int64_t nq;
  int k, w;
  uint32_t* out_idx;
  float* out_dist;
  int64_t* out_pos;
  int only_tree;
  int pos_all;  // positions of every tree into out_pos[t * nq + query], no lists
  int vec4;  // d % 4 == 0 and both matrices 16-byte aligned
  int top;   // the K prefix words lie in the top bit level (d >= 64K)
};

// Query prefix from the top bits, the warp taking 32 coordinates per ballot:
// key bit i (i < 64K) is the XOR of the permuted, reflected top bits of
// coordinates 0..i; word w holds bits 64w .. 64w+63, most significant first.
__device__ __forceinline__ void warp_top_prefix(const uint8_t* __restrict__ qc, int bits, int K,
                                                const int32_t* __restrict__ pi, const uint32_t* __restrict__ rb,
                                                uint64_t* qp, int lane) {
  uint32_t carry = 0;
  for (int w = 0; w < K; ++w) {
    uint32_t half[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = w * 64 + h * 32 + lane;
      const uint32_t bit = (((uint32_t)qc[__ldg(pi + i)] >> (bits - 1)) ^ (__ldg(rb + (i >> 5)) >> lane)) & 1u;
      uint32_t v = xor_scan_msb(__brev(__ballot_sync(FULL, bit)));
      if (carry) v = ~v;
      carry = v & 1u;
      half[h] = v;
    }
    if (lane == 0) qp[w] = ((uint64_t)half[0] << 32) | half[1];
  }
}

// Warp-wide bound over the sorted prefixes in [lo, n): each round the 32
// lanes probe 32 evenly spaced positions of [lo, hi) (one round trip), a
// ballot keeps the sub-interval that holds the first position whose prefix is
// not below the query's (le = false) or above it (le = true). About log32(n)
// rounds instead of log2(n) dependent steps.
__device__ __forceinline__ int64_t warp_bound(const uint64_t* __restrict__ pre, int64_t n, int K, const uint64_t* qp,
                                              bool le, int64_t lo, int lane) {
  int64_t hi = n;  // answer in [lo, hi]
  while (hi - lo > 0) {
    const int64_t len = hi - lo;
    const int64_t step = (len + 31) / 32;
    const int64_t m = lo + (int64_t)lane * step;
    bool below = false;  // position m lies before the answer
    if (m < hi) {
      const int c = cmp_prefix(pre, n, K, m, qp);
      below = le ? (c <= 0) : (c < 0);
    }
    const uint32_t bm = __ballot_sync(FULL, below);
    const int cnt = __popc(bm);  // lanes 0 .. cnt-1 are below (monotone)
    if (cnt == 0) {
      hi = lo;
    } else {
      const int64_t mlast = lo + (int64_t)(cnt - 1) * step;
      const int64_t nhi = lo + (int64_t)cnt * step;
      lo = mlast + 1;
      hi = nhi < hi ? nhi : hi;
    }
  }
  return lo;
}

// Bitonic sort of one (distance, index) pair per lane across the warp,
// ascending by (distance, index).
__device__ __forceinline__ void warp_sort(float& dv, uint32_t& iv, int lane) {
#pragma unroll
  for (int kk = 2; kk <= 32; kk <<= 1) {
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      const float od = __shfl_xor_sync(FULL, dv, j);
      const uint32_t oi = __shfl_xor_sync(FULL, iv, j);
      const bool up = (lane & kk) == 0;
      const bool lower = (lane & j) == 0;
      const bool other_less = lessp(od, oi, dv, iv);
      const bool take = (lower == up) ? other_less : !other_less && !(od == dv && oi == iv);
      if (take) {
        dv = od;
        iv = oi;
      }
    }
  }
}

// Transposing butterfly: lane l holds v[u] = its partial for candidate u;
// afterwards v[0] of lane l is the sum over all lanes of the partials for
// candidate l. Step s pairs lanes l and l ^ s; the lane whose bit s is set
// keeps the upper half of the remaining candidates.
__device__ __forceinline__ float warp_transpose_sum(float (&v)[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = up ? v[i] : v[i + s];
      const float keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(FULL, send, s);
    }
  }
  return v[0];
}

// Top-k list held across the warp: entry e = 32 s + lane in slot s.
template <int S>
struct WarpList {
  float dv[S];
  uint32_t iv[S];

  __device__ __forceinline__ void init() {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      dv[s] = INFINITY;
      iv[s] = 0xffffffffu;
    }
  }
  // Entry k - 1 (the one a candidate must beat).
  __device__ __forceinline__ void last(int k, float& d, uint32_t& i) const {
    const int s = (k - 1) >> 5, l = (k - 1) & 31;
    float ds = dv[0];
    uint32_t is = iv[0];
#pragma unroll
    for (int t = 1; t < S; ++t)
      if (s == t) {
        ds = dv[t];
        is = iv[t];
      }
    d = __shfl_sync(FULL, ds, l);
    i = __shfl_sync(FULL, is, l);
  }
  // Inserts (cd, ci) unless ci is already listed; entries at or beyond k are
  // scratch.
  __device__ __forceinline__ void insert(float cd, uint32_t ci, int k, int lane) {
    bool dup = false;
    int pos = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const bool valid = 32 * s + lane < k;
      dup |= __ballot_sync(FULL, valid && iv[s] == ci) != 0;
      pos += __popc(__ballot_sync(FULL, valid && lessp(dv[s], iv[s], cd, ci)));
    }
    if (dup) return;
    float cd_prev[S];
    uint32_t ci_prev[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      // entry e - 1: lane - 1 of the same slot, or lane 31 of the slot below
      float up_d = __shfl_up_sync(FULL, dv[s], 1);
      uint32_t up_i = __shfl_up_sync(FULL, iv[s], 1);
      const float wrap_d = __shfl_sync(FULL, dv[s > 0 ? s - 1 : 0], 31);
      const uint32_t wrap_i = __shfl_sync(FULL, iv[s > 0 ? s - 1 : 0], 31);
      if (lane == 0) {
        up_d = wrap_d;
        up_i = wrap_i;
      }
      cd_prev[s] = up_d;
      ci_prev[s] = up_i;
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int e = 32 * s + lane;
      if (e > pos) {
        dv[s] = cd_prev[s];
        iv[s] = ci_prev[s];
      } else if (e == pos) {
        dv[s] = cd;
        iv[s] = ci;
      }
    }
  }
};

template <int S>
__global__ void __launch_bounds__(SWARPS * 32) search_kernel(SearchArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const size_t per_warp = search_per_warp(a.K, a.d);
  unsigned char* base = smraw + per_warp * wib;
  uint64_t* qp = reinterpret_cast<uint64_t*>(base);
  uint32_t* cpid = reinterpret_cast<uint32_t*>(qp + a.K);
  uint8_t* Yq = reinterpret_cast<uint8_t*>(cpid + 32);
  uint8_t* Yd = Yq + a.d;

  const int64_t qi = (int64_t)blockIdx.x * SWARPS + wib;
  if (qi >= a.nq) return;
  const uint8_t* qc = a.qcodes + (size_t)qi * a.d;
  const float* qv = a.q + (size_t)qi * a.d;

  WarpList<S> list;
  list.init();

  const int t_begin = a.only_tree >= 0 ? a.only_tree : 0;
  const int t_end = a.only_tree >= 0 ? a.only_tree + 1 : a.T;
  for (int t = t_begin; t < t_end; ++t) {
    const int32_t* pi = a.pi + (size_t)t * a.d;
    const uint32_t* rb = a.rbits + (size_t)t * a.W32;
    const uint64_t* pre = a.prefix + (size_t)t * a.K * a.n;
    const uint32_t* sig = a.sigma + (size_t)t * a.n;
    if (a.top) {
      warp_top_prefix(qc, a.bits, a.K, pi, rb, qp, lane);
    } else if (lane == 0) {
      hf_load_coords_codes(qc, a.d, a.bits, a.L, pi, rb, Yq);
      hf_skilling(Yq, a.d, a.L);
      for (int w = 0; w < a.K; ++w) qp[w] = hf_pack_word(Yq, a.d, a.L, w);
    }
    __syncwarp();
    const int64_t lo = warp_bound(pre, a.n, a.K, qp, false, 0, lane);
    int64_t pos = lo;
    // [lo, lo2): positions whose prefix equals the query's
    if (a.K < a.W && lo < a.n && cmp_prefix(pre, a.n, a.K, lo, qp) == 0) {
      const int64_t lo2 = warp_bound(pre, a.n, a.K, qp, true, lo, lane);
      if (lane == 0) {
        // equal prefixes: lower bound by full key inside [lo, lo2)
        hf_load_coords_codes(qc, a.d, a.bits, a.bits, pi, rb, Yq);
        hf_skilling(Yq, a.d, a.bits);
        int64_t l = lo, h = lo2;
        while (l < h) {
          const int64_t mid = (l + h) >> 1;
          hf_load_coords_planes(a.planes, a.n, a.d, a.W32, a.bits, pi, rb, sig[mid], Yd);
          hf_skilling(Yd, a.d, a.bits);
          if (full_key_less(Yd, Yq, a.d, a.bits, a.W)) l = mid + 1;
          else h = mid;
        }
        pos = l;
      }
      pos = __shfl_sync(FULL, pos, 0);
    }
    if (a.only_tree >= 0 || a.pos_all) {
      if (lane == 0) a.out_pos[a.pos_all ? (size_t)t * a.nq + qi : (size_t)qi] = pos;
      continue;
    }
    const int64_t c0 = pos - a.w > 0 ? pos - a.w : 0;
    const int64_t c1 = pos + a.w < a.n ? pos + a.w : a.n;
    for (int64_t cb = c0; cb < c1; cb += 32) {
      const int64_t c = cb + lane;
      uint32_t pid = c < c1 ? __ldg(sig + c) : 0xffffffffu;
      float dist;
      if (a.vec4) {
        cpid[lane] = pid;
        __syncwarp();
        float part[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) part[u] = 0.f;
        for (int m = 4 * lane; m < a.d; m += 128) {
          const float4 qa = __ldg(reinterpret_cast<const float4*>(qv + m));
          // 8 candidate rows per group: all 8 loads are issued before any is
          // used (an empty slot reads the query's own row; its result is
          // discarded)
#pragma unroll
          for (int u0 = 0; u0 < 32; u0 += 16) {
            float4 xb[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const uint32_t p = cpid[u0 + u];
              const float* row = p != 0xffffffffu ? a.x + (size_t)p * a.d : qv;
              xb[u] = __ldg(reinterpret_cast<const float4*>(row + m));
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              float e = qa.x - xb[u].x;
              float acc = fmaf(e, e, part[u0 + u]);
              e = qa.y - xb[u].y;
              acc = fmaf(e, e, acc);
              e = qa.z - xb[u].z;
              acc = fmaf(e, e, acc);
              e = qa.w - xb[u].w;
              part[u0 + u] = fmaf(e, e, acc);
            }
          }
        }
        dist = warp_transpose_sum(part, lane);
        __syncwarp();
      } else {
        // one lane per candidate over the whole vector
        dist = 0.f;
        if (pid != 0xffffffffu) {
          const float* xv = a.x + (size_t)pid * a.d;
          for (int j = 0; j < a.d; ++j) {
            const float e = __ldg(qv + j) - __ldg(xv + j);
            dist = fmaf(e, e, dist);
          }
        }
      }
      if (pid == 0xffffffffu) dist = INFINITY;
      warp_sort(dist, pid, lane);
      // merge in ascending order; stop at the first that cannot enter
      for (int u = 0; u < 32; ++u) {
        const float cd = __shfl_sync(FULL, dist, u);
        const uint32_t ci = __shfl_sync(FULL, pid, u);
        if (ci == 0xffffffffu) break;
        float kd;
        uint32_t ki;
        list.last(a.k, kd, ki);
        if (!lessp(cd, ci, kd, ki)) break;
        list.insert(cd, ci, a.k, lane);
      }
    }
  }
  if (a.only_tree >= 0 || a.pos_all) return;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int e = 32 * s + lane;
    if (e < a.k) {
      a.out_idx[(size_t)qi * a.k + e] = list.iv[s];
      a.out_dist[(size_t)qi * a.k + e] = list.dv[s];
    }
  }
}

template <int S>
int launch_s(const SearchArgs& a, size_t smem, cudaStream_t s) {
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute((const void*)search_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
    return HF_ECUDA;
  search_kernel<S><<<hf_blocks(a.nq, SWARPS), SWARPS * 32, smem, s>>>(a);
  hf_after_launch("search_kernel", s);
  return HF_OK;
}

}  // namespace

int launch_search(const hf_forest* f, const float* q, const uint8_t* qcodes, int64_t nq, int k, int w,
                  uint32_t* out_idx, float* out_dist, int64_t* out_pos, int only_tree, cudaStream_t s) {
  if (k < 1 || k > 64) return HF_EINVAL;
  SearchArgs a;
  a.x = f->x;
  a.n = f->n;
  a.d = f->d;
  a.bits = f->bits;
  a.K = f->K;
  a.L = f->L;
  a.W = f->W;
  a.W32 = f->W32;
  a.T = f->T;
  a.planes = f->planes;
  a.pi = f->pi;
  a.rbits = f->rbits;
  a.prefix = f->prefix;
  a.sigma = f->sigma;
  a.q = q;
  a.qcodes = qcodes;
  a.nq = nq;
  a.k = k;
  a.w = w;
  a.out_idx = out_idx;
  a.out_dist = out_dist;
  a.out_pos = out_pos;
  a.only_tree = only_tree >= 0 ? only_tree : -1;
  a.pos_all = only_tree == -2;
  if (a.pos_all && !out_pos) return HF_EINVAL;
  a.vec4 = (f->d % 4 == 0) && ((reinterpret_cast<uintptr_t>(f->x) & 15) == 0) &&
           ((reinterpret_cast<uintptr_t>(q) & 15) == 0);
  a.top = f->d >= 64 * f->K;
  const size_t smem = search_per_warp(f->K, f->d) * SWARPS;
  const int rc = k <= 32 ? launch_s<1>(a, smem, s) : launch_s<2>(a, smem, s);
  if (rc != HF_OK) return rc;
  return cudaGetLastError() == cudaSuccess ? HF_OK : HF_ECUDA;
}

// ---------------------------------------------------------------------------
// Search with the second-stage filter and the master-order expansion
// (Algorithm 1, both filters).
//
// One warp per query, after the positions of every tree are known:
//  * Hamming stage: the window candidates of each tree go 32 at a time, one
//    per lane; a lane XORs its candidate's sketch with the query's (held in
//    shared memory) and counts the bits; the 32 counts are sorted across the
//    warp and merged into a warp-held list of the k2 smallest (Hamming
//    distance, index), duplicates across trees dropped on insertion.
//  * Expansion: entry e of the expanded set is survivor e / (2h + 1) shifted by
//    e % (2h + 1) - h positions in the master order (order 0), clipped. The
//    rows come from the master-ordered copy of the points, so the 2h + 1 rows
//    of one survivor are adjacent in memory.
//  * Final stage: the expanded entries are scored with the same float32
//    exact-difference distance and transposing butterfly as the plain search
//    and merged into the warp-held top-k list.
// ---------------------------------------------------------------------------
namespace {

constexpr int SK_MAX_WORDS = 16;  // sketches up to 1024 bits

struct SketchSearchArgs {
  const float* q;
  int64_t nq;
  int d;
  const float* xm;         // n x d, row p = point sig0[p]
  const uint32_t* sig0;    // master order
  const uint32_t* posm;    // inverse of the master order
  const uint32_t* sigma;   // T x n orders
  const int64_t* pos;      // T x nq lower-bound positions
  const uint64_t* sk;      // n x words
  const uint64_t* qsk;     // nq x words
  int words;
  int64_t n;
  int T, w, k2, h, k;
  uint32_t* out_idx;
  float* out_dist;
  int vec4;
};

template <int S2, int S>
__global__ void __launch_bounds__(SWARPS * 32) sketch_search_kernel(SketchSearchArgs a) {
  __shared__ uint64_t s_q[SWARPS][SK_MAX_WORDS];
  __shared__ uint32_t s_c2[SWARPS][32 * S2];
  __shared__ uint32_t s_id[SWARPS][32];
  __shared__ uint32_t s_row[SWARPS][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t qi = (int64_t)blockIdx.x * SWARPS + wib;
  if (qi >= a.nq) return;
  if (lane < a.words) s_q[wib][lane] = a.qsk[(size_t)qi * a.words + lane];
  __syncwarp();

  // Hamming stage
  WarpList<S2> l2;
  l2.init();
  for (int t = 0; t < a.T; ++t) {
    const int64_t pos = a.pos[(size_t)t * a.nq + qi];
    const uint32_t* sig = a.sigma + (size_t)t * a.n;
    const int64_t c0 = pos - a.w > 0 ? pos - a.w : 0;
    const int64_t c1 = pos + a.w < a.n ? pos + a.w : a.n;
    for (int64_t cb = c0; cb < c1; cb += 32) {
      const int64_t c = cb + lane;
      uint32_t pid = c < c1 ? __ldg(sig + c) : 0xffffffffu;
      float hd = INFINITY;
      if (pid != 0xffffffffu) {
        const uint64_t* row = a.sk + (size_t)pid * a.words;
        int hm = 0;
        for (int u = 0; u < a.words; ++u) hm += __popcll(s_q[wib][u] ^ __ldg(row + u));
        hd = (float)hm;
      }
      warp_sort(hd, pid, lane);
      for (int u = 0; u < 32; ++u) {
        const float cd = __shfl_sync(FULL, hd, u);
        const uint32_t ci = __shfl_sync(FULL, pid, u);
        if (ci == 0xffffffffu) break;
        float kd;
        uint32_t ki;
        l2.last(a.k2, kd, ki);
        if (!lessp(cd, ci, kd, ki)) break;
        l2.insert(cd, ci, a.k2, lane);
      }
    }
  }
#pragma unroll
  for (int s2 = 0; s2 < S2; ++s2) s_c2[wib][32 * s2 + lane] = 32 * s2 + lane < a.k2 ? l2.iv[s2] : 0xffffffffu;
  __syncwarp();

  // expansion and final stage
  const float* qv = a.q + (size_t)qi * a.d;
  WarpList<S> list;
  list.init();
  const int span = 2 * a.h + 1;
  const int64_t E = (int64_t)a.k2 * span;
  for (int64_t eb = 0; eb < E; eb += 32) {
    const int64_t e = eb + lane;
    uint32_t pid = 0xffffffffu, row = 0;
    if (e < E) {
      const int u = (int)(e / span), o = (int)(e % span) - a.h;
      const uint32_t c = s_c2[wib][u];
      if (c != 0xffffffffu) {
        const int64_t p = (int64_t)__ldg(a.posm + c) + o;
        if (p >= 0 && p < a.n) {
          row = (uint32_t)p;
          pid = __ldg(a.sig0 + p);
        }
      }
    }
    float dist;
    if (a.vec4) {
      s_id[wib][lane] = pid;
      s_row[wib][lane] = row;
      __syncwarp();
      float part[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) part[u] = 0.f;
      for (int m = 4 * lane; m < a.d; m += 128) {
        const float4 qa = __ldg(reinterpret_cast<const float4*>(qv + m));
#pragma unroll
        for (int u0 = 0; u0 < 32; u0 += 16) {
          float4 xb[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            // an empty entry reads master row 0; its result is discarded
            xb[u] = __ldg(reinterpret_cast<const float4*>(a.xm + (size_t)s_row[wib][u0 + u] * a.d + m));
          }
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            float ee = qa.x - xb[u].x;
            float acc = fmaf(ee, ee, part[u0 + u]);
            ee = qa.y - xb[u].y;
            acc = fmaf(ee, ee, acc);
            ee = qa.z - xb[u].z;
            acc = fmaf(ee, ee, acc);
            ee = qa.w - xb[u].w;
            part[u0 + u] = fmaf(ee, ee, acc);
          }
        }
      }
      dist = warp_transpose_sum(part, lane);
      __syncwarp();
    } else {
      dist = 0.f;
      if (pid != 0xffffffffu) {
        const float* xv = a.xm + (size_t)row * a.d;
        for (int j = 0; j < a.d; ++j) {
          const float ee = __ldg(qv + j) - __ldg(xv + j);
          dist = fmaf(ee, ee, dist);
        }
      }
    }
    if (pid == 0xffffffffu) dist = INFINITY;
    warp_sort(dist, pid, lane);
    for (int u = 0; u < 32; ++u) {
      const float cd = __shfl_sync(FULL, dist, u);
      const uint32_t ci = __shfl_sync(FULL, pid, u);
      if (ci == 0xffffffffu) break;
      float kd;
      uint32_t ki;
      list.last(a.k, kd, ki);
      if (!lessp(cd, ci, kd, ki)) break;
      list.insert(cd, ci, a.k, lane);
    }
  }
#pragma unroll
  for (int s2 = 0; s2 < S; ++s2) {
    const int e = 32 * s2 + lane;
    if (e < a.k) {
      a.out_idx[(size_t)qi * a.k + e] = list.iv[s2];
      a.out_dist[(size_t)qi * a.k + e] = list.dv[s2];
    }
  }
}

// Master-ordered copy of the points and the inverse of the master order.
__global__ void master_layout_kernel(const float* __restrict__ x, int64_t n, int d, const uint32_t* __restrict__ sig0,
                                     float* __restrict__ xm, uint32_t* __restrict__ posm) {
  const int64_t total = n * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / d;
    const int j = (int)(e - p * d);
    const uint32_t id = __ldg(sig0 + p);
    xm[e] = __ldg(x + (size_t)id * d + j);
    if (j == 0) posm[id] = (uint32_t)p;
  }
}

// Exact k nearest neighbours of given rows among the points of their own set
// (the whole matrix when unsegmented), the row itself excluded: one warp per
// row, every point of the set scored 32 at a time with the search's float32
// exact-difference distance and merged into the warp-held list.
template <int S>
__global__ void __launch_bounds__(SWARPS * 32)
exact_rows_kernel(const float* __restrict__ x, int64_t n, int d, const int64_t* __restrict__ rows, int nrows,
                  const uint32_t* __restrict__ segr, const int64_t* __restrict__ segoff, int k, int vec4,
                  uint32_t* __restrict__ out_idx, float* __restrict__ out_dist) {
  __shared__ uint32_t s_id[SWARPS][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t wi = (int64_t)blockIdx.x * SWARPS + wib;
  if (wi >= nrows) return;
  const int64_t r = rows[wi];
  const float* qv = x + (size_t)r * d;
  int64_t lo = 0, hi = n;
  if (segr) {
    const uint32_t sg = __ldg(segr + r);
    lo = __ldg(segoff + sg);
    hi = __ldg(segoff + sg + 1);
  }
  WarpList<S> list;
  list.init();
  for (int64_t cb = lo; cb < hi; cb += 32) {
    const int64_t c = cb + lane;
    uint32_t pid = (c < hi && c != r) ? (uint32_t)c : 0xffffffffu;
    float dist;
    if (vec4) {
      s_id[wib][lane] = pid;
      __syncwarp();
      float part[32];
#pragma unroll
      for (int u = 0; u < 32; ++u) part[u] = 0.f;
      for (int m = 4 * lane; m < d; m += 128) {
        const float4 qa = __ldg(reinterpret_cast<const float4*>(qv + m));
#pragma unroll
        for (int u0 = 0; u0 < 32; u0 += 16) {
          float4 xb[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const uint32_t p = s_id[wib][u0 + u];
            const float* row = p != 0xffffffffu ? x + (size_t)p * d : qv;
            xb[u] = __ldg(reinterpret_cast<const float4*>(row + m));
          }
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            float e = qa.x - xb[u].x;
            float acc = fmaf(e, e, part[u0 + u]);
            e = qa.y - xb[u].y;
            acc = fmaf(e, e, acc);
            e = qa.z - xb[u].z;
            acc = fmaf(e, e, acc);
            e = qa.w - xb[u].w;
            part[u0 + u] = fmaf(e, e, acc);
          }
        }
      }
      dist = warp_transpose_sum(part, lane);
      __syncwarp();
    } else {
      dist = 0.f;
      if (pid != 0xffffffffu) {
        const float* xv = x + (size_t)pid * d;
        for (int j = 0; j < d; ++j) {
          const float e = __ldg(qv + j) - __ldg(xv + j);
          dist = fmaf(e, e, dist);
        }
      }
    }
    if (pid == 0xffffffffu) dist = INFINITY;
    warp_sort(dist, pid, lane);
    for (int u = 0; u < 32; ++u) {
      const float cd = __shfl_sync(FULL, dist, u);
      const uint32_t ci = __shfl_sync(FULL, pid, u);
      if (ci == 0xffffffffu) break;
      float kd;
      uint32_t ki;
      list.last(k, kd, ki);
      if (!lessp(cd, ci, kd, ki)) break;
      list.insert(cd, ci, k, lane);
    }
  }
#pragma unroll
  for (int s2 = 0; s2 < S; ++s2) {
    const int e = 32 * s2 + lane;
    if (e < k) {
      out_idx[(size_t)wi * k + e] = list.iv[s2];
      out_dist[(size_t)wi * k + e] = list.dv[s2];
    }
  }
}

// out[j][c] = lists[rows[j]][c] for c < k (lists have kp slots per row).
__global__ void gather_list_rows_kernel(const uint32_t* __restrict__ lists, int kp, const int64_t* __restrict__ rows,
                                        int nrows, int k, uint32_t* __restrict__ out) {
  const int64_t total = (int64_t)nrows * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / k;
    out[e] = lists[(size_t)rows[j] * kp + (e - j * k)];
  }
}

template <int S2, int S>
int launch_ss(const SketchSearchArgs& a, cudaStream_t s) {
  sketch_search_kernel<S2, S><<<hf_blocks(a.nq, SWARPS), SWARPS * 32, 0, s>>>(a);
  hf_after_launch("sketch_search_kernel", s);
  return HF_OK;
}

template <int S>
int launch_ss_k2(const SketchSearchArgs& a, cudaStream_t s) {
  if (a.k2 <= 32) return launch_ss<1, S>(a, s);
  if (a.k2 <= 64) return launch_ss<2, S>(a, s);
  if (a.k2 <= 128) return launch_ss<4, S>(a, s);
  if (a.k2 <= 256) return launch_ss<8, S>(a, s);
  if (a.k2 <= 512) return launch_ss<16, S>(a, s);
  return launch_ss<32, S>(a, s);
}

}  // namespace

int launch_exact_rows(const hf_forest* f, const int64_t* rows, int nrows, int k, uint32_t* out_idx, float* out_dist,
                      cudaStream_t s) {
  if (k < 1 || k > 64 || nrows < 1) return HF_EINVAL;
  const int vec4 = f->d % 4 == 0 && (reinterpret_cast<uintptr_t>(f->x) & 15) == 0;
  const uint32_t* segr = f->nseg > 1 ? f->seg : nullptr;
  const int64_t* segoff = f->nseg > 1 ? f->seg_off : nullptr;
  if (k <= 32)
    exact_rows_kernel<1><<<hf_blocks(nrows, SWARPS), SWARPS * 32, 0, s>>>(f->x, f->n, f->d, rows, nrows, segr, segoff,
                                                                          k, vec4, out_idx, out_dist);
  else
    exact_rows_kernel<2><<<hf_blocks(nrows, SWARPS), SWARPS * 32, 0, s>>>(f->x, f->n, f->d, rows, nrows, segr, segoff,
                                                                          k, vec4, out_idx, out_dist);
  hf_after_launch("exact_rows_kernel", s);
  return HF_OK;
}

void launch_gather_list_rows(const uint32_t* lists, int kp, const int64_t* rows, int nrows, int k, uint32_t* out,
                             cudaStream_t s) {
  gather_list_rows_kernel<<<hf_blocks((int64_t)nrows * k, 256, 152 * 4), 256, 0, s>>>(lists, kp, rows, nrows, k, out);
  hf_after_launch("gather_list_rows_kernel", s);
}

void launch_master_layout(const float* x, int64_t n, int d, const uint32_t* sig0, float* xm, uint32_t* posm,
                          cudaStream_t s) {
  master_layout_kernel<<<hf_blocks(n * d, 256, 152 * 16), 256, 0, s>>>(x, n, d, sig0, xm, posm);
  hf_after_launch("master_layout_kernel", s);
}

int launch_sketch_search(const hf_forest* f, const float* q, int64_t nq, const int64_t* pos, const uint64_t* qsk,
                         int k, int w, int k2, int h, uint32_t* out_idx, float* out_dist, cudaStream_t s) {
  if (k < 1 || k > 64 || k2 < 1 || k2 > HF_MAX_K2 || h < 0 || !f->sketch || !f->xm || !f->posm) return HF_EINVAL;
  const int words = f->sketch_bits / 64;
  if (words < 1 || words > SK_MAX_WORDS) return HF_EINVAL;
  SketchSearchArgs a;
  a.q = q;
  a.nq = nq;
  a.d = f->d;
  a.xm = f->xm;
  a.sig0 = f->sigma;
  a.posm = f->posm;
  a.sigma = f->sigma;
  a.pos = pos;
  a.sk = f->sketch;
  a.qsk = qsk;
  a.words = words;
  a.n = f->n;
  a.T = f->T;
  a.w = w;
  a.k2 = k2;
  a.h = h;
  a.k = k;
  a.out_idx = out_idx;
  a.out_dist = out_dist;
  a.vec4 = (f->d % 4 == 0) && ((reinterpret_cast<uintptr_t>(f->xm) & 15) == 0) &&
           ((reinterpret_cast<uintptr_t>(q) & 15) == 0);
  return k <= 32 ? launch_ss_k2<1>(a, s) : launch_ss_k2<2>(a, s);
}

// ---------------------------------------------------------------------------
// Allocation-free search.
//
// hf_search allocates a device buffer for the queries' quantized codes on
// every call. Some callers cannot allocate device memory while they run: a
// serving process that holds a fixed memory budget carved out up front, a
// host runtime that owns all device memory through its own pool, or a worker
// that must not take the allocator's locks on its latency path. For them,
// hf_search_static keeps that scratch in a fixed array that lives in this
// library's device image: every GPU that loads the library holds
// HF_STATIC_QUERY_BYTES of it until the process exits.
//
// The array's host-side name is only a stand-in for the device symbol, so the
// host looks up its device address with cudaGetSymbolAddress, once per
// device, with that device current, and passes that address to the kernels.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

__device__ __align__(256) uint8_t g_static_qcodes[HF_STATIC_QUERY_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
uint8_t* g_static_addr[kMaxDevices] = {};

// Device address of g_static_qcodes on the current device (looked up on the
// first call per device).
int static_qcodes_address(uint8_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return HF_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_qcodes) != cudaSuccess || !p) {
      cudaGetLastError();
      return HF_ECUDA;
    }
    g_static_addr[dev] = static_cast<uint8_t*>(p);
  }
  *out = g_static_addr[dev];
  return HF_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int hf_search_static(hf_forest* f, const float* queries, int64_t nq, int32_t k, int32_t w,
                                int32_t* out_idx, float* out_dist, void* stream) {
  if (!f || nq < 0 || k < 1 || k > HF_MAX_K || w < 1) return HF_EINVAL;
  if (f->mode == 3) return HF_ENOTIMPL;  // the sketch form needs per-call scratch
  if (f->nseg > 1) return HF_ENOTIMPL;   // segmented orders carry no search prefixes
  if (nq == 0) return HF_OK;
  if (!queries || !out_idx || !out_dist) return HF_EINVAL;
  if ((uint64_t)nq * (uint64_t)f->d > (uint64_t)HF_STATIC_QUERY_BYTES) return HF_EINVAL;
  if (!on_device(queries) || !on_device(out_idx) || !on_device(out_dist)) return HF_EINVAL;
  uint8_t* qc = nullptr;
  int rc = static_qcodes_address(&qc);
  if (rc != HF_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();  // an earlier call's error was reported by that call
  launch_quantize_codes(queries, nq, f->d, f->lo, f->scale, f->bits, qc, f->err, s);
  rc = launch_search(f, queries, qc, nq, k, w, reinterpret_cast<uint32_t*>(out_idx), out_dist, nullptr, -1, s);
  // the same synchronisation and status mapping as every other entry point
  const int rc2 = hf_finish(f, s);
  return rc != HF_OK ? rc : rc2;
}
