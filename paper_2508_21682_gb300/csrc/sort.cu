// Hilbert sort: stable LSD radix sort of the K-word key prefixes, then the
// fix-up that orders runs of equal prefixes by full key.
//
// Paper, Section 2: the Hilbert order is a total order over the points; the
// paper sorts with a key-free CPU algorithm whose details it does not give.
// Here the order is "ascending (full key, point index)": the prefix words are
// sorted with 8-bit digits, least significant first; each pass is one
// single-pass binning kernel with decoupled look-back (Merrill & Garland 2016;
// Adinets & Merrill 2022, "Onesweep"). The input starts in point order, so
// equal prefixes stay in index order; the fix-up then reorders each run of
// equal prefixes by its full keys.
//
// The trees of a batch are sorted together: one launch per pass covers every
// tree, and tile tickets interleave the trees (ticket g is tile g / TB of tree
// g % TB), so the tiles in flight at any time are spread over all trees and
// each tree's look-back chain stays short.
//
// The look-back is the only wait between blocks. Tiles take tickets from an
// atomic counter, so a tile only ever waits for tiles that started before it;
// each wait is bounded by a %globaltimer deadline, after which the tile sets
// the error word (HF_ETIMEOUT), publishes a value and finishes.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "hf_internal.cuh"
#include "hilbert_device.cuh"

namespace {

constexpr int NT = 256;
constexpr int IPT = 8;
constexpr int TILE = NT * IPT;  // 2048 keys per tile
constexpr int WARPS = NT / 32;
constexpr uint32_t FLAG_AGG = 1u << 30;
constexpr uint32_t FLAG_PRE = 2u << 30;
constexpr uint32_t VAL_MASK = (1u << 30) - 1u;
constexpr int LB = 16;  // predecessor status words read per look-back round

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Digit histograms of all 8 bytes of all K prefix words (order-independent).
// Tree blockIdx.y: keys at pk + y * pk_ts, histograms at hist + y * K * 8 * 256.
__global__ void digit_hist_kernel(const uint64_t* __restrict__ pk, int64_t pk_ts, int64_t n, int K,
                                  uint32_t* __restrict__ hist) {
  extern __shared__ uint32_t sh[];  // [K*8][256]
  pk += blockIdx.y * pk_ts;
  hist += (size_t)blockIdx.y * K * 8 * 256;
  const int nh = K * 8 * 256;
  for (int i = threadIdx.x; i < nh; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    for (int w = 0; w < K; ++w) {
      const uint64_t key = __ldg(pk + (size_t)w * n + e);
#pragma unroll
      for (int b = 0; b < 8; ++b) atomicAdd(&sh[(w * 8 + b) * 256 + ((key >> (8 * b)) & 255)], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nh; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Exclusive scan of each 256-bin histogram (one block per histogram).
__global__ void hist_scan_kernel(uint32_t* __restrict__ hist) {
  __shared__ uint32_t s[256];
  uint32_t* h = hist + blockIdx.x * 256;
  s[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int i = 0; i < 256; ++i) {
      const uint32_t c = s[i];
      s[i] = run;
      run += c;
    }
  }
  __syncthreads();
  h[threadIdx.x] = s[threadIdx.x];
}

struct PassSmem {
  uint64_t keys[TILE];
  uint32_t vals[TILE];
  uint32_t whist[WARPS][256];
  uint32_t tile_start[256];
  uint32_t gbase[256];
  uint32_t scan[WARPS];
  uint32_t tile;
};

// One pass over the trees of a batch. Each array is given as the first
// tree's pointer plus the element stride between trees.
struct PassArgs {
  const uint64_t* keys_in;
  int64_t keys_in_ts;
  const uint32_t* vals_in;  // null: identity (first pass)
  int64_t vals_in_ts;
  const uint64_t* gather_src;
  int64_t gather_src_ts;
  uint64_t* keys_out;
  int64_t keys_out_ts;
  uint32_t* vals_out;
  int64_t vals_out_ts;
  const uint32_t* goff;  // exclusive digit offsets of this pass
  int64_t goff_ts;
  uint32_t* status;      // [TB][ntiles + 1][256]
  uint32_t* ticket;
  int* err;
  int64_t n, ntiles;
  uint64_t spin_ns;
  int shift, TB, stall;
};

// One LSD pass: bins the keys of one tile by `digit = key >> shift & 255`.
// GATHER: the key of the element at position e is gather_src[vals_in[e]]
// (the next prefix word, fetched in the current order).
template <bool GATHER>
__global__ void __launch_bounds__(NT, 5) onesweep_kernel(const PassArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  PassSmem& S = *reinterpret_cast<PassSmem*>(smraw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) S.tile = atomicAdd(a.ticket, 1u);
  for (int i = tid; i < WARPS * 256; i += NT) (&S.whist[0][0])[i] = 0;
  __syncthreads();
  const int64_t tr = S.tile % (uint32_t)a.TB;
  const int64_t tile = S.tile / (uint32_t)a.TB;
  const int64_t n = a.n, ntiles = a.ntiles;
  const int shift = a.shift;
  const uint64_t* __restrict__ keys_in = GATHER ? nullptr : a.keys_in + tr * a.keys_in_ts;
  const uint32_t* __restrict__ vals_in = a.vals_in ? a.vals_in + tr * a.vals_in_ts : nullptr;
  const uint64_t* __restrict__ gather_src = GATHER ? a.gather_src + tr * a.gather_src_ts : nullptr;
  uint64_t* __restrict__ keys_out = a.keys_out + tr * a.keys_out_ts;
  uint32_t* __restrict__ vals_out = a.vals_out + tr * a.vals_out_ts;
  const uint32_t* __restrict__ goff = a.goff + tr * a.goff_ts;
  uint32_t* __restrict__ status = a.status + (size_t)tr * (ntiles + 1) * 256;
  int* err = a.err;
  const int64_t base = tile * TILE;

  uint64_t k[IPT];
  uint32_t v[IPT];
  uint32_t rk[IPT];
  uint32_t dg[IPT];
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const int64_t e = base + warp * 32 * IPT + j * 32 + lane;
    if (e < n) {
      // read once per pass: streaming loads leave L2 to the pass's output
      v[j] = vals_in ? __ldcs(vals_in + e) : (uint32_t)e;
      if (GATHER) {
        // values are point indices < n unless an earlier pass gave up its
        // look-back (error word set); never read outside the source then
        if (v[j] >= (uint64_t)n) {
          hf_raise(err, HF_ERRBIT_TIMEOUT);
          v[j] = 0;
        }
        k[j] = __ldg(gather_src + v[j]);
      } else {
        k[j] = __ldcs(reinterpret_cast<const unsigned long long*>(keys_in) + e);
      }
      dg[j] = (uint32_t)(k[j] >> shift) & 255u;
    } else {
      v[j] = 0;
      k[j] = 0;
      dg[j] = 256u;  // sentinel: no element
    }
  }
  // Stable ranking within the warp: items are ordered by (j, lane).
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    const uint32_t peers = __match_any_sync(0xffffffffu, dg[j]);
    const uint32_t before = __popc(peers & lt);
    uint32_t basec = 0;
    if (dg[j] < 256u) basec = S.whist[warp][dg[j]];
    __syncwarp();
    if (dg[j] < 256u && before == 0) S.whist[warp][dg[j]] = basec + __popc(peers);
    __syncwarp();
    rk[j] = basec + before;
  }
  __syncthreads();

  // Per digit: exclusive offsets across warps and the tile's count.
  const int dgt = tid;  // NT == 256 == radix
  uint32_t cnt = 0;
#pragma unroll
  for (int w = 0; w < WARPS; ++w) {
    const uint32_t c = S.whist[w][dgt];
    S.whist[w][dgt] = cnt;
    cnt += c;
  }

  // The tile's counts are published first (its successors can use them at
  // once); the tile-local offsets and the scatter into shared memory run
  // before this tile waits for its own predecessors.
  uint32_t* st = status + tile * 256 + dgt;
  st_relaxed(st, (tile == 0 ? FLAG_PRE : FLAG_AGG) | cnt);

  // Tile-local exclusive scan of the digit counts (warp scans + warp totals),
  // folded into the per-warp offsets.
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) S.scan[warp] = incl;
  __syncthreads();
  uint32_t woff = 0;
#pragma unroll
  for (int w = 0; w < WARPS; ++w)
    if (w < warp) woff += S.scan[w];
  const uint32_t tstart = woff + incl - cnt;
  S.tile_start[dgt] = tstart;
#pragma unroll
  for (int w = 0; w < WARPS; ++w) S.whist[w][dgt] += tstart;
  __syncthreads();

  // Scatter into shared memory in digit order.
#pragma unroll
  for (int j = 0; j < IPT; ++j) {
    if (dg[j] < 256u) {
      const uint32_t lp = S.whist[warp][dg[j]] + rk[j];
      S.keys[lp] = k[j];
      S.vals[lp] = v[j];
    }
  }

  // Decoupled look-back for this digit. LB predecessor status words are read
  // at once (independent loads, one round trip), then consumed in order:
  // aggregates are added until an inclusive prefix ends the walk; a word that
  // is not ready yet is re-read from there on the next round.
  uint32_t excl = 0;
  if (tile > 0) {
    int64_t pred = tile - 1;
    const uint64_t t0 = globaltimer();
    uint32_t spins = 0;
    for (;;) {
      uint32_t sv[LB];
#pragma unroll
      for (int i = 0; i < LB; ++i) {
        // test hook: tile 1 watches the spare status row that nothing writes
        const int64_t pt = pred - i;
        const uint32_t* ps = (a.stall && tr == 0 && tile == 1) ? status + ntiles * 256 + dgt : status + pt * 256 + dgt;
        sv[i] = pt >= 0 ? ld_relaxed(ps) : FLAG_PRE;  // before tile 0: prefix 0
      }
      int used = 0;
      bool done = false;
#pragma unroll
      for (int i = 0; i < LB; ++i) {
        if (used != i) break;  // stopped at an earlier word
        const uint32_t flag = sv[i] & ~VAL_MASK;
        if (flag == 0) break;
        excl += sv[i] & VAL_MASK;
        ++used;
        if (flag == FLAG_PRE) {
          done = true;
          break;
        }
      }
      if (done) break;
      pred -= used;
      if (used == 0 && (++spins & 15u) == 0 && (globaltimer() - t0 > a.spin_ns || spins > (1u << 28))) {
        hf_raise(err, HF_ERRBIT_TIMEOUT);
        break;
      }
    }
    st_relaxed(st, FLAG_PRE | ((excl + cnt) & VAL_MASK));
  }
  S.gbase[dgt] = goff[dgt] + excl;
  __syncthreads();

  // Write out coalesced (runs of equal digits go to consecutive positions).
  const int valid = (int)(n - base < TILE ? n - base : TILE);
  for (int e = tid; e < valid; e += NT) {
    const uint64_t key = S.keys[e];
    const uint32_t dgi = (uint32_t)(key >> shift) & 255u;
    const uint32_t pos = S.gbase[dgi] + (uint32_t)e - S.tile_start[dgi];
    keys_out[pos] = key;
    vals_out[pos] = S.vals[e];
  }
}

// Sorted prefix words 1..K-1: out[w][p] = pk[w][sigma[p]].
__global__ void gather_prefix_kernel(const uint64_t* __restrict__ pk, const uint32_t* __restrict__ sigma,
                                     int64_t n, int K, uint64_t* __restrict__ out,
                                     const int* __restrict__ err) {
  if (*(volatile const int*)err) return;  // the order is not valid: skip
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = sigma[p];
    if (i >= (uint64_t)n) continue;
    for (int w = 1; w < K; ++w) out[(size_t)w * n + p] = __ldg(pk + (size_t)w * n + i);
  }
}

__device__ __forceinline__ bool prefix_eq(const uint64_t* __restrict__ pre, int64_t n, int K,
                                          int64_t a, int64_t b) {
  for (int w = 0; w < K; ++w)
    if (pre[(size_t)w * n + a] != pre[(size_t)w * n + b]) return false;
  return true;
}

// Finds maximal runs of >= 2 equal prefixes. Small runs go to `runs`, runs
// longer than small_cap to `big`.
__global__ void tie_find_kernel(const uint64_t* __restrict__ pre, int64_t n, int K, int small_cap,
                                uint2* __restrict__ runs, uint2* __restrict__ big, int64_t big_cap,
                                uint32_t* __restrict__ counters) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m + 1 < n;
       m += (int64_t)gridDim.x * blockDim.x) {
    if (!prefix_eq(pre, n, K, m, m + 1)) continue;
    if (m > 0 && prefix_eq(pre, n, K, m - 1, m)) continue;
    int64_t len = 2;
    while (m + len < n && prefix_eq(pre, n, K, m, m + len)) ++len;
    if (len <= small_cap) {
      const uint32_t r = atomicAdd(&counters[0], 1u);
      runs[r] = make_uint2((uint32_t)m, (uint32_t)len);
    } else {
      const uint32_t r = atomicAdd(&counters[1], 1u);
      if (r < big_cap) big[r] = make_uint2((uint32_t)m, (uint32_t)len);
      atomicAdd(&counters[2], (uint32_t)len);
    }
  }
}


__device__ __forceinline__ bool full_less(const uint64_t* a, uint32_t ia, const uint64_t* b,
                                          uint32_t ib, int W) {
  for (int w = 0; w < W; ++w)
    if (a[w] != b[w]) return a[w] < b[w];
  return ia < ib;
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

// One block per small run (grid-stride over runs). The run's prefixes (words
// 0..K-1) are equal, so the order inside it is decided by the following key
// words K..K2-1. When the key kernel computed them (kpre > K) they are read
// from pkx[w][point]; otherwise they are computed here: they lie in the top
// Lf bit levels, and the top Lf levels of a key equal the Lf-bit key of the
// coordinates' top Lf bits, so they cost a transform with Lf levels only
// (with Lf = 1 a running XOR, which a warp forms with ballots).
// Each point's rank = number of run members below it by (words K..K2-1,
// index). Only if two members also tie on those words does the block compute
// full keys (into its own slice of global scratch) and rank by (full key,
// index). Shared layout: tk[cap][K2-K], pt[cap], rank[cap], Y[blockDim][d].
__global__ void tie_small_kernel(const uint32_t* __restrict__ planes, int64_t n, int d, int W32,
                                 int bits, int W, int K, int K2, int Lf, int cap,
                                 const uint64_t* __restrict__ pkx, int kpre,
                                 const int32_t* __restrict__ pi, const uint32_t* __restrict__ rbits,
                                 const uint2* __restrict__ runs, const uint32_t* __restrict__ counters,
                                 uint32_t* __restrict__ sigma, uint64_t* __restrict__ fk_scratch,
                                 const int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_tie;
  if (*(volatile const int*)err) return;  // the order is not valid: skip
  const int KT = K2 - K;
  uint64_t* tk = reinterpret_cast<uint64_t*>(smraw);
  uint32_t* pt = reinterpret_cast<uint32_t*>(tk + (size_t)cap * KT);
  uint32_t* rank = pt + cap;
  uint8_t* Y = reinterpret_cast<uint8_t*>(rank + cap) + (size_t)threadIdx.x * d;
  uint64_t* fk = fk_scratch + (size_t)blockIdx.x * cap * W;
  const uint32_t nruns = counters[0];
  for (uint32_t r = blockIdx.x; r < nruns; r += gridDim.x) {
    const uint2 run = runs[r];
    const int len = (int)run.y;  // <= cap by construction
    if (threadIdx.x == 0) s_tie = 0;
    if (kpre <= K && Lf == 1) {
      // Words K .. K2-1 lie in the top bit level: one warp per member forms
      // them with ballots over the permuted, reflected top bits (plane 0),
      // carrying the parity of the first 64K bits.
      const int lane = threadIdx.x & 31;
      for (int e = threadIdx.x >> 5; e < len; e += blockDim.x >> 5) {
        const uint32_t p = sigma[run.x + e];
        if (lane == 0) pt[e] = p;
        if (p >= (uint64_t)n) continue;  // cannot happen for a valid order
        const uint32_t* row = planes + (size_t)p * W32;
        uint32_t carry = 0, hi = 0;
        for (int h = 0; h < 2 * K2; ++h) {
          const int c = __ldg(pi + 32 * h + lane);
          const uint32_t bit = ((__ldg(row + (c >> 5)) >> (c & 31)) ^ (__ldg(rbits + h) >> lane)) & 1u;
          const uint32_t bal = __ballot_sync(0xffffffffu, bit);
          if (h < 2 * K) {
            carry ^= __popc(bal) & 1u;
            continue;
          }
          uint32_t v = xor_scan_msb(__brev(bal));
          if (carry) v = ~v;
          carry = v & 1u;
          if (h & 1) {
            if (lane == 0) tk[(size_t)e * KT + (h >> 1) - K] = ((uint64_t)hi << 32) | v;
          } else {
            hi = v;
          }
        }
      }
    } else {
      for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const uint32_t p = sigma[run.x + e];
        pt[e] = p;
        if (p >= (uint64_t)n) continue;  // cannot happen for a valid order
        if (kpre > K) {
          for (int w = 0; w < KT; ++w) tk[(size_t)e * KT + w] = __ldg(pkx + (size_t)(K + w) * n + p);
        } else {
          hf_load_coords_planes(planes, n, d, W32, Lf, pi, rbits, p, Y);
          hf_skilling(Y, d, Lf);
          for (int w = 0; w < KT; ++w) tk[(size_t)e * KT + w] = hf_pack_word(Y, d, Lf, K + w);
        }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < len; e += blockDim.x) {
      uint32_t rk = 0;
      bool tie = false;
      for (int g = 0; g < len; ++g) {
        int c = 0;
        for (int w = 0; w < KT && c == 0; ++w) {
          const uint64_t a = tk[(size_t)g * KT + w], b = tk[(size_t)e * KT + w];
          c = a < b ? -1 : (a > b ? 1 : 0);
        }
        if (c == 0 && g != e) tie = true;
        rk += (c < 0 || (c == 0 && pt[g] < pt[e])) ? 1u : 0u;
      }
      rank[e] = rk;
      if (tie) s_tie = 1;
    }
    __syncthreads();
    if (s_tie && K2 < W) {
      // rare: the next words tie as well, rank by full keys
      for (int e = threadIdx.x; e < len; e += blockDim.x) {
        const uint32_t p = pt[e];
        if (p >= (uint64_t)n) continue;
        hf_load_coords_planes(planes, n, d, W32, bits, pi, rbits, p, Y);
        hf_skilling(Y, d, bits);
        for (int w = 0; w < W; ++w) fk[(size_t)e * W + w] = hf_pack_word(Y, d, bits, w);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < len; e += blockDim.x) {
        uint32_t rk = 0;
        for (int g = 0; g < len; ++g)
          rk += full_less(fk + (size_t)g * W, pt[g], fk + (size_t)e * W, pt[e], W) ? 1u : 0u;
        rank[e] = rk;
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < len; e += blockDim.x) sigma[run.x + rank[e]] = pt[e];
    __syncthreads();
  }
}

// Big runs: full keys into global scratch, then a bitonic network over all
// big-run elements of one tree ordered by (run, full key, point).
__global__ void big_fill_kernel(const uint32_t* __restrict__ planes, int64_t n, int d, int W32,
                                int bits, int W, const int32_t* __restrict__ pi,
                                const uint32_t* __restrict__ rbits, const uint2* __restrict__ big,
                                const uint32_t* __restrict__ offs, int nbig,
                                const uint32_t* __restrict__ sigma, uint64_t* __restrict__ fk,
                                uint32_t* __restrict__ item_pt, uint32_t* __restrict__ item_run,
                                uint8_t* __restrict__ yscratch) {
  const int r = blockIdx.x;
  if (r >= nbig) return;
  const uint2 run = big[r];
  uint8_t* y = yscratch + ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * d;
  for (uint32_t e = threadIdx.x; e < run.y; e += blockDim.x) {
    const uint32_t slot = offs[r] + e;
    const uint32_t p = sigma[run.x + e];
    item_pt[slot] = p;
    item_run[slot] = (uint32_t)r;
    hf_load_coords_planes(planes, n, d, W32, bits, pi, rbits, p, y);
    hf_skilling(y, d, bits);
    for (int w = 0; w < W; ++w) fk[(size_t)slot * W + w] = hf_pack_word(y, d, bits, w);
  }
}

__device__ __forceinline__ bool item_less(uint32_t a, uint32_t b, const uint64_t* fk,
                                          const uint32_t* pt, const uint32_t* rn, int W,
                                          uint32_t total) {
  const bool va = a < total, vb = b < total;
  if (va != vb) return va;  // padding sorts last
  if (!va) return false;
  if (rn[a] != rn[b]) return rn[a] < rn[b];
  return full_less(fk + (size_t)a * W, pt[a], fk + (size_t)b * W, pt[b], W);
}

__global__ void bitonic_step_kernel(uint32_t* __restrict__ ord, uint32_t m, uint32_t j, uint32_t kk,
                                    const uint64_t* __restrict__ fk, const uint32_t* __restrict__ pt,
                                    const uint32_t* __restrict__ rn, int W, uint32_t total) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint32_t l = i ^ j;
  if (l <= i) return;
  const uint32_t a = ord[i], b = ord[l];
  const bool up = (i & kk) == 0;
  const bool sw = up ? item_less(b, a, fk, pt, rn, W, total) : item_less(a, b, fk, pt, rn, W, total);
  if (sw) {
    ord[i] = b;
    ord[l] = a;
  }
}

__global__ void big_write_kernel(const uint32_t* __restrict__ ord, uint32_t total,
                                 const uint32_t* __restrict__ pt, const uint32_t* __restrict__ rn,
                                 const uint2* __restrict__ big, const uint32_t* __restrict__ offs,
                                 uint32_t* __restrict__ sigma) {
  const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= total) return;
  const uint32_t it = ord[s];
  const uint32_t r = rn[it];
  sigma[big[r].x + (s - offs[r])] = pt[it];
}

__global__ void iota_kernel(uint32_t* a, uint32_t m) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) a[i] = i;
}

constexpr int TIE_THREADS = 64;
constexpr int TIE_BLOCKS = 152 * 2;

struct TieGeom {
  int K2, Lf, cap;
  size_t smem;
};

// Words K..K2-1 (up to four) break ties; they lie in the top Lf levels.
// With kpre > K the key kernel already computed words K..kpre-1.
TieGeom tie_geom(int W, int d, int bits, int K, int kpre) {
  TieGeom g;
  g.K2 = kpre > K ? kpre : (K + 4 < W ? K + 4 : W);
  const int64_t lf = ((int64_t)64 * g.K2 + d - 1) / d;
  g.Lf = (int)(lf < bits ? lf : bits);
  const int KT = g.K2 - K;
  const size_t y = (size_t)TIE_THREADS * d;
  const size_t per = (size_t)KT * 8 + 8;
  size_t cap = (96 * 1024 - (y < 96 * 1024 ? y : 96 * 1024)) / per;
  if (cap > 256) cap = 256;
  if (cap < 2) cap = 2;
  g.cap = (int)cap;
  g.smem = (size_t)g.cap * per + y;
  return g;
}

}  // namespace

static cudaError_t set_attr(const void* fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Sorts trees t0 .. t0 + tb - 1 (their key words are at f->pk, tree j of the
// batch at f->pk + j * K2 * n) into f->prefix / f->sigma, then fixes each
// tree's runs of equal prefixes.
int sort_batch(hf_forest* f, int t0, int tb, cudaStream_t s) {
  const int64_t n = f->n;
  const int K = f->K, K2 = f->K2;
  const int64_t ntiles = (n + TILE - 1) / TILE;
  const int passes = 8 * K;
  const size_t per_pass = (size_t)tb * (ntiles + 1) * 256 + 1;  // status rows (+ spare row per tree) + ticket
  const int64_t pk_ts = (int64_t)K2 * n;
  const int64_t hist_ts = (int64_t)K * 8 * 256;
  uint32_t* status = f->sort.status;

  cudaMemsetAsync(f->sort.hist, 0, (size_t)tb * hist_ts * sizeof(uint32_t), s);
  cudaMemsetAsync(status, 0, per_pass * passes * sizeof(uint32_t), s);
  const size_t hsm = (size_t)hist_ts * sizeof(uint32_t);
  set_attr((const void*)digit_hist_kernel, hsm);
  digit_hist_kernel<<<dim3(hf_blocks(n, 512, 152 * 8 / tb + 1), (unsigned)tb), 512, hsm, s>>>(f->pk, pk_ts, n, K,
                                                                                            f->sort.hist);
  hf_after_launch("digit_hist_kernel", s);
  hist_scan_kernel<<<(unsigned)(tb * K * 8), 256, 0, s>>>(f->sort.hist);
  hf_after_launch("hist_scan_kernel", s);

  const size_t psm = sizeof(PassSmem);
  set_attr((const void*)onesweep_kernel<false>, psm);
  set_attr((const void*)onesweep_kernel<true>, psm);

  PassArgs a{};
  a.err = f->err;
  a.n = n;
  a.ntiles = ntiles;
  a.spin_ns = (uint64_t)f->spin_limit_us * 1000ull;
  a.TB = tb;
  a.goff_ts = hist_ts;
  a.gather_src_ts = pk_ts;
  const unsigned grid = (unsigned)(ntiles * tb);
  int pass = 0;
  for (int w = K - 1; w >= 0; --w) {
    for (int b = 0; b < 8; ++b, ++pass) {
      const bool gather = (w < K - 1) && b == 0;
      const bool last = pass == passes - 1;
      if (pass == 0) {
        a.keys_in = f->pk + (size_t)(K - 1) * n;
        a.keys_in_ts = pk_ts;
        a.vals_in = nullptr;
        a.vals_in_ts = 0;
      }
      a.gather_src = gather ? f->pk + (size_t)w * n : nullptr;
      if (last) {
        a.keys_out = f->prefix + (size_t)t0 * K * n;  // word 0 of each tree's prefix
        a.keys_out_ts = (int64_t)K * n;
        a.vals_out = f->sigma + (size_t)t0 * n;
        a.vals_out_ts = n;
      } else {
        a.keys_out = (pass & 1) ? f->sort.keys_b : f->sort.keys_a;
        a.keys_out_ts = n;
        a.vals_out = (pass & 1) ? f->sort.vals_b : f->sort.vals_a;
        a.vals_out_ts = n;
      }
      a.goff = f->sort.hist + (size_t)(w * 8 + b) * 256;
      a.status = status + per_pass * pass;
      a.ticket = a.status + (size_t)tb * (ntiles + 1) * 256;
      a.shift = 8 * b;
      a.stall = (f->test_stall && pass == 0) ? 1 : 0;
      if (gather)
        onesweep_kernel<true><<<grid, NT, psm, s>>>(a);
      else
        onesweep_kernel<false><<<grid, NT, psm, s>>>(a);
      hf_after_launch("onesweep_kernel", s);
      a.keys_in = a.keys_out;
      a.keys_in_ts = a.keys_out_ts;
      a.vals_in = a.vals_out;
      a.vals_in_ts = a.vals_out_ts;
    }
  }
  for (int j = 0; j < tb; ++j) {
    const int t = t0 + j;
    const uint64_t* pkt = f->pk + (size_t)j * pk_ts;
    uint64_t* pre = f->prefix + (size_t)t * K * n;
    uint32_t* sig = f->sigma + (size_t)t * n;
    if (K > 1) {
      gather_prefix_kernel<<<hf_blocks(n, 256, 152 * 8), 256, 0, s>>>(pkt, sig, n, K, pre, f->err);
      hf_after_launch("gather_prefix_kernel", s);
    }
    // Equal prefixes: find runs, fix the small ones on the device right
    // away. With K == W the prefix is the whole key: equal prefixes are equal
    // keys, already in index order.
    if (K < f->W) {
      const TieGeom tg = tie_geom(f->W, f->d, f->bits, K, K2);
      uint32_t* ctr = f->tie.counters + (size_t)t * 4;
      cudaMemsetAsync(ctr, 0, 4 * sizeof(uint32_t), s);
      tie_find_kernel<<<hf_blocks(n, 256, 152 * 8), 256, 0, s>>>(pre, n, K, tg.cap, f->tie.runs,
                                                                f->tie.big_runs + (size_t)t * f->tie.big_cap,
                                                                f->tie.big_cap, ctr);
      hf_after_launch("tie_find_kernel", s);
      set_attr((const void*)tie_small_kernel, tg.smem);
      tie_small_kernel<<<TIE_BLOCKS, TIE_THREADS, tg.smem, s>>>(
          f->planes, n, f->d, f->W32, f->bits, f->W, K, tg.K2, tg.Lf, tg.cap, pkt, K2, f->pi + (size_t)t * f->d,
          f->rbits + (size_t)t * f->W32, f->tie.runs, ctr, sig, f->tie.fk, f->err);
      hf_after_launch("tie_small_kernel", s);
    }
  }
  return cudaGetLastError() == cudaSuccess ? HF_OK : HF_ECUDA;
}

// Segmented forest: one more stable LSD pass per tree, keyed by the set of
// each point (the most significant digit of the order), gathered through the
// current order. Equal sets keep their relative order, so every set's points
// stay in their own Hilbert order and set s occupies positions off[s] ..
// off[s+1]-1. Up to 256 sets (one 8-bit digit).
int segment_pass(hf_forest* f, const uint64_t* seg64, cudaStream_t s) {
  const int64_t n = f->n;
  const int nseg = f->nseg;
  if (nseg < 2 || nseg > 256) return HF_EINVAL;
  const int64_t ntiles = (n + TILE - 1) / TILE;
  std::vector<uint32_t> goff(256, (uint32_t)n);
  for (int g = 0; g < nseg; ++g) goff[g] = (uint32_t)f->seg_off_h[g];
  if (cudaMemcpyAsync(f->sort.hist, goff.data(), 256 * sizeof(uint32_t), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return HF_ECUDA;
  const size_t psm = sizeof(PassSmem);
  set_attr((const void*)onesweep_kernel<true>, psm);
  for (int t0 = 0; t0 < f->T; t0 += f->TB) {
    const int tb = f->T - t0 < f->TB ? f->T - t0 : f->TB;
    const size_t words = (size_t)tb * (ntiles + 1) * 256 + 1;
    cudaMemsetAsync(f->sort.status, 0, words * sizeof(uint32_t), s);
    PassArgs a{};
    a.err = f->err;
    a.n = n;
    a.ntiles = ntiles;
    a.spin_ns = (uint64_t)f->spin_limit_us * 1000ull;
    a.TB = tb;
    a.vals_in = f->sigma + (size_t)t0 * n;
    a.vals_in_ts = n;
    a.gather_src = seg64;
    a.gather_src_ts = 0;
    a.keys_out = f->sort.keys_a;
    a.keys_out_ts = n;
    a.vals_out = f->sort.vals_a;
    a.vals_out_ts = n;
    a.goff = f->sort.hist;
    a.goff_ts = 0;
    a.status = f->sort.status;
    a.ticket = f->sort.status + (size_t)tb * (ntiles + 1) * 256;
    a.shift = 0;
    onesweep_kernel<true><<<(unsigned)(ntiles * tb), NT, psm, s>>>(a);
    hf_after_launch("onesweep_kernel<segment>", s);
    cudaMemcpyAsync(f->sigma + (size_t)t0 * n, f->sort.vals_a, (size_t)tb * n * sizeof(uint32_t),
                    cudaMemcpyDeviceToDevice, s);
  }
  return cudaGetLastError() == cudaSuccess ? HF_OK : HF_ECUDA;
}

// Host side of the big-run path; called after the build's sync, when the
// host knows how many big runs tree t has.
int tie_fixup_big(hf_forest* f, int t, uint32_t nbig, cudaStream_t s) {
  if (nbig == 0) return HF_OK;
  if (nbig > f->tie.big_cap) return HF_ECUDA;
  const int64_t n = f->n;
  std::vector<uint2> runs(nbig);
  if (cudaMemcpy(runs.data(), f->tie.big_runs + (size_t)t * f->tie.big_cap, nbig * sizeof(uint2),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return HF_ECUDA;
  std::vector<uint32_t> offs(nbig);
  uint64_t total = 0;
  for (uint32_t r = 0; r < nbig; ++r) {
    offs[r] = (uint32_t)total;
    total += runs[r].y;
  }
  uint32_t m = 1;
  while (m < total) m <<= 1;
  const int W = f->W;
  const int tt = 64;
  uint64_t* fk = nullptr;
  uint32_t *pt = nullptr, *rn = nullptr, *ord = nullptr, *doffs = nullptr;
  uint8_t* ys = nullptr;
  uint2* druns = f->tie.big_runs + (size_t)t * f->tie.big_cap;
  int rc = HF_OK;
  auto take = [&](void** p, size_t bytes) {
    if (rc == HF_OK && hf_dalloc_bytes(p, bytes, s) != cudaSuccess) {
      cudaGetLastError();
      rc = HF_ENOMEM;
    }
  };
  take((void**)&fk, (size_t)total * W * 8);
  take((void**)&pt, total * 4);
  take((void**)&rn, total * 4);
  take((void**)&ord, (size_t)m * 4);
  take((void**)&doffs, nbig * 4);
  take((void**)&ys, (size_t)nbig * tt * f->d);
  if (rc == HF_OK) {
    cudaMemcpyAsync(doffs, offs.data(), nbig * 4, cudaMemcpyHostToDevice, s);
    uint32_t* sig = f->sigma + (size_t)t * n;
    big_fill_kernel<<<nbig, tt, 0, s>>>(f->planes, n, f->d, f->W32, f->bits, W, f->pi + (size_t)t * f->d,
                                        f->rbits + (size_t)t * f->W32, druns, doffs, (int)nbig, sig, fk, pt,
                                        rn, ys);
    hf_after_launch("big_fill_kernel", s);
    iota_kernel<<<hf_blocks(m, 256), 256, 0, s>>>(ord, m);
    hf_after_launch("iota_kernel", s);
    for (uint32_t kk = 2; kk <= m; kk <<= 1)
      for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
        bitonic_step_kernel<<<hf_blocks(m, 256), 256, 0, s>>>(ord, m, j, kk, fk, pt, rn, W, (uint32_t)total);
        hf_after_launch("bitonic_step_kernel", s);
      }
    big_write_kernel<<<hf_blocks(total, 256), 256, 0, s>>>(ord, (uint32_t)total, pt, rn, druns, doffs, sig);
    hf_after_launch("big_write_kernel", s);
  }
  // stream-ordered frees: the pool hands the memory to the next user of s
  // without a device-wide synchronisation
  hf_dfree_bytes(fk, s);
  hf_dfree_bytes(pt, s);
  hf_dfree_bytes(rn, s);
  hf_dfree_bytes(ord, s);
  hf_dfree_bytes(doffs, s);
  hf_dfree_bytes(ys, s);
  if (rc == HF_OK && cudaGetLastError() != cudaSuccess) rc = HF_ECUDA;
  return rc;
}

size_t tie_scratch_words(int W, int d, int bits, int K, int K2) {
  const TieGeom g = tie_geom(W, d, bits, K, K2);
  return (size_t)TIE_BLOCKS * g.cap * W;
}

size_t sort_status_words(int64_t n, int K, int tb) {
  const int64_t ntiles = (n + TILE - 1) / TILE;
  return ((size_t)tb * (ntiles + 1) * 256 + 1) * 8 * K;
}

int tie_small_cap(int W, int d, int bits, int K, int K2) { return tie_geom(W, d, bits, K, K2).cap; }
