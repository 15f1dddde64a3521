// Window distances on the tensor cores (tcgen05), then an exact re-rank.
//
// Paper, Algorithm 2: each sort contributes, for every point, the points
// around its position as candidates; the final selection is by vector
// distance. The distance step is the only dense contraction of the path. For
// the 128 points at positions [s, s+128) of one order (a row tile) and the
// points at positions [s - W8, s + 128 + W8) (W8 = w rounded up to 8; the
// column range, Ncol = 128 + 2 W8 positions), the squared distances are
//   d2(p, q) = |x_p|^2 + |x_q|^2 - 2 <x_p, x_q>,
// and the inner products are a 128 x Ncol Gram band. tcgen05.mma computes it
// with FP32 accumulation in tensor memory from BF16 operands (kind::f16) or
// from FP8 e4m3 operands with one scale per vector (kind::f8f6f4; x ~ s q, so
// <x_p, x_q> ~ s_p s_q <q_p, q_q>).
//
// The column range is cut into units of at most 256 columns (one MMA each per
// K step, N <= 256). When it fits one unit (W8 <= 64) the 128 owned rows are
// rows W8 .. W8+127 of that unit's staged rows, so both operands read one
// copy; otherwise the owned rows (the A operand) are staged once per tile in
// a resident region, one slot per 128-byte K chunk, each slot refilled for the
// next tile as soon as the tile's last MMA that reads it has completed. The
// unit's rows (the B operand) stream through a ring of K-chunk stages. Rows
// live in shared memory in the 128-byte-swizzled K-major layout.
//
// The epilogue reads each row's band (its 2w neighbours in the order) out of
// tensor memory and merges the estimated distances into the point's top-KP
// list (KP >= k + slack). Two halves of four warps share a tile: half h takes
// the 32-column chunks of parity h, each half keeps its own list for the row,
// and at the end of the tile half 1 hands its list to half 0 through shared
// memory, which merges it and writes the point's list back.
//
// After the last tree, rerank_kernel recomputes every listed candidate's
// distance in float32 with exact coordinate differences from the float32
// points, so the expansion's cancellation and the operand rounding never
// reach the result; the list is re-sorted and the first k columns are the
// answer.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <math.h>

#include "hf_internal.cuh"
#include "topk_list.cuh"

namespace {

constexpr int GB = 128;        // owned positions per tile = MMA M

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Whole warp: allocates `ncols` tensor-memory columns, writes the base
// address to *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A * B^T, A: M x 16, B: N x 16, both K-major BF16 in shared memory.
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The same with e4m3 A and B (K = 32 per instruction, 32 bytes per row).
__device__ __forceinline__ void mma_f8(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrives on *bar once all MMAs issued so far by this thread have completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
        "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
        "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
        "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO); the leading offset is unused for this layout.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t desc = 0;
  desc |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  desc |= (uint64_t)1 << 16;                  // leading byte offset (unused): 16 B
  desc |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: 1024 B
  desc |= (uint64_t)1 << 46;                  // descriptor version for tcgen05
  desc |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return desc;
}

// BF16 copy of the points (row pitch dp, a multiple of 64, zero padded) and
// per point (squared norm of the BF16-rounded row, scale 1).
__global__ void prepare_bf16_kernel(const float* __restrict__ x, int64_t n, int d, int dp,
                                    __nv_bfloat16* __restrict__ xb, float2* __restrict__ meta) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    float s = 0.f;
    for (int c = lane; c < dp; c += 32) {
      const float v = c < d ? x[i * d + c] : 0.f;
      const __nv_bfloat16 b = __float2bfloat16_rn(v);
      xb[i * dp + c] = b;
      const float r = __bfloat162float(b);
      s = fmaf(r, r, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) meta[i] = make_float2(s, 1.0f);
  }
}

// FP8 e4m3 copy of the points with one scale per vector: s = max|x| / 448
// (448 is the largest finite e4m3 value), q = e4m3(x / s) rounded to nearest
// with saturation, row pitch dp (a multiple of 128, zero padded); per point
// (float32 squared norm of x, s). A zero row gets s = 1 and q = 0.
__global__ void prepare_fp8_kernel(const float* __restrict__ x, int64_t n, int d, int dp,
                                   uint8_t* __restrict__ xq, float2* __restrict__ meta) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nw) {
    float m = 0.f, s2 = 0.f;
    for (int c = lane; c < d; c += 32) {
      const float v = x[i * d + c];
      m = fmaxf(m, fabsf(v));
      s2 = fmaf(v, v, s2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    const float sc = m > 0.f ? m / 448.0f : 1.0f;
    for (int c = 2 * lane; c < dp; c += 64) {
      const float v0 = c < d ? x[i * d + c] / sc : 0.f;
      const float v1 = c + 1 < d ? x[i * d + c + 1] / sc : 0.f;
      const __nv_fp8x2_storage_t p = __nv_cvt_float2_to_fp8x2(make_float2(v0, v1), __NV_SATFINITE, __NV_E4M3);
      *reinterpret_cast<__nv_fp8x2_storage_t*>(xq + i * dp + c) = p;
    }
    if (lane == 0) meta[i] = make_float2(s2, sc);
  }
}

// Rows of the operand copy in the order of one tree: xs[p] = xq[sigma[p]]
// (rowb bytes each, moved in 16-byte pieces) and ms[p] = meta[sigma[p]], so
// that the Gram kernel reads every unit's rows as one contiguous range.
__global__ void gather_rows_kernel(const uint8_t* __restrict__ xq, const float2* __restrict__ meta,
                                   const uint32_t* __restrict__ sigma, int64_t n, int rowb,
                                   uint8_t* __restrict__ xs, float2* __restrict__ ms) {
  const int per = rowb >> 4;  // 16-byte pieces per row
  const int64_t total = n * per;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / per;
    const int c = (int)(e - p * per);
    const uint32_t id = __ldg(sigma + p);
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(xq + (size_t)id * rowb) + c);
    __stcs(reinterpret_cast<uint4*>(xs + (size_t)p * rowb) + c, v);
    if (c == 0) ms[p] = __ldg(meta + id);
  }
}

struct GramArgs {
  const float2* ms;        // per position of this tree: (squared norm, scale)
  const uint32_t* sigma;   // order of this tree: position -> point
  const int32_t* tile_w;   // per-tile window of this tree, or null (uniform w)
  const uint16_t* pw;      // per-point window, or null (uniform w)
  const uint32_t* segr;    // segmented forest: set of each point, or null
  const int64_t* segoff;   // segmented forest: first position of each set (+ end)
  int64_t n;
  int nk;                  // K chunks of 128 bytes per row
  int elem_per_chunk;      // 64 (BF16) or 128 (FP8) elements per chunk
  int w;                   // window when tile_w is null
  int stages;              // B ring stages
  uint32_t a_off, b_off, slot_off, x_off, bar_off;  // shared-memory layout
  uint32_t b_stage_bytes;
  uint32_t* lidx;
  float* ldist;
  int* err;
  uint64_t spin_limit;
};

// ---------------------------------------------------------------------------
// Persistent, warp-specialised band kernel. One block per SM loops over row
// tiles t = blockIdx.x + i * gridDim.x and, within a tile, over its units
// (unit j = columns [256 j, 256 j + Nj) of the tile's column range). The
// operand rows are in the tree's position order (gather_rows_kernel), so a
// unit's rows are positions [c_lo + 256 j, c_lo + 256 j + Nj) and the tile's
// own rows positions [s, s + 128).
//   warp 0      TMA producer (one lane): per K chunk of a unit, boxes of 32
//               rows x 128 bytes into the B ring (128-byte swizzle, rows
//               outside the matrix zero-filled);
//   warp 1      MMA issuer (one lane): per unit, all K chunks into one of two
//               tensor-memory accumulators (256 columns each); it also owns
//               the tensor-memory allocation;
//   warp 2      prep: per unit, the (norm, scale, id) of its columns (and, for
//               the first unit, of the tile's own rows) into one of NSLOT
//               slots;
//   warp 3      A producer (one lane): per tile with several units, the own
//               rows into the resident A region, chunk kc once the previous
//               tile's last MMA reading it has completed;
//   warps 4..11 epilogue: a warp owns tensor-memory lanes 32 (warp % 4) ..
//               + 31 (tile rows) and, in half h = (warp - 4) / 4, the
//               32-column chunks of parity h.
// Every barrier wait is bounded (spin_limit ns of %globaltimer); when one
// gives up, the block raises the error word, every role leaves, and tensor
// memory is freed after a bounded wait for MMAs in flight.
// ---------------------------------------------------------------------------
constexpr int NSLOT = 4;           // staged (norm, scale, id) units: the prep warp runs ahead
constexpr int SLOT_COLS = 256;     // column entries per slot
constexpr int SLOT_ENTS = SLOT_COLS + GB;  // + the tile's own rows
constexpr int XE = 16;             // list entries handed over per exchange round
constexpr int TW = 0;              // TMA producer warp
constexpr int MW = 1;              // MMA warp
constexpr int PW = 2;              // prep warp
constexpr int AW = 3;              // A (own rows) producer warp
constexpr int EW0 = 4;             // first epilogue warp
constexpr int PT = (EW0 + 8) * 32;
constexpr uint32_t TMEM_ALL = 512; // two accumulators of 256 columns
constexpr int MAX_STAGES = 4;
constexpr int BOX_ROWS = 32;       // rows per TMA box

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}
// One arrival that also expects `bytes` of asynchronous transfers.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// A 2-D box of the tensor map at (x elements, y rows) into shared memory;
// completion is counted in bytes on *bar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

struct Bars {
  uint64_t full[MAX_STAGES], empty[MAX_STAGES];
  uint64_t afull[32], aempty[32];    // per resident A chunk (K chunks <= 32)
  uint64_t tfull[2], tempty[2];
  uint64_t mfull[NSLOT], mempty[NSLOT];
  uint64_t xfull[4], xempty[4];
  uint32_t tslot;
  int abort;
};

// A slot holds, for SLOT_ENTS entries (the unit's SLOT_COLS columns, then
// the tile's GB own rows), three arrays: squared norm (+inf outside the
// matrix), scale (FP8 form only) and point index.
struct SlotView {
  float* nrm;
  float* sc;
  uint32_t* id;
};
template <bool F8>
__device__ __forceinline__ SlotView slot_view(unsigned char* slots, int sl) {
  constexpr int words = F8 ? 3 : 2;
  float* b = reinterpret_cast<float*>(slots) + (size_t)sl * words * SLOT_ENTS;
  SlotView v;
  v.nrm = b;
  v.sc = F8 ? b + SLOT_ENTS : nullptr;
  v.id = reinterpret_cast<uint32_t*>(b + (F8 ? 2 : 1) * SLOT_ENTS);
  return v;
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait (limit in nanoseconds of %globaltimer); on timeout raises the
// error word and the block's abort flag; returns early once another role has
// aborted.
__device__ __forceinline__ bool pwait(uint64_t* bar, uint32_t parity, uint64_t limit_ns, volatile int* abort,
                                      int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  uint32_t it = 0;
  // try_wait suspends the thread for a while before it reports "not yet",
  // so the loop does not spin hot
  while (!mbar_try_wait(bar, parity)) {
    if ((++it & 15u) == 0) {
      if (*abort) return false;
      if (gtimer() - t0 > limit_ns) {
        *abort = 1;
        hf_raise(err, HF_ERRBIT_TIMEOUT);
        return false;
      }
    }
  }
  return true;
}

// The tile's window (0 = no row of the tile takes part), W8, column count
// and unit count.
struct TileGeom {
  int w, W8, ncol, J;
};
__device__ __forceinline__ TileGeom tile_geom(const GramArgs& a, int64_t t) {
  TileGeom g;
  g.w = a.tile_w ? __ldg(a.tile_w + t) : a.w;
  if (g.w <= 0) {
    g.w = g.W8 = g.ncol = g.J = 0;
    return g;
  }
  g.W8 = (g.w + 7) & ~7;
  g.ncol = GB + 2 * g.W8;
  g.J = (g.ncol + SLOT_COLS - 1) / SLOT_COLS;
  return g;
}


// v[j] of a register array (j known only at run time): a 5-level select tree.
__device__ __forceinline__ uint32_t pick32(const uint32_t (&v)[32], int j) {
  uint32_t a16[16], a8[8], a4[4], a2[2];
#pragma unroll
  for (int i = 0; i < 16; ++i) a16[i] = (j & 16) ? v[i + 16] : v[i];
#pragma unroll
  for (int i = 0; i < 8; ++i) a8[i] = (j & 8) ? a16[i + 8] : a16[i];
#pragma unroll
  for (int i = 0; i < 4; ++i) a4[i] = (j & 4) ? a8[i + 4] : a8[i];
#pragma unroll
  for (int i = 0; i < 2; ++i) a2[i] = (j & 2) ? a4[i + 2] : a4[i];
  return (j & 1) ? a2[1] : a2[0];
}

template <int KP, bool F8>
__global__ void __launch_bounds__(PT, 1) gram_band_kernel(GramArgs a, const __grid_constant__ CUtensorMap xmap) {
  extern __shared__ unsigned char smraw[];
  unsigned char* base = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
  unsigned char* aregion = base + a.a_off;
  unsigned char* bring = base + a.b_off;
  unsigned char* slots = base + a.slot_off;
  float* xd = reinterpret_cast<float*>(base + a.x_off);            // [XE][128] distances
  uint32_t* xi = reinterpret_cast<uint32_t*>(xd + XE * GB);        // [XE][128] indices
  Bars& S = *reinterpret_cast<Bars*>(base + a.bar_off);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (a.n + GB - 1) / GB;
  const uint64_t lim = a.spin_limit;
  const int nk = a.nk, stages = a.stages;

  if (warp == MW) tmem_alloc(&S.tslot, TMEM_ALL);
  if (tid == 0) {
    for (int i = 0; i < stages; ++i) {
      mbar_init(&S.full[i], 1);
      mbar_init(&S.empty[i], 1);
    }
    for (int i = 0; i < nk; ++i) {
      mbar_init(&S.afull[i], 1);
      mbar_init(&S.aempty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.tfull[i], 1);
      mbar_init(&S.tempty[i], 8);
    }
    for (int i = 0; i < NSLOT; ++i) {
      mbar_init(&S.mfull[i], 32);
      mbar_init(&S.mempty[i], 8);
    }
    for (int i = 0; i < 4; ++i) {
      mbar_init(&S.xfull[i], 32);
      mbar_init(&S.xempty[i], 32);
    }
    S.abort = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tslot;
  volatile int* abort = &S.abort;

  if (warp == TW) {
    // ---------------- TMA producer (one lane)
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      const uint32_t chunk_box = (uint32_t)BOX_ROWS * 128u;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const TileGeom g = tile_geom(a, t);
        const int64_t s = t * GB, c_lo = s - g.W8;
        for (int j = 0; j < g.J && ok; ++j) {
          const int nj = min(SLOT_COLS, g.ncol - SLOT_COLS * j);
          const int nbox = (nj + BOX_ROWS - 1) / BOX_ROWS;
          const int y0 = (int)(c_lo + (int64_t)SLOT_COLS * j);
          for (int kc = 0; kc < nk; ++kc, ++it) {
            const int x = kc * a.elem_per_chunk;
            const int st = it % stages;
            if (!pwait(&S.empty[st], ((it / stages) & 1) ^ 1, lim, abort, a.err)) {
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(&S.full[st], (uint32_t)nbox * chunk_box);
            const uint32_t d0 = smem_u32(bring + (size_t)st * a.b_stage_bytes);
            for (int b = 0; b < nbox; ++b) tma_load_2d(d0 + (uint32_t)b * chunk_box, &xmap, x, y0 + b * BOX_ROWS, &S.full[st]);
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == AW) {
    // ---------------- A producer (one lane): the tile's own rows, chunk kc
    // as soon as the previous tile's last MMA reading chunk kc has completed
    // (a thread of its own, so the B ring of the next tile never waits for it)
    if (lane == 0) {
      uint32_t auses = 0;
      bool ok = true;
      const uint32_t chunk_box = (uint32_t)BOX_ROWS * 128u;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const TileGeom g = tile_geom(a, t);
        if (g.J <= 1) continue;
        const int64_t s = t * GB;
        for (int kc = 0; kc < nk; ++kc) {
          if (!pwait(&S.aempty[kc], (auses & 1) ^ 1, lim, abort, a.err)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&S.afull[kc], (uint32_t)GB * 128u);
          const uint32_t d0 = smem_u32(aregion + (size_t)kc * GB * 128);
#pragma unroll
          for (int b = 0; b < GB / BOX_ROWS; ++b)
            tma_load_2d(d0 + (uint32_t)b * chunk_box, &xmap, kc * a.elem_per_chunk, (int)s + b * BOX_ROWS,
                        &S.afull[kc]);
        }
        ++auses;
      }
    }
    __syncwarp();
  } else if (warp == PW) {
    // ---------------- prep warp: per unit, the (norm, scale, id) of its
    // columns and (first unit) of the tile's own rows into a slot, ahead of
    // the MMA and the epilogue (contiguous reads: the tree's order)
    uint32_t u = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      const TileGeom g = tile_geom(a, t);
      const int64_t s = t * GB, c_lo = s - g.W8;
      for (int j = 0; j < g.J && ok; ++j, ++u) {
        const int sl = u % NSLOT;
        const int nj = min(SLOT_COLS, g.ncol - SLOT_COLS * j);
        if (!pwait(&S.mempty[sl], ((u / NSLOT) & 1) ^ 1, lim, abort, a.err)) {
          ok = false;
          break;
        }
        const SlotView se = slot_view<F8>(slots, sl);
        // rows outside the matrix get an infinite norm: they never pass a screen
#pragma unroll
        for (int m = 0; m < SLOT_ENTS / 32; ++m) {
          const int e = lane + 32 * m;
          int64_t pos;
          bool valid;
          if (e < SLOT_COLS) {
            pos = c_lo + (int64_t)SLOT_COLS * j + e;
            valid = e < nj && pos >= 0 && pos < a.n;
          } else {
            pos = s + (e - SLOT_COLS);
            valid = j == 0 && pos < a.n;
          }
          const uint32_t id = valid ? __ldg(a.sigma + pos) : 0xffffffffu;
          const float2 mt = valid ? __ldg(a.ms + pos) : make_float2(INFINITY, 0.f);
          se.nrm[e] = mt.x;
          if (F8) se.sc[e] = mt.y;
          se.id[e] = id;
          // the own rows' lists into L2: the epilogue reads them when it
          // starts the tile, a few units from now
          if (e >= SLOT_COLS && valid) {
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.ldist + (size_t)id * KP));
            asm volatile("prefetch.global.L2 [%0];" ::"l"(a.lidx + (size_t)id * KP));
          }
        }
        mbar_arrive(&S.mfull[sl]);
      }
    }
  } else if (warp == MW) {
    // ---------------- MMA issuer (one lane)
    if (lane == 0) {
      uint32_t it = 0, u = 0, auses = 0;
      const uint32_t bb = smem_u32(bring), ab = smem_u32(aregion);
      // FP32 accumulator; BF16 A and B (kind::f16) or e4m3 A and B
      // (kind::f8f6f4); both K-major; M >> 4 at bit 24, N >> 3 at bit 17
      const uint32_t id0 = (1u << 4) | (F8 ? 0u : ((1u << 7) | (1u << 10))) | ((uint32_t)(GB >> 4) << 24);
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x) {
        const TileGeom g = tile_geom(a, t);
        for (int j = 0; j < g.J; ++j, ++u) {
          const int buf = u & 1;
          const uint32_t use = u >> 1;
          if (!pwait(&S.tempty[buf], (use & 1) ^ 1, lim, abort, a.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t acc = tmem + (uint32_t)(buf * 256);
          const int nj = min(SLOT_COLS, g.ncol - SLOT_COLS * j);
          const uint32_t idesc = id0 | ((uint32_t)(nj >> 3) << 17);
          for (int kc = 0; kc < nk; ++kc, ++it) {
            const int st = it % stages;
            if (!pwait(&S.full[st], (it / stages) & 1, lim, abort, a.err) ||
                (g.J > 1 && !pwait(&S.afull[kc], auses & 1, lim, abort, a.err))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t chunk = bb + (uint32_t)(st * a.b_stage_bytes);
            const uint32_t achunk = g.J == 1 ? chunk + (uint32_t)(g.W8 >> 3) * 1024u : ab + (uint32_t)kc * GB * 128u;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t bdesc = smem_desc(chunk + ks * 32);
              const uint64_t adesc = smem_desc(achunk + ks * 32);
              if (F8)
                mma_f8(acc, adesc, bdesc, idesc, (kc | ks) != 0);
              else
                mma_bf16(acc, adesc, bdesc, idesc, (kc | ks) != 0);
            }
            mma_commit(&S.empty[st]);
            if (g.J > 1 && j == g.J - 1) mma_commit(&S.aempty[kc]);
          }
          if (!ok) break;
          mma_commit(&S.tfull[buf]);
        }
        if (g.J > 1) ++auses;
      }
    }
    __syncwarp();
  } else if (warp >= EW0) {
    // ---------------- epilogue: warp EW0 + q + 4 h owns tensor-memory lanes
    // 32 q .. 32 q + 31 (tile rows) and the 32-column chunks of parity h
    const int h = (warp - EW0) >> 2;
    const int q = warp & 3;       // a warp may access TMEM lanes 32 (warp % 4) .. + 31
    const int r = q * 32 + lane;  // tile row = TMEM lane
    uint32_t u = 0, xr = 0;
    bool ok = true;
    // waits and exits are warp-uniform: tcgen05.ld is .sync.aligned
    auto wwait = [&](uint64_t* bar, uint32_t par) {
      return __all_sync(0xffffffffu, pwait(bar, par, lim, abort, a.err));
    };
    for (int64_t t = blockIdx.x; t < ntiles && ok && !__any_sync(0xffffffffu, *abort); t += gridDim.x) {
      const TileGeom g = tile_geom(a, t);
      if (g.J == 0) continue;
      const int64_t p = t * GB + r;
      const bool rowok = p < a.n;
      ListK<KP> L;
      float ni = 0.f, c2 = 2.0f;
      uint32_t ip = 0xffffffffu;
      int wlo = 0, whi = -1;
      for (int j = 0; j < g.J; ++j, ++u) {
        const int sl = u % NSLOT, buf = u & 1;
        const uint32_t use = u >> 1;
        if (!wwait(&S.mfull[sl], (u / NSLOT) & 1)) {
          ok = false;
          break;
        }
        const SlotView se = slot_view<F8>(slots, sl);
        if (j == 0) {
          ip = se.id[SLOT_COLS + r];
          ni = se.nrm[SLOT_COLS + r];
          c2 = F8 ? 2.0f * se.sc[SLOT_COLS + r] : 2.0f;
          int wr = g.w;
          if (rowok && a.pw) wr = min(wr, (int)__ldg(a.pw + ip));
          // the row's band: columns [r + W8 - wr, r + W8 + wr] except r + W8
          wlo = r + g.W8 - wr;
          whi = rowok ? r + g.W8 + wr : -1;
          if (rowok && a.segr) {
            // segmented forest: only the positions of the row's own set
            // (column c is position t * GB - W8 + c)
            const uint32_t sg = __ldg(a.segr + ip);
            const int64_t cbase = t * GB - g.W8;
            const int64_t plo = __ldg(a.segoff + sg) - cbase, phi = __ldg(a.segoff + sg + 1) - 1 - cbase;
            if (plo > wlo) wlo = (int)plo;
            if (phi < whi) whi = (int)phi;
          }
          // both halves start from the point's list (fetched while the MMAs
          // run), so both screen against its current last entry; half 0
          // writes the merged list back
          if (rowok)
            L.load(a.ldist + (size_t)ip * KP, a.lidx + (size_t)ip * KP);
          else
            L.clear();
        }
        if (!wwait(&S.tfull[buf], use & 1)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int u0 = SLOT_COLS * j;
        const int wb_hi = 32 * q + 31 + 2 * g.W8;  // last band column of the warp
        const int diag = r + g.W8;
        // chunks [c0, c0 + 32) of the warp's band inside this unit, parity h
        int c0 = max(32 * q, u0);
        if (((c0 >> 5) & 1) != h) c0 += 32;
        for (; c0 <= wb_hi && c0 < u0 + SLOT_COLS; c0 += 64) {
          __syncwarp();  // reconverge after the divergent inserts
          uint32_t v[32];
          tmem_ld32(tmem + (uint32_t)(buf * 256) + ((uint32_t)(32 * q) << 16) + (uint32_t)(c0 - u0), v);
          const int lo = wlo - c0 > 0 ? wlo - c0 : 0;
          const int hi = whi - c0 < 31 ? whi - c0 : 31;
          uint32_t wm = 0;
          if (lo <= hi) wm = (0xffffffffu >> (31 - hi + lo)) << lo;
          if (diag >= c0 && diag < c0 + 32) wm &= ~(1u << (diag - c0));
          // screen: column c passes when its estimate d2 = ni + (n_c - 2 c2' dot)
          // is at most the list's current last entry (ties pass; the offer
          // decides); with ti = last - ni (finite even for an unfilled list),
          // the sign bit of ti - (n_c - ...) marks a miss, and the misses of
          // the 32 columns are gathered by funnel shifts
          const float ti = fminf(L.d[KP - 1], 3.0e38f) - ni;
          const float* cn = se.nrm + (c0 - u0);
          uint32_t miss = 0;
#pragma unroll
          for (int q4 = 0; q4 < 8; ++q4) {
            const float4 nn = *reinterpret_cast<const float4*>(cn + 4 * q4);
            float4 ss = make_float4(1.f, 1.f, 1.f, 1.f);
            if (F8) ss = *reinterpret_cast<const float4*>(se.sc + (c0 - u0) + 4 * q4);
            const float nv[4] = {nn.x, nn.y, nn.z, nn.w};
            const float sv[4] = {ss.x, ss.y, ss.z, ss.w};
            // two columns per packed FP32 pair instruction (fma.rn.f32x2,
            // sub.rn.f32x2: each lane of the pair rounds as the scalar form)
#pragma unroll
            for (int e = 0; e < 4; e += 2) {
              const int jj = 4 * q4 + e;
              const float m0 = F8 ? -c2 * sv[e] : -2.0f, m1 = F8 ? -c2 * sv[e + 1] : -2.0f;
              uint32_t p0, p1, d0, d1;
              asm("{\n .reg .b64 a, m, nn, t, p, dd;\n"
                  " mov.b64 a, {%4, %5};\n mov.b64 m, {%6, %7};\n mov.b64 nn, {%8, %9};\n mov.b64 t, {%10, %10};\n"
                  " fma.rn.f32x2 p, a, m, nn;\n sub.rn.f32x2 dd, t, p;\n"
                  " mov.b64 {%0, %1}, p;\n mov.b64 {%2, %3}, dd;\n}"
                  : "=r"(p0), "=r"(p1), "=r"(d0), "=r"(d1)
                  : "r"(v[jj]), "r"(v[jj + 1]), "f"(m0), "f"(m1), "f"(nv[e]), "f"(nv[e + 1]), "f"(ti));
              v[jj] = p0;  // the partial estimates replace the dot products
              v[jj + 1] = p1;
              miss = __funnelshift_l(d0, miss, 1);
              miss = __funnelshift_l(d1, miss, 1);
            }
          }
          uint32_t hm = __brev(~miss) & wm;
          while (hm) {
            const int jj = __ffs(hm) - 1;
            hm &= hm - 1;
            L.offer(__uint_as_float(pick32(v, jj)) + ni, se.id[(c0 - u0) + jj]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&S.tempty[buf]);
          mbar_arrive(&S.mempty[sl]);
        }
      }
      if (!ok) break;
      // half 1 hands its list to half 0 in rounds of XE entries
      for (int e0 = 0; e0 < KP && ok; e0 += XE, ++xr) {
        if (h == 1) {
          if (!wwait(&S.xempty[q], (xr & 1) ^ 1)) {
            ok = false;
            break;
          }
#pragma unroll
          for (int e = 0; e < XE; ++e) {
            xd[e * GB + r] = L.d[e0 + e];
            xi[e * GB + r] = L.i[e0 + e];
          }
          mbar_arrive(&S.xfull[q]);
        } else {
          if (!wwait(&S.xfull[q], xr & 1)) {
            ok = false;
            break;
          }
#pragma unroll 1
          for (int e = 0; e < XE; ++e) L.offer(xd[e * GB + r], xi[e * GB + r]);
          mbar_arrive(&S.xempty[q]);
        }
      }
      if (ok && h == 0 && rowok) L.store(a.ldist + (size_t)ip * KP, a.lidx + (size_t)ip * KP);
    }
  }
  // teardown: the last commit completes before tensor memory is freed
  tc_fence_before();
  __syncthreads();
  if (warp == MW) {
    if (*abort) {
      // MMAs may still be in flight after an abort: give them a bounded time
      const uint64_t t0 = gtimer();
      while (gtimer() - t0 < lim) {
      }
    }
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_ALL);
  }
}

// Transposing butterfly over NV candidates (NV = 16 or 32): lane l holds
// v[u] = its partial sum for candidate u; afterwards the return value of lane
// l is the total over all lanes for candidate l % NV.
template <int NV>
__device__ __forceinline__ float warp_transpose_sum(float (&v)[NV], int lane) {
#pragma unroll
  for (int s = NV / 2; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = up ? v[i] : v[i + s];
      const float keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  float r = v[0];
#pragma unroll
  for (int o = NV; o < 32; o <<= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  return r;
}

// Exact re-rank: one warp per point, points taken in the order of the first
// tree (consecutive warps then share most candidate rows in L2). Listed
// candidates are scored up to 32 at a time with float32 exact differences:
// every lane reads its coordinates of each candidate row (the warp reads a row
// in coalesced 512-byte pieces when rows are float4-aligned) and keeps one
// partial sum per candidate; a transposing butterfly gives candidate j's
// distance in lane j. The KP entries are then re-sorted by (distance, index);
// empty slots stay (+inf, 0xffffffff). Slots kc.. of the incoming list are
// dropped (kc = KP keeps all).
template <int KP>
__global__ void __launch_bounds__(256, 6) rerank_kernel(const float* __restrict__ x, int64_t n, int d,
                                                     const uint32_t* __restrict__ order, int vec4, int kc,
                                                     uint32_t* __restrict__ lidx, float* __restrict__ ldist) {
  constexpr int PER = (KP + 31) / 32;
  constexpr int NV = KP < 32 ? KP : 32;  // candidates per round
  __shared__ uint32_t s_c[256 / 32][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t wi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wi >= n) return;
  const int64_t i = order ? (int64_t)__ldg(order + wi) : wi;
  const float* xi = x + (size_t)i * d;
  float dd[PER];
  uint32_t id[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    id[u] = 32 * u + lane < kc ? lidx[(size_t)i * KP + 32 * u + lane] : 0xffffffffu;
    dd[u] = INFINITY;
  }
#pragma unroll
  for (int g = 0; g < PER; ++g) {
    s_c[wib][lane] = id[g];
    __syncwarp();
    float part[NV];
#pragma unroll
    for (int u = 0; u < NV; ++u) part[u] = 0.f;
    if (vec4) {
      for (int m = 4 * lane; m < d; m += 128) {
        const float4 xa = __ldg(reinterpret_cast<const float4*>(xi + m));
#pragma unroll
        for (int u = 0; u < NV; ++u) {
          const uint32_t c = s_c[wib][u];
          if (c != 0xffffffffu) {
            const float4 xb = __ldg(reinterpret_cast<const float4*>(x + (size_t)c * d + m));
            float e = xa.x - xb.x;
            float acc = fmaf(e, e, part[u]);
            e = xa.y - xb.y;
            acc = fmaf(e, e, acc);
            e = xa.z - xb.z;
            acc = fmaf(e, e, acc);
            e = xa.w - xb.w;
            part[u] = fmaf(e, e, acc);
          }
        }
      }
    } else {
      for (int m = lane; m < d; m += 32) {
        const float xa = __ldg(xi + m);
#pragma unroll
        for (int u = 0; u < NV; ++u) {
          const uint32_t c = s_c[wib][u];
          if (c != 0xffffffffu) {
            const float e = xa - __ldg(x + (size_t)c * d + m);
            part[u] = fmaf(e, e, part[u]);
          }
        }
      }
    }
    const float dist = warp_transpose_sum<NV>(part, lane);
    if (id[g] != 0xffffffffu) dd[g] = dist;
    __syncwarp();
  }
  // rank of each lane's entries among all KP entries by (distance, index,
  // slot): unique even among empty slots; padding slots (>= KP) rank last
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int myslot = u * 32 + lane;
    uint32_t rk = 0;
#pragma unroll
    for (int v = 0; v < PER; ++v)
      for (int src = 0; src < 32; ++src) {
        const float od = __shfl_sync(0xffffffffu, dd[v], src);
        const uint32_t oi = __shfl_sync(0xffffffffu, id[v], src);
        const int os = v * 32 + src;
        const bool lt = lessp(od, oi, dd[u], id[u]) || (od == dd[u] && oi == id[u] && os < myslot);
        rk += lt ? 1u : 0u;
      }
    if (myslot < KP) {
      ldist[(size_t)i * KP + rk] = dd[u];
      lidx[(size_t)i * KP + rk] = id[u];
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct GramPlan {
  int ok = 0;
  int rowb = 0, nk = 0, stages = 0;
  uint32_t a_off = 0, b_off = 0, slot_off = 0, x_off = 0, bar_off = 0, b_stage_bytes = 0;
  size_t smem = 0;
};

int max_smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 227 * 1024;
  }
  return v;
}

// Shared-memory layout for the widest window wmax of a launch.
GramPlan gram_plan(int d, int wmax, bool f8, int smem_cap) {
  GramPlan p;
  p.rowb = f8 ? (d + 127) / 128 * 128 : (d + 63) / 64 * 128;
  p.nk = p.rowb / 128;
  if (wmax < 1 || p.nk > 32) return p;
  const int W8 = (wmax + 7) & ~7;
  const int ncol = GB + 2 * W8;
  const int J = (ncol + SLOT_COLS - 1) / SLOT_COLS;
  const int stage_rows = (J == 1 ? ncol : SLOT_COLS) + BOX_ROWS - 1;  // whole boxes
  p.b_stage_bytes = (uint32_t)(stage_rows / BOX_ROWS * BOX_ROWS) * 128u;
  const size_t a_bytes = J > 1 ? (size_t)p.nk * GB * 128 : 0;
  const size_t slot_bytes = (size_t)NSLOT * SLOT_ENTS * (f8 ? 12 : 8);
  const size_t x_bytes = (size_t)2 * XE * GB * 4;
  const size_t bar_bytes = (sizeof(Bars) + 127) / 128 * 128;
  size_t off = 0;
  p.a_off = (uint32_t)off;
  off += a_bytes;
  p.b_off = (uint32_t)off;  // 1024-aligned: a_bytes is a multiple of 16 KB
  const size_t fixed = a_bytes + slot_bytes + x_bytes + bar_bytes + 1024;
  if ((size_t)smem_cap <= fixed) return p;
  int st = (int)(((size_t)smem_cap - fixed) / p.b_stage_bytes);
  if (st > MAX_STAGES) st = MAX_STAGES;
  if (st < 2) return p;
  p.stages = st;
  off += (size_t)st * p.b_stage_bytes;  // stage sizes are multiples of 4 KB
  p.slot_off = (uint32_t)off;
  off += slot_bytes;
  p.x_off = (uint32_t)off;
  off += x_bytes;
  p.bar_off = (uint32_t)off;
  off += bar_bytes;
  p.smem = off + 1024;
  // one block per SM: it holds all 512 tensor-memory columns, so it also asks
  // for more than half of the SM's shared memory
  if (p.smem < 120 * 1024) p.smem = 120 * 1024;
  p.ok = 1;
  return p;
}

// Tensor map of the position-ordered operand rows xs [n][rowb bytes]: boxes
// of 128 bytes x 32 rows, 128-byte swizzle (the layout the MMA descriptors
// read), zero fill outside the matrix.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int make_row_map(CUtensorMap* map, const void* xs, int64_t n, int rowb, bool f8) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
      cudaGetLastError();
      return HF_ECUDA;
    }
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  const int esz = f8 ? 1 : 2;
  const cuuint64_t gdim[2] = {(cuuint64_t)(rowb / esz), (cuuint64_t)n};
  const cuuint64_t gstride[1] = {(cuuint64_t)rowb};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)BOX_ROWS};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        const_cast<void*>(xs), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? HF_OK : HF_ECUDA;
}

template <int KP, bool F8>
int launch_band(const GramArgs& a, const CUtensorMap& map, size_t smem, cudaStream_t s) {
  if (cudaFuncSetAttribute((const void*)gram_band_kernel<KP, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return HF_ECUDA;
  int sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = (a.n + GB - 1) / GB;
  const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);
  gram_band_kernel<KP, F8><<<grid, PT, smem, s>>>(a, map);
  hf_after_launch(F8 ? "gram_band_kernel<fp8>" : "gram_band_kernel<bf16>", s);
  return HF_OK;
}

}  // namespace

int gram_supported(int d, int w, int form) {
  if (form != 1 && form != 2) return 0;
  return gram_plan(d, w, form == 2, max_smem_optin()).ok;
}

size_t gram_row_bytes(int d, int form) { return form == 2 ? (size_t)(d + 127) / 128 * 128 : (size_t)(d + 63) / 64 * 128; }

void launch_prepare_operands(const float* x, int64_t n, int d, int form, void* xq, float2* meta, cudaStream_t s) {
  const unsigned blocks = hf_blocks(n * 32, 256, 152 * 16);
  if (form == 2) {
    prepare_fp8_kernel<<<blocks, 256, 0, s>>>(x, n, d, (int)gram_row_bytes(d, 2), static_cast<uint8_t*>(xq), meta);
    hf_after_launch("prepare_fp8_kernel", s);
  } else {
    prepare_bf16_kernel<<<blocks, 256, 0, s>>>(x, n, d, (int)gram_row_bytes(d, 1) / 2,
                                               static_cast<__nv_bfloat16*>(xq), meta);
    hf_after_launch("prepare_bf16_kernel", s);
  }
}

void launch_gather_rows(const void* xq, const float2* meta, int form, int64_t n, int d, const uint32_t* sigma,
                        void* xs, float2* ms, cudaStream_t s) {
  const int rowb = (int)gram_row_bytes(d, form);
  gather_rows_kernel<<<hf_blocks(n * (rowb / 16), 256, 152 * 32), 256, 0, s>>>(
      static_cast<const uint8_t*>(xq), meta, sigma, n, rowb, static_cast<uint8_t*>(xs), ms);
  hf_after_launch("gather_rows_kernel", s);
}

int launch_gram_window(int form, int64_t n, int d, const uint32_t* sigma, int w, const int32_t* tile_w,
                       const uint16_t* pw, int kp, uint32_t* li, float* ld, int* err, const void* xs, const float2* ms,
                       cudaStream_t s, const uint32_t* segr, const int64_t* segoff) {
  const bool f8 = form == 2;
  const GramPlan p = gram_plan(d, w, f8, max_smem_optin());
  if (!p.ok) return HF_EINVAL;
  alignas(64) CUtensorMap map;
  const int rc = make_row_map(&map, xs, n, p.rowb, f8);
  if (rc != HF_OK) return rc;
  GramArgs a;
  a.ms = ms;
  a.sigma = sigma;
  a.tile_w = tile_w;
  a.pw = pw;
  a.segr = segr;
  a.segoff = segoff;
  a.n = n;
  a.nk = p.nk;
  a.elem_per_chunk = f8 ? 128 : 64;
  a.w = w;
  a.stages = p.stages;
  a.a_off = p.a_off;
  a.b_off = p.b_off;
  a.slot_off = p.slot_off;
  a.x_off = p.x_off;
  a.bar_off = p.bar_off;
  a.b_stage_bytes = p.b_stage_bytes;
  a.lidx = li;
  a.ldist = ld;
  a.err = err;
  a.spin_limit = 2000000000ull;  // 2 s per wait (globaltimer nanoseconds)
  switch (kp * 2 + (f8 ? 1 : 0)) {
    case 32: return launch_band<16, false>(a, map, p.smem, s);
    case 33: return launch_band<16, true>(a, map, p.smem, s);
    case 64: return launch_band<32, false>(a, map, p.smem, s);
    case 65: return launch_band<32, true>(a, map, p.smem, s);
    default: return HF_EINVAL;
  }
}

int launch_rerank(const float* x, int64_t n, int d, const uint32_t* order, int kp, int kc, uint32_t* li, float* ld,
                  cudaStream_t s) {
  const unsigned blocks = hf_blocks(n * 32, 256);
  const int vec4 = d % 4 == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  if (kc < 1 || kc > kp) return HF_EINVAL;
  switch (kp) {
    case 16: rerank_kernel<16><<<blocks, 256, 0, s>>>(x, n, d, order, vec4, kc, li, ld); break;
    case 32: rerank_kernel<32><<<blocks, 256, 0, s>>>(x, n, d, order, vec4, kc, li, ld); break;
    case 64: rerank_kernel<64><<<blocks, 256, 0, s>>>(x, n, d, order, vec4, kc, li, ld); break;
    default: return HF_EINVAL;
  }
  hf_after_launch("rerank_kernel", s);
  return HF_OK;
}
