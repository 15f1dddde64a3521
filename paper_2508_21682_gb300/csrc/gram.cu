// Window distances on the tensor cores (tcgen05), then an exact re-rank.
//
// Paper, Algorithm 2: candidates are the neighbours around each position of
// every sort; the final selection is by vector distance. The distance step is
// the only dense contraction of the path: the squared distances between the
// B = 128 points at positions [s, s+128) of one order and the N = 128 + 2 W8
// points at positions [s - W8, s + 128 + W8) (W8 = w rounded up to 8) are
//   d2(p, q) = |x_p|^2 + |x_q|^2 - 2 <x_p, x_q>,
// and the inner products of a whole block are one 128 x N Gram tile. Here the
// tile is computed by tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation
// in tensor memory): the N gathered rows are staged once in shared memory in
// the 128-byte-swizzled K-major layout; the 128 owned rows are rows W8 ..
// W8+127 of that same tile, so both operands read one copy. The epilogue reads
// each row's band (2w columns) out of tensor memory and merges approximate
// distances (of the BF16-rounded vectors, expanded form) into the point's
// top-KP list, KP >= 2k.
//
// After the last tree, rerank_kernel recomputes every listed candidate's
// distance in float32 with exact coordinate differences from the float32
// points, so the expansion's cancellation and the BF16 rounding never reach
// the result; the list is re-sorted and the first k columns are the answer.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "hf_internal.cuh"
#include "topk_list.cuh"

namespace {

constexpr int GB = 128;        // owned positions per block = MMA M
constexpr int KC = 64;         // BF16 elements per 128-byte K chunk

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
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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

// 16-byte asynchronous copy global -> shared (zero fill when !valid).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  const int sz = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// BF16 copy of the points (row pitch dp, a multiple of 64, zero padded) and
// the FP32 squared norms of the BF16-rounded rows.
__global__ void prepare_bf16_kernel(const float* __restrict__ x, int64_t n, int d, int dp,
                                    __nv_bfloat16* __restrict__ xb, float* __restrict__ nrm) {
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
    if (lane == 0) nrm[i] = s;
  }
}

struct GramArgs {
  const __nv_bfloat16* xb;
  const float* nrm;
  const uint32_t* sigma;
  int64_t n;
  int dp, w, W8, N;
  uint32_t idesc;
  uint32_t* lidx;
  float* ldist;
  int* err;
  uint64_t spin_limit;
};

// ---------------------------------------------------------------------------
// Persistent, warp-specialised Gram kernel. One block per SM loops over tiles
// (tile t = blockIdx.x + i * gridDim.x). Warps 0..3 (loaders) stage the
// tile's row ids and norms in one of NSLOT slots (so they can run up to
// NSLOT - 1 tiles ahead of the epilogue) and gather its rows into a ring of
// STAGES K-chunk buffers with 16-byte asynchronous copies into the swizzled
// layout; each thread keeps DEPTH chunks in flight and, once the oldest has
// landed, issues a proxy fence and its arrival on that chunk's "full"
// barrier. Warp 4 (MMA) issues the chunk's four K = 16 MMAs into one of two
// tensor-memory accumulators and releases the chunk buffer through
// tcgen05.commit. Warps 5..8 and 9..12 form two epilogue groups that take
// alternate tiles (one accumulator each): each thread owns one row
// (tensor-memory lane), screens its band and merges into the point's list,
// then releases the accumulator and the staged slot.
// Every wait on a barrier is bounded; when one gives up, the block raises the
// error word, every role leaves its loop, and tensor memory is freed after a
// bounded wait for MMAs in flight.
// ---------------------------------------------------------------------------
constexpr int STAGES = 4;
constexpr int NSLOT = 4;           // staged (norm, id) rows: tiles the loaders may run ahead
constexpr int DEPTH = 3;           // K chunks a loader keeps in flight (< STAGES)
constexpr int PER = 16;            // 16-byte pieces per loader thread and chunk
constexpr int LW = 4;              // loader warps (warps 0..3)
constexpr int MW = LW;             // MMA warp
constexpr int EW0 = LW + 1;        // first epilogue warp (two groups of 4)
constexpr int PT = (LW + 1 + 8) * 32;
constexpr uint32_t TMEM_ALL = 512; // two accumulators of 256 columns

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}

struct PersistSmem {
  uint64_t full[STAGES], empty[STAGES];
  uint64_t tfull[2], tempty[2];
  uint64_t mfull[NSLOT], mempty[NSLOT];
  uint32_t tslot;
  int abort;
};

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
  while (!mbar_try_wait(bar, parity)) {
    __nanosleep(64);  // leave issue slots to the warps doing work
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

template <int KP>
__global__ void __launch_bounds__(PT, 1) gram_window_kernel(GramArgs a) {
  extern __shared__ unsigned char smraw[];
  unsigned char* base = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
  const int N = a.N, nk = a.dp / KC;
  const size_t stage_bytes = (size_t)N * 128;
  const int NP = N + 32;  // padded: an epilogue chunk may run past column N - 1
  float2* mnid = reinterpret_cast<float2*>(base + STAGES * stage_bytes);  // [NSLOT][NP] (norm, id bits)
  float* cbd = reinterpret_cast<float*>(mnid + NSLOT * NP);               // [32][256]
  uint32_t* cbi = reinterpret_cast<uint32_t*>(cbd + 256 * 32);            // [32][256]
  PersistSmem& S = *reinterpret_cast<PersistSmem*>(cbi + 256 * 32);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (a.n + GB - 1) / GB;
  const uint64_t lim = a.spin_limit;

  if (warp == MW) tmem_alloc(&S.tslot, TMEM_ALL);
  if (tid == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&S.full[i], LW * 32);
      mbar_init(&S.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&S.tfull[i], 1);
      mbar_init(&S.tempty[i], 4);
    }
    for (int i = 0; i < NSLOT; ++i) {
      mbar_init(&S.mfull[i], 1);
      mbar_init(&S.mempty[i], 4);
    }
    S.abort = 0;
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S.tslot;
  volatile int* abort = &S.abort;

  if (warp < LW) {
    // ---------------- loaders: 128 threads
    const int lt = tid;  // 0 .. 127
    uint32_t it = 0;     // chunk counter across tiles
    int pending = 0;     // chunks issued but not yet marked full
    int tl = 0;
    // Row ids (and then norms) of the next tile are loaded into registers
    // while the current tile streams, so a tile starts without a dependent
    // pair of global round trips. Thread lt stages rows lt + 128 j.
    constexpr int RPT = 3;  // ceil((N + 32) / 128) for N <= 256
    uint32_t npid[RPT];
    float nnrm[RPT];
    auto fetch_ids = [&](int64_t tt) {
      const int64_t rr0 = tt * GB - a.W8;
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        const int r = lt + j * LW * 32;
        const int64_t p = rr0 + r;
        npid[j] = (tt < ntiles && r < N && p >= 0 && p < a.n) ? __ldg(a.sigma + p) : 0xffffffffu;
      }
    };
    auto fetch_norms = [&]() {
#pragma unroll
      for (int j = 0; j < RPT; ++j)
        nnrm[j] = npid[j] != 0xffffffffu ? __ldg(a.nrm + npid[j]) : __uint_as_float(0x7fc00000u);
    };
    fetch_ids(blockIdx.x);
    fetch_norms();
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
      const int slot = tl % NSLOT;
      const uint32_t suse = (uint32_t)(tl / NSLOT);
      if (!pwait(&S.mempty[slot], (suse & 1) ^ 1, lim, abort, a.err)) break;
      float2* snid = mnid + slot * NP;
      // rows outside the matrix get a NaN norm: their distances never pass a screen
#pragma unroll
      for (int j = 0; j < RPT; ++j) {
        const int r = lt + j * LW * 32;
        if (r < NP) snid[r] = make_float2(nnrm[j], __uint_as_float(npid[j]));
      }
      fetch_ids(t + gridDim.x);
      asm volatile("bar.sync 1, %0;" ::"r"(LW * 32) : "memory");  // loaders only
      if (lt == 0) mbar_arrive(&S.mfull[slot]);
      // this thread's pieces: the same (row, 16-byte column) in every chunk,
      // so sources and swizzled destinations are formed once per tile
      const __nv_bfloat16* src[PER];
      uint32_t dsto[PER];
      uint32_t lmask = 0, smask = 0;  // pieces to load / to store
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = lt + q * LW * 32;
        const int r = e >> 3, j = e & 7;
        const uint32_t pid = e < N * 8 ? __float_as_uint(snid[r].y) : 0xffffffffu;
        src[q] = a.xb + (pid != 0xffffffffu ? (size_t)pid * a.dp : 0) + j * 8;
        dsto[q] = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
        if (e < N * 8) smask |= 1u << q;
        if (pid != 0xffffffffu) lmask |= 1u << q;
      }
      bool ok = true;
      for (int kc = 0; kc < nk; ++kc, ++it) {
        const int st = it % STAGES;
        if (!pwait(&S.empty[st], ((it / STAGES) & 1) ^ 1, lim, abort, a.err)) {
          ok = false;
          break;
        }
        const uint32_t dst0 = smem_u32(base + st * stage_bytes);
#pragma unroll
        for (int q = 0; q < PER; ++q)
          if ((smask >> q) & 1u) cp_async16(dst0 + dsto[q], src[q] + kc * KC, (lmask >> q) & 1u);
        cp_async_commit();
        // keep DEPTH chunks in flight: once the oldest has landed, make its
        // stores visible to the tensor core and mark its stage full
        if (++pending == DEPTH) {
          cp_async_wait<DEPTH - 1>();
          fence_proxy_async_smem();
          mbar_arrive(&S.full[(it - (DEPTH - 1)) % STAGES]);
          --pending;
        }
      }
      fetch_norms();  // the next tile's ids have arrived by now
      if (!ok) break;
      if (nk < DEPTH) {
        // a later tile's accumulator wait must not depend on this tile's
        // chunks still being held back
        cp_async_wait<0>();
        fence_proxy_async_smem();
        for (; pending > 0; --pending) mbar_arrive(&S.full[(it - pending) % STAGES]);
      }
    }
    // the last chunks (also after an abort: no copy may be in flight at exit)
    cp_async_wait<0>();
    fence_proxy_async_smem();
    for (; pending > 0; --pending) mbar_arrive(&S.full[(it - pending) % STAGES]);
  } else if (warp == MW) {
    // ---------------- MMA issuer (one lane)
    if (lane == 0) {
      uint32_t it = 0;
      int tl = 0;
      const uint32_t sb = smem_u32(base);
      for (int64_t t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x, ++tl) {
        const int buf = tl & 1;
        const uint32_t use = (uint32_t)(tl >> 1);
        if (!pwait(&S.tempty[buf], (use & 1) ^ 1, lim, abort, a.err)) break;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(buf * 256);
        for (int kc = 0; kc < nk; ++kc, ++it) {
          const int st = it % STAGES;
          if (!pwait(&S.full[st], (it / STAGES) & 1, lim, abort, a.err)) break;
          tc_fence_after();
          const uint32_t chunk = sb + (uint32_t)(st * stage_bytes);
#pragma unroll
          for (int ks = 0; ks < KC / 16; ++ks) {
            const uint64_t bdesc = smem_desc(chunk + ks * 32);
            const uint64_t adesc = smem_desc(chunk + (a.W8 >> 3) * 1024 + ks * 32);
            mma_bf16(acc, adesc, bdesc, a.idesc, (kc | ks) != 0);
          }
          mma_commit(&S.empty[st]);
        }
        mma_commit(&S.tfull[buf]);
      }
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: group 0 = warps 5..8 (accumulator 0, even
    // tiles), group 1 = warps 9..12 (accumulator 1, odd tiles); within a
    // group, warp w owns tensor-memory lanes 32 (w % 4) .. + 31
    const int grp = (warp - EW0) >> 2;
    const int quarter = warp & 3;
    const int r = quarter * 32 + lane;  // tile row = TMEM lane
    // staged candidates: entry u of thread `slot` at [u][slot] (conflict-free)
    const int slot = grp * 128 + r;
    float* mybd = cbd + slot;
    uint32_t* mybi = cbi + slot;
    const int buf = grp;
    int tl = grp;
    for (int64_t t = blockIdx.x + (int64_t)grp * gridDim.x; t < ntiles && !*abort;
         t += 2 * (int64_t)gridDim.x, tl += 2) {
      const uint32_t use = (uint32_t)(tl >> 1);
      const int sl = tl % NSLOT;
      if (!pwait(&S.mfull[sl], (tl / NSLOT) & 1, lim, abort, a.err)) break;
      // the row's list is fetched while the tile's MMAs run
      const float2* snid = mnid + sl * NP;
      const int64_t p = t * GB + r;
      const bool rowok = p < a.n;
      ListK<KP> L;
      const float2 own = snid[r + a.W8];
      const uint32_t ip = __float_as_uint(own.y);
      if (rowok) L.load(a.ldist + (size_t)ip * KP, a.lidx + (size_t)ip * KP);
      if (!pwait(&S.tfull[buf], use & 1, lim, abort, a.err)) break;
      tc_fence_after();
      const float np_ = own.x;
      // the row's band: columns [r + W8 - w, r + W8 + w] except r + W8 itself
      const int wlo = r + a.W8 - a.w, whi = r + a.W8 + a.w, diag = r + a.W8;
      const int cfirst = 32 * quarter;
      const int clast = 32 * quarter + 31 + 2 * a.W8;
      for (int c0 = cfirst; c0 <= clast && c0 < N; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(tmem + (uint32_t)(buf * 256) + ((uint32_t)(32 * quarter) << 16) + (uint32_t)c0, v);
        const int lo = wlo - c0 > 0 ? wlo - c0 : 0;
        const int hi = whi - c0 < 31 ? whi - c0 : 31;
        uint32_t wm = 0;
        if (rowok && lo <= hi) wm = (0xffffffffu >> (31 - hi + lo)) << lo;
        if (diag >= c0 && diag < c0 + 32) wm &= ~(1u << (diag - c0));
        // screen against the current last entry (ties pass; the offer decides)
        const float td = L.d[KP - 1];
        int m = 0;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const float2 e = snid[c0 + jj];
          const float d2 = np_ + e.x - 2.0f * __uint_as_float(v[jj]);
          // branch-free: always write slot m, keep it only on a hit (m <= jj,
          // so 32 slots suffice)
          mybd[m * 256] = d2;
          mybi[m * 256] = __float_as_uint(e.y);
          m += (((wm >> jj) & 1u) && d2 <= td) ? 1 : 0;
        }
#pragma unroll 1
        for (int u = 0; u < m; ++u) L.offer(mybd[u * 256], mybi[u * 256]);
      }
      if (rowok) L.store(a.ldist + (size_t)ip * KP, a.lidx + (size_t)ip * KP);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&S.tempty[buf]);
        mbar_arrive(&S.mempty[sl]);
      }
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
// empty slots stay (+inf, 0xffffffff).
template <int KP>
__global__ void __launch_bounds__(256, 6) rerank_kernel(const float* __restrict__ x, int64_t n, int d,
                                                     const uint32_t* __restrict__ order, int vec4,
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
    id[u] = 32 * u + lane < KP ? lidx[(size_t)i * KP + 32 * u + lane] : 0xffffffffu;
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

size_t gram_smem(int N, int dp) {
  (void)dp;
  return (size_t)STAGES * N * 128 + (size_t)NSLOT * (N + 32) * 8 + (size_t)256 * 32 * 8 + sizeof(PersistSmem) + 1024;
}

template <int KP>
int launch_gram_kp(const GramArgs& a, size_t smem, cudaStream_t s) {
  if (cudaFuncSetAttribute((const void*)gram_window_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return HF_ECUDA;
  int sms = 152;
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = (a.n + GB - 1) / GB;
  const unsigned grid = (unsigned)(ntiles < sms ? ntiles : sms);
  gram_window_kernel<KP><<<grid, PT, smem, s>>>(a);
  hf_after_launch("gram_window_kernel", s);
  return HF_OK;
}

}  // namespace

int gram_supported(int d, int w) {
  const int dp = (d + KC - 1) / KC * KC;
  const int W8 = (w + 7) / 8 * 8;
  const int N = GB + 2 * W8;
  return W8 <= 64 && N * 8 <= 16 * LW * 32 && gram_smem(N, dp) <= 220 * 1024;
}

void launch_prepare_bf16(const float* x, int64_t n, int d, void* xb, float* nrm, cudaStream_t s) {
  const int dp = (d + KC - 1) / KC * KC;
  prepare_bf16_kernel<<<hf_blocks(n * 32, 256, 152 * 16), 256, 0, s>>>(x, n, d, dp,
                                                                      static_cast<__nv_bfloat16*>(xb), nrm);
  hf_after_launch("prepare_bf16_kernel", s);
}

size_t bf16_pitch(int d) { return (size_t)(d + KC - 1) / KC * KC; }

int launch_gram_window(const void* xb, const float* nrm, int64_t n, int d, const uint32_t* sigma, int w, int kp,
                       uint32_t* li, float* ld, int* err, cudaStream_t s) {
  GramArgs a;
  a.xb = static_cast<const __nv_bfloat16*>(xb);
  a.nrm = nrm;
  a.sigma = sigma;
  a.n = n;
  a.dp = (int)bf16_pitch(d);
  a.w = w;
  a.W8 = (w + 7) / 8 * 8;
  a.N = GB + 2 * a.W8;
  // kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
  // K-major, N >> 3 at bit 17, M >> 4 at bit 24
  a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(a.N >> 3) << 17) | ((uint32_t)(GB >> 4) << 24);
  a.lidx = li;
  a.ldist = ld;
  a.err = err;
  a.spin_limit = 2000000000ull;  // 2 s per wait (globaltimer nanoseconds)
  // one block per SM (it holds all 512 tensor-memory columns): each block asks
  // for more than half of the SM's shared memory
  size_t smem = gram_smem(a.N, a.dp);
  if (smem < 120 * 1024) smem = 120 * 1024;
  switch (kp) {
    case 16: return launch_gram_kp<16>(a, smem, s);
    case 32: return launch_gram_kp<32>(a, smem, s);
    case 64: return launch_gram_kp<64>(a, smem, s);
    default: return HF_EINVAL;
  }
}

int launch_rerank(const float* x, int64_t n, int d, const uint32_t* order, int kp, uint32_t* li, float* ld,
                  cudaStream_t s) {
  const unsigned blocks = hf_blocks(n * 32, 256);
  const int vec4 = d % 4 == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  switch (kp) {
    case 16: rerank_kernel<16><<<blocks, 256, 0, s>>>(x, n, d, order, vec4, li, ld); break;
    case 32: rerank_kernel<32><<<blocks, 256, 0, s>>>(x, n, d, order, vec4, li, ld); break;
    case 64: rerank_kernel<64><<<blocks, 256, 0, s>>>(x, n, d, order, vec4, li, ld); break;
    default: return HF_EINVAL;
  }
  hf_after_launch("rerank_kernel", s);
  return HF_OK;
}
