// Learned per-point budget: labels from the forest, a small MLP trained and
// run on the tensor cores, and per-tree windows for the band kernel.
//
// The paper's method spends one budget (the number of sorts and the window
// around each position, Algorithm 2) on every point; its Table 2 trades
// recall against that budget. Points differ in how much of it they need: a
// point in a small, well separated cluster finds its neighbours in a narrow
// window of few orders, one inside a large cluster needs many wide ones. This
// unit learns that need from the coordinates:
//   labels  for each point of a sample, the cheapest (T, w) on a grid at
//           which at least `min_hits` of its k exact neighbours lie within w
//           positions of it in one of the first T orders (label_kernel);
//   model   an MLP d -> 256 -> 256 -> 2 with GELU, BF16 weights and
//           activations, FP32 accumulation on tcgen05, predicting
//           (log2 w, log2 T); trained with Adam on a mean squared error by
//           the forward and backward kernels below;
//   use     per tree t, point i takes part with window w_i while t < T_i
//           (tree_budget_kernel): the band kernel gets each point's window
//           and each tile's largest one, so tiles of easy points do less
//           work and tiles whose points are all done are skipped.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <string.h>

#include <vector>

#include "hf_internal.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace tcx;

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ---------------------------------------------------------------------------
// GEMM on the tensor cores: C = A B^T (+ bias, GELU) for the MLP.
// A: M x K BF16 (row pitch lda), B: N x K BF16 (pitch ldb), both K-major;
// M a multiple of 128, K of 64, N of 16. One block of 128 threads per
// 128 x nt tile: per 64-wide K chunk the A and B rows are staged in the
// 128-byte-swizzled layout (cp.async), one thread issues four K = 16 MMAs
// into the tensor-memory accumulator and commits them to a barrier that
// every thread waits on (bounded) before the next chunk; the epilogue reads
// the accumulator (warp w: rows 32 w .. 32 w + 31) 16 columns at a time.
// ---------------------------------------------------------------------------
// EPI_SIGN: bit j of row m = (C[m][j] > 0), 16 bits per uint16 of the
// output row (the sketch of the second stage); C is the uint16 output and
// ldc its row pitch in uint16 units.
enum { EPI_STORE = 0, EPI_BIAS_GELU = 1, EPI_BIAS = 2, EPI_SIGN = 3 };

struct GemmArgs {
  const __nv_bfloat16* A;
  const __nv_bfloat16* B;
  int lda, ldb, M, N, K, nt;
  float* C;  // fp32 result (the pre-activation in EPI_BIAS_GELU)
  int ldc;
  const float* bias;   // [N]
  __nv_bfloat16* H;    // GELU(C) in BF16 (EPI_BIAS_GELU)
  int ldh;
  int* err;
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
// d/dz of z Phi(z) = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_grad(float z) {
  const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * __expf(-0.5f * z * z);
  return cdf + z * pdf;
}

template <int EPI>
__global__ void __launch_bounds__(128, 1) mlp_gemm_kernel(GemmArgs g) {
  extern __shared__ unsigned char smraw[];
  unsigned char* base = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
  unsigned char* sa = base;           // 128 rows x 128 bytes
  unsigned char* sb = base + 16384;   // nt rows x 128 bytes
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * g.nt;
  const int nt = min(g.nt, g.N - n0);
  const uint32_t tcols = nt <= 32 ? 32u : (nt <= 64 ? 64u : (nt <= 128 ? 128u : 256u));
  if (warp == 0) tmem_alloc(&tslot, tcols);
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tslot;
  // FP32 accumulator, BF16 A and B, both K-major; N >> 3 at bit 17, M >> 4 at 24
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  const int nk = g.K / 64;
  bool ok = true;
  for (int kc = 0; kc < nk && ok; ++kc) {
    const uint32_t da = smem_u32(sa), db = smem_u32(sb);
    for (int e = tid; e < 128 * 8; e += 128) {
      const int r = e >> 3, pc = e & 7;
      const bool v = m0 + r < g.M;
      cp_async16(da + swz(r, pc), g.A + (size_t)(v ? m0 + r : 0) * g.lda + kc * 64 + pc * 8, v);
    }
    for (int e = tid; e < nt * 8; e += 128) {
      const int r = e >> 3, pc = e & 7;
      cp_async16(db + swz(r, pc), g.B + (size_t)(n0 + r) * g.ldb + kc * 64 + pc * 8, true);
    }
    cp_async_wait_all();
    fence_proxy_async_smem();  // the copies (generic proxy) are read by the tensor core
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        mma_bf16(tmem, smem_desc(da + ks * 32), smem_desc(db + ks * 32), idesc, (kc | ks) != 0);
      mma_commit(&bar);
    }
    // the chunk's MMAs must be done before the tiles are overwritten (and
    // before the epilogue): a bounded wait (2 s), agreed by all threads
    bool done = mbar_try_wait(&bar, kc & 1);
    if (!done) {
      const uint64_t t0 = gtimer();
      while (!(done = mbar_try_wait(&bar, kc & 1)) && gtimer() - t0 < 2000000000ull) {
      }
    }
    ok = !__syncthreads_or(!done);
    tc_fence_after();
  }
  if (!ok) {
    if (tid == 0) hf_raise(g.err, HF_ERRBIT_TIMEOUT);
  } else {
    const int m = m0 + warp * 32 + lane;
    for (int c = 0; c < nt; c += 16) {
      uint32_t v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      if (m < g.M && EPI == EPI_SIGN) {
        uint32_t bitsv = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) bitsv |= (__uint_as_float(v[j]) > 0.f ? 1u : 0u) << j;
        reinterpret_cast<uint16_t*>(g.C)[(size_t)m * g.ldc + (n0 + c) / 16] = (uint16_t)bitsv;
      } else if (m < g.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int n = n0 + c + j;
          float z = __uint_as_float(v[j]);
          if (EPI != EPI_STORE) z += g.bias[n];
          g.C[(size_t)m * g.ldc + n] = z;
          if (EPI == EPI_BIAS_GELU) g.H[(size_t)m * g.ldh + n] = __float2bfloat16_rn(gelu(z));
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, tcols);
  }
}

constexpr size_t GEMM_SMEM = 16384 + 256 * 128 + 1024;

template <int EPI>
int gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K, int nt, float* C,
         int ldc, const float* bias, __nv_bfloat16* H, int ldh, int* err, cudaStream_t s) {
  if (M < 1 || K % 64 || N % 16 || nt % 16 || nt > 256 || N % nt) return HF_EINVAL;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute((const void*)mlp_gemm_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)GEMM_SMEM) != cudaSuccess)
      return HF_ECUDA;
    attr = true;
  }
  GemmArgs g{A, B, lda, ldb, M, N, K, nt, C, ldc, bias, H, ldh, err};
  mlp_gemm_kernel<EPI><<<dim3((M + 127) / 128, N / nt), 128, GEMM_SMEM, s>>>(g);
  hf_after_launch("mlp_gemm_kernel", s);
  return HF_OK;
}

// ---------------------------------------------------------------------------
// Elementwise and layout kernels of the training step
// ---------------------------------------------------------------------------
// dst[c][r] = src[r][c] for r < R, c < C (BF16); dst row pitch ldd, rows of
// dst up to Cpad and columns up to Rpad are zero-filled.
__global__ void transpose_bf16_kernel(const __nv_bfloat16* __restrict__ src, int lds, int R, int C,
                                      __nv_bfloat16* __restrict__ dst, int ldd, int Rpad, int Cpad) {
  __shared__ __nv_bfloat16 tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < R && c < C) ? src[(size_t)r * lds + c] : __float2bfloat16_rn(0.f);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < Cpad && r < Rpad) dst[(size_t)c * ldd + r] = tile[threadIdx.x][i];
  }
}

// Mean squared error over the 2 outputs: L = 1/(2B) sum (y - t)^2;
// dY = (y - t) / B as BF16 in dy [B][64] (columns >= 2 zero) and its
// transpose dyt [128][B] (rows >= 2 zero); db3 += column sums; loss += L.
__global__ void loss_grad_kernel(const float* __restrict__ y, int ldy, const float* __restrict__ tgt, int B,
                                 __nv_bfloat16* __restrict__ dy, __nv_bfloat16* __restrict__ dyt, float* db3,
                                 float* loss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  float g0 = 0.f, g1 = 0.f, l = 0.f;
  if (b < B) {
    const float e0 = y[(size_t)b * ldy] - tgt[2 * b], e1 = y[(size_t)b * ldy + 1] - tgt[2 * b + 1];
    g0 = e0 / B;
    g1 = e1 / B;
    l = 0.5f * (e0 * e0 + e1 * e1) / B;
    for (int c = 0; c < 64; ++c) dy[(size_t)b * 64 + c] = __float2bfloat16_rn(c == 0 ? g0 : (c == 1 ? g1 : 0.f));
    dyt[b] = __float2bfloat16_rn(g0);
    dyt[(size_t)B + b] = __float2bfloat16_rn(g1);
    for (int r = 2; r < 128; ++r) dyt[(size_t)r * B + b] = __float2bfloat16_rn(0.f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    g0 += __shfl_xor_sync(0xffffffffu, g0, o);
    g1 += __shfl_xor_sync(0xffffffffu, g1, o);
    l += __shfl_xor_sync(0xffffffffu, l, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(db3, g0);
    atomicAdd(db3 + 1, g1);
    atomicAdd(loss, l);
  }
}

// dZ = dH * gelu'(Z) (dH, Z: [B][H] fp32): dz as BF16 [B][H] and transposed
// dzt [H][B]; db += column sums of the unrounded dZ. Block: 32 x 8 threads
// over a 32 x 32 tile.
__global__ void gelu_back_kernel(const float* __restrict__ dh, const float* __restrict__ z, int B, int H,
                                 __nv_bfloat16* __restrict__ dz, __nv_bfloat16* __restrict__ dzt, float* db) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  float colsum = 0.f;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    float v = 0.f;
    if (r < B && c < H) {
      v = dh[(size_t)r * H + c] * gelu_grad(z[(size_t)r * H + c]);
      dz[(size_t)r * H + c] = __float2bfloat16_rn(v);
    }
    tile[i][threadIdx.x] = v;
    colsum += v;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (c < H && r < B) dzt[(size_t)c * B + r] = __float2bfloat16_rn(tile[threadIdx.x][i]);
  }
  if (c0 + (int)threadIdx.x < H) atomicAdd(db + c0 + threadIdx.x, colsum);
}

// Adam step on one parameter tensor (fp32 master w, moments m, v, gradient
// g of `rows x cols`, gradient row pitch ldg); the BF16 copy wb [rows][cols]
// and, when wt is set, the transposed BF16 copy wt [cols][ldt] (rows padded
// with zeros up to ldt) are refreshed.
__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int ldg, int rows, int cols, float lr, float b1, float b2,
                            float eps, float c1, float c2, __nv_bfloat16* __restrict__ wb,
                            __nv_bfloat16* __restrict__ wt, int ldt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int r = e / cols, c = e % cols;
  const float gr = g[(size_t)r * ldg + c];
  const float mm = b1 * m[e] + (1.f - b1) * gr;
  const float vv = b2 * v[e] + (1.f - b2) * gr * gr;
  m[e] = mm;
  v[e] = vv;
  const float ww = w[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  w[e] = ww;
  if (wb) wb[e] = __float2bfloat16_rn(ww);
  if (wt) wt[(size_t)c * ldt + r] = __float2bfloat16_rn(ww);
}

__global__ void accumulate_kernel(float* acc, const float* v) { *acc += *v; }

__global__ void f32_to_bf16_kernel(const float* __restrict__ x, int64_t rows, int cols, int ld,
                                   __nv_bfloat16* __restrict__ out, int ldo) {
  const int64_t total = rows * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ld;
    const int c = (int)(e - r * ld);
    out[(size_t)r * ldo + c] = __float2bfloat16_rn(c < cols ? x[(size_t)r * cols + c] : 0.f);
  }
}

// ---------------------------------------------------------------------------
// Labels and per-tree budgets
// ---------------------------------------------------------------------------
__global__ void inverse_order_kernel(const uint32_t* __restrict__ sigma, int64_t n, int32_t* __restrict__ pos) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    pos[sigma[p]] = (int32_t)p;
}

constexpr int MAX_GRID = 16;

// One thread per point i: for each exact neighbour e (knn [n][k], -1 = none)
// the smallest position gap |p_t(i) - p_t(e)| over the first T trees, for
// each T of the grid; then the cheapest cell (cost T (128 + 2 w)) of the
// (T, w) grid at which at least min_hits neighbours are within w, else the
// last (largest) cell. Writes (log2 w, log2 T) and the cell index.
__global__ void label_kernel(const int32_t* __restrict__ pos, int64_t n, const int32_t* __restrict__ knn, int k,
                             const int32_t* __restrict__ tg, int ntg, const int32_t* __restrict__ wg, int nwg,
                             int min_hits, float* __restrict__ out, int32_t* __restrict__ cell) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int hits[MAX_GRID][MAX_GRID];
  for (int a = 0; a < ntg; ++a)
    for (int b = 0; b < nwg; ++b) hits[a][b] = 0;
  for (int j = 0; j < k; ++j) {
    const int32_t e = knn[i * k + j];
    if (e < 0) continue;
    int gmin = 0x7fffffff, t = 0;
    for (int a = 0; a < ntg; ++a) {
      for (; t < tg[a]; ++t) {
        const int g = abs(pos[(size_t)t * n + i] - pos[(size_t)t * n + e]);
        gmin = g < gmin ? g : gmin;
      }
      for (int b = 0; b < nwg; ++b) hits[a][b] += gmin <= wg[b] ? 1 : 0;
    }
  }
  int best = ntg * nwg - 1;
  double bc = 1e300;
  for (int a = 0; a < ntg; ++a)
    for (int b = 0; b < nwg; ++b) {
      const double c = (double)tg[a] * (128.0 + 2.0 * wg[b]);
      if (hits[a][b] >= min_hits && c < bc) {
        bc = c;
        best = a * nwg + b;
      }
    }
  cell[i] = best;
  out[2 * i] = log2f((float)wg[best % nwg]);
  out[2 * i + 1] = log2f((float)tg[best / nwg]);
}

// Tree t: point i takes part with window w_i while t < T_i. pw[i] gets its
// window (0: not this tree); tile_w[tile] the largest over the tile's 128
// positions. One block of 128 threads per tile.
__global__ void tree_budget_kernel(const uint32_t* __restrict__ sigma, int64_t n, int t,
                                   const int32_t* __restrict__ wpt, const int32_t* __restrict__ tpt,
                                   uint16_t* __restrict__ pw, int32_t* __restrict__ tile_w) {
  __shared__ int red[4];
  const int64_t p = (int64_t)blockIdx.x * 128 + threadIdx.x;
  int wr = 0;
  if (p < n) {
    const uint32_t id = sigma[p];
    wr = t < tpt[id] ? min(wpt[id], 65535) : 0;
    pw[id] = (uint16_t)wr;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wr = max(wr, __shfl_xor_sync(0xffffffffu, wr, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = wr;
  __syncthreads();
  if (threadIdx.x == 0) tile_w[blockIdx.x] = max(max(red[0], red[1]), max(red[2], red[3]));
}

}  // namespace

// ---------------------------------------------------------------------------
// The model
// ---------------------------------------------------------------------------
struct hf_mlp {
  int d = 0, dp = 0;  // input dimension and its pitch (a multiple of 64)
  int device = 0;
  static constexpr int H = 256, OUTP = 16;  // hidden width; padded output rows
  // fp32 masters, Adam moments, BF16 copies (W [out][in]) and transposes
  float *w1 = nullptr, *b1 = nullptr, *w2 = nullptr, *b2 = nullptr, *w3 = nullptr, *b3 = nullptr;
  float* mom = nullptr;  // m and v of all parameters
  __nv_bfloat16 *w1b = nullptr, *w2b = nullptr, *w2t = nullptr, *w3b = nullptr, *w3t = nullptr;
  int64_t nparam = 0;
  int step = 0;
  int* err = nullptr;
  // batch scratch
  int bcap = 0;
  __nv_bfloat16 *xb = nullptr, *xt = nullptr, *h1 = nullptr, *h1t = nullptr, *h2 = nullptr, *h2t = nullptr;
  __nv_bfloat16 *dy = nullptr, *dyt = nullptr, *dz2 = nullptr, *dz2t = nullptr, *dz1 = nullptr, *dz1t = nullptr;
  float *z1 = nullptr, *z2 = nullptr, *y = nullptr, *dh2 = nullptr, *dh1 = nullptr, *tgt = nullptr;
  float* grad = nullptr;  // dW1, db1, dW2, db2, dW3 (128 rows), db3
  float* loss = nullptr;
};

namespace {

int64_t mlp_param_count(int d) {
  return (int64_t)256 * d + 256 + 256 * 256 + 256 + (int64_t)hf_mlp::OUTP * 256 + hf_mlp::OUTP;
}

void mlp_free_batch(hf_mlp* m) {
  void* ptrs[] = {m->xb, m->xt, m->h1, m->h1t, m->h2, m->h2t, m->dy, m->dyt, m->dz2, m->dz2t, m->dz1, m->dz1t,
                  m->z1, m->z2, m->y, m->dh2, m->dh1, m->tgt, m->grad, m->loss};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  m->xb = m->xt = m->h1 = m->h1t = m->h2 = m->h2t = m->dy = m->dyt = m->dz2 = m->dz2t = m->dz1 = m->dz1t = nullptr;
  m->z1 = m->z2 = m->y = m->dh2 = m->dh1 = m->tgt = m->grad = m->loss = nullptr;
  m->bcap = 0;
}

// Batch buffers for up to B rows (B a multiple of 128).
int mlp_reserve(hf_mlp* m, int B) {
  if (B <= m->bcap) return HF_OK;
  mlp_free_batch(m);
  const int H = hf_mlp::H;
  bool ok = true;
  auto take = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) ok = false;
  };
  take((void**)&m->xb, (size_t)B * m->dp * 2);
  take((void**)&m->xt, (size_t)m->dp * B * 2);
  take((void**)&m->h1, (size_t)B * H * 2);
  take((void**)&m->h1t, (size_t)H * B * 2);
  take((void**)&m->h2, (size_t)B * H * 2);
  take((void**)&m->h2t, (size_t)H * B * 2);
  take((void**)&m->dy, (size_t)B * 64 * 2);
  take((void**)&m->dyt, (size_t)128 * B * 2);
  take((void**)&m->dz2, (size_t)B * H * 2);
  take((void**)&m->dz2t, (size_t)H * B * 2);
  take((void**)&m->dz1, (size_t)B * H * 2);
  take((void**)&m->dz1t, (size_t)H * B * 2);
  take((void**)&m->z1, (size_t)B * H * 4);
  take((void**)&m->z2, (size_t)B * H * 4);
  take((void**)&m->y, (size_t)B * hf_mlp::OUTP * 4);
  take((void**)&m->dh2, (size_t)B * H * 4);
  take((void**)&m->dh1, (size_t)B * H * 4);
  take((void**)&m->tgt, (size_t)B * 2 * 4);
  take((void**)&m->grad, (size_t)(H * m->dp + H + H * H + H + 128 * H + hf_mlp::OUTP) * 4);
  take((void**)&m->loss, 4);
  if (!ok) {
    cudaGetLastError();
    mlp_free_batch(m);
    return HF_ENOMEM;
  }
  m->bcap = B;
  return HF_OK;
}

// Gradient layout inside m->grad: dW1 [256][dp], db1 [256], dW2 [256][256],
// db2 [256], dW3 [128][256] (rows >= 2 zero), db3 [16].
struct GradView {
  float *w1, *b1, *w2, *b2, *w3, *b3;
};
GradView grad_view(hf_mlp* m) {
  GradView g;
  g.w1 = m->grad;
  g.b1 = g.w1 + (size_t)256 * m->dp;
  g.w2 = g.b1 + 256;
  g.b2 = g.w2 + 256 * 256;
  g.w3 = g.b2 + 256;
  g.b3 = g.w3 + 128 * 256;
  return g;
}

// Input rows x (fp32, row pitch d) -> m->xb (BF16, pitch dp, zero padded),
// rows [B0, B) zero.
void stage_input(hf_mlp* m, const float* x, int rows, int B, cudaStream_t s) {
  f32_to_bf16_kernel<<<hf_blocks((int64_t)rows * m->dp, 256, 152 * 8), 256, 0, s>>>(x, rows, m->d, m->dp, m->xb,
                                                                                    m->dp);
  hf_after_launch("f32_to_bf16_kernel", s);
  if (B > rows) cudaMemsetAsync(m->xb + (size_t)rows * m->dp, 0, (size_t)(B - rows) * m->dp * 2, s);
}

int mlp_forward_batch(hf_mlp* m, int B, cudaStream_t s) {
  const int H = hf_mlp::H;
  int rc = gemm<EPI_BIAS_GELU>(m->xb, m->dp, m->w1b, m->dp, B, H, m->dp, 256, m->z1, H, m->b1, m->h1, H, m->err, s);
  if (rc == HF_OK)
    rc = gemm<EPI_BIAS_GELU>(m->h1, H, m->w2b, H, B, H, H, 256, m->z2, H, m->b2, m->h2, H, m->err, s);
  if (rc == HF_OK)
    rc = gemm<EPI_BIAS>(m->h2, H, m->w3b, H, B, hf_mlp::OUTP, H, 16, m->y, hf_mlp::OUTP, m->b3, nullptr, 0, m->err,
                        s);
  return rc;
}

void transpose(const __nv_bfloat16* src, int lds, int R, int C, __nv_bfloat16* dst, int ldd, int Rpad, int Cpad,
               cudaStream_t s) {
  dim3 grid((Cpad + 31) / 32, (Rpad + 31) / 32);
  transpose_bf16_kernel<<<grid, dim3(32, 8), 0, s>>>(src, lds, R, C, dst, ldd, Rpad, Cpad);
  hf_after_launch("transpose_bf16_kernel", s);
}

// Gradients of the batch's loss into m->grad (forward included).
int mlp_backward_batch(hf_mlp* m, int B, cudaStream_t s) {
  const int H = hf_mlp::H;
  const GradView gv = grad_view(m);
  int rc = mlp_forward_batch(m, B, s);
  if (rc != HF_OK) return rc;
  cudaMemsetAsync(m->grad, 0, (size_t)(H * m->dp + H + H * H + H + 128 * H + hf_mlp::OUTP) * 4, s);
  cudaMemsetAsync(m->loss, 0, 4, s);
  transpose(m->xb, m->dp, B, m->dp, m->xt, B, B, m->dp, s);
  transpose(m->h1, H, B, H, m->h1t, B, B, H, s);
  transpose(m->h2, H, B, H, m->h2t, B, B, H, s);
  loss_grad_kernel<<<(B + 127) / 128, 128, 0, s>>>(m->y, hf_mlp::OUTP, m->tgt, B, m->dy, m->dyt, gv.b3, m->loss);
  hf_after_launch("loss_grad_kernel", s);
  // layer 3: dW3 = dY^T H2, dH2 = dY W3
  rc = gemm<EPI_STORE>(m->dyt, B, m->h2t, B, 128, H, B, 256, gv.w3, H, nullptr, nullptr, 0, m->err, s);
  if (rc == HF_OK) rc = gemm<EPI_STORE>(m->dy, 64, m->w3t, 64, B, H, 64, 256, m->dh2, H, nullptr, nullptr, 0, m->err, s);
  if (rc != HF_OK) return rc;
  const dim3 eg(H / 32, B / 32), eb(32, 8);
  gelu_back_kernel<<<eg, eb, 0, s>>>(m->dh2, m->z2, B, H, m->dz2, m->dz2t, gv.b2);
  hf_after_launch("gelu_back_kernel", s);
  // layer 2: dW2 = dZ2^T H1, dH1 = dZ2 W2
  rc = gemm<EPI_STORE>(m->dz2t, B, m->h1t, B, H, H, B, 256, gv.w2, H, nullptr, nullptr, 0, m->err, s);
  if (rc == HF_OK) rc = gemm<EPI_STORE>(m->dz2, H, m->w2t, H, B, H, H, 256, m->dh1, H, nullptr, nullptr, 0, m->err, s);
  if (rc != HF_OK) return rc;
  gelu_back_kernel<<<eg, eb, 0, s>>>(m->dh1, m->z1, B, H, m->dz1, m->dz1t, gv.b1);
  hf_after_launch("gelu_back_kernel", s);
  // layer 1: dW1 = dZ1^T X
  const int nt1 = m->dp % 256 == 0 ? 256 : (m->dp % 128 == 0 ? 128 : 64);
  return gemm<EPI_STORE>(m->dz1t, B, m->xt, B, H, m->dp, B, nt1, gv.w1, m->dp, nullptr, nullptr, 0, m->err, s);
}

void mlp_adam(hf_mlp* m, float lr, cudaStream_t s) {
  const int H = hf_mlp::H;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  m->step += 1;
  const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
  const GradView gv = grad_view(m);
  float* mm = m->mom;
  float* vv = m->mom + m->nparam;
  int64_t off = 0;
  auto one = [&](float* w, const float* g, int ldg, int rows, int cols, __nv_bfloat16* wb, __nv_bfloat16* wt,
                 int ldt) {
    const int cnt = rows * cols;
    adam_kernel<<<(cnt + 255) / 256, 256, 0, s>>>(w, mm + off, vv + off, g, ldg, rows, cols, lr, b1, b2, eps, c1, c2,
                                                   wb, wt, ldt);
    hf_after_launch("adam_kernel", s);
    off += cnt;
  };
  one(m->w1, gv.w1, m->dp, H, m->dp, m->w1b, nullptr, 0);
  one(m->b1, gv.b1, H, 1, H, nullptr, nullptr, 0);
  one(m->w2, gv.w2, H, H, H, m->w2b, m->w2t, H);
  one(m->b2, gv.b2, H, 1, H, nullptr, nullptr, 0);
  one(m->w3, gv.w3, H, 2, H, m->w3b, m->w3t, 64);  // rows 2..15 stay zero
  one(m->b3, gv.b3, hf_mlp::OUTP, 1, 2, nullptr, nullptr, 0);
}

// splitmix64-driven uniform initialisation (fan-in scaled), on the host.
uint64_t sm64(uint64_t& s) {
  s += 0x9E3779B97F4A7C15ull;
  uint64_t z = s;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int hf_mlp_create(int32_t d, uint64_t seed, hf_mlp** out) {
  if (!out) return HF_EINVAL;
  *out = nullptr;
  if (d < 1 || d > HF_MAX_D) return HF_EINVAL;
  hf_mlp* m = new hf_mlp();
  m->d = d;
  m->dp = (d + 63) / 64 * 64;
  cudaGetDevice(&m->device);
  const int H = hf_mlp::H;
  m->nparam = mlp_param_count(m->dp);
  // host initial values: W ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)), b = 0
  std::vector<float> hw1((size_t)H * m->dp, 0.f), hw2((size_t)H * H), hw3((size_t)hf_mlp::OUTP * H, 0.f);
  uint64_t st = seed;
  auto uni = [&](float a) { return (float)(((sm64(st) >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0) * a; };
  for (int o = 0; o < H; ++o)
    for (int i = 0; i < d; ++i) hw1[(size_t)o * m->dp + i] = uni(1.f / sqrtf((float)d));
  for (auto& v : hw2) v = uni(1.f / 16.f);
  for (int o = 0; o < 2; ++o)
    for (int i = 0; i < H; ++i) hw3[(size_t)o * H + i] = uni(1.f / 16.f);
  bool ok = true;
  auto take = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false;
  };
  take((void**)&m->w1, hw1.size() * 4);
  take((void**)&m->b1, H * 4);
  take((void**)&m->w2, hw2.size() * 4);
  take((void**)&m->b2, H * 4);
  take((void**)&m->w3, hw3.size() * 4);
  take((void**)&m->b3, hf_mlp::OUTP * 4);
  take((void**)&m->mom, (size_t)2 * m->nparam * 4);
  take((void**)&m->w1b, hw1.size() * 2);
  take((void**)&m->w2b, hw2.size() * 2);
  take((void**)&m->w2t, hw2.size() * 2);
  take((void**)&m->w3b, hw3.size() * 2);
  take((void**)&m->w3t, (size_t)H * 64 * 2);
  take((void**)&m->err, 4);
  if (!ok) {
    cudaGetLastError();
    hf_mlp_free(m);
    return HF_ENOMEM;
  }
  cudaMemcpy(m->w1, hw1.data(), hw1.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(m->w2, hw2.data(), hw2.size() * 4, cudaMemcpyHostToDevice);
  cudaMemcpy(m->w3, hw3.data(), hw3.size() * 4, cudaMemcpyHostToDevice);
  cudaMemset(m->b1, 0, H * 4);
  cudaMemset(m->b2, 0, H * 4);
  cudaMemset(m->b3, 0, hf_mlp::OUTP * 4);
  cudaMemset(m->mom, 0, (size_t)2 * m->nparam * 4);
  cudaMemset(m->w3t, 0, (size_t)H * 64 * 2);
  cudaMemset(m->err, 0, 4);
  *out = m;
  return hf_mlp_set_params(m, nullptr);
}

int hf_mlp_free(hf_mlp* m) {
  if (!m) return HF_OK;
  cudaDeviceSynchronize();
  mlp_free_batch(m);
  void* ptrs[] = {m->w1, m->b1, m->w2, m->b2, m->w3, m->b3, m->mom, m->w1b, m->w2b, m->w2t, m->w3b, m->w3t, m->err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete m;
  return HF_OK;
}

int hf_mlp_param_count(const hf_mlp* m, int64_t* out) {
  if (!m || !out) return HF_EINVAL;
  *out = (int64_t)256 * m->d + 256 + 256 * 256 + 256 + 2 * 256 + 2;
  return HF_OK;
}

// Packed parameter order (host floats): W1 [256][d], b1 [256], W2 [256][256],
// b2 [256], W3 [2][256], b3 [2].
int hf_mlp_get_params(const hf_mlp* m, float* out) {
  if (!m || !out) return HF_EINVAL;
  const int H = hf_mlp::H, d = m->d, dp = m->dp;
  std::vector<float> w1((size_t)H * dp);
  if (cudaMemcpy(w1.data(), m->w1, w1.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return HF_ECUDA;
  float* o = out;
  for (int r = 0; r < H; ++r) memcpy(o + (size_t)r * d, w1.data() + (size_t)r * dp, (size_t)d * 4);
  o += (size_t)H * d;
  cudaMemcpy(o, m->b1, H * 4, cudaMemcpyDeviceToHost);
  o += H;
  cudaMemcpy(o, m->w2, (size_t)H * H * 4, cudaMemcpyDeviceToHost);
  o += H * H;
  cudaMemcpy(o, m->b2, H * 4, cudaMemcpyDeviceToHost);
  o += H;
  cudaMemcpy(o, m->w3, (size_t)2 * H * 4, cudaMemcpyDeviceToHost);
  o += 2 * H;
  return cudaMemcpy(o, m->b3, 2 * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? HF_OK : HF_ECUDA;
}

// Sets the fp32 masters (params in the packed order; NULL keeps them) and
// refreshes the BF16 copies and transposes.
int hf_mlp_set_params(hf_mlp* m, const float* params) {
  if (!m) return HF_EINVAL;
  const int H = hf_mlp::H, d = m->d, dp = m->dp;
  std::vector<float> w1((size_t)H * dp, 0.f), w2((size_t)H * H), w3((size_t)hf_mlp::OUTP * H, 0.f), b1(H), b2(H),
      b3(hf_mlp::OUTP, 0.f);
  if (params) {
    const float* p = params;
    for (int r = 0; r < H; ++r) memcpy(w1.data() + (size_t)r * dp, p + (size_t)r * d, (size_t)d * 4);
    p += (size_t)H * d;
    memcpy(b1.data(), p, H * 4);
    p += H;
    memcpy(w2.data(), p, (size_t)H * H * 4);
    p += H * H;
    memcpy(b2.data(), p, H * 4);
    p += H;
    memcpy(w3.data(), p, (size_t)2 * H * 4);
    p += 2 * H;
    memcpy(b3.data(), p, 2 * 4);
    cudaMemcpy(m->w1, w1.data(), w1.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(m->b1, b1.data(), H * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(m->w2, w2.data(), w2.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(m->b2, b2.data(), H * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(m->w3, w3.data(), w3.size() * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(m->b3, b3.data(), hf_mlp::OUTP * 4, cudaMemcpyHostToDevice);
  } else {
    cudaMemcpy(w1.data(), m->w1, w1.size() * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(w2.data(), m->w2, w2.size() * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(w3.data(), m->w3, w3.size() * 4, cudaMemcpyDeviceToHost);
  }
  // BF16 copies (round to nearest even) and transposes
  auto bf = [](float f) { return __float2bfloat16_rn(f); };
  std::vector<__nv_bfloat16> a(w1.size()), b(w2.size()), bt(w2.size()), c(w3.size()), ct((size_t)H * 64, bf(0.f));
  for (size_t i = 0; i < w1.size(); ++i) a[i] = bf(w1[i]);
  for (int o = 0; o < H; ++o)
    for (int i = 0; i < H; ++i) {
      b[(size_t)o * H + i] = bf(w2[(size_t)o * H + i]);
      bt[(size_t)i * H + o] = b[(size_t)o * H + i];
    }
  for (size_t i = 0; i < w3.size(); ++i) c[i] = bf(w3[i]);
  for (int o = 0; o < 2; ++o)
    for (int i = 0; i < H; ++i) ct[(size_t)i * 64 + o] = c[(size_t)o * H + i];
  cudaMemcpy(m->w1b, a.data(), a.size() * 2, cudaMemcpyHostToDevice);
  cudaMemcpy(m->w2b, b.data(), b.size() * 2, cudaMemcpyHostToDevice);
  cudaMemcpy(m->w2t, bt.data(), bt.size() * 2, cudaMemcpyHostToDevice);
  cudaMemcpy(m->w3b, c.data(), c.size() * 2, cudaMemcpyHostToDevice);
  const cudaError_t e = cudaMemcpy(m->w3t, ct.data(), ct.size() * 2, cudaMemcpyHostToDevice);
  return e == cudaSuccess ? HF_OK : HF_ECUDA;
}

int hf_mlp_predict(hf_mlp* m, const float* x, int64_t n, float* out, void* stream) {
  if (!m || !x || !out || n < 0) return HF_EINVAL;
  if (n == 0) return HF_OK;
  if (!on_device(x)) return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  const int B = 8192;
  int rc = mlp_reserve(m, B);
  for (int64_t r0 = 0; r0 < n && rc == HF_OK; r0 += B) {
    const int rows = (int)(n - r0 < B ? n - r0 : B);
    const int Bp = (rows + 127) / 128 * 128;
    stage_input(m, x + (size_t)r0 * m->d, rows, Bp, s);
    rc = mlp_forward_batch(m, Bp, s);
    if (rc == HF_OK && cudaMemcpy2DAsync(out + (size_t)r0 * 2, 8, m->y, hf_mlp::OUTP * 4, 8, rows,
                                         cudaMemcpyDefault, s) != cudaSuccess)
      rc = HF_ECUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return HF_ECUDA;
  int word = 0;
  cudaMemcpy(&word, m->err, 4, cudaMemcpyDeviceToHost);
  if (word) {
    cudaMemset(m->err, 0, 4);
    return HF_ETIMEOUT;
  }
  return rc;
}

// Gradients of L = 1/(2B) sum (y - t)^2 over one batch (B rows, a multiple of
// 128 up to 8192) in the packed parameter order; also the loss.
int hf_mlp_grads(hf_mlp* m, const float* x, const float* targets, int32_t B, float* out_grads, float* out_loss,
                 void* stream) {
  if (!m || !x || !targets || B < 128 || B % 128 || B > 8192) return HF_EINVAL;
  if (!on_device(x)) return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  int rc = mlp_reserve(m, B);
  if (rc != HF_OK) return rc;
  stage_input(m, x, B, B, s);
  cudaMemcpyAsync(m->tgt, targets, (size_t)B * 2 * 4, cudaMemcpyDefault, s);
  rc = mlp_backward_batch(m, B, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return HF_ECUDA;
  if (rc != HF_OK) return rc;
  if (out_loss) cudaMemcpy(out_loss, m->loss, 4, cudaMemcpyDeviceToHost);
  if (out_grads) {
    const int H = hf_mlp::H, d = m->d, dp = m->dp;
    const GradView gv = grad_view(m);
    std::vector<float> g1((size_t)H * dp);
    cudaMemcpy(g1.data(), gv.w1, g1.size() * 4, cudaMemcpyDeviceToHost);
    float* o = out_grads;
    for (int r = 0; r < H; ++r) memcpy(o + (size_t)r * d, g1.data() + (size_t)r * dp, (size_t)d * 4);
    o += (size_t)H * d;
    cudaMemcpy(o, gv.b1, H * 4, cudaMemcpyDeviceToHost);
    o += H;
    cudaMemcpy(o, gv.w2, (size_t)H * H * 4, cudaMemcpyDeviceToHost);
    o += H * H;
    cudaMemcpy(o, gv.b2, H * 4, cudaMemcpyDeviceToHost);
    o += H;
    cudaMemcpy(o, gv.w3, (size_t)2 * H * 4, cudaMemcpyDeviceToHost);
    o += 2 * H;
    cudaMemcpy(o, gv.b3, 2 * 4, cudaMemcpyDeviceToHost);
  }
  int word = 0;
  cudaMemcpy(&word, m->err, 4, cudaMemcpyDeviceToHost);
  if (word) {
    cudaMemset(m->err, 0, 4);
    return HF_ETIMEOUT;
  }
  return cudaGetLastError() == cudaSuccess ? HF_OK : HF_ECUDA;
}

// Trains for `steps` Adam steps on batches of B rows taken in order (with
// wrap-around) from the device-resident training set x (n x d fp32) and
// targets (n x 2); the mean loss of the last `report` steps goes to
// *out_loss.
int hf_mlp_train(hf_mlp* m, const float* x, const float* targets, int64_t n, int32_t B, int32_t steps, float lr,
                 float* out_loss, void* stream) {
  if (!m || !x || !targets || n < B || B < 128 || B % 128 || B > 8192 || steps < 0) return HF_EINVAL;
  if (!on_device(x) || !on_device(targets)) return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  int rc = mlp_reserve(m, B);
  float* lacc = nullptr;
  if (rc == HF_OK && cudaMalloc(&lacc, 4) != cudaSuccess) rc = HF_ENOMEM;
  if (rc != HF_OK) return rc;
  cudaMemsetAsync(lacc, 0, 4, s);
  const int report = steps < 50 ? steps : 50;
  int64_t r0 = 0;
  for (int st = 0; st < steps && rc == HF_OK; ++st) {
    if (r0 + B > n) r0 = 0;
    stage_input(m, x + (size_t)r0 * m->d, B, B, s);
    cudaMemcpyAsync(m->tgt, targets + (size_t)r0 * 2, (size_t)B * 2 * 4, cudaMemcpyDeviceToDevice, s);
    rc = mlp_backward_batch(m, B, s);
    if (rc == HF_OK) mlp_adam(m, lr, s);
    if (rc == HF_OK && st >= steps - report) {
      accumulate_kernel<<<1, 1, 0, s>>>(lacc, m->loss);
      hf_after_launch("accumulate_kernel", s);
    }
    r0 += B;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = HF_ECUDA;
  float lsum = 0.f;
  cudaMemcpy(&lsum, lacc, 4, cudaMemcpyDeviceToHost);
  if (out_loss) *out_loss = report > 0 ? lsum / report : 0.f;
  cudaFree(lacc);
  int word = 0;
  cudaMemcpy(&word, m->err, 4, cudaMemcpyDeviceToHost);
  if (word) {
    cudaMemset(m->err, 0, 4);
    return HF_ETIMEOUT;
  }
  return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Forest-side helpers (called from api.cu)
// ---------------------------------------------------------------------------
int launch_budget_labels(const uint32_t* sigma, int T, int64_t n, const int32_t* knn, int k, const int32_t* tg,
                         int ntg, const int32_t* wg, int nwg, int min_hits, float* out, int32_t* cell, int32_t* pos,
                         cudaStream_t s) {
  if (ntg < 1 || nwg < 1 || ntg > MAX_GRID || nwg > MAX_GRID) return HF_EINVAL;
  for (int t = 0; t < T; ++t) {
    inverse_order_kernel<<<hf_blocks(n, 256, 152 * 8), 256, 0, s>>>(sigma + (size_t)t * n, n, pos + (size_t)t * n);
    hf_after_launch("inverse_order_kernel", s);
  }
  label_kernel<<<hf_blocks(n, 128), 128, 0, s>>>(pos, n, knn, k, tg, ntg, wg, nwg, min_hits, out, cell);
  hf_after_launch("label_kernel", s);
  return HF_OK;
}

void launch_tree_budget(const uint32_t* sigma, int64_t n, int t, const int32_t* wpt, const int32_t* tpt, uint16_t* pw,
                        int32_t* tile_w, cudaStream_t s) {
  tree_budget_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(sigma, n, t, wpt, tpt, pw, tile_w);
  hf_after_launch("tree_budget_kernel", s);
}

// Sketches: bit j of point i = (<x_i, r_j> > 0) for the rows r_j of R, from
// the BF16 copies (xb: n x dp, rb: bits x dp), FP32 accumulation.
int launch_sketch(const void* xb, int64_t n, int dp, const void* rb, int bits, uint64_t* sketch, int* err,
                  cudaStream_t s) {
  if (bits < 64 || bits % 64 || bits > 1024 || n > (int64_t)1 << 30) return HF_EINVAL;
  const int nt = bits % 256 == 0 ? 256 : (bits % 128 == 0 ? 128 : 64);
  return gemm<EPI_SIGN>(static_cast<const __nv_bfloat16*>(xb), dp, static_cast<const __nv_bfloat16*>(rb), dp, (int)n,
                        bits, dp, nt, reinterpret_cast<float*>(sketch), bits / 16, nullptr, nullptr, 0, err, s);
}

void launch_f32_to_bf16(const float* x, int64_t rows, int cols, int ld, void* out, cudaStream_t s) {
  f32_to_bf16_kernel<<<hf_blocks(rows * ld, 256, 152 * 8), 256, 0, s>>>(x, rows, cols, ld,
                                                                        static_cast<__nv_bfloat16*>(out), ld);
  hf_after_launch("f32_to_bf16_kernel", s);
}
