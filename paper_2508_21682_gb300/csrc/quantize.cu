// Per-axis range and b-bit quantization of the points.
//
// The paper quantizes vectors for its distance stage (Section 3, 4-bit codes)
// but does not say how coordinates are discretised for the Hilbert sort. This
// library fixes: lo_j = min_i x_ij, hi_j = max_i x_ij, scale_j =
// (float)(2^b / (double)(float)(hi_j - lo_j)) (0 for a flat axis), and
// code = clamp(floor(fl32(fl32(x - lo) * scale)), 0, 2^b - 1), each step a
// separately rounded float32 operation (__fsub_rn / __fmul_rn, never fused).
//
// Codes are stored as b bit planes, plane 0 holding the most significant bit:
// planes[l][i][m] bit j = bit (b-1-l) of the code of coordinate 32m + j of
// point i. A key prefix that needs only the top level reads one plane
// (d/8 bytes per point) instead of the whole code row.
#include <cuda_runtime.h>
#include <math.h>

#include "hf_internal.cuh"

namespace {

constexpr int RANGE_THREADS = 256;

// Each thread owns one column group of `vec` consecutive columns for the whole
// run, because the total thread count is a multiple of d / vec; it keeps a
// running min / max and writes them to partial[thread].
template <int VEC>
__global__ void range_partial_kernel(const float* __restrict__ x, int64_t total_vec, int d,
                                     int64_t nthreads, float* __restrict__ pmin,
                                     float* __restrict__ pmax, int* __restrict__ err) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nthreads) return;
  float mn[VEC], mx[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    mn[v] = INFINITY;
    mx[v] = -INFINITY;
  }
  bool bad = false;
  for (int64_t e = t; e < total_vec; e += nthreads) {
    if (VEC == 4) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(x) + e);
      const float vals[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int v = 0; v < VEC; ++v) {
        bad |= !isfinite(vals[v]);
        mn[v] = fminf(mn[v], vals[v]);
        mx[v] = fmaxf(mx[v], vals[v]);
      }
    } else {
      const float val = __ldg(x + e);
      bad |= !isfinite(val);
      mn[0] = fminf(mn[0], val);
      mx[0] = fmaxf(mx[0], val);
    }
  }
  if (bad) hf_raise(err, HF_ERRBIT_NONFINITE);
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    pmin[t * VEC + v] = mn[v];
    pmax[t * VEC + v] = mx[v];
  }
}

// One block per column c: the partials of threads t with (t*VEC) % d == c - v
// are reduced by the block's threads, then across the block.
__global__ void range_final_kernel(const float* __restrict__ pmin, const float* __restrict__ pmax,
                                   int64_t nthreads, int vec, int d, int bits,
                                   float* __restrict__ lo, float* __restrict__ scale) {
  __shared__ float smn[32], smx[32];
  const int c = blockIdx.x;
  const int groups = d / vec;  // threads per "row" of column groups
  const int g = c / vec, v = c % vec;
  float mn = INFINITY, mx = -INFINITY;
  for (int64_t t = g + (int64_t)threadIdx.x * groups; t < nthreads; t += (int64_t)blockDim.x * groups) {
    mn = fminf(mn, pmin[t * vec + v]);
    mx = fmaxf(mx, pmax[t * vec + v]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    smn[wid] = mn;
    smx[wid] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      mn = fminf(mn, smn[w]);
      mx = fmaxf(mx, smx[w]);
    }
    lo[c] = mn;
    const float width = __fsub_rn(mx, mn);
    scale[c] = width > 0.0f ? (float)((double)(1u << bits) / (double)width) : 0.0f;
  }
}

__device__ __forceinline__ uint32_t quantize_one(float x, float lo, float scale, int bits) {
  const float diff = __fsub_rn(x, lo);
  const float prod = __fmul_rn(diff, scale);
  const float fl = floorf(prod);
  const float top = (float)((1u << bits) - 1u);
  const float cl = fminf(fmaxf(fl, 0.0f), top);
  return (uint32_t)cl;
}

// 8 x 8 bit-matrix transpose of a 64-bit word: bit c of byte u moves to
// bit u of byte c (delta swaps of 7, 14 and 28 positions).
__device__ __forceinline__ uint64_t transpose8x8(uint64_t x) {
  uint64_t t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
  x = x ^ t ^ (t << 7);
  t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
  x = x ^ t ^ (t << 14);
  t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
  x = x ^ t ^ (t << 28);
  return x;
}

// One warp per point. The warp first copies the point's row into its
// shared-memory slot (16-byte loads when rows are 16-byte aligned, all issued
// before any is used). Lane j then takes groups of 8 consecutive coordinates
// (8g .. 8g+7, g = j, j + 32, ...): it quantizes them, packs the 8 codes
// (aligned to 8 bits) into one 64-bit word and transposes it as an 8 x 8 bit
// matrix, so that byte 7 - l holds bit plane l of the 8 coordinates: byte g
// of the point's plane-l row. The plane rows (W32 words each) are collected
// in shared memory and written out contiguously.
constexpr int QP_THREADS = 256;

__global__ void __launch_bounds__(QP_THREADS)
quantize_planes_kernel(const float* __restrict__ x, int64_t n, int d, int W32, const float* __restrict__ lo0,
                       const float* __restrict__ scale0, int bits, int vec4, const uint32_t* __restrict__ seg,
                       uint32_t* __restrict__ planes) {
  extern __shared__ __align__(16) float qsm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int rowf = 32 * W32;                       // staged floats (>= d)
  const int wstride = (rowf + bits * W32 + 3) & ~3;  // floats per warp, keeps 16-byte alignment
  float* row_s = qsm + (size_t)wib * wstride;
  uint32_t* word_s = reinterpret_cast<uint32_t*>(row_s + rowf);  // [bits][W32]
  uint8_t* byte_s = reinterpret_cast<uint8_t*>(word_s);          // [bits][4 W32]
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int groups = 4 * W32;
  for (int64_t i = warp; i < n; i += nwarps) {
    const float* row = x + (size_t)i * d;
    // segmented rows take their own set's range
    const size_t so = seg ? (size_t)__ldg(seg + i) * d : 0;
    const float* __restrict__ lo = lo0 + so;
    const float* __restrict__ scale = scale0 + so;
    if (vec4) {
      for (int f = lane; f < (d >> 2); f += 32)
        reinterpret_cast<float4*>(row_s)[f] = __ldg(reinterpret_cast<const float4*>(row) + f);
    } else {
      for (int c = lane; c < d; c += 32) row_s[c] = __ldg(row + c);
    }
    __syncwarp();
    for (int g = lane; g < groups; g += 32) {
      const int c0 = 8 * g;
      uint32_t w0 = 0, w1 = 0;  // codes of coordinates c0 .. c0+3 and c0+4 .. c0+7, one per byte
      if (vec4 && c0 + 8 <= d) {
        const float4 xa = *reinterpret_cast<const float4*>(row_s + c0);
        const float4 xb = *reinterpret_cast<const float4*>(row_s + c0 + 4);
        const float4 la = __ldg(reinterpret_cast<const float4*>(lo + c0));
        const float4 lb = __ldg(reinterpret_cast<const float4*>(lo + c0 + 4));
        const float4 sa = __ldg(reinterpret_cast<const float4*>(scale + c0));
        const float4 sb = __ldg(reinterpret_cast<const float4*>(scale + c0 + 4));
        w0 = quantize_one(xa.x, la.x, sa.x, bits) | (quantize_one(xa.y, la.y, sa.y, bits) << 8) |
             (quantize_one(xa.z, la.z, sa.z, bits) << 16) | (quantize_one(xa.w, la.w, sa.w, bits) << 24);
        w1 = quantize_one(xb.x, lb.x, sb.x, bits) | (quantize_one(xb.y, lb.y, sb.y, bits) << 8) |
             (quantize_one(xb.z, lb.z, sb.z, bits) << 16) | (quantize_one(xb.w, lb.w, sb.w, bits) << 24);
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = c0 + u;
          const uint32_t code = c < d ? quantize_one(row_s[c], __ldg(lo + c), __ldg(scale + c), bits) : 0u;
          if (u < 4) w0 |= code << (8 * u);
          else w1 |= code << (8 * (u - 4));
        }
      }
      // align every code to 8 bits (the shift stays inside each byte)
      const uint64_t packed = ((uint64_t)w1 << 32 | w0) << (8 - bits);
      const uint64_t tr = transpose8x8(packed);
      for (int l = 0; l < bits; ++l) byte_s[l * groups + g] = (uint8_t)(tr >> (8 * (7 - l)));
    }
    __syncwarp();
    for (int l = 0; l < bits; ++l)
      for (int m = lane; m < W32; m += 32) planes[((size_t)l * n + i) * W32 + m] = word_s[l * W32 + m];
    __syncwarp();
  }
}

__global__ void quantize_codes_kernel(const float* __restrict__ x, int64_t total, int d,
                                      const float* __restrict__ lo,
                                      const float* __restrict__ scale, int bits,
                                      uint8_t* __restrict__ codes, int* __restrict__ err) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float v = x[e];
    if (!isfinite(v)) {
      hf_raise(err, HF_ERRBIT_NONFINITE);
      codes[e] = 0;
      continue;
    }
    const int c = (int)(e % d);
    codes[e] = (uint8_t)quantize_one(v, lo[c], scale[c], bits);
  }
}

__global__ void planes_to_codes_kernel(const uint32_t* __restrict__ planes, int64_t n, int d,
                                       int W32, int bits, uint8_t* __restrict__ codes) {
  const int64_t total = n * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / d;
    const int c = (int)(e - i * d);
    uint32_t v = 0;
    for (int l = 0; l < bits; ++l)
      v = (v << 1) | ((planes[((size_t)l * n + i) * W32 + (c >> 5)] >> (c & 31)) & 1u);
    codes[e] = (uint8_t)v;
  }
}

// Range of every set of a segmented matrix: block (set, 32-column chunk);
// lane j of each warp keeps the min / max of column 32 c + j over the warp's
// rows of the set, then the block's warps are combined. Same lo / scale
// formula as range_final_kernel.
__global__ void seg_range_kernel(const float* __restrict__ x, int d, const int64_t* __restrict__ off, int nchunks,
                                 int bits, float* __restrict__ lo, float* __restrict__ scale, int* __restrict__ err) {
  __shared__ float smn[8][32], smx[8][32];
  const int set = blockIdx.x / nchunks, ch = blockIdx.x % nchunks;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = 32 * ch + lane;
  const int64_t r0 = off[set], r1 = off[set + 1];
  float mn = INFINITY, mx = -INFINITY;
  bool bad = false;
  if (c < d) {
    for (int64_t r = r0 + warp; r < r1; r += 8) {
      const float v = __ldg(x + (size_t)r * d + c);
      bad |= !isfinite(v);
      mn = fminf(mn, v);
      mx = fmaxf(mx, v);
    }
  }
  if (bad) hf_raise(err, HF_ERRBIT_NONFINITE);
  smn[warp][lane] = mn;
  smx[warp][lane] = mx;
  __syncthreads();
  if (warp == 0 && c < d) {
    for (int w = 1; w < 8; ++w) {
      mn = fminf(mn, smn[w][lane]);
      mx = fmaxf(mx, smx[w][lane]);
    }
    lo[(size_t)set * d + c] = mn;
    const float width = __fsub_rn(mx, mn);
    scale[(size_t)set * d + c] = width > 0.0f ? (float)((double)(1u << bits) / (double)width) : 0.0f;
  }
}

// Set index of every row of a segmented matrix (binary search of the offsets).
__global__ void seg_of_row_kernel(const int64_t* __restrict__ off, int nseg, int64_t n, uint32_t* __restrict__ seg,
                                  uint64_t* __restrict__ seg64) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nseg - 1;  // last set whose offset is <= i
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(off + mid) <= i) lo = mid;
      else hi = mid - 1;
    }
    seg[i] = (uint32_t)lo;
    if (seg64) seg64[i] = (uint64_t)lo;
  }
}

int64_t range_threads(int64_t n, int d, int vec) {
  const int64_t groups = d / vec;
  int64_t target = 152 * 2048;
  int64_t reps = (target + groups - 1) / groups;
  const int64_t rows_max = n;  // no more threads than rows per column group
  if (reps > rows_max) reps = rows_max;
  if (reps < 1) reps = 1;
  return reps * groups;
}

}  // namespace

size_t range_scratch_bytes(int64_t n, int d) {
  const int vec = (d % 4 == 0) ? 4 : 1;
  return (size_t)range_threads(n, d, vec) * vec * 2 * sizeof(float);
}

void launch_range(const float* x, int64_t n, int d, float* lo, float* scale, int bits, int* err,
                  void* scratch, size_t scratch_bytes, cudaStream_t s) {
  const bool v4 = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
  const int vec = v4 ? 4 : 1;
  int64_t nthreads = range_threads(n, d, (d % 4 == 0) ? 4 : 1);
  if (!v4) nthreads = range_threads(n, d, 1);
  float* pmin = static_cast<float*>(scratch);
  float* pmax = pmin + nthreads * vec;
  (void)scratch_bytes;
  const int64_t total_vec = n * d / vec;
  const unsigned blocks = hf_blocks(nthreads, RANGE_THREADS);
  if (v4)
    range_partial_kernel<4><<<blocks, RANGE_THREADS, 0, s>>>(x, total_vec, d, nthreads, pmin, pmax, err);
  else
    range_partial_kernel<1><<<blocks, RANGE_THREADS, 0, s>>>(x, total_vec, d, nthreads, pmin, pmax, err);
  hf_after_launch("range_partial_kernel", s);
  range_final_kernel<<<d, 256, 0, s>>>(pmin, pmax, nthreads, vec, d, bits, lo, scale);
  hf_after_launch("range_final_kernel", s);
}

void launch_seg_range(const float* x, int d, const int64_t* off, int nseg, int bits, float* lo, float* scale, int* err,
                      cudaStream_t s) {
  const int nchunks = (d + 31) / 32;
  seg_range_kernel<<<(unsigned)(nseg * nchunks), 256, 0, s>>>(x, d, off, nchunks, bits, lo, scale, err);
  hf_after_launch("seg_range_kernel", s);
}

void launch_seg_of_row(const int64_t* off, int nseg, int64_t n, uint32_t* seg, uint64_t* seg64, cudaStream_t s) {
  seg_of_row_kernel<<<hf_blocks(n, 256, 152 * 8), 256, 0, s>>>(off, nseg, n, seg, seg64);
  hf_after_launch("seg_of_row_kernel", s);
}

void launch_quantize_planes(const float* x, int64_t n, int d, const float* lo, const float* scale,
                            int bits, uint32_t* planes, int* err, cudaStream_t s, const uint32_t* seg) {
  (void)err;
  const int W32 = (d + 31) / 32;
  const int vec4 = d % 4 == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  const size_t smem = (size_t)(QP_THREADS / 32) * ((32 * W32 + bits * W32 + 3) & ~3) * 4;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute((const void*)quantize_planes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  quantize_planes_kernel<<<hf_blocks(n * 32, QP_THREADS, 152 * 16), QP_THREADS, smem, s>>>(x, n, d, W32, lo, scale,
                                                                                          bits, vec4, seg, planes);
  hf_after_launch("quantize_planes_kernel", s);
}

void launch_quantize_codes(const float* x, int64_t n, int d, const float* lo, const float* scale,
                           int bits, uint8_t* codes, int* err, cudaStream_t s) {
  const int64_t total = n * d;
  quantize_codes_kernel<<<hf_blocks(total, 256, 152 * 16), 256, 0, s>>>(x, total, d, lo, scale, bits,
                                                                       codes, err); hf_after_launch("quantize_codes_kernel", s);
}

void launch_planes_to_codes(const uint32_t* planes, int64_t n, int d, int bits, uint8_t* codes,
                            cudaStream_t s) {
  const int W32 = (d + 31) / 32;
  planes_to_codes_kernel<<<hf_blocks(n * d, 256, 152 * 16), 256, 0, s>>>(planes, n, d, W32, bits, codes); hf_after_launch("planes_to_codes_kernel", s);
}
