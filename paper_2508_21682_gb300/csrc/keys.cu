// Hilbert key prefixes (what the radix sort orders) and full keys (for the
// tie fix-up, search and inspection).
//
// Paper, Section 2 and Algorithm 2: every sort uses its own random axis order
// and orders the points along the Hilbert curve. Here the curve is Skilling's
// transposed index; the sort compares the first K 64-bit words of the key and
// resolves equal prefixes with the full key afterwards.
//
// Two prefix paths:
//  * top-level path (the first 64K key bits all lie in bit level 0, i.e.
//    d >= 64K): those bits are the running XOR of the permuted, reflected top
//    bits of coordinates 0 .. 64K-1. Each block stages the plane-0 rows of its
//    points in shared memory and every thread gathers, XOR-scans and packs its
//    point's bits word by word.
//  * general path: each thread forms the top L bits of all d coordinates in
//    shared memory and runs the transform with L levels.
#include <cuda_runtime.h>

#include "hf_internal.cuh"
#include "hilbert_device.cuh"

namespace {

constexpr int TOP_THREADS = 128;

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

__global__ void __launch_bounds__(TOP_THREADS)
prefix_top_kernel(const uint32_t* __restrict__ plane0, int64_t n, int d, int W32, int K,
                  const int32_t* __restrict__ pi, const uint32_t* __restrict__ rbits,
                  uint64_t* __restrict__ pk) {
  extern __shared__ uint32_t sm[];
  const int nbits = 64 * K;                 // bits needed, all from plane 0
  int32_t* s_pi = reinterpret_cast<int32_t*>(sm);  // [nbits]
  uint32_t* s_r = sm + nbits;                      // [nbits / 32]
  uint32_t* s_rows = s_r + nbits / 32;             // [TOP_THREADS][W32 + 1]
  const int stride = W32 + 1;

  for (int i = threadIdx.x; i < nbits; i += blockDim.x) s_pi[i] = pi[i];
  for (int i = threadIdx.x; i < nbits / 32; i += blockDim.x) {
    // reflection bits of permuted axes 32i .. 32i+31, reordered MSB-first so
    // that bit 31 belongs to axis 32i
    s_r[i] = __brev(rbits[i]);
  }
  const int64_t p0 = (int64_t)blockIdx.x * TOP_THREADS;
  const int rows = (int)((n - p0) < TOP_THREADS ? (n - p0) : TOP_THREADS);
  for (int e = threadIdx.x; e < rows * W32; e += blockDim.x) {
    const int r = e / W32, m = e - r * W32;
    s_rows[r * stride + m] = __ldg(plane0 + (p0 + r) * W32 + m);
  }
  __syncthreads();
  if ((int)threadIdx.x >= rows) return;
  const uint32_t* row = s_rows + threadIdx.x * stride;
  uint32_t carry = 0;  // parity of all earlier bits
  const int64_t p = p0 + threadIdx.x;
  for (int w = 0; w < K; ++w) {
    uint32_t half[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int base = w * 64 + h * 32;
      uint32_t v = 0;
#pragma unroll 8
      for (int j = 0; j < 32; ++j) {
        const int c = s_pi[base + j];
        v = (v << 1) | ((row[c >> 5] >> (c & 31)) & 1u);
      }
      v ^= s_r[base >> 5];
      v = xor_scan_msb(v);
      if (carry) v = ~v;
      carry = v & 1u;
      half[h] = v;
    }
    pk[(size_t)w * n + p] = ((uint64_t)half[0] << 32) | half[1];
  }
}

// General path: one thread per point, Y in shared memory.
__global__ void prefix_general_kernel(const uint32_t* __restrict__ planes, int64_t n, int d,
                                      int W32, int K, int L, const int32_t* __restrict__ pi,
                                      const uint32_t* __restrict__ rbits,
                                      uint64_t* __restrict__ pk) {
  extern __shared__ uint8_t smb[];
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  uint8_t* Y = smb + (size_t)threadIdx.x * d;
  hf_load_coords_planes(planes, n, d, W32, L, pi, rbits, p, Y);
  hf_skilling(Y, d, L);
  for (int w = 0; w < K; ++w) pk[(size_t)w * n + p] = hf_pack_word(Y, d, L, w);
}

__global__ void full_keys_planes_kernel(const uint32_t* __restrict__ planes, int64_t n, int d,
                                        int W32, int bits, int W, const int32_t* __restrict__ pi,
                                        const uint32_t* __restrict__ rbits,
                                        uint64_t* __restrict__ out) {
  extern __shared__ uint8_t smb[];
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  uint8_t* Y = smb + (size_t)threadIdx.x * d;
  hf_load_coords_planes(planes, n, d, W32, bits, pi, rbits, p, Y);
  hf_skilling(Y, d, bits);
  for (int w = 0; w < W; ++w) out[(size_t)p * W + w] = hf_pack_word(Y, d, bits, w);
}

__global__ void full_keys_codes_kernel(const uint8_t* __restrict__ codes, int64_t n, int d,
                                       int bits, int W, const int32_t* __restrict__ pi,
                                       const uint32_t* __restrict__ rbits,
                                       uint64_t* __restrict__ out) {
  extern __shared__ uint8_t smb[];
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  uint8_t* Y = smb + (size_t)threadIdx.x * d;
  hf_load_coords_codes(codes + (size_t)p * d, d, bits, bits, pi, rbits, Y);
  hf_skilling(Y, d, bits);
  for (int w = 0; w < W; ++w) out[(size_t)p * W + w] = hf_pack_word(Y, d, bits, w);
}

int threads_for_bytes_per_thread(int bytes) {
  int t = 256;
  while (t > 32 && (size_t)t * bytes > 96 * 1024) t >>= 1;
  return t;
}

void set_smem(const void* fn, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

void launch_prefix_keys(const uint32_t* planes, int64_t n, int d, int bits, int K, int L,
                        const int32_t* pi, const uint32_t* rbits, uint64_t* pk, cudaStream_t s) {
  const int W32 = (d + 31) / 32;
  if (L == 1 && d >= 64 * K) {
    const size_t smem = (size_t)(64 * K + 2 * K + TOP_THREADS * (W32 + 1)) * sizeof(uint32_t);
    set_smem((const void*)prefix_top_kernel, smem);
    prefix_top_kernel<<<hf_blocks(n, TOP_THREADS), TOP_THREADS, smem, s>>>(planes, n, d, W32, K, pi,
                                                                           rbits, pk); hf_after_launch("prefix_top_kernel", s);
    return;
  }
  const int t = threads_for_bytes_per_thread(d);
  const size_t smem = (size_t)t * d;
  set_smem((const void*)prefix_general_kernel, smem);
  prefix_general_kernel<<<hf_blocks(n, t), t, smem, s>>>(planes, n, d, W32, K, L, pi, rbits, pk); hf_after_launch("prefix_general_kernel", s);
  (void)bits;
}

void launch_full_keys_planes(const uint32_t* planes, int64_t n, int d, int bits, int W,
                             const int32_t* pi, const uint32_t* rbits, uint64_t* out,
                             cudaStream_t s) {
  const int W32 = (d + 31) / 32;
  const int t = threads_for_bytes_per_thread(d);
  const size_t smem = (size_t)t * d;
  set_smem((const void*)full_keys_planes_kernel, smem);
  full_keys_planes_kernel<<<hf_blocks(n, t), t, smem, s>>>(planes, n, d, W32, bits, W, pi, rbits, out); hf_after_launch("full_keys_planes_kernel", s);
}

void launch_full_keys_codes(const uint8_t* codes, int64_t n, int d, int bits, int W,
                            const int32_t* pi, const uint32_t* rbits, uint64_t* out,
                            cudaStream_t s) {
  const int t = threads_for_bytes_per_thread(d);
  const size_t smem = (size_t)t * d;
  set_smem((const void*)full_keys_codes_kernel, smem);
  full_keys_codes_kernel<<<hf_blocks(n, t), t, smem, s>>>(codes, n, d, bits, W, pi, rbits, out); hf_after_launch("full_keys_codes_kernel", s);
}
