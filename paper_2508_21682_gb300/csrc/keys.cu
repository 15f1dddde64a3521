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
//    bits of coordinates 0 .. 64K-1. It works on plane 0 in bit-sliced form
//    (one 32-bit word per group of 32 points and coordinate, made once per
//    build): a warp takes one group, lane l reads the word of permuted
//    coordinate 32h + l, an XOR scan across the lanes gives key bits
//    32h .. 32h+31 of all 32 points at once, and a bit-matrix transpose across
//    the warp hands each point its 32 key bits.
//  * general path (the prefix reaches below the top level, L >= 2 levels):
//    the same bit-sliced idea one level deeper -- the transform runs on
//    32-point words, one lane per group of 32 points, with the top L planes
//    sliced and the key words packed by warp transposes (prefix_bitsliced_kernel
//    below); one thread per point only where a warp's tile would not fit in
//    shared memory.
#include <cuda_runtime.h>

#include "hf_internal.cuh"
#include "hilbert_device.cuh"

namespace {

// 32 x 32 bit-matrix transpose across the warp: lane l holds row l (bit j =
// entry (l, j)); afterwards lane j holds column j (bit l = entry (l, j)).
// Stage s swaps the off-diagonal s x s blocks between lanes l and l ^ s: a
// lane keeps the bit positions whose bit s equals its own lane bit s and takes
// the others from its partner's word moved by s positions -- up for the lower
// lane, down for the upper one. Both moves are one rotation (by 32 - s or s):
// the bits that wrap around land only in kept positions. Per stage that is a
// shuffle, a funnel shift and one three-input logic op; the keep masks and
// rotation amounts depend on the lane alone.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    uint32_t mlo = 0;  // bit positions p with (p & s) == 0
#pragma unroll
    for (int p = 0; p < 32; ++p)
      if (!(p & s)) mlo |= 1u << p;
    const bool up = (lane & s) != 0;
    const uint32_t keep = up ? ~mlo : mlo;
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, s);
    const uint32_t moved = __funnelshift_r(y, y, up ? s : 32 - s);
    x = (x & keep) | (moved & ~keep);
  }
  return x;
}

// Bit-sliced plane 0: p0t[g][c] bit j = top bit of coordinate c of point
// 32g + j (0 past the last point). One warp per (group, plane word): lane j
// reads point 32g + j's word m, the transpose leaves coordinate 32m + c's word
// in lane c.
__global__ void plane0_slice_kernel(const uint32_t* __restrict__ plane0, int64_t n, int d, int W32,
                                    uint32_t* __restrict__ p0t) {
  const int lane = threadIdx.x & 31;
  const int64_t G = (n + 31) / 32;
  const int64_t tasks = G * W32;
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < tasks;
       e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t g = e / W32;
    const int m = (int)(e - g * W32);
    const int64_t p = g * 32 + lane;
    uint32_t x = p < n ? __ldg(plane0 + (size_t)p * W32 + m) : 0u;
    x = warp_transpose32(x, lane);
    const int c = m * 32 + lane;
    if (c < d) p0t[(size_t)g * d + c] = x;
  }
}

// Top-level prefix words 0 .. K-1 from the bit-sliced plane 0, one warp per
// group of 32 points. For half-word h, lane l takes key bit i = 32h + l: the
// word of permuted axis pi[i] (inverted when the axis is reflected) holds
// that bit's input for all 32 points; an inclusive XOR scan over the lanes
// plus the running carry of the earlier halves gives key bit i for all 32
// points, and the transpose (bit-reversed: the key is packed most significant
// bit first) gives point j its 32 bits 32h .. 32h+31.
template <int H>
__global__ void prefix_sliced_kernel(const uint32_t* __restrict__ p0t, int64_t n, int d, int K,
                                     const int32_t* __restrict__ pi, const uint32_t* __restrict__ rbits,
                                     uint64_t* __restrict__ pk) {
  constexpr int GW = 2;  // point groups per warp and round: their loads are in flight together
  const int lane = threadIdx.x & 31;
  const int64_t G = (n + 31) / 32;
  const int nh = 2 * K;  // 32-bit halves of the prefix (nh <= H)
  // the tree's permuted axes and reflection bits of this lane, once per warp
  int ax[H];
  uint32_t flip[H];
#pragma unroll
  for (int h = 0; h < H; ++h) {
    ax[h] = h < nh ? __ldg(pi + 32 * h + lane) : 0;
    flip[h] = h < nh ? 0u - ((__ldg(rbits + h) >> lane) & 1u) : 0u;
  }
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g0 < G; g0 += GW * nw) {
    // every word of both groups is loaded before any is used
    uint32_t v[GW][H];
#pragma unroll
    for (int q = 0; q < GW; ++q) {
      const int64_t g = g0 + q * nw;
      const uint32_t* row = p0t + (size_t)(g < G ? g : 0) * d;
#pragma unroll
      for (int h = 0; h < H; ++h) v[q][h] = (h < nh && g < G) ? __ldg(row + ax[h]) ^ flip[h] : 0u;
    }
#pragma unroll
    for (int q = 0; q < GW; ++q) {
      const int64_t g = g0 + q * nw;
      if (g >= G) break;
      const int64_t p = g * 32 + lane;
      uint32_t carry = 0, hi = 0;
#pragma unroll
      for (int h = 0; h < H; ++h) {
        if (h >= nh) break;
        uint32_t x = v[q][h];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x ^= t;
        }
        x ^= carry;
        carry = __shfl_sync(0xffffffffu, x, 31);
        const uint32_t half = __brev(warp_transpose32(x, lane));
        if (h & 1) {
          if (p < n) pk[(size_t)(h >> 1) * n + p] = ((uint64_t)hi << 32) | half;
        } else {
          hi = half;
        }
      }
    }
  }
}

// General path (L >= 2 top levels) in bit-sliced form. A warp takes `gpw`
// point groups (32 points each); lane j owns group g0 + j and keeps one 32-bit
// word per (level l, permuted coordinate i) -- bit p = level-l bit of
// coordinate i of point 32(g0 + j) + p -- in row l*d + i of its column of the
// warp's shared-memory tile (row stride `rs`, odd, so that a row's columns,
// a column's 32 consecutive rows and any 32 distinct rows of one 32-row span
// fall in distinct banks). Row l*d + i is also key bit l*d + i from the top,
// so the packing at the end reads rows in order.
//
// Skilling's map on whole words: at level q the points whose coordinate i has
// bit q set (mask c) invert the lower levels of coordinate 0, the others
// exchange the lower levels of coordinates 0 and i; with f = x0 ^ xi that is
// x0 ^= c | f and xi ^= f & ~c on every lower level. The Gray step is a
// running XOR over the coordinates, and the final correction of level r is
// the XOR of the last coordinate's levels above r. One lane thus transforms
// 32 points at once; loading (point-major planes -> sliced words) and packing
// (sliced words -> point-major key words) are 32 x 32 bit transposes across
// the warp, one group at a time.
template <int L>
__global__ void prefix_bitsliced_kernel(const uint32_t* __restrict__ planes, int64_t n, int d, int W32, int K,
                                        int gpw, int rs, const int32_t* __restrict__ pi,
                                        const uint32_t* __restrict__ rbits, uint64_t* __restrict__ pk) {
  extern __shared__ uint32_t smk[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  const int rows = L * d;
  int* inv = reinterpret_cast<int*>(smk);  // inv[pi[i]] = i
  uint32_t* S = smk + d + (size_t)warp * rows * rs;
  for (int i = threadIdx.x; i < d; i += blockDim.x) inv[__ldg(pi + i)] = i;
  __syncthreads();
  const int64_t G = (n + 31) / 32;
  const int nhalf = 2 * K;
  for (int64_t g0 = ((int64_t)blockIdx.x * nwb + warp) * gpw; g0 < G; g0 += (int64_t)gridDim.x * nwb * gpw) {
    const int ng = (int)(G - g0 < gpw ? G - g0 : gpw);
    // 1. slice: plane word m of level l for the group's 32 points, transposed,
    //    leaves coordinate 32m + lane's word in this lane; it goes to the row of
    //    its permuted position, inverted when that position is reflected. The
    //    L loads of the next (group, plane word) are in flight meanwhile.
    const int tasks = ng * W32;
    uint32_t v[L];
    auto load = [&](int e, uint32_t* dst) {
      const int j = e / W32, m = e - j * W32;
      const int64_t p = (g0 + j) * 32 + lane;
#pragma unroll
      for (int l = 0; l < L; ++l) dst[l] = p < n ? __ldg(planes + ((size_t)l * n + p) * W32 + m) : 0u;
    };
    load(0, v);
    for (int e = 0; e < tasks; ++e) {
      uint32_t nx[L];
      if (e + 1 < tasks) {
        load(e + 1, nx);
      } else {
#pragma unroll
        for (int l = 0; l < L; ++l) nx[l] = 0u;
      }
      const int j = e / W32, m = e - j * W32;
      const int c = m * 32 + lane;
      int i = 0;
      uint32_t flip = 0u;
      if (c < d) {
        i = inv[c];
        flip = 0u - ((__ldg(rbits + (i >> 5)) >> (i & 31)) & 1u);
      }
#pragma unroll
      for (int l = 0; l < L; ++l) {
        const uint32_t x = warp_transpose32(v[l], lane);
        if (c < d) S[(size_t)(l * d + i) * rs + j] = x ^ flip;
        v[l] = nx[l];
      }
    }
    __syncwarp();
    // 2. transform column `lane`
    if (lane < ng) {
      uint32_t* col = S + lane;
      uint32_t x0[L];
#pragma unroll
      for (int l = 0; l < L; ++l) x0[l] = col[(size_t)(l * d) * rs];
#pragma unroll
      for (int q = 0; q < L - 1; ++q) {
        const uint32_t c0 = x0[q];  // coordinate 0 against itself: inversion only
#pragma unroll
        for (int r = q + 1; r < L; ++r) x0[r] ^= c0;
        for (int i = 1; i < d; ++i) {
          const uint32_t c = col[(size_t)(q * d + i) * rs];
#pragma unroll
          for (int r = q + 1; r < L; ++r) {
            uint32_t* a = col + (size_t)(r * d + i) * rs;
            const uint32_t xi = *a;
            const uint32_t f = x0[r] ^ xi;
            x0[r] ^= c | f;
            *a = xi ^ (f & ~c);
          }
        }
      }
      uint32_t run[L], t[L];
#pragma unroll
      for (int l = 0; l < L; ++l) run[l] = x0[l];
      for (int i = 1; i < d; ++i) {
#pragma unroll
        for (int l = 0; l < L; ++l) {
          uint32_t* a = col + (size_t)(l * d + i) * rs;
          run[l] ^= *a;
          *a = run[l];
        }
      }
      uint32_t acc = 0;
#pragma unroll
      for (int l = 0; l < L; ++l) {
        t[l] = acc;
        acc ^= run[l];
      }
#pragma unroll
      for (int l = 0; l < L; ++l) col[(size_t)(l * d) * rs] = x0[l] ^ t[l];
      for (int i = 1; i < d; ++i) {
#pragma unroll
        for (int l = 1; l < L; ++l) col[(size_t)(l * d + i) * rs] ^= t[l];
      }
    }
    __syncwarp();
    // 3. pack: half h of group j's key words is rows 32h .. 32h+31 of column
    //    j, transposed (bit-reversed: most significant bit first)
    for (int j = 0; j < ng; ++j) {
      const int64_t p = (g0 + j) * 32 + lane;
      uint32_t hi = 0;
      for (int h = 0; h < nhalf; ++h) {
        const int b = 32 * h + lane;
        uint32_t x = b < rows ? S[(size_t)b * rs + j] : 0u;
        x = __brev(warp_transpose32(x, lane));
        if (h & 1) {
          if (p < n) pk[(size_t)(h >> 1) * n + p] = ((uint64_t)hi << 32) | x;
        } else {
          hi = x;
        }
      }
    }
    __syncwarp();
  }
}

// Per-thread general path: one thread per point, Y in shared memory. Used
// where the sliced tile of one warp would not fit in shared memory.
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

template <int L>
void bitsliced_launch(unsigned blocks, int threads, size_t smem, const uint32_t* planes, int64_t n, int d, int W32,
                      int K, int gpw, int rs, const int32_t* pi, const uint32_t* rbits, uint64_t* pk, cudaStream_t s) {
  set_smem((const void*)prefix_bitsliced_kernel<L>, smem);
  prefix_bitsliced_kernel<L><<<blocks, threads, smem, s>>>(planes, n, d, W32, K, gpw, rs, pi, rbits, pk);
}

// The bit-sliced general path; false (nothing launched) when one warp's tile
// does not fit in shared memory. Groups per warp: as few as give about 16
// warps per SM (the kernel is latency-bound: 8 or 32 per SM measured slower),
// up to one per lane.
bool launch_prefix_bitsliced(const uint32_t* planes, int64_t n, int d, int W32, int K, int L, const int32_t* pi,
                             const uint32_t* rbits, uint64_t* pk, cudaStream_t s) {
  constexpr int64_t kWarpsWanted = 152 * 16;
  constexpr size_t kSmemCap = 200 * 1024;
  const int64_t G = (n + 31) / 32;
  const int64_t want = (G + kWarpsWanted - 1) / kWarpsWanted;
  const int gpw = want < 1 ? 1 : (want > 32 ? 32 : (int)want);
  const int rs = gpw | 1;
  const size_t per_warp = (size_t)L * d * rs * sizeof(uint32_t);
  int nwb = 4;
  while (nwb > 1 && d * sizeof(int) + nwb * per_warp > kSmemCap) nwb >>= 1;
  const size_t smem = d * sizeof(int) + nwb * per_warp;
  if (smem > kSmemCap) return false;
  const int64_t warps = (G + gpw - 1) / gpw;
  int64_t blocks = (warps + nwb - 1) / nwb;
  if (blocks > 152 * 32) blocks = 152 * 32;
  const int thr = 32 * nwb;
  switch (L) {
    case 2: bitsliced_launch<2>((unsigned)blocks, thr, smem, planes, n, d, W32, K, gpw, rs, pi, rbits, pk, s); break;
    case 3: bitsliced_launch<3>((unsigned)blocks, thr, smem, planes, n, d, W32, K, gpw, rs, pi, rbits, pk, s); break;
    case 4: bitsliced_launch<4>((unsigned)blocks, thr, smem, planes, n, d, W32, K, gpw, rs, pi, rbits, pk, s); break;
    case 5: bitsliced_launch<5>((unsigned)blocks, thr, smem, planes, n, d, W32, K, gpw, rs, pi, rbits, pk, s); break;
    case 6: bitsliced_launch<6>((unsigned)blocks, thr, smem, planes, n, d, W32, K, gpw, rs, pi, rbits, pk, s); break;
    case 7: bitsliced_launch<7>((unsigned)blocks, thr, smem, planes, n, d, W32, K, gpw, rs, pi, rbits, pk, s); break;
    default: bitsliced_launch<8>((unsigned)blocks, thr, smem, planes, n, d, W32, K, gpw, rs, pi, rbits, pk, s); break;
  }
  hf_after_launch("prefix_bitsliced_kernel", s);
  return true;
}

}  // namespace

bool prefix_top_path(int d, int K, int L) { return L == 1 && d >= 64 * K; }

void launch_plane0_slice(const uint32_t* planes, int64_t n, int d, uint32_t* p0t, cudaStream_t s) {
  const int W32 = (d + 31) / 32;
  const int64_t tasks = (n + 31) / 32 * W32;
  plane0_slice_kernel<<<hf_blocks(tasks * 32, 256, 152 * 16), 256, 0, s>>>(planes, n, d, W32, p0t);
  hf_after_launch("plane0_slice_kernel", s);
}

void launch_prefix_keys(const uint32_t* planes, const uint32_t* p0t, int64_t n, int d, int bits, int K, int L,
                        const int32_t* pi, const uint32_t* rbits, uint64_t* pk, cudaStream_t s) {
  const int W32 = (d + 31) / 32;
  if (prefix_top_path(d, K, L) && p0t) {
    const int64_t G = (n + 31) / 32;
    const unsigned blocks = hf_blocks(G * 32, 256, 152 * 16);
    if (K <= 2)
      prefix_sliced_kernel<4><<<blocks, 256, 0, s>>>(p0t, n, d, K, pi, rbits, pk);
    else if (K <= 4)
      prefix_sliced_kernel<8><<<blocks, 256, 0, s>>>(p0t, n, d, K, pi, rbits, pk);
    else
      prefix_sliced_kernel<16><<<blocks, 256, 0, s>>>(p0t, n, d, K, pi, rbits, pk);
    hf_after_launch("prefix_sliced_kernel", s);
    return;
  }
  if (L >= 2 && L <= 8 && launch_prefix_bitsliced(planes, n, d, W32, K, L, pi, rbits, pk, s)) return;
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
