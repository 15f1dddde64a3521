// Window distances and top-k merge (plain float32 form).
//
// Paper, Algorithm 2: for the point j at position i of a sort's Hilbert order,
// the neighbours around position i are appended to its candidate set; the
// final selection keeps the top k by vector distance. Here the window is w
// positions on each side, the distance is the float32 squared Euclidean
// distance with exact coordinate differences, and each point's list (k pairs
// of (distance, index), ascending) is merged tree by tree, so the candidate
// set is never materialised.
//
// One block owns B consecutive positions [s, s+B). Every unordered pair of
// positions (p, q), p < q <= p + w, with at least one end owned by the block
// is scored once: rows p in [s - wr, s + B) against offsets delta = q - p in
// [1, wr] (wr = w rounded up to 8; offsets above w are masked). The rows
// [s - wr, s + B + wr) of the gathered point matrix are staged in shared
// memory DC coordinates at a time; each thread accumulates a 4-row x 8-offset
// unit of the band in registers. The band of distances then sits in shared
// memory, and the thread owning position p merges its right neighbours
// (p, p + delta) and left neighbours (p - delta, p) into point sigma[p]'s list.
// Pairs whose two ends belong to different blocks are scored by both blocks
// (the same arithmetic in the same order, so both see the same value).
#include <cuda_runtime.h>
#include <math.h>

#include "hf_internal.cuh"

namespace {

constexpr int WNT = 256;   // threads per block
constexpr int DC = 32;     // coordinates staged per chunk
constexpr int XS = DC + 4; // padded row stride of the staged chunk (floats)
constexpr int UR = 4;      // rows per thread unit
constexpr int UC = 8;      // offsets per thread unit

struct WinGeom {
  int B;   // owned positions per block
  int wr;  // w rounded up to a multiple of UC
  int NR;  // staged rows = B + 2 wr
  int units;
};

__device__ __forceinline__ bool lessp(float da, uint32_t ia, float db, uint32_t ib) {
  return da < db || (da == db && ia < ib);
}

template <int UPT>
__global__ void __launch_bounds__(WNT)
window_kernel(const float* __restrict__ x, int64_t n, int d, const uint32_t* __restrict__ sigma, int w,
              int k, int B, int wr, int vec4, uint32_t* __restrict__ lidx, float* __restrict__ ldist) {
  extern __shared__ __align__(16) float smem[];
  const int NR = B + 2 * wr;
  const int nband = B + wr;  // band rows
  float* xs = smem;                                   // [NR][XS]
  float* band = xs + (size_t)NR * XS;                 // [nband][wr]
  uint32_t* srow = reinterpret_cast<uint32_t*>(band + (size_t)nband * wr);  // [NR] point ids
  float* ld = reinterpret_cast<float*>(srow + NR);    // [k][B]
  uint32_t* li = reinterpret_cast<uint32_t*>(ld + (size_t)k * B);  // [k][B]

  const int64_t s = (int64_t)blockIdx.x * B;
  const int64_t r0 = s - wr;  // global position of staged row 0
  for (int r = threadIdx.x; r < NR; r += WNT) {
    const int64_t p = r0 + r;
    srow[r] = (p >= 0 && p < n) ? sigma[p] : 0xffffffffu;
  }

  const int ogroups = wr / UC;
  const int units = (nband / UR) * ogroups;
  float acc[UPT][UR][UC];
#pragma unroll
  for (int u = 0; u < UPT; ++u)
#pragma unroll
    for (int a = 0; a < UR; ++a)
#pragma unroll
      for (int c = 0; c < UC; ++c) acc[u][a][c] = 0.f;
  __syncthreads();

  for (int c0 = 0; c0 < d; c0 += DC) {
    const int dc = min(DC, d - c0);
    // stage rows r0 .. r0 + NR - 1, coordinates c0 .. c0 + dc - 1 (zero padded)
    if (vec4) {
      const int per_row = DC / 4;
      for (int e = threadIdx.x; e < NR * per_row; e += WNT) {
        const int r = e / per_row, q = e - r * per_row;
        const uint32_t pid = srow[r];
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (pid != 0xffffffffu && 4 * q < dc)
          v = __ldg(reinterpret_cast<const float4*>(x + (size_t)pid * d + c0) + q);
        *reinterpret_cast<float4*>(xs + r * XS + 4 * q) = v;
      }
    } else {
      for (int e = threadIdx.x; e < NR * DC; e += WNT) {
        const int r = e / DC, q = e - r * DC;
        const uint32_t pid = srow[r];
        float v = 0.f;
        if (pid != 0xffffffffu && q < dc) v = __ldg(x + (size_t)pid * d + c0 + q);
        xs[r * XS + q] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
      const int unit = threadIdx.x + u * WNT;
      if (unit < units) {
        const int g = unit / ogroups, o = unit - g * ogroups;
        const int pr = UR * g;            // band row of the unit's first row (= staged row)
        const int qr = pr + 1 + UC * o;   // staged row of (first row, first offset)
        for (int j = 0; j < DC; j += 4) {
          float4 a[UR], b[UR + UC - 1];
#pragma unroll
          for (int t = 0; t < UR; ++t) a[t] = *reinterpret_cast<const float4*>(xs + (pr + t) * XS + j);
#pragma unroll
          for (int t = 0; t < UR + UC - 1; ++t) b[t] = *reinterpret_cast<const float4*>(xs + (qr + t) * XS + j);
#pragma unroll
          for (int t = 0; t < UR; ++t)
#pragma unroll
            for (int c = 0; c < UC; ++c) {
              float e0 = a[t].x - b[t + c].x;
              float e1 = a[t].y - b[t + c].y;
              float e2 = a[t].z - b[t + c].z;
              float e3 = a[t].w - b[t + c].w;
              float v = acc[u][t][c];
              v = fmaf(e0, e0, v);
              v = fmaf(e1, e1, v);
              v = fmaf(e2, e2, v);
              v = fmaf(e3, e3, v);
              acc[u][t][c] = v;
            }
        }
      }
    }
    __syncthreads();
  }

  // band[row][delta-1]: row = staged row of p (p = r0 + row), valid pairs only
#pragma unroll
  for (int u = 0; u < UPT; ++u) {
    const int unit = threadIdx.x + u * WNT;
    if (unit < units) {
      const int g = unit / ogroups, o = unit - g * ogroups;
#pragma unroll
      for (int t = 0; t < UR; ++t)
#pragma unroll
        for (int c = 0; c < UC; ++c) {
          const int row = UR * g + t;
          const int delta = 1 + UC * o + c;
          const int64_t p = r0 + row, q = p + delta;
          const bool ok = delta <= w && p >= 0 && q < n && (p >= s || q >= s) && p < s + B;
          band[row * wr + delta - 1] = ok ? acc[u][t][c] : INFINITY;
        }
    }
  }
  __syncthreads();

  // merge: thread t owns position s + t
  for (int t = threadIdx.x; t < B; t += WNT) {
    const int64_t p = s + t;
    if (p >= n) continue;
    const int rowp = t + wr;  // staged row of p
    const uint32_t ip = srow[rowp];
    for (int j = 0; j < k; ++j) {
      ld[j * B + t] = ldist[(size_t)ip * k + j];
      li[j * B + t] = lidx[(size_t)ip * k + j];
    }
    float wd = ld[(k - 1) * B + t];
    uint32_t wi = li[(k - 1) * B + t];
    for (int side = 0; side < 2; ++side) {
      for (int delta = 1; delta <= w; ++delta) {
        float cd;
        uint32_t ci;
        if (side == 0) {  // right neighbour (p, p + delta)
          if (p + delta >= n) break;
          cd = band[rowp * wr + delta - 1];
          ci = srow[rowp + delta];
        } else {  // left neighbour (p - delta, p)
          if (p - delta < 0) break;
          cd = band[(rowp - delta) * wr + delta - 1];
          ci = srow[rowp - delta];
        }
        if (!lessp(cd, ci, wd, wi)) continue;
        bool dup = false;
        for (int j = 0; j < k; ++j) dup |= (li[j * B + t] == ci);
        if (dup) continue;
        int j = k - 1;
        while (j > 0 && lessp(cd, ci, ld[(j - 1) * B + t], li[(j - 1) * B + t])) {
          ld[j * B + t] = ld[(j - 1) * B + t];
          li[j * B + t] = li[(j - 1) * B + t];
          --j;
        }
        ld[j * B + t] = cd;
        li[j * B + t] = ci;
        wd = ld[(k - 1) * B + t];
        wi = li[(k - 1) * B + t];
      }
    }
    for (int j = 0; j < k; ++j) {
      ldist[(size_t)ip * k + j] = ld[j * B + t];
      lidx[(size_t)ip * k + j] = li[j * B + t];
    }
  }
}

__global__ void list_init_kernel(uint32_t* __restrict__ idx, float* __restrict__ dist, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    idx[e] = 0xffffffffu;
    dist[e] = INFINITY;
  }
}

size_t window_smem(int B, int wr, int k) {
  const int NR = B + 2 * wr;
  return ((size_t)NR * XS + (size_t)(B + wr) * wr) * sizeof(float) + (size_t)NR * 4 +
         (size_t)k * B * 8;
}

template <int UPT>
int launch_upt(const float* x, int64_t n, int d, const uint32_t* sigma, int w, int k, int B, int wr,
               uint32_t* li, float* ldd, cudaStream_t s) {
  const size_t smem = window_smem(B, wr, k);
  if (cudaFuncSetAttribute((const void*)window_kernel<UPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return HF_ECUDA;
  const unsigned blocks = hf_blocks(n, B);
  // 16-byte loads need every row start 16-byte aligned
  const int vec4 = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
  window_kernel<UPT><<<blocks, WNT, smem, s>>>(x, n, d, sigma, w, k, B, wr, vec4, li, ldd); hf_after_launch("window_kernel<UPT>", s);
  return HF_OK;
}

}  // namespace

void launch_list_init(uint32_t* idx, float* dist, int64_t count, cudaStream_t s) {
  list_init_kernel<<<hf_blocks(count, 256, 152 * 8), 256, 0, s>>>(idx, dist, count); hf_after_launch("list_init_kernel", s);
}

// Chooses B so that (B + wr) / 4 * wr / 8 units fill a multiple of the block.
int launch_window_graph(const float* x, int64_t n, int d, const uint32_t* sigma, int w, int k,
                        uint32_t* list_idx, float* list_dist, cudaStream_t s) {
  const int wr = (w + UC - 1) / UC * UC;
  // units = (B + wr) * wr / 32; pick B (multiple of 4) for ~1..4 units/thread
  int upt;
  if (wr <= 32) upt = 1;
  else if (wr <= 64) upt = 2;
  else upt = 4;
  if (wr > 128) return HF_ENOTIMPL;
  int B = (upt * WNT * 32) / wr - wr;  // largest B with units <= upt * WNT
  B = B / UR * UR;
  if (B < 16) return HF_ENOTIMPL;
  if (B > 512) B = 512;
  while (window_smem(B, wr, k) > 220 * 1024 && B > 16) B -= 16;
  switch (upt) {
    case 1: return launch_upt<1>(x, n, d, sigma, w, k, B, wr, list_idx, list_dist, s);
    case 2: return launch_upt<2>(x, n, d, sigma, w, k, B, wr, list_idx, list_dist, s);
    default: return launch_upt<4>(x, n, d, sigma, w, k, B, wr, list_idx, list_dist, s);
  }
}
