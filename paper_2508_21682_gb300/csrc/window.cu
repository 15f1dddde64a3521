// Window distances and top-k merge (plain float32 form).
//
// Paper, Algorithm 2: in every sort, the points lying a few places before and
// after a point in that sort's Hilbert order join its candidates, and the
// best k candidates by vector distance are the result. Here the window is w
// positions on each side, the distance is the float32 squared Euclidean
// distance with exact coordinate differences, and each point's list (k pairs
// of (distance, index), ascending) is merged tree by tree, so the candidate
// set is never materialised.
//
// Work split. A block owns B consecutive positions [s, s+B) and one band of
// 32 offsets [dlo, dlo+31] (w > 32 takes several launches, one per band).
// Every pair (p, p + delta), delta in the band, with at least one end owned
// by the block is scored once per block: rows p in [s - dhi, s + B) (dhi =
// dlo + 31) against the band's offsets. Each thread owns an 8-row x 8-offset
// unit of that rectangle and keeps its 64 sums in registers; B + dhi = 512
// rows make 256 units, one per thread. The rows [s - dhi, s + B + dhi) of the
// point matrix (gathered through sigma) are staged in shared memory 16
// coordinates at a time, coordinate-major (xs[c][row]) so that a thread reads
// 4 consecutive rows of one coordinate with one 16-byte load, by 4-byte
// cp.async copies double-buffered against the arithmetic. The finished band
// of distances reuses the staging buffers; then the thread owning position p
// merges the band's right neighbours (p, p + delta) and left neighbours
// (p - delta, p) into point sigma[p]'s list, held in registers.
//
// Pairs with ends in two blocks are scored by both, with the same arithmetic
// in the same coordinate order, so both see the same value; (x_p - x_q)^2 and
// (x_q - x_p)^2 are equal, so a pair scores the same in every tree.
#include <cuda_runtime.h>
#include <math.h>

#include "hf_internal.cuh"
#include "topk_list.cuh"

namespace {

// Threads per block = units per block: 256 for bands up to offset 480 and
// 512 (two blocks' worth of unit rows) beyond, where B = ROWS - dhi would
// otherwise fall below 32 owned positions.
constexpr int DC = 16;          // coordinates per staged chunk
constexpr int UR = 8;           // rows per unit
constexpr int UC = 8;           // offsets per unit
constexpr int WB = 32;          // offsets per band (launch)
constexpr int OG = WB / UC;     // offset groups per band
__host__ __device__ constexpr int rows_of(int nt) { return nt * UR * UC / WB; }  // unit rows: B + dhi

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(dst);
  const int sz = valid ? 4 : 0;  // 0: zero-fill, nothing read
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(saddr), "l"(src), "r"(sz) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Row pitch of the staging buffers: a multiple of 4 floats (16-byte loads)
// with an odd number of 16-byte groups, so that rows 8 apart do not share
// banks.
__host__ __device__ __forceinline__ int staging_pitch(int NR) {
  const int p = (NR + 3) & ~3;
  return ((p >> 2) & 1) ? p : p + 4;
}

// Slot of staged row r inside a coordinate column: rows move in groups of 4
// (one 16-byte load); group index bit 3 is folded into bit 0 so that the five
// b-blocks a quarter-warp reads (groups 2m + q, five consecutive m) fall into
// five different bank quads.
__device__ __forceinline__ int rslot(int r) {
  const int gq = r >> 2;
  return ((gq ^ ((gq >> 3) & 1)) << 2) | (r & 3);
}

// Stage coordinates [c0, c0 + DC) of staged rows [0, NR) into buf[c][row].
// Lanes take 16 consecutive coordinates of 2 rows: 64-byte global segments.
__device__ __forceinline__ void stage_chunk(float* buf, int NRP, int NR, const uint32_t* srow,
                                            const float* __restrict__ x, int d, int c0) {
  for (int e = threadIdx.x; e < NR * DC; e += blockDim.x) {
    const int r = e >> 4, c = e & (DC - 1);
    const uint32_t pid = srow[r];
    const bool ok = pid != 0xffffffffu && c0 + c < d;
    const float* src = ok ? x + (size_t)pid * d + c0 + c : x;
    cp_async4(buf + c * NRP + rslot(r), src, ok);
  }
}



// One band of offsets [dlo, dlo + WB - 1] for the block's positions.
// HAM: the rows are binary sketches (d 32-bit words each) and the distance is
// their Hamming distance (the paper's second-stage filter); otherwise float32
// squared Euclidean distance with exact coordinate differences.
template <int KP, int NT, bool HAM>
__global__ void __launch_bounds__(NT, 512 / NT)
window_kernel(const float* __restrict__ x, int64_t n, int d, const uint32_t* __restrict__ sigma, int w,
              int B, int dlo, uint32_t* __restrict__ lidx, float* __restrict__ ldist,
              const uint32_t* __restrict__ segr, const int64_t* __restrict__ segoff) {
  constexpr int ROWS = rows_of(NT);
  extern __shared__ __align__(16) float smem[];
  const int dhi = dlo + WB - 1;
  const int NR = B + 2 * dhi;  // staged rows
  const int NRP = staging_pitch((NR + 7) & ~7);
  float* buf0 = smem;
  float* buf1 = smem + DC * NRP;
  const int stage_floats = 2 * DC * NRP > ROWS * WB ? 2 * DC * NRP : ROWS * WB;
  uint32_t* srow = reinterpret_cast<uint32_t*>(smem + stage_floats);
  float* band = smem;  // [ROWS][WB], after the distance phase

  const int64_t s = (int64_t)blockIdx.x * B;
  const int64_t r0 = s - dhi;  // position of staged row 0
  for (int r = threadIdx.x; r < NR; r += NT) {
    const int64_t p = r0 + r;
    srow[r] = (p >= 0 && p < n) ? __ldg(sigma + p) : 0xffffffffu;
  }
  __syncthreads();

  // unit of this thread: staged rows pr .. pr+7, offsets dlo + 8o .. dlo + 8o + 7
  const int g = threadIdx.x / OG, o = threadIdx.x % OG;
  const int pr = UR * g;
  const int br = pr + dlo - 1 + UC * o;  // staged row of b[0] (a multiple of 8)

  float acc[UR][UC];
#pragma unroll
  for (int t = 0; t < UR; ++t)
#pragma unroll
    for (int c = 0; c < UC; ++c) acc[t][c] = 0.f;

  const int nchunks = (d + DC - 1) / DC;
  stage_chunk(buf0, NRP, NR, srow, x, d, 0);
  cp_async_commit();
  for (int ch = 0; ch < nchunks; ++ch) {
    float* cur = (ch & 1) ? buf1 : buf0;
    float* nxt = (ch & 1) ? buf0 : buf1;
    if (ch + 1 < nchunks) stage_chunk(nxt, NRP, NR, srow, x, d, (ch + 1) * DC);
    cp_async_commit();
    cp_async_wait_1();
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < DC; ++j) {
      const float* col = cur + j * NRP;
      float a[UR], b[16];
      *reinterpret_cast<float4*>(a) = *reinterpret_cast<const float4*>(col + rslot(pr));
      *reinterpret_cast<float4*>(a + 4) = *reinterpret_cast<const float4*>(col + rslot(pr + 4));
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(b + 4 * q) = *reinterpret_cast<const float4*>(col + rslot(br + 4 * q));
#pragma unroll
      for (int t = 0; t < UR; ++t)
#pragma unroll
        for (int c = 0; c < UC; ++c) {
          if (HAM) {
            // integer popcount sums kept in the float registers' bits
            const uint32_t xr = __float_as_uint(a[t]) ^ __float_as_uint(b[1 + t + c]);
            acc[t][c] = __uint_as_float(__float_as_uint(acc[t][c]) + (uint32_t)__popc(xr));
          } else {
            const float e = a[t] - b[1 + t + c];
            acc[t][c] = fmaf(e, e, acc[t][c]);
          }
        }
    }
    __syncthreads();
  }
  cp_async_wait_0();
  __syncthreads();

  // band[row][delta - dlo], row = staged row of p (rows < ROWS)
#pragma unroll
  for (int t = 0; t < UR; ++t)
#pragma unroll
    for (int c = 0; c < UC; ++c)
      band[(pr + t) * WB + UC * o + c] = HAM ? (float)__float_as_uint(acc[t][c]) : acc[t][c];
  __syncthreads();

  // merge: positions s + tt, tt < B; the point's list is held in registers
  const int wtop = min(dhi, w);
  for (int tt = threadIdx.x; tt < B; tt += NT) {
    const int64_t p = s + tt;
    if (p >= n) break;
    const int rowp = tt + dhi;  // staged row of p
    const uint32_t ip = srow[rowp];
    ListK<KP> L;
    L.load(ldist + (size_t)ip * KP, lidx + (size_t)ip * KP);
    // positions of p's set (segmented forest: the set's block of the order)
    int64_t plo = 0, phi = n;
    if (segr) {
      const uint32_t sg = __ldg(segr + ip);
      plo = __ldg(segoff + sg);
      phi = __ldg(segoff + sg + 1);
    }
    const int rmax = (int)(phi - 1 - p < wtop ? phi - 1 - p : wtop);  // right: (p, p + delta)
    for (int delta = dlo; delta <= rmax; ++delta) L.offer(band[rowp * WB + delta - dlo], srow[rowp + delta]);
    const int lmax = (int)(p - plo < wtop ? p - plo : wtop);  // left: (p - delta, p)
    for (int delta = dlo; delta <= lmax; ++delta)
      L.offer(band[(rowp - delta) * WB + delta - dlo], srow[rowp - delta]);
    L.store(ldist + (size_t)ip * KP, lidx + (size_t)ip * KP);
  }
}

__global__ void list_init_kernel(uint32_t* __restrict__ idx, float* __restrict__ dist, int64_t count) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    idx[e] = 0xffffffffu;
    dist[e] = INFINITY;
  }
}

size_t window_smem(int B, int dhi, int rows) {
  const int NR = B + 2 * dhi;
  const size_t staging = (size_t)2 * DC * staging_pitch((NR + 7) & ~7);
  const size_t bandf = (size_t)rows * WB;
  return ((staging > bandf ? staging : bandf) + (size_t)NR) * 4;
}

template <int KP, int NT, bool HAM>
int launch_band(const float* x, int64_t n, int d, const uint32_t* sigma, int w, int dlo, uint32_t* li, float* ldd,
                cudaStream_t s, const uint32_t* segr, const int64_t* segoff) {
  const int dhi = dlo + WB - 1;
  const int B = rows_of(NT) - dhi;
  const size_t smem = window_smem(B, dhi, rows_of(NT));
  if (B < 32 || smem > 227 * 1024) return HF_ENOTIMPL;
  if (cudaFuncSetAttribute((const void*)window_kernel<KP, NT, HAM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return HF_ECUDA;
  window_kernel<KP, NT, HAM><<<hf_blocks(n, B), NT, smem, s>>>(x, n, d, sigma, w, B, dlo, li, ldd, segr, segoff);
  hf_after_launch(HAM ? "window_kernel<hamming>" : "window_kernel", s);
  return HF_OK;
}

// nt: block threads (256 or 512; 0 picks 256 while its blocks keep 32
// positions, else 512)
template <int KP, bool HAM>
int launch_kp(const float* x, int64_t n, int d, const uint32_t* sigma, int w, uint32_t* li, float* ldd,
              cudaStream_t s, const uint32_t* segr, const int64_t* segoff, int nt) {
  for (int dlo = 1; dlo <= w; dlo += WB) {
    const int dhi = dlo + WB - 1;
    const bool small = nt == 256 || (nt == 0 && rows_of(256) - dhi >= 32);
    const int rc = small ? launch_band<KP, 256, HAM>(x, n, d, sigma, w, dlo, li, ldd, s, segr, segoff)
                         : launch_band<KP, 512, HAM>(x, n, d, sigma, w, dlo, li, ldd, s, segr, segoff);
    if (rc != HF_OK) return rc;
  }
  return HF_OK;
}

}  // namespace

void launch_list_init(uint32_t* idx, float* dist, int64_t count, cudaStream_t s) {
  list_init_kernel<<<hf_blocks(count, 256, 152 * 8), 256, 0, s>>>(idx, dist, count);
  hf_after_launch("list_init_kernel", s);
}

int window_list_pitch(int k) { return k <= 16 ? 16 : (k <= 32 ? 32 : 64); }

// One launch per band of 32 offsets; w up to HF_PLAIN_MAX_W (B >= 32 and
// the staging within shared memory). Lists have window_list_pitch(k) slots
// per point.
int launch_window_graph(const float* x, int64_t n, int d, const uint32_t* sigma, int w, int kp,
                        uint32_t* list_idx, float* list_dist, cudaStream_t s, const uint32_t* segr,
                        const int64_t* segoff, int nt) {
  if (nt != 0 && nt != 256 && nt != 512) return HF_EINVAL;
  switch (kp) {
    case 16: return launch_kp<16, false>(x, n, d, sigma, w, list_idx, list_dist, s, segr, segoff, nt);
    case 32: return launch_kp<32, false>(x, n, d, sigma, w, list_idx, list_dist, s, segr, segoff, nt);
    case 64: return launch_kp<64, false>(x, n, d, sigma, w, list_idx, list_dist, s, segr, segoff, nt);
    default: return HF_EINVAL;
  }
}

int launch_window_hamming(const uint32_t* sketch, int64_t n, int words, const uint32_t* sigma, int w, int kp,
                          uint32_t* list_idx, float* list_dist, cudaStream_t s, const uint32_t* segr,
                          const int64_t* segoff) {
  const float* x = reinterpret_cast<const float*>(sketch);  // staged as raw 32-bit words
  switch (kp) {
    case 16: return launch_kp<16, true>(x, n, words, sigma, w, list_idx, list_dist, s, segr, segoff, 0);
    case 32: return launch_kp<32, true>(x, n, words, sigma, w, list_idx, list_dist, s, segr, segoff, 0);
    case 64: return launch_kp<64, true>(x, n, words, sigma, w, list_idx, list_dist, s, segr, segoff, 0);
    default: return HF_EINVAL;
  }
}
