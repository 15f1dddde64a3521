// Batched query search.
//
// Paper, Section 2: since the Hilbert order is a total order, binary search
// locates an arbitrary point in a sorted set; Algorithm 1 then takes the
// candidates near each query's position in every tree and keeps the top k by
// vector distance. The paper simulates a collective Hilbert sort of all queries
// on the CPU; here every query is located independently, which parallelises
// trivially.
//
// One warp per query, looping over the trees, so the query's top-k list stays
// in shared memory for the whole search. Per tree, lane 0 computes the query's
// key prefix; the warp locates it among the sorted prefixes with 32-way
// probing rounds; when the query's prefix equals some data prefixes, lane 0
// refines the position inside that run by comparing full keys (computed on
// demand from the bit planes). The window's candidates are scored 32 at a
// time, one per lane over the whole vector (sequential float32 sum with exact
// differences), sorted across the warp, and merged in ascending order until
// the first one that cannot enter the list.
#include <cuda_runtime.h>
#include <math.h>

#include "hf_internal.cuh"
#include "hilbert_device.cuh"

namespace {

constexpr int SWARPS = 4;

// Shared bytes per warp: list (k floats + k ids), query prefix (K words), two
// coordinate scratch rows (d bytes each), rounded to 16.
__host__ __device__ __forceinline__ size_t search_per_warp(int k, int K, int d) {
  return ((size_t)k * 8 + (size_t)K * 8 + 2 * (size_t)d + 15) & ~(size_t)15;
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
  int vec4;  // d % 4 == 0 and both matrices 16-byte aligned
  const uint64_t* qkeys;  // [nq][T][K] query key prefixes, or null: computed in the search kernel
};

// Key prefixes of every (query, tree) pair, one thread each, so the search
// kernel's lanes do not wait on a serial transform.
__global__ void query_keys_kernel(const uint8_t* __restrict__ qcodes, int64_t nq, int d, int bits, int K, int L,
                                  int T, int W32, const int32_t* __restrict__ pi, const uint32_t* __restrict__ rbits,
                                  uint64_t* __restrict__ out) {
  extern __shared__ uint8_t smy[];
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nq * T) return;
  const int64_t qi = e / T;
  const int t = (int)(e - qi * T);
  uint8_t* Y = smy + (size_t)threadIdx.x * d;
  hf_load_coords_codes(qcodes + (size_t)qi * d, d, bits, L, pi + (size_t)t * d, rbits + (size_t)t * W32, Y);
  hf_skilling(Y, d, L);
  for (int w = 0; w < K; ++w) out[(size_t)e * K + w] = hf_pack_word(Y, d, L, w);
}

// Warp-wide lower bound over the sorted prefixes: each round the 32 lanes
// probe 32 evenly spaced positions of [lo, hi) (one round trip), a ballot
// keeps the sub-interval that holds the first position whose prefix is not
// below the query's (le = false) or above it (le = true). About log32(n)
// rounds instead of log2(n) dependent steps.
__device__ __forceinline__ int64_t warp_bound(const uint64_t* __restrict__ pre, int64_t n, int K, const uint64_t* qp,
                                              bool le, int lane) {
  int64_t lo = 0, hi = n;  // answer in [lo, hi]
  while (hi - lo > 0) {
    const int64_t len = hi - lo;
    const int64_t step = (len + 31) / 32;
    const int64_t m = lo + (int64_t)lane * step;
    bool below = false;  // position m lies before the answer
    if (m < hi) {
      const int c = cmp_prefix(pre, n, K, m, qp);
      below = le ? (c <= 0) : (c < 0);
    }
    const uint32_t bm = __ballot_sync(0xffffffffu, below);
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
      const float od = __shfl_xor_sync(0xffffffffu, dv, j);
      const uint32_t oi = __shfl_xor_sync(0xffffffffu, iv, j);
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

__global__ void __launch_bounds__(SWARPS * 32) search_kernel(SearchArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const size_t per_warp = search_per_warp(a.k, a.K, a.d);
  unsigned char* base = smraw + per_warp * wib;
  float* ldst = reinterpret_cast<float*>(base);
  uint32_t* lidx = reinterpret_cast<uint32_t*>(ldst + a.k);
  uint64_t* qp = reinterpret_cast<uint64_t*>(lidx + a.k);  // 8k bytes in: 8-byte aligned
  uint8_t* Yq = reinterpret_cast<uint8_t*>(qp + a.K);
  uint8_t* Yd = Yq + a.d;

  const int64_t qi = (int64_t)blockIdx.x * SWARPS + wib;
  if (qi >= a.nq) return;
  const uint8_t* qc = a.qcodes + (size_t)qi * a.d;
  const float* qv = a.q + (size_t)qi * a.d;

  for (int j = lane; j < a.k; j += 32) {
    ldst[j] = INFINITY;
    lidx[j] = 0xffffffffu;
  }
  __syncwarp();

  const int t_begin = a.only_tree >= 0 ? a.only_tree : 0;
  const int t_end = a.only_tree >= 0 ? a.only_tree + 1 : a.T;
  for (int t = t_begin; t < t_end; ++t) {
    const int32_t* pi = a.pi + (size_t)t * a.d;
    const uint32_t* rb = a.rbits + (size_t)t * a.W32;
    const uint64_t* pre = a.prefix + (size_t)t * a.K * a.n;
    const uint32_t* sig = a.sigma + (size_t)t * a.n;
    if (a.qkeys) {
      if (lane < a.K) qp[lane] = __ldg(a.qkeys + ((size_t)qi * a.T + t) * a.K + lane);
    } else if (lane == 0) {
      hf_load_coords_codes(qc, a.d, a.bits, a.L, pi, rb, Yq);
      hf_skilling(Yq, a.d, a.L);
      for (int w = 0; w < a.K; ++w) qp[w] = hf_pack_word(Yq, a.d, a.L, w);
    }
    __syncwarp();
    // [lo, lo2): positions whose prefix equals the query's
    int64_t lo = warp_bound(pre, a.n, a.K, qp, false, lane);
    const int64_t lo2 = warp_bound(pre, a.n, a.K, qp, true, lane);
    int64_t pos = lo;
    if (lo2 > lo && a.K < a.W) {
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
      pos = __shfl_sync(0xffffffffu, pos, 0);
    }
    if (a.only_tree >= 0) {
      if (lane == 0) a.out_pos[qi] = pos;
      continue;
    }
    const int64_t c0 = pos - a.w > 0 ? pos - a.w : 0;
    const int64_t c1 = pos + a.w < a.n ? pos + a.w : a.n;
    for (int64_t cb = c0; cb < c1; cb += 32) {
      // lane j scores candidate cb + j over the whole vector
      const int64_t c = cb + lane;
      float dist = INFINITY;
      uint32_t pid = 0xffffffffu;
      if (c < c1) {
        pid = __ldg(sig + c);
        const float* xv = a.x + (size_t)pid * a.d;
        float acc = 0.f;
        if (a.vec4) {
          for (int j = 0; j < a.d; j += 4) {
            const float4 qa = __ldg(reinterpret_cast<const float4*>(qv + j));
            const float4 xa = __ldg(reinterpret_cast<const float4*>(xv + j));
            float e = qa.x - xa.x;
            acc = fmaf(e, e, acc);
            e = qa.y - xa.y;
            acc = fmaf(e, e, acc);
            e = qa.z - xa.z;
            acc = fmaf(e, e, acc);
            e = qa.w - xa.w;
            acc = fmaf(e, e, acc);
          }
        } else {
          for (int j = 0; j < a.d; ++j) {
            const float e = __ldg(qv + j) - __ldg(xv + j);
            acc = fmaf(e, e, acc);
          }
        }
        dist = acc;
      }
      warp_sort(dist, pid, lane);
      // merge in ascending order; stop at the first that cannot enter
      for (int u = 0; u < 32; ++u) {
        const float cd = __shfl_sync(0xffffffffu, dist, u);
        const uint32_t ci = __shfl_sync(0xffffffffu, pid, u);
        if (ci == 0xffffffffu) break;
        if (!lessp(cd, ci, ldst[a.k - 1], lidx[a.k - 1])) break;
        if (lane == 0) {
          bool dup = false;
          for (int j = 0; j < a.k; ++j) dup |= (lidx[j] == ci);
          if (!dup) {
            int j = a.k - 1;
            while (j > 0 && lessp(cd, ci, ldst[j - 1], lidx[j - 1])) {
              ldst[j] = ldst[j - 1];
              lidx[j] = lidx[j - 1];
              --j;
            }
            ldst[j] = cd;
            lidx[j] = ci;
          }
        }
        __syncwarp();
      }
    }
  }
  if (a.only_tree >= 0) return;
  __syncwarp();
  for (int j = lane; j < a.k; j += 32) {
    a.out_idx[(size_t)qi * a.k + j] = lidx[j];
    a.out_dist[(size_t)qi * a.k + j] = ldst[j];
  }
}

}  // namespace

int launch_search(const hf_forest* f, const float* q, const uint8_t* qcodes, int64_t nq, int k, int w,
                  uint32_t* out_idx, float* out_dist, int64_t* out_pos, int only_tree, cudaStream_t s,
                  uint64_t* qkeys) {
  SearchArgs a;
  a.qkeys = nullptr;
  if (qkeys && only_tree < 0) {
    int t = 256;
    while (t > 32 && (size_t)t * f->d > 96 * 1024) t >>= 1;
    const size_t sm = (size_t)t * f->d;
    if (sm > 48 * 1024)
      cudaFuncSetAttribute((const void*)query_keys_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    query_keys_kernel<<<hf_blocks(nq * f->T, t), t, sm, s>>>(qcodes, nq, f->d, f->bits, f->K, f->L, f->T, f->W32,
                                                               f->pi, f->rbits, qkeys);
    hf_after_launch("query_keys_kernel", s);
    a.qkeys = qkeys;
  }
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
  a.only_tree = only_tree;
  a.vec4 = (f->d % 4 == 0) && ((reinterpret_cast<uintptr_t>(f->x) & 15) == 0) &&
           ((reinterpret_cast<uintptr_t>(q) & 15) == 0);
  const size_t smem = search_per_warp(k, f->K, f->d) * SWARPS;
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute((const void*)search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess)
    return HF_ECUDA;
  search_kernel<<<hf_blocks(nq, SWARPS), SWARPS * 32, smem, s>>>(a); hf_after_launch("search_kernel", s);
  return cudaGetLastError() == cudaSuccess ? HF_OK : HF_ECUDA;
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
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return HF_ECUDA;
  if (rc != HF_OK) return rc;
  int word = 0;
  if (cudaMemcpy(&word, f->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HF_ECUDA;
  if (word) {
    cudaMemset(f->err, 0, sizeof(int));
    return (word & HF_ERRBIT_NONFINITE) ? HF_ENONFINITE : HF_ETIMEOUT;
  }
  return HF_OK;
}
