// C-ABI entry points and the host runtime around the kernels: argument
// checks, host/device buffer resolution, the forest's allocations, the
// per-tree loop, the device error word and per-phase CUDA-event timings.
#include <cuda_runtime.h>
#include <string.h>

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "hf_internal.cuh"

size_t sort_status_words(int64_t n, int K, int tb);
int tie_small_cap(int W, int d, int bits, int K, int K2);
size_t tie_scratch_words(int W, int d, int bits, int K, int K2);

namespace {

constexpr uint64_t GOLDEN_GAMMA = 0x9E3779B97F4A7C15ull;

uint64_t splitmix64_next(uint64_t& state) {
  state += GOLDEN_GAMMA;
  uint64_t z = state;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// 1: device-accessible, 0: host memory, -1: error
int classify(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? 1 : 0;
}

// Device memory comes from a library-owned, stream-ordered pool per device:
// a buffer freed at the end of one call (on that call's stream) is handed to
// the next call without a device-wide synchronisation or a trip to the
// driver. The pool keeps up to a quarter of the device's memory (64 GiB at
// most) cached between calls; hf_trim_pool returns it.
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};

cudaMemPool_t device_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    size_t fr = 0, tot = 0;
    uint64_t keep = 64ull << 30;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && tot / 4 < keep) keep = tot / 4;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

}  // namespace

cudaError_t hf_dalloc_bytes(void** p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  cudaMemPool_t pool = device_pool();
  if (!pool) return cudaErrorMemoryAllocation;
  return cudaMallocFromPoolAsync(p, bytes ? bytes : 1, pool, s);
}

void hf_dfree_bytes(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

namespace {

cudaError_t dalloc_bytes(void** p, size_t bytes, cudaStream_t s) { return hf_dalloc_bytes(p, bytes, s); }

template <typename T>
cudaError_t dalloc(T** p, size_t count, cudaStream_t s) {
  void* v = nullptr;
  const cudaError_t e = dalloc_bytes(&v, (count ? count : 1) * sizeof(T), s);
  *p = static_cast<T*>(v);
  return e;
}

// Frees in stream order on s: the caller has finished (or enqueued on s)
// every use of p.
template <typename T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(reinterpret_cast<void*>(p), s);
  p = nullptr;
}

int map_cuda(cudaError_t e) {
  if (e == cudaSuccess) return HF_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? HF_ENOMEM : HF_ECUDA;
}

}  // namespace

// Synchronises, reads and clears the error word, maps to a status.
int hf_finish(hf_forest* f, cudaStream_t s) {
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return map_cuda(e);
  e = cudaGetLastError();
  if (e != cudaSuccess) return map_cuda(e);
  int word = 0;
  if (cudaMemcpy(&word, f->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HF_ECUDA;
  if (word) cudaMemset(f->err, 0, sizeof(int));
  if (word & HF_ERRBIT_NONFINITE) return HF_ENONFINITE;
  if (word & HF_ERRBIT_TIMEOUT) return HF_ETIMEOUT;
  return HF_OK;
}

namespace {

int finish(hf_forest* f, cudaStream_t s) { return hf_finish(f, s); }

void free_build_scratch(hf_forest* f, cudaStream_t s) {
  dfree(f->pk, s);
  dfree(f->p0t, s);
  dfree(f->sort.keys_a, s);
  dfree(f->sort.keys_b, s);
  dfree(f->sort.vals_a, s);
  dfree(f->sort.vals_b, s);
  dfree(f->sort.status, s);
  dfree(f->sort.hist, s);
  dfree(f->tie.runs, s);
  dfree(f->tie.big_runs, s);
  dfree(f->tie.counters, s);
  dfree(f->tie.fk, s);
}

void destroy(hf_forest* f, cudaStream_t s) {
  if (!f) return;
  free_build_scratch(f, s);
  dfree(f->x_owned, s);
  dfree(f->lo, s);
  dfree(f->scale, s);
  dfree(f->planes, s);
  dfree(f->pi, s);
  dfree(f->rbits, s);
  dfree(f->prefix, s);
  dfree(f->sigma, s);
  dfree(f->err, s);
  dfree(f->xb, s);
  dfree(f->xmeta, s);
  dfree(f->sketch, s);
  dfree(f->sketch_r, s);
  dfree(f->xm, s);
  dfree(f->posm, s);
  dfree(f->seg_off, s);
  dfree(f->seg, s);
  dfree(f->plan_li, s);
  dfree(f->plan_ld, s);
  dfree(f->plan_xs, s);
  dfree(f->plan_ms, s);
  if (f->side) {
    cudaStreamSynchronize(s);  // the stream-ordered frees above run before the side stream goes
    cudaStreamDestroy(f->side);
  }
  delete f;
}

int parse_options(hf_forest* f, const char* opts) {
  if (!opts) return HF_OK;
  std::string s(opts);
  size_t i = 0;
  while (i < s.size()) {
    size_t j = s.find(',', i);
    if (j == std::string::npos) j = s.size();
    std::string kv = s.substr(i, j - i);
    i = j + 1;
    if (kv.empty()) continue;
    size_t eq = kv.find('=');
    if (eq == std::string::npos) return HF_EINVAL;
    std::string key = kv.substr(0, eq), val = kv.substr(eq + 1);
    char* end = nullptr;
    long long v = strtoll(val.c_str(), &end, 10);
    if (end == val.c_str() || *end) return HF_EINVAL;
    if (key == "prefix_words") {
      if (v < 1 || v > 8) return HF_EINVAL;
      f->K = (int)v;
    } else if (key == "sort_batch") {
      if (v < 1) return HF_EINVAL;
      f->sort_batch_max = (int)v;
    } else if (key == "spin_limit_us") {
      if (v < 1) return HF_EINVAL;
      f->spin_limit_us = v;
    } else if (key == "test_stall") {
      f->test_stall = v ? 1 : 0;
    } else {
      return HF_EINVAL;
    }
  }
  return HF_OK;
}

// Per-call CUDA-event spans. Every event is created by mark(), owned by the
// Timer and destroyed exactly once (an event may end one span and start the
// next).
struct Timer {
  hf_forest* f;
  cudaStream_t s;
  std::vector<cudaEvent_t> events;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> spans[HF_NTIMINGS];
  explicit Timer(hf_forest* ff, cudaStream_t ss) : f(ff), s(ss) {}
  cudaEvent_t mark() { return mark_on(s); }
  cudaEvent_t mark_on(cudaStream_t st) {
    cudaEvent_t e = nullptr;
    if (f->timing && cudaEventCreate(&e) == cudaSuccess) {
      events.push_back(e);
      cudaEventRecord(e, st);
    }
    return e;
  }
  void span(int slot, cudaEvent_t a, cudaEvent_t b) {
    if (a && b) spans[slot].push_back({a, b});
  }
  // after a sync
  void collect(std::initializer_list<int> slots) {
    for (int sl : slots) {
      float tot = 0.f;
      for (auto& p : spans[sl]) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.first, p.second);
        tot += ms;
      }
      if (!spans[sl].empty()) f->timings[sl] = tot;
    }
  }
  Timer(const Timer&) = delete;
  Timer& operator=(const Timer&) = delete;
  ~Timer() {
    for (cudaEvent_t e : events) cudaEventDestroy(e);
  }
};

}  // namespace

// Kernels launched by this library in this process (diagnostic counter).
static std::atomic<uint64_t> g_launches{0};

void hf_after_launch(const char* what, cudaStream_t s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  static const int on = [] {
    const char* v = getenv("HF_DEBUG");
    return v && *v && *v != '0';
  }();
  if (!on) return;
  // peek: the error stays set for the entry point's final check
  cudaError_t e = cudaPeekAtLastError();
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (e == cudaSuccess && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
    e = cudaStreamSynchronize(s);  // no synchronisation while a graph is being captured
  fprintf(stderr, "[hf] %s: %s\n", what, cudaGetErrorString(e));
  fflush(stderr);
}

void hf_tree_params_host(uint64_t seed, int tree, int d, int32_t* pi, uint8_t* r) {
  uint64_t state = seed + (uint64_t)(tree + 1) * GOLDEN_GAMMA;
  for (int j = 0; j < d; ++j) pi[j] = j;
  for (int j = d - 1; j >= 1; --j) {
    const uint64_t m = splitmix64_next(state) % (uint64_t)(j + 1);
    const int32_t tmp = pi[j];
    pi[j] = pi[m];
    pi[m] = tmp;
  }
  for (int j = 0; j < d; ++j) r[j] = (uint8_t)(splitmix64_next(state) >> 63);
}

extern "C" {

const char* hf_status_string(int status) {
  switch (status) {
    case HF_OK: return "ok";
    case HF_EINVAL: return "invalid argument";
    case HF_ENOMEM: return "device allocation failed";
    case HF_ECUDA: return "CUDA error";
    case HF_ENONFINITE: return "non-finite input value";
    case HF_ETIMEOUT: return "bounded wait between blocks timed out";
    case HF_ESTATE: return "forest does not hold the needed state";
    case HF_ENOTIMPL: return "not implemented for these arguments";
    default: return "unknown status";
  }
}

uint64_t hf_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int hf_tree_params(uint64_t seed, int32_t tree, int32_t d, int32_t* pi, uint8_t* r) {
  if (!pi || !r || d < 1 || d > HF_MAX_D || tree < 0) return HF_EINVAL;
  hf_tree_params_host(seed, tree, d, pi, r);
  return HF_OK;
}

int hf_build(const float* points, int64_t n, int32_t d, int32_t T, int32_t bits, uint64_t seed,
             void* stream, hf_forest** out) {
  return hf_build_opts(points, n, d, T, bits, seed, nullptr, stream, out);
}

static int build_impl(const float* points, int64_t n, int32_t d, int32_t T, int32_t bits, uint64_t seed,
                      const char* options, int nseg, const int64_t* seg_off, void* stream, hf_forest** out) {
  if (out) *out = nullptr;
  if (!points || !out || n < 2 || n > HF_MAX_N || d < 1 || d > HF_MAX_D || T < 1 || bits < 1 ||
      bits > HF_MAX_BITS)
    return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();  // an earlier call's error was reported by that call
  hf_forest* f = new hf_forest();
  f->nseg = nseg;
  if (nseg > 1) f->seg_off_h.assign(seg_off, seg_off + nseg + 1);
  f->n = n;
  f->d = d;
  f->T = T;
  f->bits = bits;
  f->seed = seed;
  f->W = (int)(((int64_t)d * bits + 63) / 64);
  f->W32 = (d + 31) / 32;
  f->K = f->W < 2 ? f->W : 2;
  int rc = parse_options(f, options);
  if (rc == HF_OK && f->K > f->W) rc = HF_EINVAL;
  if (rc != HF_OK) {
    delete f;
    return rc;
  }
  {
    const int64_t need = ((int64_t)64 * f->K + d - 1) / d;
    f->L = (int)(need < bits ? need : bits);
    // With L > 1, words past the sorted prefix that come from the same L top
    // levels are computed with it (up to four): they settle equal prefixes
    // cheaply. On the top-level path (L = 1) the fix-up forms them itself
    // with ballots for the tied points only, which costs less than computing
    // them for every point.
    f->K2 = f->K;
    if (f->L > 1)
      while (f->K2 < f->W && f->K2 < f->K + 4 && (int64_t)64 * (f->K2 + 1) <= (int64_t)d * f->L) ++f->K2;
  }
  cudaGetDevice(&f->device);

  Timer tm(f, s);
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess && x != cudaSuccess) e = x;
  };
  const int dev = classify(points);
  if (dev == 1) {
    f->x = points;
  } else {
    chk(dalloc(&f->x_owned, (size_t)n * d, s));
    if (e == cudaSuccess)
      chk(cudaMemcpyAsync(f->x_owned, points, (size_t)n * d * sizeof(float), cudaMemcpyHostToDevice, s));
    f->x = f->x_owned;
  }
  const int K = f->K, W32 = f->W32;
  // Trees are keyed and sorted in batches of TB (all of them when the
  // batch's scratch fits in half of the free device memory, 16 GiB at most).
  {
    const int64_t ntiles = (n + 2047) / 2048;  // sort tiles (status words per tile)
    const double per_tree = (double)n * (8.0 * f->K2 + 24.0) + (double)(ntiles + 1) * 256 * 4 * 8 * K;
    size_t fr = 0, tot = 0;
    double budget = 16.0 * (1ull << 30);
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && 0.5 * (double)fr < budget) budget = 0.5 * (double)fr;
    else cudaGetLastError();
    const double tbd = budget / per_tree;
    f->TB = tbd >= T ? T : (tbd < 1.0 ? 1 : (int)tbd);
    if (f->sort_batch_max > 0 && f->TB > f->sort_batch_max) f->TB = f->sort_batch_max;
  }
  const int TB = f->TB;
  chk(dalloc(&f->lo, (size_t)nseg * d, s));
  chk(dalloc(&f->scale, (size_t)nseg * d, s));
  uint64_t* seg64 = nullptr;
  if (nseg > 1) {
    chk(dalloc(&f->seg_off, (size_t)nseg + 1, s));
    chk(dalloc(&f->seg, (size_t)n, s));
    chk(dalloc(&seg64, (size_t)n, s));
  }
  chk(dalloc(&f->planes, (size_t)bits * n * W32, s));
  chk(dalloc(&f->pi, (size_t)T * d, s));
  chk(dalloc(&f->rbits, (size_t)T * W32, s));
  chk(dalloc(&f->prefix, (size_t)T * K * n, s));
  chk(dalloc(&f->sigma, (size_t)T * n, s));
  chk(dalloc(&f->err, 1, s));
  chk(dalloc(&f->pk, (size_t)TB * f->K2 * n, s));
  const bool sliced = prefix_top_path(d, f->K2, f->L);
  if (sliced) chk(dalloc(&f->p0t, (size_t)((n + 31) / 32) * d, s));
  chk(dalloc(&f->sort.keys_a, (size_t)TB * n, s));
  chk(dalloc(&f->sort.keys_b, (size_t)TB * n, s));
  chk(dalloc(&f->sort.vals_a, (size_t)TB * n, s));
  chk(dalloc(&f->sort.vals_b, (size_t)TB * n, s));
  chk(dalloc(&f->sort.status, sort_status_words(n, K, TB), s));
  chk(dalloc(&f->sort.hist, (size_t)TB * K * 8 * 256, s));
  const int cap = tie_small_cap(f->W, d, bits, K, f->K2);
  f->tie.big_cap = n / (cap + 1) + 1;
  chk(dalloc(&f->tie.runs, (size_t)(n / 2 + 1), s));
  chk(dalloc(&f->tie.big_runs, (size_t)T * f->tie.big_cap, s));
  chk(dalloc(&f->tie.counters, (size_t)T * 4, s));
  chk(dalloc(&f->tie.fk, K < f->W ? tie_scratch_words(f->W, d, bits, K, f->K2) : 1, s));
  void* rscratch = nullptr;
  const size_t rbytes = range_scratch_bytes(n, d);
  chk(dalloc_bytes(&rscratch, rbytes, s));
  if (e != cudaSuccess) {
    dfree(rscratch, s);
    dfree(seg64, s);
    destroy(f, s);
    return map_cuda(e);
  }
  cudaMemsetAsync(f->err, 0, sizeof(int), s);
  if (nseg > 1) {
    cudaMemcpyAsync(f->seg_off, f->seg_off_h.data(), (size_t)(nseg + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    launch_seg_of_row(f->seg_off, nseg, n, f->seg, seg64, s);
  }
  cudaMemsetAsync(f->tie.counters, 0, (size_t)T * 4 * sizeof(uint32_t), s);

  // per-tree permutations and reflection masks (host, then one upload)
  std::vector<int32_t> hpi((size_t)T * d);
  std::vector<uint32_t> hr((size_t)T * W32, 0u);
  std::vector<uint8_t> r(d);
  for (int t = 0; t < T; ++t) {
    hf_tree_params_host(seed, t, d, hpi.data() + (size_t)t * d, r.data());
    for (int j = 0; j < d; ++j)
      if (r[j]) hr[(size_t)t * W32 + (j >> 5)] |= 1u << (j & 31);
  }
  cudaMemcpyAsync(f->pi, hpi.data(), hpi.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(f->rbits, hr.data(), hr.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s);

  cudaEvent_t a0 = tm.mark();
  if (nseg > 1)
    launch_seg_range(f->x, d, f->seg_off, nseg, bits, f->lo, f->scale, f->err, s);
  else
    launch_range(f->x, n, d, f->lo, f->scale, bits, f->err, rscratch, rbytes, s);
  launch_quantize_planes(f->x, n, d, f->lo, f->scale, bits, f->planes, f->err, s, nseg > 1 ? f->seg : nullptr);
  if (sliced) launch_plane0_slice(f->planes, n, d, f->p0t, s);
  cudaEvent_t a1 = tm.mark();
  tm.span(0, a0, a1);
  for (int t0 = 0; t0 < T && rc == HF_OK; t0 += TB) {
    const int tb = T - t0 < TB ? T - t0 : TB;
    cudaEvent_t k0 = tm.mark();
    for (int j = 0; j < tb; ++j) {
      const int t = t0 + j;
      launch_prefix_keys(f->planes, f->p0t, n, d, bits, f->K2, f->L, f->pi + (size_t)t * d, f->rbits + (size_t)t * W32,
                         f->pk + (size_t)j * f->K2 * n, s);
    }
    cudaEvent_t k1 = tm.mark();
    rc = sort_batch(f, t0, tb, s);
    cudaEvent_t k2 = tm.mark();
    tm.span(1, k0, k1);
    tm.span(2, k1, k2);
  }
  if (rc == HF_OK) rc = finish(f, s);
  // runs of equal prefixes longer than the on-device cap
  if (rc == HF_OK) {
    std::vector<uint32_t> ctr((size_t)T * 4);
    if (cudaMemcpy(ctr.data(), f->tie.counters, ctr.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) rc = HF_ECUDA;
    cudaEvent_t b0 = tm.mark();
    for (int t = 0; t < T && rc == HF_OK; ++t) rc = tie_fixup_big(f, t, ctr[(size_t)t * 4 + 1], s);
    cudaEvent_t b1 = tm.mark();
    tm.span(3, b0, b1);
    if (rc == HF_OK && nseg > 1) {
      cudaEvent_t c0 = tm.mark();
      rc = segment_pass(f, seg64, s);
      cudaEvent_t c1 = tm.mark();
      tm.span(2, c0, c1);
    }
    if (rc == HF_OK) rc = finish(f, s);
  }
  dfree(rscratch, s);
  dfree(seg64, s);
  if (rc == HF_OK) {
    tm.collect({0, 1, 2, 3});
    // keys, prefix gather and tie kernels per tree; histogram, scan and 8K
    // passes per batch
    const int nb = (T + TB - 1) / TB;
    f->timings[6] = (float)(T * (1 + (K > 1 ? 1 : 0) + (K < f->W ? 2 : 0)) + nb * (2 + 8 * K));
  }
  free_build_scratch(f, s);
  if (rc != HF_OK) {
    destroy(f, s);
    return rc;
  }
  *out = f;
  return HF_OK;
}

int hf_build_opts(const float* points, int64_t n, int32_t d, int32_t T, int32_t bits, uint64_t seed,
                  const char* options, void* stream, hf_forest** out) {
  return build_impl(points, n, d, T, bits, seed, options, 1, nullptr, stream, out);
}

int hf_build_segmented(const float* points, const int64_t* offsets, int32_t nsets, int32_t d, int32_t T, int32_t bits,
                       uint64_t seed, const char* options, void* stream, hf_forest** out) {
  if (out) *out = nullptr;
  if (!offsets || nsets < 1 || nsets > HF_MAX_SETS || offsets[0] != 0) return HF_EINVAL;
  for (int g = 0; g < nsets; ++g)
    if (offsets[g + 1] - offsets[g] < 2) return HF_EINVAL;  // every set holds two points at least
  if (nsets == 1) return build_impl(points, offsets[1], d, T, bits, seed, options, 1, nullptr, stream, out);
  return build_impl(points, offsets[nsets], d, T, bits, seed, options, nsets, offsets, stream, out);
}

int hf_free(hf_forest* f) {
  if (!f) return HF_OK;
  cudaDeviceSynchronize();  // no use of the forest's memory is still in flight
  destroy(f, 0);
  return HF_OK;
}

int hf_trim_pool(void) {
  cudaMemPool_t pool = device_pool();
  if (!pool) return HF_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
    cudaGetLastError();
    return HF_ECUDA;
  }
  return HF_OK;
}

int hf_set_option(hf_forest* f, const char* key, int64_t value) {
  if (!f || !key) return HF_EINVAL;
  std::string k(key);
  if (k == "mode") {
    if (value < 0 || value > 3) return HF_EINVAL;
    f->mode = (int)value;
  } else if (k == "sketch_k2") {
    if (value < 1 || value > HF_MAX_K2) return HF_EINVAL;
    f->sketch_k2 = (int)value;
  } else if (k == "expand_h") {
    if (value < 0 || value > (1 << 20)) return HF_EINVAL;
    f->expand_h = (int)value;
  } else if (k == "tensor_slack") {
    if (value < -1 || value > 64) return HF_EINVAL;
    f->tensor_slack = (int)value;
  } else if (k == "timing") {
    f->timing = value ? 1 : 0;
  } else {
    return HF_EINVAL;
  }
  return HF_OK;
}

int hf_get_timings(const hf_forest* f, float* out_ms, int32_t cap) {
  if (!f || !out_ms || cap < 0) return HF_EINVAL;
  for (int i = 0; i < cap && i < HF_NTIMINGS; ++i) out_ms[i] = f->timings[i];
  return HF_OK;
}

int hf_info(const hf_forest* f, int64_t* out, int32_t cap) {
  if (!f || !out || cap < 0) return HF_EINVAL;
  const int64_t v[8] = {f->n, f->d, f->T, f->bits, f->W, f->K, f->K2, f->L};
  for (int i = 0; i < cap && i < 8; ++i) out[i] = v[i];
  return HF_OK;
}

}  // extern "C"

namespace {

// The graph over the first T_use trees. wpt / tpt (device, per point; both or
// neither): point i takes part in tree t < tpt[i] with window wpt[i] (w is
// then the largest window); the tensor forms only.
int knn_graph_impl(hf_forest* f, int32_t k, int32_t w, const int32_t* wpt, const int32_t* tpt, int T_use,
                   int32_t* out_idx, float* out_dist, cudaStream_t s) {
  cudaGetLastError();  // an earlier call's error was reported by that call
  const int64_t n = f->n;
  const bool budget = wpt != nullptr;
  // Plain mode: the window kernel keeps the top kp >= k per point by exact
  // float32 distance. Tensor mode: the Gram kernel keeps the top kp >= k + 1
  // (by default) by the BF16 expansion, then the re-rank orders them by exact
  // float32 distance. Either way the first k columns are the result.
  // form: 0 plain, 1 BF16 Gram, 2 FP8 Gram, 3 sketches (Hamming screen)
  const int form = f->mode == 3 ? 3 : (f->mode >= 1 && gram_supported(f->d, w, f->mode) ? f->mode : 0);
  const bool tensor = form == 1 || form == 2;
  const bool sketchf = form == 3;
  if (sketchf && !f->sketch) return HF_ESTATE;            // hf_set_sketch first
  if (sketchf && f->sketch_k2 > HF_MAX_K) return HF_ENOTIMPL;  // the band lists hold at most 64
  if (f->nseg > 1 && budget) return HF_ENOTIMPL;                 // segmented forests: uniform windows
  if (!tensor && w > HF_PLAIN_MAX_W) return HF_ENOTIMPL;  // widest window the plain band launches cover
  if (!tensor && budget) return HF_ENOTIMPL;              // per-point windows: tensor forms only
  f->timings[8] = (float)form;  // the form that runs
  const int slack = f->tensor_slack < 0 ? 1 : f->tensor_slack;
  const int kp = window_list_pitch(tensor ? k + slack : (sketchf ? (f->sketch_k2 > k ? f->sketch_k2 : k) : k));
  if (tensor && kp > 32) return HF_ENOTIMPL;  // tensor lists hold at most 32 entries
  uint32_t* li = nullptr;
  float* ldd = nullptr;
  // tensor forms: two trees' rows in their orders (the next tree's rows are
  // gathered on a side stream while the Gram band of this tree runs)
  void* xs[2] = {nullptr, nullptr};
  float2* ms[2] = {nullptr, nullptr};
  uint16_t* pw = nullptr;     // per-point windows of one tree
  int32_t* tile_w = nullptr;  // per-tile windows of one tree
  cudaError_t e = dalloc(&li, (size_t)n * kp, s);
  if (e == cudaSuccess) e = dalloc(&ldd, (size_t)n * kp, s);
  if (e == cudaSuccess && budget) e = dalloc(&pw, (size_t)n, s);
  if (e == cudaSuccess && budget) e = dalloc(&tile_w, (size_t)(n + 127) / 128, s);
  for (int b = 0; b < (T_use > 1 ? 2 : 1) && tensor; ++b) {
    if (e == cudaSuccess) e = dalloc_bytes(&xs[b], (size_t)n * gram_row_bytes(f->d, form), s);
    if (e == cudaSuccess) e = dalloc(&ms[b], (size_t)n, s);
  }
  if (e == cudaSuccess && tensor && !f->side) e = cudaStreamCreateWithFlags(&f->side, cudaStreamNonBlocking);
  if (e == cudaSuccess && tensor && f->xform != form) {
    dfree(f->xb, s);
    dfree(f->xmeta, s);
    f->xform = 0;
    e = dalloc_bytes(&f->xb, (size_t)n * gram_row_bytes(f->d, form), s);
    if (e == cudaSuccess) e = dalloc(&f->xmeta, (size_t)n, s);
    if (e == cudaSuccess) {
      launch_prepare_operands(f->x, n, f->d, form, f->xb, f->xmeta, s);
      f->xform = form;
    }
  }
  cudaEvent_t ev[5] = {};  // gathered[2], band done[2], side stream idle
  for (int i = 0; i < 5 && e == cudaSuccess && tensor; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    for (cudaEvent_t x : ev)
      if (x) cudaEventDestroy(x);
    dfree(li, s);
    dfree(ldd, s);
    for (int b = 0; b < 2; ++b) {
      dfree(xs[b], s);
      dfree(ms[b], s);
    }
    dfree(pw, s);
    dfree(tile_w, s);
    return map_cuda(e);
  }
  Timer tm(f, s);
  cudaEvent_t a0 = tm.mark();
  launch_list_init(li, ldd, n * kp, s);
  int rc = HF_OK;
  cudaStream_t side = f->side;
  auto gather = [&](int t) {  // tree t's rows into buffer t % 2, on the side stream
    const int b = T_use > 1 ? (t & 1) : 0;
    cudaEvent_t g0 = tm.mark_on(side);
    launch_gather_rows(f->xb, f->xmeta, form, n, f->d, f->sigma + (size_t)t * n, xs[b], ms[b], side);
    cudaEvent_t g1 = tm.mark_on(side);
    tm.span(9, g0, g1);
    cudaEventRecord(ev[b], side);
  };
  if (tensor) {
    cudaEventRecord(ev[4], s);  // operands prepared, lists initialised
    cudaStreamWaitEvent(side, ev[4], 0);
    gather(0);
  }
  for (int t = 0; t < T_use && rc == HF_OK; ++t) {
    if (tensor) {
      const int b = T_use > 1 ? (t & 1) : 0;
      const uint32_t* sig = f->sigma + (size_t)t * n;
      if (budget) launch_tree_budget(sig, n, t, wpt, tpt, pw, tile_w, s);
      cudaStreamWaitEvent(s, ev[b], 0);
      cudaEvent_t m0 = tm.mark();
      rc = launch_gram_window(form, n, f->d, sig, w, tile_w, pw, kp, li, ldd, f->err, xs[b], ms[b], s, f->seg,
                              f->seg_off);
      cudaEvent_t m1 = tm.mark();
      tm.span(10, m0, m1);
      cudaEventRecord(ev[2 + b], s);
      if (rc == HF_OK && t + 1 < T_use) {
        // buffer (t + 1) % 2 was read by tree t - 1's band
        if (t >= 1) cudaStreamWaitEvent(side, ev[2 + ((t + 1) & 1)], 0);
        gather(t + 1);
      }
    } else if (sketchf) {
      rc = launch_window_hamming(reinterpret_cast<const uint32_t*>(f->sketch), n, f->sketch_bits / 32,
                                 f->sigma + (size_t)t * n, w, kp, li, ldd, s, f->seg, f->seg_off);
    } else
      rc = launch_window_graph(f->x, n, f->d, f->sigma + (size_t)t * n, w, kp, li, ldd, s, f->seg, f->seg_off);
  }
  if (tensor) {
    // nothing of the side stream may outlive the buffers freed on s
    cudaEventRecord(ev[4], side);
    cudaStreamWaitEvent(s, ev[4], 0);
  }
  cudaEvent_t a1 = tm.mark();
  // every form's returned distances come from the re-rank's float32 exact
  // differences with the butterfly sum (relative error below 1.1e-6 at
  // d = 384); the plain window kernel's sequential sums only select
  if (rc == HF_OK)
    rc = launch_rerank(f->x, n, f->d, f->sigma, kp, sketchf ? (f->sketch_k2 > k ? f->sketch_k2 : k) : kp, li, ldd, s);
  cudaEvent_t a2 = tm.mark();
  tm.span(4, a0, a1);
  tm.span(7, a1, a2);
  // First k of kp columns into the caller's buffers. A host buffer gets the
  // columns packed on the device first and one contiguous copy (a strided
  // copy of n rows of 4k bytes straight to the host moves at a fraction of
  // the link's rate).
  auto deliver = [&](void* out, const void* lists) -> int {
    const size_t row = (size_t)k * 4, bytes = row * (size_t)n;
    if (classify(out) == 1)
      return map_cuda(cudaMemcpy2DAsync(out, row, lists, (size_t)kp * 4, row, (size_t)n, cudaMemcpyDefault, s));
    void* packed = nullptr;
    int r = map_cuda(dalloc_bytes(&packed, bytes, s));
    if (r == HF_OK)
      r = map_cuda(cudaMemcpy2DAsync(packed, row, lists, (size_t)kp * 4, row, (size_t)n, cudaMemcpyDefault, s));
    if (r == HF_OK) r = map_cuda(cudaMemcpyAsync(out, packed, bytes, cudaMemcpyDefault, s));
    dfree(packed, s);
    return r;
  };
  if (rc == HF_OK) rc = deliver(out_idx, li);
  if (rc == HF_OK) rc = deliver(out_dist, ldd);
  int rc2 = finish(f, s);
  if (rc == HF_OK) rc = rc2;
  f->timings[9] = 0.f;
  f->timings[10] = 0.f;
  if (rc == HF_OK) tm.collect({4, 7, 9, 10});
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  dfree(li, s);
  dfree(ldd, s);
  for (int b = 0; b < 2; ++b) {
    dfree(xs[b], s);
    dfree(ms[b], s);
  }
  dfree(pw, s);
  dfree(tile_w, s);
  return rc;
}

}  // namespace

extern "C" {

int hf_knn_graph(hf_forest* f, int32_t k, int32_t w, int32_t* out_idx, float* out_dist, void* stream) {
  if (!f || !out_idx || !out_dist || k < 1 || k > HF_MAX_K || w < 1) return HF_EINVAL;
  return knn_graph_impl(f, k, w, nullptr, nullptr, f->T, out_idx, out_dist, static_cast<cudaStream_t>(stream));
}

int hf_knn_graph_budget(hf_forest* f, int32_t k, const int32_t* w_pt, const int32_t* T_pt, int32_t w_max,
                        int32_t T_max, int32_t* out_idx, float* out_dist, void* stream) {
  if (!f || !w_pt || !T_pt || !out_idx || !out_dist || k < 1 || k > HF_MAX_K || w_max < 1 || w_max > 65535 ||
      T_max < 1 || T_max > f->T)
    return HF_EINVAL;
  if (classify(w_pt) != 1 || classify(T_pt) != 1) return HF_EINVAL;
  return knn_graph_impl(f, k, w_max, w_pt, T_pt, T_max, out_idx, out_dist, static_cast<cudaStream_t>(stream));
}

// ---- enqueue-only graph, CUDA graphs, exact rows, autotuner ---------------

int hf_graph_plan(hf_forest* f, int32_t k, int32_t w, int32_t threads, void* stream) {
  if (!f || k < 1 || k > HF_MAX_K || w < 1) return HF_EINVAL;
  if (threads != 0 && threads != 256 && threads != 512) return HF_EINVAL;
  if (f->mode == 3) return HF_ENOTIMPL;
  const int form = f->mode;  // 0 plain, 1 BF16 Gram, 2 FP8 Gram
  if (form == 0 && w > HF_PLAIN_MAX_W) return HF_ENOTIMPL;
  if (form != 0 && !gram_supported(f->d, w, form)) return HF_ENOTIMPL;  // no silent change of form here
  const int slack = f->tensor_slack < 0 ? 1 : f->tensor_slack;
  const int kp = window_list_pitch(form ? k + slack : k);
  if (form && kp > 32) return HF_ENOTIMPL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  const int64_t n = f->n;
  cudaError_t e = cudaSuccess;
  if (kp != f->plan_kp || !f->plan_li) {
    dfree(f->plan_li, s);
    dfree(f->plan_ld, s);
    e = dalloc(&f->plan_li, (size_t)n * kp, s);
    if (e == cudaSuccess) e = dalloc(&f->plan_ld, (size_t)n * kp, s);
  }
  if (e == cudaSuccess && form && (form != f->plan_form || !f->plan_xs)) {
    dfree(f->plan_xs, s);
    dfree(f->plan_ms, s);
    e = dalloc_bytes(&f->plan_xs, (size_t)n * gram_row_bytes(f->d, form), s);
    if (e == cudaSuccess) e = dalloc(&f->plan_ms, (size_t)n, s);
  }
  if (e == cudaSuccess && form && f->xform != form) {
    dfree(f->xb, s);
    dfree(f->xmeta, s);
    f->xform = 0;
    e = dalloc_bytes(&f->xb, (size_t)n * gram_row_bytes(f->d, form), s);
    if (e == cudaSuccess) e = dalloc(&f->xmeta, (size_t)n, s);
    if (e == cudaSuccess) {
      launch_prepare_operands(f->x, n, f->d, form, f->xb, f->xmeta, s);
      f->xform = form;
    }
  }
  if (e != cudaSuccess) {
    dfree(f->plan_li, s);
    dfree(f->plan_ld, s);
    dfree(f->plan_xs, s);
    dfree(f->plan_ms, s);
    f->plan_kp = 0;
    return map_cuda(e);
  }
  f->plan_k = k;
  f->plan_w = w;
  f->plan_kp = kp;
  f->plan_nt = threads;
  f->plan_form = form;
  return finish(f, s);
}

// Enqueues list init, per tree the window launches (plain) or the row gather
// and the Gram band launch (tensor forms), the re-rank (tensor forms) and
// the copy of the first k columns; no allocation, no synchronisation.
static int enqueue_graph(hf_forest* f, int32_t* out_idx, float* out_dist, cudaStream_t s) {
  const int64_t n = f->n;
  const int kp = f->plan_kp, k = f->plan_k, form = f->plan_form;
  launch_list_init(f->plan_li, f->plan_ld, n * kp, s);
  int rc = HF_OK;
  for (int t = 0; t < f->T && rc == HF_OK; ++t) {
    const uint32_t* sig = f->sigma + (size_t)t * n;
    if (form) {
      launch_gather_rows(f->xb, f->xmeta, form, n, f->d, sig, f->plan_xs, f->plan_ms, s);
      rc = launch_gram_window(form, n, f->d, sig, f->plan_w, nullptr, nullptr, kp, f->plan_li, f->plan_ld, f->err,
                              f->plan_xs, f->plan_ms, s, f->seg, f->seg_off);
    } else {
      rc = launch_window_graph(f->x, n, f->d, sig, f->plan_w, kp, f->plan_li, f->plan_ld, s, f->seg, f->seg_off,
                               f->plan_nt);
    }
  }
  if (rc == HF_OK) rc = launch_rerank(f->x, n, f->d, f->sigma, kp, kp, f->plan_li, f->plan_ld, s);
  if (rc != HF_OK) return rc;
  if (out_idx &&
      cudaMemcpy2DAsync(out_idx, (size_t)k * 4, f->plan_li, (size_t)kp * 4, (size_t)k * 4, (size_t)n,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return HF_ECUDA;
  if (out_dist &&
      cudaMemcpy2DAsync(out_dist, (size_t)k * 4, f->plan_ld, (size_t)kp * 4, (size_t)k * 4, (size_t)n,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return HF_ECUDA;
  return HF_OK;
}

int hf_knn_graph_enqueue(hf_forest* f, int32_t* out_idx, float* out_dist, void* stream) {
  if (!f || !out_idx || !out_dist) return HF_EINVAL;
  if (!f->plan_li) return HF_ESTATE;
  if (classify(out_idx) != 1 || classify(out_dist) != 1) return HF_EINVAL;
  return enqueue_graph(f, out_idx, out_dist, static_cast<cudaStream_t>(stream));
}

int hf_status(hf_forest* f, void* stream) {
  if (!f) return HF_EINVAL;
  return finish(f, static_cast<cudaStream_t>(stream));
}

int hf_capture_begin(void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!s) return HF_EINVAL;  // the legacy default stream cannot be captured
  return map_cuda(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
}

int hf_capture_end(void* stream, void** exec) {
  if (!exec) return HF_EINVAL;
  *exec = nullptr;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(static_cast<cudaStream_t>(stream), &g);
  if (e != cudaSuccess) return map_cuda(e);
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return map_cuda(e);
  *exec = x;
  return HF_OK;
}

int hf_graph_launch(void* exec, void* stream) {
  if (!exec) return HF_EINVAL;
  return map_cuda(cudaGraphLaunch(static_cast<cudaGraphExec_t>(exec), static_cast<cudaStream_t>(stream)));
}

int hf_graph_destroy(void* exec) {
  if (!exec) return HF_OK;
  return map_cuda(cudaGraphExecDestroy(static_cast<cudaGraphExec_t>(exec)));
}

int hf_exact_knn_rows(hf_forest* f, const int64_t* rows, int32_t nrows, int32_t k, int32_t* out_idx,
                      float* out_dist, void* stream) {
  if (!f || !rows || !out_idx || !out_dist || nrows < 1 || k < 1 || k > HF_MAX_K) return HF_EINVAL;
  for (int32_t j = 0; j < nrows; ++j)
    if (rows[j] < 0 || rows[j] >= f->n) return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  int64_t* rd = nullptr;
  uint32_t* oi = nullptr;
  float* od = nullptr;
  cudaError_t e = dalloc(&rd, (size_t)nrows, s);
  if (e == cudaSuccess) e = dalloc(&oi, (size_t)nrows * k, s);
  if (e == cudaSuccess) e = dalloc(&od, (size_t)nrows * k, s);
  int rc = map_cuda(e);
  if (rc == HF_OK) rc = map_cuda(cudaMemcpyAsync(rd, rows, (size_t)nrows * 8, cudaMemcpyHostToDevice, s));
  if (rc == HF_OK) rc = launch_exact_rows(f, rd, nrows, k, oi, od, s);
  if (rc == HF_OK) rc = map_cuda(cudaMemcpyAsync(out_idx, oi, (size_t)nrows * k * 4, cudaMemcpyDefault, s));
  if (rc == HF_OK) rc = map_cuda(cudaMemcpyAsync(out_dist, od, (size_t)nrows * k * 4, cudaMemcpyDefault, s));
  const int rc2 = finish(f, s);
  dfree(rd, s);
  dfree(oi, s);
  dfree(od, s);
  return rc != HF_OK ? rc : rc2;
}

int hf_autotune(hf_forest* f, int32_t k, double target_recall, int32_t sample, int32_t w_max, int32_t forms,
                int32_t* out_form, int32_t* out_w, int32_t* out_threads, double* out_recall, float* out_ms,
                void* stream) {
  if (!f || k < 1 || k > HF_MAX_K || sample < 1 || w_max < 1 || !(target_recall >= 0.0 && target_recall <= 1.0) ||
      (forms & 7) == 0 || (forms & ~7))
    return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ladder_all[] = {2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 704, 1024, 1536, 2048};
  // sample rows spread evenly over the matrix (so over the sets by size)
  const int m = (int)(sample < f->n ? sample : f->n);
  std::vector<int64_t> rows(m);
  for (int j = 0; j < m; ++j) rows[j] = (int64_t)(((__int128)j * f->n) / m);
  std::vector<int32_t> ex((size_t)m * k);
  std::vector<float> exd((size_t)m * k);
  int rc = hf_exact_knn_rows(f, rows.data(), m, k, ex.data(), exd.data(), stream);
  if (rc != HF_OK) return rc;
  int64_t* rd = nullptr;
  uint32_t* got_d = nullptr;
  cudaError_t e = dalloc(&rd, (size_t)m, s);
  if (e == cudaSuccess) e = dalloc(&got_d, (size_t)m * k, s);
  rc = map_cuda(e);
  if (rc == HF_OK) rc = map_cuda(cudaMemcpyAsync(rd, rows.data(), (size_t)m * 8, cudaMemcpyHostToDevice, s));
  std::vector<uint32_t> got((size_t)m * k);
  auto recall_at = [&](int w, double* rec) -> int {
    int r = hf_graph_plan(f, k, w, 0, stream);
    if (r == HF_OK) r = enqueue_graph(f, nullptr, nullptr, s);
    if (r == HF_OK) launch_gather_list_rows(f->plan_li, f->plan_kp, rd, m, k, got_d, s);
    if (r == HF_OK) r = map_cuda(cudaMemcpyAsync(got.data(), got_d, got.size() * 4, cudaMemcpyDeviceToHost, s));
    const int r2 = finish(f, s);
    if (r != HF_OK) return r;
    if (r2 != HF_OK) return r2;
    int64_t hit = 0, tot = 0;
    for (int j = 0; j < m; ++j) {
      const int32_t* ej = ex.data() + (size_t)j * k;
      const uint32_t* gj = got.data() + (size_t)j * k;
      for (int a = 0; a < k; ++a) {
        if (ej[a] < 0) continue;
        ++tot;
        for (int b = 0; b < k; ++b)
          if (gj[b] == (uint32_t)ej[a]) {
            ++hit;
            break;
          }
      }
    }
    *rec = tot ? (double)hit / (double)tot : 1.0;
    return HF_OK;
  };
  // CUDA-event time of the planned graph (mean of 3 after a warm-up)
  auto time_plan = [&](float* ms_out) -> int {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int r = enqueue_graph(f, nullptr, nullptr, s);
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3 && r == HF_OK; ++rep) r = enqueue_graph(f, nullptr, nullptr, s);
    cudaEventRecord(e1, s);
    const int r2 = finish(f, s);
    float ms = 0.f;
    if (r == HF_OK && r2 == HF_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) r = HF_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = ms / 3.f;
    return r != HF_OK ? r : r2;
  };
  const int mode0 = f->mode, slack0 = f->tensor_slack;
  int best_form = -1, best_w = 0, best_nt = 0, best_slack = -1;
  double best_rec = -1.0;
  float best_ms = 0.f;
  bool best_hit = false;
  // variants: the plain form; each Gram form with the shortest list that
  // holds k + 1 candidates and with 32 slots (more candidates for the re-rank)
  struct Variant {
    int form, slack;
  };
  std::vector<Variant> variants;
  if (forms & 1) variants.push_back({0, -1});
  for (int form = 1; form <= 2; ++form) {
    if (!(forms & (1 << form))) continue;
    if (k + 1 <= 16) variants.push_back({form, 16 - k});
    if (k + 1 <= 32) variants.push_back({form, 32 - k});
  }
  for (const Variant& var : variants) {
    if (rc != HF_OK) break;
    const int form = var.form;
    f->mode = form;
    f->tensor_slack = var.slack;
    std::vector<int> ladder;
    for (int w : ladder_all)
      if (w <= w_max && (form == 0 ? w <= HF_PLAIN_MAX_W : gram_supported(f->d, w, form) != 0)) ladder.push_back(w);
    if (ladder.empty()) continue;
    // smallest rung reaching the target (recall grows with w)
    int lo = 0, hi = (int)ladder.size() - 1, pick = hi;
    double pick_rec = -1.0;
    while (rc == HF_OK && lo <= hi) {
      const int mid = (lo + hi) / 2;
      double rec = 0.0;
      rc = recall_at(ladder[mid], &rec);
      if (rc != HF_OK) break;
      if (rec >= target_recall) {
        pick = mid;
        pick_rec = rec;
        hi = mid - 1;
      } else {
        lo = mid + 1;
      }
    }
    if (rc != HF_OK) break;
    const bool hit = pick_rec >= 0.0;
    if (!hit) rc = recall_at(ladder[pick], &pick_rec);
    if (rc != HF_OK) break;
    // block size (plain form: 256 or 512 threads; the Gram kernel is persistent)
    const int nts[2] = {256, 512};
    for (int v = 0; v < (form == 0 ? 2 : 1) && rc == HF_OK; ++v) {
      const int nt = form == 0 ? nts[v] : 0;
      if (hf_graph_plan(f, k, ladder[pick], nt, stream) != HF_OK) continue;
      float ms = 0.f;
      if (time_plan(&ms) != HF_OK) {
        cudaGetLastError();  // a block size whose blocks cannot hold 32 positions is skipped
        continue;
      }
      // a form that reaches the target beats one that does not; then time
      const bool better = best_form < 0 || (hit && !best_hit) ||
                          (hit == best_hit && (hit ? ms < best_ms : pick_rec > best_rec));
      if (better) {
        best_form = form;
        best_slack = var.slack;
        best_w = ladder[pick];
        best_nt = nt;
        best_rec = pick_rec;
        best_ms = ms;
        best_hit = hit;
      }
    }
  }
  if (rc == HF_OK && best_form < 0) rc = HF_ENOTIMPL;
  if (rc == HF_OK) {
    f->mode = best_form;
    f->tensor_slack = best_slack;
    rc = hf_graph_plan(f, k, best_w, best_nt, stream);
  } else {
    f->mode = mode0;
    f->tensor_slack = slack0;
  }
  dfree(rd, s);
  dfree(got_d, s);
  if (rc == HF_OK) {
    if (out_form) *out_form = best_form | (best_form ? (f->plan_kp << 8) : 0);
    if (out_w) *out_w = best_w;
    if (out_threads) *out_threads = best_nt;
    if (out_recall) *out_recall = best_rec;
    if (out_ms) *out_ms = best_ms;
  }
  return rc;
}

int hf_set_sketch(hf_forest* f, const float* R, int32_t bits, void* stream) {
  if (!f || !R || bits < 64 || bits > 1024 || bits % 64) return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  const int d = f->d, dp = (d + 63) / 64 * 64;
  const int64_t n = f->n;
  float* rd = nullptr;
  void *rb = nullptr, *xbt = nullptr;
  uint64_t* sk = nullptr;
  cudaError_t e = cudaSuccess;
  const bool dev_r = classify(R) == 1;
  if (!dev_r) e = dalloc(&rd, (size_t)bits * d, s);
  if (e == cudaSuccess) e = dalloc_bytes(&rb, (size_t)bits * dp * 2, s);
  if (e == cudaSuccess) e = dalloc_bytes(&xbt, (size_t)n * dp * 2, s);
  if (e == cudaSuccess) e = dalloc(&sk, (size_t)n * (bits / 64), s);
  int rc = map_cuda(e);
  if (rc == HF_OK) {
    if (!dev_r) cudaMemcpyAsync(rd, R, (size_t)bits * d * 4, cudaMemcpyHostToDevice, s);
    launch_f32_to_bf16(dev_r ? R : rd, bits, d, dp, rb, s);
    launch_f32_to_bf16(f->x, n, d, dp, xbt, s);
    rc = launch_sketch(xbt, n, dp, rb, bits, sk, f->err, s);
  }
  const int rc2 = finish(f, s);
  if (rc == HF_OK) rc = rc2;
  dfree(rd, s);
  dfree(xbt, s);
  if (rc == HF_OK) {
    dfree(f->sketch, s);
    dfree(f->sketch_r, s);
    f->sketch = sk;
    f->sketch_r = rb;
    f->sketch_bits = bits;
  } else {
    dfree(sk, s);
    dfree(rb, s);
  }
  return rc;
}

int hf_debug_sketch(hf_forest* f, uint64_t* out, void* stream) {
  if (!f || !out) return HF_EINVAL;
  if (!f->sketch) return HF_ESTATE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  const int rc = map_cuda(cudaMemcpyAsync(out, f->sketch, (size_t)f->n * (f->sketch_bits / 64) * 8,
                                          cudaMemcpyDefault, s));
  const int rc2 = finish(f, s);
  return rc != HF_OK ? rc : rc2;
}

int hf_budget_labels(hf_forest* f, const int32_t* knn, int32_t k, const int32_t* t_grid, int32_t nt,
                     const int32_t* w_grid, int32_t nw, int32_t min_hits, float* out_targets, int32_t* out_cell,
                     void* stream) {
  if (!f || !knn || !t_grid || !w_grid || !out_targets || !out_cell || k < 1 || k > HF_MAX_K || nt < 1 || nw < 1 ||
      nt > 16 || nw > 16 || min_hits < 0 || min_hits > k)
    return HF_EINVAL;
  if (f->nseg > 1) return HF_ENOTIMPL;
  if (classify(knn) != 1 || classify(out_targets) != 1 || classify(out_cell) != 1) return HF_EINVAL;
  int tmax = 0;
  for (int i = 0; i < nt; ++i) {
    if (t_grid[i] < 1 || t_grid[i] > f->T || (i && t_grid[i] <= t_grid[i - 1])) return HF_EINVAL;
    tmax = t_grid[i];
  }
  for (int i = 0; i < nw; ++i)
    if (w_grid[i] < 1 || (i && w_grid[i] <= w_grid[i - 1])) return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();
  int32_t *pos = nullptr, *tg = nullptr, *wg = nullptr;
  cudaError_t e = dalloc(&pos, (size_t)tmax * f->n, s);
  if (e == cudaSuccess) e = dalloc(&tg, (size_t)nt, s);
  if (e == cudaSuccess) e = dalloc(&wg, (size_t)nw, s);
  int rc = map_cuda(e);
  if (rc == HF_OK) {
    cudaMemcpyAsync(tg, t_grid, (size_t)nt * 4, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(wg, w_grid, (size_t)nw * 4, cudaMemcpyHostToDevice, s);
    rc = launch_budget_labels(f->sigma, tmax, f->n, knn, k, tg, nt, wg, nw, min_hits, out_targets, out_cell, pos, s);
  }
  const int rc2 = finish(f, s);
  dfree(pos, s);
  dfree(tg, s);
  dfree(wg, s);
  return rc != HF_OK ? rc : rc2;
}

// Sketch form of the search (Algorithm 1 with both filters): positions of
// every tree, query sketches, then one warp per query for the Hamming stage,
// the master-order expansion and the final float32 stage. The master-ordered
// copy of the points is built on the first such call and kept.
static int sketch_search(hf_forest* f, const float* q, const uint8_t* qc, int64_t nq, int k, int w, uint32_t* li,
                         float* ldd, cudaStream_t s) {
  if (!f->sketch || !f->sketch_r) return HF_ESTATE;
  if (!f->sigma) return HF_ESTATE;
  const int d = f->d, dp = (d + 63) / 64 * 64, words = f->sketch_bits / 64;
  cudaError_t e = cudaSuccess;
  if (!f->xm) {
    e = dalloc(&f->xm, (size_t)f->n * d, s);
    if (e == cudaSuccess) e = dalloc(&f->posm, (size_t)f->n, s);
    if (e != cudaSuccess) {
      dfree(f->xm, s);
      dfree(f->posm, s);
      f->xm = nullptr;
      f->posm = nullptr;
      return map_cuda(e);
    }
    launch_master_layout(f->x, f->n, d, f->sigma, f->xm, f->posm, s);
  }
  int64_t* pos = nullptr;
  void* qb = nullptr;
  uint64_t* qsk = nullptr;
  e = dalloc(&pos, (size_t)f->T * nq, s);
  if (e == cudaSuccess) e = dalloc_bytes(&qb, (size_t)nq * dp * 2, s);
  if (e == cudaSuccess) e = dalloc(&qsk, (size_t)nq * words, s);
  int rc = map_cuda(e);
  if (rc == HF_OK) rc = launch_search(f, q, qc, nq, k, w, nullptr, nullptr, pos, -2, s);
  if (rc == HF_OK) {
    launch_f32_to_bf16(q, nq, d, dp, qb, s);
    rc = launch_sketch(qb, nq, dp, f->sketch_r, f->sketch_bits, qsk, f->err, s);
  }
  if (rc == HF_OK) rc = launch_sketch_search(f, q, nq, pos, qsk, k, w, f->sketch_k2, f->expand_h, li, ldd, s);
  dfree(pos, s);
  dfree(qb, s);
  dfree(qsk, s);
  return rc;
}

int hf_search(hf_forest* f, const float* queries, int64_t nq, int32_t k, int32_t w, int32_t* out_idx,
              float* out_dist, void* stream) {
  if (!f || nq < 0 || k < 1 || k > HF_MAX_K || w < 1) return HF_EINVAL;
  if (f->nseg > 1) return HF_ENOTIMPL;
  if (nq == 0) return HF_OK;
  if (!queries || !out_idx || !out_dist || nq > HF_MAX_N) return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();  // an earlier call's error was reported by that call
  const int d = f->d;
  const size_t cnt = (size_t)nq * k;
  const bool dev_q = classify(queries) == 1;
  const bool dev_i = classify(out_idx) == 1, dev_d = classify(out_dist) == 1;
  float* qd = nullptr;
  uint8_t* qc = nullptr;
  uint32_t* li = dev_i ? reinterpret_cast<uint32_t*>(out_idx) : nullptr;
  float* ldd = dev_d ? out_dist : nullptr;
  cudaError_t e = cudaSuccess;
  if (!dev_q) e = dalloc(&qd, (size_t)nq * d, s);
  if (e == cudaSuccess) e = dalloc(&qc, (size_t)nq * d, s);
  if (e == cudaSuccess && !li) e = dalloc(&li, cnt, s);
  if (e == cudaSuccess && !ldd) e = dalloc(&ldd, cnt, s);
  int rc = map_cuda(e);
  Timer tm(f, s);
  if (rc == HF_OK) {
    if (!dev_q) rc = map_cuda(cudaMemcpyAsync(qd, queries, (size_t)nq * d * 4, cudaMemcpyHostToDevice, s));
    const float* qsrc = dev_q ? queries : qd;
    cudaEvent_t a0 = tm.mark();
    launch_quantize_codes(qsrc, nq, d, f->lo, f->scale, f->bits, qc, f->err, s);
    if (rc == HF_OK && f->mode == 3)
      rc = sketch_search(f, qsrc, qc, nq, k, w, li, ldd, s);
    else if (rc == HF_OK)
      rc = launch_search(f, qsrc, qc, nq, k, w, li, ldd, nullptr, -1, s);
    cudaEvent_t a1 = tm.mark();
    tm.span(5, a0, a1);
    if (rc == HF_OK && !dev_i) rc = map_cuda(cudaMemcpyAsync(out_idx, li, cnt * 4, cudaMemcpyDeviceToHost, s));
    if (rc == HF_OK && !dev_d) rc = map_cuda(cudaMemcpyAsync(out_dist, ldd, cnt * 4, cudaMemcpyDeviceToHost, s));
    int rc2 = finish(f, s);
    if (rc == HF_OK) rc = rc2;
    if (rc == HF_OK) tm.collect({5});
  }
  dfree(qd, s);
  dfree(qc, s);
  if (!dev_i) dfree(li, s);
  if (!dev_d) dfree(ldd, s);
  return rc;
}

// ---- inspection exports ----------------------------------------------------

int hf_debug_codes(hf_forest* f, uint8_t* out_codes, void* stream) {
  if (!f || !out_codes) return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();  // an earlier call's error was reported by that call
  const size_t cnt = (size_t)f->n * f->d;
  const bool dev = classify(out_codes) == 1;
  uint8_t* c = dev ? out_codes : nullptr;
  if (!dev && dalloc(&c, cnt, s) != cudaSuccess) return HF_ENOMEM;
  launch_planes_to_codes(f->planes, f->n, f->d, f->bits, c, s);
  int rc = HF_OK;
  if (!dev) rc = map_cuda(cudaMemcpyAsync(out_codes, c, cnt, cudaMemcpyDeviceToHost, s));
  int rc2 = finish(f, s);
  if (!dev) dfree(c, s);
  return rc ? rc : rc2;
}

int hf_debug_keys(hf_forest* f, int32_t tree, uint64_t* out_keys, void* stream) {
  if (!f || !out_keys || tree < 0 || tree >= f->T) return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();  // an earlier call's error was reported by that call
  const size_t cnt = (size_t)f->n * f->W;
  const bool dev = classify(out_keys) == 1;
  uint64_t* kk = dev ? out_keys : nullptr;
  if (!dev && dalloc(&kk, cnt, s) != cudaSuccess) return HF_ENOMEM;
  launch_full_keys_planes(f->planes, f->n, f->d, f->bits, f->W, f->pi + (size_t)tree * f->d,
                          f->rbits + (size_t)tree * f->W32, kk, s);
  int rc = HF_OK;
  if (!dev) rc = map_cuda(cudaMemcpyAsync(out_keys, kk, cnt * 8, cudaMemcpyDeviceToHost, s));
  int rc2 = finish(f, s);
  if (!dev) dfree(kk, s);
  return rc ? rc : rc2;
}

int hf_debug_prefix(hf_forest* f, int32_t tree, uint64_t* out_words, void* stream) {
  if (!f || !out_words || tree < 0 || tree >= f->T) return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();  // an earlier call's error was reported by that call
  const size_t cnt = (size_t)f->n * f->K2;
  const bool dev = classify(out_words) == 1;
  uint64_t* kk = dev ? out_words : nullptr;
  if (!dev && dalloc(&kk, cnt, s) != cudaSuccess) return HF_ENOMEM;
  // the build freed its bit-sliced plane 0; it is made again so that the
  // words come from the same kernel as in the build
  uint32_t* p0t = nullptr;
  if (prefix_top_path(f->d, f->K2, f->L)) {
    if (dalloc(&p0t, (size_t)((f->n + 31) / 32) * f->d, s) != cudaSuccess) {
      if (!dev) dfree(kk, s);
      return HF_ENOMEM;
    }
    launch_plane0_slice(f->planes, f->n, f->d, p0t, s);
  }
  launch_prefix_keys(f->planes, p0t, f->n, f->d, f->bits, f->K2, f->L, f->pi + (size_t)tree * f->d,
                     f->rbits + (size_t)tree * f->W32, kk, s);
  int rc = HF_OK;
  if (!dev) rc = map_cuda(cudaMemcpyAsync(out_words, kk, cnt * 8, cudaMemcpyDeviceToHost, s));
  int rc2 = finish(f, s);
  dfree(p0t, s);
  if (!dev) dfree(kk, s);
  return rc ? rc : rc2;
}

int hf_debug_order(hf_forest* f, int32_t tree, uint32_t* out_sigma, void* stream) {
  if (!f || !out_sigma || tree < 0 || tree >= f->T) return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();  // an earlier call's error was reported by that call
  int rc = map_cuda(cudaMemcpyAsync(out_sigma, f->sigma + (size_t)tree * f->n, (size_t)f->n * 4,
                                    cudaMemcpyDefault, s));
  int rc2 = finish(f, s);
  return rc ? rc : rc2;
}

int hf_debug_locate(hf_forest* f, int32_t tree, const float* queries, int64_t nq, int64_t* out_pos,
                    void* stream) {
  if (!f || tree < 0 || tree >= f->T || nq < 0) return HF_EINVAL;
  if (f->nseg > 1) return HF_ENOTIMPL;
  if (nq == 0) return HF_OK;
  if (!queries || !out_pos) return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();  // an earlier call's error was reported by that call
  const int d = f->d;
  const bool dev_q = classify(queries) == 1, dev_o = classify(out_pos) == 1;
  float* qd = nullptr;
  uint8_t* qc = nullptr;
  int64_t* po = dev_o ? out_pos : nullptr;
  cudaError_t e = cudaSuccess;
  if (!dev_q) e = dalloc(&qd, (size_t)nq * d, s);
  if (e == cudaSuccess) e = dalloc(&qc, (size_t)nq * d, s);
  if (e == cudaSuccess && !po) e = dalloc(&po, (size_t)nq, s);
  int rc = map_cuda(e);
  if (rc == HF_OK) {
    if (!dev_q) cudaMemcpyAsync(qd, queries, (size_t)nq * d * 4, cudaMemcpyHostToDevice, s);
    const float* qsrc = dev_q ? queries : qd;
    launch_quantize_codes(qsrc, nq, d, f->lo, f->scale, f->bits, qc, f->err, s);
    rc = launch_search(f, qsrc, qc, nq, 1, 1, nullptr, nullptr, po, tree, s);
    if (rc == HF_OK && !dev_o) rc = map_cuda(cudaMemcpyAsync(out_pos, po, (size_t)nq * 8, cudaMemcpyDeviceToHost, s));
    int rc2 = finish(f, s);
    if (rc == HF_OK) rc = rc2;
  }
  dfree(qd, s);
  dfree(qc, s);
  if (!dev_o) dfree(po, s);
  return rc;
}

int hf_debug_keys_from_codes(const uint8_t* codes, int64_t n, int32_t d, int32_t bits, uint64_t* out_keys,
                             void* stream) {
  if (!codes || !out_keys || n < 1 || n > HF_MAX_N || d < 1 || d > HF_MAX_D || bits < 1 || bits > HF_MAX_BITS)
    return HF_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaGetLastError();  // an earlier call's error was reported by that call
  const int W = (int)(((int64_t)d * bits + 63) / 64);
  const bool dev_c = classify(codes) == 1, dev_o = classify(out_keys) == 1;
  uint8_t* cd = nullptr;
  uint64_t* kk = dev_o ? out_keys : nullptr;
  cudaError_t e = cudaSuccess;
  if (!dev_c) e = dalloc(&cd, (size_t)n * d, s);
  if (e == cudaSuccess && !kk) e = dalloc(&kk, (size_t)n * W, s);
  int rc = map_cuda(e);
  if (rc == HF_OK) {
    if (!dev_c) cudaMemcpyAsync(cd, codes, (size_t)n * d, cudaMemcpyHostToDevice, s);
    launch_full_keys_codes(dev_c ? codes : cd, n, d, bits, W, nullptr, nullptr, kk, s);
    if (!dev_o) cudaMemcpyAsync(out_keys, kk, (size_t)n * W * 8, cudaMemcpyDeviceToHost, s);
    cudaError_t se = cudaStreamSynchronize(s);
    if (se == cudaSuccess) se = cudaGetLastError();
    rc = map_cuda(se);
  }
  dfree(cd, s);
  if (!dev_o) dfree(kk, s);
  return rc;
}

}  // extern "C"
