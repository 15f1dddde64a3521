// Plain CPU oracle of the Hilbert forest path, in C++ -- TEST INFRASTRUCTURE
// ONLY.
//
// A second, independent statement of what oracle/hilbert_forest.py computes,
// written as scalar loops over points, coordinates and trees. Only the test
// suite (through oracle/c_oracle.py) and the bench's CPU arms load it; the
// CUDA library never does, and the two share no code, header or table.
//
// What it follows (arXiv 2508.21682, "Hilbert Forest in the SISAP 2025
// Indexing Challenge"):
//  * Section 2: points are ordered along a Hilbert curve; that order is a
//    total order in which binary search places any point; a forest is several
//    such orders.
//  * Algorithm 2 (Section 4, the kNN graph): for every sort, shuffle the
//    coordinate axes, order all points along the curve, and give each point
//    the points a few places before and after it as candidates; keep the k
//    candidates nearest by vector distance.
//  * Algorithm 1 (Section 3, search): in every tree, place the query in the
//    order and take the points around that place as candidates; keep the k
//    nearest.
// Where the paper is silent the conventions are the ones the numpy oracle
// states (curve: Skilling 2004, transposed index; quantization: per-axis
// min/max, b bits, separately rounded float32 steps; axis order: splitmix64
// and a Fisher-Yates shuffle plus one reflection bit per axis; equal keys by
// point index; window of w positions on each side; candidate sets are sets
// without the point itself; squared Euclidean distance in double, ties by
// index; missing slots (-1, +inf)).
//
// Built with -ffp-contract=off: no multiply-add is fused, so every float32
// step of the quantization is the separately rounded operation the
// convention names, and every distance is the plain left-to-right sum.
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

// splitmix64 (Steele, Lea and Flood, OOPSLA 2014): add the golden-ratio
// increment to the state, then two xor-shift-multiply rounds and a final
// xor-shift of the new state.
struct SplitMix64 {
  uint64_t state;
  uint64_t next() {
    state += kGamma;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

// Tree t's axis order and reflections: the generator starts at
// seed + (t + 1) * gamma; pi starts as the identity and, for j = d-1 down to
// 1, entries j and next() mod (j + 1) are exchanged; then each axis j draws
// its reflection bit as the top bit of next().
void tree_params(uint64_t seed, int tree, int d, int64_t* pi, uint8_t* r) {
  SplitMix64 g{seed + (uint64_t)(tree + 1) * kGamma};
  for (int j = 0; j < d; ++j) pi[j] = j;
  for (int j = d - 1; j >= 1; --j) {
    const uint64_t m = g.next() % (uint64_t)(j + 1);
    std::swap(pi[j], pi[m]);
  }
  for (int j = 0; j < d; ++j) r[j] = (uint8_t)(g.next() >> 63);
}

// Per-axis range: lo = min, hi = max over the points; width = hi - lo in
// float32; scale = 2^b / width evaluated in double and rounded to float32
// once, 0 for a flat axis. Returns false on a non-finite value.
bool axis_range(const float* x, int64_t n, int d, int bits, float* lo, float* scale) {
  for (int j = 0; j < d; ++j) {
    float mn = x[j], mx = x[j];
    for (int64_t i = 0; i < n; ++i) {
      const float v = x[(size_t)i * d + j];
      if (!std::isfinite(v)) return false;
      if (v < mn) mn = v;
      if (v > mx) mx = v;
    }
    const float width = mx - mn;
    lo[j] = mn;
    scale[j] = width > 0.0f ? (float)((double)(1u << bits) / (double)width) : 0.0f;
  }
  return true;
}

// code = clamp(floor(fl32(fl32(x - lo) * scale)), 0, 2^b - 1).
bool quantize(const float* x, int64_t n, int d, int bits, const float* lo, const float* scale, uint16_t* codes) {
  const double top = (double)((1u << bits) - 1u);
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < d; ++j) {
      const float v = x[(size_t)i * d + j];
      if (!std::isfinite(v)) return false;
      const float diff = v - lo[j];
      const float prod = diff * scale[j];
      double c = std::floor((double)prod);
      if (c < 0.0) c = 0.0;
      if (c > top) c = top;
      codes[(size_t)i * d + j] = (uint16_t)c;
    }
  return true;
}

}  // namespace

namespace {

// Skilling's axes-to-transpose map (J. Skilling, "Programming the Hilbert
// curve", AIP Conf. Proc. 707, 2004) on one point, in place. X[0..d) are the
// permuted, reflected coordinates, `bits` bits each.
//  1. Undo excess work, from the top bit level q = bits-1 down to q = 1 with
//     P = 2^q - 1, coordinates i = 0 .. d-1 in turn: if bit q of X[i] is set,
//     invert the low q bits of X[0]; otherwise exchange the low q bits of X[0]
//     and X[i].
//  2. Gray encode: X[i] ^= X[i-1] for i = 1 .. d-1, in turn.
//  3. t = XOR of (2^q - 1) over the levels q = bits-1 .. 1 at which X[d-1]
//     has its bit set; every X[i] ^= t.
void skilling_transpose(uint32_t* X, int d, int bits) {
  for (int q = bits - 1; q >= 1; --q) {
    const uint32_t P = (1u << q) - 1u;
    for (int i = 0; i < d; ++i) {
      if ((X[i] >> q) & 1u) {
        X[0] ^= P;
      } else {
        const uint32_t t = (X[0] ^ X[i]) & P;
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  for (int i = 1; i < d; ++i) X[i] ^= X[i - 1];
  uint32_t t = 0;
  for (int q = bits - 1; q >= 1; --q)
    if ((X[d - 1] >> q) & 1u) t ^= (1u << q) - 1u;
  for (int i = 0; i < d; ++i) X[i] ^= t;
}

int key_words(int d, int bits) { return (int)(((int64_t)d * bits + 63) / 64); }

// The key is the bit string, most significant first, of level l = 0 .. bits-1
// (level 0 = the top bit) of X[0], X[1], ..., X[d-1]; key bit g = l*d + i is
// bit (bits-1-l) of X[i], and it sits in word g / 64 at bit 63 - g % 64. The
// last word is zero-padded at its low end.
void pack_key(const uint32_t* X, int d, int bits, uint64_t* key) {
  const int W = key_words(d, bits);
  for (int w = 0; w < W; ++w) key[w] = 0;
  for (int l = 0; l < bits; ++l)
    for (int i = 0; i < d; ++i) {
      const int64_t g = (int64_t)l * d + i;
      const uint64_t bit = (X[i] >> (bits - 1 - l)) & 1u;
      key[g / 64] |= bit << (63 - g % 64);
    }
}

// Full key of one code row under tree (pi, r).
void row_key(const uint16_t* code, int d, int bits, const int64_t* pi, const uint8_t* r, uint32_t* X,
             uint64_t* key) {
  const uint32_t full = (1u << bits) - 1u;
  for (int j = 0; j < d; ++j) X[j] = (uint32_t)code[pi[j]] ^ (r[j] ? full : 0u);
  skilling_transpose(X, d, bits);
  pack_key(X, d, bits, key);
}

// Lexicographic comparison of two W-word keys: -1, 0 or 1.
int key_cmp(const uint64_t* a, const uint64_t* b, int W) {
  for (int w = 0; w < W; ++w) {
    if (a[w] < b[w]) return -1;
    if (a[w] > b[w]) return 1;
  }
  return 0;
}

// sigma: point indices ordered by (key, index) ascending (Section 2: the
// Hilbert order; equal keys by index).
void hilbert_order(const uint64_t* keys, int64_t n, int W, int64_t* sigma) {
  std::vector<int64_t> idx((size_t)n);
  for (int64_t i = 0; i < n; ++i) idx[(size_t)i] = i;
  std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
    const int c = key_cmp(keys + (size_t)a * W, keys + (size_t)b * W, W);
    return c != 0 ? c < 0 : a < b;
  });
  for (int64_t i = 0; i < n; ++i) sigma[i] = idx[(size_t)i];
}

// Lower bound: the number of points whose key is smaller than qkey (Section 2:
// binary search in a Hilbert order). Counted over all points, so it needs no
// order at all.
int64_t keys_below(const uint64_t* keys, int64_t n, int W, const uint64_t* qkey) {
  int64_t c = 0;
  for (int64_t i = 0; i < n; ++i)
    if (key_cmp(keys + (size_t)i * W, qkey, W) < 0) ++c;
  return c;
}

}  // namespace

namespace {

constexpr double kInf = std::numeric_limits<double>::infinity();

// Squared Euclidean distance in double, coordinates summed left to right.
double sq_dist(const float* a, const float* b, int d) {
  double s = 0.0;
  for (int j = 0; j < d; ++j) {
    const double t = (double)a[j] - (double)b[j];
    s += t * t;
  }
  return s;
}

// The k best of a candidate multiset by (distance to v, index): repeats and
// the owner (owner >= 0) removed first; (-1, +inf) where fewer than k remain.
void top_k(const float* x, int d, const float* v, int64_t owner, std::vector<int64_t>& cand, int k, int64_t* out_i,
           double* out_d) {
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  std::vector<std::pair<double, int64_t>> scored;
  scored.reserve(cand.size());
  for (int64_t c : cand)
    if (c >= 0 && c != owner) scored.emplace_back(sq_dist(v, x + (size_t)c * d, d), c);
  std::sort(scored.begin(), scored.end());
  for (int j = 0; j < k; ++j) {
    const bool ok = j < (int)scored.size();
    out_i[j] = ok ? scored[(size_t)j].second : -1;
    out_d[j] = ok ? scored[(size_t)j].first : kInf;
  }
}

}  // namespace

extern "C" {

// Tree t's permutation pi[d] (int64) and reflection bits r[d].
void hfo_tree_params(uint64_t seed, int32_t tree, int32_t d, int64_t* pi, uint8_t* r) {
  tree_params(seed, tree, d, pi, r);
}

// Skilling's transposed index of n points (rows of `coords`, d coordinates of
// `bits` bits, uint32) into X (same shape).
void hfo_transpose(const uint32_t* coords, int64_t n, int32_t d, int32_t bits, uint32_t* X) {
  for (int64_t i = 0; i < n; ++i) {
    for (int j = 0; j < d; ++j) X[(size_t)i * d + j] = coords[(size_t)i * d + j];
    skilling_transpose(X + (size_t)i * d, d, bits);
  }
}

// Keys of n transposed indices X (n x d, `bits` bits each): n x W words.
void hfo_pack_key(const uint32_t* X, int64_t n, int32_t d, int32_t bits, uint64_t* keys) {
  const int W = key_words(d, bits);
  for (int64_t i = 0; i < n; ++i) pack_key(X + (size_t)i * d, d, bits, keys + (size_t)i * W);
}

// The forest: lo, scale (d each), codes (n x d), and per tree t the full keys
// keys[t][i][0..W) (point order) and the order sigma[t][0..n). Returns 0, or
// -1 on a non-finite input or bad sizes.
int32_t hfo_forest(const float* x, int64_t n, int32_t d, int32_t T, int32_t bits, uint64_t seed, float* lo,
                   float* scale, uint16_t* codes, uint64_t* keys, int64_t* sigma) {
  if (n < 1 || d < 1 || T < 1 || bits < 1 || bits > 16) return -1;
  if (!axis_range(x, n, d, bits, lo, scale)) return -1;
  if (!quantize(x, n, d, bits, lo, scale, codes)) return -1;
  const int W = key_words(d, bits);
  std::vector<int64_t> pi((size_t)d);
  std::vector<uint8_t> r((size_t)d);
  std::vector<uint32_t> X((size_t)d);
  for (int t = 0; t < T; ++t) {
    tree_params(seed, t, d, pi.data(), r.data());
    uint64_t* kt = keys + (size_t)t * n * W;
    for (int64_t i = 0; i < n; ++i)
      row_key(codes + (size_t)i * d, d, bits, pi.data(), r.data(), X.data(), kt + (size_t)i * W);
    hilbert_order(kt, n, W, sigma + (size_t)t * n);
  }
  return 0;
}

// Algorithm 2 over the given orders: each point's candidates are the points
// at positions p - w .. p + w (p its own position, itself excluded) of every
// order, as a set; the result is its k nearest by (double squared distance,
// index). out_i / out_d: n x k.
int32_t hfo_knn_graph(const float* x, int64_t n, int32_t d, const int64_t* sigma, int32_t T, int32_t w, int32_t k,
                      int64_t* out_i, double* out_d) {
  if (n < 1 || d < 1 || T < 1 || w < 0 || k < 1) return -1;
  std::vector<int64_t> pos((size_t)T * n);
  for (int t = 0; t < T; ++t)
    for (int64_t p = 0; p < n; ++p) pos[(size_t)t * n + sigma[(size_t)t * n + p]] = p;
  std::vector<int64_t> cand;
  for (int64_t i = 0; i < n; ++i) {
    cand.clear();
    for (int t = 0; t < T; ++t) {
      const int64_t p = pos[(size_t)t * n + i];
      for (int64_t o = -w; o <= w; ++o) {
        const int64_t q = p + o;
        if (o != 0 && q >= 0 && q < n) cand.push_back(sigma[(size_t)t * n + q]);
      }
    }
    top_k(x, d, x + (size_t)i * d, i, cand, k, out_i + (size_t)i * k, out_d + (size_t)i * k);
  }
  return 0;
}

// Algorithm 1's first stage and final selection: each query is quantized with
// the forest's lo / scale (clamped), keyed in every tree, and placed at its
// lower bound p among the tree's keys; the candidates are the points at
// positions p - w .. p + w - 1 of that order; the result is the k nearest of
// their union by (double squared distance, index). keys / sigma as
// hfo_forest returns them.
int32_t hfo_search(const float* x, int64_t n, int32_t d, int32_t T, int32_t bits, uint64_t seed, const float* lo,
                   const float* scale, const uint64_t* keys, const int64_t* sigma, const float* q, int64_t nq,
                   int32_t w, int32_t k, int64_t* out_i, double* out_d) {
  if (n < 1 || d < 1 || T < 1 || bits < 1 || bits > 16 || nq < 0 || w < 0 || k < 1) return -1;
  const int W = key_words(d, bits);
  std::vector<uint16_t> qc((size_t)d);
  std::vector<int64_t> pi((size_t)T * d);
  std::vector<uint8_t> r((size_t)T * d);
  for (int t = 0; t < T; ++t) tree_params(seed, t, d, pi.data() + (size_t)t * d, r.data() + (size_t)t * d);
  std::vector<uint32_t> X((size_t)d);
  std::vector<uint64_t> qk((size_t)W);
  std::vector<int64_t> cand;
  for (int64_t j = 0; j < nq; ++j) {
    if (!quantize(q + (size_t)j * d, 1, d, bits, lo, scale, qc.data())) return -1;
    cand.clear();
    for (int t = 0; t < T; ++t) {
      row_key(qc.data(), d, bits, pi.data() + (size_t)t * d, r.data() + (size_t)t * d, X.data(), qk.data());
      const int64_t p = keys_below(keys + (size_t)t * n * W, n, W, qk.data());
      for (int64_t o = -w; o < w; ++o) {
        const int64_t s = p + o;
        if (s >= 0 && s < n) cand.push_back(sigma[(size_t)t * n + s]);
      }
    }
    top_k(x, d, q + (size_t)j * d, -1, cand, k, out_i + (size_t)j * k, out_d + (size_t)j * k);
  }
  return 0;
}

// Exact k nearest of m rows (point indices, each excluding itself) or, when
// rows is null, of m queries q: every point scored, (double squared distance,
// index) order.
int32_t hfo_brute_force(const float* x, int64_t n, int32_t d, const int64_t* rows, const float* q, int64_t m,
                        int32_t k, int64_t* out_i, double* out_d) {
  if (n < 1 || d < 1 || m < 0 || k < 1 || (!rows && !q)) return -1;
  std::vector<int64_t> all((size_t)n);
  for (int64_t i = 0; i < n; ++i) all[(size_t)i] = i;
  std::vector<int64_t> cand;
  for (int64_t j = 0; j < m; ++j) {
    cand = all;
    const int64_t owner = rows ? rows[j] : -1;
    const float* v = rows ? x + (size_t)owner * d : q + (size_t)j * d;
    top_k(x, d, v, owner, cand, k, out_i + (size_t)j * k, out_d + (size_t)j * k);
  }
  return 0;
}

}  // extern "C"
