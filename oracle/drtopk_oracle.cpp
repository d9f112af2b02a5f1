// CPU oracle for delegate-centric top-k (Dr. Top-k, SC'21, arXiv 2109.08219).
//
// TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
// reference that the CUDA path is checked against. Only the tests, the smoke
// entry and the benchmark's CPU-baseline leg may load it. It shares no code,
// header, table or helper with the CUDA library, and the CUDA library never
// calls it.
//
// Every function follows one passage of the paper:
//   * oracle_map_keys / oracle_unmap_keys : order-preserving 32-bit key map.
//     The paper works on unsigned ints only (Sec. 5, "each data entry is an
//     unsigned integer"); i32 and f32 are mapped to u32 so that the unsigned
//     order equals the signed / IEEE total order (reading G13).
//   * oracle_topk / oracle_kth : the problem statement (Sec. 1): the k
//     largest elements of V, and the k-th largest. Ties are broken by the
//     smallest index and the top-k is returned sorted by (key desc, idx asc)
//     (readings G11, G12).
//   * oracle_delegates : Rule 1 (maximum delegate, Sec. 3.1) generalised by
//     Rule 3 (beta delegates, Sec. 3.3): the beta largest elements of each
//     subrange of 2^alpha consecutive elements.
//   * oracle_threshold : Rule 2 (Sec. 3.2): the k-th largest delegate, a
//     lower bound on the k-th largest element of V.
//   * oracle_candidates : concatenation with filtering (Sec. 3.2, Sec. 3.3,
//     Sec. 4.1): subranges whose maximum delegate is below the threshold are
//     skipped; a subrange whose beta delegates all reach the threshold is
//     scanned and its elements >= threshold are kept; otherwise only its
//     delegates >= threshold are kept (readings G1-G3: ">= threshold").
//   * oracle_drtopk : the four steps in the paper's order (delegate vector,
//     first top-k, concatenation, second top-k; Eq. 1).
//   * oracle_alpha_rule4 : Rule 4 / Eq. 9 with const = 3 and floor rounding
//     (Sec. 4.2; the paper's worked value alpha(2^30, 2^24) = 4).
//   * oracle_bottomk / oracle_kth_smallest : the other criterion of the
//     problem statement (Sec. 1, Sec. 2: "the k largest or smallest"): the k
//     smallest elements ordered by (key asc, idx asc), and the k-th smallest.
//   * oracle_topk_merge : the distributed form's final step (Sec. 4.4): the
//     plain top-k of a set of (key, global index) pairs, whatever their order.
//   * oracle_topk_omp : the same result as oracle_topk computed by chunks on
//     several threads (each thread's local top-k, then the top-k of their
//     union); only the timed multi-core CPU baseline uses it.
//
// Library primitives used as single steps: std::nth_element (selection) and
// std::sort / std::stable_sort.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

enum { U32 = 0, I32 = 1, F32 = 2 };

// Order-preserving map of the raw 32-bit pattern of one key to an unsigned
// 32-bit value whose unsigned order is the key's order.
uint32_t map_key(int dtype, uint32_t bits) {
  if (dtype == U32) return bits;
  if (dtype == I32) return bits ^ 0x80000000u;  // two's complement -> offset binary
  // f32: negative floats (sign bit 1) order reversed -> flip all bits;
  // non-negative floats -> set the sign bit so they sort above all negatives.
  if (bits & 0x80000000u) return ~bits;
  return bits | 0x80000000u;
}

uint32_t unmap_key(int dtype, uint32_t m) {
  if (dtype == U32) return m;
  if (dtype == I32) return m ^ 0x80000000u;
  if (m & 0x80000000u) return m & 0x7FFFFFFFu;  // was non-negative
  return ~m;                                     // was negative
}

struct Pair {
  uint32_t key;  // mapped key
  int64_t idx;   // position in V
};

// The total order of the problem statement: larger key first, then smaller index.
bool before(const Pair& a, const Pair& b) {
  if (a.key != b.key) return a.key > b.key;
  return a.idx < b.idx;
}

// The smallest criterion: smaller key first, then smaller index.
bool before_smallest(const Pair& a, const Pair& b) {
  if (a.key != b.key) return a.key < b.key;
  return a.idx < b.idx;
}

bool valid_dtype(int d) { return d == U32 || d == I32 || d == F32; }

}  // namespace

extern "C" {

// a0 key map over an array (raw bits in, mapped u32 out).
int oracle_map_keys(int dtype, const uint32_t* in, int64_t n, uint32_t* out) {
  if (!valid_dtype(dtype) || n < 0) return 1;
  for (int64_t i = 0; i < n; ++i) out[i] = map_key(dtype, in[i]);
  return 0;
}

int oracle_unmap_keys(int dtype, const uint32_t* in, int64_t n, uint32_t* out) {
  if (!valid_dtype(dtype) || n < 0) return 1;
  for (int64_t i = 0; i < n; ++i) out[i] = unmap_key(dtype, in[i]);
  return 0;
}

// Plain definition of top-k (Sec. 1): order all positions by (key desc,
// idx asc) and return the first k, in that order, as original key bits and
// int32 indices. Returns 0 on success, 2 when k is out of [1, n].
int oracle_topk(int dtype, const uint32_t* keys, int64_t n, int64_t k,
                uint32_t* out_keys, int32_t* out_idx) {
  if (!valid_dtype(dtype)) return 3;
  if (k < 1 || k > n) return 2;
  std::vector<Pair> p(static_cast<size_t>(n));
  for (int64_t i = 0; i < n; ++i) p[i] = Pair{map_key(dtype, keys[i]), i};
  std::nth_element(p.begin(), p.begin() + (k - 1), p.end(), before);
  std::sort(p.begin(), p.begin() + k, before);
  for (int64_t j = 0; j < k; ++j) {
    out_keys[j] = unmap_key(dtype, p[j].key);
    out_idx[j] = static_cast<int32_t>(p[j].idx);
  }
  return 0;
}

// Plain definition of k-selection (Sec. 1): the key at position k of the
// same order (original bits).
int oracle_kth(int dtype, const uint32_t* keys, int64_t n, int64_t k,
               uint32_t* out_kth) {
  if (!valid_dtype(dtype)) return 3;
  if (k < 1 || k > n) return 2;
  std::vector<uint32_t> m(static_cast<size_t>(n));
  for (int64_t i = 0; i < n; ++i) m[i] = map_key(dtype, keys[i]);
  std::nth_element(m.begin(), m.begin() + (k - 1), m.end(),
                   [](uint32_t a, uint32_t b) { return a > b; });
  *out_kth = unmap_key(dtype, m[k - 1]);
  return 0;
}

// Plain definition of the smallest criterion (Sec. 1, Sec. 2): order all
// positions by (key asc, idx asc) and return the first k, in that order.
int oracle_bottomk(int dtype, const uint32_t* keys, int64_t n, int64_t k,
                   uint32_t* out_keys, int32_t* out_idx) {
  if (!valid_dtype(dtype)) return 3;
  if (k < 1 || k > n) return 2;
  std::vector<Pair> p(static_cast<size_t>(n));
  for (int64_t i = 0; i < n; ++i) p[i] = Pair{map_key(dtype, keys[i]), i};
  std::nth_element(p.begin(), p.begin() + (k - 1), p.end(), before_smallest);
  std::sort(p.begin(), p.begin() + k, before_smallest);
  for (int64_t j = 0; j < k; ++j) {
    out_keys[j] = unmap_key(dtype, p[j].key);
    out_idx[j] = static_cast<int32_t>(p[j].idx);
  }
  return 0;
}

// The k-th smallest key (original bits).
int oracle_kth_smallest(int dtype, const uint32_t* keys, int64_t n, int64_t k,
                        uint32_t* out_kth) {
  if (!valid_dtype(dtype)) return 3;
  if (k < 1 || k > n) return 2;
  std::vector<uint32_t> m(static_cast<size_t>(n));
  for (int64_t i = 0; i < n; ++i) m[i] = map_key(dtype, keys[i]);
  std::nth_element(m.begin(), m.begin() + (k - 1), m.end());
  *out_kth = unmap_key(dtype, m[k - 1]);
  return 0;
}

// Final step of the distributed form (Sec. 4.4): the top-k of m pairs
// (key bits, int64 global index) in any order, by (key desc, idx asc), or
// by (key asc, idx asc) when smallest != 0.
int oracle_topk_merge(int dtype, const uint32_t* keys, const int64_t* gidx, int64_t m,
                      int64_t k, int smallest, uint32_t* out_keys, int64_t* out_gidx) {
  if (!valid_dtype(dtype)) return 3;
  if (k < 1 || k > m) return 2;
  std::vector<Pair> p(static_cast<size_t>(m));
  for (int64_t i = 0; i < m; ++i) p[i] = Pair{map_key(dtype, keys[i]), gidx[i]};
  auto order = smallest ? before_smallest : before;
  std::nth_element(p.begin(), p.begin() + (k - 1), p.end(), order);
  std::sort(p.begin(), p.begin() + k, order);
  for (int64_t j = 0; j < k; ++j) {
    out_keys[j] = unmap_key(dtype, p[j].key);
    out_gidx[j] = p[j].idx;
  }
  return 0;
}

// Multi-core variant of oracle_topk, for the timed CPU baseline only: the
// positions are split into one contiguous chunk per thread; each thread
// keeps its chunk's top-min(k, chunk) by nth_element; the union of these
// holds the answer (an element of the top-k is in its own chunk's top-k),
// and one nth_element + sort over the union gives it. threads <= 0: all
// available. *used receives the thread count.
int oracle_topk_omp(int dtype, const uint32_t* keys, int64_t n, int64_t k, int threads,
                    uint32_t* out_keys, int32_t* out_idx, int* used) {
  if (!valid_dtype(dtype)) return 3;
  if (k < 1 || k > n) return 2;
  int T = 1;
#ifdef _OPENMP
  T = threads > 0 ? threads : omp_get_max_threads();
#endif
  if (T < 1) T = 1;
  if (used) *used = T;
  std::vector<std::vector<Pair>> local(static_cast<size_t>(T));
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(static, 1)
#endif
  for (int t = 0; t < T; ++t) {
    const int64_t lo = n * t / T, hi = n * (t + 1) / T;
    std::vector<Pair>& p = local[static_cast<size_t>(t)];
    p.resize(static_cast<size_t>(hi - lo));
    for (int64_t i = lo; i < hi; ++i) p[i - lo] = Pair{map_key(dtype, keys[i]), i};
    const int64_t kk = std::min<int64_t>(k, hi - lo);
    if (kk > 0 && kk < hi - lo) {
      std::nth_element(p.begin(), p.begin() + (kk - 1), p.end(), before);
      p.resize(static_cast<size_t>(kk));
    }
  }
  std::vector<Pair> u;
  for (auto& p : local) u.insert(u.end(), p.begin(), p.end());
  std::nth_element(u.begin(), u.begin() + (k - 1), u.end(), before);
  std::sort(u.begin(), u.begin() + k, before);
  for (int64_t j = 0; j < k; ++j) {
    out_keys[j] = unmap_key(dtype, u[j].key);
    out_idx[j] = static_cast<int32_t>(u[j].idx);
  }
  return 0;
}

// Rule 1 / Rule 3 (Sec. 3.1, 3.3): for each subrange S_i of 2^alpha
// consecutive mapped keys (the last one may be shorter), the beta largest
// elements m_i^0 >= ... >= m_i^{beta-1}, ties ordered by smaller index.
// Output layout: d_keys[i*beta + j], d_idx[i*beta + j] (global index).
// A subrange with fewer than beta elements fills its missing slots with
// key 0 and index -1 (not part of D). Returns the number of subranges.
int64_t oracle_delegates(const uint32_t* mapped, int64_t n, int alpha, int beta,
                         uint32_t* d_keys, int64_t* d_idx) {
  if (n < 0 || alpha < 0 || alpha > 30 || beta < 1) return -1;
  const int64_t len = int64_t(1) << alpha;
  const int64_t S = (n + len - 1) / len;
  for (int64_t i = 0; i < S; ++i) {
    const int64_t lo = i * len;
    const int64_t hi = std::min(n, lo + len);
    std::vector<Pair> p;
    for (int64_t t = lo; t < hi; ++t) p.push_back(Pair{mapped[t], t});
    std::sort(p.begin(), p.end(), before);
    for (int j = 0; j < beta; ++j) {
      if (j < static_cast<int64_t>(p.size())) {
        d_keys[i * beta + j] = p[j].key;
        d_idx[i * beta + j] = p[j].idx;
      } else {
        d_keys[i * beta + j] = 0;
        d_idx[i * beta + j] = -1;
      }
    }
  }
  return S;
}

// Rule 2 (Sec. 3.2): tau = min(topk(D)), the k-th largest element of the
// delegate multiset D (slots with index -1 are not in D). When D holds fewer
// than k elements no delegate bound exists and tau is the smallest mapped
// key, 0 (reading G10): every element then qualifies.
int oracle_threshold(const uint32_t* d_keys, const int64_t* d_idx, int64_t m,
                     int64_t k, uint32_t* tau) {
  if (m < 0 || k < 1) return 2;
  std::vector<uint32_t> d;
  for (int64_t j = 0; j < m; ++j)
    if (d_idx[j] >= 0) d.push_back(d_keys[j]);
  if (static_cast<int64_t>(d.size()) < k) {
    *tau = 0;
    return 0;
  }
  std::nth_element(d.begin(), d.begin() + (k - 1), d.end(),
                   [](uint32_t a, uint32_t b) { return a > b; });
  *tau = d[k - 1];
  return 0;
}

// Concatenation with filtering (Rules 1-3; Sec. 3.2, 3.3, 4.1). For each
// subrange, in index order:
//   * m^0 < tau            : skipped (Rule 1 in its threshold form, G1);
//   * all beta delegates >= tau and the subrange holds more than beta
//     elements             : scanned; every element >= tau is kept (Rule 2, G2);
//   * otherwise            : only the delegates >= tau are kept (Rule 3, G3).
// Kept elements are written as (mapped key, global index) in index order
// within each subrange. Returns the candidate count (which may exceed cap;
// then only cap entries are written); *scanned receives the number of
// scanned subranges.
int64_t oracle_candidates(const uint32_t* mapped, int64_t n, int alpha, int beta,
                          const uint32_t* d_keys, const int64_t* d_idx,
                          uint32_t tau, uint32_t* c_keys, int64_t* c_idx,
                          int64_t cap, int64_t* scanned) {
  if (n < 0 || alpha < 0 || alpha > 30 || beta < 1) return -1;
  const int64_t len = int64_t(1) << alpha;
  const int64_t S = (n + len - 1) / len;
  int64_t cnt = 0, sc = 0;
  auto keep = [&](uint32_t key, int64_t idx) {
    if (cnt < cap) {
      c_keys[cnt] = key;
      c_idx[cnt] = idx;
    }
    ++cnt;
  };
  for (int64_t i = 0; i < S; ++i) {
    const int64_t lo = i * len;
    const int64_t hi = std::min(n, lo + len);
    const uint32_t* dk = d_keys + i * beta;
    const int64_t* di = d_idx + i * beta;
    if (dk[0] < tau) continue;
    const bool full = (hi - lo) > beta;
    if (full && dk[beta - 1] >= tau) {
      ++sc;
      for (int64_t t = lo; t < hi; ++t)
        if (mapped[t] >= tau) keep(mapped[t], t);
    } else {
      std::vector<Pair> q;
      for (int j = 0; j < beta; ++j)
        if (di[j] >= 0 && dk[j] >= tau) q.push_back(Pair{dk[j], di[j]});
      std::sort(q.begin(), q.end(),
                [](const Pair& a, const Pair& b) { return a.idx < b.idx; });
      for (const Pair& p : q) keep(p.key, p.idx);
    }
  }
  if (scanned) *scanned = sc;
  return cnt;
}

// The method end to end, in the paper's order (Eq. 1): delegate vector,
// first top-k (threshold), concatenation with filtering, second top-k over
// the concatenated vector. The second top-k uses the plain definition.
// stats (optional, 4 entries): [tau (mapped), |C|, scanned subranges, S].
int oracle_drtopk(int dtype, const uint32_t* keys, int64_t n, int64_t k,
                  int alpha, int beta, uint32_t* out_keys, int32_t* out_idx,
                  int64_t* stats) {
  if (!valid_dtype(dtype)) return 3;
  if (k < 1 || k > n) return 2;
  if (alpha < 0 || alpha > 30 || beta < 1) return 1;
  std::vector<uint32_t> mapped(static_cast<size_t>(n));
  for (int64_t i = 0; i < n; ++i) mapped[i] = map_key(dtype, keys[i]);
  const int64_t len = int64_t(1) << alpha;
  const int64_t S = (n + len - 1) / len;
  std::vector<uint32_t> dk(static_cast<size_t>(S * beta));
  std::vector<int64_t> di(static_cast<size_t>(S * beta));
  oracle_delegates(mapped.data(), n, alpha, beta, dk.data(), di.data());
  uint32_t tau = 0;
  oracle_threshold(dk.data(), di.data(), S * beta, k, &tau);
  int64_t scanned = 0;
  const int64_t c = oracle_candidates(mapped.data(), n, alpha, beta, dk.data(),
                                      di.data(), tau, nullptr, nullptr, 0,
                                      &scanned);
  std::vector<uint32_t> ck(static_cast<size_t>(c));
  std::vector<int64_t> ci(static_cast<size_t>(c));
  oracle_candidates(mapped.data(), n, alpha, beta, dk.data(), di.data(), tau,
                    ck.data(), ci.data(), c, &scanned);
  if (c < k) return 4;  // cannot happen when Rules 1-3 hold (|C| >= k)
  std::vector<Pair> p(static_cast<size_t>(c));
  for (int64_t j = 0; j < c; ++j) p[j] = Pair{ck[j], ci[j]};
  std::nth_element(p.begin(), p.begin() + (k - 1), p.end(), before);
  std::sort(p.begin(), p.begin() + k, before);
  for (int64_t j = 0; j < k; ++j) {
    out_keys[j] = unmap_key(dtype, p[j].key);
    out_idx[j] = static_cast<int32_t>(p[j].idx);
  }
  if (stats) {
    stats[0] = tau;
    stats[1] = c;
    stats[2] = scanned;
    stats[3] = S;
  }
  return 0;
}

// Rule 4 / Eq. 9 (Sec. 4.2): alpha = 1/2 (log2|V| - log2 k + const), with
// const = 3 as the paper tunes it, rounded down (the paper's alpha(2^30,
// 2^24) = 4 from 4.5). No clamping: that is a design choice of the library.
int oracle_alpha_rule4(int64_t n, int64_t k, double cnst) {
  if (n < 1 || k < 1) return -1;
  const double a = 0.5 * (std::log2(static_cast<double>(n)) -
                          std::log2(static_cast<double>(k)) + cnst);
  return static_cast<int>(std::floor(a));
}

}  // extern "C"
