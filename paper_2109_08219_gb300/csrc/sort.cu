// Output ordering: the k winners W (unique (key, ~idx) composites) are
// sorted descending, i.e. by key descending then index ascending (the
// output order of top-k; the paper leaves it unstated), and written as the
// input dtype's key bits plus int32 indices.
// When the k-th key is tau (tie mode), W holds G (all keys > tau, unsorted)
// followed by the ties at tau in index order, which are already in output
// order: only the first |G| entries are sorted (m below).
//   * k <= 4096: one CTA bitonic-sorts W in shared memory;
//   * 4096 < k <= 2^21: bucketed by the bits below the common prefix,
//     buckets sorted by warps in registers (the bucketed sort below);
//   * larger k: a stable LSD radix sort of the complemented composites
//     (ascending) with 8-bit digits. One kernel histograms all 8 digits at
//     once; each digit pass is then a single kernel: tiles of 8192 are taken
//     in order from an atomic counter, ranked stably in shared memory, and
//     their global offsets come from a decoupled look-back over the earlier
//     tiles' per-digit counts (bounded waits). A digit equal for all k
//     entries is skipped.
#include "common.cuh"
#include "launch.h"

namespace drtopk {
namespace {

constexpr int kSmallSort = 4096;
constexpr int kSortThreads = 512;
constexpr int kItems = 16;
constexpr int kTile = kSortThreads * kItems;  // 8192
constexpr int kHistThreads = 256;
constexpr uint64_t kFlagAgg = uint64_t(1) << 32;
constexpr uint64_t kFlagIncl = uint64_t(2) << 32;
constexpr uint32_t kLookbackSpin = 1u << 22;


__device__ __forceinline__ void st_relaxed(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void write_out(uint64_t c, int64_t j, int64_t k, int dtype,
                                          uint32_t* out_keys, int32_t* out_idx,
                                          uint32_t* out_kth, Ctl* ctl) {
  const uint32_t key = unmap_key(dtype, comp_key(c));
  if (out_keys) out_keys[j] = key;
  if (out_idx) out_idx[j] = static_cast<int32_t>(comp_idx(c));
  if (j == k - 1) {
    ctl->kth_mapped = comp_key(c);
    if (out_kth) *out_kth = key;
  }
}

// Entries of W that need sorting: all k, or |G| when the tail of W holds
// the ties at tau in index order.
__device__ __forceinline__ int64_t sort_count(const Ctl* ctl, int64_t k) {
  return __ldcg(&ctl->mode) == kModeTies ? static_cast<int64_t>(__ldcg(&ctl->g_count)) : k;
}

__global__ void __launch_bounds__(1024) small_sort_kernel(const uint64_t* w, int k, int dtype,
                                                          uint32_t* out_keys, int32_t* out_idx,
                                                          uint32_t* out_kth, Ctl* ctl,
                                                          uint32_t* err_out) {
  __shared__ uint64_t s[kSmallSort];
  if (threadIdx.x == 0) report_errors(ctl, err_out);
  const int m = static_cast<int>(sort_count(ctl, k));
  int P = 1;
  while (P < m) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = (i < m) ? w[i] : 0ull;
  __syncthreads();
  // bitonic sort, descending
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int j = i ^ stride;
        if (j > i) {
          const bool desc = (i & size) == 0;
          const uint64_t a = s[i], b = s[j];
          if ((a < b) == desc) {
            s[i] = b;
            s[j] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    write_out(i < m ? s[i] : w[i], i, k, dtype, out_keys, out_idx, out_kth, ctl);
}

struct SortParams {
  uint64_t* buf[2];
  uint64_t* status;  // [8][ntiles][256] look-back words (flag << 32 | count)
  int64_t k;
  int64_t ntiles;
  Ctl* ctl;
  uint32_t* err_out;
};

// pass p: digit p (0 = least significant byte) of ~c
__device__ __forceinline__ uint32_t sdigit(uint64_t c, int pass) {
  return static_cast<uint32_t>((~c) >> (8 * pass)) & 255u;
}

__global__ void __launch_bounds__(kHistThreads) sort_hist_all_kernel(SortParams p) {
  __shared__ uint32_t sh[8][256];
  for (int i = threadIdx.x; i < 8 * 256; i += kHistThreads) (&sh[0][0])[i] = 0;
  __syncthreads();
  const uint64_t* src = p.buf[0];
  const uint32_t lane = lane_id();
  const int64_t m = sort_count(p.ctl, p.k);
  for (int64_t b = int64_t(blockIdx.x) * kHistThreads; b < m;
       b += int64_t(gridDim.x) * kHistThreads) {
    const int64_t i = b + threadIdx.x;
    const bool act = i < m;
    const uint32_t am = __ballot_sync(0xFFFFFFFFu, act);
    if (act) {
      const uint64_t c = src[i];
      const int leader = __ffs(am) - 1;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint32_t d = sdigit(c, q);
        // a digit equal across the warp (common: high key bytes) adds once
        if (__all_sync(am, d == __shfl_sync(am, d, leader))) {
          if (static_cast<int>(lane) == leader) atomicAdd(&sh[q][d], __popc(am));
        } else {
          atomicAdd(&sh[q][d], 1u);
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 8 * 256; i += kHistThreads) {
    const uint32_t v = (&sh[0][0])[i];
    if (v) atomicAdd(&(&p.ctl->sort_hist[0][0])[i], v);
  }
  if (last_block(&p.ctl->sort_ticket)) {
    // exclusive offsets per digit, all 8 digit histograms at once (thread d
    // owns bin d of every digit); a digit that holds all k entries is skipped
    __syncthreads();
    uint32_t v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = __ldcg(&p.ctl->sort_hist[q][threadIdx.x]);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t e = block_scan_excl<kHistThreads>(v[q], nullptr);
      p.ctl->sort_hist[q][threadIdx.x] = e;
      const int full = __syncthreads_or(v[q] == static_cast<uint32_t>(m));
      if (threadIdx.x == 0) p.ctl->sort_skip[q] = full ? 1u : 0u;
    }
  }
}

__global__ void __launch_bounds__(kSortThreads, 1) sort_pass_kernel(SortParams p, int pass) {
  Ctl* ctl = p.ctl;
  uint32_t skip[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) skip[q] = __ldcg(&ctl->sort_skip[q]);
  if (skip[pass]) return;
  uint32_t par = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) par ^= (q < pass && skip[q] == 0) ? 1u : 0u;
  const uint64_t* src = p.buf[par];
  uint64_t* dst = p.buf[par ^ 1u];

  constexpr int kWarpsS = kSortThreads / 32;
  constexpr int kPerWarp = kTile / kWarpsS;  // consecutive tile positions per warp
  __shared__ uint32_t s_tile;
  __shared__ uint32_t wcnt[kWarpsS][256];
  __shared__ uint32_t s_off[256];
  __shared__ uint32_t s_start[256];
  extern __shared__ __align__(16) uint64_t s_el[];  // kTile entries, then kTile u16 ranks
  uint16_t* s_rank = reinterpret_cast<uint16_t*>(s_el + kTile);
  const int64_t m = sort_count(ctl, p.k);
  if (threadIdx.x == 0) s_tile = atomicAdd(&ctl->sort_tiles[pass], 1u);
  for (int q = threadIdx.x; q < kWarpsS * 256; q += kSortThreads) (&wcnt[0][0])[q] = 0;
  __syncthreads();
  const int64_t tile = s_tile;
  if (tile * kTile >= m) return;  // beyond the entries to sort (nobody waits on it)
  const int warp = threadIdx.x >> 5;
  const uint32_t lane = lane_id();
  const int64_t w0 = tile * kTile + int64_t(warp) * kPerWarp;

  // stable ranking: warp w owns kPerWarp consecutive tile positions, 32 per
  // round; warp-private digit counters, no block barrier per round. The
  // rank inside (warp, digit) is kept in shared memory.
  uint64_t c[kItems];
  const uint32_t lt = lanemask_lt32();
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = w0 + r * 32 + lane;
    c[r] = (i < m) ? src[i] : 0ull;
  }
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = w0 + r * 32 + lane;
    const bool act = i < m;
    const uint32_t am = __ballot_sync(0xFFFFFFFFu, act);
    if (act) {
      const uint32_t d = sdigit(c[r], pass);
      const uint32_t peers = peers8(am, d);
      const uint32_t before = wcnt[warp][d];
      s_rank[warp * kPerWarp + r * 32 + lane] = static_cast<uint16_t>(before + __popc(peers & lt));
      __syncwarp(am);
      if ((peers & lt) == 0) wcnt[warp][d] = before + __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();

  // per digit: exclusive offsets of the warps inside the tile, then the
  // decoupled look-back over the earlier tiles (thread d handles digit d)
  if (threadIdx.x < 256) {
    const int d = threadIdx.x;
    uint32_t cnt = 0;
    for (int q = 0; q < kWarpsS; ++q) {
      const uint32_t v = wcnt[q][d];
      wcnt[q][d] = cnt;
      cnt += v;
    }
    uint64_t* st = p.status + (int64_t(pass) * p.ntiles) * 256;
    uint32_t excl = 0;
    if (tile == 0) {
      st_relaxed(&st[d], kFlagIncl | cnt);
    } else {
      st_relaxed(&st[tile * 256 + d], kFlagAgg | cnt);
      // windowed look-back: read kWin predecessors per round trip, add
      // their counts back to the nearest inclusive prefix
      constexpr int kWin = 8;
      int64_t t = tile - 1;
      uint32_t spins = 0;
      bool found = false;
      while (t >= 0 && !found) {
        uint64_t v[kWin];
#pragma unroll
        for (int j = 0; j < kWin; ++j)
          v[j] = (t - j >= 0) ? ld_relaxed(&st[(t - j) * 256 + d]) : kFlagIncl;
        int used = 0;
        bool stall = false;
#pragma unroll
        for (int j = 0; j < kWin; ++j) {
          if (!stall && !found) {
            const uint64_t f = v[j] & ~uint64_t(0xFFFFFFFFu);
            if (f == 0) {
              stall = true;
            } else {
              excl += static_cast<uint32_t>(v[j]);
              ++used;
              if (f == kFlagIncl) found = true;
            }
          }
        }
        t -= used;
        if (stall && ++spins > kLookbackSpin) {
          atomicOr(&ctl->error, kErrTimeout);
          break;
        }
      }
      st_relaxed(&st[tile * 256 + d], kFlagIncl | (excl + cnt));
    }
    s_off[d] = __ldcg(&ctl->sort_hist[pass][d]) + excl;
    s_start[d] = cnt;
  }
  __syncthreads();
  // tile-local start of each digit run (exclusive scan of the 256 counts)
  {
    const uint32_t v = threadIdx.x < 256 ? s_start[threadIdx.x] : 0u;
    const uint32_t e = block_scan_excl<kSortThreads>(v, nullptr);
    if (threadIdx.x < 256) s_start[threadIdx.x] = e;
  }
  __syncthreads();
  // reorder the tile by digit in shared memory, then write each digit's run
  // to consecutive global positions (coalesced)
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = w0 + r * 32 + lane;
    if (i < m) {
      const uint32_t d = sdigit(c[r], pass);
      s_el[s_start[d] + wcnt[warp][d] + s_rank[warp * kPerWarp + r * 32 + lane]] = c[r];
    }
  }
  __syncthreads();
  const int64_t tcount = imin64(kTile, m - tile * kTile);
  for (int j = threadIdx.x; j < tcount; j += kSortThreads) {
    const uint64_t e = s_el[j];
    const uint32_t d = sdigit(e, pass);
    dst[s_off[d] + (j - s_start[d])] = e;
  }
}

// --------------------------------------------------- bucketed output sort ---
// For 4096 < k <= kBucketMaxK. The m entries of W to sort are unique
// composites; all of them share the bits above their highest varying bit.
// Bucket = the bb bits just below that common prefix, bb chosen so that a
// bucket holds about 32 entries on average (bb = ceil(log2 m) - 5, 1..15),
// numbered so that a larger bucket holds larger composites. The common
// prefix comes from the range the entries are known to lie in: [the k-th
// composite found by the second select, key_max's largest composite] in
// select mode, [(tau + 1) << 32, same] for G in tie mode. Counting pass
// (atomics aggregated per warp), one-CTA scan of the counts in descending
// bucket order, atomic scatter (the order inside a bucket does not matter:
// every bucket is sorted in full afterwards). Then one warp sorts a bucket
// of up to 128 entries in registers (bitonic network over shuffles) and
// writes its outputs; larger buckets (entries that share many bits, e.g.
// clustered keys) are listed and sorted by whole CTAs: in shared memory up
// to kGroupCap entries, else in chunks merged by merge path, exact but
// slower.
constexpr int kBktMaxBits = 15;
constexpr int kBktMax = 1 << kBktMaxBits;
constexpr int kBktThreads = 256;
constexpr int kWarpSortMax = 128;
constexpr int kGroupCap = 8192;
constexpr int kBigThreads = 512;
constexpr int64_t kBucketMaxK = int64_t(1) << 21;

struct BktHdr {                  // zeroed before the sort
  uint32_t nbig;                 // buckets listed for the CTA path
  uint32_t pad[7];
};
// Layout of the sort status region: header, then count, off, cursor and
// the big-bucket list, kBktMax words each.
struct BktParams {
  uint64_t* w;         // W: entries [0, m) to sort, ties after them
  uint64_t* w2;        // bucketed entries
  BktHdr* hdr;
  uint32_t* count;
  uint32_t* off;       // first output position of each bucket
  uint32_t* cursor;    // scatter cursors, start at off
  uint32_t* big;       // buckets of more than kWarpSortMax entries
  Ctl* ctl;
  uint32_t* err_out;
  int64_t k;
  int full_range;      // entries may lie anywhere below key_max (ablations)
};

// Bucket bits (bb) and shift of the current sort, from m and the bounds.
struct BktGeom {
  int bb;
  uint32_t shift;
};
__device__ __forceinline__ BktGeom bkt_geom(const Ctl* ctl, int64_t m, int full_range) {
  int lg = 0;
  while ((int64_t(1) << lg) < m) ++lg;  // ceil(log2 m)
  int bb = lg - 5;
  bb = bb < 1 ? 1 : (bb > kBktMaxBits ? kBktMaxBits : bb);
  const uint64_t hi = (static_cast<uint64_t>(__ldcg(&ctl->key_max)) << 32) | 0xFFFFFFFFull;
  // (ablations keep entries below tau in G: no lower bound then)
  const uint64_t lo = full_range ? 0ull
                      : __ldcg(&ctl->mode) == kModeTies
                          ? (static_cast<uint64_t>(__ldcg(&ctl->tau)) + 1) << 32
                          : __ldcg(&ctl->gsel.prefix);
  const unsigned long long vary = lo ^ hi;
  BktGeom g{bb, 0u};
  if (vary != 0) {
    const int top = 63 - __clzll(static_cast<long long>(vary));
    g.shift = static_cast<uint32_t>(top >= bb - 1 ? top - (bb - 1) : 0);
  }
  return g;
}

__global__ void __launch_bounds__(kBktThreads) bkt_count_kernel(BktParams p) {
  const int64_t m = sort_count(p.ctl, p.k);
  const BktGeom g = bkt_geom(p.ctl, m, p.full_range);
  const uint32_t mask = (1u << g.bb) - 1u;
  const uint32_t lane = lane_id();
  for (int64_t base = int64_t(blockIdx.x) * kBktThreads + (threadIdx.x & ~31u); base < m;
       base += int64_t(gridDim.x) * kBktThreads) {
    const int64_t i = base + lane;
    const bool act = i < m;
    const uint32_t am = __ballot_sync(0xFFFFFFFFu, act);
    if (act) {
      const uint32_t b = static_cast<uint32_t>(p.w[i] >> g.shift) & mask;
      const uint32_t peers = __match_any_sync(am, b);
      if (static_cast<int>(lane) == __ffs(peers) - 1) atomicAdd(&p.count[b], __popc(peers));
    }
  }
}

// One CTA: offsets in descending bucket order, cursors, big-bucket list.
// Output-order slot t holds bucket nb - 1 - t. The counts are staged in
// shared memory (row of 32 slots per thread, padded to 33 words: no bank
// conflicts); thread th scans slots [32 th, 32 th + 32) after one block
// scan of the per-thread sums.
constexpr int kScanSmemWords = (kBktMax / 32) * 33;
__global__ void __launch_bounds__(1024) bkt_scan_kernel(BktParams p) {
  extern __shared__ uint32_t s_cnt[];  // kScanSmemWords
  const int64_t m = sort_count(p.ctl, p.k);
  const int nb = 1 << bkt_geom(p.ctl, m, p.full_range).bb;
  auto at = [](int t) { return (t >> 5) * 33 + (t & 31); };
  for (int t = threadIdx.x; t < kBktMax; t += 1024)
    s_cnt[at(t)] = t < nb ? __ldcg(&p.count[nb - 1 - t]) : 0u;
  __syncthreads();
  uint32_t sum = 0;
#pragma unroll 8
  for (int j = 0; j < 32; ++j) sum += s_cnt[threadIdx.x * 33 + j];
  uint32_t run = block_scan_excl<1024>(sum, nullptr);
#pragma unroll 8
  for (int j = 0; j < 32; ++j) {
    const uint32_t c = s_cnt[threadIdx.x * 33 + j];
    s_cnt[threadIdx.x * 33 + j] = run;
    if (c > static_cast<uint32_t>(kWarpSortMax))
      p.big[atomicAdd(&p.hdr->nbig, 1u)] = static_cast<uint32_t>(nb - 1 - (threadIdx.x * 32 + j));
    run += c;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nb; t += 1024) {
    const uint32_t o = s_cnt[at(t)];
    p.off[nb - 1 - t] = o;
    p.cursor[nb - 1 - t] = o;
  }
}

__global__ void __launch_bounds__(kBktThreads) bkt_scatter_kernel(BktParams p) {
  const int64_t m = sort_count(p.ctl, p.k);
  const BktGeom g = bkt_geom(p.ctl, m, p.full_range);
  const uint32_t mask = (1u << g.bb) - 1u;
  const uint32_t lane = lane_id();
  const uint32_t lt = lanemask_lt32();
  for (int64_t base = int64_t(blockIdx.x) * kBktThreads + (threadIdx.x & ~31u); base < m;
       base += int64_t(gridDim.x) * kBktThreads) {
    const int64_t i = base + lane;
    const bool act = i < m;
    const uint64_t c = act ? p.w[i] : 0ull;
    const uint32_t b = static_cast<uint32_t>(c >> g.shift) & mask;
    const uint32_t am = __ballot_sync(0xFFFFFFFFu, act);
    if (act) {
      const uint32_t peers = __match_any_sync(am, b);
      const int leader = __ffs(peers) - 1;
      uint32_t pos = 0;
      if (static_cast<int>(lane) == leader) pos = atomicAdd(&p.cursor[b], __popc(peers));
      pos = __shfl_sync(peers, pos, leader) + __popc(peers & lt);
      p.w2[pos] = c;
    }
  }
}

// Descending bitonic sort of the P = 32 * E entries v[e] of a warp (entry
// index e * 32 + lane): strides below 32 exchange across lanes by shuffles,
// larger strides between a lane's own registers.
template <int E>
__device__ __forceinline__ void warp_bitonic_desc(uint64_t (&v)[E]) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int size = 2; size <= 32 * E; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      if (stride >= 32) {
        const int es = stride >> 5;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int e2 = e ^ es;
          if (e < e2) {
            const bool desc = ((e * 32 + static_cast<int>(lane)) & size) == 0;
            const uint64_t a = v[e], b = v[e2];
            if ((a < b) == desc) {
              v[e] = b;
              v[e2] = a;
            }
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, v[e], stride);
          const bool desc = ((e * 32 + static_cast<int>(lane)) & size) == 0;
          const bool lower = (lane & static_cast<uint32_t>(stride)) == 0;
          const bool keep_max = lower == desc;
          v[e] = keep_max ? (v[e] > o ? v[e] : o) : (v[e] < o ? v[e] : o);
        }
      }
    }
  }
}

template <int E>
__device__ __forceinline__ void warp_sort_bucket(const BktParams& p, int64_t o, int n, int dtype,
                                                 uint32_t* out_keys, int32_t* out_idx,
                                                 uint32_t* out_kth) {
  const uint32_t lane = lane_id();
  uint64_t v[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * 32 + static_cast<int>(lane);
    v[e] = i < n ? p.w2[o + i] : 0ull;  // 0 is below every composite
  }
  warp_bitonic_desc<E>(v);
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = e * 32 + static_cast<int>(lane);
    if (i < n) write_out(v[e], o + i, p.k, dtype, out_keys, out_idx, out_kth, p.ctl);
  }
}

// One warp per bucket of up to kWarpSortMax entries; also copies the ties
// that follow G (already in output order).
__global__ void __launch_bounds__(kBktThreads) bkt_warp_finish_kernel(BktParams p, int dtype,
                                                                      uint32_t* out_keys,
                                                                      int32_t* out_idx,
                                                                      uint32_t* out_kth) {
  if (blockIdx.x == 0 && threadIdx.x == 0) report_errors(p.ctl, p.err_out);
  const int64_t m = sort_count(p.ctl, p.k);
  for (int64_t j = m + int64_t(blockIdx.x) * kBktThreads + threadIdx.x; j < p.k;
       j += int64_t(gridDim.x) * kBktThreads)
    write_out(p.w[j], j, p.k, dtype, out_keys, out_idx, out_kth, p.ctl);
  if (m == 0) return;
  const int nb = 1 << bkt_geom(p.ctl, m, p.full_range).bb;
  const int warps = static_cast<int>(gridDim.x) * (kBktThreads / 32);
  for (int b = static_cast<int>(blockIdx.x) * (kBktThreads / 32) + (threadIdx.x >> 5); b < nb;
       b += warps) {
    const int n = static_cast<int>(__ldcg(&p.count[b]));
    if (n == 0 || n > kWarpSortMax) continue;  // uniform over the warp
    const int64_t o = __ldcg(&p.off[b]);
    if (n <= 32) warp_sort_bucket<1>(p, o, n, dtype, out_keys, out_idx, out_kth);
    else if (n <= 64) warp_sort_bucket<2>(p, o, n, dtype, out_keys, out_idx, out_kth);
    else warp_sort_bucket<4>(p, o, n, dtype, out_keys, out_idx, out_kth);
  }
}

// Descending bitonic sort of s[0, N), N a power of two, by the whole CTA.
__device__ __forceinline__ void cta_bitonic_desc(uint64_t* s, int N) {
  for (int size = 2; size <= N; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int q = threadIdx.x; q < (N >> 1); q += blockDim.x) {
        const int i = 2 * q - (q & (stride - 1));
        const int j = i + stride;
        const bool desc = (i & size) == 0;
        const uint64_t a = s[i], b = s[j];
        if ((a < b) == desc) {
          s[i] = b;
          s[j] = a;
        }
      }
      __syncthreads();
    }
  }
}

// Loads src[0, n) (n <= kGroupCap) into s, pads to a power of two with 0
// (below every composite) and sorts descending.
__device__ __forceinline__ void cta_sort_chunk(const uint64_t* src, int n, uint64_t* s) {
  int N = 1;
  while (N < n) N <<= 1;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s[i] = i < n ? src[i] : 0ull;
  __syncthreads();
  cta_bitonic_desc(s, N);
}

// Merges the descending runs a[0, na) and b[0, nb) (disjoint values) into
// dst[0, na + nb): each thread finds its output range's split by a merge
// path search and merges that range.
__device__ void cta_merge_desc(const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb,
                               uint64_t* dst) {
  const int64_t L = na + nb;
  const int64_t T = blockDim.x;
  const int64_t d0 = L * threadIdx.x / T, d1 = L * (threadIdx.x + 1) / T;
  int64_t lo = d0 > nb ? d0 - nb : 0, hi = d0 < na ? d0 : na;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] > b[d0 - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  int64_t i = lo, j = d0 - lo;
  for (int64_t d = d0; d < d1; ++d) {
    if (i < na && (j >= nb || a[i] > b[j])) dst[d] = a[i++];
    else dst[d] = b[j++];
  }
}

// Buckets of more than kWarpSortMax entries, one CTA each: in shared memory
// up to kGroupCap entries; else sorted chunks of kGroupCap merged pairwise,
// ping-ponging between the bucket's range of w2 and the same range of W
// (consumed by the scatter).
__global__ void __launch_bounds__(kBigThreads) bkt_big_finish_kernel(BktParams p, int dtype,
                                                                     uint32_t* out_keys,
                                                                     int32_t* out_idx,
                                                                     uint32_t* out_kth) {
  extern __shared__ __align__(16) uint64_t s_grp[];  // kGroupCap entries
  const uint32_t nbig = __ldcg(&p.hdr->nbig);
  for (uint32_t t = blockIdx.x; t < nbig; t += gridDim.x) {
    const uint32_t b = __ldcg(&p.big[t]);
    const int64_t P0 = __ldcg(&p.off[b]);
    const int64_t size = __ldcg(&p.count[b]);
    if (size <= kGroupCap) {
      cta_sort_chunk(p.w2 + P0, static_cast<int>(size), s_grp);
      for (int i = threadIdx.x; i < size; i += kBigThreads)
        write_out(s_grp[i], P0 + i, p.k, dtype, out_keys, out_idx, out_kth, p.ctl);
      __syncthreads();
      continue;
    }
    uint64_t* bufs[2] = {p.w2 + P0, p.w + P0};
    for (int64_t c0 = 0; c0 < size; c0 += kGroupCap) {
      const int n = static_cast<int>(imin64(kGroupCap, size - c0));
      cta_sort_chunk(bufs[0] + c0, n, s_grp);
      for (int i = threadIdx.x; i < n; i += kBigThreads) bufs[0][c0 + i] = s_grp[i];
      __syncthreads();
    }
    int src = 0;
    for (int64_t r = kGroupCap; r < size; r <<= 1) {
      for (int64_t s0 = 0; s0 < size; s0 += 2 * r) {
        const int64_t na = imin64(r, size - s0);
        const int64_t nb = imin64(r, size - s0 - na);
        cta_merge_desc(bufs[src] + s0, na, bufs[src] + s0 + na, nb, bufs[src ^ 1] + s0);
      }
      __syncthreads();
      src ^= 1;
    }
    for (int64_t i = threadIdx.x; i < size; i += kBigThreads)
      write_out(bufs[src][i], P0 + i, p.k, dtype, out_keys, out_idx, out_kth, p.ctl);
    __syncthreads();
  }
}

__global__ void finalize_kernel(SortParams p, int dtype, uint32_t* out_keys, int32_t* out_idx,
                                uint32_t* out_kth) {
  if (blockIdx.x == 0 && threadIdx.x == 0) report_errors(p.ctl, p.err_out);
  uint32_t skip[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) skip[q] = __ldcg(&p.ctl->sort_skip[q]);
  uint32_t par = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) par ^= (skip[q] == 0) ? 1u : 0u;
  const uint64_t* src = p.buf[par];
  const int64_t m = sort_count(p.ctl, p.k);
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < p.k;
       j += int64_t(gridDim.x) * blockDim.x)
    write_out(j < m ? src[j] : p.buf[0][j], j, p.k, dtype, out_keys, out_idx, out_kth, p.ctl);
}

}  // namespace

size_t sort_status_words(int64_t k) {
  if (k <= kSmallSort) return 0;
  if (k <= kBucketMaxK) return (sizeof(BktHdr) + size_t(4) * kBktMax * 4 + 7) / 8;
  const int64_t nt = (k + kTile - 1) / kTile;
  return static_cast<size_t>(8 * nt * 256);
}

cudaError_t launch_sort_output(const Work& w, void* out_keys, int32_t* out_idx, void* out_kth,
                               int sms, cudaStream_t s) {
  if (w.k <= kSmallSort) {
    small_sort_kernel<<<1, 1024, 0, s>>>(w.w, static_cast<int>(w.k), w.dtype,
                                         static_cast<uint32_t*>(out_keys), out_idx,
                                         static_cast<uint32_t*>(out_kth), w.ctl, w.err_out);
    note_launch();
    return cudaGetLastError();
  }
  if (w.k <= kBucketMaxK) {
    BktParams q;
    q.w = w.w;
    q.w2 = w.w2;
    q.hdr = reinterpret_cast<BktHdr*>(w.sort_status);
    q.count = reinterpret_cast<uint32_t*>(q.hdr + 1);
    q.off = q.count + kBktMax;
    q.cursor = q.off + kBktMax;
    q.big = q.cursor + kBktMax;
    q.ctl = w.ctl;
    q.err_out = w.err_out;
    q.k = w.k;
    q.full_range = w.ablate != 0;
    // the header and the counts of as many buckets as k can use
    int lg = 0;
    while ((int64_t(1) << lg) < w.k) ++lg;
    const int bbmax = std::max(1, std::min(kBktMaxBits, lg - 5));
    cudaError_t e = cudaMemsetAsync(q.hdr, 0, sizeof(BktHdr) + (size_t(4) << bbmax), s);
    if (e != cudaSuccess) return e;
    const int g = static_cast<int>(
        std::min<int64_t>((w.k + kBktThreads * 8 - 1) / (kBktThreads * 8), int64_t(sms) * 4));
    bkt_count_kernel<<<g, kBktThreads, 0, s>>>(q);
    cudaFuncSetAttribute(bkt_scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kScanSmemWords * 4);
    bkt_scan_kernel<<<1, 1024, kScanSmemWords * 4, s>>>(q);
    bkt_scatter_kernel<<<g, kBktThreads, 0, s>>>(q);
    const int gw = static_cast<int>(std::min<int64_t>(
        std::max<int64_t>((int64_t(1) << bbmax) / (kBktThreads / 32), 1), int64_t(sms) * 8));
    bkt_warp_finish_kernel<<<gw, kBktThreads, 0, s>>>(q, w.dtype,
                                                      static_cast<uint32_t*>(out_keys), out_idx,
                                                      static_cast<uint32_t*>(out_kth));
    const int dsm = kGroupCap * 8;
    cudaFuncSetAttribute(bkt_big_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm);
    bkt_big_finish_kernel<<<sms, kBigThreads, dsm, s>>>(q, w.dtype, static_cast<uint32_t*>(out_keys),
                                                        out_idx, static_cast<uint32_t*>(out_kth));
    note_launch(5);
    return cudaGetLastError();
  }
  SortParams p;
  p.buf[0] = w.w;
  p.buf[1] = w.w2;
  p.status = w.sort_status;
  p.k = w.k;
  p.ntiles = (w.k + kTile - 1) / kTile;
  p.ctl = w.ctl;
  p.err_out = w.err_out;
  cudaError_t e = cudaMemsetAsync(p.status, 0, sort_status_words(w.k) * 8, s);
  if (e != cudaSuccess) return e;
  const int gh = static_cast<int>(std::min<int64_t>((w.k + kHistThreads * 16 - 1) / (kHistThreads * 16),
                                                     int64_t(sms) * 2));
  sort_hist_all_kernel<<<gh, kHistThreads, 0, s>>>(p);
  const size_t dsm = static_cast<size_t>(kTile) * (8 + 2);
  cudaFuncSetAttribute(sort_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(dsm));
  for (int pass = 0; pass < 8; ++pass)
    sort_pass_kernel<<<static_cast<unsigned>(p.ntiles), kSortThreads, dsm, s>>>(p, pass);
  const int g = static_cast<int>(std::min<int64_t>((w.k + 255) / 256, int64_t(sms) * 8));
  finalize_kernel<<<g, 256, 0, s>>>(p, w.dtype, static_cast<uint32_t*>(out_keys), out_idx,
                                    static_cast<uint32_t*>(out_kth));
  note_launch(10);
  return cudaGetLastError();
}

}  // namespace drtopk
