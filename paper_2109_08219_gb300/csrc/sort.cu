// Output ordering: the k winners W (unique (key, ~idx) composites) are
// sorted descending, i.e. by key descending then index ascending (the
// output order of top-k; the paper leaves it unstated), and written as the
// input dtype's key bits plus int32 indices.
// When the k-th key is tau (tie mode), W holds G (all keys > tau, unsorted)
// followed by the ties at tau in index order, which are already in output
// order: only the first |G| entries are sorted (m below).
//   * k <= 4096: one CTA bitonic-sorts W in shared memory;
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
