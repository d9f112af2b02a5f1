// Output ordering: the k winners W (unique (key, ~idx) composites) are
// sorted descending, i.e. by key descending then index ascending (the
// output order of top-k; the paper leaves it unstated), and written as the
// input dtype's key bits plus int32 indices.
//   * k <= 4096: one CTA bitonic-sorts W in shared memory;
//   * larger k: a stable LSD radix sort of the complemented composites
//     (ascending) with 8-bit digits. One kernel histograms all 8 digits at
//     once; each digit pass is then a single kernel: tiles of 4096 are taken
//     in order from an atomic counter, ranked stably in shared memory, and
//     their global offsets come from a decoupled look-back over the earlier
//     tiles' per-digit counts (bounded waits). A digit equal for all k
//     entries is skipped.
#include "common.cuh"
#include "launch.h"

namespace drtopk {
namespace {

constexpr int kSmallSort = 4096;
constexpr int kSortThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kSortThreads * kItems;  // 4096
constexpr uint64_t kFlagAgg = uint64_t(1) << 32;
constexpr uint64_t kFlagIncl = uint64_t(2) << 32;
constexpr uint32_t kLookbackSpin = 1u << 22;

__device__ __forceinline__ uint32_t lanemask_lt_s() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

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

__global__ void __launch_bounds__(1024) small_sort_kernel(const uint64_t* w, int k, int dtype,
                                                          uint32_t* out_keys, int32_t* out_idx,
                                                          uint32_t* out_kth, Ctl* ctl) {
  __shared__ uint64_t s[kSmallSort];
  int P = 1;
  while (P < k) P <<= 1;
  for (int i = threadIdx.x; i < P; i += blockDim.x) s[i] = (i < k) ? w[i] : 0ull;
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
    write_out(s[i], i, k, dtype, out_keys, out_idx, out_kth, ctl);
}

struct SortParams {
  uint64_t* buf[2];
  uint64_t* status;  // [8][ntiles][256] look-back words (flag << 32 | count)
  int64_t k;
  int64_t ntiles;
  Ctl* ctl;
};

// pass p: digit p (0 = least significant byte) of ~c
__device__ __forceinline__ uint32_t sdigit(uint64_t c, int pass) {
  return static_cast<uint32_t>((~c) >> (8 * pass)) & 255u;
}

__global__ void __launch_bounds__(kSortThreads) sort_hist_all_kernel(SortParams p) {
  __shared__ uint32_t sh[8][256];
  for (int i = threadIdx.x; i < 8 * 256; i += kSortThreads) (&sh[0][0])[i] = 0;
  __syncthreads();
  const uint64_t* src = p.buf[0];
  for (int64_t i = int64_t(blockIdx.x) * kSortThreads + threadIdx.x; i < p.k;
       i += int64_t(gridDim.x) * kSortThreads) {
    const uint64_t c = src[i];
#pragma unroll
    for (int q = 0; q < 8; ++q) atomicAdd(&sh[q][sdigit(c, q)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 8 * 256; i += kSortThreads) {
    const uint32_t v = (&sh[0][0])[i];
    if (v) atomicAdd(&(&p.ctl->sort_hist[0][0])[i], v);
  }
  if (last_block(&p.ctl->sort_ticket)) {
    if (threadIdx.x < 8) {
      // exclusive offsets per digit; a digit that holds all k entries is skipped
      uint32_t* h = p.ctl->sort_hist[threadIdx.x];
      uint32_t run = 0, skip = 0;
      for (int d = 0; d < 256; ++d) {
        const uint32_t v = __ldcg(&h[d]);
        if (v == static_cast<uint32_t>(p.k)) skip = 1;
        h[d] = run;
        run += v;
      }
      p.ctl->sort_skip[threadIdx.x] = skip;
    }
  }
}

__global__ void __launch_bounds__(kSortThreads) sort_pass_kernel(SortParams p, int pass) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->sort_skip[pass])) return;
  uint32_t par = 0;
  for (int q = 0; q < pass; ++q) par ^= (__ldcg(&ctl->sort_skip[q]) == 0);
  const uint64_t* src = p.buf[par];
  uint64_t* dst = p.buf[par ^ 1u];

  __shared__ uint32_t s_tile;
  __shared__ uint32_t base[256];
  __shared__ uint32_t wcnt[kSortThreads / 32][256];
  __shared__ uint32_t s_off[256];
  if (threadIdx.x == 0) s_tile = atomicAdd(&ctl->sort_tiles[pass], 1u);
  for (int d = threadIdx.x; d < 256; d += kSortThreads) base[d] = 0;
  __syncthreads();
  const int64_t tile = s_tile;
  const int warp = threadIdx.x >> 5;
  const int64_t t0 = tile * kTile;

  uint64_t c[kItems];
  uint32_t rank[kItems];
  // stable ranking inside the tile: element order = (round, warp, lane)
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    for (int q = threadIdx.x; q < (kSortThreads / 32) * 256; q += kSortThreads)
      (&wcnt[0][0])[q] = 0;
    __syncthreads();
    const int64_t i = t0 + r * kSortThreads + threadIdx.x;
    const bool act = i < p.k;
    uint32_t d = 0, rk = 0;
    const uint32_t am = __ballot_sync(0xFFFFFFFFu, act);
    c[r] = 0;
    if (act) {
      c[r] = src[i];
      d = sdigit(c[r], pass);
      const uint32_t peers = __match_any_sync(am, d);
      rk = __popc(peers & lanemask_lt_s());
      if (rk == 0) wcnt[warp][d] = __popc(peers);
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < 256; dd += kSortThreads) {
      uint32_t run = base[dd];
      for (int q = 0; q < kSortThreads / 32; ++q) {
        const uint32_t v = wcnt[q][dd];
        wcnt[q][dd] = run;
        run += v;
      }
      base[dd] = run;
    }
    __syncthreads();
    rank[r] = act ? wcnt[warp][d] + rk : 0u;
    __syncthreads();  // wcnt is cleared again by the next round
  }

  // decoupled look-back: thread d publishes this tile's count of digit d and
  // adds the earlier tiles' counts
  {
    const int d = threadIdx.x;  // 256 threads = 256 digits
    uint64_t* st = p.status + (int64_t(pass) * p.ntiles) * 256;
    const uint32_t cnt = base[d];
    uint32_t excl = 0;
    if (tile == 0) {
      st_relaxed(&st[d], kFlagIncl | cnt);
    } else {
      st_relaxed(&st[tile * 256 + d], kFlagAgg | cnt);
      int64_t t = tile - 1;
      uint32_t spins = 0;
      while (t >= 0) {
        const uint64_t v = ld_relaxed(&st[t * 256 + d]);
        const uint64_t f = v & ~uint64_t(0xFFFFFFFFu);
        if (f == 0) {
          if (++spins > kLookbackSpin) {
            atomicOr(&ctl->error, kErrTimeout);
            break;
          }
          continue;
        }
        excl += static_cast<uint32_t>(v);
        if (f == kFlagIncl) break;
        --t;
      }
      st_relaxed(&st[tile * 256 + d], kFlagIncl | (excl + cnt));
    }
    s_off[d] = __ldcg(&ctl->sort_hist[pass][d]) + excl;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = t0 + r * kSortThreads + threadIdx.x;
    if (i < p.k) dst[s_off[sdigit(c[r], pass)] + rank[r]] = c[r];
  }
}

__global__ void finalize_kernel(SortParams p, int dtype, uint32_t* out_keys, int32_t* out_idx,
                                uint32_t* out_kth) {
  uint32_t par = 0;
  for (int q = 0; q < 8; ++q) par ^= (__ldcg(&p.ctl->sort_skip[q]) == 0);
  const uint64_t* src = p.buf[par];
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < p.k;
       j += int64_t(gridDim.x) * blockDim.x)
    write_out(src[j], j, p.k, dtype, out_keys, out_idx, out_kth, p.ctl);
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
                                         static_cast<uint32_t*>(out_kth), w.ctl);
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
  cudaError_t e = cudaMemsetAsync(p.status, 0, sort_status_words(w.k) * 8, s);
  if (e != cudaSuccess) return e;
  const int gh = static_cast<int>(std::min<int64_t>(p.ntiles, int64_t(sms) * 4));
  sort_hist_all_kernel<<<gh, kSortThreads, 0, s>>>(p);
  for (int pass = 0; pass < 8; ++pass)
    sort_pass_kernel<<<static_cast<unsigned>(p.ntiles), kSortThreads, 0, s>>>(p, pass);
  const int g = static_cast<int>(std::min<int64_t>((w.k + 255) / 256, int64_t(sms) * 8));
  finalize_kernel<<<g, 256, 0, s>>>(p, w.dtype, static_cast<uint32_t*>(out_keys), out_idx,
                                    static_cast<uint32_t*>(out_kth));
  note_launch(10);
  return cudaGetLastError();
}

}  // namespace drtopk
