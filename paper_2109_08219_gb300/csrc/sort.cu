// Output ordering: the k winners W (unique (key, ~idx) composites) are
// sorted descending, i.e. by key descending then index ascending (the
// output order of top-k; the paper leaves it unstated), and written as the
// input dtype's key bits plus int32 indices.
//   * k <= 4096: one CTA bitonic-sorts W in shared memory;
//   * larger k: a stable LSD radix sort with 8-bit digits over the
//     complemented composites (ascending), 3 kernels per digit; a digit that
//     is the same for all k entries is skipped on the device.
#include "common.cuh"
#include "launch.h"

namespace drtopk {
namespace {

constexpr int kSmallSort = 4096;
constexpr int kSortThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kSortThreads * kItems;  // 4096

__device__ __forceinline__ uint32_t lanemask_lt_s() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
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
  uint32_t* hist;  // [256][nblk] digit-major counts, then [2] flags per pass
  int64_t k;
  int64_t nblk;
  Ctl* ctl;
};

// pass p: digit p (0 = least significant byte) of ~c
__device__ __forceinline__ uint32_t sdigit(uint64_t c, int pass) {
  return static_cast<uint32_t>((~c) >> (8 * pass)) & 255u;
}

__global__ void __launch_bounds__(kSortThreads) sort_hist_kernel(SortParams p, int pass) {
  __shared__ uint32_t sh[256];
  for (int i = threadIdx.x; i < 256; i += kSortThreads) sh[i] = 0;
  __syncthreads();
  const uint64_t* src = p.buf[__ldcg(&p.ctl->sort_cur) & 1];
  const int64_t t0 = int64_t(blockIdx.x) * kTile;
  for (int r = 0; r < kItems; ++r) {
    const int64_t i = t0 + r * kSortThreads + threadIdx.x;
    if (i < p.k) atomicAdd(&sh[sdigit(src[i], pass)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += kSortThreads) p.hist[int64_t(d) * p.nblk + blockIdx.x] = sh[d];
}

// Exclusive scan over the digit-major counts; flags[pass] = 1 when one digit
// holds every entry (the pass is skipped).
__global__ void __launch_bounds__(1024) sort_scan_kernel(SortParams p, int pass) {
  __shared__ uint32_t part[1024];
  __shared__ uint32_t s_skip;
  const int64_t total = 256 * p.nblk;
  const int64_t per = (total + 1023) / 1024;
  const int64_t lo = threadIdx.x * per;
  const int64_t hi = imin64(total, lo + per);
  uint32_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += p.hist[i];
  part[threadIdx.x] = s;
  if (threadIdx.x == 0) s_skip = 0;
  __syncthreads();
  // a digit holds everything iff its nblk counts sum to k
  if (threadIdx.x < 256) {
    uint64_t ds = 0;
    for (int64_t b = 0; b < p.nblk; ++b) ds += p.hist[int64_t(threadIdx.x) * p.nblk + b];
    if (ds == static_cast<uint64_t>(p.k)) s_skip = 1;
  }
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t v = threadIdx.x >= static_cast<unsigned>(o) ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - s;
  for (int64_t i = lo; i < hi; ++i) {
    const uint32_t v = p.hist[i];
    p.hist[i] = run;
    run += v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t cur = p.ctl->sort_cur & 1;
    p.hist[total + 2 * pass] = s_skip;
    p.hist[total + 2 * pass + 1] = cur;  // source buffer of this pass
    if (!s_skip) p.ctl->sort_cur = cur ^ 1u;
  }
}

__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(SortParams p, int pass) {
  const int64_t total = 256 * p.nblk;
  if (__ldcg(&p.hist[total + 2 * pass]) != 0) return;
  const uint32_t cur = __ldcg(&p.hist[total + 2 * pass + 1]);
  const uint64_t* src = p.buf[cur];
  uint64_t* dst = p.buf[cur ^ 1u];
  __shared__ uint32_t base[256];
  __shared__ uint32_t wcnt[kSortThreads / 32][256];
  const int warp = threadIdx.x >> 5;
  const uint32_t lane = threadIdx.x & 31u;
  for (int d = threadIdx.x; d < 256; d += kSortThreads) base[d] = p.hist[int64_t(d) * p.nblk + blockIdx.x];
  const int64_t t0 = int64_t(blockIdx.x) * kTile;
  for (int r = 0; r < kItems; ++r) {
    for (int q = threadIdx.x; q < (kSortThreads / 32) * 256; q += kSortThreads)
      (&wcnt[0][0])[q] = 0;
    __syncthreads();
    const int64_t i = t0 + r * kSortThreads + threadIdx.x;
    const bool act = i < p.k;
    uint64_t c = 0;
    uint32_t d = 0, rank = 0;
    const uint32_t am = __ballot_sync(0xFFFFFFFFu, act);
    if (act) {
      c = src[i];
      d = sdigit(c, pass);
      const uint32_t peers = __match_any_sync(am, d);
      rank = __popc(peers & lanemask_lt_s());
      if (rank == 0) wcnt[warp][d] = __popc(peers);
    }
    __syncthreads();
    // per digit: offsets of the warps in order, then advance the base
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
    if (act) dst[wcnt[warp][d] + rank] = c;
    __syncthreads();
  }
}

__global__ void finalize_kernel(SortParams p, int dtype, uint32_t* out_keys, int32_t* out_idx,
                                uint32_t* out_kth) {
  const uint64_t* src = p.buf[__ldcg(&p.ctl->sort_cur) & 1];
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < p.k;
       j += int64_t(gridDim.x) * blockDim.x)
    write_out(src[j], j, p.k, dtype, out_keys, out_idx, out_kth, p.ctl);
}

}  // namespace

size_t sort_hist_words(int64_t k) {
  if (k <= kSmallSort) return 0;
  const int64_t nblk = (k + kTile - 1) / kTile;
  return static_cast<size_t>(256 * nblk + 16);
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
  p.hist = w.sort_hist;
  p.k = w.k;
  p.nblk = (w.k + kTile - 1) / kTile;
  p.ctl = w.ctl;
  const int nb = static_cast<int>(p.nblk);
  for (int pass = 0; pass < 8; ++pass) {
    sort_hist_kernel<<<nb, kSortThreads, 0, s>>>(p, pass);
    sort_scan_kernel<<<1, 1024, 0, s>>>(p, pass);
    sort_scatter_kernel<<<nb, kSortThreads, 0, s>>>(p, pass);
  }
  int g = static_cast<int>(std::min<int64_t>((w.k + 255) / 256, int64_t(sms) * 8));
  finalize_kernel<<<g, 256, 0, s>>>(p, w.dtype, static_cast<uint32_t*>(out_keys), out_idx,
                                    static_cast<uint32_t*>(out_kth));
  note_launch(25);
  return cudaGetLastError();
}

}  // namespace drtopk
