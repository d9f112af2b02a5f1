// Delegate pass: the one step that streams all n keys (Sec. 3.1 Rule 1,
// Sec. 3.3 Rule 3, Sec. 4.1 delegate vector construction, Sec. 4.3).
//
// For each subrange S_i of 2^alpha consecutive keys it writes the beta
// largest keys m_i^0 >= ... >= m_i^{beta-1} (order-mapped) and, for each, the
// 32-key segment of S_i it came from. Among equal keys the smaller index
// wins: within a segment the j-th equal delegate is the j-th occurrence,
// and across segments the smaller segment wins. Exact positions are
// recovered from (key, segment, occurrence) only for the few delegates that
// are ever emitted.
//
// GB300 design (replaces the paper's warp-per-subrange shuffles and its
// shared-memory transposition for small subranges):
//   * persistent grid, 2 CTAs of 256 threads per SM;
//   * each CTA streams 32 KB chunks (8192 keys) with cp.async.bulk (TMA,
//     1-D) into a 3-stage shared-memory ring completed on mbarriers, with an
//     L2 evict-first hint (the keys are read once);
//   * thread t owns keys [32t, 32t+32) of a chunk and reads them as eight
//     16-byte words in a rotated order (conflict-free banks); its top-beta
//     is kept by value only (2*beta-1 integer min/max per key);
//   * per-thread lists of (key, segment) composites are merged with
//     bitonic merges over warp shuffles, then across warps in shared memory;
//   * the histogram of the delegates' top 8 bits (first digit of the
//     threshold select) is fused into the epilogue.
#include "common.cuh"
#include "delegate_core.cuh"
#include "launch.h"

namespace drtopk {
namespace {

constexpr int kThreads = 256;
constexpr int kChunkKeys = 8192;
constexpr int kKPT = 32;  // keys per thread per chunk
constexpr int kStages = 3;
constexpr int kChunkBytes = kChunkKeys * 4;
constexpr int kWarps = kThreads / 32;

struct DelegParams {
  const uint32_t* keys;
  int64_t n;
  int64_t S;
  int alpha;
  int64_t nchunks;
  uint32_t* dkeys;
  uint16_t* dsegs;
  Ctl* ctl;
  int fuse_hist;
  int select_last;  // the launch's last block resolves the first threshold digit
  uint32_t k;
};

template <int B>
__device__ __forceinline__ void write_delegates(const DelegParams& p, int64_t sub,
                                                const uint64_t* c, uint32_t* sh_hist,
                                                uint32_t& kmax) {
  // c: descending composites (B entries); kmax: running maximum key
  kmax = max(kmax, dc_key(c[0]));
#pragma unroll
  for (int j = 0; j < B; ++j) {
    const uint32_t key = dc_key(c[j]);
    const uint32_t seg = (c[j] == 0) ? kNoSeg : dc_seg(c[j]);
    p.dkeys[sub * B + j] = key;
    p.dsegs[sub * B + j] = static_cast<uint16_t>(seg);
    if (p.fuse_hist) atomicAdd(&sh_hist[key >> 24], 1u);
  }
}

// Block-sequence of chunks: the j-th chunk this block processes, or -1.
__device__ __forceinline__ int64_t chunk_of(const DelegParams& p, int64_t j, int cps_log) {
  const int64_t G = gridDim.x;
  if (cps_log == 0) {
    const int64_t c = blockIdx.x + j * G;
    return c < p.nchunks ? c : -1;
  }
  const int64_t sub = blockIdx.x + (j >> cps_log) * G;
  if (sub >= p.S) return -1;
  const int64_t c = (sub << cps_log) + (j & ((int64_t(1) << cps_log) - 1));
  return c < p.nchunks ? c : -1;
}

template <bool TMA>
__device__ __forceinline__ void issue_chunk(const DelegParams& p, int64_t c, uint32_t* dst,
                                            uint64_t* bar, uint64_t pol) {
  // thread 0 only (TMA) ; all threads (plain)
  const int64_t start = c * kChunkKeys;
  const int64_t cnt = imin64(kChunkKeys, p.n - start);
  if constexpr (TMA) {
    const uint32_t bytes = static_cast<uint32_t>(cnt) * 4u;
    const uint32_t bulk = bytes & ~15u;
    const uint32_t tail_from = bulk / 4u;
    for (uint32_t t = tail_from; t < static_cast<uint32_t>(cnt); ++t) dst[t] = p.keys[start + t];
    if (bulk) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bar, bulk);
      tma_load_1d(dst, p.keys + start, bulk, bar, pol);
    } else {
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
    }
  } else {
    for (int i = threadIdx.x; i < cnt; i += kThreads) dst[i] = __ldg(p.keys + start + i);
  }
}

template <int DT, int B, bool TMA>
__global__ void __launch_bounds__(kThreads, 2) delegate_kernel(DelegParams p) {
  constexpr int P = Pow2<B>::v;
  extern __shared__ __align__(128) uint32_t smem[];
  uint32_t* buf = smem;  // kStages * kChunkKeys
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ uint32_t sh_hist[256];
  __shared__ uint64_t sh_lists[kWarps][P];

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int alpha = p.alpha;
  const int cps_log = alpha > 13 ? alpha - 13 : 0;  // chunks per subrange (log2)

  for (int i = tid; i < 256; i += kThreads) sh_hist[i] = 0;
  uint64_t pol = 0;
  if constexpr (TMA) {
    if (tid == 0) {
      for (int s = 0; s < kStages; ++s) mbar_init(&full_bar[s], 1);
      fence_mbar_init();
    }
    pol = l2_evict_first_policy();
  }
  __syncthreads();

  if constexpr (TMA) {
    if (tid == 0) {
      for (int s = 0; s < kStages; ++s) {
        const int64_t c = chunk_of(p, s, cps_log);
        if (c < 0) break;
        issue_chunk<true>(p, c, buf + s * kChunkKeys, &full_bar[s], pol);
      }
    }
  }

  uint32_t kmax = 0;  // largest delegate key this thread wrote
  // running list across chunks (alpha > 13)
  uint64_t run[P];
#pragma unroll
  for (int i = 0; i < P; ++i) run[i] = 0;

  for (int64_t j = 0;; ++j) {
    const int64_t c = chunk_of(p, j, cps_log);
    if (c < 0) break;
    const int stage = static_cast<int>(j % kStages);
    uint32_t* cb = buf + stage * kChunkKeys;
    bool ok = true;
    if constexpr (TMA) {
      ok = mbar_wait_bounded(&full_bar[stage], static_cast<uint32_t>((j / kStages) & 1));
    } else {
      issue_chunk<false>(p, c, cb, nullptr, 0);
    }
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(&p.ctl->error, kErrTimeout);
        if constexpr (TMA) {
          // copies still in flight land in this CTA's shared memory: let
          // them complete (bounded) before the CTA exits
          for (int64_t jj = j; jj < j + kStages && chunk_of(p, jj, cps_log) >= 0; ++jj)
            mbar_wait_bounded(&full_bar[jj % kStages], static_cast<uint32_t>((jj / kStages) & 1));
        }
      }
      return;
    }

    const int64_t cstart = c * kChunkKeys;
    const int64_t seg_start = cstart + tid * kKPT;
    const int64_t valid = p.n - seg_start;  // keys of this thread's segment present
    const bool full = valid >= kKPT;
    const uint4* sv = reinterpret_cast<const uint4*>(cb + tid * kKPT);
    const int rot = tid & 7;

    if (alpha < 5) {
      // each thread owns 32 / 2^alpha whole subranges; segment = subrange
      const int sub_keys = 1 << alpha;
      const int words = sub_keys >> 2;  // 16-byte words per subrange
      const int nsub = kKPT >> alpha;
      for (int s0 = 0; s0 < nsub; ++s0) {
        const int s = (s0 + rot) & (nsub - 1);
        const int64_t sub = (seg_start >> alpha) + s;
        if (sub >= p.S) continue;
        uint32_t m[B];
#pragma unroll
        for (int i = 0; i < B; ++i) m[i] = 0;
        int r = 0;
        if (full) {
          for (int w = 0; w < words; ++w) insert4<DT, B>(m, sv[s * words + w]);
          r = sub_keys;
        } else {
          const int64_t lo = s * sub_keys;
          for (int e = 0; e < sub_keys; ++e) {
            if (lo + e < valid) {
              insert_val<B>(m, map_key<DT>(cb[tid * kKPT + lo + e]));
              ++r;
            }
          }
        }
        uint64_t cc[B];
#pragma unroll
        for (int i = 0; i < B; ++i) cc[i] = (i < r) ? make_dc(m[i], 0) : 0;
        write_delegates<B>(p, sub, cc, sh_hist, kmax);
      }
    } else {
      // value-only top-B of the thread's 32-key segment
      uint32_t m[B];
#pragma unroll
      for (int i = 0; i < B; ++i) m[i] = 0;
      int r;
      if (full) {
#pragma unroll
        for (int w = 0; w < 8; ++w) insert4<DT, B>(m, sv[(w + rot) & 7]);
        r = kKPT;
      } else {
        r = 0;
        for (int e = 0; e < kKPT; ++e) {
          if (e < valid) {
            insert_val<B>(m, map_key<DT>(cb[tid * kKPT + e]));
            ++r;
          }
        }
      }
      // segment index of this thread inside its subrange
      const int64_t sub = seg_start >> alpha;
      const uint32_t seg = static_cast<uint32_t>((seg_start - (sub << alpha)) >> 5);
      uint64_t a[P];
#pragma unroll
      for (int i = 0; i < P; ++i) a[i] = (i < B && i < r) ? make_dc(m[i < B ? i : 0], seg) : 0;

      if (alpha <= 13) {
        const int g_log = alpha - 5;  // log2 threads per subrange
        const int wl = g_log < 5 ? g_log : 5;
        for (int l = 0; l < wl; ++l) shfl_merge<P>(a, 1 << l);
        if (g_log <= 5) {
          if ((lane & ((1 << g_log) - 1)) == 0 && sub < p.S) write_delegates<B>(p, sub, a, sh_hist, kmax);
        } else {
          // 2^(g_log-5) warps per subrange: merge their lists in shared memory
          if (lane == 0) {
#pragma unroll
            for (int i = 0; i < P; ++i) sh_lists[warp][i] = a[i];
          }
          __syncthreads();
          const int wps_log = g_log - 5;           // warps per subrange (log2)
          const int nsub_chunk = kWarps >> wps_log;  // subranges in this chunk
          if (warp < nsub_chunk) {
            uint64_t b[P];
            const int src = warp * (1 << wps_log) + (lane & ((1 << wps_log) - 1));
#pragma unroll
            for (int i = 0; i < P; ++i) b[i] = sh_lists[src][i];
            for (int l = 0; l < wps_log; ++l) shfl_merge<P>(b, 1 << l);
            const int64_t sub2 = (cstart >> alpha) + warp;
            if (lane == 0 && sub2 < p.S) write_delegates<B>(p, sub2, b, sh_hist, kmax);
          }
        }
      } else {
        // subrange spans several chunks: accumulate, merge at its last chunk
        merge_desc<P>(run, a);
        const int64_t cps = int64_t(1) << cps_log;
        const bool last_of_sub = ((c & (cps - 1)) == cps - 1) || (c == p.nchunks - 1);
        if (last_of_sub) {
          for (int l = 0; l < 5; ++l) shfl_merge<P>(run, 1 << l);
          if (lane == 0) {
#pragma unroll
            for (int i = 0; i < P; ++i) sh_lists[warp][i] = run[i];
          }
          __syncthreads();
          if (warp == 0) {
            uint64_t b[P];
#pragma unroll
            for (int i = 0; i < P; ++i) b[i] = sh_lists[lane & 7][i];
            for (int l = 0; l < 3; ++l) shfl_merge<P>(b, 1 << l);
            if (lane == 0) write_delegates<B>(p, c >> cps_log, b, sh_hist, kmax);
          }
#pragma unroll
          for (int i = 0; i < P; ++i) run[i] = 0;
        }
      }
    }
    __syncthreads();  // stage fully consumed
    if constexpr (TMA) {
      if (tid == 0) {
        const int64_t cn = chunk_of(p, j + kStages, cps_log);
        if (cn >= 0) issue_chunk<true>(p, cn, cb, &full_bar[stage], pol);
      }
    }
  }

  {
    // the largest key of V is the largest delegate
    const uint32_t wm = __reduce_max_sync(0xFFFFFFFFu, kmax);
    if (lane == 0 && wm) atomicMax(&p.ctl->key_max, wm);
  }
  if (p.fuse_hist) {
    __syncthreads();
    for (int i = tid; i < 256; i += kThreads) {
      const uint32_t v = sh_hist[i];
      if (v) atomicAdd(&p.ctl->dsel.hist[0][i], v);
    }
    if (p.select_last && last_block(&p.ctl->dsel.ticket[0])) {
      if (warp == 0) {
        if (lane == 0) p.ctl->dsel.k_rem = p.k;
        __syncwarp();
        select_digit<4>(&p.ctl->dsel, 0, 32, false);
      }
    }
  }
}

template <int DT, int B>
cudaError_t launch_deleg_t(const DelegParams& p, bool tma, int sms, cudaStream_t s) {
  const size_t smem = static_cast<size_t>(kStages) * kChunkBytes;
  int64_t units = (p.alpha > 13) ? p.S : p.nchunks;
  int64_t grid = std::min<int64_t>(units, static_cast<int64_t>(sms) * 2);
  if (grid < 1) grid = 1;
  if (tma) {
    auto k = delegate_kernel<DT, B, true>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    k<<<static_cast<unsigned>(grid), kThreads, smem, s>>>(p);
  } else {
    auto k = delegate_kernel<DT, B, false>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    k<<<static_cast<unsigned>(grid), kThreads, smem, s>>>(p);
  }
  return cudaGetLastError();
}

template <int DT>
cudaError_t launch_deleg_b(const DelegParams& p, int beta, bool tma, int sms, cudaStream_t s) {
  switch (beta) {
    case 1: return launch_deleg_t<DT, 1>(p, tma, sms, s);
    case 2: return launch_deleg_t<DT, 2>(p, tma, sms, s);
    case 3: return launch_deleg_t<DT, 3>(p, tma, sms, s);
    case 4: return launch_deleg_t<DT, 4>(p, tma, sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_delegates(const Work& w, const void* keys, bool fuse_hist, int sms,
                             cudaStream_t s) {
  return launch_delegates_range(w, keys, 0, w.S, fuse_hist, true, sms, s);
}

cudaError_t launch_delegates_range(const Work& w, const void* keys, int64_t sub0, int64_t sub1,
                                   bool fuse_hist, bool select_last, int sms, cudaStream_t s) {
  // subranges [sub0, sub1) as an array of their own: keys and delegate
  // slots offset by whole subranges (positions inside a subrange and the
  // segments stored with the delegates do not change)
  DelegParams p;
  const int64_t k0 = sub0 << w.alpha;
  p.keys = static_cast<const uint32_t*>(keys) + k0;
  p.n = imin64(w.n, sub1 << w.alpha) - k0;
  p.S = sub1 - sub0;
  p.alpha = w.alpha;
  p.nchunks = (p.n + kChunkKeys - 1) / kChunkKeys;
  p.dkeys = w.dkeys + sub0 * w.beta;
  p.dsegs = w.dsegs + sub0 * w.beta;
  p.ctl = w.ctl;
  p.fuse_hist = fuse_hist ? 1 : 0;
  p.select_last = select_last ? 1 : 0;
  p.k = static_cast<uint32_t>(w.k);
  if (p.n <= 0 || p.S <= 0) return cudaErrorInvalidValue;
  const bool tma = (reinterpret_cast<uintptr_t>(p.keys) & 15u) == 0;
  note_launch();
  switch (w.dtype) {
    case DRTOPK_U32: return launch_deleg_b<DRTOPK_U32>(p, w.beta, tma, sms, s);
    case DRTOPK_I32: return launch_deleg_b<DRTOPK_I32>(p, w.beta, tma, sms, s);
    case DRTOPK_F32: return launch_deleg_b<DRTOPK_F32>(p, w.beta, tma, sms, s);
    case DRTOPK_U32 | kSmallest: return launch_deleg_b<DRTOPK_U32 | kSmallest>(p, w.beta, tma, sms, s);
    case DRTOPK_I32 | kSmallest: return launch_deleg_b<DRTOPK_I32 | kSmallest>(p, w.beta, tma, sms, s);
    case DRTOPK_F32 | kSmallest: return launch_deleg_b<DRTOPK_F32 | kSmallest>(p, w.beta, tma, sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace drtopk
