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
//   * persistent grid, 3 CTAs of 256 threads per SM;
//   * each CTA streams 32 KB chunks (8192 keys) with cp.async.bulk (TMA,
//     1-D) into a 2-stage shared-memory ring completed on mbarriers, with an
//     L2 evict-first hint (the keys are read once);
//   * thread t owns keys [32t, 32t+32) of a chunk and reads them as eight
//     16-byte words in a rotated order (conflict-free banks); its top-beta
//     is kept by value only (2*beta-1 integer min/max per key);
//   * per-thread lists of (key, segment) composites are merged with
//     bitonic merges over warp shuffles, then across warps in shared memory;
//   * the histogram of the delegates' top 8 bits (first digit of the
//     threshold select) is fused into the epilogue.
// For alpha in [5, 10] on large arrays the same kernel also runs as the
// passes of the speculative compaction (Ctl::spec_on): a sample pass over
// every 128th chunk that sets a bound t_lo below the expected tau, a records
// pass that stores only the subranges whose largest delegate reaches t_lo,
// and a fallback pass (the full pass behind a device-side condition) that
// writes the full arrays when the records cannot stand in for them.
#include "common.cuh"
#include "delegate_core.cuh"
#include "launch.h"

namespace drtopk {
namespace {

constexpr int kThreads = 256;
constexpr int kChunkKeys = 8192;
constexpr int kKPT = 32;  // keys per thread per chunk
constexpr int kStages = 2;
constexpr int kCtasPerSm = 3;  // 3 x (2 x 32 KB ring + static) per SM
constexpr int kChunkBytes = kChunkKeys * 4;
constexpr int kWarps = kThreads / 32;

// Passes of the delegate kernel (the speculative compaction is described
// with Ctl::spec_on).
constexpr int kPassFull = 0;    // store every subrange's delegates
constexpr int kPassSample = 1;  // histogram the delegates of every kSampStride-th chunk
constexpr int kPassSpec = 2;    // store records of subranges reaching t_lo (nothing when declined)
constexpr int kPassFallback = 3;  // store every subrange's delegates when p.only_if holds
constexpr int kSampStride = 128;
constexpr int kSampBins = 2048;  // top 11 bits
constexpr int kRecStage = 320;   // records staged per CTA (three CTAs per SM must fit)

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
  int only_if;      // fallback pass: 1 when Ctl::need_full; 2 when the
                    // records stand in and the query is in tie mode
  int64_t d_total;  // delegate slots of the whole array (sample decision)
  uint32_t* rec_keys;
  uint16_t* rec_segs;
  uint32_t* rec_sub;
  int64_t rec_cap;
};

template <int B>
__device__ __forceinline__ void write_delegates(const DelegParams& p, int64_t sub,
                                                const uint64_t* c, uint32_t* sh_hist,
                                                uint32_t& kmax, bool fuse) {
  // c: descending composites (B entries); kmax: running maximum key
  kmax = max(kmax, dc_key(c[0]));
#pragma unroll
  for (int j = 0; j < B; ++j) {
    const uint32_t key = dc_key(c[j]);
    const uint32_t seg = (c[j] == 0) ? kNoSeg : dc_seg(c[j]);
    p.dkeys[sub * B + j] = key;
    p.dsegs[sub * B + j] = static_cast<uint16_t>(seg);
    if (fuse) atomicAdd(&sh_hist[key >> 24], 1u);
  }
}

// Histogram of a sampled subrange's delegates (top 11 bits).
template <int B>
__device__ __forceinline__ void sample_delegates(const uint64_t* c, uint32_t* sh_samp, uint32_t& cnt) {
#pragma unroll
  for (int j = 0; j < B; ++j) {
    if (c[j] != 0) {
      atomicAdd(&sh_samp[dc_key(c[j]) >> 21], 1u);
      ++cnt;
    }
  }
}

// Records pass: the histogram and the running maximum for every subrange;
// a record (subrange, delegates, segments) staged when its largest
// delegate reaches t_lo; `above` counts the delegates >= t_lo.
template <int B>
__device__ __forceinline__ void record_delegates(int64_t sub, const uint64_t* c,
                                                 uint32_t t_lo, uint32_t* sh_hist, uint32_t& kmax,
                                                 uint32_t* rs_cnt, uint32_t* rs_sub, uint32_t* rs_keys,
                                                 uint16_t* rs_segs, uint32_t& above) {
  kmax = max(kmax, dc_key(c[0]));
#pragma unroll
  for (int j = 0; j < B; ++j) atomicAdd(&sh_hist[dc_key(c[j]) >> 24], 1u);
  if (dc_key(c[0]) >= t_lo) {
    const uint32_t slot = atomicAdd(rs_cnt, 1u);
    rs_sub[slot] = static_cast<uint32_t>(sub);
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const uint32_t key = dc_key(c[j]);
      rs_keys[slot * B + j] = key;
      rs_segs[slot * B + j] = static_cast<uint16_t>((c[j] == 0) ? kNoSeg : dc_seg(c[j]));
      above += (c[j] != 0 && key >= t_lo) ? 1u : 0u;
    }
  }
}

// Stores the `nst` staged records (all threads; nst read by every thread
// after a block barrier, before this call) at one reserved range of the
// record arrays; past their capacity the overflow is flagged instead.
template <int B>
__device__ __forceinline__ void flush_records(const DelegParams& p, uint32_t nst, uint32_t* rs_base,
                                              uint32_t* rs_cnt, const uint32_t* rs_sub,
                                              const uint32_t* rs_keys, const uint16_t* rs_segs) {
  if (threadIdx.x == 0) *rs_base = atomicAdd(&p.ctl->rec_count, nst);
  __syncthreads();
  const uint64_t base = *rs_base;
  for (uint32_t i = threadIdx.x; i < nst; i += kThreads) {
    const uint64_t r = base + i;
    if (r < static_cast<uint64_t>(p.rec_cap)) {
      p.rec_sub[r] = rs_sub[i];
#pragma unroll
      for (int j = 0; j < B; ++j) {
        p.rec_keys[r * B + j] = rs_keys[i * B + j];
        p.rec_segs[r * B + j] = rs_segs[i * B + j];
      }
    }
  }
  if (threadIdx.x == 0) {
    if (base + nst > static_cast<uint64_t>(p.rec_cap)) p.ctl->rec_over = 1;
    *rs_cnt = 0;  // the next appends follow the next block barrier
  }
}

// Last block of the sample pass: t_lo = the start of the highest 11-bit
// bin whose count from the top reaches 1.5x the expected number of sampled
// delegates above tau (k scaled by the sampled share of the delegates),
// plus 8 standard deviations and 64; records are used when the delegates
// >= t_lo, scaled up, stay within 80 % of the record capacity.
__device__ void sample_decide(const DelegParams& p) {
  constexpr int per = kSampBins / kThreads;  // bins per thread, from the top
  __shared__ uint32_t s_acc;
  if (threadIdx.x == 0) s_acc = 0;
  uint32_t c[per];
  uint32_t sum = 0;
#pragma unroll
  for (int j = 0; j < per; ++j) {
    c[j] = __ldcg(&p.ctl->samp_hist[kSampBins - 1 - (threadIdx.x * per + j)]);
    sum += c[j];
  }
  const uint32_t excl = block_scan_excl<kThreads>(sum, nullptr);  // (synchronizes)
  const double sn = static_cast<double>(__ldcg(&p.ctl->samp_n));
  const double scale = static_cast<double>(p.d_total) / (sn > 0.0 ? sn : 1.0);
  const double target = static_cast<double>(p.k) / scale;
  const double need = 1.5 * target + 8.0 * sqrt(target) + 64.0;
  // too few sampled delegates: decline
  if (sn >= 4096.0 && static_cast<double>(excl) < need && static_cast<double>(excl) + sum >= need) {
    double acc = excl;
    int j = 0;
    for (; j < per - 1; ++j) {
      acc += c[j];
      if (acc >= need) break;
    }
    if (j == per - 1) acc = static_cast<double>(excl) + sum;
    const uint32_t bin = static_cast<uint32_t>(kSampBins - 1 - (threadIdx.x * per + j));
    const double est = acc * scale * 1.1;
    if (bin > 0 && est <= 0.8 * static_cast<double>(p.rec_cap)) {
      p.ctl->t_lo = bin << 21;
      p.ctl->spec_on = 1;
      s_acc = 1;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && !s_acc) {
    // declined: the fallback pass is the delegate pass of this query
    p.ctl->need_full = 1;
    p.ctl->need_hist = 1;
  }
}

// Block-sequence of chunks: the j-th chunk this block processes, or -1
// (always -1 for a fallback pass whose condition does not hold: the pass
// then ends without an early return, which keeps its code as the full
// pass's).
template <int MODE = kPassFull>
__device__ __forceinline__ int64_t chunk_of(const DelegParams& p, int64_t j, int cps_log,
                                            bool skip = false) {
  const int64_t G = gridDim.x;
  if constexpr (MODE == kPassFallback || MODE == kPassSpec) {
    if (skip) return -1;
  }
  if constexpr (MODE == kPassSample) {
    const int64_t c = (blockIdx.x + j * G) * kSampStride;
    return c < p.nchunks ? c : -1;
  }
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

template <int DT, int B, bool TMA, int MODE = kPassFull>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) delegate_kernel(DelegParams p) {
  constexpr int P = Pow2<B>::v;
  // a fallback pass runs only when its condition holds, a records pass
  // only when the sample accepted (uniform over the grid)
  bool skip = false;
  bool fuse = p.fuse_hist != 0, sel = p.select_last != 0;
  if constexpr (MODE == kPassFallback) {
    skip = (p.only_if == 1) ? !__ldcg(&p.ctl->need_full)
                            : !(__ldcg(&p.ctl->spec_on) && __ldcg(&p.ctl->mode) == kModeTies);
    if (!skip && blockIdx.x == 0 && threadIdx.x == 0) p.ctl->full_written = 1;
    // after a declined sample this is the query's delegate pass
    fuse = sel = !skip && p.only_if == 1 && __ldcg(&p.ctl->need_hist) != 0;
  }
  extern __shared__ __align__(128) uint32_t smem[];
  uint32_t* buf = smem;  // kStages * kChunkKeys
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ uint32_t sh_hist[256];
  __shared__ uint64_t sh_lists[kWarps][P];
  // sample pass: histogram; records pass: the staged records
  __shared__ uint32_t sh_samp[MODE == kPassSample ? kSampBins : 1];
  __shared__ uint32_t rs_sub[MODE == kPassSpec ? kRecStage : 1];
  __shared__ uint32_t rs_keys[MODE == kPassSpec ? kRecStage * B : 1];
  __shared__ uint16_t rs_segs[MODE == kPassSpec ? kRecStage * B : 1];
  __shared__ uint32_t rs_cnt, rs_base;
  uint32_t samp_cnt = 0, above = 0;
  bool spec = false;
  uint32_t t_lo = 0;
  if constexpr (MODE == kPassSpec) {
    spec = __ldcg(&p.ctl->spec_on) != 0;
    t_lo = __ldcg(&p.ctl->t_lo);
    skip = !spec;
    fuse = fuse && spec;
    sel = sel && spec;
  }

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int alpha = p.alpha;
  const int cps_log = alpha > 13 ? alpha - 13 : 0;  // chunks per subrange (log2)

  for (int i = tid; i < 256; i += kThreads) sh_hist[i] = 0;
  if constexpr (MODE == kPassSample)
    for (int i = tid; i < kSampBins; i += kThreads) sh_samp[i] = 0;
  if (MODE == kPassSpec && tid == 0) rs_cnt = 0;
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
        const int64_t c = chunk_of<MODE>(p, s, cps_log, skip);
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
    const int64_t c = chunk_of<MODE>(p, j, cps_log, skip);
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
          for (int64_t jj = j; jj < j + kStages && chunk_of<MODE>(p, jj, cps_log, skip) >= 0; ++jj)
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
        write_delegates<B>(p, sub, cc, sh_hist, kmax, fuse);
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
          if ((lane & ((1 << g_log) - 1)) == 0 && sub < p.S) {
            if constexpr (MODE == kPassSample) {
              sample_delegates<B>(a, sh_samp, samp_cnt);
            } else if constexpr (MODE == kPassSpec) {
              record_delegates<B>(sub, a, t_lo, sh_hist, kmax, &rs_cnt, rs_sub, rs_keys, rs_segs,
                                  above);
            } else {
              write_delegates<B>(p, sub, a, sh_hist, kmax, fuse);
            }
          }
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
            if (lane == 0 && sub2 < p.S) write_delegates<B>(p, sub2, b, sh_hist, kmax, fuse);
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
            if (lane == 0) write_delegates<B>(p, c >> cps_log, b, sh_hist, kmax, fuse);
          }
#pragma unroll
          for (int i = 0; i < P; ++i) run[i] = 0;
        }
      }
    }
    __syncthreads();  // stage fully consumed
    if constexpr (TMA) {
      if (tid == 0) {
        const int64_t cn = chunk_of<MODE>(p, j + kStages, cps_log, skip);
        if (cn >= 0) issue_chunk<true>(p, cn, cb, &full_bar[stage], pol);
      }
    }
    if constexpr (MODE == kPassSpec) {
      const uint32_t nst = rs_cnt;  // no append is in flight after the barrier
      // flush while the next chunk's subranges (8192 >> alpha) still fit
      if (nst > static_cast<uint32_t>(kRecStage - (kChunkKeys >> alpha)))
        flush_records<B>(p, nst, &rs_base, &rs_cnt, rs_sub, rs_keys, rs_segs);
    }
  }
  if constexpr (MODE == kPassSpec) {
    if (spec) {  // else the sample declined: the fallback pass does it all
      __syncthreads();
      const uint32_t nst = rs_cnt;
      if (nst) flush_records<B>(p, nst, &rs_base, &rs_cnt, rs_sub, rs_keys, rs_segs);
      const uint32_t wa = __reduce_add_sync(0xFFFFFFFFu, above);
      if (lane == 0 && wa) atomicAdd(&p.ctl->n_above, wa);
      if (tid == 0) p.ctl->spec_used = 1;
    }
  }
  if constexpr (MODE == kPassSample) {
    __syncthreads();
    for (int i = tid; i < kSampBins; i += kThreads) {
      const uint32_t v = sh_samp[i];
      if (v) atomicAdd(&p.ctl->samp_hist[i], v);
    }
    const uint32_t wc = __reduce_add_sync(0xFFFFFFFFu, samp_cnt);
    if (lane == 0 && wc) atomicAdd(&p.ctl->samp_n, wc);
    if (last_block(&p.ctl->samp_ticket)) sample_decide(p);
    return;
  }

  {
    // the largest key of V is the largest delegate
    const uint32_t wm = __reduce_max_sync(0xFFFFFFFFu, kmax);
    if (lane == 0 && wm) atomicMax(&p.ctl->key_max, wm);
  }
  if (fuse) {
    __syncthreads();
    for (int i = tid; i < 256; i += kThreads) {
      const uint32_t v = sh_hist[i];
      if (v) atomicAdd(&p.ctl->dsel.hist[0][i], v);
    }
    if (sel && last_block(&p.ctl->dsel.ticket[0])) {
      if (warp == 0) {
        if (lane == 0) p.ctl->dsel.k_rem = p.k;
        __syncwarp();
        select_digit<4>(&p.ctl->dsel, 0, 32, false);
      }
      if constexpr (MODE == kPassSpec) {
        // tau >= t_lo iff at least k delegates are >= t_lo: else, or when
        // the records overflowed, the full arrays are written next
        if (tid == 0 && __ldcg(&p.ctl->spec_on) &&
            (__ldcg(&p.ctl->n_above) < p.k || __ldcg(&p.ctl->rec_over))) {
          p.ctl->need_full = 1;
          p.ctl->spec_on = 0;
        }
      }
    }
  }
}

template <int DT, int B, int MODE>
cudaError_t launch_deleg_t(const DelegParams& p, bool tma, int sms, cudaStream_t s) {
  const size_t smem = static_cast<size_t>(kStages) * kChunkBytes;
  int64_t units = (p.alpha > 13) ? p.S : p.nchunks;
  if (MODE == kPassSample) units = (p.nchunks + kSampStride - 1) / kSampStride;
  int64_t grid = std::min<int64_t>(units, static_cast<int64_t>(sms) * kCtasPerSm);
  if (grid < 1) grid = 1;
  if (tma || MODE != kPassFull) {
    auto k = delegate_kernel<DT, B, true, MODE>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    k<<<static_cast<unsigned>(grid), kThreads, smem, s>>>(p);
  } else {
    auto k = delegate_kernel<DT, B, false, kPassFull>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    k<<<static_cast<unsigned>(grid), kThreads, smem, s>>>(p);
  }
  return cudaGetLastError();
}

template <int DT, int MODE>
cudaError_t launch_deleg_b(const DelegParams& p, int beta, bool tma, int sms, cudaStream_t s) {
  switch (beta) {
    case 1: return launch_deleg_t<DT, 1, MODE>(p, tma, sms, s);
    case 2: return launch_deleg_t<DT, 2, MODE>(p, tma, sms, s);
    case 3: return launch_deleg_t<DT, 3, MODE>(p, tma, sms, s);
    case 4: return launch_deleg_t<DT, 4, MODE>(p, tma, sms, s);
  }
  return cudaErrorInvalidValue;
}

template <int MODE>
cudaError_t launch_deleg_mode(const Work& w, const DelegParams& p, bool tma, int sms, cudaStream_t s) {
  note_launch();
  switch (w.dtype) {
    case DRTOPK_U32: return launch_deleg_b<DRTOPK_U32, MODE>(p, w.beta, tma, sms, s);
    case DRTOPK_I32: return launch_deleg_b<DRTOPK_I32, MODE>(p, w.beta, tma, sms, s);
    case DRTOPK_F32: return launch_deleg_b<DRTOPK_F32, MODE>(p, w.beta, tma, sms, s);
    case DRTOPK_U32 | kSmallest: return launch_deleg_b<DRTOPK_U32 | kSmallest, MODE>(p, w.beta, tma, sms, s);
    case DRTOPK_I32 | kSmallest: return launch_deleg_b<DRTOPK_I32 | kSmallest, MODE>(p, w.beta, tma, sms, s);
    case DRTOPK_F32 | kSmallest: return launch_deleg_b<DRTOPK_F32 | kSmallest, MODE>(p, w.beta, tma, sms, s);
  }
  return cudaErrorInvalidValue;
}

// Parameters of the pass over subranges [sub0, sub1) as an array of their
// own: keys and delegate slots offset by whole subranges (positions inside
// a subrange and the segments stored with the delegates do not change).
DelegParams deleg_params(const Work& w, const void* keys, int64_t sub0, int64_t sub1, bool fuse_hist,
                         bool select_last) {
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
  p.only_if = 0;
  p.d_total = w.S * w.beta;
  p.rec_keys = w.rec_keys;
  p.rec_segs = w.rec_segs;
  p.rec_sub = w.rec_sub;
  p.rec_cap = w.rec_cap;
  return p;
}

}  // namespace

bool spec_eligible(const Work& w, const void* keys) {
  return w.rec_cap > 0 && w.alpha >= 5 && w.alpha <= 10 && w.ablate == 0 &&
         (reinterpret_cast<uintptr_t>(keys) & 15u) == 0;
}

cudaError_t launch_delegates(const Work& w, const void* keys, bool fuse_hist, int sms,
                             cudaStream_t s) {
  return launch_delegates_range(w, keys, 0, w.S, fuse_hist, true, sms, s);
}

cudaError_t launch_delegates_range(const Work& w, const void* keys, int64_t sub0, int64_t sub1,
                                   bool fuse_hist, bool select_last, int sms, cudaStream_t s) {
  const DelegParams p = deleg_params(w, keys, sub0, sub1, fuse_hist, select_last);
  if (p.n <= 0 || p.S <= 0) return cudaErrorInvalidValue;
  const bool tma = (reinterpret_cast<uintptr_t>(p.keys) & 15u) == 0;
  return launch_deleg_mode<kPassFull>(w, p, tma, sms, s);
}

cudaError_t launch_delegates_spec(const Work& w, const void* keys, int sms, cudaStream_t s) {
  if (!spec_eligible(w, keys)) return launch_delegates(w, keys, true, sms, s);
  const DelegParams p = deleg_params(w, keys, 0, w.S, true, true);
  cudaError_t e = launch_deleg_mode<kPassSample>(w, p, true, sms, s);
  if (e == cudaSuccess) e = launch_deleg_mode<kPassSpec>(w, p, true, sms, s);
  if (e == cudaSuccess) e = launch_delegates_fallback(w, keys, 1, sms, s);
  return e;
}

cudaError_t launch_delegates_fallback(const Work& w, const void* keys, int cond, int sms,
                                      cudaStream_t s) {
  DelegParams p = deleg_params(w, keys, 0, w.S, false, false);
  p.only_if = cond;
  return launch_deleg_mode<kPassFallback>(w, p, true, sms, s);
}

}  // namespace drtopk
