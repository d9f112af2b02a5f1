// Shared device-side definitions of the drtopk CUDA library (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "drtopk.h"

namespace drtopk {

// ---------------------------------------------------------------- limits ---
constexpr int kMaxBeta = 4;
constexpr int kMinAlpha = 2;
constexpr int kMaxAlpha = 16;
// Bounded waits: an mbarrier wait gives up after kWaitNs nanoseconds of the
// GPU's global timer (a bulk copy lands in microseconds), a look-back wait
// after a bounded number of polls; either sets kErrTimeout in the control
// block instead of hanging.
constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s

// Device error flags (Ctl::error).
constexpr uint32_t kErrTimeout = 1u;
constexpr uint32_t kErrOverflowG = 2u;
constexpr uint32_t kErrOverflowW = 4u;
constexpr uint32_t kErrTieRank = 8u;

// Query modes decided on the device after the filter.
constexpr uint32_t kModeSelect = 0;  // |{x > tau}| >= k: select among them
constexpr uint32_t kModeTies = 1;    // |{x > tau}| < k: k-th key is tau

// ------------------------------------------------------------- key map -----
// Order-preserving map of a raw 32-bit key to u32 (unsigned order == key
// order). u32: identity. i32: flip the sign bit. f32: negative floats flip
// all bits, non-negative floats set the sign bit.
//
// Internal key types: the dtype (DRTOPK_U32 / I32 / F32) plus kSmallest for
// the smallest-k criterion (Sec. 1 and Sec. 2 name "largest or smallest"):
// the mapped key is complemented, so the k largest mapped keys are the k
// smallest keys, and the tie rule (smallest index first) is unchanged.
constexpr int kSmallest = 4;
__host__ __device__ constexpr int base_dtype(int dt) { return dt & 3; }

template <int DT>
__device__ __forceinline__ uint32_t map_key(uint32_t b) {
  constexpr int B = DT & 3;
  uint32_t m;
  if constexpr (B == DRTOPK_U32) {
    m = b;
  } else if constexpr (B == DRTOPK_I32) {
    m = b ^ 0x80000000u;
  } else {
    m = b ^ (static_cast<uint32_t>(static_cast<int32_t>(b) >> 31) | 0x80000000u);
  }
  if constexpr ((DT & kSmallest) != 0) m = ~m;
  return m;
}

__host__ __device__ __forceinline__ uint32_t unmap_key(int dt, uint32_t m) {
  if (dt & kSmallest) m = ~m;
  const int b = dt & 3;
  if (b == DRTOPK_U32) return m;
  if (b == DRTOPK_I32) return m ^ 0x80000000u;
  return (m & 0x80000000u) ? (m & 0x7FFFFFFFu) : ~m;
}

// Output composite: larger key first, then smaller index. Unique per element.
__device__ __forceinline__ uint64_t make_comp(uint32_t mkey, uint32_t idx) {
  return (static_cast<uint64_t>(mkey) << 32) | static_cast<uint32_t>(~idx);
}
__device__ __forceinline__ uint32_t comp_key(uint64_t c) { return static_cast<uint32_t>(c >> 32); }
__device__ __forceinline__ uint32_t comp_idx(uint64_t c) { return ~static_cast<uint32_t>(c); }

// Delegate composite used while merging per-thread lists: (key, segment)
// with the smaller segment first among equal keys. An empty slot is 0,
// which loses every tie against a real element (its ~seg is never 0).
constexpr uint32_t kNoSeg = 0xFFFFu;
__device__ __forceinline__ uint64_t make_dc(uint32_t key, uint32_t seg) {
  return (static_cast<uint64_t>(key) << 32) | static_cast<uint32_t>(0xFFFFu - seg);
}
__device__ __forceinline__ uint32_t dc_key(uint64_t c) { return static_cast<uint32_t>(c >> 32); }
__device__ __forceinline__ uint32_t dc_seg(uint64_t c) { return 0xFFFFu - static_cast<uint32_t>(c & 0xFFFFu); }

// ---------------------------------------------------- radix select state ---
// Most-significant-digit radix select with 8-bit digits (Sec. 4.1 uses
// radix top-k with 8-bit digits for both selections). hist[p] counts the
// digit p of the keys that still match the selected prefix; the last block
// of each pass picks the digit that holds the k_rem-th largest key.
template <int NPASS>
struct SelState {
  uint32_t hist[NPASS][256];
  uint32_t ticket[NPASS];
  uint32_t level;    // number of resolved digits
  uint32_t k_rem;    // rank (1-based, from the top) inside the current bucket
  uint32_t bucket;   // count of the current bucket
  uint32_t done;     // set once the bucket count equals k_rem (top-k mode)
  uint64_t prefix;   // resolved digits, most significant first, left-aligned
};

// Capacities of the direct tie path's lists (Ctl::ts, tc) and the largest
// set of scanned subranges it reads again.
constexpr uint32_t kTieSCap = 1024;
constexpr uint32_t kTieCandCap = 1024;
constexpr uint32_t kTieScanMax = 4096;

// Control block of one query, zeroed by the host before the first launch.
struct Ctl {
  SelState<4> dsel;  // threshold select over the delegate keys
  SelState<8> gsel;  // second select over (key, idx) composites
  uint32_t tau;      // threshold (mapped)
  uint32_t tau_ready;
  uint32_t mode;
  uint32_t need;     // ties at tau still needed (mode == kModeTies)
  uint32_t g_count;  // composites written to G
  uint32_t w_count;  // outputs written to W
  uint32_t error;
  uint32_t scanned;
  uint32_t tie_scanned;
  uint32_t filter_ticket;
  uint32_t kth_mapped;
  uint32_t ds_count;       // delegate keys surviving the first threshold digit
  uint32_t scanq_count;    // subranges queued for the filter scan
  uint32_t tie_ticket;     // next listed tile of the dense tie count
  uint32_t tie_cut_inv;    // ~(first listed tile not needed); 0: none yet
  uint32_t stage_count[10];  // survivors entering each second-select stage
  uint32_t ds_inplace;       // threshold passes 2-3 read the delegate keys in place
  uint32_t sort_ticket;
  uint32_t sort_tiles[8];    // dynamic tile ids of the output radix sort
  uint32_t sort_hist[8][256];  // digit counts of the output composites
  uint32_t sort_skip[8];
  uint32_t rq_count;         // delegates queued for position resolution
  uint32_t thr_lo_inv;       // ~(smallest delegate key in the first-digit bucket)
  uint32_t thr_hi;           // largest delegate key in the first-digit bucket
  uint32_t thr_done;         // tau found after digit 1 (the bucket holds one value)
  // speculative compaction of the delegate vector (large arrays, alpha in
  // [5, 10]): a sample of the chunks sets t_lo below the expected tau; the
  // delegate pass then stores only the records of subranges whose largest
  // delegate is >= t_lo, and the threshold and classification read those.
  // Exact: when fewer than k delegates are >= t_lo (tau < t_lo), the
  // records overflow, or the query ends in tie mode (the tie path reads
  // every subrange's delegates), the full delegate arrays are written by
  // another pass before they are needed.
  uint32_t spec_on;          // the records stand in for the delegate arrays
  uint32_t spec_used;        // the delegate pass stored records (statistics)
  uint32_t t_lo;
  uint32_t rec_count;        // records stored
  uint32_t rec_over;         // more records than their capacity
  uint32_t n_above;          // delegates >= t_lo
  uint32_t need_full;        // the full delegate arrays must be written
  uint32_t need_hist;        // ... and their first-digit histogram taken (the
                             // sample declined: the records pass did nothing)
  uint32_t full_written;     // a fallback pass wrote them (statistics)
  uint32_t samp_n;           // delegates of the sampled chunks
  uint32_t samp_ticket;
  uint32_t samp_hist[2048];  // sampled delegates by their top 11 bits
  uint32_t tie_nlist;        // tiles listed for the tie emission
  uint32_t tie_dense;        // the listed tiles are read whole (bulk copies)
  uint32_t g_total;          // |G| = |{x > tau}| at the mode decision
  uint32_t key_max;          // largest mapped key of V (from the delegate pass)
  uint32_t g_lvl0;           // first composite digit of G that can vary
  // two-pass filter scan of large scan sets: counting pass, then a cut key
  uint32_t two_pass;         // the scan set was counted first
  uint32_t scan_total;       // scanned keys > tau (counting pass)
  uint32_t g_all;            // |{x > tau}| when counted first
  uint32_t cut_key;          // the writing pass keeps keys >= cut_key (and > tau)
  uint32_t cnt_ticket;
  uint32_t scan_ticket;
  uint32_t fhist[2048];      // keys > tau by their 11 bits below the common prefix
  uint32_t tie_sum;          // ties counted so far by the dense tie count
  // direct tie path: where ties at tau can be, collected by the filter
  uint32_t ts_count;         // subranges outside the scan holding a delegate == tau
  uint32_t tc_count;         // positions of keys equal to tau found
  uint32_t tie_fast_bad;     // a list overflowed: use the tile pipeline
  uint32_t tie_fast;         // the ties were placed directly
  uint32_t tie_reads;        // subranges read for the direct tie path
  uint32_t tie_dticket;
  uint32_t ts[kTieSCap];     // subranges
  uint32_t tc[kTieCandCap];  // positions
};

// First digit level (byte of the (key, ~idx) composite, 0 = top) that can
// differ between the composites of G: G's keys lie in (tau, key_max] (in
// [0, key_max] when Rule 2's filtering is off), so the leading bytes that
// the interval's ends share are the same for all of them; 4 when the key
// itself is fixed. The second select starts at this digit.
__device__ __forceinline__ int g_first_level(const Ctl* ctl, bool no_filter) {
  const uint32_t hi = *reinterpret_cast<const volatile uint32_t*>(&ctl->key_max);
  const uint32_t tau = *reinterpret_cast<const volatile uint32_t*>(&ctl->tau);
  const uint32_t lo = (no_filter || tau == 0xFFFFFFFFu) ? 0u : tau + 1;
  const uint32_t x = lo ^ hi;
  return x == 0 ? 4 : (__clz(x) >> 3);
}
__device__ __forceinline__ uint32_t comp_digit(uint64_t c, int level) {
  return static_cast<uint32_t>(c >> (56 - 8 * level)) & 255u;
}

// Ablations of the method (drtopk_topk_ablate): Rule 2's filtering off
// (every subrange whose maximum delegate reaches tau is concatenated whole),
// and the first top-k stopped one digit early (Sec. 3.3's shortcut: tau is
// the k-th delegate with its low 8 bits cleared, a lower threshold).
constexpr int kAblateNoFilter = 1;
constexpr int kAblateSkipLastDigit = 2;

// Device views of the workspace of one query.
struct Work {
  uint32_t* dkeys;    // [S * beta] delegate keys (mapped), descending
  uint16_t* dsegs;    // [S * beta] delegate segment ids (kNoSeg = pad)
  uint32_t* ds;       // [S * beta] delegate keys surviving the first digit
  uint32_t* scanq;    // [S] subranges queued for the filter scan
  uint32_t* rq;       // [rq_cap] delegates > tau to place (subrange << 2 | slot)
  int64_t rq_cap;
  uint64_t* g;        // [g_cap] composites of {x > tau}
  uint64_t* sv;       // [g_cap] second-select ping-pong buffer
  uint64_t* w;        // [k] winners (unsorted), later sorted
  uint64_t* w2;       // [k] sort ping-pong buffer
  uint64_t* tstat;    // tie path: tie_bytes(S, alpha) bytes (look-back words, then
                      // per-tile lower bounds, their prefixes and the tile list)
  uint64_t* sort_status;  // [8 * tiles * 256] look-back words of the sort
  Ctl* ctl;
  int64_t n;
  int64_t S;
  int64_t g_cap;
  int64_t k;
  int alpha;
  int beta;
  int dtype;
  int ablate;         // kAblate* flags, 0 for the method as stated
  uint32_t* err_out;  // device-visible word the query's last kernel ORs its
                      // error flags into (nullptr: not reported there)
  // speculative compaction (spec): records of subranges whose largest
  // delegate reaches t_lo; rec_cap records at most (0: not planned)
  uint32_t* rec_keys;  // [rec_cap * beta]
  uint16_t* rec_segs;  // [rec_cap * beta]
  uint32_t* rec_sub;   // [rec_cap] subrange of each record
  int64_t rec_cap;
};

// Which delegate rows the threshold and the classification read: every
// subrange (row r = subrange r), or the records of the speculative
// compaction (row r = subrange sub[r]).
struct DView {
  const uint32_t* keys;  // [rows * beta]
  const uint16_t* segs;
  const uint32_t* sub;   // nullptr: rows are subranges
  int64_t rows;
  __device__ __forceinline__ int64_t subrange(int64_t r) const { return sub ? int64_t(__ldcg(sub + r)) : r; }
};
__device__ __forceinline__ DView delegate_view(const Ctl* ctl, const uint32_t* dkeys, const uint16_t* dsegs,
                                               int64_t S, const uint32_t* rk, const uint16_t* rs,
                                               const uint32_t* rsub) {
  if (rk && __ldcg(&ctl->spec_on)) return DView{rk, rs, rsub, int64_t(__ldcg(&ctl->rec_count))};
  return DView{dkeys, dsegs, nullptr, S};
}

// Called by one thread of the last kernel of a query, after every earlier
// kernel of the query has finished: ORs the query's device error flags into
// the caller-visible report word (host-mapped memory or a device word).
__device__ __forceinline__ void report_errors(const Ctl* ctl, uint32_t* err_out) {
  const uint32_t e = *reinterpret_cast<const volatile uint32_t*>(&ctl->error);
  if (e && err_out) {
    volatile uint32_t* q = err_out;
    *q = *q | e;
    __threadfence_system();
  }
}

// -------------------------------------------------------- small helpers ---
__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier + TMA bulk copy (inline PTX) --------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait on an mbarrier phase: false once limit_ns nanoseconds passed
// without the phase completing (the clock is read every 64 polls).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = kWaitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 0 && global_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_evict_normal_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// 1-D bulk copy global -> shared, completion counted on `bar` in bytes.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// ---- warp-aggregated append ------------------------------------------------
// Each lane contributes `cnt` items; returns the lane's first slot.
__device__ __forceinline__ uint32_t warp_append(uint32_t* counter, uint32_t cnt) {
  const uint32_t lane = lane_id();
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= static_cast<uint32_t>(o)) incl += v;
  }
  const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
  uint32_t base = 0;
  if (lane == 31 && total) base = atomicAdd(counter, total);
  base = __shfl_sync(0xFFFFFFFFu, base, 31);
  return base + incl - cnt;
}

// ---- block-aggregated append -------------------------------------------------
// Every thread of the block calls this with its item count; one atomicAdd per
// block reserves the block's range. Returns the thread's first slot.
template <int NT>
__device__ __forceinline__ uint32_t block_append(uint32_t* counter, uint32_t cnt) {
  __shared__ uint32_t s_w[NT / 32];
  __shared__ uint32_t s_base;
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= static_cast<uint32_t>(o)) incl += v;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < NT / 32; ++w) {
      const uint32_t t = s_w[w];
      s_w[w] = run;
      run += t;
    }
    s_base = run ? atomicAdd(counter, run) : 0u;
  }
  __syncthreads();
  const uint32_t r = s_base + s_w[warp] + incl - cnt;
  __syncthreads();
  return r;
}

// Warp-contiguous reservation for one or two output arrays. Each warp
// passes its totals (same value in every lane); one atomic per counter per
// block reserves the block's range; every warp gets a contiguous sub-range
// so that its lanes can write coalesced rounds (ballot + popc ranks).
template <int NT>
__device__ __forceinline__ void block_reserve2(uint32_t* ctr0, uint32_t t0, uint32_t* ctr1,
                                               uint32_t t1, uint32_t& b0, uint32_t& b1) {
  __shared__ uint32_t s[2][NT / 32];
  __shared__ uint32_t s_base[2];
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  if (lane == 0) {
    s[0][warp] = t0;
    s[1][warp] = t1;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const int c = threadIdx.x;
    uint32_t run = 0;
    for (int w = 0; w < NT / 32; ++w) {
      const uint32_t t = s[c][w];
      s[c][w] = run;
      run += t;
    }
    uint32_t* ctr = c ? ctr1 : ctr0;
    s_base[c] = (run && ctr) ? atomicAdd(ctr, run) : 0u;
  }
  __syncthreads();
  b0 = s_base[0] + s[0][warp];
  b1 = s_base[1] + s[1][warp];
  __syncthreads();
}

__device__ __forceinline__ uint32_t lanemask_lt32() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Block-wide exclusive scan of one value per thread (NT threads); *total
// (optional) receives the block sum.
template <int NT>
__device__ __forceinline__ uint32_t block_scan_excl(uint32_t v, uint32_t* total) {
  __shared__ uint32_t wsum[NT / 32];
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= static_cast<uint32_t>(o)) incl += t;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0, tot = 0;
#pragma unroll
  for (int q = 0; q < NT / 32; ++q) {
    if (q < warp) wpre += wsum[q];
    tot += wsum[q];
  }
  __syncthreads();
  if (total) *total = tot;
  return wpre + incl - v;
}

// Shared-memory staging of a variable-size output: items are gathered in a
// block buffer of CAP entries and copied to the global array with one
// atomicAdd per flush (coalesced). All threads of the block call these.
template <typename T, int NT>
__device__ __forceinline__ void stage_flush(T* buf, uint32_t* s_fill, uint32_t* gctr, T* gdst,
                                            uint64_t gcap, uint32_t* err, uint32_t ebit) {
  __shared__ uint32_t s_base;
  __syncthreads();
  const uint32_t f = *s_fill;
  if (threadIdx.x == 0) s_base = f ? atomicAdd(gctr, f) : 0u;
  __syncthreads();
  const uint64_t b = s_base;
  for (uint32_t j = threadIdx.x; j < f; j += NT) {
    if (b + j < gcap) gdst[b + j] = buf[j];
    else atomicOr(err, ebit);
  }
  __syncthreads();
  if (threadIdx.x == 0) *s_fill = 0;
  __syncthreads();
}

// Per-warp variant: a warp gathers items in its own shared buffer of CAP
// entries (a prefix over the lanes, no block barrier) and copies them out
// with one atomicAdd per flush. All 32 lanes call reserve/flush with the
// same arguments; `fill` stays warp-uniform.
template <typename T, int CAP>
struct WarpStage {
  T* buf;
  uint32_t fill;

  __device__ __forceinline__ void flush(uint32_t* gctr, T* gdst, uint64_t gcap, uint32_t* err,
                                        uint32_t ebit) {
    __syncwarp();
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t base = 0;
    if (lane == 0 && fill) base = atomicAdd(gctr, fill);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (uint32_t j = lane; j < fill; j += 32) {
      if (uint64_t(base) + j < gcap) gdst[base + j] = buf[j];
      else atomicOr(err, ebit);
    }
    __syncwarp();
    fill = 0;
  }

  // Reserves `cnt` consecutive slots for every lane (prefix over the warp;
  // at most CAP in total), flushing first when they do not fit; returns the
  // lane's first slot in buf. The lanes write their slots before the next
  // call.
  __device__ __forceinline__ uint32_t reserve(uint32_t cnt, uint32_t* gctr, T* gdst, uint64_t gcap,
                                              uint32_t* err, uint32_t ebit) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= static_cast<uint32_t>(o)) incl += t;
    }
    const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (fill + tot > CAP) flush(gctr, gdst, gcap, err, ebit);
    const uint32_t pos = fill + incl - cnt;
    fill += tot;
    return pos;
  }
};

// Reserves cnt staged slots for the calling thread (flushing first when the
// buffer cannot take this round); returns the first slot in buf. The caller
// writes buf[slot .. slot + cnt) before the next stage call.
template <typename T, int NT, int CAP>
__device__ __forceinline__ uint32_t stage_reserve(T* buf, uint32_t* s_fill, uint32_t cnt,
                                                  uint32_t* gctr, T* gdst, uint64_t gcap,
                                                  uint32_t* err, uint32_t ebit) {
  uint32_t total;
  const uint32_t excl = block_scan_excl<NT>(cnt, &total);
  if (*s_fill + total > CAP) stage_flush<T, NT>(buf, s_fill, gctr, gdst, gcap, err, ebit);
  const uint32_t slot = *s_fill + excl;
  __syncthreads();
  if (threadIdx.x == 0) *s_fill += total;
  return slot;
}

// Lanes of `am` whose 8-bit value d equals the calling lane's (radix-rank
// peer mask from 8 ballots; cheaper than a generic match on this GPU).
__device__ __forceinline__ uint32_t peers8(uint32_t am, uint32_t d) {
  uint32_t peers = am;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const uint32_t bal = __ballot_sync(am, (d >> b) & 1u);
    peers &= ((d >> b) & 1u) ? bal : ~bal;
  }
  return peers;
}

// Thread-local run-length aggregation of shared-histogram increments: equal
// consecutive bins (skewed or tied data) cost one shared atomic per run.
struct RunHist {
  uint32_t bin = 0xFFFFFFFFu;
  uint32_t cnt = 0;
  __device__ __forceinline__ void add(uint32_t* sh, uint32_t b) {
    if (b != bin) {
      if (cnt) atomicAdd(&sh[bin], cnt);
      bin = b;
      cnt = 1;
    } else {
      ++cnt;
    }
  }
  __device__ __forceinline__ void flush(uint32_t* sh) {
    if (cnt) atomicAdd(&sh[bin], cnt);
    cnt = 0;
  }
};

// ---- last-block-done helper --------------------------------------------------
// Called by all threads after a block has published its partial results
// with global atomics. Returns true in exactly one block: the last to arrive.
__device__ __forceinline__ bool last_block(uint32_t* ticket) {
  __shared__ uint32_t s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t t = atomicAdd(ticket, 1u);
    s_last = (t == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Same for a grid of which only the first `nact` blocks take part.
__device__ __forceinline__ bool last_block_of(uint32_t* ticket, uint32_t nact) {
  __shared__ uint32_t s_last2;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t t = atomicAdd(ticket, 1u);
    s_last2 = (t == nact - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (s_last2) __threadfence();
  return s_last2 != 0;
}

// Number of blocks that have work when `count` items are processed
// `per_step` at a time by a grid-stride loop (at least 1).
__device__ __forceinline__ uint32_t active_blocks(int64_t count, int64_t per_step) {
  int64_t a = (count + per_step - 1) / per_step;
  if (a > static_cast<int64_t>(gridDim.x)) a = gridDim.x;
  if (a < 1) a = 1;
  return static_cast<uint32_t>(a);
}

// Picks the digit holding the k_rem-th largest of the histogram `h` (in
// global memory, read with L2-coherent loads) and advances the selection.
// Executed by warp 0 of the last block only. Returns the bucket count.
template <int NPASS>
__device__ inline void select_digit(SelState<NPASS>* st, int pass, int total_bits,
                                    bool allow_done) {
  const uint32_t lane = lane_id();
  uint32_t c[8];
  uint32_t sum = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    c[j] = __ldcg(&st->hist[pass][lane * 8 + j]);
    sum += c[j];
  }
  // suffix sums over lanes: above[l] = sum of lanes > l
  uint32_t incl = sum;  // inclusive suffix
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t v = __shfl_down_sync(0xFFFFFFFFu, incl, o);
    if (lane + o < 32) incl += v;
  }
  const uint32_t above = incl - sum;
  const uint32_t k_rem = st->k_rem;
  // the lane whose bins hold the k_rem-th largest: above < k_rem <= incl
  const bool mine = (above < k_rem) && (k_rem <= incl);
  const uint32_t who = __ffs(__ballot_sync(0xFFFFFFFFu, mine));
  if (who != 0 && lane == who - 1) {
    uint32_t acc = above;
    int d = 7;
    for (; d > 0; --d) {
      if (acc + c[d] >= k_rem) break;
      acc += c[d];
    }
    const uint32_t digit = lane * 8 + d;
    const uint32_t nk = k_rem - acc;
    const int shift = total_bits - 8 * (pass + 1);
    st->prefix |= static_cast<uint64_t>(digit) << shift;
    st->k_rem = nk;
    st->bucket = c[d];
    st->level = pass + 1;
    if (allow_done && c[d] == nk) st->done = 1;
    __threadfence();
  }
}

}  // namespace drtopk
