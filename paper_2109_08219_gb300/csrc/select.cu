// First top-k (threshold), concatenation with filtering, tie ranking and the
// second top-k (Sec. 3.2 Rule 2, Sec. 3.3 Rule 3, Sec. 4.1).
//
// Exactness argument (the paper states Rules 1-3 for distinct keys; this
// version also covers ties). tau = k-th largest delegate <= k-th largest
// key of V because the delegates are elements of V (Rule 2). Let
// G = {x > tau}:
//   * a subrange with m^{beta-1} > tau is scanned; its elements > tau go to G.
//     Fewer than k delegates exceed tau, so fewer than k/beta subranges are
//     scanned and |G| < floor((k-1)/beta) * 2^alpha + k (the workspace bound);
//   * in any other subrange every element > tau is a delegate (non-delegates
//     are <= m^{beta-1} <= tau), so its delegates > tau are emitted (Rule 3).
// If |G| >= k the k-th key is above tau and the answer lies in G: an exact
// MSD radix select over (key, ~idx) composites finds it. Otherwise the k-th
// key equals tau (at least k keys are >= tau) and the answer is G plus the
// k - |G| smallest indices holding tau; these are found by prefix sums of
// per-subrange tie counts taken in index order, reading a subrange again
// only when its count is not already known from its delegates and an
// earlier prefix could still be short.
//
// GB300 organisation: every variable-size output is gathered in shared
// memory and appended with one atomic per block step or per warp flush
// (block_reserve2, stage_reserve / stage_flush, WarpStage); uneven work
// (scanned subranges, tie counts) goes through global queues that all
// warps of the grid drain; each radix pass keeps only the survivors of the
// previous digit.
#include "common.cuh"
#include "launch.h"

namespace drtopk {
namespace {

constexpr int kThreads = 256;
constexpr int kScanKPT = 16;  // virtual keys per thread per filter-scan step

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ void zero_hist(uint32_t* sh) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) sh[i] = 0;
}

__device__ __forceinline__ void flush_hist(const uint32_t* sh, uint32_t* g) {
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    const uint32_t v = sh[i];
    if (v) atomicAdd(&g[i], v);
  }
}

__device__ __forceinline__ int64_t sub_len(int64_t i, int alpha, int64_t n) {
  const int64_t lo = i << alpha;
  return imin64(int64_t(1) << alpha, n - lo);
}

// Exact position of a delegate: the (r+1)-th key equal to K (mapped) in
// segment `seg` of subrange i. -1 when absent (cannot happen).
template <int DT>
__device__ int64_t resolve_pos(const uint32_t* keys, int64_t n, int alpha, int64_t i,
                               uint32_t seg, uint32_t K, int r) {
  const int64_t gran = alpha < 5 ? (int64_t(1) << alpha) : 32;
  const int64_t lo = (i << alpha) + seg * gran;
  const int64_t hi = imin64(imin64(n, lo + gran), (i + 1) << alpha);
  if (hi - lo == gran && (reinterpret_cast<uintptr_t>(keys + lo) & 15u) == 0) {
    // whole segment, 16-byte aligned: issue every load at once
    const uint4* v4 = reinterpret_cast<const uint4*>(keys + lo);
    const int words = static_cast<int>(gran >> 2);
    uint4 v[8];
#pragma unroll
    for (int w = 0; w < 8; ++w)
      if (w < words) v[w] = __ldg(v4 + w);
    int cnt = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      if (w < words) {
        const uint32_t e[4] = {v[w].x, v[w].y, v[w].z, v[w].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (map_key<DT>(e[q]) == K) {
            if (cnt == r) return lo + 4 * w + q;
            ++cnt;
          }
        }
      }
    }
    return -1;
  }
  int cnt = 0;
  for (int64_t t = lo; t < hi; ++t) {
    if (map_key<DT>(__ldg(keys + t)) == K) {
      if (cnt == r) return t;
      ++cnt;
    }
  }
  return -1;
}

// Occurrence rank of delegate j among the earlier delegates with the same
// (key, segment) in row dk/ds.
template <int B>
__device__ __forceinline__ int occ_rank(const uint32_t* dk, const uint16_t* ds, int j) {
  int r = 0;
#pragma unroll
  for (int q = 0; q < B; ++q)
    if (q < j && dk[q] == dk[j] && ds[q] == ds[j]) ++r;
  return r;
}

// The beta delegate keys of subrange i (contiguous in the workspace, which
// is 256-byte aligned): one vector load for beta 2 and 4.
template <int B>
__device__ __forceinline__ void load_dkeys(const uint32_t* dkeys, int64_t i, uint32_t (&d)[B]) {
  if constexpr (B == 2) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(dkeys) + i);
    d[0] = v.x;
    d[1] = v.y;
  } else if constexpr (B == 4) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(dkeys) + i);
    d[0] = v.x;
    d[1] = v.y;
    d[2] = v.z;
    d[3] = v.w;
  } else {
#pragma unroll
    for (int j = 0; j < B; ++j) d[j] = __ldg(dkeys + i * B + j);
  }
}

int grid_for(int64_t work, int per_block, int sms, int per_sm) {
  int64_t g = (work + per_block - 1) / per_block;
  const int64_t cap = static_cast<int64_t>(sms) * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

// ------------------------------------------------------------ threshold ---
// Loads 16 consecutive-in-blocks keys per thread: word q (0..3) of thread t
// in block step `base` covers keys base + (q * NT + t) * 4 .. + 3.
template <int NT>
__device__ __forceinline__ void load16(const uint32_t* a, int64_t count, int64_t base,
                                       uint32_t (&v)[16]) {
  // full words load unconditionally (clamped to the last full word); the
  // ragged tail (count not a multiple of 4) is patched with scalar loads
  const int64_t last_full = (count >> 2) - 1;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t w = (base >> 2) + int64_t(q) * NT + threadIdx.x;
    const int64_t wc = w < last_full ? w : (last_full < 0 ? 0 : last_full);
    uint4 x = make_uint4(0, 0, 0, 0);
    if (last_full >= 0) x = __ldcg(reinterpret_cast<const uint4*>(a) + wc);
    v[q * 4 + 0] = x.x; v[q * 4 + 1] = x.y; v[q * 4 + 2] = x.z; v[q * 4 + 3] = x.w;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t w = (base >> 2) + int64_t(q) * NT + threadIdx.x;
    if (w > last_full) {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[q * 4 + e] = (w * 4 + e < count) ? a[w * 4 + e] : 0u;
    }
  }
}

constexpr int kThrStageCap = kThreads * 16;

// Digit 1 pass: keep the delegate keys whose first digit is the selected
// one (compacted into ds) and histogram their second digit. When the first
// digit's bucket is large (ties, few distinct values) nothing is copied and
// the later passes read the delegate keys in place.
__global__ void __launch_bounds__(kThreads) thr_compact_kernel(const uint32_t* dkeys_all,
                                                               int64_t count_all, uint32_t* ds,
                                                               Ctl* ctl, int allow_done,
                                                               const uint32_t* rec_keys, int beta) {
  // every delegate key, or the records' keys (their rows hold every key
  // >= t_lo, and tau >= t_lo: the same k-th largest)
  const DView dv = delegate_view(ctl, dkeys_all, nullptr, count_all / beta, rec_keys, nullptr, nullptr);
  const uint32_t* dkeys = dv.keys;
  const int64_t count = dv.rows * beta;
  __shared__ uint32_t sh[256];
  constexpr int kWCap = kThrStageCap / (kThreads / 32);
  __shared__ uint32_t sbuf[kThrStageCap];
  zero_hist(sh);
  __syncthreads();
  SelState<4>* st = &ctl->dsel;
  const uint32_t d0 = static_cast<uint32_t>(__ldcg(&st->prefix)) >> 24;
  const bool inplace = uint64_t(__ldcg(&st->bucket)) * 8 > static_cast<uint64_t>(count);
  if (inplace && blockIdx.x == 0 && threadIdx.x == 0) ctl->ds_inplace = 1;
  RunHist rh;
  // kept keys are staged per warp (no block barrier in the loop)
  WarpStage<uint32_t, kWCap> stg{sbuf + (threadIdx.x >> 5) * kWCap, 0u};
  uint32_t lo = 0xFFFFFFFFu, hi = 0;  // range of the bucket's keys
  const int64_t step = int64_t(gridDim.x) * kThreads * 16;
  for (int64_t base = int64_t(blockIdx.x) * kThreads * 16; base < count; base += step) {
    uint32_t v[16];
    load16<kThreads>(dkeys, count, base, v);
    const bool full = base + kThreads * 16 <= count;  // no bounds checks needed
    uint32_t hit = 0;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      bool in = true;
      if (!full) in = base + (int64_t(e >> 2) * kThreads + threadIdx.x) * 4 + (e & 3) < count;
      if (in && (v[e] >> 24) == d0) hit |= 1u << e;
    }
    if (__any_sync(0xFFFFFFFFu, hit != 0)) {  // the bucket is small: most warp steps skip this
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        if ((hit >> e) & 1u) {
          rh.add(sh, (v[e] >> 16) & 255u);
          lo = min(lo, v[e]);
          hi = max(hi, v[e]);
        }
      }
      if (!inplace) {
        uint32_t pos = stg.reserve(__popc(hit), &ctl->ds_count, ds, ~uint64_t(0), &ctl->error, 0u);
#pragma unroll
        for (int e = 0; e < 16; ++e)
          if ((hit >> e) & 1u) stg.buf[pos++] = v[e];
      }
    }
  }
  if (!inplace) stg.flush(&ctl->ds_count, ds, ~uint64_t(0), &ctl->error, 0u);
  rh.flush(sh);
  lo = __reduce_min_sync(0xFFFFFFFFu, lo);
  hi = __reduce_max_sync(0xFFFFFFFFu, hi);
  if ((threadIdx.x & 31) == 0 && hi >= lo) {
    atomicMax(&ctl->thr_lo_inv, ~lo);
    atomicMax(&ctl->thr_hi, hi);
  }
  __syncthreads();
  flush_hist(sh, st->hist[1]);
  if (last_block(&st->ticket[1])) {
    if (threadIdx.x < 32) select_digit<4>(st, 1, 32, false);
    if (threadIdx.x == 0) {
      // every key of the bucket holding the k-th delegate is the same: it is
      // tau, and the digit 2 and 3 passes have nothing left to decide
      const uint32_t blo = ~__ldcg(&ctl->thr_lo_inv), bhi = __ldcg(&ctl->thr_hi);
      if (allow_done && blo == bhi) {
        ctl->tau = bhi;
        __threadfence();
        ctl->tau_ready = 1;
        ctl->thr_done = 1;
      }
    }
  }
}

// Digit 2 and 3 passes over the compacted survivors (or the delegate keys).
__global__ void __launch_bounds__(kThreads) thr_pass_kernel(const uint32_t* dsv,
                                                            const uint32_t* dkeys_all,
                                                            int64_t dcount_all, Ctl* ctl,
                                                            int pass, int last_pass,
                                                            const uint32_t* rec_keys, int beta) {
  if (__ldcg(&ctl->thr_done)) return;  // tau already known
  const DView dv = delegate_view(ctl, dkeys_all, nullptr, dcount_all / beta, rec_keys, nullptr, nullptr);
  const uint32_t* dkeys = dv.keys;
  const int64_t dcount = dv.rows * beta;
  __shared__ uint32_t sh[256];
  zero_hist(sh);
  __syncthreads();
  SelState<4>* st = &ctl->dsel;
  const bool inplace = __ldcg(&ctl->ds_inplace) != 0;
  const uint32_t* ds = inplace ? dkeys : dsv;
  const int64_t count = inplace ? dcount : static_cast<int64_t>(__ldcg(&ctl->ds_count));
  const uint32_t prefix = static_cast<uint32_t>(__ldcg(&st->prefix));
  const uint32_t mask = 0xFFFFFFFFu << (32 - 8 * pass);
  const uint32_t want = prefix & mask;
  const int sh_d = 24 - 8 * pass;
  const uint32_t nact = active_blocks(count, int64_t(kThreads) * 16);
  if (blockIdx.x >= nact) return;
  RunHist rh;
  const int64_t step = int64_t(nact) * kThreads * 16;
  for (int64_t base = int64_t(blockIdx.x) * kThreads * 16; base < count; base += step) {
    uint32_t v[16];
    load16<kThreads>(ds, count, base, v);
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int64_t i = base + (int64_t(e >> 2) * kThreads + threadIdx.x) * 4 + (e & 3);
      if (i < count && (v[e] & mask) == want) rh.add(sh, (v[e] >> sh_d) & 255u);
    }
  }
  rh.flush(sh);
  __syncthreads();
  flush_hist(sh, st->hist[pass]);
  if (last_block_of(&st->ticket[pass], nact)) {
    if (threadIdx.x < 32) {
      select_digit<4>(st, pass, 32, false);
      if (pass == last_pass && threadIdx.x == 0) {
        __threadfence();
        ctl->tau = static_cast<uint32_t>(__ldcg(&st->prefix));
        ctl->tau_ready = 1;
      }
    }
  }
}

// --------------------------------------------------------------- filter ---
struct FilterParams {
  const uint32_t* keys;
  int64_t n, S, g_cap, k;
  int alpha;
  const uint32_t* dkeys;
  const uint16_t* dsegs;
  const uint32_t* rec_keys;  // speculative compaction's records (nullptr: none)
  const uint16_t* rec_segs;
  const uint32_t* rec_sub;
  uint32_t* scanq;
  uint64_t* g;
  Ctl* ctl;
  uint32_t* rq;   // delegates > tau to place: subrange << 2 | delegate slot
  int64_t rq_cap;
  uint64_t* w;    // winners (top-k only): the direct tie path writes its ties
  int kth_only;
  int no_filter;  // ablation: Rule 2 off
};

// The direct tie path is tried for top-k with Rule 2's filtering as stated.
__device__ __forceinline__ bool tie_direct_on(const FilterParams& p) {
  return !p.kth_only && !p.no_filter;
}


// Appends this lane's value (when `has`) to one of the direct tie path's
// capped lists, one atomic per warp (all lanes call it). Past the cap the
// entry is dropped, tie_fast_bad is set and `stop` makes the warp skip its
// later appends.
__device__ __forceinline__ void tie_append(bool has, uint32_t v, uint32_t* count, uint32_t* buf,
                                           uint32_t cap, Ctl* ctl, bool& stop) {
  const uint32_t m = __ballot_sync(0xFFFFFFFFu, has && !stop);
  if (m == 0) return;
  const int leader = __ffs(m) - 1;
  uint32_t base = 0;
  if (static_cast<int>(lane_id()) == leader) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (base + __popc(m) > cap) {
    stop = true;
    if (static_cast<int>(lane_id()) == leader) ctl->tie_fast_bad = 1;
  }
  if ((m >> lane_id()) & 1u) {
    const uint32_t slot = base + __popc(m & lanemask_lt());
    if (slot < cap) buf[slot] = v;
  }
}

// Each thread classifies 4 subranges per step: skip (m^0 <= tau), queue
// for a scan (m^{beta-1} > tau: Rule 3 says every element may qualify) or
// emit its delegates > tau (Rule 3: they are all of its elements > tau).
// Queue entries and emitted delegate slots are staged per warp in shared
// memory.
constexpr int kClsSub = 4;
constexpr int kClsGCap = kThreads * kClsSub * 4;
constexpr int kClsQCap = kThreads * kClsSub * 2;

template <int DT, int B>
__global__ void __launch_bounds__(kThreads) filter_classify_kernel(FilterParams p) {
  constexpr int kWR = kClsGCap / (kThreads / 32);
  constexpr int kWQ = kClsQCap / (kThreads / 32);
  __shared__ uint32_t rbuf[kClsGCap];
  __shared__ uint32_t qbuf[kClsQCap];
  // queue entries and requests are staged per warp (no block barrier)
  const int warp = threadIdx.x >> 5;
  WarpStage<uint32_t, kWQ> sq{qbuf + warp * kWQ, 0u};
  WarpStage<uint32_t, kWR> sr{rbuf + warp * kWR, 0u};
  const uint32_t tau = __ldcg(&p.ctl->tau);
  const int alpha = p.alpha;
  uint32_t nscan = 0;
  const int64_t per_step = int64_t(kThreads) * kClsSub;
  // rows: every subrange, or the records of the speculative compaction
  // (subranges not recorded have m^0 < t_lo <= tau: skipped either way)
  const DView dv = delegate_view(p.ctl, p.dkeys, p.dsegs, p.S, p.rec_keys, p.rec_segs, p.rec_sub);
  const int64_t rows = dv.rows;
  // the next step's delegates are loaded before this step is classified
  // (double-buffered in registers)
  uint32_t dk[kClsSub][B], nk[kClsSub][B];
  auto load_step = [&](int64_t b) {
#pragma unroll
    for (int u = 0; u < kClsSub; ++u) {
      const int64_t r = b + int64_t(u) * kThreads + threadIdx.x;
      if (r < rows) {
        load_dkeys<B>(dv.keys, r, nk[u]);
      } else {
#pragma unroll
        for (int j = 0; j < B; ++j) nk[u][j] = 0u;
      }
    }
  };
  load_step(int64_t(blockIdx.x) * per_step);
  for (int64_t base = int64_t(blockIdx.x) * per_step; base < rows;
       base += int64_t(gridDim.x) * per_step) {
#pragma unroll
    for (int u = 0; u < kClsSub; ++u)
#pragma unroll
      for (int j = 0; j < B; ++j) dk[u][j] = nk[u][j];
    if (base + int64_t(gridDim.x) * per_step < rows) load_step(base + int64_t(gridDim.x) * per_step);
    uint32_t scanm = 0;  // subranges to scan (bit u)
    uint32_t emitm = 0;  // delegate slots to place (bit u * B + j)
#pragma unroll
    for (int u = 0; u < kClsSub; ++u) {
      const int64_t r = base + int64_t(u) * kThreads + threadIdx.x;
      const int64_t i = r < rows ? dv.subrange(r) : 0;
      if (p.no_filter) {
        // Rule 1 alone: a subrange whose maximum delegate reaches tau is kept whole
        if (r < rows && dk[u][0] >= tau) scanm |= 1u << u;
      } else if (r < rows && dk[u][0] > tau) {
        if (dk[u][B - 1] > tau && sub_len(i, alpha, p.n) > B) {
          scanm |= 1u << u;
        } else {
          // its keys > tau are exactly its delegates > tau (Rule 3); their
          // positions are resolved by filter_resolve_kernel
#pragma unroll
          for (int j = 0; j < B; ++j) emitm |= (dk[u][j] > tau) ? (1u << (u * B + j)) : 0u;
        }
      }
    }
    if (__any_sync(0xFFFFFFFFu, scanm != 0)) {
      uint32_t pos = sq.reserve(__popc(scanm), &p.ctl->scanq_count, p.scanq, ~uint64_t(0),
                                &p.ctl->error, 0u);
#pragma unroll
      for (int u = 0; u < kClsSub; ++u) {
        if ((scanm >> u) & 1u) {
          const int64_t r = base + int64_t(u) * kThreads + threadIdx.x;
          sq.buf[pos++] = static_cast<uint32_t>(dv.subrange(r));
        }
      }
      nscan += __popc(scanm);
    }
    if (__any_sync(0xFFFFFFFFu, emitm != 0)) {
      uint32_t pos = sr.reserve(__popc(emitm), &p.ctl->rq_count, p.rq,
                                static_cast<uint64_t>(p.rq_cap), &p.ctl->error, kErrOverflowG);
#pragma unroll
      for (int u = 0; u < kClsSub; ++u)
#pragma unroll
        for (int j = 0; j < B; ++j)
          if ((emitm >> (u * B + j)) & 1u)  // row << 2 | slot
            sr.buf[pos++] = static_cast<uint32_t>((base + int64_t(u) * kThreads + threadIdx.x) << 2) |
                            static_cast<uint32_t>(j);
    }
  }
  sq.flush(&p.ctl->scanq_count, p.scanq, ~uint64_t(0), &p.ctl->error, 0u);
  sr.flush(&p.ctl->rq_count, p.rq, static_cast<uint64_t>(p.rq_cap), &p.ctl->error, kErrOverflowG);
  nscan = __reduce_add_sync(0xFFFFFFFFu, nscan);
  if ((threadIdx.x & 31) == 0 && nscan) atomicAdd(&p.ctl->scanned, nscan);
}

// Fine digit of the keys above tau for the counting pass of large scan
// sets: the 11 bits just below the bits that every key in (tau, key_max]
// shares. cut(b) = the smallest key whose fine digit is b.
constexpr int kFineBins = 2048;
struct FineGeom {
  uint32_t sh;    // digit = (key >> sh) & (kFineBins - 1)
  uint32_t pref;  // the shared leading bits
};
__device__ __forceinline__ FineGeom fine_geom(const Ctl* ctl) {
  const uint32_t hi = __ldcg(&ctl->key_max);
  const uint32_t tau = __ldcg(&ctl->tau);
  const uint32_t lo = tau == 0xFFFFFFFFu ? hi : tau + 1;
  const uint32_t x = lo ^ hi;
  const int pb = x ? __clz(x) : 32;
  FineGeom g;
  g.sh = static_cast<uint32_t>(32 - pb - 11 > 0 ? 32 - pb - 11 : 0);
  g.pref = pb ? (hi & (0xFFFFFFFFu << (32 - pb))) : 0u;
  return g;
}

// Counting pass first when the scan set is large (sorted inputs with large
// k): then only the keys from the bucket holding the k-th key upwards are
// written, not every key above tau.
__device__ __forceinline__ bool two_pass_wanted(int no_filter, int64_t total, int64_t k) {
  const int64_t lim = 4 * k > (int64_t(1) << 17) ? 4 * k : (int64_t(1) << 17);
  return !no_filter && total > lim;
}

// The query mode, decided once G is complete (warp 0 of the filter's last
// block): select the k-th of G when |{x > tau}| >= k, else ties at tau.
__device__ __forceinline__ void decide_mode(Ctl* ctl, int64_t k, int lvl0, bool kth_only) {
  const uint32_t g = __ldcg(&ctl->two_pass) ? __ldcg(&ctl->g_all) : __ldcg(&ctl->g_count);
  if (threadIdx.x == 0) ctl->g_total = g;
  if (static_cast<int64_t>(g) >= k) {
    if (threadIdx.x == 0) {
      ctl->mode = kModeSelect;
      ctl->gsel.k_rem = static_cast<uint32_t>(k);
      // the leading digits common to all of G are known: they are the
      // first lvl0 bytes of key_max; the selection starts after them
      const uint64_t km = static_cast<uint64_t>(__ldcg(&ctl->key_max)) << 32;
      ctl->gsel.prefix = lvl0 ? (km & (~0ull << (64 - 8 * lvl0))) : 0ull;
      ctl->g_lvl0 = static_cast<uint32_t>(lvl0);
    }
    __syncwarp();
    __threadfence();
    select_digit<8>(&ctl->gsel, lvl0, 64, !kth_only);
  } else if (threadIdx.x == 0) {
    ctl->mode = kModeTies;
    ctl->need = static_cast<uint32_t>(k - g);
    ctl->kth_mapped = __ldcg(&ctl->tau);
  }
}

// Positions of the queued delegates: the occurrence-th key equal to the
// delegate in its 32-key segment, found by one coalesced read per request
// and a vote. A warp takes 32 requests (lane u decodes request u), then
// reads their segments 8 at a time (broadcast by shuffles, 8 reads in
// flight); lane u keeps the composite of request u. The composites join G
// (staged per block) and the histogram of their first digit. The last block
// decides the query mode (G large enough, or ties at tau).
constexpr int kResCap = kThreads * 4;

template <int DT, int B>
__global__ void __launch_bounds__(kThreads) filter_resolve_kernel(FilterParams p) {
  __shared__ uint32_t sh[256];
  __shared__ uint32_t fh[kFineBins];
  __shared__ uint64_t gbuf[kResCap];
  __shared__ uint32_t g_fill;
  zero_hist(sh);
  for (int i = threadIdx.x; i < kFineBins; i += kThreads) fh[i] = 0;
  if (threadIdx.x == 0) g_fill = 0;
  __syncthreads();
  Ctl* ctl = p.ctl;
  const int64_t nq = __ldcg(&ctl->rq_count);
  const int alpha = p.alpha;
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const int lvl0 = g_first_level(ctl, p.no_filter != 0);
  const FineGeom fg = fine_geom(ctl);
  // the counting pass of a large scan set needs these keys in its histogram
  const bool fine = two_pass_wanted(p.no_filter, int64_t(__ldcg(&ctl->scanq_count)) << alpha, p.k);
  // requests are (row << 2 | slot) of the classification's rows
  const DView dv = delegate_view(ctl, p.dkeys, p.dsegs, p.S, p.rec_keys, p.rec_segs, p.rec_sub);
  for (int64_t b0 = int64_t(blockIdx.x) * kThreads; b0 < nq; b0 += int64_t(gridDim.x) * kThreads) {
    const int64_t q = b0 + threadIdx.x;  // this lane's request
    uint32_t key = 0;
    int64_t lo = 0, hi = 0;
    int occ = 0;
    if (q < nq) {
      const uint32_t r = p.rq[q];
      const int64_t row = r >> 2;
      const int64_t i = dv.subrange(row);
      const int j = static_cast<int>(r & 3u);
      uint32_t dk[B];
      uint16_t ds[B];
#pragma unroll
      for (int z = 0; z < B; ++z) {
        dk[z] = dv.keys[row * B + z];
        ds[z] = dv.segs[row * B + z];
      }
      // register selects (j is data-dependent): no local-memory arrays
      uint32_t sj = 0;
#pragma unroll
      for (int z = 0; z < B; ++z) {
        if (z == j) {
          key = dk[z];
          sj = ds[z];
        }
      }
#pragma unroll
      for (int z = 0; z < B; ++z) occ += (z < j && dk[z] == key && ds[z] == sj) ? 1 : 0;
      lo = (i << alpha) + int64_t(sj) * 32;
      hi = imin64(imin64(p.n, lo + 32), (i + 1) << alpha);
    }
    uint64_t item = 0;
    const bool has = q < nq;
#pragma unroll
    for (int g8 = 0; g8 < 4; ++g8) {
      uint32_t x[8], kk[8];
      int64_t l8[8], h8[8];
      int o8[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int src = g8 * 8 + u;
        kk[u] = __shfl_sync(0xFFFFFFFFu, key, src);
        l8[u] = __shfl_sync(0xFFFFFFFFu, lo, src);
        h8[u] = __shfl_sync(0xFFFFFFFFu, hi, src);
        o8[u] = __shfl_sync(0xFFFFFFFFu, occ, src);
        x[u] = l8[u] + lane < h8[u] ? __ldg(p.keys + l8[u] + lane) : 0u;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        uint32_t bal = __ballot_sync(0xFFFFFFFFu, l8[u] + lane < h8[u] && map_key<DT>(x[u]) == kk[u]);
        for (int z = 0; z < o8[u]; ++z) bal &= bal - 1;
        if (static_cast<int>(lane) == g8 * 8 + u && has) {
          if (bal == 0) atomicOr(&ctl->error, kErrTieRank);
          item = make_comp(key, static_cast<uint32_t>(lo + (bal ? __ffs(bal) - 1 : 0)));
        }
      }
    }
    (void)warp;
    const uint32_t slot = stage_reserve<uint64_t, kThreads, kResCap>(
        gbuf, &g_fill, has ? 1u : 0u, &ctl->g_count, p.g, static_cast<uint64_t>(p.g_cap),
        &ctl->error, kErrOverflowG);
    if (has) {
      gbuf[slot] = item;
      atomicAdd(&sh[comp_digit(item, lvl0)], 1u);
      if (fine) atomicAdd(&fh[(comp_key(item) >> fg.sh) & (kFineBins - 1)], 1u);
    }
  }
  stage_flush<uint64_t, kThreads>(gbuf, &g_fill, &ctl->g_count, p.g, static_cast<uint64_t>(p.g_cap),
                                  &ctl->error, kErrOverflowG);
  flush_hist(sh, ctl->gsel.hist[lvl0]);
  if (fine) {
    for (int i = threadIdx.x; i < kFineBins; i += kThreads) {
      const uint32_t v = fh[i];
      if (v) atomicAdd(&ctl->fhist[i], v);
    }
  }
}

// All queued subranges read as one virtual array of nq * 2^alpha keys,
// 2048 per block step. The queue entries a step needs are staged in shared
// memory one step ahead (ScanQ), so a step waits for one round trip (its
// keys), not two (entry, then key). Kept keys are appended with one atomic
// per block step.
constexpr int kScanStep = kThreads * kScanKPT;     // virtual keys per block step
constexpr int kScanQ = kScanStep >> kMinAlpha;     // queue entries per step at most
constexpr int kScanQPer = kScanQ / kThreads;

struct ScanQ {
  uint32_t (*s)[kScanQ];  // [2][kScanQ] in shared memory
  uint32_t r[kScanQPer];  // entries of the next step, in flight
  int64_t nq;
  int alpha;

  // entries of the step starting at virtual key b (a multiple of kScanStep)
  __device__ __forceinline__ int64_t first(int64_t b) const { return b >> alpha; }
  __device__ __forceinline__ int64_t count(int64_t b) const {
    const int64_t c = ((b + kScanStep - 1) >> alpha) - (b >> alpha) + 1;
    return c < kScanQ ? c : kScanQ;
  }
  __device__ __forceinline__ void fetch(const uint32_t* scanq, int64_t b) {
    const int64_t q0 = first(b), c = count(b);
#pragma unroll
    for (int e = 0; e < kScanQPer; ++e) {
      const int64_t j = threadIdx.x + e * kThreads;
      r[e] = (j < c && q0 + j < nq) ? __ldg(scanq + q0 + j) : 0u;
    }
  }
  __device__ __forceinline__ void put(int buf) {
#pragma unroll
    for (int e = 0; e < kScanQPer; ++e) s[buf][threadIdx.x + e * kThreads] = r[e];
  }
  // position of virtual key v of the step starting at b
  __device__ __forceinline__ int64_t pos(int buf, int64_t b, int64_t v) const {
    return (int64_t(s[buf][(v >> alpha) - (b >> alpha)]) << alpha) + (v & ((int64_t(1) << alpha) - 1));
  }
};

// Direct tie path, placement (block-wide, in the last block of the
// collection kernel below): every key equal to tau was listed (delegates
// equal to tau, keys of the subranges read); when the lists did not
// overflow, the `need` smallest positions go to W after G in index order
// (rank = number of listed positions below), and the tile pipeline of the
// tie path is skipped.
__device__ __noinline__ void tie_direct(Ctl* ctl, uint64_t* w) {
  __shared__ uint32_t s_pos[kTieCandCap];
  if (__ldcg(&ctl->mode) != kModeTies || __ldcg(&ctl->tie_fast_bad)) return;  // uniform
  const uint32_t T = __ldcg(&ctl->tc_count);
  const uint32_t need = __ldcg(&ctl->need);
  if (T > kTieCandCap || T < need) return;  // uniform; the tile pipeline decides
  const uint32_t g = __ldcg(&ctl->g_count);
  const uint32_t tau = __ldcg(&ctl->tau);
  for (uint32_t e = threadIdx.x; e < T; e += blockDim.x) s_pos[e] = __ldcg(&ctl->tc[e]);
  __syncthreads();
  for (uint32_t e = threadIdx.x; e < T; e += blockDim.x) {
    const uint32_t pe = s_pos[e];
    uint32_t rank = 0;
    for (uint32_t f = 0; f < T; ++f) rank += s_pos[f] < pe ? 1u : 0u;
    if (rank < need) w[g + rank] = make_comp(tau, pe);
  }
  if (threadIdx.x == 0) {
    ctl->tie_fast = 1;
    atomicAdd(&ctl->w_count, need);
    const uint32_t nr = __ldcg(&ctl->tie_reads);
    if (nr) atomicAdd(&ctl->tie_scanned, nr);
  }
}

// Direct tie path, step 1 (after the filter, mode ties only): the
// subranges outside the scan that hold a delegate equal to tau, from one
// pass over the delegate keys. Skipped from the start when the threshold
// select counted more delegates equal to tau than the list can take
// (dense ties: the tile pipeline takes them).
template <int B>
__global__ void __launch_bounds__(kThreads) filter_tfind_kernel(FilterParams p) {
  Ctl* ctl = p.ctl;
  if (!tie_direct_on(p) || __ldcg(&ctl->mode) != kModeTies) return;
  if (__ldcg(&ctl->tau_ready) &&
      uint64_t(__ldcg(&ctl->dsel.bucket)) > uint64_t(kTieSCap) * B) {
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->tie_fast_bad = 1;
    return;
  }
  const uint32_t tau = __ldcg(&ctl->tau);
  bool tstop = false;
  for (int64_t b0 = int64_t(blockIdx.x) * kThreads + (threadIdx.x & ~31u); b0 < p.S && !tstop;
       b0 += int64_t(gridDim.x) * kThreads) {
    const int64_t i = b0 + lane_id();
    bool in = false;
    if (i < p.S) {
      uint32_t dk[B];
      load_dkeys<B>(p.dkeys, i, dk);
      bool eq = false;
#pragma unroll
      for (int j = 0; j < B; ++j) eq |= dk[j] == tau;
      const bool scanned = dk[B - 1] > tau && sub_len(i, p.alpha, p.n) > B;
      in = eq && !scanned;
    }
    tie_append(in, static_cast<uint32_t>(i), &ctl->ts_count, ctl->ts, kTieSCap, ctl, tstop);
  }
}

// Direct tie path, step 2 (one warp per subrange): every key equal to tau
// lies in a listed subrange (one holding a delegate equal to tau, outside
// the scan) or in a scanned one. A listed subrange whose beta-th delegate is below
// tau (or that holds at most beta keys) has all its ties among its
// delegates: each is placed by a vote over its 32-key segment; any other
// listed subrange, and every scanned one, is read whole (8 loads per lane
// in flight). Positions go to Ctl::tc; an overflow leaves the ties to the
// tile pipeline. The last block ranks the positions (tie_direct).
template <int DT, int B>
__global__ void __launch_bounds__(kThreads) filter_ties_kernel(FilterParams p) {
  Ctl* ctl = p.ctl;
  if (!tie_direct_on(p) || __ldcg(&ctl->mode) != kModeTies || __ldcg(&ctl->tie_fast_bad)) return;
  const int64_t nts = __ldcg(&ctl->ts_count);
  const int64_t nsc = __ldcg(&ctl->scanq_count);
  if (nsc > kTieScanMax) return;  // uniform: the tile pipeline takes the ties
  const uint32_t tau = __ldcg(&ctl->tau);
  const int alpha = p.alpha;
  const uint32_t lane = lane_id();
  const int64_t gw = (int64_t(blockIdx.x) * kThreads + threadIdx.x) >> 5;
  const int64_t nw = int64_t(gridDim.x) * (kThreads / 32);
  bool tstop = false;
  uint32_t reads = 0;
  for (int64_t e = gw; e < nts + nsc && !tstop; e += nw) {
    const int64_t i = e < nts ? __ldcg(&ctl->ts[e]) : __ldg(p.scanq + (e - nts));
    const int64_t lo = i << alpha;
    const int64_t len = sub_len(i, alpha, p.n);
    uint32_t dk[B];
    uint16_t ds[B];
    bool rd = e >= nts;
    if (!rd) {
#pragma unroll
      for (int z = 0; z < B; ++z) {
        dk[z] = p.dkeys[i * B + z];
        ds[z] = p.dsegs[i * B + z];
      }
      rd = dk[B - 1] == tau && len > B;
    }
    if (rd) {
      ++reads;
      for (int64_t off = 0; off < len && !tstop; off += 256) {
        uint32_t x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int64_t o = off + q * 32 + lane;
          x[q] = o < len ? __ldg(p.keys + lo + o) : 0u;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int64_t o = off + q * 32 + lane;
          tie_append(o < len && map_key<DT>(x[q]) == tau, static_cast<uint32_t>(lo + o),
                     &ctl->tc_count, ctl->tc, kTieCandCap, ctl, tstop);
        }
      }
    } else {
      // the delegates equal to tau: the occurrence-th such key of the segment
      const int64_t gran = alpha < 5 ? (int64_t(1) << alpha) : 32;
#pragma unroll
      for (int j = 0; j < B; ++j) {
        if (j < len && dk[j] == tau) {  // uniform over the warp
          int occ = 0;
#pragma unroll
          for (int z = 0; z < B; ++z) occ += (z < j && dk[z] == tau && ds[z] == ds[j]) ? 1 : 0;
          const int64_t s0 = lo + int64_t(ds[j]) * gran;
          const int64_t s1 = imin64(imin64(p.n, s0 + gran), lo + (int64_t(1) << alpha));
          uint32_t bal = __ballot_sync(
              0xFFFFFFFFu, s0 + lane < s1 && map_key<DT>(__ldg(p.keys + s0 + lane)) == tau);
          for (int z = 0; z < occ; ++z) bal &= bal - 1;
          if (bal == 0 && lane == 0) atomicOr(&ctl->error, kErrTieRank);
          tie_append(lane == 0 && bal != 0, static_cast<uint32_t>(s0 + __ffs(bal) - 1),
                     &ctl->tc_count, ctl->tc, kTieCandCap, ctl, tstop);
        }
      }
    }
  }
  if (lane == 0 && reads) atomicAdd(&ctl->tie_reads, reads);
  if (last_block(&ctl->tie_dticket)) tie_direct(ctl, p.w);
}

// Counting pass over a large scan set (two_pass_wanted): the keys > tau by
// their fine digit (with the delegates the resolve kernel placed, already
// counted there). The last block finds the bucket b holding the k-th key
// from the top and sets cut_key = cut(b): the writing pass then keeps only
// keys >= cut_key, a superset of the answer. With fewer than k keys above
// tau every one of them is kept (ties at tau follow).
// Slot u of this thread in the scan step at virtual key `base`. VEC (key
// array 16-byte aligned): four consecutive virtual keys per 16-byte load
// (they lie in one subrange, at a multiple of 4 from its start, since
// subranges hold at least 4 keys); else one key per slot, strided.
template <bool VEC>
__device__ __forceinline__ int64_t scan_vkey(int64_t base, int u) {
  if constexpr (VEC)
    return base + 4 * (int64_t(threadIdx.x) + int64_t(kThreads) * (u >> 2)) + (u & 3);
  else
    return base + threadIdx.x + int64_t(u) * kThreads;
}

// Loads this thread's keys of the step (raw bits); bit u of *hit marks a
// slot that holds a key of the array.
template <bool VEC>
__device__ __forceinline__ void scan_load(const uint32_t* keys, int64_t n, const ScanQ& sq,
                                          int cur, int64_t base, int64_t total,
                                          uint32_t (&x)[kScanKPT], uint32_t& hit) {
  hit = 0;
  if constexpr (VEC) {
#pragma unroll
    for (int j = 0; j < kScanKPT / 4; ++j) {
      const int64_t v0 = scan_vkey<true>(base, 4 * j);
      const int64_t g0 = v0 < total ? sq.pos(cur, base, v0) : n;
      if (g0 + 3 < n) {
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(keys + g0));
        x[4 * j + 0] = w.x;
        x[4 * j + 1] = w.y;
        x[4 * j + 2] = w.z;
        x[4 * j + 3] = w.w;
        hit |= 0xFu << (4 * j);
      } else {
        // the ragged end of the array (or beyond the step)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const bool ok = g0 + e < n;
          x[4 * j + e] = ok ? __ldg(keys + g0 + e) : 0u;
          if (ok) hit |= 1u << (4 * j + e);
        }
      }
    }
  } else {
#pragma unroll
    for (int u = 0; u < kScanKPT; ++u) {
      const int64_t v = scan_vkey<false>(base, u);
      const int64_t gi = v < total ? sq.pos(cur, base, v) : n;
      const bool ok = gi < n;
      x[u] = __ldg(keys + (ok ? gi : 0));
      if (ok) hit |= 1u << u;
    }
  }
}

template <int DT, bool VEC>
__global__ void __launch_bounds__(kThreads) filter_count_kernel(FilterParams p) {
  __shared__ uint32_t fh[kFineBins];
  __shared__ uint32_t s_q[2][kScanQ];
  __shared__ uint32_t s_cnt;
  Ctl* ctl = p.ctl;
  const int64_t nq = __ldcg(&ctl->scanq_count);
  const int64_t total = nq << p.alpha;
  if (!two_pass_wanted(p.no_filter, total, p.k)) return;  // uniform over the grid
  const uint32_t nact = active_blocks(total, kScanStep);
  if (blockIdx.x >= nact) return;
  for (int i = threadIdx.x; i < kFineBins; i += kThreads) fh[i] = 0;
  if (threadIdx.x == 0) s_cnt = 0;
  const uint32_t tau = __ldcg(&ctl->tau);
  const FineGeom fg = fine_geom(ctl);
  const int64_t step = int64_t(nact) * kScanStep;
  const int64_t b0 = int64_t(blockIdx.x) * kScanStep;
  ScanQ sq{s_q, {}, nq, p.alpha};
  if (b0 < total) {
    sq.fetch(p.scanq, b0);
    sq.put(0);
  }
  __syncthreads();
  uint32_t cnt = 0;
  int cur = 0;
  for (int64_t base = b0; base < total; base += step) {
    uint32_t x[kScanKPT];
    uint32_t hit;
    scan_load<VEC>(p.keys, p.n, sq, cur, base, total, x, hit);
    const bool more = base + step < total;
    if (more) sq.fetch(p.scanq, base + step);
#pragma unroll
    for (int u = 0; u < kScanKPT; ++u) {
      const uint32_t m = map_key<DT>(x[u]);
      if (((hit >> u) & 1u) && m > tau) {
        atomicAdd(&fh[(m >> fg.sh) & (kFineBins - 1)], 1u);
        ++cnt;
      }
    }
    if (more) sq.put(cur ^ 1);
    __syncthreads();
    cur ^= 1;
  }
  cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s_cnt, cnt);
  __syncthreads();
  for (int i = threadIdx.x; i < kFineBins; i += kThreads) {
    const uint32_t v = fh[i];
    if (v) atomicAdd(&ctl->fhist[i], v);
  }
  if (threadIdx.x == 0 && s_cnt) atomicAdd(&ctl->scan_total, s_cnt);
  if (last_block_of(&ctl->cnt_ticket, nact)) {
    // the placed delegates (resolve kernel, earlier on the stream) are in
    // g_count and in fhist already
    const uint64_t g_all = uint64_t(__ldcg(&ctl->g_count)) + __ldcg(&ctl->scan_total);
    const uint64_t k = static_cast<uint64_t>(p.k);
    // thread t owns the 8 bins from the top [2047 - 8t - 7, 2047 - 8t]
    constexpr int per = kFineBins / kThreads;
    uint32_t c[per];
    uint32_t sum = 0;
#pragma unroll
    for (int j = 0; j < per; ++j) {
      c[j] = __ldcg(&ctl->fhist[kFineBins - 1 - (threadIdx.x * per + j)]);
      sum += c[j];
    }
    const uint32_t above = block_scan_excl<kThreads>(sum, nullptr);
    if (g_all >= k && above < k && uint64_t(above) + sum >= k) {
      uint32_t acc = above;
      int j = 0;
      for (; j < per - 1; ++j) {
        if (uint64_t(acc) + c[j] >= k) break;
        acc += c[j];
      }
      const uint32_t b = static_cast<uint32_t>(kFineBins - 1 - (threadIdx.x * per + j));
      ctl->cut_key = fg.pref | (b << fg.sh);
    }
    if (threadIdx.x == 0) {
      if (g_all < k) ctl->cut_key = 0u;  // every key > tau is needed
      ctl->g_all = static_cast<uint32_t>(g_all);
      ctl->two_pass = 1;
    }
  }
}

template <int DT, bool VEC>
__global__ void __launch_bounds__(kThreads) filter_scan_kernel(FilterParams p) {
  __shared__ uint32_t sh[256];
  __shared__ uint32_t s_q[2][kScanQ];
  zero_hist(sh);
  const int lvl0 = g_first_level(p.ctl, p.no_filter != 0);
  const uint32_t tau = __ldcg(&p.ctl->tau);
  // after a counting pass only keys >= cut_key are written
  const uint32_t cut = __ldcg(&p.ctl->two_pass) ? __ldcg(&p.ctl->cut_key) : 0u;
  const int64_t nq = __ldcg(&p.ctl->scanq_count);
  const int64_t total = nq << p.alpha;
  const uint32_t nact = active_blocks(total, kScanStep);
  if (blockIdx.x >= nact) return;
  RunHist rh;
  const int64_t step = int64_t(nact) * kScanStep;
  const int64_t b0 = int64_t(blockIdx.x) * kScanStep;
  ScanQ sq{s_q, {}, nq, p.alpha};
  if (b0 < total) {
    sq.fetch(p.scanq, b0);
    sq.put(0);
  }
  __syncthreads();
  const uint32_t lt = lanemask_lt();
  int cur = 0;
  for (int64_t base = b0; base < total; base += step) {
    uint32_t x[kScanKPT];
    uint32_t hit;
    scan_load<VEC>(p.keys, p.n, sq, cur, base, total, x, hit);
    const bool more = base + step < total;
    if (more) sq.fetch(p.scanq, base + step);  // in flight with this step's keys
#pragma unroll
    for (int u = 0; u < kScanKPT; ++u) {
      x[u] = map_key<DT>(x[u]);
      if (!((x[u] > tau && x[u] >= cut) || p.no_filter)) hit &= ~(1u << u);
    }
    const uint32_t wt = __reduce_add_sync(0xFFFFFFFFu, __popc(hit));
    uint32_t wb, unused;
    block_reserve2<kThreads>(&p.ctl->g_count, wt, nullptr, 0, wb, unused);
    uint32_t run = 0;
#pragma unroll
    for (int u = 0; u < kScanKPT; ++u) {
      const bool h = (hit >> u) & 1u;
      const uint32_t bal = __ballot_sync(0xFFFFFFFFu, h);
      if (h) {
        const int64_t v = scan_vkey<VEC>(base, u);
        const uint32_t slot = wb + run + __popc(bal & lt);
        const uint64_t cmp = make_comp(x[u], static_cast<uint32_t>(sq.pos(cur, base, v)));
        if (slot < p.g_cap) p.g[slot] = cmp;
        else atomicOr(&p.ctl->error, kErrOverflowG);
        rh.add(sh, comp_digit(cmp, lvl0));
      }
      run += __popc(bal);
    }
    if (more) sq.put(cur ^ 1);
    __syncthreads();
    cur ^= 1;
  }
  rh.flush(sh);
  __syncthreads();
  flush_hist(sh, p.ctl->gsel.hist[lvl0]);
  // G is complete once every active block is here: decide the mode
  if (last_block_of(&p.ctl->scan_ticket, nact)) {
    if (threadIdx.x < 32) decide_mode(p.ctl, p.k, lvl0, p.kth_only != 0);
  }
}

// --------------------------------------------------------- second select ---
// Stage s (1..8) reads the composites that match the digits selected so far
// (stage 1: all of G) and decides digit level lvl0 + s - 1, where lvl0
// leading digits are common to all of G: larger digit -> winner
// (written to W), equal -> survivor for stage s+1 (or winner when the
// bucket is exactly what is still needed), smaller -> dropped. The last
// block selects the next digit from the survivors' histogram.
struct GSelParams {
  uint64_t* g;
  uint64_t* sv;
  uint64_t* w;
  int64_t g_cap, k;
  Ctl* ctl;
  int kth_only;
};

constexpr int kGIpt = 16;
constexpr int kGCap = kThreads * kGIpt;  // one step's worth per buffer

__global__ void __launch_bounds__(kThreads) gstage_kernel(GSelParams p, int s) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeSelect) return;
  // stage s decides digit lvl0 + s - 1 (the digits before lvl0 are common
  // to all of G); k-selection stops once the four key digits are known
  const int level = static_cast<int>(__ldcg(&ctl->g_lvl0)) + s - 1;
  if (level > 7 || (p.kth_only && level > 2)) return;
  const int64_t count = (s == 1) ? imin64(__ldcg(&ctl->g_count), p.g_cap)
                                 : static_cast<int64_t>(__ldcg(&ctl->stage_count[s]));
  if (count == 0) return;  // uniform over the grid: nothing survived
  const uint32_t nact = active_blocks(count, int64_t(kThreads) * kGIpt);
  if (blockIdx.x >= nact) return;
  __shared__ uint32_t sh[256];
  extern __shared__ __align__(16) uint64_t gsm[];
  uint64_t* wbuf = gsm;           // winners staged
  uint64_t* sbuf = gsm + kGCap;   // survivors staged
  __shared__ uint32_t w_fill, s_fill;
  zero_hist(sh);
  if (threadIdx.x == 0) {
    w_fill = 0;
    s_fill = 0;
  }
  __syncthreads();
  const uint64_t* src = (s & 1) ? p.g : p.sv;
  uint64_t* dst = (s & 1) ? p.sv : p.g;
  const uint64_t prefix = __ldcg(&ctl->gsel.prefix);
  const uint32_t d = static_cast<uint32_t>(prefix >> (56 - 8 * level)) & 255u;
  const bool done = __ldcg(&ctl->gsel.done) != 0;
  const bool last = (level == 7);
  const int nsh = 48 - 8 * level;  // next digit shift
  RunHist rh;
  const int64_t stepn = int64_t(nact) * kThreads * kGIpt;
  // the next step's composites are loaded before this step's block scan and
  // staging (double-buffered in registers)
  uint64_t c[kGIpt], nc[kGIpt];
  auto load_step = [&](int64_t b) {
#pragma unroll
    for (int u = 0; u < kGIpt; ++u)
      nc[u] = __ldcg(src + imin64(b + threadIdx.x + int64_t(u) * kThreads, count - 1));
  };
  load_step(int64_t(blockIdx.x) * kThreads * kGIpt);
  for (int64_t base = int64_t(blockIdx.x) * kThreads * kGIpt; base < count; base += stepn) {
    uint32_t win = 0, sur = 0;
#pragma unroll
    for (int u = 0; u < kGIpt; ++u) c[u] = nc[u];
    if (base + stepn < count) load_step(base + stepn);
#pragma unroll
    for (int u = 0; u < kGIpt; ++u) {
      const int64_t i = base + threadIdx.x + int64_t(u) * kThreads;
      const uint32_t dg = static_cast<uint32_t>(c[u] >> (56 - 8 * level)) & 255u;
      if (i < count) {
        if (dg > d || (dg == d && (done || last))) win |= 1u << u;
        else if (dg == d) sur |= 1u << u;
      }
    }
    if (p.kth_only) win = 0;  // k-selection keeps no winners
    // one block scan reserves both staged outputs (16-bit fields)
    uint32_t tot;
    const uint32_t ex = block_scan_excl<kThreads>(__popc(win) | (__popc(sur) << 16), &tot);
    if (w_fill + (tot & 0xFFFFu) > kGCap)
      stage_flush<uint64_t, kThreads>(wbuf, &w_fill, &ctl->w_count, p.w, static_cast<uint64_t>(p.k),
                                      &ctl->error, kErrOverflowW);
    if (s_fill + (tot >> 16) > kGCap)
      stage_flush<uint64_t, kThreads>(sbuf, &s_fill, &ctl->stage_count[s + 1], dst,
                                      static_cast<uint64_t>(p.g_cap), &ctl->error, kErrOverflowG);
    uint32_t ws = w_fill + (ex & 0xFFFFu);
    uint32_t ss = s_fill + (ex >> 16);
    __syncthreads();
    if (threadIdx.x == 0) {
      w_fill += tot & 0xFFFFu;
      s_fill += tot >> 16;
    }
#pragma unroll
    for (int u = 0; u < kGIpt; ++u) {
      if (win & (1u << u)) wbuf[ws++] = c[u];
      if (sur & (1u << u)) {
        sbuf[ss++] = c[u];
        if (nsh >= 0) rh.add(sh, static_cast<uint32_t>(c[u] >> nsh) & 255u);
      }
    }
  }
  stage_flush<uint64_t, kThreads>(wbuf, &w_fill, &ctl->w_count, p.w, static_cast<uint64_t>(p.k),
                                  &ctl->error, kErrOverflowW);
  stage_flush<uint64_t, kThreads>(sbuf, &s_fill, &ctl->stage_count[s + 1], dst,
                                  static_cast<uint64_t>(p.g_cap), &ctl->error, kErrOverflowG);
  if (last || done) return;  // no further digit to select (uniform)
  rh.flush(sh);
  __syncthreads();
  flush_hist(sh, ctl->gsel.hist[level + 1]);
  if (last_block_of(&ctl->gsel.ticket[level + 1], nact)) {
    if (threadIdx.x < 32) select_digit<8>(&ctl->gsel, level + 1, 64, !p.kth_only);
  }
}

// ------------------------------------------------------------ tie path ----
// Mode kModeTies (|G| < k, the k-th key is tau): the answer is G plus the
// `need` smallest indices holding tau (reading R1). The subranges are cut
// into tiles of consecutive subranges:
//   A  per tile, a lower bound of its ties from the delegates alone (exact
//      unless some subrange's beta delegates all reach tau: "inexact");
//   B  one block: exclusive prefixes of the lower bounds, the last tile that
//      can matter (the first whose lower-bound prefix reaches `need`), and
//      the list, in index order, of the tiles up to it that hold ties or are
//      inexact; dense when most of their subranges must be read;
//   C  exact tie counts of the listed tiles (dense: whole tiles by bulk
//      copies, handed out in index order until the counted ones hold
//      `need`; sparse: the few subranges of interest, a warp each), one-block
//      prefixes of the counts in list order and the cut, then the tiles
//      before the cut write their ties to W[|G| + prefix + rank] in index
//      order, in parallel.
// Sparse ties (one tie needed among distinct keys) touch one tile; dense
// ties (all keys equal) read the tiles before the cut plus at most one
// round of tiles in flight, twice.
struct TieParams {
  const uint32_t* keys;
  int64_t n, S, k;
  int alpha;
  const uint32_t* dkeys;
  const uint16_t* dsegs;
  uint64_t* tstat;   // per list entry: flag << 32 | correction (aggregate or inclusive)
  uint32_t* tlb;     // per tile: lower bound | inexact << 31
  uint32_t* lbpre;   // per tile: exclusive prefix of the lower bounds
  uint32_t* list;    // tiles to visit, index order; bit 31: no inexact tile before
  int64_t tsub;      // subranges per tile (a power of two)
  int tsub_log;
  int64_t ntiles;
  const uint64_t* g;
  uint64_t* w;
  Ctl* ctl;
};

constexpr int kTieTileKeys = 32768;     // keys per tile (at least one subrange)
constexpr int kTieTileMaxSub = 1024;    // subranges per tile at most
constexpr int kTieMaxSeg = 2048;        // 32-key segments per tile at most (alpha = 16)
constexpr int kTiePlanChunk = 8192;     // tiles per shared-memory pass of the plan
constexpr uint32_t kTieInexact = 0x80000000u;
// tile word: bits 0-15 lower bound, 16-29 inexact subranges, 31 inexact flag
__device__ __forceinline__ uint32_t tlb_lb(uint32_t v) { return v & 0xFFFFu; }
__device__ __forceinline__ uint32_t tlb_ninex(uint32_t v) { return (v >> 16) & 0x3FFFu; }

// Ties at tau a subrange holds by its delegates, and whether non-delegates
// may hold more (all beta delegates reach tau and the subrange is longer).
// A delegate slot is real iff its index is below the subrange's length (the
// delegate pass pads only the slots a short subrange cannot fill), so the
// segment ids are not read here.
template <int B>
__device__ __forceinline__ uint32_t tie_lb_of(const TieParams& p, int64_t i, uint32_t tau,
                                              bool* inexact) {
  uint32_t dk[B];
#pragma unroll
  for (int j = 0; j < B; ++j) dk[j] = p.dkeys[i * B + j];
  uint32_t c = 0;
  *inexact = false;
  if (dk[0] >= tau) {
    const int64_t len = sub_len(i, p.alpha, p.n);
#pragma unroll
    for (int j = 0; j < B; ++j) c += (dk[j] == tau && j < len) ? 1u : 0u;
    *inexact = dk[B - 1] >= tau && len > B;
  }
  return c;
}

// A warp owns whole tiles: chunks of max(tsub, 32) consecutive subranges
// (one tile, or 32 / tsub tiles of tsub lanes each), 8 subranges in flight
// per lane. Each subrange adds (ties it surely holds) | (inexact << 16) to
// its lane's sum; the sums of a tile are reduced in the warp and its word is
// stored whole (no atomics, no block barrier).
template <int B>
__global__ void __launch_bounds__(kThreads) tie_lb_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies || __ldcg(&ctl->tie_fast)) return;
  const uint32_t tau = __ldcg(&ctl->tau);
  const uint32_t lane = lane_id();
  constexpr int kU = 8;
  const int grp = p.tsub < 32 ? static_cast<int>(p.tsub) : 32;
  const int64_t csub = p.tsub < 32 ? 32 : p.tsub;
  const int64_t nchunks = (p.S + csub - 1) / csub;
  const int64_t nw = int64_t(gridDim.x) * (kThreads / 32);
  for (int64_t ch = int64_t(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5); ch < nchunks;
       ch += nw) {
    const int64_t i0 = ch * csub;
    const int64_t i1 = imin64(p.S, i0 + csub);
    uint32_t acc = 0;
    for (int64_t b = i0; b < i1; b += 32 * kU) {
      uint32_t dk[kU][B];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t i = b + u * 32 + lane;
        if (i < i1) {
          load_dkeys<B>(p.dkeys, i, dk[u]);
        } else {
#pragma unroll
          for (int q = 0; q < B; ++q) dk[u][q] = 0u;
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int64_t i = b + u * 32 + lane;
        if (i < i1 && dk[u][0] >= tau) {
          const int64_t len = sub_len(i, p.alpha, p.n);
          uint32_t c = 0;
#pragma unroll
          for (int q = 0; q < B; ++q) c += (dk[u][q] == tau && q < len) ? 1u : 0u;
          const uint32_t x = (dk[u][B - 1] >= tau && len > B) ? 1u : 0u;
          acc += c | (x << 16);
        }
      }
    }
    // lb <= B * tsub <= 4096 and inexact <= tsub <= 1024: the packed sums
    // cannot carry into each other
    if (grp == 32) {
      acc = __reduce_add_sync(0xFFFFFFFFu, acc);
    } else {
      for (int o = 1; o < grp; o <<= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    }
    const int64_t first = i0 + (grp == 32 ? 0 : int64_t(lane));
    if ((lane & (grp - 1)) == 0 && first < p.S) {
      const uint32_t ninex = acc >> 16;
      p.tlb[first >> p.tsub_log] = (acc & 0xFFFFu) | (ninex << 16) | (ninex ? kTieInexact : 0u);
    }
  }
}

// The tile words are staged through shared memory in chunks (coalesced
// global reads and writes); each thread scans 8 consecutive tiles of a chunk.
__global__ void __launch_bounds__(1024) tie_plan_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies || __ldcg(&ctl->tie_fast)) return;
  const uint32_t need = __ldcg(&ctl->need);
  constexpr int kPer = kTiePlanChunk / 1024;
  __shared__ uint32_t buf[kTiePlanChunk + kTiePlanChunk / 32];  // padded: no bank conflicts
  __shared__ int64_t s_last;
  auto pad = [](int j) { return j + (j >> 5); };
  const int64_t nt = p.ntiles;
  const int tid = threadIdx.x;
  if (tid == 0) s_last = nt - 1;
  // pass 1: exclusive prefixes of the lower bounds; the first tile whose
  // inclusive prefix reaches `need` is the last one that can matter
  uint32_t base = 0;
  for (int64_t c0 = 0; c0 < nt; c0 += kTiePlanChunk) {
    const int cn = static_cast<int>(imin64(kTiePlanChunk, nt - c0));
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      const int j = e * 1024 + tid;
      if (j < cn) buf[pad(j)] = tlb_lb(p.tlb[c0 + j]);
    }
    __syncthreads();
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      const int j = tid * kPer + e;
      v[e] = j < cn ? buf[pad(j)] : 0u;
      sum += v[e];
    }
    uint32_t tot;
    uint32_t run = base + block_scan_excl<1024>(sum, &tot);
    int64_t first = -1;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      const int j = tid * kPer + e;
      if (j < cn) {
        buf[pad(j)] = run;
        if (first < 0 && run + v[e] >= need) first = c0 + j;
      }
      run += v[e];
    }
    if (first >= 0)
      atomicMin(reinterpret_cast<unsigned long long*>(&s_last), static_cast<unsigned long long>(first));
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      const int j = e * 1024 + tid;
      if (j < cn) p.lbpre[c0 + j] = buf[pad(j)];
    }
    base += tot;
    __syncthreads();
  }
  const int64_t last = s_last;
  // pass 2: the list of tiles up to `last` that hold ties or are inexact,
  // each marked when no inexact tile precedes it
  uint32_t lbase = 0, xbase = 0;
  uint64_t nin = 0;  // inexact subranges up to `last` (this thread's share)
  for (int64_t c0 = 0; c0 <= last; c0 += kTiePlanChunk) {
    const int cn = static_cast<int>(imin64(kTiePlanChunk, last + 1 - c0));
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      const int j = e * 1024 + tid;
      if (j < cn) buf[pad(j)] = p.tlb[c0 + j];
    }
    __syncthreads();
    uint32_t v[kPer], ci = 0, cx = 0;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      const int j = tid * kPer + e;
      v[e] = j < cn ? buf[pad(j)] : 0u;
      ci += v[e] != 0 ? 1u : 0u;  // holds ties or is inexact
      cx += (v[e] & kTieInexact) ? 1u : 0u;
      nin += tlb_ninex(v[e]);
    }
    uint32_t ti, tx;
    uint32_t bi = lbase + block_scan_excl<1024>(ci, &ti);
    uint32_t bx = xbase + block_scan_excl<1024>(cx, &tx);
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      const int j = tid * kPer + e;
      if (j < cn && v[e] != 0)
        p.list[bi++] = static_cast<uint32_t>(c0 + j) | (bx == 0 ? kTieInexact : 0u);
      bx += (v[e] & kTieInexact) ? 1u : 0u;
    }
    lbase += ti;
    xbase += tx;
    __syncthreads();
  }
  // dense when most subranges up to `last` must be read: their tiles come
  // whole by bulk copies; else a few subranges per tile, read directly
  __shared__ unsigned long long s_nin;
  if (tid == 0) s_nin = 0;
  __syncthreads();
  if (nin) atomicAdd(&s_nin, static_cast<unsigned long long>(nin));
  __syncthreads();
  if (tid == 0) {
    ctl->tie_nlist = lbase;
    const int64_t subs = imin64(p.S, (last + 1) * p.tsub);
    ctl->tie_dense = (2 * static_cast<int64_t>(s_nin) > subs) ? 1u : 0u;
  }
}

__device__ __forceinline__ void tie_copy_g(const TieParams& p, uint32_t g) {
  // G is part of the answer, in front of the ties
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < g;
       j += int64_t(gridDim.x) * blockDim.x)
    p.w[j] = p.g[j];
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&p.ctl->w_count, g);
}

__device__ __forceinline__ void tie_finish(const TieParams& p, uint32_t read_subs,
                                           uint32_t emitted) {
  const uint32_t lane = lane_id();
  read_subs = __reduce_add_sync(0xFFFFFFFFu, read_subs);
  if (lane == 0 && read_subs) atomicAdd(&p.ctl->tie_scanned, read_subs);
  emitted = __reduce_add_sync(0xFFFFFFFFu, emitted);
  if (lane == 0 && emitted) atomicAdd(&p.ctl->w_count, emitted);
}

// Dense ties (most listed subranges must be read), in three kernels:
//   1. tie_dcount: the listed tiles are handed out in index order (ticket)
//      and their keys equal to tau counted, whole tiles streamed with
//      16-byte loads; a CTA stops once the tiles counted so far hold `need`
//      ties (every tile handed out after that lies past the cut, since the
//      counted ones all precede it);
//   2. tie_scan (shared with the sparse path): exclusive prefixes of the
//      counts in list order and the cut;
//   3. tie_dplace: the tiles before the cut, in parallel: a ballot per
//      32-key segment read straight from global memory (many segments in
//      flight per warp), prefixes over the segments, ties written from the
//      bitmasks.
constexpr int kDenseThreads = 1024;

__device__ __forceinline__ void tie_tile_range(const TieParams& p, int64_t t, int64_t* klo,
                                               int64_t* khi) {
  const int64_t i_lo = t * p.tsub;
  const int64_t nsub = imin64(p.tsub, p.S - i_lo);
  *klo = i_lo << p.alpha;
  *khi = imin64(p.n, (i_lo + nsub) << p.alpha);
}

template <int DT>
__global__ void __launch_bounds__(kDenseThreads) tie_dcount_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies || __ldcg(&ctl->tie_dense) == 0) return;
  const uint32_t tau = __ldcg(&ctl->tau);
  const uint32_t need = __ldcg(&ctl->need);
  const int64_t nl = __ldcg(&ctl->tie_nlist);
  const bool vec = (reinterpret_cast<uintptr_t>(p.keys) & 15u) == 0;
  __shared__ int64_t s_j;
  __shared__ uint32_t s_w[kDenseThreads / 32];
  const int tid = threadIdx.x;
  uint32_t read_subs = 0;
  for (;;) {
    if (tid == 0) {
      s_j = -1;
      if (__ldcg(&ctl->tie_sum) < need) {
        const int64_t j = atomicAdd(&ctl->tie_ticket, 1u);
        if (j < nl) s_j = j;
      }
    }
    __syncthreads();
    const int64_t j = s_j;
    if (j < 0) break;
    int64_t klo, khi;
    tie_tile_range(p, p.list[j] & ~kTieInexact, &klo, &khi);
    uint32_t c = 0;
    // 8 words of 4 keys per thread in flight (a 32768-key tile in one round)
    for (int64_t x0 = klo + int64_t(tid) * 4; x0 < khi; x0 += int64_t(kDenseThreads) * 32) {
      uint4 w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t x = x0 + int64_t(u) * kDenseThreads * 4;
        if (vec && x + 3 < khi) {
          w[u] = __ldg(reinterpret_cast<const uint4*>(p.keys + x));  // kept for tie_dplace
        } else {
          w[u].x = x < khi ? p.keys[x] : 0u;
          w[u].y = x + 1 < khi ? p.keys[x + 1] : 0u;
          w[u].z = x + 2 < khi ? p.keys[x + 2] : 0u;
          w[u].w = x + 3 < khi ? p.keys[x + 3] : 0u;
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t x = x0 + int64_t(u) * kDenseThreads * 4;
        c += (x < khi && map_key<DT>(w[u].x) == tau) ? 1u : 0u;
        c += (x + 1 < khi && map_key<DT>(w[u].y) == tau) ? 1u : 0u;
        c += (x + 2 < khi && map_key<DT>(w[u].z) == tau) ? 1u : 0u;
        c += (x + 3 < khi && map_key<DT>(w[u].w) == tau) ? 1u : 0u;
      }
    }
    c = __reduce_add_sync(0xFFFFFFFFu, c);
    if (lane_id() == 0) s_w[tid >> 5] = c;
    __syncthreads();
    if (tid < 32) {
      uint32_t tot = __reduce_add_sync(0xFFFFFFFFu, s_w[tid]);
      if (tid == 0) {
        p.tstat[j] = tot;
        __threadfence();
        atomicAdd(&ctl->tie_sum, tot);
        read_subs += static_cast<uint32_t>((khi - klo + (int64_t(1) << p.alpha) - 1) >> p.alpha);
      }
    }
    __syncthreads();
  }
  tie_finish(p, read_subs, 0u);
}

template <int DT>
__global__ void __launch_bounds__(kDenseThreads) tie_dplace_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies || __ldcg(&ctl->tie_dense) == 0) return;
  const uint32_t tau = __ldcg(&ctl->tau);
  const uint32_t need = __ldcg(&ctl->need);
  const uint32_t g = __ldcg(&ctl->g_count);
  const int64_t cut = ~__ldcg(&ctl->tie_cut_inv);
  const int64_t nl = imin64(__ldcg(&ctl->tie_nlist), cut);
  tie_copy_g(p, g);
  __shared__ uint32_t s_bits[kTieMaxSeg];
  __shared__ uint32_t s_pre[kTieMaxSeg];
  constexpr int kWarpsD = kDenseThreads / 32;
  constexpr int kInFlight = 32;  // segments per warp per round: a 32768-key tile in one
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const uint32_t lane = lane_id();
  const uint32_t lt = lanemask_lt();
  uint32_t emitted = 0;
  for (int64_t j = blockIdx.x; j < nl; j += gridDim.x) {
    int64_t klo, khi;
    tie_tile_range(p, p.list[j] & ~kTieInexact, &klo, &khi);
    const uint32_t E = static_cast<uint32_t>(p.tstat[j]);
    const int nseg = static_cast<int>((khi - klo + 31) >> 5);
    // segment warp + kWarpsD * q of the tile (all warps, interleaved)
    for (int q0 = 0; q0 * kWarpsD < nseg; q0 += kInFlight) {
      uint32_t v[kInFlight];
#pragma unroll
      for (int q = 0; q < kInFlight; ++q) {
        const int64_t x = klo + int64_t(warp + kWarpsD * (q0 + q)) * 32 + lane;
        v[q] = x < khi ? __ldcs(p.keys + x) : 0u;
      }
#pragma unroll
      for (int q = 0; q < kInFlight; ++q) {
        const int sg = warp + kWarpsD * (q0 + q);
        const int64_t x = klo + int64_t(sg) * 32 + lane;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, x < khi && map_key<DT>(v[q]) == tau);
        if (lane == 0 && sg < nseg) s_bits[sg] = bal;
      }
    }
    __syncthreads();
    // exclusive prefixes of the segment counts (2 consecutive per thread)
    const uint32_t c0 = 2 * tid < nseg ? __popc(s_bits[2 * tid]) : 0u;
    const uint32_t c1 = 2 * tid + 1 < nseg ? __popc(s_bits[2 * tid + 1]) : 0u;
    const uint32_t ex = block_scan_excl<kDenseThreads>(c0 + c1, nullptr);
    if (2 * tid < nseg) s_pre[2 * tid] = ex;
    if (2 * tid + 1 < nseg) s_pre[2 * tid + 1] = ex + c0;
    __syncthreads();
    for (int sg = warp; sg < nseg; sg += kDenseThreads / 32) {
      const uint32_t bits = s_bits[sg];
      const uint32_t r0 = E + s_pre[sg];
      if (bits == 0 || r0 >= need) continue;
      if ((bits >> lane) & 1u) {
        const uint32_t r = r0 + __popc(bits & lt);
        if (r < need) {
          p.w[g + r] = make_comp(tau, static_cast<uint32_t>(klo + int64_t(sg) * 32 + lane));
          ++emitted;
        }
      }
    }
    __syncthreads();  // the bitmasks are rebuilt for the next tile
  }
  tie_finish(p, 0u, emitted);
}

// Sparse ties work per tile on its few "interesting" subranges (ties among
// the delegates, or a subrange that must be read): they are listed in index
// order, counted (a warp per subrange read, coalesced 32-key votes),
// prefixed, and in step 3 written, a warp each.
struct TieSparseSmem {
  uint16_t sub[kTieTileMaxSub];  // interesting subranges, index order; bit 15: read
  uint32_t cnt[kTieTileMaxSub];  // their tie counts, then exclusive prefixes
  uint32_t n;                    // how many
};

template <int DT, int B>
__device__ uint32_t tie_sparse_tile(const TieParams& p, int64_t t, uint32_t tau,
                                    TieSparseSmem& sm, uint32_t& read_subs) {
  const int tid = threadIdx.x;
  const uint32_t lane = lane_id();
  const int warp = tid >> 5;
  const int alpha = p.alpha;
  const int64_t i_lo = t * p.tsub;
  const int nsub = static_cast<int>(imin64(p.tsub, p.S - i_lo));
  constexpr int kPerT = kTieTileMaxSub / kThreads;
  // classify kPerT consecutive subranges per thread, list them in order
  uint32_t c[kPerT];
  uint8_t flag[kPerT];  // 0 none, 1 delegates, 2 read
  uint32_t mine = 0;
#pragma unroll
  for (int e = 0; e < kPerT; ++e) {
    const int ii = tid * kPerT + e;
    c[e] = 0;
    flag[e] = 0;
    if (ii < nsub) {
      bool x;
      c[e] = tie_lb_of<B>(p, i_lo + ii, tau, &x);
      const bool rd = alpha < 5 ? (c[e] > 0 || x) : x;
      flag[e] = rd ? 2 : (c[e] > 0 ? 1 : 0);
    }
    mine += flag[e] ? 1u : 0u;
  }
  uint32_t ni;
  uint32_t pos = block_scan_excl<kThreads>(mine, &ni);
#pragma unroll
  for (int e = 0; e < kPerT; ++e) {
    if (flag[e]) {
      sm.sub[pos] = static_cast<uint16_t>((tid * kPerT + e) | (flag[e] == 2 ? 0x8000 : 0));
      sm.cnt[pos] = flag[e] == 2 ? 0u : c[e];
      ++pos;
      if (flag[e] == 2) ++read_subs;
    }
  }
  __syncthreads();
  // exact counts of the subranges read: a warp each, 4 segments in flight
  for (uint32_t q = warp; q < ni; q += kThreads / 32) {
    const uint32_t e = sm.sub[q];
    if (!(e & 0x8000)) continue;
    const int64_t i = i_lo + (e & 0x7FFF);
    const int64_t lo = i << alpha;
    const int64_t len = sub_len(i, alpha, p.n);
    uint32_t cntq = 0;
    for (int64_t off = 0; off < len; off += 128) {
      uint32_t v[4];
      bool on[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t x = off + u * 32 + lane;
        on[u] = x < len;
        v[u] = on[u] ? __ldg(p.keys + lo + x) : 0u;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        cntq += __popc(__ballot_sync(0xFFFFFFFFu, on[u] && map_key<DT>(v[u]) == tau));
    }
    if (lane == 0) sm.cnt[q] = cntq;
  }
  __syncthreads();
  // exclusive prefixes (kPerT consecutive entries per thread)
  uint32_t v[kPerT], sum = 0;
#pragma unroll
  for (int e = 0; e < kPerT; ++e) {
    const uint32_t q = tid * kPerT + e;
    v[e] = q < ni ? sm.cnt[q] : 0u;
    sum += v[e];
  }
  uint32_t tot;
  uint32_t run = block_scan_excl<kThreads>(sum, &tot);
#pragma unroll
  for (int e = 0; e < kPerT; ++e) {
    const uint32_t q = tid * kPerT + e;
    if (q < ni) sm.cnt[q] = run;  // prefix; the count is recomputed where needed
    run += v[e];
  }
  if (tid == 0) sm.n = ni;
  __syncthreads();
  return tot;
}

// Sparse ties, step 1: exact tie count of every listed tile, in parallel.
template <int DT, int B>
__global__ void __launch_bounds__(kThreads, 4) tie_count_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies || __ldcg(&ctl->tie_dense) != 0 || __ldcg(&ctl->tie_fast))
    return;
  const uint32_t tau = __ldcg(&ctl->tau);
  const int64_t nl = __ldcg(&ctl->tie_nlist);
  __shared__ TieSparseSmem sm;
  uint32_t read_subs = 0;
  for (int64_t j = blockIdx.x; j < nl; j += gridDim.x) {
    const int64_t t = p.list[j] & ~kTieInexact;
    const uint32_t tot = tie_sparse_tile<DT, B>(p, t, tau, sm, read_subs);
    if (threadIdx.x == 0) p.tstat[j] = tot;
  }
}

// Ties, step 2 (one block, dense and sparse): exclusive prefixes of the
// tiles' exact counts in list order (in place), and the cut.
__global__ void __launch_bounds__(1024) tie_scan_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies || __ldcg(&ctl->tie_fast)) return;
  const uint32_t need = __ldcg(&ctl->need);
  const int64_t nl = __ldcg(&ctl->tie_nlist);
  constexpr int kPer = kTiePlanChunk / 1024;
  __shared__ uint32_t buf[kTiePlanChunk + kTiePlanChunk / 32];
  __shared__ int64_t s_cut;
  auto pad = [](int j) { return j + (j >> 5); };
  const int tid = threadIdx.x;
  if (tid == 0) s_cut = nl;
  uint64_t base = 0;
  for (int64_t c0 = 0; c0 < nl; c0 += kTiePlanChunk) {
    const int cn = static_cast<int>(imin64(kTiePlanChunk, nl - c0));
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      const int jj = e * 1024 + tid;
      if (jj < cn) buf[pad(jj)] = static_cast<uint32_t>(p.tstat[c0 + jj]);
    }
    __syncthreads();
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      const int jj = tid * kPer + e;
      v[e] = jj < cn ? buf[pad(jj)] : 0u;
      sum += v[e];
    }
    uint32_t tot;
    uint64_t run = base + block_scan_excl<1024>(sum, &tot);
    int64_t cut = -1;
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      const int jj = tid * kPer + e;
      if (jj < cn) {
        buf[pad(jj)] = static_cast<uint32_t>(run < need ? run : need);
        if (cut < 0 && run >= need) cut = c0 + jj;
      }
      run += v[e];
    }
    if (cut >= 0) atomicMin(reinterpret_cast<unsigned long long*>(&s_cut), static_cast<unsigned long long>(cut));
    __syncthreads();
#pragma unroll
    for (int e = 0; e < kPer; ++e) {
      const int jj = e * 1024 + tid;
      if (jj < cn) p.tstat[c0 + jj] = buf[pad(jj)];
    }
    base += tot;
    __syncthreads();
  }
  if (tid == 0) ctl->tie_cut_inv = ~static_cast<uint32_t>(s_cut);  // first list entry not needed
}

// Sparse ties, step 3: the tiles before the cut write their ties, in
// parallel (their prefixes are known), a warp per interesting subrange.
template <int DT, int B>
__global__ void __launch_bounds__(kThreads, 4) tie_place_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies || __ldcg(&ctl->tie_dense) != 0) return;
  if (__ldcg(&ctl->tie_fast)) {  // ties placed by the filter: G goes in front
    tie_copy_g(p, __ldcg(&ctl->g_count));
    return;
  }
  const uint32_t tau = __ldcg(&ctl->tau);
  const uint32_t need = __ldcg(&ctl->need);
  const uint32_t g = __ldcg(&ctl->g_count);
  const int64_t cut = ~__ldcg(&ctl->tie_cut_inv);
  const int64_t nl = imin64(__ldcg(&ctl->tie_nlist), cut);
  tie_copy_g(p, g);
  __shared__ TieSparseSmem sm;
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const int alpha = p.alpha;
  uint32_t read_subs = 0, emitted = 0;
  for (int64_t j = blockIdx.x; j < nl; j += gridDim.x) {
    const int64_t t = p.list[j] & ~kTieInexact;
    const uint32_t E = static_cast<uint32_t>(p.tstat[j]);
    tie_sparse_tile<DT, B>(p, t, tau, sm, read_subs);
    const int64_t i_lo = t * p.tsub;
    for (uint32_t q = warp; q < sm.n; q += kThreads / 32) {
      const uint32_t r0 = E + sm.cnt[q];
      if (r0 >= need) continue;
      const uint32_t e = sm.sub[q];
      const int64_t i = i_lo + (e & 0x7FFF);
      if (e & 0x8000) {
        // read in index order and rank the ties
        const int64_t lo = i << alpha;
        const int64_t len = sub_len(i, alpha, p.n);
        uint32_t run = 0;
        for (int64_t off = 0; off < len && r0 + run < need; off += 32) {
          const int64_t x = off + lane;
          const bool is_t = x < len && map_key<DT>(__ldg(p.keys + lo + x)) == tau;
          const uint32_t bal = __ballot_sync(0xFFFFFFFFu, is_t);
          const uint32_t r = r0 + run + __popc(bal & lanemask_lt());
          if (is_t && r < need) {
            p.w[g + r] = make_comp(tau, static_cast<uint32_t>(lo + x));
            ++emitted;
          }
          run += __popc(bal);
        }
      } else {
        // every tie is a delegate: D lists equal keys in index order; the
        // position is the occurrence-th key equal to tau in its segment
        uint32_t dk[B];
        uint16_t ds[B];
#pragma unroll
        for (int z = 0; z < B; ++z) {
          dk[z] = p.dkeys[i * B + z];
          ds[z] = p.dsegs[i * B + z];
        }
        uint32_t r = r0;
#pragma unroll
        for (int z = 0; z < B; ++z) {
          if (dk[z] == tau && ds[z] != kNoSeg && r < need) {
            const int o = occ_rank<B>(dk, ds, z);
            const int64_t lo = (i << alpha) + int64_t(ds[z]) * 32;
            const int64_t hi = imin64(imin64(p.n, lo + 32), (i + 1) << alpha);
            const bool m = lo + lane < hi && map_key<DT>(__ldg(p.keys + lo + lane)) == tau;
            uint32_t bal = __ballot_sync(0xFFFFFFFFu, m);
            for (int y = 0; y < o; ++y) bal &= bal - 1;
            if (lane == 0) {
              if (bal == 0) atomicOr(&ctl->error, kErrTieRank);
              p.w[g + r] = make_comp(tau, static_cast<uint32_t>(lo + (bal ? __ffs(bal) - 1 : 0)));
              ++emitted;
            }
            ++r;
          }
        }
      }
    }
    __syncthreads();
  }
  tie_finish(p, read_subs, emitted);
}

// ----------------------------------------------------------- k-th output ---
__global__ void write_kth_kernel(Ctl* ctl, int dtype, uint32_t* out, uint32_t* err_out) {
  report_errors(ctl, err_out);
  const uint32_t mode = __ldcg(&ctl->mode);
  const uint32_t m = (mode == kModeTies) ? __ldcg(&ctl->tau)
                                         : static_cast<uint32_t>(__ldcg(&ctl->gsel.prefix) >> 32);
  ctl->kth_mapped = m;
  if (out) *out = unmap_key(dtype, m);
}

// Self-test of the bounded waits: one CTA waits on an mbarrier phase that
// nothing completes, with the wait the bulk-copy rings use, and reports the
// timeout through the report word the way a query's last kernel does.
__global__ void wait_selftest_kernel(uint64_t limit_ns, uint32_t* err_out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
  if (!ok && threadIdx.x == 0 && err_out) {
    volatile uint32_t* q = err_out;
    *q = *q | kErrTimeout;
    __threadfence_system();
  }
}

// ------------------------------------------------- delegate stage output ---
template <int DT, int B>
__global__ void resolve_kernel(const uint32_t* keys, int64_t n, int64_t S, int alpha,
                               const uint32_t* dkeys, const uint16_t* dsegs, int32_t* d_idx) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= S) return;
  uint32_t dk[B];
  uint16_t ds[B];
#pragma unroll
  for (int j = 0; j < B; ++j) {
    dk[j] = dkeys[i * B + j];
    ds[j] = dsegs[i * B + j];
  }
#pragma unroll
  for (int j = 0; j < B; ++j) {
    if (ds[j] == kNoSeg) {
      d_idx[i * B + j] = -1;
    } else {
      const int r = occ_rank<B>(dk, ds, j);
      d_idx[i * B + j] = static_cast<int32_t>(resolve_pos<DT>(keys, n, alpha, i, ds[j], dk[j], r));
    }
  }
}

}  // namespace


cudaError_t launch_threshold(const Work& w, int sms, cudaStream_t s) {
  const int64_t count = w.S * w.beta;
  const int g1 = grid_for(count, kThreads * 16, sms, 4);
  // the one-value shortcut after digit 1 is off under the ablation that
  // stops the select one digit early (its tau must stay the truncated one)
  thr_compact_kernel<<<g1, kThreads, 0, s>>>(w.dkeys, count, w.ds, w.ctl,
                                             (w.ablate & kAblateSkipLastDigit) ? 0 : 1,
                                             w.rec_keys, w.beta);
  const int g2 = grid_for(count, kThreads * 8, sms, 4);
  // the shortcut stops after digit 2: tau = the k-th delegate's top 24 bits
  // (low byte 0), a lower threshold, still exact (the tie reading holds for
  // any tau with at least k keys >= tau)
  const bool skip_last = (w.ablate & kAblateSkipLastDigit) != 0;
  thr_pass_kernel<<<g2, kThreads, 0, s>>>(w.ds, w.dkeys, count, w.ctl, 2, skip_last ? 2 : 3,
                                          w.rec_keys, w.beta);
  if (!skip_last)
    thr_pass_kernel<<<g2, kThreads, 0, s>>>(w.ds, w.dkeys, count, w.ctl, 3, 3, w.rec_keys, w.beta);
  note_launch(skip_last ? 2 : 3);
  return cudaGetLastError();
}

// fb: the work of a query whose delegate pass may have stored records
// only; in tie mode its full delegate arrays are written before the tie
// path reads them (nullptr: not such a query)
template <int DT, int B>
static void filter_t(const FilterParams& p, int g1, int g2, int g3, int g4, int g5,
                     cudaStream_t s, const Work* fb, int sms) {
  filter_classify_kernel<DT, B><<<g1, kThreads, 0, s>>>(p);
  filter_resolve_kernel<DT, B><<<g3, kThreads, 0, s>>>(p);
  if ((reinterpret_cast<uintptr_t>(p.keys) & 15u) == 0) {
    filter_count_kernel<DT, true><<<g2, kThreads, 0, s>>>(p);
    filter_scan_kernel<DT, true><<<g2, kThreads, 0, s>>>(p);
  } else {
    filter_count_kernel<DT, false><<<g2, kThreads, 0, s>>>(p);
    filter_scan_kernel<DT, false><<<g2, kThreads, 0, s>>>(p);
  }
  if (fb) launch_delegates_fallback(*fb, p.keys, 2, sms, s);
  filter_tfind_kernel<B><<<g5, kThreads, 0, s>>>(p);
  filter_ties_kernel<DT, B><<<g4, kThreads, 0, s>>>(p);
}

cudaError_t launch_filter(const Work& w, const void* keys, bool kth_only, int sms,
                          cudaStream_t s) {
  FilterParams p;
  p.keys = static_cast<const uint32_t*>(keys);
  p.n = w.n;
  p.S = w.S;
  p.g_cap = w.g_cap;
  p.k = w.k;
  p.alpha = w.alpha;
  p.dkeys = w.dkeys;
  p.dsegs = w.dsegs;
  p.rec_keys = w.rec_keys;
  p.rec_segs = w.rec_segs;
  p.rec_sub = w.rec_sub;
  p.scanq = w.scanq;
  p.g = w.g;
  p.ctl = w.ctl;
  p.kth_only = kth_only ? 1 : 0;
  p.no_filter = (w.ablate & kAblateNoFilter) ? 1 : 0;
  p.rq = w.rq;
  p.rq_cap = w.rq_cap;
  p.w = w.w;
  const int g1 = grid_for(w.S, kThreads, sms, 8);
  // requests to resolve: at most rq_cap, one per thread per block step
  const int g3 = grid_for(w.rq_cap, kThreads, sms, 4);
  // scanned keys are bounded by the G capacity (or n when tau = 0)
  const int g2 = grid_for(w.g_cap, kScanStep, sms, 6);
  // direct tie path: a warp per listed or scanned subrange
  const int g4 = grid_for(int64_t(kTieSCap) + kTieScanMax, kThreads / 32, sms, 1);
  const int g5 = grid_for(w.S, kThreads, sms, 4);
  const Work* fb = (!kth_only && spec_eligible(w, keys)) ? &w : nullptr;
#define DRTOPK_FILTER_CASE(DTV)                              \
  switch (w.beta) {                                          \
    case 1: filter_t<DTV, 1>(p, g1, g2, g3, g4, g5, s, fb, sms); break;       \
    case 2: filter_t<DTV, 2>(p, g1, g2, g3, g4, g5, s, fb, sms); break;       \
    case 3: filter_t<DTV, 3>(p, g1, g2, g3, g4, g5, s, fb, sms); break;       \
    default: filter_t<DTV, 4>(p, g1, g2, g3, g4, g5, s, fb, sms); break;      \
  }
  switch (w.dtype) {
    case DRTOPK_U32: DRTOPK_FILTER_CASE(DRTOPK_U32); break;
    case DRTOPK_I32: DRTOPK_FILTER_CASE(DRTOPK_I32); break;
    case DRTOPK_F32: DRTOPK_FILTER_CASE(DRTOPK_F32); break;
    case DRTOPK_U32 | kSmallest: DRTOPK_FILTER_CASE(DRTOPK_U32 | kSmallest); break;
    case DRTOPK_I32 | kSmallest: DRTOPK_FILTER_CASE(DRTOPK_I32 | kSmallest); break;
    case DRTOPK_F32 | kSmallest: DRTOPK_FILTER_CASE(DRTOPK_F32 | kSmallest); break;
    default: return cudaErrorInvalidValue;
  }
#undef DRTOPK_FILTER_CASE
  note_launch(6);
  return cudaGetLastError();
}

int64_t tie_tile_subs(int alpha) {
  const int64_t t = kTieTileKeys >> alpha;
  return t < 1 ? 1 : (t > kTieTileMaxSub ? kTieTileMaxSub : t);
}
int64_t tie_tiles(int64_t S, int alpha) {
  const int64_t t = tie_tile_subs(alpha);
  return (S + t - 1) / t;
}
size_t tie_bytes(int64_t S, int alpha) { return static_cast<size_t>(tie_tiles(S, alpha)) * 20; }

cudaError_t launch_ties(const Work& w, const void* keys, int sms, cudaStream_t s) {
  TieParams p;
  p.keys = static_cast<const uint32_t*>(keys);
  p.n = w.n;
  p.S = w.S;
  p.k = w.k;
  p.alpha = w.alpha;
  p.dkeys = w.dkeys;
  p.dsegs = w.dsegs;
  p.tsub = tie_tile_subs(w.alpha);
  p.tsub_log = 0;
  while ((int64_t(1) << p.tsub_log) < p.tsub) ++p.tsub_log;
  p.ntiles = tie_tiles(w.S, w.alpha);
  p.tstat = w.tstat;
  p.tlb = reinterpret_cast<uint32_t*>(w.tstat + p.ntiles);
  p.lbpre = p.tlb + p.ntiles;
  p.list = p.lbpre + p.ntiles;
  p.g = w.g;
  p.w = w.w;
  p.ctl = w.ctl;
  // look-back words and tile lower bounds start at zero
  cudaError_t e = cudaMemsetAsync(w.tstat, 0, static_cast<size_t>(p.ntiles) * 12, s);
  if (e != cudaSuccess) return e;
  // tie_lb: one warp per chunk of max(tsub, 32) subranges
  const int64_t lb_chunks = (p.S + std::max<int64_t>(p.tsub, 32) - 1) / std::max<int64_t>(p.tsub, 32);
  const int ga = static_cast<int>(
      std::min<int64_t>((lb_chunks + kThreads / 32 - 1) / (kThreads / 32), int64_t(sms) * 8));
  const int gd = static_cast<int>(std::min<int64_t>(p.ntiles, int64_t(sms) * 2));
  const int gs = static_cast<int>(std::min<int64_t>(p.ntiles, int64_t(sms) * 4));
#define DRTOPK_TIE_CASE(DTV, BV)                                                       \
  tie_lb_kernel<BV><<<ga, kThreads, 0, s>>>(p);                                        \
  tie_plan_kernel<<<1, 1024, 0, s>>>(p);                                               \
  tie_dcount_kernel<DTV><<<gd, kDenseThreads, 0, s>>>(p);                              \
  tie_count_kernel<DTV, BV><<<gs, kThreads, 0, s>>>(p);                                \
  tie_scan_kernel<<<1, 1024, 0, s>>>(p);                                               \
  tie_dplace_kernel<DTV><<<gd, kDenseThreads, 0, s>>>(p);                              \
  tie_place_kernel<DTV, BV><<<gs, kThreads, 0, s>>>(p);
#define DRTOPK_TIE_BETA(DTV)                    \
  switch (w.beta) {                             \
    case 1: DRTOPK_TIE_CASE(DTV, 1) break;      \
    case 2: DRTOPK_TIE_CASE(DTV, 2) break;      \
    case 3: DRTOPK_TIE_CASE(DTV, 3) break;      \
    default: DRTOPK_TIE_CASE(DTV, 4) break;     \
  }
  switch (w.dtype) {
    case DRTOPK_U32: DRTOPK_TIE_BETA(DRTOPK_U32); break;
    case DRTOPK_I32: DRTOPK_TIE_BETA(DRTOPK_I32); break;
    case DRTOPK_F32: DRTOPK_TIE_BETA(DRTOPK_F32); break;
    case DRTOPK_U32 | kSmallest: DRTOPK_TIE_BETA(DRTOPK_U32 | kSmallest); break;
    case DRTOPK_I32 | kSmallest: DRTOPK_TIE_BETA(DRTOPK_I32 | kSmallest); break;
    case DRTOPK_F32 | kSmallest: DRTOPK_TIE_BETA(DRTOPK_F32 | kSmallest); break;
    default: return cudaErrorInvalidValue;
  }
#undef DRTOPK_TIE_BETA
#undef DRTOPK_TIE_CASE
  note_launch(7);
  return cudaGetLastError();
}

cudaError_t launch_gselect(const Work& w, bool kth_only, int sms, cudaStream_t s) {
  GSelParams p;
  p.g = w.g;
  p.sv = w.sv;
  p.w = w.w;
  p.g_cap = w.g_cap;
  p.k = w.k;
  p.ctl = w.ctl;
  p.kth_only = kth_only ? 1 : 0;
  const int grid = grid_for(w.g_cap, kThreads * kGIpt, sms, 2);
  const size_t dsm = size_t(2) * kGCap * sizeof(uint64_t);
  cudaFuncSetAttribute(gstage_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(dsm));
  // k-selection needs the 4 key digits (stages 1-3 decide digits 0-2 and
  // select digit 3); top-k resolves all 8 digits of the composite.
  const int last = kth_only ? 3 : 8;
  for (int st = 1; st <= last; ++st) gstage_kernel<<<grid, kThreads, dsm, s>>>(p, st);
  note_launch(last);
  return cudaGetLastError();
}

cudaError_t launch_write_kth(const Work& w, void* out_kth, cudaStream_t s) {
  write_kth_kernel<<<1, 1, 0, s>>>(w.ctl, w.dtype, static_cast<uint32_t*>(out_kth), w.err_out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_wait_selftest(uint32_t timeout_us, uint32_t* err_out, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(static_cast<uint64_t>(timeout_us) * 1000ull, err_out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_resolve_delegates(const Work& w, const void* keys, int32_t* d_idx,
                                     cudaStream_t s) {
  const int64_t grid = (w.S + 255) / 256;
  const uint32_t* k = static_cast<const uint32_t*>(keys);
#define DRTOPK_RES_CASE(DTV)                                                                     \
  switch (w.beta) {                                                                              \
    case 1: resolve_kernel<DTV, 1><<<grid, 256, 0, s>>>(k, w.n, w.S, w.alpha, w.dkeys, w.dsegs, d_idx); break; \
    case 2: resolve_kernel<DTV, 2><<<grid, 256, 0, s>>>(k, w.n, w.S, w.alpha, w.dkeys, w.dsegs, d_idx); break; \
    case 3: resolve_kernel<DTV, 3><<<grid, 256, 0, s>>>(k, w.n, w.S, w.alpha, w.dkeys, w.dsegs, d_idx); break; \
    default: resolve_kernel<DTV, 4><<<grid, 256, 0, s>>>(k, w.n, w.S, w.alpha, w.dkeys, w.dsegs, d_idx); break; \
  }
  switch (w.dtype) {
    case DRTOPK_U32: DRTOPK_RES_CASE(DRTOPK_U32); break;
    case DRTOPK_I32: DRTOPK_RES_CASE(DRTOPK_I32); break;
    default: DRTOPK_RES_CASE(DRTOPK_F32); break;
  }
#undef DRTOPK_RES_CASE
  note_launch();
  return cudaGetLastError();
}

}  // namespace drtopk
