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
// GB300 organisation: every variable-size output is appended with one
// atomic per block (block_append); uneven work (scanned subranges, tie
// counts) goes through global queues that all warps of the grid drain; each
// radix pass keeps only the survivors of the previous digit.
#include "common.cuh"
#include "launch.h"

namespace drtopk {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kInexact = 0x80000000u;  // tie count is a lower bound
constexpr uint32_t kScanned = 0x40000000u;  // tie count came from a scan
constexpr uint32_t kCountMask = 0x3FFFFFFFu;
constexpr int kTieSubPerThread = 8;
constexpr int kTieSubPerBlock = kThreads * kTieSubPerThread;
constexpr int kScanKPT = 32;  // virtual keys per thread per filter-scan step

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

int grid_for(int64_t work, int per_block, int sms, int per_sm) {
  int64_t g = (work + per_block - 1) / per_block;
  const int64_t cap = static_cast<int64_t>(sms) * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

// ------------------------------------------------------------ threshold ---
// Digit 1 pass: keep the delegate keys whose first digit is the selected
// one (compacted into ds) and histogram their second digit.
__global__ void __launch_bounds__(kThreads) thr_compact_kernel(const uint32_t* dkeys,
                                                               int64_t count, uint32_t* ds,
                                                               Ctl* ctl) {
  __shared__ uint32_t sh[256];
  zero_hist(sh);
  __syncthreads();
  SelState<4>* st = &ctl->dsel;
  const uint32_t d0 = static_cast<uint32_t>(__ldcg(&st->prefix)) >> 24;
  RunHist rh;
  const int64_t step = int64_t(gridDim.x) * kThreads * 16;
  for (int64_t base = int64_t(blockIdx.x) * kThreads * 16; base < count; base += step) {
    uint32_t v[16];
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i0 = base + (int64_t(q) * kThreads + threadIdx.x) * 4;
      if (i0 + 3 < count) {
        const uint4 x = __ldcg(reinterpret_cast<const uint4*>(dkeys + i0));
        v[q * 4 + 0] = x.x; v[q * 4 + 1] = x.y; v[q * 4 + 2] = x.z; v[q * 4 + 3] = x.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) v[q * 4 + e] = (i0 + e < count) ? dkeys[i0 + e] : 0u;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const bool ok = (i0 + e < count) && ((v[q * 4 + e] >> 24) == d0);
        c += ok;
      }
    }
    uint32_t slot = block_append<kThreads>(&ctl->ds_count, c);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t i0 = base + (int64_t(q) * kThreads + threadIdx.x) * 4;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const uint32_t x = v[q * 4 + e];
        if ((i0 + e < count) && ((x >> 24) == d0)) {
          ds[slot++] = x;
          rh.add(sh, (x >> 16) & 255u);
        }
      }
    }
  }
  rh.flush(sh);
  __syncthreads();
  flush_hist(sh, st->hist[1]);
  if (last_block(&st->ticket[1])) {
    if (threadIdx.x < 32) select_digit<4>(st, 1, 32, false);
  }
}

// Digit 2 and 3 passes over the compacted survivors.
__global__ void __launch_bounds__(kThreads) thr_pass_kernel(const uint32_t* ds, Ctl* ctl,
                                                            int pass) {
  __shared__ uint32_t sh[256];
  zero_hist(sh);
  __syncthreads();
  SelState<4>* st = &ctl->dsel;
  const int64_t count = __ldcg(&ctl->ds_count);
  const uint32_t prefix = static_cast<uint32_t>(__ldcg(&st->prefix));
  const uint32_t mask = 0xFFFFFFFFu << (32 - 8 * pass);
  const uint32_t want = prefix & mask;
  const int sh_d = 24 - 8 * pass;
  RunHist rh;
  for (int64_t i = int64_t(blockIdx.x) * kThreads + threadIdx.x; i < count;
       i += int64_t(gridDim.x) * kThreads) {
    const uint32_t x = ds[i];
    if ((x & mask) == want) rh.add(sh, (x >> sh_d) & 255u);
  }
  rh.flush(sh);
  __syncthreads();
  flush_hist(sh, st->hist[pass]);
  if (last_block(&st->ticket[pass])) {
    if (threadIdx.x < 32) {
      select_digit<4>(st, pass, 32, false);
      if (pass == 3 && threadIdx.x == 0) {
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
  uint32_t* scanq;
  uint64_t* g;
  Ctl* ctl;
  int kth_only;
};

// One thread per subrange: skip it (m^0 <= tau), queue it for a scan
// (m^{beta-1} > tau: Rule 3 says every element may qualify) or emit its
// delegates > tau (Rule 3: they are all of its elements > tau).
template <int DT, int B>
__global__ void __launch_bounds__(kThreads) filter_classify_kernel(FilterParams p) {
  __shared__ uint32_t sh[256];
  zero_hist(sh);
  __syncthreads();
  const uint32_t tau = __ldcg(&p.ctl->tau);
  const int alpha = p.alpha;
  uint32_t nscan = 0;
  for (int64_t base = int64_t(blockIdx.x) * kThreads; base < p.S;
       base += int64_t(gridDim.x) * kThreads) {
    const int64_t i = base + threadIdx.x;
    uint32_t dk[B];
    uint16_t ds[B];
    int cls = 0;  // 0 none, 1 delegates only, 2 scan
    if (i < p.S) {
#pragma unroll
      for (int j = 0; j < B; ++j) {
        dk[j] = p.dkeys[i * B + j];
        ds[j] = p.dsegs[i * B + j];
      }
      if (dk[0] > tau) cls = (dk[B - 1] > tau && sub_len(i, alpha, p.n) > B) ? 2 : 1;
    }
    const uint32_t qs = block_append<kThreads>(&p.ctl->scanq_count, cls == 2);
    if (cls == 2) {
      p.scanq[qs] = static_cast<uint32_t>(i);
      ++nscan;
    }
    uint64_t items[B];
    uint32_t cnt = 0;
    if (cls == 1) {
#pragma unroll
      for (int j = 0; j < B; ++j) {
        if (dk[j] > tau) {
          const int r = occ_rank<B>(dk, ds, j);
          const int64_t pos = resolve_pos<DT>(p.keys, p.n, alpha, i, ds[j], dk[j], r);
          if (pos < 0) atomicOr(&p.ctl->error, kErrTieRank);
          items[cnt++] = make_comp(dk[j], static_cast<uint32_t>(pos));
        }
      }
    }
    const uint32_t slot = block_append<kThreads>(&p.ctl->g_count, cnt);
    for (uint32_t e = 0; e < cnt; ++e) {
      const uint64_t s = uint64_t(slot) + e;
      if (s < static_cast<uint64_t>(p.g_cap)) p.g[s] = items[e];
      else atomicOr(&p.ctl->error, kErrOverflowG);
      atomicAdd(&sh[static_cast<uint32_t>(items[e] >> 56)], 1u);
    }
  }
  __syncthreads();
  flush_hist(sh, p.ctl->gsel.hist[0]);
  if (nscan) atomicAdd(&p.ctl->scanned, nscan);
}

// All queued subranges read as one virtual array of nq * 2^alpha keys,
// 8192 per block step, appended with one atomic per block step. The last
// block decides the query mode.
template <int DT>
__global__ void __launch_bounds__(kThreads) filter_scan_kernel(FilterParams p) {
  __shared__ uint32_t sh[256];
  zero_hist(sh);
  __syncthreads();
  const uint32_t tau = __ldcg(&p.ctl->tau);
  const int alpha = p.alpha;
  const int64_t nq = __ldcg(&p.ctl->scanq_count);
  const int64_t total = nq << alpha;
  const int64_t mask = (int64_t(1) << alpha) - 1;
  RunHist rh;
  const int64_t step = int64_t(gridDim.x) * kThreads * kScanKPT;
  for (int64_t base = int64_t(blockIdx.x) * kThreads * kScanKPT; base < total; base += step) {
    uint32_t x[kScanKPT];
    uint32_t hit = 0;
#pragma unroll
    for (int u = 0; u < kScanKPT; ++u) {
      const int64_t v = base + threadIdx.x + int64_t(u) * kThreads;
      x[u] = 0;
      if (v < total) {
        const int64_t gi = (int64_t(__ldg(p.scanq + (v >> alpha))) << alpha) + (v & mask);
        if (gi < p.n) {
          x[u] = map_key<DT>(__ldg(p.keys + gi));
          if (x[u] > tau) hit |= 1u << u;
        }
      }
    }
    uint32_t slot = block_append<kThreads>(&p.ctl->g_count, __popc(hit));
#pragma unroll
    for (int u = 0; u < kScanKPT; ++u) {
      if (hit & (1u << u)) {
        const int64_t v = base + threadIdx.x + int64_t(u) * kThreads;
        const int64_t gi = (int64_t(__ldg(p.scanq + (v >> alpha))) << alpha) + (v & mask);
        if (slot < p.g_cap) p.g[slot] = make_comp(x[u], static_cast<uint32_t>(gi));
        else atomicOr(&p.ctl->error, kErrOverflowG);
        ++slot;
        rh.add(sh, x[u] >> 24);
      }
    }
  }
  rh.flush(sh);
  __syncthreads();
  flush_hist(sh, p.ctl->gsel.hist[0]);
  if (last_block(&p.ctl->filter_ticket)) {
    if (threadIdx.x < 32) {
      Ctl* ctl = p.ctl;
      const uint32_t g = __ldcg(&ctl->g_count);
      const uint64_t k = static_cast<uint64_t>(p.k);
      if (g >= k) {
        if (threadIdx.x == 0) {
          ctl->mode = kModeSelect;
          ctl->gsel.k_rem = static_cast<uint32_t>(k);
        }
        __syncwarp();
        __threadfence();
        select_digit<8>(&ctl->gsel, 0, 64, !p.kth_only);
      } else if (threadIdx.x == 0) {
        ctl->mode = kModeTies;
        ctl->need = static_cast<uint32_t>(k - g);
        ctl->kth_mapped = tau;
      }
    }
  }
}

// --------------------------------------------------------- second select ---
// Stage s (1..8) reads the composites that match the digits selected so far
// (stage 1: all of G) and decides digit level s-1: larger digit -> winner
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

__global__ void __launch_bounds__(kThreads) gstage_kernel(GSelParams p, int s) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeSelect) return;
  const int level = s - 1;
  const int64_t count = (s == 1) ? imin64(__ldcg(&ctl->g_count), p.g_cap)
                                 : static_cast<int64_t>(__ldcg(&ctl->stage_count[s]));
  if (count == 0) return;  // uniform over the grid: nothing survived
  __shared__ uint32_t sh[256];
  zero_hist(sh);
  __syncthreads();
  const uint64_t* src = (s & 1) ? p.g : p.sv;
  uint64_t* dst = (s & 1) ? p.sv : p.g;
  const uint64_t prefix = __ldcg(&ctl->gsel.prefix);
  const uint32_t d = static_cast<uint32_t>(prefix >> (56 - 8 * level)) & 255u;
  const bool done = __ldcg(&ctl->gsel.done) != 0;
  const bool last = (level == 7);
  const int nsh = 48 - 8 * level;  // next digit shift
  RunHist rh;
  constexpr int IPT = 8;
  const int64_t stepn = int64_t(gridDim.x) * kThreads * IPT;
  for (int64_t base = int64_t(blockIdx.x) * kThreads * IPT; base < count; base += stepn) {
    uint64_t c[IPT];
    uint32_t win = 0, sur = 0;
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      const int64_t i = base + threadIdx.x + int64_t(u) * kThreads;
      c[u] = 0;
      if (i < count) {
        c[u] = src[i];
        const uint32_t dg = static_cast<uint32_t>(c[u] >> (56 - 8 * level)) & 255u;
        if (dg > d || (dg == d && (done || last))) win |= 1u << u;
        else if (dg == d) sur |= 1u << u;
      }
    }
    if (!p.kth_only) {
      uint32_t ws = block_append<kThreads>(&ctl->w_count, __popc(win));
#pragma unroll
      for (int u = 0; u < IPT; ++u) {
        if (win & (1u << u)) {
          if (ws < p.k) p.w[ws] = c[u];
          else atomicOr(&ctl->error, kErrOverflowW);
          ++ws;
        }
      }
    }
    uint32_t ss = block_append<kThreads>(&ctl->stage_count[s + 1], __popc(sur));
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
      if (sur & (1u << u)) {
        dst[ss++] = c[u];
        if (nsh >= 0) rh.add(sh, static_cast<uint32_t>(c[u] >> nsh) & 255u);
      }
    }
  }
  if (last || done) return;  // no further digit to select (uniform)
  rh.flush(sh);
  __syncthreads();
  flush_hist(sh, ctl->gsel.hist[level + 1]);
  if (last_block(&ctl->gsel.ticket[level + 1])) {
    if (threadIdx.x < 32) select_digit<8>(&ctl->gsel, level + 1, 64, !p.kth_only);
  }
}

// ------------------------------------------------------------ tie path ----
struct TieParams {
  const uint32_t* keys;
  int64_t n, S, k;
  int alpha;
  const uint32_t* dkeys;
  const uint16_t* dsegs;
  uint32_t* tcnt;
  uint32_t* bsum1;   // block sums of the lower bounds, scanned in place
  uint32_t* bsum2;   // block sums after exact counts, scanned in place
  int64_t nblk;
  uint32_t* q1;      // subranges needing an exact tie count
  uint32_t* q2;      // subranges emitting ties
  uint32_t* q2pre;   // their tie prefixes
  const uint64_t* g;
  uint64_t* w;
  Ctl* ctl;
};

// Block-wide exclusive scan of one value per thread (256 threads).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t wsum[kThreads / 32];
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
  for (int q = 0; q < kThreads / 32; ++q) {
    if (q < warp) wpre += wsum[q];
    tot += wsum[q];
  }
  __syncthreads();
  if (total) *total = tot;
  return wpre + incl - v;
}

template <int B>
__global__ void __launch_bounds__(kThreads) tie_lb_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies) return;
  const uint32_t tau = __ldcg(&ctl->tau);
  const int64_t i0 = int64_t(blockIdx.x) * kTieSubPerBlock + threadIdx.x * kTieSubPerThread;
  uint32_t sum = 0;
  for (int e = 0; e < kTieSubPerThread; ++e) {
    const int64_t i = i0 + e;
    if (i >= p.S) break;
    uint32_t dk[B];
    uint16_t ds[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
      dk[j] = p.dkeys[i * B + j];
      ds[j] = p.dsegs[i * B + j];
    }
    const int64_t len = sub_len(i, p.alpha, p.n);
    uint32_t t;
    if (dk[0] < tau) {
      t = 0;
    } else if (dk[B - 1] > tau && len > B) {
      t = kInexact;  // scanned by the filter; its ties were not counted
    } else {
      uint32_t c = 0;
#pragma unroll
      for (int j = 0; j < B; ++j) c += (dk[j] == tau && ds[j] != kNoSeg) ? 1u : 0u;
      t = c | ((dk[B - 1] == tau && len > B) ? kInexact : 0u);
    }
    p.tcnt[i] = t;
    sum += t & kCountMask;
  }
  uint32_t tot;
  block_excl_scan(sum, &tot);
  if (threadIdx.x == 0) {
    p.bsum1[blockIdx.x] = tot;
    p.bsum2[blockIdx.x] = tot;
  }
}

// Exclusive scan of nblk block sums in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) scan_blocks_kernel(uint32_t* a, int64_t nblk, Ctl* ctl) {
  if (__ldcg(&ctl->mode) != kModeTies) return;
  __shared__ uint32_t part[1024];
  const int64_t per = (nblk + 1023) / 1024;
  const int64_t lo = threadIdx.x * per;
  const int64_t hi = imin64(nblk, lo + per);
  uint32_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += a[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t v = threadIdx.x >= static_cast<unsigned>(o) ? part[threadIdx.x - o] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = part[threadIdx.x] - s;
  for (int64_t i = lo; i < hi; ++i) {
    const uint32_t v = a[i];
    a[i] = run;
    run += v;
  }
}

// Per-thread exclusive prefixes of the 8 tie counts it owns, offset by the
// block's scanned sum: pre[e] = number of ties (as counted) before subrange e.
__device__ __forceinline__ void tie_prefixes(const TieParams& p, const uint32_t* bscan,
                                             uint32_t (&t)[kTieSubPerThread],
                                             uint32_t (&pre)[kTieSubPerThread]) {
  const int64_t i0 = int64_t(blockIdx.x) * kTieSubPerBlock + threadIdx.x * kTieSubPerThread;
  uint32_t sum = 0;
#pragma unroll
  for (int e = 0; e < kTieSubPerThread; ++e) {
    const int64_t i = i0 + e;
    t[e] = (i < p.S) ? p.tcnt[i] : 0u;
    pre[e] = sum;
    sum += t[e] & kCountMask;
  }
  const uint32_t off = block_excl_scan(sum, nullptr) + bscan[blockIdx.x];
#pragma unroll
  for (int e = 0; e < kTieSubPerThread; ++e) pre[e] += off;
}

// Queue the subranges whose tie count is only a lower bound and whose
// prefix is still below `need`: only they can hold a needed tie we cannot
// place yet.
__global__ void __launch_bounds__(kThreads) tie_enqueue_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies) return;
  const uint32_t need = __ldcg(&ctl->need);
  uint32_t t[kTieSubPerThread], pre[kTieSubPerThread];
  tie_prefixes(p, p.bsum1, t, pre);
  const int64_t i0 = int64_t(blockIdx.x) * kTieSubPerBlock + threadIdx.x * kTieSubPerThread;
  uint32_t c = 0;
#pragma unroll
  for (int e = 0; e < kTieSubPerThread; ++e) c += ((t[e] & kInexact) && pre[e] < need);
  uint32_t slot = block_append<kThreads>(&ctl->tieq1_count, c);
#pragma unroll
  for (int e = 0; e < kTieSubPerThread; ++e)
    if ((t[e] & kInexact) && pre[e] < need) p.q1[slot++] = static_cast<uint32_t>(i0 + e);
}

// Exact tie counts of the queued subranges, one warp per subrange over the
// whole grid; the block sums used for the second scan are corrected in place.
template <int DT>
__global__ void __launch_bounds__(kThreads) tie_count_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies) return;
  const uint32_t tau = __ldcg(&ctl->tau);
  const int64_t nq = __ldcg(&ctl->tieq1_count);
  const uint32_t lane = lane_id();
  const int64_t warps = int64_t(gridDim.x) * (kThreads / 32);
  uint32_t done = 0;
  for (int64_t q = int64_t(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5); q < nq;
       q += warps) {
    const int64_t i = p.q1[q];
    const int64_t lo = i << p.alpha;
    const int64_t len = sub_len(i, p.alpha, p.n);
    uint32_t c = 0;
    for (int64_t off = lane; off < len; off += 32)
      c += (map_key<DT>(__ldg(p.keys + lo + off)) == tau);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (lane == 0) {
      const uint32_t old = p.tcnt[i] & kCountMask;
      p.tcnt[i] = c | kScanned;
      atomicAdd(&p.bsum2[i / kTieSubPerBlock], c - old);
      ++done;
    }
  }
  if (done) atomicAdd(&ctl->tie_scanned, done);
}

// Queue the subranges that hold needed ties (exact prefix below `need`) and
// copy G, which is part of the answer, in front of the ties in W.
__global__ void __launch_bounds__(kThreads) tie_emit_enqueue_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies) return;
  const uint32_t need = __ldcg(&ctl->need);
  const uint32_t g = __ldcg(&ctl->g_count);  // < k in this mode
  for (int64_t j = int64_t(blockIdx.x) * kThreads + threadIdx.x; j < g;
       j += int64_t(gridDim.x) * kThreads)
    p.w[j] = p.g[j];
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctl->w_count, g);
  uint32_t t[kTieSubPerThread], pre[kTieSubPerThread];
  tie_prefixes(p, p.bsum2, t, pre);
  const int64_t i0 = int64_t(blockIdx.x) * kTieSubPerBlock + threadIdx.x * kTieSubPerThread;
  uint32_t c = 0;
#pragma unroll
  for (int e = 0; e < kTieSubPerThread; ++e) c += ((t[e] & kCountMask) > 0 && pre[e] < need);
  uint32_t slot = block_append<kThreads>(&ctl->tieq2_count, c);
#pragma unroll
  for (int e = 0; e < kTieSubPerThread; ++e) {
    if ((t[e] & kCountMask) > 0 && pre[e] < need) {
      p.q2[slot] = static_cast<uint32_t>(i0 + e);
      p.q2pre[slot] = pre[e];
      ++slot;
    }
  }
}

// Emit the ties of the queued subranges in index order, one warp each.
template <int DT, int B>
__global__ void __launch_bounds__(kThreads) tie_emit_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies) return;
  const uint32_t tau = __ldcg(&ctl->tau);
  const uint32_t need = __ldcg(&ctl->need);
  const uint32_t g = __ldcg(&ctl->g_count);
  const int64_t nq = __ldcg(&ctl->tieq2_count);
  const uint32_t lane = lane_id();
  const int64_t warps = int64_t(gridDim.x) * (kThreads / 32);
  uint32_t emitted_total = 0;
  for (int64_t q = int64_t(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5); q < nq;
       q += warps) {
    const int64_t i = p.q2[q];
    const uint32_t base = p.q2pre[q];
    const uint32_t tt = p.tcnt[i];
    uint32_t emitted = 0;
    if (tt & kScanned) {
      // read the subrange in index order and rank its ties
      const int64_t lo = i << p.alpha;
      const int64_t len = sub_len(i, p.alpha, p.n);
      uint32_t run = 0;
      for (int64_t off = 0; off < len && base + run < need; off += 32) {
        const int64_t tix = off + lane;
        const bool is_t = (tix < len) && (map_key<DT>(__ldg(p.keys + lo + tix)) == tau);
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, is_t);
        const uint32_t r = base + run + __popc(bal & lanemask_lt());
        if (is_t && r < need) {
          p.w[g + r] = make_comp(tau, static_cast<uint32_t>(lo + tix));
          ++emitted;
        }
        run += __popc(bal);
      }
    } else if (lane == 0) {
      // every tie of this subrange is a delegate; D lists equal keys in
      // index order (segment, then occurrence)
      uint32_t dk[B];
      uint16_t ds[B];
#pragma unroll
      for (int j = 0; j < B; ++j) {
        dk[j] = p.dkeys[i * B + j];
        ds[j] = p.dsegs[i * B + j];
      }
      uint32_t r = base;
#pragma unroll
      for (int j = 0; j < B; ++j) {
        if (dk[j] == tau && ds[j] != kNoSeg && r < need) {
          const int o = occ_rank<B>(dk, ds, j);
          const int64_t pos = resolve_pos<DT>(p.keys, p.n, p.alpha, i, ds[j], tau, o);
          if (pos < 0) atomicOr(&ctl->error, kErrTieRank);
          p.w[g + r] = make_comp(tau, static_cast<uint32_t>(pos));
          ++r;
          ++emitted;
        }
      }
    }
    emitted_total += emitted;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) emitted_total += __shfl_xor_sync(0xFFFFFFFFu, emitted_total, o);
  if (lane == 0 && emitted_total) atomicAdd(&ctl->w_count, emitted_total);
}

// ----------------------------------------------------------- k-th output ---
__global__ void write_kth_kernel(Ctl* ctl, int dtype, uint32_t* out) {
  const uint32_t mode = __ldcg(&ctl->mode);
  const uint32_t m = (mode == kModeTies) ? __ldcg(&ctl->tau)
                                         : static_cast<uint32_t>(__ldcg(&ctl->gsel.prefix) >> 32);
  ctl->kth_mapped = m;
  if (out) *out = unmap_key(dtype, m);
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

int64_t tie_blocks(int64_t S) { return (S + kTieSubPerBlock - 1) / kTieSubPerBlock; }

cudaError_t launch_threshold(const Work& w, int sms, cudaStream_t s) {
  const int64_t count = w.S * w.beta;
  const int g1 = grid_for(count, kThreads * 16, sms, 4);
  thr_compact_kernel<<<g1, kThreads, 0, s>>>(w.dkeys, count, w.ds, w.ctl);
  const int g2 = grid_for(count, kThreads * 8, sms, 4);
  thr_pass_kernel<<<g2, kThreads, 0, s>>>(w.ds, w.ctl, 2);
  thr_pass_kernel<<<g2, kThreads, 0, s>>>(w.ds, w.ctl, 3);
  note_launch(3);
  return cudaGetLastError();
}

template <int DT, int B>
static void filter_t(const FilterParams& p, int g1, int g2, cudaStream_t s) {
  filter_classify_kernel<DT, B><<<g1, kThreads, 0, s>>>(p);
  filter_scan_kernel<DT><<<g2, kThreads, 0, s>>>(p);
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
  p.scanq = w.scanq;
  p.g = w.g;
  p.ctl = w.ctl;
  p.kth_only = kth_only ? 1 : 0;
  const int g1 = grid_for(w.S, kThreads, sms, 8);
  // scanned keys are bounded by the G capacity (or n when tau = 0)
  const int g2 = grid_for(w.g_cap, kThreads * kScanKPT, sms, 8);
#define DRTOPK_FILTER_CASE(DTV)                              \
  switch (w.beta) {                                          \
    case 1: filter_t<DTV, 1>(p, g1, g2, s); break;           \
    case 2: filter_t<DTV, 2>(p, g1, g2, s); break;           \
    case 3: filter_t<DTV, 3>(p, g1, g2, s); break;           \
    default: filter_t<DTV, 4>(p, g1, g2, s); break;          \
  }
  switch (w.dtype) {
    case DRTOPK_U32: DRTOPK_FILTER_CASE(DRTOPK_U32); break;
    case DRTOPK_I32: DRTOPK_FILTER_CASE(DRTOPK_I32); break;
    default: DRTOPK_FILTER_CASE(DRTOPK_F32); break;
  }
#undef DRTOPK_FILTER_CASE
  note_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_ties(const Work& w, const void* keys, int sms, cudaStream_t s) {
  TieParams p;
  p.keys = static_cast<const uint32_t*>(keys);
  p.n = w.n;
  p.S = w.S;
  p.k = w.k;
  p.alpha = w.alpha;
  p.dkeys = w.dkeys;
  p.dsegs = w.dsegs;
  p.tcnt = w.tcnt;
  p.nblk = tie_blocks(w.S);
  p.bsum1 = w.bsum;
  p.bsum2 = w.bsum + p.nblk;
  p.q1 = w.tieq;
  p.q2 = w.tieq + w.S;
  p.q2pre = w.scanq;  // the filter's queue is no longer needed
  p.g = w.g;
  p.w = w.w;
  p.ctl = w.ctl;
  const int grid = static_cast<int>(p.nblk);
  const int gq = grid_for(w.S, kThreads / 32, sms, 8);
#define DRTOPK_TIE_CASE(DTV)                                                        \
  switch (w.beta) {                                                                 \
    case 1: tie_lb_kernel<1><<<grid, kThreads, 0, s>>>(p); break;                   \
    case 2: tie_lb_kernel<2><<<grid, kThreads, 0, s>>>(p); break;                   \
    case 3: tie_lb_kernel<3><<<grid, kThreads, 0, s>>>(p); break;                   \
    default: tie_lb_kernel<4><<<grid, kThreads, 0, s>>>(p); break;                  \
  }                                                                                 \
  scan_blocks_kernel<<<1, 1024, 0, s>>>(p.bsum1, p.nblk, p.ctl);                    \
  tie_enqueue_kernel<<<grid, kThreads, 0, s>>>(p);                                  \
  tie_count_kernel<DTV><<<gq, kThreads, 0, s>>>(p);                                 \
  scan_blocks_kernel<<<1, 1024, 0, s>>>(p.bsum2, p.nblk, p.ctl);                    \
  tie_emit_enqueue_kernel<<<grid, kThreads, 0, s>>>(p);                             \
  switch (w.beta) {                                                                 \
    case 1: tie_emit_kernel<DTV, 1><<<gq, kThreads, 0, s>>>(p); break;              \
    case 2: tie_emit_kernel<DTV, 2><<<gq, kThreads, 0, s>>>(p); break;              \
    case 3: tie_emit_kernel<DTV, 3><<<gq, kThreads, 0, s>>>(p); break;              \
    default: tie_emit_kernel<DTV, 4><<<gq, kThreads, 0, s>>>(p); break;             \
  }
  switch (w.dtype) {
    case DRTOPK_U32: DRTOPK_TIE_CASE(DRTOPK_U32); break;
    case DRTOPK_I32: DRTOPK_TIE_CASE(DRTOPK_I32); break;
    default: DRTOPK_TIE_CASE(DRTOPK_F32); break;
  }
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
  const int grid = grid_for(w.g_cap, kThreads * 8, sms, 8);
  // k-selection needs the 4 key digits (stages 1-3 decide digits 0-2 and
  // select digit 3); top-k resolves all 8 digits of the composite.
  const int last = kth_only ? 3 : 8;
  for (int st = 1; st <= last; ++st) gstage_kernel<<<grid, kThreads, 0, s>>>(p, st);
  note_launch(last);
  return cudaGetLastError();
}

cudaError_t launch_write_kth(const Work& w, void* out_kth, cudaStream_t s) {
  write_kth_kernel<<<1, 1, 0, s>>>(w.ctl, w.dtype, static_cast<uint32_t*>(out_kth));
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
