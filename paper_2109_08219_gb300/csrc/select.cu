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

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Shared-memory histogram add, aggregated over lanes with the same bin.
__device__ __forceinline__ void hist_add(uint32_t* sh, uint32_t bin, bool active) {
  const uint32_t am = __ballot_sync(0xFFFFFFFFu, active);
  if (active) {
    const uint32_t peers = __match_any_sync(am, bin);
    if ((lanemask_lt() & peers) == 0) atomicAdd(&sh[bin], __popc(peers));
  }
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

// ------------------------------------------------------------ threshold ---
__global__ void __launch_bounds__(kThreads) thr_pass_kernel(const uint32_t* dkeys, int64_t count,
                                                            Ctl* ctl, int pass) {
  __shared__ uint32_t sh[256];
  for (int i = threadIdx.x; i < 256; i += kThreads) sh[i] = 0;
  __syncthreads();
  SelState<4>* st = &ctl->dsel;
  const uint32_t prefix = static_cast<uint32_t>(__ldcg(&st->prefix));
  const uint32_t mask = 0xFFFFFFFFu << (32 - 8 * pass);
  const uint32_t want = prefix & mask;
  const int sh_d = 24 - 8 * pass;
  const int64_t warps_total = int64_t(gridDim.x) * (kThreads / 32);
  const int64_t gw = int64_t(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5);
  const uint32_t lane = lane_id();
  for (int64_t base = gw * 128; base < count; base += warps_total * 128) {
    const int64_t i0 = base + lane * 4;
    uint32_t v[4];
    if (i0 + 3 < count) {
      const uint4 q = *reinterpret_cast<const uint4*>(dkeys + i0);
      v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[e] = (i0 + e < count) ? dkeys[i0 + e] : 0;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const bool act = (i0 + e < count) && ((v[e] & mask) == want);
      hist_add(sh, (v[e] >> sh_d) & 255u, act);
    }
  }
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
  uint64_t* g;
  Ctl* ctl;
  int kth_only;
};

template <int DT>
__device__ __forceinline__ void emit_g(const FilterParams& p, uint32_t* sh, const uint64_t* items,
                                       int cnt) {
  const uint32_t slot = warp_append(&p.ctl->g_count, cnt);
  for (int e = 0; e < cnt; ++e) {
    const uint64_t s = uint64_t(slot) + e;
    if (s < static_cast<uint64_t>(p.g_cap)) p.g[s] = items[e];
    else atomicOr(&p.ctl->error, kErrOverflowG);
  }
}

template <int DT, int B>
__global__ void __launch_bounds__(kThreads) filter_kernel(FilterParams p) {
  __shared__ uint32_t sh[256];
  for (int i = threadIdx.x; i < 256; i += kThreads) sh[i] = 0;
  __syncthreads();
  const uint32_t tau = __ldcg(&p.ctl->tau);
  const uint32_t lane = lane_id();
  const int64_t warps_total = int64_t(gridDim.x) * (kThreads / 32);
  const int64_t gw = int64_t(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5);
  const int alpha = p.alpha;

  for (int64_t base = gw * 32; base < p.S; base += warps_total * 32) {
    const int64_t i = base + lane;
    uint32_t dk[B];
    uint16_t ds[B];
    int cls = 0;  // 0 none, 1 delegates only, 2 scan
    int64_t len = 0;
    if (i < p.S) {
#pragma unroll
      for (int j = 0; j < B; ++j) {
        dk[j] = p.dkeys[i * B + j];
        ds[j] = p.dsegs[i * B + j];
      }
      len = sub_len(i, alpha, p.n);
      if (dk[0] > tau) cls = (dk[B - 1] > tau && len > B) ? 2 : 1;
    }
    // delegates-only subranges: their delegates > tau are all of {x > tau}
    uint64_t items[B];
#pragma unroll
    for (int j = 0; j < B; ++j) items[j] = 0;
    int cnt = 0;
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
    for (int e = 0; e < B; ++e) hist_add(sh, static_cast<uint32_t>(items[e < cnt ? e : 0] >> 56), e < cnt);
    emit_g<DT>(p, sh, items, cnt);

    // scanned subranges: the whole warp reads each one
    uint32_t scan_mask = __ballot_sync(0xFFFFFFFFu, cls == 2);
    if (lane == 0 && scan_mask) atomicAdd(&p.ctl->scanned, __popc(scan_mask));
    while (scan_mask) {
      const int src = __ffs(scan_mask) - 1;
      scan_mask &= scan_mask - 1;
      const int64_t si = base + src;
      const int64_t lo = si << alpha;
      const int64_t slen = sub_len(si, alpha, p.n);
      for (int64_t off = 0; off < slen; off += 128) {
        uint64_t it[4];
        int c2 = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int64_t t = off + u * 32 + lane;
          if (t < slen) {
            const uint32_t x = map_key<DT>(__ldg(p.keys + lo + t));
            if (x > tau) it[c2++] = make_comp(x, static_cast<uint32_t>(lo + t));
          }
        }
        for (int e = 0; e < 4; ++e) hist_add(sh, static_cast<uint32_t>(it[e < c2 ? e : 0] >> 56), e < c2);
        const uint32_t slot = warp_append(&p.ctl->g_count, c2);
        for (int e = 0; e < c2; ++e) {
          const uint64_t s = uint64_t(slot) + e;
          if (s < static_cast<uint64_t>(p.g_cap)) p.g[s] = it[e];
          else atomicOr(&p.ctl->error, kErrOverflowG);
        }
      }
    }
  }
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
struct GSelParams {
  uint64_t* g;
  uint64_t* sv;
  uint64_t* w;
  int64_t g_cap, k;
  Ctl* ctl;
  int kth_only;
};

__global__ void __launch_bounds__(kThreads) gpart_kernel(GSelParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeSelect) return;
  __shared__ uint32_t sh[256];
  for (int i = threadIdx.x; i < 256; i += kThreads) sh[i] = 0;
  __syncthreads();
  const uint32_t gcount =
      static_cast<uint32_t>(imin64(__ldcg(&ctl->g_count), p.g_cap));  // overflow is flagged
  const uint32_t d0 = static_cast<uint32_t>(__ldcg(&ctl->gsel.prefix) >> 56);
  const bool done0 = __ldcg(&ctl->gsel.done) != 0;
  const uint32_t lane = lane_id();
  const int64_t warps_total = int64_t(gridDim.x) * (kThreads / 32);
  const int64_t gw = int64_t(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5);
  for (int64_t base = gw * 32; base < gcount; base += warps_total * 32) {
    const int64_t i = base + lane;
    uint64_t c = 0;
    int kind = 0;  // 1 winner, 2 survivor
    if (i < gcount) {
      c = p.g[i];
      const uint32_t dg = static_cast<uint32_t>(c >> 56);
      if (dg > d0 || (dg == d0 && done0)) kind = 1;
      else if (dg == d0) kind = 2;
    }
    if (!p.kth_only) {
      const uint32_t slot = warp_append(&ctl->w_count, kind == 1);
      if (kind == 1) {
        if (slot < p.k) p.w[slot] = c;
        else atomicOr(&ctl->error, kErrOverflowW);
      }
    }
    const uint32_t s2 = warp_append(&ctl->sv_count, kind == 2);
    if (kind == 2) p.sv[s2] = c;
    hist_add(sh, static_cast<uint32_t>(c >> 48) & 255u, kind == 2);
  }
  __syncthreads();
  flush_hist(sh, ctl->gsel.hist[1]);
  if (last_block(&ctl->gsel.ticket[1])) {
    if (threadIdx.x < 32 && !done0) select_digit<8>(&ctl->gsel, 1, 64, !p.kth_only);
  }
}

__global__ void __launch_bounds__(kThreads) gpass_kernel(GSelParams p, int pass) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeSelect) return;
  if (__ldcg(&ctl->gsel.done) != 0) return;
  __shared__ uint32_t sh[256];
  for (int i = threadIdx.x; i < 256; i += kThreads) sh[i] = 0;
  __syncthreads();
  const uint32_t cnt = __ldcg(&ctl->sv_count);
  const uint64_t prefix = __ldcg(&ctl->gsel.prefix);
  const uint64_t mask = ~uint64_t(0) << (64 - 8 * pass);
  const uint64_t want = prefix & mask;
  const int sh_d = 56 - 8 * pass;
  const uint32_t lane = lane_id();
  const int64_t warps_total = int64_t(gridDim.x) * (kThreads / 32);
  const int64_t gw = int64_t(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5);
  for (int64_t base = gw * 32; base < cnt; base += warps_total * 32) {
    const int64_t i = base + lane;
    uint64_t c = 0;
    bool act = false;
    if (i < cnt) {
      c = p.sv[i];
      act = (c & mask) == want;
    }
    hist_add(sh, static_cast<uint32_t>(c >> sh_d) & 255u, act);
  }
  __syncthreads();
  flush_hist(sh, ctl->gsel.hist[pass]);
  if (last_block(&ctl->gsel.ticket[pass])) {
    if (threadIdx.x < 32) select_digit<8>(&ctl->gsel, pass, 64, !p.kth_only);
  }
}

__global__ void __launch_bounds__(kThreads) gemit_kernel(GSelParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeSelect) return;
  const uint32_t level = __ldcg(&ctl->gsel.level);
  const bool done = __ldcg(&ctl->gsel.done) != 0;
  if (level <= 1 && done) return;  // the partition already wrote every winner
  const uint64_t T = __ldcg(&ctl->gsel.prefix);
  const uint32_t cnt = __ldcg(&ctl->sv_count);
  const uint32_t lane = lane_id();
  const int64_t warps_total = int64_t(gridDim.x) * (kThreads / 32);
  const int64_t gw = int64_t(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5);
  for (int64_t base = gw * 32; base < cnt; base += warps_total * 32) {
    const int64_t i = base + lane;
    uint64_t c = 0;
    bool win = false;
    if (i < cnt) {
      c = p.sv[i];
      win = c >= T;
    }
    const uint32_t slot = warp_append(&ctl->w_count, win);
    if (win) {
      if (slot < p.k) p.w[slot] = c;
      else atomicOr(&ctl->error, kErrOverflowW);
    }
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
  uint32_t* bsum1;
  uint32_t* bsum2;
  int64_t nblk;
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
  if (threadIdx.x == 0) p.bsum1[blockIdx.x] = tot;
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
__device__ __forceinline__ uint32_t tie_prefixes(const TieParams& p, const uint32_t* bscan,
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
  uint32_t total;
  const uint32_t off = block_excl_scan(sum, &total) + bscan[blockIdx.x];
#pragma unroll
  for (int e = 0; e < kTieSubPerThread; ++e) pre[e] += off;
  return total;
}

template <int DT>
__global__ void __launch_bounds__(kThreads) tie_exact_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies) return;
  const uint32_t tau = __ldcg(&ctl->tau);
  const uint32_t need = __ldcg(&ctl->need);
  __shared__ uint32_t q_sub[kTieSubPerBlock];
  __shared__ uint32_t q_n;
  __shared__ uint32_t delta;
  if (threadIdx.x == 0) {
    q_n = 0;
    delta = 0;
  }
  __syncthreads();
  uint32_t t[kTieSubPerThread], pre[kTieSubPerThread];
  const uint32_t old_total = tie_prefixes(p, p.bsum1, t, pre);
#pragma unroll
  for (int e = 0; e < kTieSubPerThread; ++e) {
    if ((t[e] & kInexact) && pre[e] < need) {
      const uint32_t s = atomicAdd(&q_n, 1u);
      q_sub[s] = static_cast<uint32_t>(threadIdx.x * kTieSubPerThread + e);
    }
  }
  __syncthreads();
  const uint32_t nq = q_n;
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  for (uint32_t q = warp; q < nq; q += kThreads / 32) {
    const int64_t i = int64_t(blockIdx.x) * kTieSubPerBlock + q_sub[q];
    const int64_t lo = i << p.alpha;
    const int64_t len = sub_len(i, p.alpha, p.n);
    uint32_t c = 0;
    for (int64_t off = lane; off < len; off += 32) c += (map_key<DT>(__ldg(p.keys + lo + off)) == tau);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (lane == 0) {
      const uint32_t old = p.tcnt[i] & kCountMask;
      p.tcnt[i] = c | kScanned;
      atomicAdd(&delta, c - old);
      atomicAdd(&ctl->tie_scanned, 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) p.bsum2[blockIdx.x] = old_total + delta;
}

template <int DT, int B>
__global__ void __launch_bounds__(kThreads) tie_emit_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies) return;
  const uint32_t tau = __ldcg(&ctl->tau);
  const uint32_t need = __ldcg(&ctl->need);
  const uint32_t g = __ldcg(&ctl->g_count);  // < k in this mode
  // G is part of the answer: copy it in front of the ties
  for (int64_t j = int64_t(blockIdx.x) * kThreads + threadIdx.x; j < g;
       j += int64_t(gridDim.x) * kThreads)
    p.w[j] = p.g[j];
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctl->w_count, g);

  __shared__ uint32_t q_sub[kTieSubPerBlock];
  __shared__ uint32_t q_pre[kTieSubPerBlock];
  __shared__ uint32_t q_n;
  if (threadIdx.x == 0) q_n = 0;
  __syncthreads();
  uint32_t t[kTieSubPerThread], pre[kTieSubPerThread];
  tie_prefixes(p, p.bsum2, t, pre);
#pragma unroll
  for (int e = 0; e < kTieSubPerThread; ++e) {
    if ((t[e] & kCountMask) > 0 && pre[e] < need) {
      const uint32_t s = atomicAdd(&q_n, 1u);
      q_sub[s] = static_cast<uint32_t>(threadIdx.x * kTieSubPerThread + e);
      q_pre[s] = pre[e];
    }
  }
  __syncthreads();
  const uint32_t nq = q_n;
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  for (uint32_t q = warp; q < nq; q += kThreads / 32) {
    const int64_t i = int64_t(blockIdx.x) * kTieSubPerBlock + q_sub[q];
    const uint32_t base = q_pre[q];
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
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) emitted += __shfl_xor_sync(0xFFFFFFFFu, emitted, o);
    if (lane == 0 && emitted) atomicAdd(&ctl->w_count, emitted);
  }
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

int grid_for(int64_t work, int per_block, int sms, int per_sm) {
  int64_t g = (work + per_block - 1) / per_block;
  const int64_t cap = static_cast<int64_t>(sms) * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

}  // namespace

cudaError_t launch_threshold(const Work& w, int sms, cudaStream_t s) {
  const int64_t count = w.S * w.beta;
  const int grid = grid_for(count, kThreads * 16, sms, 4);
  for (int pass = 1; pass <= 3; ++pass) {
    thr_pass_kernel<<<grid, kThreads, 0, s>>>(w.dkeys, count, w.ctl, pass);
    note_launch();
  }
  return cudaGetLastError();
}

template <int DT, int B>
static void filter_t(const FilterParams& p, int grid, cudaStream_t s) {
  filter_kernel<DT, B><<<grid, kThreads, 0, s>>>(p);
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
  p.g = w.g;
  p.ctl = w.ctl;
  p.kth_only = kth_only ? 1 : 0;
  const int grid = grid_for(w.S, kThreads * 4, sms, 8);
#define DRTOPK_FILTER_CASE(DTV)                           \
  switch (w.beta) {                                       \
    case 1: filter_t<DTV, 1>(p, grid, s); break;          \
    case 2: filter_t<DTV, 2>(p, grid, s); break;          \
    case 3: filter_t<DTV, 3>(p, grid, s); break;          \
    default: filter_t<DTV, 4>(p, grid, s); break;         \
  }
  switch (w.dtype) {
    case DRTOPK_U32: DRTOPK_FILTER_CASE(DRTOPK_U32); break;
    case DRTOPK_I32: DRTOPK_FILTER_CASE(DRTOPK_I32); break;
    default: DRTOPK_FILTER_CASE(DRTOPK_F32); break;
  }
#undef DRTOPK_FILTER_CASE
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_ties(const Work& w, const void* keys, int sms, cudaStream_t s) {
  (void)sms;
  TieParams p;
  p.keys = static_cast<const uint32_t*>(keys);
  p.n = w.n;
  p.S = w.S;
  p.k = w.k;
  p.alpha = w.alpha;
  p.dkeys = w.dkeys;
  p.dsegs = w.dsegs;
  p.tcnt = w.tcnt;
  p.nblk = (w.S + kTieSubPerBlock - 1) / kTieSubPerBlock;
  p.bsum1 = w.bsum;
  p.bsum2 = w.bsum + p.nblk;
  p.g = w.g;
  p.w = w.w;
  p.ctl = w.ctl;
  const int grid = static_cast<int>(p.nblk);
#define DRTOPK_TIE_CASE(DTV)                                                        \
  switch (w.beta) {                                                                 \
    case 1: tie_lb_kernel<1><<<grid, kThreads, 0, s>>>(p); break;                   \
    case 2: tie_lb_kernel<2><<<grid, kThreads, 0, s>>>(p); break;                   \
    case 3: tie_lb_kernel<3><<<grid, kThreads, 0, s>>>(p); break;                   \
    default: tie_lb_kernel<4><<<grid, kThreads, 0, s>>>(p); break;                  \
  }                                                                                 \
  scan_blocks_kernel<<<1, 1024, 0, s>>>(p.bsum1, p.nblk, p.ctl);                    \
  tie_exact_kernel<DTV><<<grid, kThreads, 0, s>>>(p);                               \
  scan_blocks_kernel<<<1, 1024, 0, s>>>(p.bsum2, p.nblk, p.ctl);                    \
  switch (w.beta) {                                                                 \
    case 1: tie_emit_kernel<DTV, 1><<<grid, kThreads, 0, s>>>(p); break;            \
    case 2: tie_emit_kernel<DTV, 2><<<grid, kThreads, 0, s>>>(p); break;            \
    case 3: tie_emit_kernel<DTV, 3><<<grid, kThreads, 0, s>>>(p); break;            \
    default: tie_emit_kernel<DTV, 4><<<grid, kThreads, 0, s>>>(p); break;           \
  }
  switch (w.dtype) {
    case DRTOPK_U32: DRTOPK_TIE_CASE(DRTOPK_U32); break;
    case DRTOPK_I32: DRTOPK_TIE_CASE(DRTOPK_I32); break;
    default: DRTOPK_TIE_CASE(DRTOPK_F32); break;
  }
#undef DRTOPK_TIE_CASE
  note_launch(5);
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
  gpart_kernel<<<grid, kThreads, 0, s>>>(p);
  const int last = kth_only ? 3 : 7;
  for (int pass = 2; pass <= last; ++pass) gpass_kernel<<<grid, kThreads, 0, s>>>(p, pass);
  int launched = 1 + (last - 1);
  if (!kth_only) {
    gemit_kernel<<<grid, kThreads, 0, s>>>(p);
    ++launched;
  }
  note_launch(launched);
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
