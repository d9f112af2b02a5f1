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
__global__ void __launch_bounds__(kThreads) thr_compact_kernel(const uint32_t* dkeys,
                                                               int64_t count, uint32_t* ds,
                                                               Ctl* ctl) {
  __shared__ uint32_t sh[256];
  __shared__ uint32_t sbuf[kThrStageCap];
  __shared__ uint32_t s_fill;
  zero_hist(sh);
  if (threadIdx.x == 0) s_fill = 0;
  __syncthreads();
  SelState<4>* st = &ctl->dsel;
  const uint32_t d0 = static_cast<uint32_t>(__ldcg(&st->prefix)) >> 24;
  const bool inplace = uint64_t(__ldcg(&st->bucket)) * 8 > static_cast<uint64_t>(count);
  if (inplace && blockIdx.x == 0 && threadIdx.x == 0) ctl->ds_inplace = 1;
  RunHist rh;
  const int64_t step = int64_t(gridDim.x) * kThreads * 16;
  for (int64_t base = int64_t(blockIdx.x) * kThreads * 16; base < count; base += step) {
    uint32_t v[16];
    load16<kThreads>(dkeys, count, base, v);
    uint32_t hit = 0;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      const int64_t i = base + (int64_t(e >> 2) * kThreads + threadIdx.x) * 4 + (e & 3);
      if (i < count && (v[e] >> 24) == d0) {
        hit |= 1u << e;
        rh.add(sh, (v[e] >> 16) & 255u);
      }
    }
    if (!inplace) {
      uint32_t slot = stage_reserve<uint32_t, kThreads, kThrStageCap>(
          sbuf, &s_fill, __popc(hit), &ctl->ds_count, ds, ~uint64_t(0), &ctl->error, 0u);
#pragma unroll
      for (int e = 0; e < 16; ++e)
        if (hit & (1u << e)) sbuf[slot++] = v[e];
    }
  }
  if (!inplace) stage_flush<uint32_t, kThreads>(sbuf, &s_fill, &ctl->ds_count, ds, ~uint64_t(0),
                                                &ctl->error, 0u);
  rh.flush(sh);
  __syncthreads();
  flush_hist(sh, st->hist[1]);
  if (last_block(&st->ticket[1])) {
    if (threadIdx.x < 32) select_digit<4>(st, 1, 32, false);
  }
}

// Digit 2 and 3 passes over the compacted survivors (or the delegate keys).
__global__ void __launch_bounds__(kThreads) thr_pass_kernel(const uint32_t* dsv,
                                                            const uint32_t* dkeys,
                                                            int64_t dcount, Ctl* ctl,
                                                            int pass) {
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

// Each thread classifies 4 subranges per step: skip (m^0 <= tau), queue
// for a scan (m^{beta-1} > tau: Rule 3 says every element may qualify) or
// emit its delegates > tau (Rule 3: they are all of its elements > tau).
// Queue entries and emitted candidates are staged in shared memory.
constexpr int kClsSub = 4;
constexpr int kClsGCap = kThreads * kClsSub * 4;
constexpr int kClsQCap = kThreads * kClsSub * 2;

template <int DT, int B>
__global__ void __launch_bounds__(kThreads) filter_classify_kernel(FilterParams p) {
  __shared__ uint32_t sh[256];
  __shared__ uint64_t gbuf[kClsGCap];
  __shared__ uint32_t qbuf[kClsQCap];
  __shared__ uint32_t g_fill, q_fill;
  zero_hist(sh);
  if (threadIdx.x == 0) {
    g_fill = 0;
    q_fill = 0;
  }
  __syncthreads();
  const uint32_t tau = __ldcg(&p.ctl->tau);
  const int alpha = p.alpha;
  uint32_t nscan = 0;
  const int64_t per_step = int64_t(kThreads) * kClsSub;
  for (int64_t base = int64_t(blockIdx.x) * per_step; base < p.S;
       base += int64_t(gridDim.x) * per_step) {
    uint32_t dk[kClsSub][B];
    uint16_t ds[kClsSub][B];
#pragma unroll
    for (int u = 0; u < kClsSub; ++u) {
      const int64_t i = base + int64_t(u) * kThreads + threadIdx.x;
#pragma unroll
      for (int j = 0; j < B; ++j) {
        dk[u][j] = (i < p.S) ? p.dkeys[i * B + j] : 0u;
        ds[u][j] = (i < p.S) ? p.dsegs[i * B + j] : static_cast<uint16_t>(kNoSeg);
      }
    }
    uint32_t scanm = 0, nitems = 0;
    uint64_t items[kClsSub * B];
#pragma unroll
    for (int u = 0; u < kClsSub; ++u) {
      const int64_t i = base + int64_t(u) * kThreads + threadIdx.x;
      if (i < p.S && dk[u][0] > tau) {
        if (dk[u][B - 1] > tau && sub_len(i, alpha, p.n) > B) {
          scanm |= 1u << u;
        } else {
#pragma unroll
          for (int j = 0; j < B; ++j) {
            if (dk[u][j] > tau) {
              const int r = occ_rank<B>(dk[u], ds[u], j);
              const int64_t pos = resolve_pos<DT>(p.keys, p.n, alpha, i, ds[u][j], dk[u][j], r);
              if (pos < 0) atomicOr(&p.ctl->error, kErrTieRank);
              items[nitems++] = make_comp(dk[u][j], static_cast<uint32_t>(pos));
            }
          }
        }
      }
    }
    uint32_t qs = stage_reserve<uint32_t, kThreads, kClsQCap>(
        qbuf, &q_fill, __popc(scanm), &p.ctl->scanq_count, p.scanq, ~uint64_t(0), &p.ctl->error, 0u);
#pragma unroll
    for (int u = 0; u < kClsSub; ++u)
      if (scanm & (1u << u)) qbuf[qs++] = static_cast<uint32_t>(base + int64_t(u) * kThreads + threadIdx.x);
    nscan += __popc(scanm);
    uint32_t gs = stage_reserve<uint64_t, kThreads, kClsGCap>(
        gbuf, &g_fill, nitems, &p.ctl->g_count, p.g, static_cast<uint64_t>(p.g_cap), &p.ctl->error,
        kErrOverflowG);
    for (uint32_t e = 0; e < nitems; ++e) {
      gbuf[gs + e] = items[e];
      atomicAdd(&sh[static_cast<uint32_t>(items[e] >> 56)], 1u);
    }
  }
  stage_flush<uint32_t, kThreads>(qbuf, &q_fill, &p.ctl->scanq_count, p.scanq, ~uint64_t(0),
                                  &p.ctl->error, 0u);
  stage_flush<uint64_t, kThreads>(gbuf, &g_fill, &p.ctl->g_count, p.g,
                                  static_cast<uint64_t>(p.g_cap), &p.ctl->error, kErrOverflowG);
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
  const uint32_t nact = active_blocks(total, int64_t(kThreads) * kScanKPT);
  if (blockIdx.x >= nact) return;
  RunHist rh;
  const int64_t step = int64_t(nact) * kThreads * kScanKPT;
  for (int64_t base = int64_t(blockIdx.x) * kThreads * kScanKPT; base < total; base += step) {
    uint32_t x[kScanKPT];
    uint32_t sq[kScanKPT];
    uint32_t hit = 0;
    // phase 1: queue entries (independent loads, all in flight)
#pragma unroll
    for (int u = 0; u < kScanKPT; ++u) {
      const int64_t v = imin64(base + threadIdx.x + int64_t(u) * kThreads, total - 1);
      sq[u] = __ldg(p.scanq + (v >> alpha));
    }
    // phase 2: keys (clamped addresses, unconditional loads)
#pragma unroll
    for (int u = 0; u < kScanKPT; ++u) {
      const int64_t v = base + threadIdx.x + int64_t(u) * kThreads;
      const int64_t gi = (int64_t(sq[u]) << alpha) + (v & mask);
      const bool ok = v < total && gi < p.n;
      x[u] = map_key<DT>(__ldg(p.keys + (ok ? gi : 0)));
      if (ok && x[u] > tau) hit |= 1u << u;
    }
    const uint32_t wt = __reduce_add_sync(0xFFFFFFFFu, __popc(hit));
    uint32_t wb, unused;
    block_reserve2<kThreads>(&p.ctl->g_count, wt, nullptr, 0, wb, unused);
    const uint32_t lt = lanemask_lt();
    uint32_t run = 0;
#pragma unroll
    for (int u = 0; u < kScanKPT; ++u) {
      const bool h = (hit >> u) & 1u;
      const uint32_t bal = __ballot_sync(0xFFFFFFFFu, h);
      if (h) {
        const int64_t v = base + threadIdx.x + int64_t(u) * kThreads;
        const int64_t gi = (int64_t(sq[u]) << alpha) + (v & mask);
        const uint32_t slot = wb + run + __popc(bal & lt);
        if (slot < p.g_cap) p.g[slot] = make_comp(x[u], static_cast<uint32_t>(gi));
        else atomicOr(&p.ctl->error, kErrOverflowG);
        rh.add(sh, x[u] >> 24);
      }
      run += __popc(bal);
    }
  }
  rh.flush(sh);
  __syncthreads();
  flush_hist(sh, p.ctl->gsel.hist[0]);
  if (last_block_of(&p.ctl->filter_ticket, nact)) {
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

constexpr int kGIpt = 16;
constexpr int kGCap = kThreads * kGIpt;  // one step's worth per buffer

__global__ void __launch_bounds__(kThreads) gstage_kernel(GSelParams p, int s) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeSelect) return;
  const int level = s - 1;
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
  for (int64_t base = int64_t(blockIdx.x) * kThreads * kGIpt; base < count; base += stepn) {
    uint64_t c[kGIpt];
    uint32_t win = 0, sur = 0;
#pragma unroll
    for (int u = 0; u < kGIpt; ++u) {
      const int64_t i = base + threadIdx.x + int64_t(u) * kThreads;
      c[u] = __ldcg(src + imin64(i, count - 1));
    }
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
  for (int64_t b = blockIdx.x; b < p.nblk; b += gridDim.x) {
  const int64_t i0 = b * kTieSubPerBlock + threadIdx.x * kTieSubPerThread;
  uint32_t sum = 0;
  uint32_t dka[kTieSubPerThread][B];
  uint16_t dsa[kTieSubPerThread][B];
#pragma unroll
  for (int e = 0; e < kTieSubPerThread; ++e) {
    const int64_t i = i0 + e;
#pragma unroll
    for (int j = 0; j < B; ++j) {
      dka[e][j] = (i < p.S) ? p.dkeys[i * B + j] : 0u;
      dsa[e][j] = (i < p.S) ? p.dsegs[i * B + j] : static_cast<uint16_t>(kNoSeg);
    }
  }
#pragma unroll
  for (int e = 0; e < kTieSubPerThread; ++e) {
    const int64_t i = i0 + e;
    if (i >= p.S) break;
    const uint32_t* dk = dka[e];
    const uint16_t* ds = dsa[e];
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
    p.bsum1[b] = tot;
    p.bsum2[b] = tot;
  }
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
__device__ __forceinline__ void tie_prefixes(const TieParams& p, const uint32_t* bscan, int64_t b,
                                             uint32_t (&t)[kTieSubPerThread],
                                             uint32_t (&pre)[kTieSubPerThread]) {
  const int64_t i0 = b * kTieSubPerBlock + threadIdx.x * kTieSubPerThread;
  uint32_t sum = 0;
#pragma unroll
  for (int e = 0; e < kTieSubPerThread; ++e) {
    const int64_t i = i0 + e;
    t[e] = (i < p.S) ? p.tcnt[i] : 0u;
    pre[e] = sum;
    sum += t[e] & kCountMask;
  }
  const uint32_t off = block_excl_scan(sum, nullptr) + bscan[b];
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
  for (int64_t b = blockIdx.x; b < p.nblk; b += gridDim.x) {
    uint32_t t[kTieSubPerThread], pre[kTieSubPerThread];
    tie_prefixes(p, p.bsum1, b, t, pre);
    const int64_t i0 = b * kTieSubPerBlock + threadIdx.x * kTieSubPerThread;
    uint32_t c = 0;
#pragma unroll
    for (int e = 0; e < kTieSubPerThread; ++e) c += ((t[e] & kInexact) && pre[e] < need);
    uint32_t slot = block_append<kThreads>(&ctl->tieq1_count, c);
#pragma unroll
    for (int e = 0; e < kTieSubPerThread; ++e)
      if ((t[e] & kInexact) && pre[e] < need) p.q1[slot++] = static_cast<uint32_t>(i0 + e);
  }
}

// Exact tie counts of the queued subranges, one warp per subrange over the
// whole grid; the block sums used for the second scan are corrected in place.
// Ties equal to tau among keys [lo, lo + len), read by one thread (len <= 64).
template <int DT>
__device__ __forceinline__ uint32_t count_eq_thread(const uint32_t* keys, int64_t lo, int64_t len,
                                                    uint32_t tau) {
  uint32_t c = 0;
  if ((len & 3) == 0 && (reinterpret_cast<uintptr_t>(keys + lo) & 15u) == 0) {
    const uint4* v4 = reinterpret_cast<const uint4*>(keys + lo);
    for (int64_t w = 0; w < (len >> 2); ++w) {
      const uint4 v = __ldg(v4 + w);
      c += (map_key<DT>(v.x) == tau) + (map_key<DT>(v.y) == tau) + (map_key<DT>(v.z) == tau) +
           (map_key<DT>(v.w) == tau);
    }
  } else {
    for (int64_t t = 0; t < len; ++t) c += (map_key<DT>(__ldg(keys + lo + t)) == tau);
  }
  return c;
}

constexpr int kTieThreadAlpha = 6;  // subranges of <= 64 keys: one thread each

template <int DT>
__global__ void __launch_bounds__(kThreads) tie_count_kernel(TieParams p) {
  Ctl* ctl = p.ctl;
  if (__ldcg(&ctl->mode) != kModeTies) return;
  const uint32_t tau = __ldcg(&ctl->tau);
  const int64_t nq = __ldcg(&ctl->tieq1_count);
  const uint32_t lane = lane_id();
  const int64_t warps = int64_t(gridDim.x) * (kThreads / 32);
  uint32_t done = 0;
  if (p.alpha <= kTieThreadAlpha) {
    const int64_t nthr = int64_t(gridDim.x) * kThreads;
    for (int64_t q0 = int64_t(blockIdx.x) * kThreads; q0 < nq; q0 += nthr) {
      const int64_t q = q0 + threadIdx.x;
      uint32_t delta = 0;
      int64_t blk = -1;
      if (q < nq) {
        const int64_t i = p.q1[q];
        const uint32_t c = count_eq_thread<DT>(p.keys, i << p.alpha, sub_len(i, p.alpha, p.n), tau);
        delta = c - (p.tcnt[i] & kCountMask);
        p.tcnt[i] = c | kScanned;
        blk = i / kTieSubPerBlock;
        ++done;
      }
      // consecutive queue entries mostly share a block sum: add once per group
      const uint32_t am = __ballot_sync(0xFFFFFFFFu, q < nq);
      if (q < nq) {
        const uint32_t peers = __match_any_sync(am, static_cast<unsigned long long>(blk));
        const uint32_t tot = __reduce_add_sync(peers, delta);
        if ((peers & lanemask_lt()) == 0) atomicAdd(&p.bsum2[blk], tot);
      }
    }
    done = __reduce_add_sync(0xFFFFFFFFu, done);
    if (lane == 0 && done) atomicAdd(&ctl->tie_scanned, done);
    return;
  }
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
  for (int64_t b = blockIdx.x; b < p.nblk; b += gridDim.x) {
    uint32_t t[kTieSubPerThread], pre[kTieSubPerThread];
    tie_prefixes(p, p.bsum2, b, t, pre);
    const int64_t i0 = b * kTieSubPerBlock + threadIdx.x * kTieSubPerThread;
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
  if (p.alpha <= kTieThreadAlpha) {
    // one thread per subrange, reading it in index order
    for (int64_t q = int64_t(blockIdx.x) * kThreads + threadIdx.x; q < nq;
         q += int64_t(gridDim.x) * kThreads) {
      const int64_t i = p.q2[q];
      uint32_t r = p.q2pre[q];
      if (p.tcnt[i] & kScanned) {
        const int64_t lo = i << p.alpha;
        const int64_t len = sub_len(i, p.alpha, p.n);
        for (int64_t t0 = 0; t0 < len && r < need; t0 += 16) {
          uint32_t v[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) v[e] = (t0 + e < len) ? __ldg(p.keys + lo + t0 + e) : 0u;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            if (t0 + e < len && r < need && map_key<DT>(v[e]) == tau) {
              p.w[g + r] = make_comp(tau, static_cast<uint32_t>(lo + t0 + e));
              ++r;
              ++emitted_total;
            }
          }
        }
      } else {
        uint32_t dk[B];
        uint16_t ds[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
          dk[j] = p.dkeys[i * B + j];
          ds[j] = p.dsegs[i * B + j];
        }
#pragma unroll
        for (int j = 0; j < B; ++j) {
          if (dk[j] == tau && ds[j] != kNoSeg && r < need) {
            const int o = occ_rank<B>(dk, ds, j);
            const int64_t pos = resolve_pos<DT>(p.keys, p.n, p.alpha, i, ds[j], tau, o);
            if (pos < 0) atomicOr(&ctl->error, kErrTieRank);
            p.w[g + r] = make_comp(tau, static_cast<uint32_t>(pos));
            ++r;
            ++emitted_total;
          }
        }
      }
    }
  }
  for (int64_t q = int64_t(blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5);
       p.alpha > kTieThreadAlpha && q < nq; q += warps) {
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
  thr_pass_kernel<<<g2, kThreads, 0, s>>>(w.ds, w.dkeys, count, w.ctl, 2);
  thr_pass_kernel<<<g2, kThreads, 0, s>>>(w.ds, w.dkeys, count, w.ctl, 3);
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
  const int grid = static_cast<int>(std::min<int64_t>(p.nblk, int64_t(sms) * 4));
  const int gq = grid_for(w.S, kThreads / 32, sms, 4);
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
