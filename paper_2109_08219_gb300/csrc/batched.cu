// Batched ragged top-k: many independent (row, k_r) queries in ONE
// persistent launch. Each CTA takes rows from an atomic counter (largest
// first) and runs the whole delegate-centric method on a row on-chip:
//   1. delegate pass (Rule 1 Sec. 3.1, Rule 3 Sec. 3.3): the row streams
//      through a 2-stage ring of 64 KB TMA bulk copies; every thread keeps
//      the top-beta of 32 keys by value; (key, segment) lists are merged
//      per subrange; the delegate vector D stays in shared memory;
//   2. threshold (Rule 2 Sec. 3.2): MSD radix select of the k-th delegate
//      over D in shared memory;
//   3. filter (Rules 2-3): subranges whose beta delegates all exceed tau
//      are read again, the others give their delegates > tau; candidates
//      G = {x > tau} go to shared memory, spilling to a per-CTA scratch;
//   4. second top-k: MSD radix select over the (key, ~index) composites of
//      G, or, when |G| < k, G plus the smallest-index ties at tau;
//   5. the k_r winners are bitonic-sorted in shared memory.
// Rows start at any 4-byte offset: each chunk is copied from the 16-byte
// boundary below it and read at a shift, with rotated scalar reads (no
// bank conflicts). Row sizes up to 4096 keys skip the delegates (direct
// select). Indices in the output are positions within the row.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "delegate_core.cuh"
#include "launch.h"

namespace drtopk {

namespace {

constexpr int kBT = 512;              // threads per CTA (one CTA per SM)
constexpr int kBWarps = kBT / 32;
constexpr int kBLogWarps = 4;
constexpr int kBLogChunk = kBLogWarps + 10;          // keys per ring stage: 32 per thread
constexpr int kBChunk = 1 << kBLogChunk;
constexpr int kBStages = 2;
static_assert((1 << kBLogWarps) == kBWarps && kBChunk == kBT * 32, "chunk geometry");
constexpr int kBStageBytes = kBChunk * 4 + 128;  // + room for the alignment shift
constexpr int kBDMax = 8192;          // delegate slots (S * beta) kept on chip
constexpr int kBGS = 4096;            // candidates kept on chip (more spill to scratch)
constexpr int kBMaxK = 4096;          // largest k_r of the batched path
constexpr int kBDirect = 4096;        // rows up to this size: always direct select
constexpr int kBDirectMax = kBStages * kBChunk;  // longest row a direct select holds on chip
constexpr int64_t kBMaxN = int64_t(1) << 24;  // longest row of the batched path
constexpr int64_t kBKeepL2 = int64_t(1) << 20;  // rows up to 1 MB: normal L2 priority

constexpr size_t kRingBytes = size_t(kBStages) * kBStageBytes;
// The ring is free after the delegate pass. The filter keeps its lists
// there; then the winners (up to kBMaxK) and the tie ranking's lists.
constexpr size_t kScanOff = 0;                          // u16 subrange list, <= kBDMax
constexpr size_t kReqOff = size_t(kBDMax) * 2;          // u64 resolve requests, <= kBDMax
constexpr size_t kTieOff = size_t(kBMaxK) * 8;          // u16 + 2 x u32 per thread
static_assert(kReqOff + size_t(kBDMax) * 8 <= kRingBytes, "filter lists exceed the ring");
static_assert(kTieOff + size_t(kBT) * 10 <= kRingBytes, "tie lists exceed the ring");
constexpr size_t kDynSmem = kRingBytes + size_t(kBDMax) * 4 + size_t(kBDMax) * 2 + size_t(kBGS) * 8;

struct BatchParams {
  uint64_t keys_base;     // base addresses of RowDesc's offsets
  uint64_t out_keys_base;
  uint64_t out_idx_base;
  const RowDesc* rows;    // processing order (largest first)
  int32_t nrows;
  uint32_t* row_ctr;      // zeroed by the host before the launch
  uint64_t* scratch;      // per-CTA candidate spill, scap entries each
  int64_t scap;
  uint32_t* err;
  unsigned long long* phase;  // kBPhases cycle counters (thread 0 of each CTA)
};

// Cycle counters of the batched kernel, summed over CTAs. Rows with
// delegates: 0 delegate pass, 1 threshold select, 2 filter, 3 second select
// (or sort of all candidates), 4 tie ranking, 5 final sort and output.
// Direct rows: 6 load, 7 select, 8 collection, 9 sort and output.
constexpr int kBPhases = 10;
static_assert(kBPhases == kBatchPhases, "phase counters");

__device__ __forceinline__ void phase_mark(const BatchParams& p, int ph, long long& tmark) {
  if (threadIdx.x == 0) {
    const long long t = clock64();
    atomicAdd(p.phase + ph, static_cast<unsigned long long>(t - tmark));
    tmark = t;
  }
}

struct Smem {
  unsigned char* ring;
  uint32_t* dkeys;
  uint16_t* dsegs;
  uint64_t* gbuf;
};

__device__ __forceinline__ uint32_t lanemask_lt_b() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ------------------------------------------------------------ chunk ring ---
struct Ring {
  uint64_t* bar;      // kBStages mbarriers
  uint64_t seq;       // chunks issued by this CTA so far (all rows)
  uint64_t pol_first;   // rows read once (long rows)
  uint64_t pol_normal;  // rows read again by the filter while still in L2
};

__device__ __forceinline__ const uint32_t* row_keys(const BatchParams& p, const RowDesc& r) {
  return reinterpret_cast<const uint32_t*>(p.keys_base + r.keys);
}
__device__ __forceinline__ uint32_t* row_out_keys(const BatchParams& p, const RowDesc& r) {
  return reinterpret_cast<uint32_t*>(p.out_keys_base + r.out_keys);
}
__device__ __forceinline__ int32_t* row_out_idx(const BatchParams& p, const RowDesc& r) {
  return reinterpret_cast<int32_t*>(p.out_idx_base + r.out_idx);
}
// Key shift of the row inside its 16-byte blocks (chunks start at
// multiples of 16 bytes from the row start, so it holds for every chunk).
__device__ __forceinline__ int row_shift(const BatchParams& p, const RowDesc& r) {
  return static_cast<int>(((p.keys_base + r.keys) & 15u) >> 2);
}

// Issues chunk c of the row into a stage buffer: one bulk copy from the
// 16-byte boundary at or below its first key (the chunk is then read at
// row_shift keys), up to the last 16-byte boundary inside the row; the keys
// after that boundary come by plain loads. The copy may read the bytes of
// the row's first 16-byte block that precede its first key (always inside
// the same allocation, whose base is at least 16-byte aligned), never bytes
// past the row. Thread 0 only.
__device__ __forceinline__ void issue_row_chunk(const BatchParams& p, const RowDesc& r, int64_t c,
                                                unsigned char* buf, uint64_t* bar, uint64_t pol) {
  const uint32_t* rk = row_keys(p, r);
  const int64_t base = static_cast<int64_t>(p.keys_base + r.keys);
  const int s = row_shift(p, r);
  const int64_t e0 = c * kBChunk;                                  // first key (row index)
  const int64_t e1 = imin64(int64_t(r.n), (c + 1) * kBChunk);      // one past
  const int64_t a0 = (base + e0 * 4) & ~int64_t(15);
  const int64_t end16 = (base + int64_t(r.n) * 4) & ~int64_t(15);
  const int64_t a1 = imin64((base + e1 * 4 + 15) & ~int64_t(15), end16);
  const int64_t bytes = a1 > a0 ? a1 - a0 : 0;
  uint32_t* dst = reinterpret_cast<uint32_t*>(buf);
  // buffer word w holds row key e0 + w - s
  const int64_t covered = e0 + bytes / 4 - s;  // first key not in the bulk copy
  for (int64_t e = (covered > e0 ? covered : e0); e < e1; ++e) dst[e - e0 + s] = rk[e];
  if (bytes > 0) {
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bar, static_cast<uint32_t>(bytes));
    tma_load_1d(buf, reinterpret_cast<const unsigned char*>(a0), static_cast<uint32_t>(bytes), bar,
                pol);
  } else {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
  }
}

// ---------------------------------------------------- block radix select ---
// Warp 0: finds the digit d (from the top) at which the descending running
// count of hist[] reaches krem; s_bc = {d, krem - count above d, hist[d]}.
// Each lane sums 8 buckets; a warp scan locates the crossing lane.
__device__ __forceinline__ void bucket_search(const uint32_t* hist, uint32_t krem, uint32_t* s_bc) {
  const int lane = threadIdx.x & 31;
  const int top = 255 - lane * 8;  // this lane's buckets: top, top-1, ..., top-7
  uint32_t h[8];
  uint32_t sum = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    h[q] = hist[top - q];
    sum += h[q];
  }
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += t;
  }
  const uint32_t hit = __ballot_sync(0xFFFFFFFFu, incl >= krem);
  const int f = hit ? __ffs(hit) - 1 : 31;
  if (lane == f) {
    uint32_t acc = incl - sum;
    int d = top - 7;
    uint32_t hd = h[7];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (acc + h[q] >= krem || q == 7) {
        d = top - q;
        hd = h[q];
        break;
      }
      acc += h[q];
    }
    s_bc[0] = static_cast<uint32_t>(d);
    s_bc[1] = krem - acc;
    s_bc[2] = hd;
  }
}

// Logical candidate array: [0, kBGS) in shared memory, then the CTA's
// scratch.
__device__ __forceinline__ uint64_t g_get(const Smem& sm, const uint64_t* scr, uint32_t i) {
  return i < kBGS ? sm.gbuf[i] : scr[i - kBGS];
}
__device__ __forceinline__ void g_put(const Smem& sm, uint64_t* scr, int64_t scap, uint32_t i,
                                      uint64_t v, uint32_t* err) {
  if (i < kBGS) sm.gbuf[i] = v;
  else if (int64_t(i - kBGS) < scap) scr[i - kBGS] = v;
  else atomicOr(err, kErrOverflowG);
}

// Warp-aggregated append of one optional item per lane to the logical G.
__device__ __forceinline__ void g_append(const Smem& sm, uint64_t* scr, int64_t scap,
                                         uint32_t* s_gcnt, bool has, uint64_t v, uint32_t* err) {
  const uint32_t bal = __ballot_sync(0xFFFFFFFFu, has);
  if (!bal) return;
  uint32_t base = 0;
  const uint32_t lane = lane_id();
  if (lane == static_cast<uint32_t>(__ffs(bal) - 1)) base = atomicAdd(s_gcnt, __popc(bal));
  base = __shfl_sync(0xFFFFFFFFu, base, __ffs(bal) - 1);
  if (has) g_put(sm, scr, scap, base + __popc(bal & lanemask_lt_b()), v, err);
}

template <class V>
__device__ __forceinline__ V warp_min(V v) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const V t = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = t < v ? t : v;
  }
  return v;
}

template <class V>
struct SelResult {
  V value;        // exact mode: the krem-th largest; else a threshold T
  uint32_t need;  // exact mode: values equal to it among the top krem
};

// The krem-th largest of cnt values get(i) (MSD radix select, Sec. 4.1's
// digits of 8 bits). When every value of the selected bucket is among the
// top krem the search stops: in exact mode the answer is the bucket's
// minimum (found by one more pass); otherwise the returned T (the bucket's
// prefix, low bits 0) still has exactly krem values >= T when the values
// are distinct. mm: one 64-bit shared word.
template <class V, bool kExact, class Get>
__device__ SelResult<V> block_select(Get get, uint32_t cnt, uint32_t krem, uint32_t* hist,
                                     uint32_t* s_bc, unsigned long long* mm) {
  constexpr int kBits = sizeof(V) * 8;
  const int tid = threadIdx.x;
  int hb = kBits;  // bits above hb are fixed in prefix
  V prefix = 0;
  while (hb > 0) {
    const int width = hb < 8 ? hb : 8;
    const int sh = hb - width;
    for (int i = tid; i < 256; i += kBT) hist[i] = 0;
    __syncthreads();
    for (uint32_t i = tid; i < cnt; i += kBT) {
      const V x = get(i);
      if (hb >= kBits || (x >> hb) == (prefix >> hb))
        atomicAdd(&hist[static_cast<uint32_t>(x >> sh) & ((1u << width) - 1u)], 1u);
    }
    __syncthreads();
    if (tid < 32) bucket_search(hist, krem, s_bc);
    __syncthreads();
    prefix |= static_cast<V>(s_bc[0]) << sh;
    krem = s_bc[1];
    const uint32_t hd = s_bc[2];
    __syncthreads();
    hb = sh;
    if (hd == krem && hb > 0) {
      if constexpr (!kExact) {
        return {prefix, 0u};
      } else {
        // the whole bucket is among the top: the answer is its minimum,
        // needed as many times as it occurs
        if (tid == 0) {
          mm[0] = ~0ull;
          s_bc[3] = 0;
        }
        __syncthreads();
        V lo = static_cast<V>(~V(0));
        for (uint32_t i = tid; i < cnt; i += kBT) {
          const V x = get(i);
          if ((x >> hb) == (prefix >> hb)) lo = x < lo ? x : lo;
        }
        lo = warp_min(lo);
        if ((tid & 31) == 0) atomicMin(&mm[0], static_cast<unsigned long long>(lo));
        __syncthreads();
        const V v = static_cast<V>(mm[0]);
        uint32_t c = 0;
        for (uint32_t i = tid; i < cnt; i += kBT) c += get(i) == v ? 1u : 0u;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        if ((tid & 31) == 0) atomicAdd(&s_bc[3], c);
        __syncthreads();
        const uint32_t need = s_bc[3];
        __syncthreads();
        return {v, need};
      }
    }
  }
  return {prefix, krem};
}

// Bitonic sort (descending) of w[0..cnt) in shared memory, cnt <= kBMaxK;
// pads w[cnt..P) with 0 (P = next power of two), which sorts last. The
// pairs q of a warp in one sweep, [32m, 32m + 32), touch only elements
// [64m, 64m + 64) while the stride is at most 32, so such consecutive
// stages need only the warp in step.
__device__ void block_sort_desc(uint64_t* w, int cnt) {
  int P = 1;
  while (P < cnt) P <<= 1;
  for (int i = cnt + threadIdx.x; i < P; i += kBT) w[i] = 0ull;
  __syncthreads();
  const int half = P >> 1;
  for (int size = 2; size <= P; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int q = threadIdx.x; q < half; q += kBT) {
        const int i = 2 * q - (q & (stride - 1));
        const int j = i + stride;
        const bool desc = (i & size) == 0;
        const uint64_t a = w[i], b = w[j];
        if ((a < b) == desc) {
          w[i] = b;
          w[j] = a;
        }
      }
      const int next = stride > 1 ? stride >> 1 : size;  // stride of the next stage
      if (stride > 32 || next > 32) __syncthreads();
      else __syncwarp();
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------ direct row --
// Rows of at most kBDirectMax keys where delegates cannot reduce the work
// (short rows, or beta * n / 32 < 2k): the row is copied into the ring and
// the k-th largest key is found by an MSD radix select over it (Sec. 4.1's
// 8-bit digits); then one ordered pass collects the keys above it and the
// smallest-index keys equal to it, which go straight to the output.
template <int DT>
__device__ void direct_row(const BatchParams& p, const RowDesc& r, const Smem& sm, Ring& ring,
                           uint32_t* hist, uint32_t* s_bc, uint32_t* s_cnt,
                           unsigned long long* mm, long long& tmark) {
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int64_t n = r.n;
  const uint32_t k = static_cast<uint32_t>(r.k);
  const int nch = static_cast<int>((n + kBChunk - 1) / kBChunk);  // <= kBStages
  const uint64_t seq0 = ring.seq;
  if (tid == 0) {
    for (int c = 0; c < nch; ++c) {
      const uint64_t q = seq0 + c;
      issue_row_chunk(p, r, c, sm.ring + (q % kBStages) * kBStageBytes, &ring.bar[q % kBStages],
                      ring.pol_first);
    }
  }
  const uint32_t* base[kBStages];
  bool ok = true;
#pragma unroll
  for (int c = 0; c < kBStages; ++c) {
    const uint64_t q = seq0 + c;
    const int shift = row_shift(p, r);
    base[c] = reinterpret_cast<const uint32_t*>(sm.ring + (q % kBStages) * kBStageBytes) + shift;
    if (c < nch) ok = mbar_wait_bounded(&ring.bar[q % kBStages], static_cast<uint32_t>((q / kBStages) & 1)) && ok;
  }
  ring.seq = seq0 + static_cast<uint64_t>(nch);
  if (__syncthreads_or(!ok)) {
    if (tid == 0) atomicOr(p.err, kErrTimeout);
    return;
  }
  static_assert(kBStages == 2, "a direct row spans at most two stage buffers");
  const uint32_t* b0 = base[0];
  const uint32_t* b1 = base[1];
  auto key_at = [&](int64_t i) -> uint32_t {
    return map_key<DT>((i < kBChunk ? b0 : b1)[i & (kBChunk - 1)]);
  };
  phase_mark(p, 6, tmark);

  // k-th largest mapped key: four 8-bit digit passes over the row on chip
  const SelResult<uint32_t> sel = block_select<uint32_t, true>(
      [&](uint32_t i) { return key_at(i); }, static_cast<uint32_t>(n), k, hist, s_bc, mm);
  const uint32_t kth = sel.value;
  const uint32_t need = sel.need;  // keys equal to kth among the top k
  phase_mark(p, 7, tmark);
  const uint32_t gt = k - need; // keys above kth

  // ordered pass: keys > kth to gbuf (any order), ties in index order to
  // the output after the gt largest
  constexpr int kU = 8;
  uint32_t* wt = hist;  // per-warp tie counts
  uint32_t tbase = 0;
  const uint32_t tie_raw = unmap_key(DT, kth);
  for (int64_t t0 = 0; t0 < n; t0 += int64_t(kBT) * kU) {
    const int64_t wb = t0 + int64_t(warp) * 32 * kU;
    uint32_t bal[kU];
    uint32_t wcount = 0;
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int64_t i = wb + u * 32 + lane;
      const uint32_t x = i < n ? key_at(i) : 0u;
      const bool big = i < n && x > kth;
      const uint32_t bb = __ballot_sync(0xFFFFFFFFu, big);
      if (bb) {
        uint32_t b0 = 0;
        if (lane == __ffs(bb) - 1) b0 = atomicAdd(&s_cnt[0], __popc(bb));
        b0 = __shfl_sync(0xFFFFFFFFu, b0, __ffs(bb) - 1);
        if (big) {
          const uint32_t slot = b0 + __popc(bb & lanemask_lt_b());
          if (slot < gt) sm.gbuf[slot] = make_comp(x, static_cast<uint32_t>(i));
          else atomicOr(p.err, kErrOverflowW);
        }
      }
      bal[u] = __ballot_sync(0xFFFFFFFFu, i < n && x == kth);
      wcount += __popc(bal[u]);
    }
    if (lane == 0) wt[warp] = wcount;
    __syncthreads();
    uint32_t pre = tbase, tot = 0;
#pragma unroll
    for (int q = 0; q < kBWarps; ++q) {
      const uint32_t c = wt[q];
      pre += q < warp ? c : 0u;
      tot += c;
    }
    if (pre < tbase + need) {
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const uint32_t rank = pre + __popc(bal[u] & lanemask_lt_b());
        if (((bal[u] >> lane) & 1u) && rank < need) {
          row_out_keys(p, r)[gt + rank] = tie_raw;
          row_out_idx(p, r)[gt + rank] = static_cast<int32_t>(wb + u * 32 + lane);
        }
        pre += __popc(bal[u]);
      }
    }
    tbase += tot;
    __syncthreads();
  }
  phase_mark(p, 8, tmark);
  block_sort_desc(sm.gbuf, static_cast<int>(gt));
  for (uint32_t j = tid; j < gt; j += kBT) {
    const uint64_t c = sm.gbuf[j];
    row_out_keys(p, r)[j] = unmap_key(DT, comp_key(c));
    row_out_idx(p, r)[j] = static_cast<int32_t>(comp_idx(c));
  }
  __syncthreads();
  phase_mark(p, 9, tmark);
}

// ------------------------------------------------------------ one row ----
template <int DT, int B>
__device__ void process_row(const BatchParams& p, const RowDesc& r, const Smem& sm, Ring& ring,
                            uint32_t* hist, uint32_t* s_bc, uint32_t* s_cnt, uint64_t* s_lists,
                            unsigned long long* mm) {
  constexpr int P = Pow2<B>::v;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int64_t n = r.n;
  const uint32_t k = static_cast<uint32_t>(r.k);
  const int alpha = r.alpha;
  uint64_t* scr = p.scratch + static_cast<int64_t>(blockIdx.x) * p.scap;
  const uint32_t* rk = row_keys(p, r);

  if (tid == 0) {
    s_cnt[0] = 0;  // |G|
    s_cnt[1] = 0;  // scan list length
    s_cnt[2] = 0;  // winners
    s_cnt[3] = 0;  // resolve requests
  }
  // the previous row wrote the ring with generic stores; the bulk copies of
  // this row write it through the async proxy
  fence_proxy_async_smem();
  __syncthreads();

  long long tmark = clock64();
  int64_t S = 0;
  uint32_t tau = 0;
  if (alpha == 0) {
    direct_row<DT>(p, r, sm, ring, hist, s_bc, s_cnt, mm, tmark);
    return;
  }
  {
    // ---------------------------------------------- 1. delegate pass ----
    S = (n + (int64_t(1) << alpha) - 1) >> alpha;
    const int64_t nch = (n + kBChunk - 1) / kBChunk;
    const int cps_log = alpha > kBLogChunk ? alpha - kBLogChunk : 0;
    const uint64_t seq0 = ring.seq;
    // rows up to kBKeepL2 bytes stay in L2 for the filter's second reads
    const uint64_t pol = n * 4 <= kBKeepL2 ? ring.pol_normal : ring.pol_first;
    if (tid == 0) {
      for (int64_t c = 0; c < kBStages && c < nch; ++c) {
        const uint64_t q = seq0 + c;
        issue_row_chunk(p, r, c, sm.ring + (q % kBStages) * kBStageBytes, &ring.bar[q % kBStages],
                        pol);
      }
    }
    uint64_t run[P];
#pragma unroll
    for (int i = 0; i < P; ++i) run[i] = 0;
    for (int64_t c = 0; c < nch; ++c) {
      const uint64_t q = seq0 + c;
      const int stage = static_cast<int>(q % kBStages);
      const bool ok = mbar_wait_bounded(&ring.bar[stage], static_cast<uint32_t>((q / kBStages) & 1));
      if (__syncthreads_or(!ok)) {
        if (tid == 0) {
          atomicOr(p.err, kErrTimeout);
          // let the copies still in flight land (bounded) before leaving
          for (int64_t c2 = c; c2 < nch && c2 < c + kBStages; ++c2) {
            const uint64_t q2 = seq0 + c2;
            mbar_wait_bounded(&ring.bar[q2 % kBStages], static_cast<uint32_t>((q2 / kBStages) & 1));
          }
        }
        __syncthreads();
        return;
      }
      const uint32_t* cb = reinterpret_cast<const uint32_t*>(sm.ring + stage * kBStageBytes);
      const int shift = row_shift(p, r);
      const int64_t seg_start = c * kBChunk + int64_t(tid) * 32;  // row-relative
      const int64_t valid = n - seg_start;
      uint32_t m[B];
#pragma unroll
      for (int i = 0; i < B; ++i) m[i] = 0;
      int cntv;
      if (valid >= 32) {
        // rotated reads: lane l starts at word l of its 32 (no bank conflicts)
#pragma unroll
        for (int j = 0; j < 32; ++j) insert1<DT, B>(m, cb[shift + tid * 32 + ((j + lane) & 31)]);
        cntv = 32;
      } else {
        cntv = 0;
        for (int j = 0; j < 32; ++j) {
          if (j < valid) {
            insert1<DT, B>(m, cb[shift + tid * 32 + j]);
            ++cntv;
          }
        }
      }
      const int64_t sub = seg_start >> alpha;
      const uint32_t seg = static_cast<uint32_t>((seg_start - (sub << alpha)) >> 5);
      uint64_t a[P];
#pragma unroll
      for (int i = 0; i < P; ++i) a[i] = (i < B && i < cntv) ? make_dc(m[i < B ? i : 0], seg) : 0ull;
      if (alpha <= kBLogChunk) {
        const int g_log = alpha - 5;
        const int wl = g_log < 5 ? g_log : 5;
        for (int l = 0; l < wl; ++l) shfl_merge<P>(a, 1 << l);
        if (g_log <= 5) {
          if ((lane & ((1 << g_log) - 1)) == 0 && sub < S) {
#pragma unroll
            for (int j = 0; j < B; ++j) {
              sm.dkeys[sub * B + j] = dc_key(a[j]);
              sm.dsegs[sub * B + j] = static_cast<uint16_t>(a[j] == 0 ? kNoSeg : dc_seg(a[j]));
            }
          }
        } else {
          if (lane == 0) {
#pragma unroll
            for (int i = 0; i < P; ++i) s_lists[warp * P + i] = a[i];
          }
          __syncthreads();
          const int wps_log = g_log - 5;
          const int nsub_chunk = kBWarps >> wps_log;
          if (warp < nsub_chunk) {
            uint64_t b[P];
            const int src = warp * (1 << wps_log) + (lane & ((1 << wps_log) - 1));
#pragma unroll
            for (int i = 0; i < P; ++i) b[i] = s_lists[src * P + i];
            for (int l = 0; l < wps_log; ++l) shfl_merge<P>(b, 1 << l);
            const int64_t sub2 = ((c * kBChunk) >> alpha) + warp;
            if (lane == 0 && sub2 < S) {
#pragma unroll
              for (int j = 0; j < B; ++j) {
                sm.dkeys[sub2 * B + j] = dc_key(b[j]);
                sm.dsegs[sub2 * B + j] = static_cast<uint16_t>(b[j] == 0 ? kNoSeg : dc_seg(b[j]));
              }
            }
          }
        }
      } else {
        merge_desc<P>(run, a);
        const int64_t cps = int64_t(1) << cps_log;
        if (((c & (cps - 1)) == cps - 1) || (c == nch - 1)) {
          for (int l = 0; l < 5; ++l) shfl_merge<P>(run, 1 << l);
          if (lane == 0) {
#pragma unroll
            for (int i = 0; i < P; ++i) s_lists[warp * P + i] = run[i];
          }
          __syncthreads();
          if (warp == 0) {
            uint64_t b[P];
#pragma unroll
            for (int i = 0; i < P; ++i) b[i] = s_lists[(lane & (kBWarps - 1)) * P + i];
            for (int l = 0; l < kBLogWarps; ++l) shfl_merge<P>(b, 1 << l);
            const int64_t sub3 = c >> cps_log;
            if (lane == 0) {
#pragma unroll
              for (int j = 0; j < B; ++j) {
                sm.dkeys[sub3 * B + j] = dc_key(b[j]);
                sm.dsegs[sub3 * B + j] = static_cast<uint16_t>(b[j] == 0 ? kNoSeg : dc_seg(b[j]));
              }
            }
          }
#pragma unroll
          for (int i = 0; i < P; ++i) run[i] = 0;
        }
      }
      __syncthreads();  // stage consumed
      if (tid == 0 && c + kBStages < nch) {
        const uint64_t qn = q + kBStages;
        issue_row_chunk(p, r, c + kBStages, sm.ring + (qn % kBStages) * kBStageBytes,
                        &ring.bar[qn % kBStages], pol);
      }
    }
    ring.seq = seq0 + static_cast<uint64_t>(nch);
    phase_mark(p, 0, tmark);

    // ------------------------------------------------- 2. threshold ----
    const int dcnt = static_cast<int>(S * B);
    if (dcnt >= static_cast<int>(k)) {
      const uint32_t* dk = sm.dkeys;
      tau = block_select<uint32_t, true>([dk](uint32_t i) { return dk[i]; },
                                         static_cast<uint32_t>(dcnt), k, hist, s_bc, mm).value;
    }
    phase_mark(p, 1, tmark);

    // ------------------------------------------------- 3. filter -------
    // (a) classify each subrange: read again when its beta-th delegate
    // exceeds tau (non-delegates may too), else its delegates > tau are
    // candidates whose positions are resolved in (b).
    uint16_t* scanl = reinterpret_cast<uint16_t*>(sm.ring + kScanOff);
    uint64_t* reql = reinterpret_cast<uint64_t*>(sm.ring + kReqOff);
    for (int64_t i0 = 0; i0 < S; i0 += kBT) {
      const int64_t i = i0 + tid;
      if (i < S) {
        uint32_t dk[B];
        uint16_t ds[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
          dk[j] = sm.dkeys[i * B + j];
          ds[j] = sm.dsegs[i * B + j];
        }
        const int64_t len = imin64(int64_t(1) << alpha, n - (i << alpha));
        if (dk[0] > tau) {
          if (dk[B - 1] > tau && len > B) {
            scanl[atomicAdd(&s_cnt[1], 1u)] = static_cast<uint16_t>(i);
          } else {
#pragma unroll
            for (int j = 0; j < B; ++j) {
              if (dk[j] > tau) {
                // the (occ+1)-th key equal to dk[j] in segment ds[j]
                uint32_t occ = 0;
#pragma unroll
                for (int q = 0; q < j; ++q) occ += (dk[q] == dk[j] && ds[q] == ds[j]) ? 1u : 0u;
                const uint64_t lo = static_cast<uint64_t>((i << alpha) + int64_t(ds[j]) * 32);
                reql[atomicAdd(&s_cnt[3], 1u)] = (uint64_t(dk[j]) << 32) | (uint64_t(occ) << 24) | lo;
              }
            }
          }
        }
      }
    }
    __syncthreads();
    // (b) resolve positions: a warp reads a 32-key segment per request
    // (coalesced), kRU requests in flight per warp
    {
      constexpr int kRU = 8;
      const uint32_t nreq = s_cnt[3];
      for (uint32_t q0 = warp * kRU; q0 < nreq; q0 += (kBT / 32) * kRU) {
        uint32_t x[kRU];
        uint64_t rq[kRU];
#pragma unroll
        for (int u = 0; u < kRU; ++u) {
          rq[u] = (q0 + u < nreq) ? reql[q0 + u] : 0ull;
          const int64_t lo = static_cast<int64_t>(rq[u] & 0xFFFFFFu);
          const int64_t hi = imin64(imin64(n, lo + 32), ((lo >> alpha) + 1) << alpha);
          x[u] = (q0 + u < nreq && lo + lane < hi) ? rk[lo + lane] : 0u;
          if (!(q0 + u < nreq && lo + lane < hi)) rq[u] |= (1ull << 31);  // lane not in segment
        }
#pragma unroll
        for (int u = 0; u < kRU; ++u) {
          if (q0 + u >= nreq) break;
          const uint32_t key = static_cast<uint32_t>(rq[u] >> 32);
          const bool m = !((rq[u] >> 31) & 1u) && map_key<DT>(x[u]) == key;
          uint32_t bal = __ballot_sync(0xFFFFFFFFu, m);
          const uint32_t occ = static_cast<uint32_t>(rq[u] >> 24) & 3u;
          for (uint32_t t = 0; t < occ; ++t) bal &= bal - 1;
          if (lane == 0) {
            const int64_t lo = static_cast<int64_t>(rq[u] & 0xFFFFFFu);
            int64_t pos = -1;
            if (bal) pos = lo + (__ffs(bal) - 1);
            else atomicOr(p.err, kErrTieRank);
            g_put(sm, scr, p.scap, atomicAdd(&s_cnt[0], 1u),
                  make_comp(key, static_cast<uint32_t>(pos)), p.err);
          }
        }
      }
    }
    // (c) read the listed subranges again: kFU keys per thread in flight
    {
      constexpr int kFU = 16;
      const uint32_t nq = s_cnt[1];
      const int64_t vtotal = int64_t(nq) << alpha;
      const int64_t vmask = (int64_t(1) << alpha) - 1;
      const uint32_t nn = static_cast<uint32_t>(n);
      for (int64_t v0 = 0; v0 < vtotal; v0 += int64_t(kBT) * kFU) {
        uint32_t x[kFU];
        uint32_t gi[kFU];
#pragma unroll
        for (int u = 0; u < kFU; ++u) {
          const int64_t v = v0 + int64_t(u) * kBT + tid;
          gi[u] = v < vtotal ? static_cast<uint32_t>((int64_t(scanl[v >> alpha]) << alpha) + (v & vmask))
                             : nn;
          x[u] = gi[u] < nn ? rk[gi[u]] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kFU; ++u) {
          const uint32_t mk = map_key<DT>(x[u]);
          const bool has = gi[u] < nn && mk > tau;
          g_append(sm, scr, p.scap, &s_cnt[0], has, make_comp(mk, gi[u]), p.err);
        }
      }
    }
    __syncthreads();
  }

  // ------------------------------------------------- 4. second top-k ----
  uint64_t* w = reinterpret_cast<uint64_t*>(sm.ring);  // winners (the ring is free)
  const uint32_t gcnt = s_cnt[0];
  phase_mark(p, 2, tmark);
  if (gcnt >= k) {
    if (gcnt <= 2 * k && gcnt <= static_cast<uint32_t>(kBMaxK)) {
      // few candidates beyond k: sorting them all is cheaper than a select
      for (uint32_t i = tid; i < gcnt; i += kBT) w[i] = g_get(sm, scr, i);
      block_sort_desc(w, static_cast<int>(gcnt));
      phase_mark(p, 3, tmark);
    } else {
      const uint64_t T = block_select<uint64_t, false>(
          [&sm, scr](uint32_t i) { return g_get(sm, scr, i); }, gcnt, k, hist, s_bc, mm).value;
      for (uint32_t i0 = 0; i0 < gcnt; i0 += kBT) {
        const uint32_t i = i0 + tid;
        uint64_t v = 0;
        bool win = false;
        if (i < gcnt) {
          v = g_get(sm, scr, i);
          win = v >= T;
        }
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, win);
        if (!bal) continue;
        uint32_t base = 0;
        if (lane == __ffs(bal) - 1) base = atomicAdd(&s_cnt[2], __popc(bal));
        base = __shfl_sync(0xFFFFFFFFu, base, __ffs(bal) - 1);
        if (win) {
          const uint32_t slot = base + __popc(bal & lanemask_lt_b());
          if (slot < k) w[slot] = v;
          else atomicOr(p.err, kErrOverflowW);
        }
      }
      phase_mark(p, 3, tmark);
      block_sort_desc(w, static_cast<int>(k));
      phase_mark(p, 5, tmark);
    }
  } else {
    // the k-th key is tau: G (all > tau, fewer than k) sorted, then the
    // smallest-index ties at tau in index order, which keeps the whole
    // output sorted
    for (uint32_t i = tid; i < gcnt; i += kBT) w[i] = g_get(sm, scr, i);
    block_sort_desc(w, static_cast<int>(gcnt));
    phase_mark(p, 3, tmark);
    const uint32_t need = k - gcnt;
    uint32_t base = 0;  // ties placed so far (uniform)
    for (int64_t i0 = 0; i0 < S && base < need; i0 += kBT) {
      const int64_t i = i0 + tid;
      uint32_t cnt = 0;
      bool scan = false;
      if (i < S) {
        const int64_t len = imin64(int64_t(1) << alpha, n - (i << alpha));
        const uint32_t m0 = sm.dkeys[i * B], mb = sm.dkeys[i * B + B - 1];
        if (m0 >= tau) {
          if (mb >= tau && len > B) {
            scan = true;  // non-delegates may equal tau
          } else {
#pragma unroll
            for (int j = 0; j < B; ++j)
              cnt += (sm.dkeys[i * B + j] == tau && sm.dsegs[i * B + j] != kNoSeg) ? 1u : 0u;
          }
        }
      }
      // exact counts of the subranges that must be read: a warp each
      __syncthreads();
      if (tid == 0) s_cnt[3] = 0;
      __syncthreads();
      uint16_t* lst = reinterpret_cast<uint16_t*>(sm.ring + kTieOff);
      if (scan) lst[atomicAdd(&s_cnt[3], 1u)] = static_cast<uint16_t>(tid);
      __syncthreads();
      uint32_t* cnts = reinterpret_cast<uint32_t*>(sm.ring + kTieOff + size_t(kBT) * 2);
      cnts[tid] = cnt;
      __syncthreads();
      const uint32_t nscan = s_cnt[3];
      for (uint32_t q = warp; q < nscan; q += kBT / 32) {
        const int64_t ii = i0 + lst[q];
        const int64_t lo = ii << alpha;
        const int64_t len = imin64(int64_t(1) << alpha, n - lo);
        uint32_t c = 0;
        for (int64_t t = lane; t < len; t += 32) c += (map_key<DT>(rk[lo + t]) == tau);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        if (lane == 0) cnts[lst[q]] = c;
      }
      __syncthreads();
      uint32_t tot;
      const uint32_t pre = base + block_scan_excl<kBT>(cnts[tid], &tot);
      // emit: delegate-exact subranges by their thread, read ones by a warp
      if (i < S && !scan && cnts[tid] > 0 && pre < need) {
        uint32_t rr = pre;
#pragma unroll
        for (int j = 0; j < B; ++j) {
          if (sm.dkeys[i * B + j] == tau && sm.dsegs[i * B + j] != kNoSeg && rr < need) {
            int occ = 0;
            for (int q = 0; q < j; ++q)
              if (sm.dkeys[i * B + q] == tau && sm.dsegs[i * B + q] == sm.dsegs[i * B + j]) ++occ;
            const int64_t lo = (i << alpha) + int64_t(sm.dsegs[i * B + j]) * 32;
            const int64_t hi = imin64(imin64(n, lo + 32), (i + 1) << alpha);
            int64_t pos = -1;
            int cq = 0;
            for (int64_t t = lo; t < hi; ++t) {
              if (map_key<DT>(rk[t]) == tau) {
                if (cq == occ) {
                  pos = t;
                  break;
                }
                ++cq;
              }
            }
            if (pos < 0) atomicOr(p.err, kErrTieRank);
            w[gcnt + rr] = make_comp(tau, static_cast<uint32_t>(pos));
            ++rr;
          }
        }
      }
      uint32_t* pres = cnts + kBT;
      pres[tid] = pre;
      __syncthreads();
      for (uint32_t q = warp; q < nscan; q += kBT / 32) {
        const int64_t ii = i0 + lst[q];
        uint32_t rr = pres[lst[q]];
        const int64_t lo = ii << alpha;
        const int64_t len = imin64(int64_t(1) << alpha, n - lo);
        for (int64_t off = 0; off < len && rr < need; off += 32) {
          const int64_t t = off + lane;
          const bool is_t = t < len && map_key<DT>(rk[lo + t]) == tau;
          const uint32_t bal = __ballot_sync(0xFFFFFFFFu, is_t);
          const uint32_t rank = rr + __popc(bal & lanemask_lt_b());
          if (is_t && rank < need) w[gcnt + rank] = make_comp(tau, static_cast<uint32_t>(lo + t));
          rr += __popc(bal);
        }
      }
      base += tot;
      __syncthreads();
    }
    __syncthreads();
    phase_mark(p, 4, tmark);
  }

  // ------------------------------------------------- 5. write ------------
  for (uint32_t j = tid; j < k; j += kBT) {
    const uint64_t c = w[j];
    row_out_keys(p, r)[j] = unmap_key(DT, comp_key(c));
    row_out_idx(p, r)[j] = static_cast<int32_t>(comp_idx(c));
  }
  __syncthreads();
  phase_mark(p, 5, tmark);
}

template <int DT>
__global__ void __launch_bounds__(kBT, 1) batched_kernel(BatchParams p) {
  extern __shared__ __align__(128) unsigned char bsm[];
  __shared__ __align__(8) uint64_t bars[kBStages];
  __shared__ uint32_t hist[256];
  __shared__ unsigned long long mm[2];
  __shared__ uint32_t s_bc[4];
  __shared__ uint32_t s_cnt[4];
  __shared__ uint32_t s_row;
  __shared__ uint64_t s_lists[kBWarps * 4];
  Smem sm;
  sm.ring = bsm;
  sm.dkeys = reinterpret_cast<uint32_t*>(bsm + kRingBytes);
  sm.dsegs = reinterpret_cast<uint16_t*>(bsm + kRingBytes + size_t(kBDMax) * 4);
  sm.gbuf = reinterpret_cast<uint64_t*>(bsm + kRingBytes + size_t(kBDMax) * 6);
  Ring ring;
  ring.bar = bars;
  ring.seq = 0;
  ring.pol_first = l2_evict_first_policy();
  ring.pol_normal = l2_evict_normal_policy();
  if (threadIdx.x == 0) {
    for (int s = 0; s < kBStages; ++s) mbar_init(&bars[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) s_row = atomicAdd(p.row_ctr, 1u);
    __syncthreads();
    const uint32_t ri = s_row;
    __syncthreads();
    if (ri >= static_cast<uint32_t>(p.nrows)) break;
    const RowDesc r = p.rows[ri];
    switch (r.beta) {
      case 1: process_row<DT, 1>(p, r, sm, ring, hist, s_bc, s_cnt, s_lists, mm); break;
      case 3: process_row<DT, 3>(p, r, sm, ring, hist, s_bc, s_cnt, s_lists, mm); break;
      case 4: process_row<DT, 4>(p, r, sm, ring, hist, s_bc, s_cnt, s_lists, mm); break;
      default: process_row<DT, 2>(p, r, sm, ring, hist, s_bc, s_cnt, s_lists, mm); break;
    }
    // a bounded wait gave up: copies may still be in flight, stop this CTA
    if (__syncthreads_or(threadIdx.x == 0 && (__ldcg(p.err) & kErrTimeout))) break;
  }
}

// Fills every key with hashed bits (tuning inputs only).
__global__ void fill_hash_kernel(uint32_t* a, int64_t n, uint64_t seed) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    uint64_t z = seed + static_cast<uint64_t>(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    a[i] = static_cast<uint32_t>((z ^ (z >> 31)) >> 32);
  }
}

}  // namespace

cudaError_t launch_batched(int dtype, uint64_t keys_base, uint64_t out_keys_base,
                           uint64_t out_idx_base, const RowDesc* rows, int32_t nrows,
                           uint32_t* row_ctr, uint64_t* scratch, int64_t scap, uint32_t* err,
                           unsigned long long* phase, int grid, cudaStream_t s) {
  BatchParams p;
  p.keys_base = keys_base;
  p.out_keys_base = out_keys_base;
  p.out_idx_base = out_idx_base;
  p.rows = rows;
  p.nrows = nrows;
  p.row_ctr = row_ctr;
  p.scratch = scratch;
  p.scap = scap;
  p.err = err;
  p.phase = phase;
  switch (dtype) {
    case DRTOPK_U32:
      cudaFuncSetAttribute(batched_kernel<DRTOPK_U32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(kDynSmem));
      batched_kernel<DRTOPK_U32><<<grid, kBT, kDynSmem, s>>>(p);
      break;
    case DRTOPK_I32:
      cudaFuncSetAttribute(batched_kernel<DRTOPK_I32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(kDynSmem));
      batched_kernel<DRTOPK_I32><<<grid, kBT, kDynSmem, s>>>(p);
      break;
    default:
      cudaFuncSetAttribute(batched_kernel<DRTOPK_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(kDynSmem));
      batched_kernel<DRTOPK_F32><<<grid, kBT, kDynSmem, s>>>(p);
      break;
  }
  note_launch();
  return cudaGetLastError();
}


// ------------------------------------------------------------------------
// Host side: per-shape parameters, plans, the C ABI.
// ------------------------------------------------------------------------
namespace {

constexpr int kTuneN0 = 10, kTuneN1 = 31;  // log2 n buckets
constexpr int kTuneK1 = 12;                // log2 k buckets 0..12
struct TuneEntry {
  int alpha = 0;  // 0: not tuned, use Rule 4
  int beta = 0;
};
std::mutex g_tune_mu;
TuneEntry g_tune[kTuneN1 - kTuneN0 + 1][kTuneK1 + 1];

int ilog2_floor(int64_t v) {
  int l = 0;
  while ((int64_t(1) << (l + 1)) <= v) ++l;
  return l;
}

// Rule 4 / Eq. 9 (Sec. 4.2), const = 3, rounded down.
int rule4(int64_t n, int64_t k) {
  return static_cast<int>(std::floor(0.5 * (std::log2(double(n)) - std::log2(double(k)) + 3.0)));
}

struct RowPlan {
  int alpha, beta;
  int64_t gneed;  // candidate capacity the row may need
};

// Parameters of one row for the on-chip path: the forced or tuned (alpha,
// beta) of the row's shape bucket, else Rule 4 and beta = 2, lowered while
// fewer than 2k delegates would exist; in every case raised so that the
// delegates fit on chip (beta * S <= kBDMax, alpha >= 5).
RowPlan plan_row(int64_t n, int64_t k, int force_alpha, int force_beta) {
  const RowPlan direct{0, 0, 0};  // on-chip select, no scratch
  if (force_alpha <= 0 && n <= kBDirect) return direct;
  int a = 0, b = 0;
  {
    const int ln = std::min(std::max(ilog2_floor(n), kTuneN0), kTuneN1) - kTuneN0;
    const int lk = std::min(ilog2_floor(k), kTuneK1);
    std::lock_guard<std::mutex> lk2(g_tune_mu);
    a = g_tune[ln][lk].alpha;
    b = g_tune[ln][lk].beta;
  }
  if (force_alpha > 0) a = force_alpha;
  if (force_beta > 0) b = force_beta;
  if (b <= 0) b = 2;
  if (a == 1) {
    if (n <= kBDirectMax) return direct;
    a = 0;  // too long to hold on chip: Rule 4
  }
  const bool from_rule4 = a <= 0;
  // fewer than 2k delegates even with one segment per subrange: the
  // delegates cannot reduce the row, select it directly when it fits
  if (from_rule4 && n <= kBDirectMax && int64_t(b) * ((n + 31) / 32) < 2 * k) return direct;
  if (from_rule4) a = rule4(n, k);
  // delegates must fit on chip: beta * S <= kBDMax
  int amin = 5;
  while (amin < 16 && b * ((n + (int64_t(1) << amin) - 1) >> amin) > kBDMax) ++amin;
  a = std::max(a, amin);
  a = std::min(a, 16);
  if (from_rule4)
    while (a > amin && int64_t(b) * ((n + (int64_t(1) << a) - 1) >> a) < 2 * k) --a;
  const int64_t S = (n + (int64_t(1) << a) - 1) >> a;
  RowPlan rp;
  rp.alpha = a;
  rp.beta = b;
  rp.gneed = (int64_t(b) * S >= k) ? std::min<int64_t>(n, ((k - 1) / b) * (int64_t(1) << a) + k) : n;
  return rp;
}

// Copies `count` entries from a host or device pointer into `dst`.
template <class T>
bool fetch_host(const T* src, size_t count, std::vector<T>& dst) {
  dst.resize(count);
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, src) == cudaSuccess &&
      (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
    return cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost) == cudaSuccess;
  }
  cudaGetLastError();  // no device, or a plain host pointer
  std::copy(src, src + count, dst.begin());
  return true;
}

}  // namespace

BatchRowPlan batch_plan_row(int64_t n, int64_t k) {
  const RowPlan rp = plan_row(n, k, 0, 0);
  return {rp.alpha, rp.beta, rp.gneed};
}
int batch_grid(int sms) { return sms; }
int64_t batch_onchip_candidates() { return kBGS; }
int64_t batch_max_k() { return kBMaxK; }
int64_t batch_max_n() { return kBMaxN; }

}  // namespace drtopk

using namespace drtopk;

struct drtopk_batch_plan {
  int dtype = 0;
  int32_t rows = 0;
  int64_t total = 0;
  int grid = 0;
  int64_t scap = 0;
  RowDesc* d_rows = nullptr;     // device, processing order
  uint32_t* d_ctl = nullptr;     // [0] row counter, [1] error flags
  unsigned long long* d_phase = nullptr;  // kBPhases cycle counters
  uint64_t* d_scratch = nullptr;
  std::vector<int32_t> alpha, beta;  // per row, row order
};

extern "C" {

drtopk_status drtopk_batch_plan_create(drtopk_dtype dtype, const int64_t* row_off_in,
                                       const int32_t* ks_in, int32_t rows, int alpha, int beta,
                                       drtopk_batch_plan** out) {
  if (!out || !row_off_in || !ks_in || rows < 1) return DRTOPK_ERR_INVALID;
  std::vector<int64_t> off_h;
  std::vector<int32_t> ks_h;
  if (!fetch_host(row_off_in, static_cast<size_t>(rows) + 1, off_h) ||
      !fetch_host(ks_in, static_cast<size_t>(rows), ks_h))
    return DRTOPK_ERR_CUDA;
  const int64_t* row_off = off_h.data();
  const int32_t* ks = ks_h.data();
  if (dtype != DRTOPK_U32 && dtype != DRTOPK_I32 && dtype != DRTOPK_F32) return DRTOPK_ERR_DTYPE;
  if (alpha < 0 || alpha > 16 || (alpha > 1 && alpha < 5) || beta < 0 || beta > kMaxBeta)
    return DRTOPK_ERR_INVALID;
  if (row_off[0] < 0) return DRTOPK_ERR_INVALID;
  std::vector<RowDesc> rd(static_cast<size_t>(rows));
  std::vector<int32_t> ra(static_cast<size_t>(rows)), rb(static_cast<size_t>(rows));
  int64_t out_pos = 0, scap = 0;
  for (int32_t r = 0; r < rows; ++r) {
    const int64_t n = row_off[r + 1] - row_off[r];
    const int64_t k = ks[r];
    if (n < 1 || n > kBMaxN) return DRTOPK_ERR_INVALID;
    if (k < 1 || k > n || k > kBMaxK) return DRTOPK_ERR_K;
    const RowPlan rp = plan_row(n, k, alpha, beta);
    rd[r].keys = static_cast<uint64_t>(row_off[r]) * 4;
    rd[r].out_keys = static_cast<uint64_t>(out_pos) * 4;
    rd[r].out_idx = static_cast<uint64_t>(out_pos) * 4;
    rd[r].n = static_cast<int32_t>(n);
    rd[r].k = static_cast<int32_t>(k);
    rd[r].alpha = rp.alpha;
    rd[r].beta = rp.beta;
    ra[r] = rp.alpha;
    rb[r] = rp.beta;
    out_pos += k;
    scap = std::max<int64_t>(scap, rp.gneed - kBGS);
  }
  // largest rows first: the CTAs that take them start earliest
  std::stable_sort(rd.begin(), rd.end(), [](const RowDesc& a, const RowDesc& b) { return a.n > b.n; });
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DRTOPK_ERR_CUDA;
  auto* pl = new drtopk_batch_plan;
  pl->dtype = dtype;
  pl->rows = rows;
  pl->total = row_off[rows];
  pl->grid = std::min<int>(sms, rows);
  pl->scap = std::max<int64_t>(scap, 1);
  pl->alpha = std::move(ra);
  pl->beta = std::move(rb);
  note_alloc(4);  // rows, control words, phase counters, scratch
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&pl->d_rows), rd.size() * sizeof(RowDesc));
  if (e == cudaSuccess)
    e = cudaMemcpy(pl->d_rows, rd.data(), rd.size() * sizeof(RowDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&pl->d_ctl), 2 * sizeof(uint32_t));
  if (e == cudaSuccess)
    e = cudaMalloc(reinterpret_cast<void**>(&pl->d_phase), kBPhases * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(pl->d_phase, 0, kBPhases * sizeof(unsigned long long));
  if (e == cudaSuccess)
    e = cudaMalloc(reinterpret_cast<void**>(&pl->d_scratch),
                   static_cast<size_t>(pl->grid) * pl->scap * sizeof(uint64_t));
  if (e != cudaSuccess) {
    cudaFree(pl->d_rows);
    cudaFree(pl->d_ctl);
    cudaFree(pl->d_phase);
    cudaFree(pl->d_scratch);
    delete pl;
    return e == cudaErrorMemoryAllocation ? DRTOPK_ERR_NOMEM : DRTOPK_ERR_CUDA;
  }
  *out = pl;
  return DRTOPK_OK;
}

drtopk_status drtopk_batch_limits(int32_t* max_k, int64_t* max_row, int32_t* direct_max,
                                  int32_t* direct_max_onchip, int32_t* max_delegates,
                                  int32_t* onchip_candidates) {
  if (max_k) *max_k = kBMaxK;
  if (max_row) *max_row = kBMaxN;
  if (direct_max) *direct_max = kBDirect;
  if (direct_max_onchip) *direct_max_onchip = kBDirectMax;
  if (max_delegates) *max_delegates = kBDMax;
  if (onchip_candidates) *onchip_candidates = kBGS;
  return DRTOPK_OK;
}

drtopk_status drtopk_batch_plan_run(drtopk_batch_plan* pl, const void* keys, void* out_keys,
                                    int32_t* out_idx, void* stream) {
  if (!pl || !keys || !out_keys || !out_idx) return DRTOPK_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(out_keys) |
       reinterpret_cast<uintptr_t>(out_idx)) & 3u)
    return DRTOPK_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(pl->d_ctl, 0, 2 * sizeof(uint32_t), s);
  if (e == cudaSuccess)
    e = launch_batched(pl->dtype, reinterpret_cast<uint64_t>(keys),
                       reinterpret_cast<uint64_t>(out_keys), reinterpret_cast<uint64_t>(out_idx),
                       pl->d_rows, pl->rows, pl->d_ctl, pl->d_scratch, pl->scap, pl->d_ctl + 1,
                       pl->d_phase, pl->grid, s);
  return e == cudaSuccess ? DRTOPK_OK : (e == cudaErrorMemoryAllocation ? DRTOPK_ERR_NOMEM : DRTOPK_ERR_CUDA);
}

drtopk_status drtopk_batch_plan_status(drtopk_batch_plan* pl, void* stream) {
  if (!pl) return DRTOPK_ERR_INVALID;
  uint32_t err = 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&err, pl->d_ctl + 1, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return DRTOPK_ERR_CUDA;
  if (err & kErrTimeout) return DRTOPK_ERR_TIMEOUT;
  return err ? DRTOPK_ERR_CUDA : DRTOPK_OK;
}

drtopk_status drtopk_batch_plan_params(const drtopk_batch_plan* pl, int32_t* alpha,
                                       int32_t* beta) {
  if (!pl || !alpha || !beta) return DRTOPK_ERR_INVALID;
  std::copy(pl->alpha.begin(), pl->alpha.end(), alpha);
  std::copy(pl->beta.begin(), pl->beta.end(), beta);
  return DRTOPK_OK;
}

drtopk_status drtopk_batch_plan_phase_cycles(drtopk_batch_plan* pl, uint64_t* out, int reset,
                                             void* stream) {
  if (!pl || !out) return DRTOPK_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long h[kBPhases];
  cudaError_t e = cudaMemcpyAsync(h, pl->d_phase, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && reset) e = cudaMemsetAsync(pl->d_phase, 0, sizeof(h), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return DRTOPK_ERR_CUDA;
  for (int i = 0; i < kBPhases; ++i) out[i] = h[i];
  return DRTOPK_OK;
}

drtopk_status drtopk_batch_plan_destroy(drtopk_batch_plan* pl) {
  if (!pl) return DRTOPK_ERR_INVALID;
  cudaDeviceSynchronize();
  cudaFree(pl->d_rows);
  cudaFree(pl->d_ctl);
  cudaFree(pl->d_phase);
  cudaFree(pl->d_scratch);
  delete pl;
  return DRTOPK_OK;
}

drtopk_status drtopk_topk_batched(const void* keys, drtopk_dtype dtype, const int64_t* row_off,
                                  const int32_t* ks, int32_t rows, void* out_keys,
                                  int32_t* out_idx, void* stream) {
  drtopk_batch_plan* pl = nullptr;
  drtopk_status st = drtopk_batch_plan_create(dtype, row_off, ks, rows, 0, 0, &pl);
  if (st != DRTOPK_OK) return st;
  st = drtopk_batch_plan_run(pl, keys, out_keys, out_idx, stream);
  if (st == DRTOPK_OK) st = drtopk_batch_plan_status(pl, stream);
  drtopk_batch_plan_destroy(pl);
  return st;
}

drtopk_status drtopk_tune_get(int32_t log2n, int32_t log2k, int* alpha, int* beta) {
  if (log2n < kTuneN0 || log2n > kTuneN1 || log2k < 0 || log2k > kTuneK1 || !alpha || !beta)
    return DRTOPK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  *alpha = g_tune[log2n - kTuneN0][log2k].alpha;
  *beta = g_tune[log2n - kTuneN0][log2k].beta;
  return DRTOPK_OK;
}

drtopk_status drtopk_tune_set(int32_t log2n, int32_t log2k, int alpha, int beta) {
  if (log2n < kTuneN0 || log2n > kTuneN1 || log2k < 0 || log2k > kTuneK1) return DRTOPK_ERR_INVALID;
  if (alpha < 0 || alpha > 16 || (alpha > 1 && alpha < 5) || beta < 0 || beta > kMaxBeta)
    return DRTOPK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[log2n - kTuneN0][log2k].alpha = alpha;
  g_tune[log2n - kTuneN0][log2k].beta = beta;
  return DRTOPK_OK;
}

// Measures, for every (log2 n, log2 k) bucket with min_log2n <= log2 n <=
// max_log2n and 2^(log2 k) <= min(4096, n / 2), the batched kernel on
// `rows_per_shape` rows of 2^log2n hashed keys with k = 2^(log2 k + 1/2):
// the direct select (rows that fit on chip) and alpha in [Rule 4 - 3,
// Rule 4 + 2] with beta in {1, 2, 3, 4}; stores the fastest choice.
drtopk_status drtopk_autotune_batched(drtopk_dtype dtype, int32_t min_log2n, int32_t max_log2n,
                                      int32_t rows_per_shape, void* stream) {
  if (min_log2n < kTuneN0 || max_log2n > 24 || min_log2n > max_log2n || rows_per_shape < 1)
    return DRTOPK_ERR_INVALID;
  if (dtype != DRTOPK_U32 && dtype != DRTOPK_I32 && dtype != DRTOPK_F32) return DRTOPK_ERR_DTYPE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t maxn = int64_t(1) << max_log2n;
  const int64_t total = maxn * rows_per_shape;
  uint32_t* d_keys = nullptr;
  uint32_t* d_ok = nullptr;
  int32_t* d_oi = nullptr;
  note_alloc(3);
  if (cudaMalloc(reinterpret_cast<void**>(&d_keys), total * 4) != cudaSuccess) return DRTOPK_ERR_NOMEM;
  if (cudaMalloc(reinterpret_cast<void**>(&d_ok), size_t(kBMaxK) * rows_per_shape * 4) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&d_oi), size_t(kBMaxK) * rows_per_shape * 4) != cudaSuccess) {
    cudaFree(d_keys);
    cudaFree(d_ok);
    return DRTOPK_ERR_NOMEM;
  }
  fill_hash_kernel<<<1024, 256, 0, s>>>(d_keys, total, 0x5EEDull);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  drtopk_status st = DRTOPK_OK;
  for (int ln = min_log2n; ln <= max_log2n && st == DRTOPK_OK; ++ln) {
    const int64_t n = int64_t(1) << ln;
    std::vector<int64_t> off(rows_per_shape + 1);
    for (int r = 0; r <= rows_per_shape; ++r) off[r] = r * n;
    if (n <= kBDirect) continue;  // always selected directly
    for (int lk = 0; lk <= kTuneK1 && (int64_t(1) << lk) <= std::min<int64_t>(kBMaxK, n / 2); ++lk) {
      // a k in the middle of the bucket [2^lk, 2^(lk+1))
      const int32_t k = static_cast<int32_t>(std::min<int64_t>(
          std::min<int64_t>(kBMaxK, n / 2), std::llround(std::exp2(lk + 0.5))));
      std::vector<int32_t> kv(rows_per_shape, k);
      const int a4 = rule4(n, k);
      std::vector<std::pair<int, int>> cand;
      if (n <= kBDirectMax) cand.push_back({1, 0});
      for (int b = 1; b <= 4; ++b)
        for (int a = std::max(5, a4 - 3); a <= std::min(16, a4 + 2); ++a) cand.push_back({a, b});
      float best = 1e30f;
      int best_a = 0, best_b = 0;
      for (const auto& ab : cand) {
        if (st != DRTOPK_OK) break;
        drtopk_batch_plan* pl = nullptr;
        if (drtopk_batch_plan_create(dtype, off.data(), kv.data(), rows_per_shape, ab.first,
                                     ab.second, &pl) != DRTOPK_OK)
          continue;
        float ms_best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
          cudaEventRecord(e0, s);
          drtopk_batch_plan_run(pl, d_keys, d_ok, d_oi, s);
          cudaEventRecord(e1, s);
          cudaEventSynchronize(e1);
          float ms = 0;
          cudaEventElapsedTime(&ms, e0, e1);
          ms_best = std::min(ms_best, ms);
        }
        if (drtopk_batch_plan_status(pl, s) != DRTOPK_OK) st = DRTOPK_ERR_CUDA;
        drtopk_batch_plan_destroy(pl);
        if (ms_best < best) {
          best = ms_best;
          best_a = ab.first;
          best_b = ab.second;
        }
      }
      if (best_a > 0) drtopk_tune_set(ln, lk, best_a, best_b);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_keys);
  cudaFree(d_ok);
  cudaFree(d_oi);
  return st;
}

}  // extern "C"
