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
