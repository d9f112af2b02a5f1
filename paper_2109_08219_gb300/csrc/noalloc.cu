// k-selection that allocates nothing: its scratch is a fixed device array
// that lives in this library for the life of the process.
//
// Who needs this: callers that must not allocate device memory while they
// serve queries. Examples are real-time or certified pipelines that forbid
// any allocation after start-up, and processes whose device memory is owned
// entirely by another allocator (a framework's caching pool sized to the
// whole GPU), where a driver allocation at query time may fail or fragment.
// drtopk_kth allocates its workspace from the stream-ordered pool on every
// call; drtopk_kth_noalloc runs the same kernels on the fixed array instead.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "launch.h"

namespace drtopk {
namespace {

// Scratch of every drtopk_kth_noalloc call on a device. Each GPU that loads
// the library holds these bytes until the process exits.
constexpr size_t kScratchBytes = size_t(64) << 20;  // 64 MiB
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr size_t kAl = 256;
size_t al(size_t b) { return (b + kAl - 1) & ~(kAl - 1); }

// Device address of the scratch array, looked up once per device (with that
// device current). Host code cannot use the array's name as an address.
std::mutex g_mu;
void* g_addr[64];

cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace drtopk

using namespace drtopk;

extern "C" drtopk_status drtopk_kth_noalloc(const void* keys, drtopk_dtype dtype, int64_t n,
                                            int64_t k, void* out_kth, void* stream) {
  if (dtype != DRTOPK_U32 && dtype != DRTOPK_I32 && dtype != DRTOPK_F32) return DRTOPK_ERR_DTYPE;
  if (n < 1 || n > 0x7FFFFFFFLL) return DRTOPK_ERR_INVALID;
  if (k < 1 || k > n) return DRTOPK_ERR_K;
  if (!keys || (reinterpret_cast<uintptr_t>(keys) & 3u) || !out_kth) return DRTOPK_ERR_INVALID;
  int alpha = 0, beta = 0;
  drtopk_status st = drtopk_plan(n, k, &alpha, &beta, nullptr);
  if (st != DRTOPK_OK) return st;

  // The kernels of the k-selection path need: control block, delegate keys
  // and segments, the delegate keys kept by the first threshold digit, the
  // queues of subranges to scan and of delegates to place, the candidates
  // above the threshold and their survivors.
  const int64_t S = (n + (int64_t(1) << alpha) - 1) >> alpha;
  int64_t g_cap = n;
  if (static_cast<int64_t>(beta) * S >= k)
    g_cap = std::min<int64_t>(n, ((k - 1) / beta) * (int64_t(1) << alpha) + k);
  const size_t o_ctl = 0;
  const size_t o_dk = o_ctl + al(sizeof(Ctl));
  const size_t o_ds = o_dk + al(static_cast<size_t>(S) * beta * 4);
  const size_t o_dsv = o_ds + al(static_cast<size_t>(S) * beta * 2);
  const size_t o_q = o_dsv + al(static_cast<size_t>(S) * beta * 4);
  // delegates > tau queued for position resolution: fewer than k, or all
  // beta S of them when there are fewer than k
  const int64_t rq_cap = std::max<int64_t>(1, std::min<int64_t>(S * beta, k));
  const size_t o_rq = o_q + al(static_cast<size_t>(S) * 4);
  const size_t o_g = o_rq + al(static_cast<size_t>(rq_cap) * 4);
  const size_t o_sv = o_g + al(static_cast<size_t>(g_cap) * 8);
  const size_t total = o_sv + al(static_cast<size_t>(g_cap) * 8);
  if (total > kScratchBytes) return DRTOPK_ERR_NOMEM;  // does not fit the fixed scratch

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DRTOPK_ERR_CUDA;
  void* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return DRTOPK_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DRTOPK_ERR_CUDA;

  char* ws = static_cast<char*>(base);
  Work w{};
  w.ctl = reinterpret_cast<Ctl*>(ws + o_ctl);
  w.dkeys = reinterpret_cast<uint32_t*>(ws + o_dk);
  w.dsegs = reinterpret_cast<uint16_t*>(ws + o_ds);
  w.ds = reinterpret_cast<uint32_t*>(ws + o_dsv);
  w.scanq = reinterpret_cast<uint32_t*>(ws + o_q);
  w.rq = reinterpret_cast<uint32_t*>(ws + o_rq);
  w.rq_cap = rq_cap;
  w.g = reinterpret_cast<uint64_t*>(ws + o_g);
  w.sv = reinterpret_cast<uint64_t*>(ws + o_sv);
  w.n = n;
  w.S = S;
  w.g_cap = g_cap;
  w.k = k;
  w.alpha = alpha;
  w.beta = beta;
  w.dtype = dtype;
  const bool fuse = static_cast<int64_t>(beta) * S >= k;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // The array keeps the previous call's contents: the control block (counters,
  // histograms, threshold) must start at zero; everything else is written
  // before it is read.
  cudaError_t e = cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), s);
  if (e == cudaSuccess) {
    e = launch_delegates(w, keys, fuse, sms, s);
    note_launch();
  }
  if (e == cudaSuccess && fuse) e = launch_threshold(w, sms, s);
  if (e == cudaSuccess) e = launch_filter(w, keys, true, sms, s);
  if (e == cudaSuccess) e = launch_gselect(w, true, sms, s);
  if (e == cudaSuccess) e = launch_write_kth(w, out_kth, s);
  if (e == cudaErrorMemoryAllocation) return DRTOPK_ERR_NOMEM;
  return e == cudaSuccess ? DRTOPK_OK : DRTOPK_ERR_CUDA;
}
