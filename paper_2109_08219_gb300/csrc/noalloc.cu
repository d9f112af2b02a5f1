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
// Device error flags of the calls since the last drtopk_sync_status.
__device__ uint32_t g_noalloc_err;

// Device addresses of the scratch array and the error word, looked up once
// per device (with that device current). Host code cannot use the arrays'
// names as addresses.
std::mutex g_mu;
void* g_addr[64];
uint32_t* g_err_addr[64];

cudaError_t scratch_address(int dev, void** out, uint32_t** err) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    void* q = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    e = cudaGetSymbolAddress(&q, g_noalloc_err);
    if (e != cudaSuccess) return e;
    g_err_addr[dev] = static_cast<uint32_t*>(q);
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  *err = g_err_addr[dev];
  return cudaSuccess;
}

}  // namespace

uint32_t take_noalloc_errors() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_addr[dev] == nullptr) return 0;  // never ran on this device
  }
  uint32_t v = 0;
  if (cudaMemcpyFromSymbol(&v, g_noalloc_err, sizeof(v)) != cudaSuccess) return kErrTimeout;
  if (v) {
    const uint32_t zero = 0;
    cudaMemcpyToSymbol(g_noalloc_err, &zero, sizeof(zero));
  }
  return v;
}

}  // namespace drtopk

using namespace drtopk;

extern "C" drtopk_status drtopk_kth_noalloc(const void* keys, drtopk_dtype dtype, int64_t n,
                                            int64_t k, void* out_kth, void* stream) {
  if (dtype != DRTOPK_U32 && dtype != DRTOPK_I32 && dtype != DRTOPK_F32) return DRTOPK_ERR_DTYPE;
  if (n < 1 || n > 0x7FFFFFFFLL) return DRTOPK_ERR_INVALID;
  if (k < 1 || k > n) return DRTOPK_ERR_K;
  if (!keys || (reinterpret_cast<uintptr_t>(keys) & 3u) || !out_kth) return DRTOPK_ERR_INVALID;
  Plan P;
  if (!make_plan(n, k, 0, 0, &P)) return DRTOPK_ERR_INVALID;
  // the k-selection workspace of drtopk_kth (control block, delegate keys
  // and segments, first-digit survivors, filter queues, the candidates
  // above the threshold and their survivors), laid out as drtopk_kth does
  const Layout L = layout(P, k, /*need_topk=*/false, /*external_dkeys=*/false);
  if (L.total > kScratchBytes) return DRTOPK_ERR_NOMEM;  // does not fit the fixed scratch

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DRTOPK_ERR_CUDA;
  void* base = nullptr;
  uint32_t* err = nullptr;
  if (scratch_address(dev, &base, &err) != cudaSuccess) return DRTOPK_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return DRTOPK_ERR_CUDA;

  Work w{};
  bind_work(w, static_cast<char*>(base), L, P, n, k, dtype);
  w.err_out = err;
  // The array keeps the previous call's contents: the query's first launch
  // zeroes the control block (counters, histograms, threshold); everything
  // else is written before it is read.
  const cudaError_t e = enqueue_query_plain(w, P, keys, /*topk=*/false, nullptr, nullptr,
                                            out_kth, sms, static_cast<cudaStream_t>(stream));
  if (e == cudaErrorMemoryAllocation) return DRTOPK_ERR_NOMEM;
  return e == cudaSuccess ? DRTOPK_OK : DRTOPK_ERR_CUDA;
}
