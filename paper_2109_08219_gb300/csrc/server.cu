// Served top-k: requests arrive at any time from any host thread; a
// scheduler thread admits them in arrival order while the device-resident
// state of the admitted requests (their keys, outputs and workspace) fits
// an HBM budget, coalesces the admitted small requests into batched
// launches (one persistent kernel over all of them, the batched form of the
// method), runs the large ones as single queries on their own streams so
// that they overlap, and retires everything by polling CUDA events. There
// is no counterpart in the paper, which answers one query per call.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "launch.h"

namespace drtopk {
namespace {

using Clock = std::chrono::steady_clock;

constexpr int kQueryStreams = 4;    // streams for single queries (overlap)
constexpr int kBatchCtxs = 2;       // batched launches in flight
constexpr int kMaxBatchRows = 4096; // rows of one batched launch
constexpr int64_t kScratchPerCta = int64_t(1) << 18;  // spilled candidates per CTA
constexpr int64_t kDefaultBatchMaxN = int64_t(1) << 20;

enum ReqState { kQueued = 0, kRunning = 1, kDone = 2 };

struct Req {
  const void* keys;
  int dtype;
  int64_t n, k;
  void* out_keys;
  int32_t* out_idx;
  size_t bytes;
  bool batched;
  int state;
  drtopk_status status;
  Clock::time_point t_submit, t_done;
};

struct BatchCtx {
  RowDesc* d_rows = nullptr;
  RowDesc* h_rows = nullptr;  // pinned staging
  uint32_t* d_ctl = nullptr;  // [0] row counter, [1] error flags
  unsigned long long* d_phase = nullptr;
  uint64_t* d_scratch = nullptr;
  uint32_t* h_err = nullptr;  // pinned copy of the error flags
  cudaStream_t stream = nullptr;
  bool busy = false;
};

struct Unit {
  cudaEvent_t ev;
  std::vector<uint64_t> tickets;
  int ctx;       // batch context, or -1 for a single query
  int err_slot;  // single query: its report word, or -1
};

// Report words of single queries in flight: host-mapped pinned words in
// blocks of 256, recycled as queries retire (scheduler thread only).
struct ErrSlots {
  static constexpr int kBlock = 256;
  std::vector<uint32_t*> host_blocks, dev_blocks;
  std::vector<int> free_slots;
  cudaError_t take(int* slot) {
    if (free_slots.empty()) {
      uint32_t* h = nullptr;
      uint32_t* d = nullptr;
      cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&h), kBlock * sizeof(uint32_t),
                                    cudaHostAllocMapped);
      note_alloc();
      if (e != cudaSuccess) return e;
      e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&d), h, 0);
      if (e != cudaSuccess) {
        cudaFreeHost(h);
        return e;
      }
      const int b = static_cast<int>(host_blocks.size());
      host_blocks.push_back(h);
      dev_blocks.push_back(d);
      for (int i = kBlock - 1; i >= 0; --i) free_slots.push_back(b * kBlock + i);
    }
    *slot = free_slots.back();
    free_slots.pop_back();
    host(*slot) = 0;
    return cudaSuccess;
  }
  uint32_t& host(int slot) { return host_blocks[slot / kBlock][slot % kBlock]; }
  uint32_t* dev(int slot) { return dev_blocks[slot / kBlock] + slot % kBlock; }
  void give(int slot) { free_slots.push_back(slot); }
  void release() {
    for (uint32_t* h : host_blocks) cudaFreeHost(h);
    host_blocks.clear();
    dev_blocks.clear();
    free_slots.clear();
  }
};

size_t single_workspace(int64_t n, int64_t k) {
  size_t ws = 0;
  if (drtopk_plan(n, k, nullptr, nullptr, &ws) != DRTOPK_OK) return 0;
  return ws;
}

// Small requests go to batched launches: rows the batched kernel takes
// (k and n within its limits, spilled candidates within the per-CTA
// scratch) up to max_n keys.
bool batchable(int flags, int64_t max_n, int64_t n, int64_t k) {
  if (flags & DRTOPK_SERVER_PLAIN) return false;
  if (n > max_n || n > batch_max_n() || k > batch_max_k()) return false;
  const BatchRowPlan rp = batch_plan_row(n, k);
  return rp.gneed - batch_onchip_candidates() <= kScratchPerCta;
}

}  // namespace
}  // namespace drtopk

using namespace drtopk;

struct drtopk_server {
  int device = 0;
  size_t budget = 0;
  size_t fixed = 0;  // the server's own device memory
  int flags = 0;
  int64_t max_batch_n = kDefaultBatchMaxN;
  int sms = 0;
  int grid = 0;

  std::mutex mu;
  std::condition_variable cv_work;  // new requests, stop
  std::condition_variable cv_done;  // completions
  std::unordered_map<uint64_t, Req> reqs;
  std::deque<uint64_t> queued;
  uint64_t next_ticket = 1;
  size_t in_use = 0;
  bool stop = false;
  drtopk_server_stats stats{};

  // owned by the scheduler thread
  cudaStream_t qs[kQueryStreams] = {};
  BatchCtx ctx[kBatchCtxs];
  std::vector<Unit> inflight;
  ErrSlots err_slots;
  std::vector<cudaEvent_t> events;
  std::vector<uint64_t> ready_small;
  int next_qs = 0;
  std::thread worker;

  cudaEvent_t get_event() {
    if (!events.empty()) {
      cudaEvent_t e = events.back();
      events.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    return e;
  }

  // Marks tickets finished (scheduler thread).
  void finish(const std::vector<uint64_t>& ts, drtopk_status st) {
    const auto now = Clock::now();
    {
      std::lock_guard<std::mutex> lk(mu);
      for (uint64_t t : ts) {
        auto it = reqs.find(t);
        if (it == reqs.end()) continue;
        Req& r = it->second;
        r.state = kDone;
        r.status = st;
        r.t_done = now;
        in_use -= r.bytes;
        ++stats.completed;
        if (st != DRTOPK_OK) ++stats.failed;
      }
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }

  bool retire() {
    bool any = false;
    for (size_t i = 0; i < inflight.size();) {
      Unit& u = inflight[i];
      const cudaError_t q = cudaEventQuery(u.ev);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      drtopk_status st = q == cudaSuccess ? DRTOPK_OK : DRTOPK_ERR_CUDA;
      if (q != cudaSuccess) cudaGetLastError();
      if (u.ctx >= 0) {
        const uint32_t e = *ctx[u.ctx].h_err;
        if (st == DRTOPK_OK && e) st = (e & kErrTimeout) ? DRTOPK_ERR_TIMEOUT : DRTOPK_ERR_INTERNAL;
        ctx[u.ctx].busy = false;
      }
      if (u.err_slot >= 0) {
        const uint32_t e = *reinterpret_cast<volatile uint32_t*>(&err_slots.host(u.err_slot));
        if (st == DRTOPK_OK) st = error_status(e);
        err_slots.give(u.err_slot);
      }
      finish(u.tickets, st);
      events.push_back(u.ev);
      inflight[i] = inflight.back();
      inflight.pop_back();
      any = true;
    }
    return any;
  }

  void launch_single(uint64_t t, const Req& r) {
    cudaStream_t s = qs[(flags & DRTOPK_SERVER_PLAIN) ? 0 : (next_qs++ % kQueryStreams)];
    int slot = -1;
    if (err_slots.take(&slot) != cudaSuccess) {
      cudaGetLastError();
      finish({t}, DRTOPK_ERR_NOMEM);
      return;
    }
    const drtopk_status st = topk_kernel_by_kernel(r.keys, r.dtype, r.n, r.k, r.out_keys,
                                                   r.out_idx, err_slots.dev(slot), s);
    if (st != DRTOPK_OK) {
      err_slots.give(slot);
      finish({t}, st);
      return;
    }
    Unit u;
    u.ev = get_event();
    u.ctx = -1;
    u.err_slot = slot;
    u.tickets.push_back(t);
    if (cudaEventRecord(u.ev, s) != cudaSuccess) {
      cudaGetLastError();
      events.push_back(u.ev);
      finish({t}, DRTOPK_ERR_CUDA);
      return;
    }
    inflight.push_back(std::move(u));
    std::lock_guard<std::mutex> lk(mu);
    ++stats.single_queries;
  }

  // Coalesces admitted small requests of one dtype into one batched launch.
  bool launch_batch() {
    int c = -1;
    for (int i = 0; i < kBatchCtxs; ++i)
      if (!ctx[i].busy) c = i;
    if (c < 0 || ready_small.empty()) return false;
    BatchCtx& bc = ctx[c];
    std::vector<uint64_t> take, keep;
    std::vector<RowDesc> rows;
    int dtype = -1;
    {
      std::lock_guard<std::mutex> lk(mu);
      dtype = reqs[ready_small.front()].dtype;
      for (uint64_t t : ready_small) {
        const Req& r = reqs[t];
        if (r.dtype != dtype || static_cast<int>(take.size()) >= kMaxBatchRows) {
          keep.push_back(t);
          continue;
        }
        take.push_back(t);
        const BatchRowPlan rp = batch_plan_row(r.n, r.k);
        RowDesc d;
        d.keys = reinterpret_cast<uint64_t>(r.keys);
        d.out_keys = reinterpret_cast<uint64_t>(r.out_keys);
        d.out_idx = reinterpret_cast<uint64_t>(r.out_idx);
        d.n = static_cast<int32_t>(r.n);
        d.k = static_cast<int32_t>(r.k);
        d.alpha = rp.alpha;
        d.beta = rp.beta;
        rows.push_back(d);
      }
    }
    ready_small.swap(keep);
    // longest rows first: the CTAs that take them start earliest
    std::stable_sort(rows.begin(), rows.end(),
                     [](const RowDesc& a, const RowDesc& b) { return a.n > b.n; });
    std::copy(rows.begin(), rows.end(), bc.h_rows);
    const int nrows = static_cast<int>(rows.size());
    cudaError_t e = cudaMemcpyAsync(bc.d_rows, bc.h_rows, nrows * sizeof(RowDesc),
                                    cudaMemcpyHostToDevice, bc.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(bc.d_ctl, 0, 2 * sizeof(uint32_t), bc.stream);
    if (e == cudaSuccess)
      e = launch_batched(dtype, 0, 0, 0, bc.d_rows, nrows, bc.d_ctl, bc.d_scratch, kScratchPerCta,
                         bc.d_ctl + 1, bc.d_phase, std::min(grid, nrows), bc.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bc.h_err, bc.d_ctl + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                          bc.stream);
    Unit u;
    u.ev = get_event();
    u.ctx = c;
    u.err_slot = -1;
    u.tickets = take;
    if (e == cudaSuccess) e = cudaEventRecord(u.ev, bc.stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      events.push_back(u.ev);
      finish(take, DRTOPK_ERR_CUDA);
      return true;
    }
    bc.busy = true;
    inflight.push_back(std::move(u));
    std::lock_guard<std::mutex> lk(mu);
    ++stats.batches;
    stats.batched_requests += take.size();
    return true;
  }

  void run() {
    cudaSetDevice(device);
    for (;;) {
      bool progress = retire();
      std::vector<uint64_t> big;
      bool done = false;
      {
        std::unique_lock<std::mutex> lk(mu);
        // admission in arrival order while the budget allows
        while (!queued.empty()) {
          Req& r = reqs[queued.front()];
          if (in_use + r.bytes > budget - fixed) break;
          in_use += r.bytes;
          stats.peak_bytes = std::max<uint64_t>(stats.peak_bytes, in_use + fixed);
          r.state = kRunning;
          (r.batched ? ready_small : big).push_back(queued.front());
          queued.pop_front();
          progress = true;
        }
        done = stop && queued.empty() && ready_small.empty() && big.empty() && inflight.empty();
        if (!progress && !done && inflight.empty() && ready_small.empty())
          cv_work.wait_for(lk, std::chrono::milliseconds(1));
      }
      if (done) break;
      for (uint64_t t : big) {
        Req r;
        {
          std::lock_guard<std::mutex> lk(mu);
          r = reqs[t];
        }
        launch_single(t, r);
      }
      while (launch_batch()) progress = true;
      if (!progress && !inflight.empty()) std::this_thread::yield();
    }
  }

  void release() {
    for (auto& c : ctx) {
      if (c.stream) cudaStreamSynchronize(c.stream);
      cudaFree(c.d_rows);
      cudaFreeHost(c.h_rows);
      cudaFree(c.d_ctl);
      cudaFree(c.d_phase);
      cudaFree(c.d_scratch);
      cudaFreeHost(c.h_err);
      if (c.stream) cudaStreamDestroy(c.stream);
      c = BatchCtx();
    }
    for (auto& s : qs) {
      if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
      s = nullptr;
    }
    for (auto& u : inflight) cudaEventDestroy(u.ev);
    inflight.clear();
    err_slots.release();
    for (auto e : events) cudaEventDestroy(e);
    events.clear();
  }
};

extern "C" {

drtopk_status drtopk_server_footprint(drtopk_dtype dtype, int64_t n, int64_t k, int flags,
                                      int64_t batch_max_n, size_t* bytes, int* batched) {
  if (dtype != DRTOPK_U32 && dtype != DRTOPK_I32 && dtype != DRTOPK_F32) return DRTOPK_ERR_DTYPE;
  if (n < 1 || n > 0x7FFFFFFFLL) return DRTOPK_ERR_INVALID;
  if (k < 1 || k > n) return DRTOPK_ERR_K;
  const bool b = batchable(flags, batch_max_n > 0 ? batch_max_n : kDefaultBatchMaxN, n, k);
  const size_t io = static_cast<size_t>(n) * 4 + static_cast<size_t>(k) * 8;
  if (bytes) *bytes = io + (b ? 0 : single_workspace(n, k));
  if (batched) *batched = b ? 1 : 0;
  return DRTOPK_OK;
}

drtopk_status drtopk_server_create_ex(size_t hbm_budget_bytes, int device, int flags,
                                      int64_t batch_max_n, drtopk_server** out) {
  if (!out || device < 0 || (flags & ~DRTOPK_SERVER_PLAIN)) return DRTOPK_ERR_INVALID;
  if (batch_max_n < 0) return DRTOPK_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return DRTOPK_ERR_CUDA;
  }
  if (device >= ndev) return DRTOPK_ERR_INVALID;
  // the set-up below runs on `device`; the caller's current device is
  // restored before returning
  int prev_dev = 0;
  if (cudaGetDevice(&prev_dev) != cudaSuccess) {
    cudaGetLastError();
    return DRTOPK_ERR_CUDA;
  }
  auto* S = new drtopk_server;
  S->device = device;
  S->budget = hbm_budget_bytes;
  S->flags = flags;
  S->max_batch_n = batch_max_n > 0 ? batch_max_n : kDefaultBatchMaxN;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, device);
  S->grid = batch_grid(S->sms);
  for (int i = 0; i < kQueryStreams && e == cudaSuccess; ++i)
    e = cudaStreamCreateWithFlags(&S->qs[i], cudaStreamNonBlocking);
  const bool batching = !(flags & DRTOPK_SERVER_PLAIN);
  for (int i = 0; i < kBatchCtxs && e == cudaSuccess && batching; ++i) {
    BatchCtx& c = S->ctx[i];
    e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
    note_alloc(6);  // rows (device and pinned), control words, phases, scratch, error word
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&c.d_rows), kMaxBatchRows * sizeof(RowDesc));
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&c.h_rows), kMaxBatchRows * sizeof(RowDesc));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&c.d_ctl), 2 * sizeof(uint32_t));
    if (e == cudaSuccess)
      e = cudaMalloc(reinterpret_cast<void**>(&c.d_phase), kBatchPhases * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c.d_phase, 0, kBatchPhases * sizeof(unsigned long long));
    const size_t scr = static_cast<size_t>(S->grid) * kScratchPerCta * sizeof(uint64_t);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&c.d_scratch), scr);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&c.h_err), sizeof(uint32_t));
    if (e == cudaSuccess) *c.h_err = 0;
    S->fixed += kMaxBatchRows * sizeof(RowDesc) + 2 * sizeof(uint32_t) + scr +
                kBatchPhases * sizeof(unsigned long long);
  }
  if (e != cudaSuccess || S->fixed >= S->budget) {
    const drtopk_status st = e != cudaSuccess
                                 ? (e == cudaErrorMemoryAllocation ? DRTOPK_ERR_NOMEM : DRTOPK_ERR_CUDA)
                                 : DRTOPK_ERR_BUDGET;
    cudaGetLastError();
    S->release();
    delete S;
    cudaSetDevice(prev_dev);
    return st;
  }
  S->worker = std::thread([S] { S->run(); });
  *out = S;
  return cudaSetDevice(prev_dev) == cudaSuccess ? DRTOPK_OK : DRTOPK_ERR_CUDA;
}

drtopk_status drtopk_server_create(size_t hbm_budget_bytes, int device, drtopk_server** out) {
  return drtopk_server_create_ex(hbm_budget_bytes, device, 0, 0, out);
}

drtopk_status drtopk_server_submit(drtopk_server* S, const void* keys, drtopk_dtype dtype,
                                   int64_t n, int64_t k, void* out_keys, int32_t* out_idx,
                                   uint64_t* ticket) {
  if (!S || !keys || !out_keys || !out_idx || !ticket) return DRTOPK_ERR_INVALID;
  if ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(out_keys) |
       reinterpret_cast<uintptr_t>(out_idx)) & 3u)
    return DRTOPK_ERR_INVALID;
  size_t bytes = 0;
  int batched = 0;
  const drtopk_status st =
      drtopk_server_footprint(dtype, n, k, S->flags, S->max_batch_n, &bytes, &batched);
  if (st != DRTOPK_OK) return st;
  if (bytes > S->budget - S->fixed) return DRTOPK_ERR_BUDGET;
  Req r;
  r.keys = keys;
  r.dtype = dtype;
  r.n = n;
  r.k = k;
  r.out_keys = out_keys;
  r.out_idx = out_idx;
  r.bytes = bytes;
  r.batched = batched != 0;
  r.state = kQueued;
  r.status = DRTOPK_PENDING;
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return DRTOPK_ERR_INVALID;
    const uint64_t t = S->next_ticket++;
    S->reqs.emplace(t, r);
    S->queued.push_back(t);
    ++S->stats.submitted;
    *ticket = t;
  }
  S->cv_work.notify_one();
  return DRTOPK_OK;
}

drtopk_status drtopk_server_poll_ex(drtopk_server* S, uint64_t ticket, double* latency_us) {
  if (!S) return DRTOPK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return DRTOPK_ERR_INVALID;
  const Req& r = it->second;
  if (r.state != kDone) return DRTOPK_PENDING;
  const drtopk_status st = r.status;
  if (latency_us)
    *latency_us = std::chrono::duration<double, std::micro>(r.t_done - r.t_submit).count();
  S->reqs.erase(it);
  return st;
}

drtopk_status drtopk_server_poll(drtopk_server* S, uint64_t ticket) {
  return drtopk_server_poll_ex(S, ticket, nullptr);
}

drtopk_status drtopk_server_wait(drtopk_server* S, uint64_t ticket, double* latency_us) {
  if (!S) return DRTOPK_ERR_INVALID;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
      auto it = S->reqs.find(ticket);
      if (it == S->reqs.end()) return DRTOPK_ERR_INVALID;
      if (it->second.state == kDone) break;
      S->cv_done.wait_for(lk, std::chrono::milliseconds(10));
    }
  }
  return drtopk_server_poll_ex(S, ticket, latency_us);
}

drtopk_status drtopk_server_get_stats(drtopk_server* S, drtopk_server_stats* out) {
  if (!S || !out) return DRTOPK_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->stats;
  out->in_use_bytes = S->in_use + S->fixed;
  out->fixed_bytes = S->fixed;
  return DRTOPK_OK;
}

drtopk_status drtopk_server_destroy(drtopk_server* S) {
  if (!S) return DRTOPK_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  int prev_dev = 0;
  const bool restore = cudaGetDevice(&prev_dev) == cudaSuccess;
  cudaSetDevice(S->device);
  S->release();
  delete S;
  if (restore) cudaSetDevice(prev_dev);
  return DRTOPK_OK;
}

}  // extern "C"
