// C ABI of the drtopk library: argument checks, parameter choice (Rule 4),
// workspace, stage orchestration on one stream, statistics and profiling.
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "launch.h"

namespace drtopk {

static std::atomic<uint64_t> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(static_cast<uint64_t>(n)); }
static std::atomic<uint64_t> g_allocs{0};
void note_alloc(int n) { g_allocs.fetch_add(static_cast<uint64_t>(n)); }

namespace {

// ------------------------------------------------------------- planning ---
int alpha_rule4(int64_t n, int64_t k) {
  // Rule 4 / Eq. 9 with const = 3, rounded down (Sec. 4.2)
  const double a = 0.5 * (std::log2(static_cast<double>(n)) - std::log2(static_cast<double>(k)) + 3.0);
  return static_cast<int>(std::floor(a));
}

constexpr size_t kAlign = 256;
size_t al(size_t b) { return (b + kAlign - 1) & ~(kAlign - 1); }

// Delegates the filter may queue for position resolution: those > tau,
// fewer than k when tau is the k-th delegate (or all beta S of them when
// there are fewer than k); every delegate under the shortcut ablation.
int64_t rq_capacity(const Plan& p, int64_t k) {
  const int64_t d = p.S * p.beta;
  if (p.ablate & kAblateSkipLastDigit) return d;
  return std::max<int64_t>(1, std::min(d, k));
}

}  // namespace

bool make_plan(int64_t n, int64_t k, int alpha, int beta, Plan* p, int ablate) {
  if (beta <= 0) beta = 2;  // Sec. 3.3: beta = 2 performs best
  if (beta < 1 || beta > kMaxBeta) return false;
  if (alpha <= 0) {
    int a = alpha_rule4(n, k);
    a = std::max(kMinAlpha, std::min(kMaxAlpha, a));
    // enough delegates for a useful threshold: beta * S >= 2k
    while (a > kMinAlpha && static_cast<int64_t>(beta) * ((n + (int64_t(1) << a) - 1) >> a) < 2 * k) --a;
    alpha = a;
  }
  if (alpha < kMinAlpha || alpha > kMaxAlpha || (int64_t(1) << alpha) < beta) return false;
  p->alpha = alpha;
  p->beta = beta;
  p->S = (n + (int64_t(1) << alpha) - 1) >> alpha;
  p->fuse_hist = static_cast<int64_t>(beta) * p->S >= k;
  if (p->fuse_hist) {
    const int64_t bound = ((k - 1) / beta) * (int64_t(1) << alpha) + k;
    p->g_cap = std::min<int64_t>(n, bound);
  } else {
    p->g_cap = n;
  }
  // the candidate bound assumes both Rule 2's filtering and tau = the exact
  // k-th delegate: without either, candidates are bounded by n only
  if (ablate & (kAblateNoFilter | kAblateSkipLastDigit)) p->g_cap = n;
  if (p->g_cap < 1) p->g_cap = 1;
  p->ablate = ablate;
  return true;
}

void plan_spec(Plan* p, int64_t n) {
  p->rec_cap = 0;
  if (p->ablate == 0 && p->fuse_hist && p->alpha >= 5 && p->alpha <= 10 && n >= (int64_t(1) << 26))
    p->rec_cap = std::max<int64_t>(1024, p->S / 4);
}

Layout layout(const Plan& p, int64_t k, bool need_topk, bool external_dkeys) {
  Layout L;
  const size_t D = static_cast<size_t>(p.S) * p.beta;
  size_t o = 0;
  L.ctl = o; o += al(sizeof(Ctl));
  L.dkeys = o; if (!external_dkeys) o += al(D * 4);
  L.dsegs = o; o += al(D * 2);
  L.ds = o; if (p.fuse_hist) o += al(D * 4);
  L.scanq = o; o += al(static_cast<size_t>(p.S) * 4);
  L.rq = o; o += al(static_cast<size_t>(rq_capacity(p, k)) * 4);
  L.g = o; o += al(static_cast<size_t>(p.g_cap) * 8);
  L.sv = o; o += al(static_cast<size_t>(p.g_cap) * 8);
  L.w = o; if (need_topk) o += al(static_cast<size_t>(k) * 8);
  L.w2 = o; if (need_topk && k > 4096) o += al(static_cast<size_t>(k) * 8);
  L.tstat = o; if (need_topk) o += al(tie_bytes(p.S, p.alpha));
  L.sstat = o; if (need_topk) o += al(sort_status_words(k) * 8);
  const size_t rc = static_cast<size_t>(p.rec_cap);
  L.rk = o; o += al(rc * p.beta * 4);
  L.rs = o; o += al(rc * p.beta * 2);
  L.rsub = o; o += al(rc * 4);
  L.total = o;
  return L;
}

void bind_work(Work& w, char* ws, const Layout& L, const Plan& P, int64_t n, int64_t k,
               int dtype) {
  w.ctl = reinterpret_cast<Ctl*>(ws + L.ctl);
  w.dkeys = reinterpret_cast<uint32_t*>(ws + L.dkeys);
  w.dsegs = reinterpret_cast<uint16_t*>(ws + L.dsegs);
  w.ds = reinterpret_cast<uint32_t*>(ws + L.ds);
  w.scanq = reinterpret_cast<uint32_t*>(ws + L.scanq);
  w.rq = reinterpret_cast<uint32_t*>(ws + L.rq);
  w.rq_cap = rq_capacity(P, k);
  w.g = reinterpret_cast<uint64_t*>(ws + L.g);
  w.sv = reinterpret_cast<uint64_t*>(ws + L.sv);
  w.w = reinterpret_cast<uint64_t*>(ws + L.w);
  w.w2 = reinterpret_cast<uint64_t*>(ws + L.w2);
  w.tstat = reinterpret_cast<uint64_t*>(ws + L.tstat);
  w.sort_status = reinterpret_cast<uint64_t*>(ws + L.sstat);
  w.n = n;
  w.S = P.S;
  w.g_cap = P.g_cap;
  w.k = k;
  w.alpha = P.alpha;
  w.beta = P.beta;
  w.dtype = dtype;
  w.ablate = P.ablate;
  w.err_out = nullptr;
  w.rec_cap = P.rec_cap;
  w.rec_keys = P.rec_cap ? reinterpret_cast<uint32_t*>(ws + L.rk) : nullptr;
  w.rec_segs = P.rec_cap ? reinterpret_cast<uint16_t*>(ws + L.rs) : nullptr;
  w.rec_sub = P.rec_cap ? reinterpret_cast<uint32_t*>(ws + L.rsub) : nullptr;
}

drtopk_status error_status(uint32_t flags) {
  if (flags == 0) return DRTOPK_OK;
  return (flags & kErrTimeout) ? DRTOPK_ERR_TIMEOUT : DRTOPK_ERR_INTERNAL;
}

namespace {

// --------------------------------------------------------------- device ---
// Per device: SM count, the library's own stream-ordered memory pool (freed
// workspace stays cached in it; the device's default pool is left as the
// process configured it) and the report word of device-side errors: one
// host-mapped word that the last kernel of every query ORs its error flags
// into, read and cleared by the next call on the device or by
// drtopk_sync_status.
constexpr int kHostChunks = 64;  // copy pieces of one drtopk_topk_host call at most
struct DevInfo {
  int sms = 0;
  cudaMemPool_t pool = nullptr;
  uint32_t* err_host = nullptr;  // mapped pinned host word
  uint32_t* err_dev = nullptr;   // its device address
  // drtopk_topk_host: the copy stream and one event per piece (plus one
  // ordering the copies after the caller's earlier work); created on first
  // use, guarded by the device's staging lock
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_ev[kHostChunks + 1] = {};
};
std::mutex g_dev_mu;
DevInfo g_dev[64];

drtopk_status dev_info(int* sms, DevInfo** out = nullptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DRTOPK_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_dev_mu);
  DevInfo& d = g_dev[dev];
  if (d.sms == 0) {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return DRTOPK_ERR_CUDA;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return DRTOPK_ERR_CUDA;
    note_alloc(2);  // the pool and the report word below
    uint64_t thr = UINT64_MAX;  // keep freed workspace cached in the pool
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr) != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return DRTOPK_ERR_CUDA;
    }
    uint32_t* h = nullptr;
    uint32_t* dp = nullptr;
    if (cudaHostAlloc(reinterpret_cast<void**>(&h), sizeof(uint32_t),
                      cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return DRTOPK_ERR_CUDA;
    }
    *h = 0;
    if (cudaHostGetDevicePointer(reinterpret_cast<void**>(&dp), h, 0) != cudaSuccess) {
      cudaFreeHost(h);
      cudaMemPoolDestroy(pool);
      return DRTOPK_ERR_CUDA;
    }
    d.pool = pool;
    d.err_host = h;
    d.err_dev = dp;
    d.sms = nsm;
  }
  *sms = d.sms;
  if (out) *out = &d;
  return DRTOPK_OK;
}

// Takes (reads and clears) the error flags reported on the device so far.
uint32_t take_errors(DevInfo* d) {
  if (!d || !d->err_host) return 0;
  return __atomic_exchange_n(d->err_host, 0u, __ATOMIC_ACQ_REL);
}

// ------------------------------------------------------------ profiling ---
struct StageRec {
  int stage;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<StageRec> g_prof;

bool profiling_on() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return g_prof_on;
}

// Records a pair of events around each stage on the launching stream.
struct StageTimer {
  cudaStream_t s;
  bool on;
  cudaEvent_t a = nullptr;
  int stage = -1;
  StageTimer(cudaStream_t st, bool enabled) : s(st), on(enabled) {}
  void begin(int st) {
    if (!on) return;
    stage = st;
    cudaEventCreate(&a);
    cudaEventRecord(a, s);
  }
  void end() {
    if (!on || stage < 0) return;
    cudaEvent_t b;
    cudaEventCreate(&b);
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back(StageRec{stage, a, b});
    stage = -1;
  }
};

drtopk_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return DRTOPK_OK;
  if (e == cudaErrorMemoryAllocation) return DRTOPK_ERR_NOMEM;
  return DRTOPK_ERR_CUDA;
}

// dtype: a drtopk_dtype, optionally with kSmallest (the smallest-k criterion)
drtopk_status check_args(const void* keys, int dtype, int64_t n, int64_t k) {
  const int b = dtype & ~kSmallest;
  if (b != DRTOPK_U32 && b != DRTOPK_I32 && b != DRTOPK_F32) return DRTOPK_ERR_DTYPE;
  if (n < 1 || n > 0x7FFFFFFFLL) return DRTOPK_ERR_INVALID;
  if (k < 1 || k > n) return DRTOPK_ERR_K;
  if (!keys || (reinterpret_cast<uintptr_t>(keys) & 3u)) return DRTOPK_ERR_INVALID;
  return DRTOPK_OK;
}

#define DRTOPK_CU(call)                          \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) {                     \
      st = cuda_status(e_);                      \
      goto done;                                 \
    }                                            \
  } while (0)

// The launches of one query after its delegate pass, in order, on stream s.
cudaError_t enqueue_after_delegates(const Work& w, const Plan& P, const void* keys, bool topk,
                                    void* out_keys, int32_t* out_idx, void* out_kth, int sms,
                                    cudaStream_t s, StageTimer& tm) {
  cudaError_t e = cudaSuccess;
  if (P.fuse_hist) {
    tm.begin(1);
    e = launch_threshold(w, sms, s);
    tm.end();
    if (e != cudaSuccess) return e;
  }
  tm.begin(2);
  e = launch_filter(w, keys, !topk, sms, s);
  tm.end();
  if (e != cudaSuccess) return e;
  if (topk) {
    tm.begin(3);
    e = launch_ties(w, keys, sms, s);
    tm.end();
    if (e != cudaSuccess) return e;
  }
  tm.begin(4);
  e = launch_gselect(w, !topk, sms, s);
  if (e == cudaSuccess && !topk) e = launch_write_kth(w, out_kth, s);
  tm.end();
  if (e != cudaSuccess) return e;
  if (topk) {
    tm.begin(5);
    e = launch_sort_output(w, out_keys, out_idx, out_kth, sms, s);
    tm.end();
  }
  return e;
}

// Every launch of one query, in order, on stream s (no allocation, no sync).
cudaError_t enqueue_query(const Work& w, const Plan& P, const void* keys, bool topk,
                          void* out_keys, int32_t* out_idx, void* out_kth, int sms,
                          cudaStream_t s, StageTimer& tm) {
  cudaError_t e = cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), s);
  if (e != cudaSuccess) return e;
  tm.begin(0);
  e = spec_eligible(w, keys) ? launch_delegates_spec(w, keys, sms, s)
                             : launch_delegates(w, keys, P.fuse_hist, sms, s);
  tm.end();
  if (e != cudaSuccess) return e;
  return enqueue_after_delegates(w, P, keys, topk, out_keys, out_idx, out_kth, sms, s, tm);
}

// ---------------------------------------------------------- graph cache ---
// Repeated calls with identical arguments on the same stream replay a CUDA
// graph of the whole query (one graph launch instead of ~30 kernel launches).
// A graph is built on the second call with a key (the last kSeenKeys keys
// are remembered), so one-off calls never pay for a capture. Each entry
// owns its workspace; entries are evicted least-recently-used past
// kGraphMaxEntries or DRTOPK_GRAPH_CACHE_BYTES (default 16 GiB) of
// workspace. Calls on a stream that is being captured launch kernel by
// kernel into that capture. DRTOPK_GRAPH_CACHE=0 disables the cache.
struct GraphKey {
  const void* keys;
  void* out_keys;
  void* out_idx;
  void* out_kth;
  int64_t n, k;
  int dtype, alpha, beta, dev;
  cudaStream_t s;
  bool operator==(const GraphKey& o) const {
    return keys == o.keys && out_keys == o.out_keys && out_idx == o.out_idx &&
           out_kth == o.out_kth && n == o.n && k == o.k && dtype == o.dtype &&
           alpha == o.alpha && beta == o.beta && dev == o.dev && s == o.s;
  }
};

struct GraphEntry {
  GraphKey key;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  char* ws = nullptr;
  size_t bytes = 0;
  cudaEvent_t done = nullptr;
  uint64_t tick = 0;
  uint64_t nlaunch = 0;
};

// Device staging of drtopk_topk_host, one buffer per device.
constexpr int kMaxDevices = 64;
struct HostStage {
  std::mutex mu;
  char* d = nullptr;
  size_t cap = 0;
};
HostStage g_hstage[kMaxDevices];

constexpr size_t kGraphMaxEntries = 64;
constexpr size_t kSeenKeys = 256;
std::mutex g_gmu;
std::vector<GraphEntry> g_graphs;
GraphKey g_seen[kSeenKeys];
size_t g_seen_next = 0;
uint64_t g_gtick = 0;
size_t g_gbytes = 0;
cudaStream_t g_capture_stream[64];

bool graph_cache_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("DRTOPK_GRAPH_CACHE");
    return !(v && v[0] == '0');
  }();
  return on;
}

size_t graph_cache_budget() {
  static const size_t b = [] {
    const char* v = std::getenv("DRTOPK_GRAPH_CACHE_BYTES");
    return v ? static_cast<size_t>(std::strtoull(v, nullptr, 10)) : (size_t(16) << 30);
  }();
  return b;
}

void destroy_entry(GraphEntry& e) {
  if (e.done) cudaEventSynchronize(e.done);
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.graph) cudaGraphDestroy(e.graph);
  if (e.ws) cudaFree(e.ws);
  if (e.done) cudaEventDestroy(e.done);
  g_gbytes -= e.bytes;
}

// Builds an entry (capture + instantiate). Caller holds g_gmu.
cudaError_t build_entry(GraphEntry& ent, const Plan& P, const Layout& L, const void* keys,
                        int dtype, int64_t n, int64_t k, bool topk, void* out_keys,
                        int32_t* out_idx, void* out_kth, int sms, int dev, uint32_t* err_out) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&ent.ws), L.total);
  note_alloc();
  if (e != cudaSuccess) return e;
  ent.bytes = L.total;
  g_gbytes += L.total;
  Work w;
  bind_work(w, ent.ws, L, P, n, k, dtype);
  w.err_out = err_out;
  if (!g_capture_stream[dev]) {
    e = cudaStreamCreateWithFlags(&g_capture_stream[dev], cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  cudaStream_t cs = g_capture_stream[dev];
  StageTimer tm(cs, false);
  const uint64_t before = drtopk_launch_count();
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  const cudaError_t ee = enqueue_query(w, P, keys, topk, out_keys, out_idx, out_kth, sms, cs, tm);
  e = cudaStreamEndCapture(cs, &ent.graph);
  ent.nlaunch = drtopk_launch_count() - before;
  g_launches.fetch_sub(ent.nlaunch);  // counted again at every replay
  if (ee != cudaSuccess) return ee;
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&ent.exec, ent.graph, 0);
  if (e != cudaSuccess) return e;
  return cudaEventCreateWithFlags(&ent.done, cudaEventDisableTiming);
}

// Replays (building on a miss) the graph of this query. Returns false when
// the graph path is not usable; the caller then runs the direct path.
bool run_graph(const Plan& P, const void* keys, int dtype, int64_t n, int64_t k, bool topk,
               void* out_keys, int32_t* out_idx, void* out_kth, int sms, uint32_t* err_out,
               cudaStream_t s, drtopk_status* st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (cap != cudaStreamCaptureStatusNone) return false;
  GraphKey key{keys, out_keys, out_idx, out_kth, n, k, dtype, P.alpha, P.beta, dev, s};
  std::lock_guard<std::mutex> lk(g_gmu);
  GraphEntry* ent = nullptr;
  for (auto& e : g_graphs)
    if (e.key == key) ent = &e;
  if (!ent) {
    // admit a key on its second call
    bool seen = false;
    for (size_t i = 0; i < kSeenKeys && !seen; ++i) seen = g_seen[i] == key;
    if (!seen) {
      g_seen[g_seen_next] = key;
      g_seen_next = (g_seen_next + 1) % kSeenKeys;
      return false;
    }
    const Layout L = layout(P, k, topk, false);
    if (L.total > graph_cache_budget()) return false;
    while (!g_graphs.empty() &&
           (g_graphs.size() >= kGraphMaxEntries || g_gbytes + L.total > graph_cache_budget())) {
      size_t v = 0;
      for (size_t i = 1; i < g_graphs.size(); ++i)
        if (g_graphs[i].tick < g_graphs[v].tick) v = i;
      destroy_entry(g_graphs[v]);
      g_graphs.erase(g_graphs.begin() + v);
    }
    GraphEntry fresh;
    fresh.key = key;
    if (build_entry(fresh, P, L, keys, dtype, n, k, topk, out_keys, out_idx, out_kth, sms, dev,
                    err_out) != cudaSuccess) {
      cudaGetLastError();
      destroy_entry(fresh);
      return false;
    }
    g_graphs.push_back(fresh);
    ent = &g_graphs.back();
  }
  ent->tick = ++g_gtick;
  cudaError_t e = cudaGraphLaunch(ent->exec, s);
  if (e == cudaSuccess) e = cudaEventRecord(ent->done, s);
  if (e == cudaSuccess) note_launch(static_cast<int>(ent->nlaunch));
  *st = cuda_status(e);
  return true;
}

// Where a query's device error flags go: the device's report word (read by
// the next call on the device and by drtopk_sync_status), a caller's word,
// or nowhere (the call reads them itself).
enum class Report { kDevice, kCaller, kNone };

drtopk_status run_query(const void* keys, int dtype, int64_t n, int64_t k, int alpha, int beta,
                        void* out_keys, int32_t* out_idx, void* out_kth, drtopk_stats* stats,
                        cudaStream_t s, bool allow_graph, int ablate = 0,
                        Report report = Report::kDevice, uint32_t* caller_err = nullptr) {
  drtopk_status st = check_args(keys, dtype, n, k);
  if (st != DRTOPK_OK) return st;
  const bool topk = out_keys != nullptr || out_idx != nullptr;
  if (!topk && !out_kth) return DRTOPK_ERR_INVALID;
  if (alpha > 0 && (alpha < kMinAlpha || alpha > kMaxAlpha)) return DRTOPK_ERR_INVALID;
  if (beta > kMaxBeta) return DRTOPK_ERR_INVALID;
  Plan P;
  if (!make_plan(n, k, alpha, beta, &P, ablate)) return DRTOPK_ERR_INVALID;
  plan_spec(&P, n);
  int sms = 0;
  DevInfo* dv = nullptr;
  st = dev_info(&sms, &dv);
  if (st != DRTOPK_OK) return st;
  if (stats) report = Report::kNone;  // read back below, with the statistics
  uint32_t* err_out = nullptr;
  if (report == Report::kDevice) {
    // an earlier asynchronous call on this device reported a device-side
    // error: return it now (this call does nothing)
    if (const uint32_t prev = take_errors(dv)) return error_status(prev);
    err_out = dv->err_dev;
  } else if (report == Report::kCaller) {
    err_out = caller_err;
  }
  const bool prof = profiling_on();
  if (ablate) allow_graph = false;  // the graph cache keys on the method as stated

  // profiled calls run the direct path: its stage events sit between launches
  if (allow_graph && !stats && !prof && graph_cache_enabled() && report == Report::kDevice &&
      run_graph(P, keys, dtype, n, k, topk, out_keys, out_idx, out_kth, sms, err_out, s, &st))
    return st;

  const Layout L = layout(P, k, topk, false);
  char* ws = nullptr;
  StageTimer tm(s, prof);
  Work w;
  {
    // the library's own pool; under a caller's stream capture the workspace
    // becomes a graph allocation node instead
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_status(e);
    e = (cap == cudaStreamCaptureStatusNone)
            ? cudaMallocFromPoolAsync(reinterpret_cast<void**>(&ws), L.total, dv->pool, s)
            : cudaMallocAsync(reinterpret_cast<void**>(&ws), L.total, s);
    note_alloc();
    if (e != cudaSuccess) return cuda_status(e);
  }
  bind_work(w, ws, L, P, n, k, dtype);
  w.err_out = err_out;
  DRTOPK_CU(enqueue_query(w, P, keys, topk, out_keys, out_idx, out_kth, sms, s, tm));
  if (stats) {
    Ctl c;
    DRTOPK_CU(cudaMemcpyAsync(&c, w.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
    DRTOPK_CU(cudaStreamSynchronize(s));
    std::memset(stats, 0, sizeof(*stats));
    stats->alpha = P.alpha;
    stats->beta = P.beta;
    stats->subranges = P.S;
    stats->tau = c.tau;
    stats->kth_mapped = c.kth_mapped;
    stats->greater = c.g_total;
    stats->ties_needed = (c.mode == kModeTies) ? c.need : 0;
    stats->scanned = c.scanned;
    stats->tie_scanned = c.tie_scanned;
    stats->survivors = c.stage_count[2];
    stats->emitted = c.w_count;
    stats->error = c.error;
    stats->delegate_path = (c.spec_used ? 1u : 0u) | (c.full_written ? 2u : 0u);
    st = error_status(c.error);
  }
done:
  {
    cudaError_t e = cudaFreeAsync(ws, s);
    if (st == DRTOPK_OK && e != cudaSuccess) st = cuda_status(e);
  }
  return st;
}

}  // namespace

drtopk_status topk_kernel_by_kernel(const void* keys, int dtype, int64_t n, int64_t k,
                                    void* out_keys, int32_t* out_idx, uint32_t* err_out,
                                    cudaStream_t s) {
  return run_query(keys, dtype, n, k, 0, 0, out_keys, out_idx, nullptr, nullptr, s, false, 0,
                   Report::kCaller, err_out);
}

cudaError_t enqueue_query_plain(const Work& w, const Plan& P, const void* keys, bool topk,
                                void* out_keys, int32_t* out_idx, void* out_kth, int sms,
                                cudaStream_t s) {
  StageTimer tm(s, false);
  return enqueue_query(w, P, keys, topk, out_keys, out_idx, out_kth, sms, s, tm);
}

}  // namespace drtopk

using namespace drtopk;

extern "C" {

const char* drtopk_status_str(drtopk_status s) {
  switch (s) {
    case DRTOPK_OK: return "DRTOPK_OK";
    case DRTOPK_ERR_INVALID: return "DRTOPK_ERR_INVALID";
    case DRTOPK_ERR_K: return "DRTOPK_ERR_K";
    case DRTOPK_ERR_DTYPE: return "DRTOPK_ERR_DTYPE";
    case DRTOPK_ERR_NOMEM: return "DRTOPK_ERR_NOMEM";
    case DRTOPK_ERR_CUDA: return "DRTOPK_ERR_CUDA";
    case DRTOPK_ERR_BUDGET: return "DRTOPK_ERR_BUDGET";
    case DRTOPK_ERR_TIMEOUT: return "DRTOPK_ERR_TIMEOUT";
    case DRTOPK_PENDING: return "DRTOPK_PENDING";
    case DRTOPK_ERR_INTERNAL: return "DRTOPK_ERR_INTERNAL";
  }
  return "DRTOPK_UNKNOWN_STATUS";
}

drtopk_status drtopk_plan(int64_t n, int64_t k, int* alpha, int* beta, size_t* workspace_bytes) {
  if (n < 1 || n > 0x7FFFFFFFLL) return DRTOPK_ERR_INVALID;
  if (k < 1 || k > n) return DRTOPK_ERR_K;
  Plan P;
  if (!make_plan(n, k, 0, 0, &P)) return DRTOPK_ERR_INVALID;
  plan_spec(&P, n);
  if (alpha) *alpha = P.alpha;
  if (beta) *beta = P.beta;
  if (workspace_bytes) *workspace_bytes = layout(P, k, true, false).total;
  return DRTOPK_OK;
}

drtopk_status drtopk_kth(const void* keys, drtopk_dtype dtype, int64_t n, int64_t k,
                         void* out_kth, void* stream) {
  if (!out_kth) return DRTOPK_ERR_INVALID;
  return run_query(keys, dtype, n, k, 0, 0, nullptr, nullptr, out_kth, nullptr,
                   static_cast<cudaStream_t>(stream), true);
}

drtopk_status drtopk_topk(const void* keys, drtopk_dtype dtype, int64_t n, int64_t k,
                          void* out_keys, int32_t* out_idx, void* stream) {
  if (!out_keys || !out_idx) return DRTOPK_ERR_INVALID;
  return run_query(keys, dtype, n, k, 0, 0, out_keys, out_idx, nullptr, nullptr,
                   static_cast<cudaStream_t>(stream), true);
}

drtopk_status drtopk_topk_ex(const void* keys, drtopk_dtype dtype, int64_t n, int64_t k,
                             int alpha, int beta, void* out_keys, int32_t* out_idx,
                             void* out_kth, drtopk_stats* stats, void* stream) {
  if ((out_keys == nullptr) != (out_idx == nullptr)) return DRTOPK_ERR_INVALID;
  if (alpha < 0 || beta < 0) return DRTOPK_ERR_INVALID;
  return run_query(keys, dtype, n, k, alpha, beta, out_keys, out_idx, out_kth, stats,
                   static_cast<cudaStream_t>(stream), true);
}

drtopk_status drtopk_select(const void* keys, drtopk_dtype dtype, int64_t n, int64_t k,
                            int flags, void* out_keys, int32_t* out_idx, void* out_kth,
                            void* stream) {
  if ((out_keys == nullptr) != (out_idx == nullptr)) return DRTOPK_ERR_INVALID;
  if (!out_keys && !out_kth) return DRTOPK_ERR_INVALID;
  if (flags & ~DRTOPK_SMALLEST) return DRTOPK_ERR_INVALID;
  if (dtype != DRTOPK_U32 && dtype != DRTOPK_I32 && dtype != DRTOPK_F32) return DRTOPK_ERR_DTYPE;
  const int dt = static_cast<int>(dtype) | ((flags & DRTOPK_SMALLEST) ? kSmallest : 0);
  return run_query(keys, dt, n, k, 0, 0, out_keys, out_idx, out_kth, nullptr,
                   static_cast<cudaStream_t>(stream), true);
}

drtopk_status drtopk_topk_merge(const void* keys, const int32_t* idx, drtopk_dtype dtype,
                                const int64_t* part_off, const int64_t* part_base,
                                int32_t parts, int64_t k, int flags, void* out_keys,
                                int64_t* out_gidx, void* stream) {
  if (!keys || !idx || !part_off || !part_base || !out_keys || !out_gidx)
    return DRTOPK_ERR_INVALID;
  if (parts < 1 || parts > kMaxMergeParts || (flags & ~DRTOPK_SMALLEST)) return DRTOPK_ERR_INVALID;
  if (dtype != DRTOPK_U32 && dtype != DRTOPK_I32 && dtype != DRTOPK_F32) return DRTOPK_ERR_DTYPE;
  if (part_off[0] < 0) return DRTOPK_ERR_INVALID;
  MergeParts mp;
  mp.parts = parts;
  for (int p = 0; p < parts; ++p) {
    if (part_off[p + 1] < part_off[p] || part_base[p] < 0) return DRTOPK_ERR_INVALID;
    mp.off[p] = part_off[p] - part_off[0];
    mp.base[p] = part_base[p];
  }
  const int64_t m = part_off[parts] - part_off[0];
  if (m < 1 || m > 0x7FFFFFFFLL) return DRTOPK_ERR_INVALID;
  if (k < 1 || k > m) return DRTOPK_ERR_K;
  const int dt = static_cast<int>(dtype) | ((flags & DRTOPK_SMALLEST) ? kSmallest : 0);
  const char* kbase = static_cast<const char*>(keys) + part_off[0] * 4;
  const int32_t* ibase = idx + part_off[0];
  int sms = 0;
  DevInfo* dv = nullptr;
  drtopk_status st = dev_info(&sms, &dv);
  if (st != DRTOPK_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // positions of the winners in the concatenated lists (stream-ordered)
  int32_t* pos = nullptr;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return cuda_status(e);
  const size_t pb = static_cast<size_t>(k) * 4;
  e = (cap == cudaStreamCaptureStatusNone)
          ? cudaMallocFromPoolAsync(reinterpret_cast<void**>(&pos), pb, dv->pool, s)
          : cudaMallocAsync(reinterpret_cast<void**>(&pos), pb, s);
  note_alloc();
  if (e != cudaSuccess) return cuda_status(e);
  // The lists are sorted as drtopk_select returns them and concatenated in
  // increasing order of their global index ranges, so among equal keys the
  // position order is the global index order: the single-query path over
  // the concatenation (ties to the smallest position) is the exact merge.
  st = run_query(kbase, dt, m, k, 0, 0, out_keys, pos, nullptr, nullptr, s, true);
  if (st == DRTOPK_OK) st = cuda_status(launch_merge_gather(mp, pos, ibase, k, out_gidx, sms, s));
  const cudaError_t e2 = cudaFreeAsync(pos, s);
  if (st == DRTOPK_OK && e2 != cudaSuccess) st = cuda_status(e2);
  return st;
}

drtopk_status drtopk_topk_ablate(const void* keys, drtopk_dtype dtype, int64_t n, int64_t k,
                                 int alpha, int beta, int flags, void* out_keys, int32_t* out_idx,
                                 drtopk_stats* stats, void* stream) {
  if (!out_keys || !out_idx) return DRTOPK_ERR_INVALID;
  if (alpha < 0 || beta < 0 || (flags & ~(DRTOPK_ABLATE_NO_FILTER | DRTOPK_ABLATE_SKIP_LAST_DIGIT)))
    return DRTOPK_ERR_INVALID;
  return run_query(keys, dtype, n, k, alpha, beta, out_keys, out_idx, nullptr, stats,
                   static_cast<cudaStream_t>(stream), false, flags);
}

drtopk_status drtopk_delegates(const void* keys, drtopk_dtype dtype, int64_t n, int alpha,
                               int beta, uint32_t* d_keys, int32_t* d_idx, void* stream) {
  drtopk_status st = check_args(keys, dtype, n, 1);
  if (st != DRTOPK_OK) return st;
  if (!d_keys || !d_idx) return DRTOPK_ERR_INVALID;
  if (alpha < kMinAlpha || alpha > kMaxAlpha || beta < 1 || beta > kMaxBeta ||
      (1 << alpha) < beta)
    return DRTOPK_ERR_INVALID;
  Plan P;
  if (!make_plan(n, 1, alpha, beta, &P)) return DRTOPK_ERR_INVALID;
  int sms = 0;
  DevInfo* dv = nullptr;
  st = dev_info(&sms, &dv);
  if (st != DRTOPK_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t bytes = al(sizeof(Ctl)) + al(static_cast<size_t>(P.S) * beta * 2);
  char* ws = nullptr;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return cuda_status(e);
  e = (cap == cudaStreamCaptureStatusNone)
          ? cudaMallocFromPoolAsync(reinterpret_cast<void**>(&ws), bytes, dv->pool, s)
          : cudaMallocAsync(reinterpret_cast<void**>(&ws), bytes, s);
  note_alloc();
  if (e != cudaSuccess) return cuda_status(e);
  Work w;
  std::memset(&w, 0, sizeof(w));
  w.ctl = reinterpret_cast<Ctl*>(ws);
  w.dkeys = d_keys;
  w.dsegs = reinterpret_cast<uint16_t*>(ws + al(sizeof(Ctl)));
  w.n = n;
  w.S = P.S;
  w.k = 1;
  w.alpha = alpha;
  w.beta = beta;
  w.dtype = dtype;
  e = cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), s);
  if (e == cudaSuccess) {
    e = launch_delegates(w, keys, false, sms, s);
  }
  if (e == cudaSuccess) e = launch_resolve_delegates(w, keys, d_idx, s);
  cudaError_t e2 = cudaFreeAsync(ws, s);
  if (e == cudaSuccess) e = e2;
  return cuda_status(e);
}

drtopk_status drtopk_topk_host(const void* keys, drtopk_dtype dtype, int64_t n, int64_t k,
                               void* out_keys, int32_t* out_idx, void* stream) {
  drtopk_status st = check_args(keys, dtype, n, k);
  if (st != DRTOPK_OK) return st;
  if (!out_keys || !out_idx) return DRTOPK_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DRTOPK_ERR_CUDA;
  int sms = 0;
  DevInfo* dv = nullptr;
  st = dev_info(&sms, &dv);
  if (st != DRTOPK_OK) return st;
  if (const uint32_t prev = take_errors(dv)) return error_status(prev);
  Plan P;
  if (!make_plan(n, k, 0, 0, &P)) return DRTOPK_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t kb = al(static_cast<size_t>(n) * 4);
  const size_t ob = al(static_cast<size_t>(k) * 4);
  // the device's staging buffer, grown to the largest call and kept
  HostStage& hs = g_hstage[dev];
  std::lock_guard<std::mutex> lk(hs.mu);
  if (hs.cap < kb + 2 * ob) {
    if (hs.d) {
      cudaError_t e = cudaFree(hs.d);  // waits for the device
      hs.d = nullptr;
      hs.cap = 0;
      if (e != cudaSuccess) return cuda_status(e);
    }
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&hs.d), kb + 2 * ob);
    note_alloc();
    if (e != cudaSuccess) {
      hs.d = nullptr;
      return cuda_status(e);
    }
    hs.cap = kb + 2 * ob;
  }
  if (!dv->copy_stream) {
    if (cudaStreamCreateWithFlags(&dv->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
      return DRTOPK_ERR_CUDA;
    for (auto& ev : dv->copy_ev)
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return DRTOPK_ERR_CUDA;
  }
  char* d = hs.d;
  const char* h = static_cast<const char*>(keys);
  const Layout L = layout(P, k, true, false);
  char* ws = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&ws), L.total, dv->pool, s);
  note_alloc();
  if (e != cudaSuccess) return cuda_status(e);
  Work w;
  bind_work(w, ws, L, P, n, k, dtype);
  w.err_out = dv->err_dev;
  // The keys go over in pieces of whole subranges (about 128 MB) on the
  // copy stream; the delegate pass of piece c runs on `stream` as soon as
  // piece c has landed, while the next pieces are still in flight. The rest
  // of the query follows the last piece.
  int64_t spc = std::max<int64_t>(1, (int64_t(32) << 20) >> P.alpha);  // subranges per piece
  while ((P.S + spc - 1) / spc > kHostChunks) spc *= 2;
  const int nc = static_cast<int>((P.S + spc - 1) / spc);
  cudaStream_t cs = dv->copy_stream;
  StageTimer tm(s, false);
  e = cudaEventRecord(dv->copy_ev[kHostChunks], s);  // after the caller's earlier work
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, dv->copy_ev[kHostChunks], 0);
  for (int c = 0; c < nc && e == cudaSuccess; ++c) {
    const int64_t k0 = (int64_t(c) * spc) << P.alpha;
    const int64_t k1 = std::min<int64_t>(n, (int64_t(c + 1) * spc) << P.alpha);
    e = cudaMemcpyAsync(d + k0 * 4, h + k0 * 4, static_cast<size_t>(k1 - k0) * 4,
                        cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(dv->copy_ev[c], cs);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(w.ctl, 0, sizeof(Ctl), s);
  for (int c = 0; c < nc && e == cudaSuccess; ++c) {
    e = cudaStreamWaitEvent(s, dv->copy_ev[c], 0);
    if (e == cudaSuccess)
      e = launch_delegates_range(w, d, int64_t(c) * spc, std::min<int64_t>(P.S, int64_t(c + 1) * spc),
                                 P.fuse_hist, c == nc - 1, sms, s);
  }
  if (e == cudaSuccess)
    e = enqueue_after_delegates(w, P, d, true, d + kb, reinterpret_cast<int32_t*>(d + kb + ob),
                                nullptr, sms, s, tm);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_keys, d + kb, static_cast<size_t>(k) * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_idx, d + kb + ob, static_cast<size_t>(k) * 4, cudaMemcpyDeviceToHost, s);
  const cudaError_t e2 = cudaFreeAsync(ws, s);
  const cudaError_t e3 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = e3;
  if (e != cudaSuccess) return cuda_status(e);
  // synchronous: the query's device-side errors are reported here
  return error_status(take_errors(dv));
}

drtopk_status drtopk_profile_begin(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& r : g_prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof.clear();
  g_prof_on = true;
  return DRTOPK_OK;
}

drtopk_status drtopk_profile_end(drtopk_profile* out) {
  std::vector<StageRec> recs;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = false;
    recs.swap(g_prof);
  }
  drtopk_status st = DRTOPK_OK;
  if (out) std::memset(out, 0, sizeof(*out));
  for (auto& r : recs) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
      st = DRTOPK_ERR_CUDA;
    else if (out && r.stage >= 0 && r.stage < DRTOPK_NUM_STAGES) {
      out->ms[r.stage] += ms;
      out->launches[r.stage] += 1;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  return st;
}

uint64_t drtopk_launch_count(void) { return g_launches.load(); }

uint64_t drtopk_alloc_count(void) { return g_allocs.load(); }

drtopk_status drtopk_sync_status(void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  int sms = 0;
  DevInfo* dv = nullptr;
  if (dev_info(&sms, &dv) != DRTOPK_OK) return DRTOPK_ERR_CUDA;
  uint32_t flags = take_errors(dv);
  flags |= take_noalloc_errors();
  return error_status(flags);
}

drtopk_status drtopk_wait_selftest(uint32_t timeout_us, void* stream) {
  if (timeout_us < 1 || timeout_us > 10000000u) return DRTOPK_ERR_INVALID;
  int sms = 0;
  DevInfo* dv = nullptr;
  drtopk_status st = dev_info(&sms, &dv);
  if (st != DRTOPK_OK) return st;
  return cuda_status(launch_wait_selftest(timeout_us, dv->err_dev,
                                          static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
