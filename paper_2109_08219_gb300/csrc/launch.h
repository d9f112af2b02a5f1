// Host-side launchers of the drtopk kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace drtopk {

// Counts every kernel this library launches (drtopk_launch_count).
void note_launch(int n = 1);
// Counts every device or pinned-host allocation this library makes
// (drtopk_alloc_count); called next to each allocating CUDA call.
void note_alloc(int n = 1);

// ------------------------------------------------------ single queries ---
// Parameters of one query: alpha (Rule 4 / Eq. 9 unless forced), beta, the
// subrange count S and the capacity of the candidates above tau.
struct Plan {
  int alpha;
  int beta;
  int64_t S;
  int64_t g_cap;
  bool fuse_hist;  // beta * S >= k: tau from the delegates, else tau = 0
  int ablate = 0;
  int64_t rec_cap = 0;  // records of the speculative compaction (0: not planned)
};
bool make_plan(int64_t n, int64_t k, int alpha, int beta, Plan* p, int ablate = 0);
// Plans the speculative compaction of the delegate vector for a query that
// runs whole on the device (large arrays with alpha in [5, 10]).
void plan_spec(Plan* p, int64_t n);

// Byte offsets of a query's workspace regions (256-byte aligned) and the
// total. need_topk = false leaves out the regions only top-k uses;
// external_dkeys leaves out the delegate keys (a caller's buffer).
struct Layout {
  size_t ctl, dkeys, dsegs, ds, scanq, rq, g, sv, w, w2, tstat, sstat, rk, rs, rsub, total;
};
Layout layout(const Plan& p, int64_t k, bool need_topk, bool external_dkeys);

// Points the device views of `w` into the workspace `ws` laid out by L.
void bind_work(Work& w, char* ws, const Layout& L, const Plan& P, int64_t n, int64_t k,
               int dtype);

// Every launch of one query, in order, on stream s (no allocation, no
// host synchronization).
cudaError_t enqueue_query_plain(const Work& w, const Plan& P, const void* keys, bool topk,
                                void* out_keys, int32_t* out_idx, void* out_kth, int sms,
                                cudaStream_t s);

// Delegate pass (delegate.cu). fuse_hist: also histogram the first digit of
// the threshold select and resolve it in the last block.
cudaError_t launch_delegates(const Work& w, const void* keys, bool fuse_hist, int sms,
                             cudaStream_t s);
// The delegate pass over subranges [sub0, sub1) only (keys is the whole
// array). The fused first-digit histogram accumulates over calls; only the
// call with select_last resolves the digit (it must come last).
cudaError_t launch_delegates_range(const Work& w, const void* keys, int64_t sub0, int64_t sub1,
                                   bool fuse_hist, bool select_last, int sms, cudaStream_t s);

// Speculative compaction of the delegate vector (Ctl::spec_on): whether a
// query can use it (records planned, alpha in [5, 10], the method as stated,
// 16-byte aligned keys); the sample pass, the records pass and the fallback
// full pass when the speculation missed (the whole delegate step of such a
// query); and the fallback full pass for a query that ends in tie mode
// (cond 2; cond 1 = when Ctl::need_full).
bool spec_eligible(const Work& w, const void* keys);
cudaError_t launch_delegates_spec(const Work& w, const void* keys, int sms, cudaStream_t s);
cudaError_t launch_delegates_fallback(const Work& w, const void* keys, int cond, int sms,
                                      cudaStream_t s);

// Threshold select passes 1..3 over the delegate keys (select.cu).
cudaError_t launch_threshold(const Work& w, int sms, cudaStream_t s);

// Filter: G = {x > tau} as (key, idx) composites + first-digit histogram;
// decides the query mode (select.cu).
cudaError_t launch_filter(const Work& w, const void* keys, bool kth_only, int sms,
                          cudaStream_t s);

// Tie ranking at tau (mode kModeTies): the `need` smallest indices with
// key == tau, written after G into W (select.cu).
cudaError_t launch_ties(const Work& w, const void* keys, int sms, cudaStream_t s);

// Second select over G (mode kModeSelect). kth_only: resolve the k-th key
// only (select.cu).
cudaError_t launch_gselect(const Work& w, bool kth_only, int sms, cudaStream_t s);

// Writes the k-th key (input dtype) to out_kth (select.cu).
cudaError_t launch_write_kth(const Work& w, void* out_kth, cudaStream_t s);

// Sorts W[0..k) descending and writes out_keys (dtype) / out_idx (sort.cu).
cudaError_t launch_sort_output(const Work& w, void* out_keys, int32_t* out_idx,
                               void* out_kth, int sms, cudaStream_t s);
size_t sort_status_words(int64_t k);

// Tiles of the tie path for S subranges of 2^alpha keys, and the bytes of
// its workspace (select.cu).
int64_t tie_tiles(int64_t S, int alpha);
size_t tie_bytes(int64_t S, int alpha);

// Resolves exact delegate positions for drtopk_delegates (select.cu).
cudaError_t launch_resolve_delegates(const Work& w, const void* keys, int32_t* d_idx,
                                     cudaStream_t s);

// drtopk_topk without the graph cache: every kernel launched on `s`
// (api.cu). For one-off queries, e.g. those of the server. The query's
// device error flags are ORed into *err_out (a device-visible word).
drtopk_status topk_kernel_by_kernel(const void* keys, int dtype, int64_t n, int64_t k,
                                    void* out_keys, int32_t* out_idx, uint32_t* err_out,
                                    cudaStream_t s);

// Status of a set of device error flags (0: DRTOPK_OK).
drtopk_status error_status(uint32_t flags);

// Takes (reads and clears) the error flags drtopk_kth_noalloc reported on
// the current device (noalloc.cu); 0 when it never ran there. Synchronous.
uint32_t take_noalloc_errors();

// One CTA waits, bounded by timeout_us, on an mbarrier phase that nothing
// completes, and ORs kErrTimeout into *err_out when the wait gives up
// (select.cu).
cudaError_t launch_wait_selftest(uint32_t timeout_us, uint32_t* err_out, cudaStream_t s);

// ---------------------------------------------------------------- merge ---
// Parts of a merge (drtopk_topk_merge), passed by value: part p occupies
// positions [off[p], off[p+1]) of the concatenated lists (off[0] = 0) and
// its local index i is the global index base[p] + i.
constexpr int kMaxMergeParts = 256;
struct MergeParts {
  int64_t off[kMaxMergeParts];
  int64_t base[kMaxMergeParts];
  int parts;
};
cudaError_t launch_merge_gather(const MergeParts& mp, const int32_t* pos, const int32_t* idx,
                                int64_t k, int64_t* out_gidx, int sms, cudaStream_t s);

// ------------------------------------------------------------- batched ---
// One row of a batch. Its keys, output keys and output indices sit at the
// byte offsets keys / out_keys / out_idx from the launch's three base
// addresses (a plan over one concatenated array uses the arrays as bases;
// the server uses base 0 and absolute addresses).
struct RowDesc {
  uint64_t keys;      // first key, 4-byte aligned
  uint64_t out_keys;  // k outputs
  uint64_t out_idx;   // k int32 indices
  int32_t n;
  int32_t k;
  int32_t alpha;   // 0: direct select (no delegates)
  int32_t beta;
};

// The batched kernel (batched.cu): one persistent CTA per SM takes rows
// [0, nrows) of `rows` through *row_ctr (zeroed before the launch).
cudaError_t launch_batched(int dtype, uint64_t keys_base, uint64_t out_keys_base,
                           uint64_t out_idx_base, const RowDesc* rows, int32_t nrows,
                           uint32_t* row_ctr, uint64_t* scratch, int64_t scap, uint32_t* err,
                           unsigned long long* phase, int grid, cudaStream_t s);

// Per-row parameters of the batched path with the default policy (tuning
// table, direct select, Rule 4): alpha 0 = direct select; gneed = candidate
// capacity the row may need (scratch holds what exceeds the on-chip part).
struct BatchRowPlan {
  int alpha, beta;
  int64_t gneed;
};
BatchRowPlan batch_plan_row(int64_t n, int64_t k);
int batch_grid(int sms);                 // CTAs of one batched launch
int64_t batch_onchip_candidates();
int64_t batch_max_k();
int64_t batch_max_n();
constexpr int kBatchPhases = 10;         // cycle counters of a batched launch

}  // namespace drtopk
