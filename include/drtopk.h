/*
 * drtopk.h - C ABI of a GB300-native delegate-centric top-k library.
 *
 * The method is Dr. Top-k (Gaihre et al., "Dr. Top-k: Delegate-Centric
 * Top-k on GPUs", SC'21, arXiv 2109.08219). Problem statement (Sec. 1): given
 * a vector V of n keys, top-k returns the k largest elements of V and
 * k-selection returns the k-th largest. The library computes both exactly:
 *   1. delegate pass (Sec. 3.1 Rule 1, Sec. 3.3 Rule 3, Sec. 4.1): V is cut
 *      into subranges of 2^alpha keys; each yields its beta largest keys;
 *   2. first top-k (Sec. 3.2 Rule 2): tau = k-th largest delegate, a lower
 *      bound on the k-th largest key of V;
 *   3. concatenation with filtering (Sec. 3.2, 3.3): only subranges whose
 *      delegates reach tau are read again; only keys that can still be in
 *      the answer are kept;
 *   4. second top-k (Sec. 4.1): an exact selection over the kept keys.
 * alpha follows Rule 4 / Eq. 9 (const = 3, rounded down) and beta = 2
 * (Sec. 3.3, beta tuning) unless the caller forces them.
 *
 * Conventions for every entry point:
 *   - Keys are 32-bit: unsigned, signed or IEEE float, named by drtopk_dtype.
 *     Order: unsigned / signed integer order; floats by IEEE total order
 *     restricted to non-NaN values (-0.0 < +0.0). NaNs are accepted and
 *     ordered by their bit pattern (positive NaNs above +inf, negative NaNs
 *     below -inf); they are not validated.
 *   - Ties are broken by the smallest index. The top-k output is sorted by
 *     (key descending, index ascending); indices are int32.
 *   - 1 <= k <= n <= 2^31 - 1. Other values return DRTOPK_ERR_K (k) or
 *     DRTOPK_ERR_INVALID (n, pointers).
 *   - Device pointers point to memory of the current CUDA device. Keys must
 *     be 4-byte aligned; 16-byte alignment takes the TMA fast path. With any
 *     alignment, bulk copies may read the bytes of the 16-byte block that
 *     holds keys[0] before keys[0] (never past the 16-byte block that holds
 *     keys[n-1]); those bytes are never part of a result.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Calls are asynchronous on `stream` unless stated otherwise:
 *     results are valid once the stream has reached the call. The input
 *     must stay alive and unmodified until then.
 *   - The library allocates its temporary workspace with the stream-ordered
 *     allocator from a memory pool of its own per device (freed workspace
 *     stays cached there; the device's default pool is left untouched) and
 *     owns it; under a caller's stream capture the workspace is a graph
 *     allocation. The caller owns every input and output buffer.
 *   - drtopk_kth, drtopk_topk and drtopk_topk_ex (without statistics) keep a
 *     cache of CUDA graphs of whole queries, keyed by every argument
 *     (pointers, sizes, dtype, alpha, beta, device, stream): the second
 *     call with a key captures a graph and later calls replay it instead of
 *     launching ~30 kernels (the first call launches kernel by kernel). Each
 *     cached entry owns a workspace; entries are evicted least-recently-used
 *     beyond 64 entries or DRTOPK_GRAPH_CACHE_BYTES (default 16 GiB) of
 *     workspace. DRTOPK_GRAPH_CACHE=0 disables the cache. Calls made while
 *     profiling (drtopk_profile_begin) or on a stream that is being captured
 *     launch kernel by kernel (into the caller's capture).
 *   - Calls return a drtopk_status and never abort. A CUDA error returns
 *     DRTOPK_ERR_CUDA; argument checks happen before any CUDA call.
 *   - Device-side errors: every wait inside a kernel is bounded; a wait
 *     that gives up (DRTOPK_ERR_TIMEOUT) or a capacity guard that fires
 *     (DRTOPK_ERR_INTERNAL) leaves that query's outputs undefined. Since
 *     calls are asynchronous, such an error is reported later: the last
 *     kernel of each query of drtopk_kth / drtopk_topk / drtopk_topk_ex
 *     (without statistics) ORs its error flags into a per-device report
 *     word, which the next of these calls on the device reads and clears
 *     (it then returns the error and does nothing), and which
 *     drtopk_sync_status reads and clears after synchronizing. Calls with
 *     statistics and the synchronous calls (drtopk_topk_host, batched
 *     plans' status, server tickets) report their own errors directly.
 */
#ifndef DRTOPK_H
#define DRTOPK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DRTOPK_U32 = 0,
  DRTOPK_I32 = 1,
  DRTOPK_F32 = 2
} drtopk_dtype;

typedef enum {
  DRTOPK_OK = 0,
  DRTOPK_ERR_INVALID = 1, /* bad n, null pointer, bad alpha/beta, bad handle */
  DRTOPK_ERR_K = 2,       /* k outside [1, n] */
  DRTOPK_ERR_DTYPE = 3,   /* dtype not one of drtopk_dtype */
  DRTOPK_ERR_NOMEM = 4,   /* workspace allocation failed */
  DRTOPK_ERR_CUDA = 5,    /* a CUDA call failed */
  DRTOPK_ERR_BUDGET = 6,  /* server: request larger than the HBM budget */
  DRTOPK_ERR_TIMEOUT = 7, /* a bounded device-side wait gave up */
  DRTOPK_PENDING = 8,     /* server: ticket not finished yet */
  DRTOPK_ERR_INTERNAL = 9 /* a device-side capacity guard fired */
} drtopk_status;

/* Human-readable name of a status. Never NULL. */
const char* drtopk_status_str(drtopk_status s);

/*
 * Synchronizes `stream`, then reads and clears the device-side error flags
 * reported on the current device since the last check (by single queries
 * and by drtopk_kth_noalloc; see the conventions above): DRTOPK_OK when
 * none, DRTOPK_ERR_TIMEOUT when a bounded wait gave up, DRTOPK_ERR_INTERNAL
 * for any other device-side flag. The flags are per device, not per stream.
 */
drtopk_status drtopk_sync_status(void* stream);

/*
 * Self-test of device-side wait handling (no counterpart in the paper):
 * launches one small kernel on `stream` that waits, bounded by timeout_us
 * microseconds (1 .. 10^7), on an mbarrier phase that nothing completes,
 * using the same bounded wait as the bulk-copy rings, and reports the
 * timeout through the device's report word like a query does. Afterwards
 * drtopk_sync_status returns DRTOPK_ERR_TIMEOUT once; the context stays
 * usable. No GPU fault is involved.
 */
drtopk_status drtopk_wait_selftest(uint32_t timeout_us, void* stream);

/*
 * Parameter choice (host only, no CUDA call). Rule 4 / Eq. 9 (Sec. 4.2):
 * alpha = floor((log2 n - log2 k + 3) / 2), clamped to [2, 16], then lowered
 * while fewer than 2k delegates would exist (beta * ceil(n / 2^alpha) < 2k)
 * and alpha > 2. beta = 2 (Sec. 3.3). *workspace_bytes receives the device
 * workspace a top-k call with these parameters allocates (may be NULL).
 */
drtopk_status drtopk_plan(int64_t n, int64_t k, int* alpha, int* beta,
                          size_t* workspace_bytes);

/*
 * k-selection (Sec. 1): out_kth[0] = the k-th largest key of keys[0..n),
 * written with the input's dtype. keys, out_kth: device pointers.
 */
drtopk_status drtopk_kth(const void* keys, drtopk_dtype dtype, int64_t n,
                         int64_t k, void* out_kth, void* stream);

/*
 * top-k (Sec. 1): out_keys[0..k) (dtype of the input) and out_idx[0..k)
 * (int32 positions in keys) receive the k largest keys, sorted by (key
 * descending, index ascending); among equal keys the smallest indices win.
 * keys, out_keys, out_idx: device pointers.
 */
drtopk_status drtopk_topk(const void* keys, drtopk_dtype dtype, int64_t n,
                          int64_t k, void* out_keys, int32_t* out_idx,
                          void* stream);

/* Criterion flag of drtopk_select and drtopk_topk_merge. */
#define DRTOPK_SMALLEST 1

/*
 * Top-k and / or k-selection by either criterion of the problem statement
 * (Sec. 1 and Sec. 2: "the k largest or smallest"; the paper describes the
 * largest). flags = 0: the k largest keys, sorted by (key descending, index
 * ascending), and the k-th largest: the results of drtopk_topk /
 * drtopk_kth. flags = DRTOPK_SMALLEST: the k smallest keys, sorted by (key
 * ascending, index ascending), and the k-th smallest; among equal keys the
 * smallest indices win. Same method: the smallest criterion complements
 * the order-mapped key, so delegates, threshold and filter keep the k
 * smallest. Give out_keys and out_idx (top-k), out_kth (k-selection), or
 * all three. keys, outputs: device pointers. Graph-cached like
 * drtopk_topk.
 */
drtopk_status drtopk_select(const void* keys, drtopk_dtype dtype, int64_t n,
                            int64_t k, int flags, void* out_keys,
                            int32_t* out_idx, void* out_kth, void* stream);

/*
 * Exchange step of the distributed form (Sec. 4.4, "Distributed Dr. Top-k":
 * each GPU computes the top-k of its own contiguous sub-vector, the lists
 * are gathered on the primary GPU, which computes the final top-k). Given
 * `parts` lists concatenated in keys / idx, list p at positions
 * [part_off[p], part_off[p+1]) holding the result of drtopk_select (same
 * flags) on a sub-vector whose position i has global index
 * part_base[p] + i, writes the final top-k: out_keys[0..k) (dtype) and
 * out_gidx[0..k) (int64 global indices), sorted and tie-broken as
 * drtopk_select does over the whole vector. Requirements (not checked):
 * each list is sorted as drtopk_select returns it, and the lists appear in
 * increasing order of disjoint global index ranges (part_base[p] + its
 * largest index < part_base[p+1]). Then among equal keys the order of
 * positions is the order of global indices, and the single-query path over
 * the concatenation is the exact merge; a list shorter than k (a
 * sub-vector with fewer than k keys) is allowed. The union holds the
 * answer: an element of the global top-k is in its own sub-vector's
 * top-k. part_off, part_base: HOST arrays (parts + 1 and parts entries,
 * 1 <= parts <= 256, part_off nondecreasing, part_off[0] >= 0);
 * keys, idx (int32, as drtopk_select writes them), out_keys, out_gidx:
 * device pointers. 1 <= k <= part_off[parts] - part_off[0] <= 2^31 - 1.
 */
drtopk_status drtopk_topk_merge(const void* keys, const int32_t* idx,
                                drtopk_dtype dtype, const int64_t* part_off,
                                const int64_t* part_base, int32_t parts,
                                int64_t k, int flags, void* out_keys,
                                int64_t* out_gidx, void* stream);

/* Per-query statistics of the delegate-centric path (Sec. 5.2 workload
 * statistics: delegate and concatenated vector sizes). */
typedef struct {
  int32_t alpha;           /* subrange size exponent used */
  int32_t beta;            /* delegates per subrange used */
  int64_t subranges;       /* S = ceil(n / 2^alpha) */
  uint32_t tau;            /* threshold, order-mapped key (Rule 2) */
  uint32_t kth_mapped;     /* k-th largest key, order-mapped */
  int64_t greater;         /* |{x > tau}|: candidates kept by the filter */
  int64_t ties_needed;     /* k - greater when greater < k, else 0 */
  int64_t scanned;         /* subranges read again by the filter (Rule 3) */
  int64_t tie_scanned;     /* subranges read again to rank ties at tau */
  int64_t survivors;       /* candidates left after the first digit of the
                              second top-k */
  int64_t emitted;         /* outputs written (equals k on success) */
  uint32_t error;          /* device error flags, 0 when none */
  uint32_t delegate_path;  /* bit 0: the delegate pass stored only the records
                              of subranges reaching a sampled bound (speculative
                              compaction of the delegate vector, 16-byte aligned
                              arrays of 2^26 keys or more with alpha in [5, 10]);
                              bit 1: a fallback pass wrote the full delegate
                              arrays (alone: the sample declined; with bit 0: the
                              bound was above tau, the records overflowed, or the
                              query ended in tie mode). 0: the full pass alone.
                              The result is exact either way. */
} drtopk_stats;

/*
 * Extended query: alpha / beta forced when > 0 (alpha in [2, 16], beta in
 * [1, 4], beta <= 2^alpha), else chosen as drtopk_plan does. Either out_keys
 * and out_idx (top-k) or out_kth (k-selection) or all three may be given;
 * when only out_kth is given the call runs k-selection. stats: HOST pointer,
 * optional; when given, the call synchronizes `stream` and fills it.
 */
drtopk_status drtopk_topk_ex(const void* keys, drtopk_dtype dtype, int64_t n,
                             int64_t k, int alpha, int beta, void* out_keys,
                             int32_t* out_idx, void* out_kth,
                             drtopk_stats* stats, void* stream);

/*
 * Ablations of the method (Sec. 5's ablation study; results stay exact):
 *   DRTOPK_ABLATE_NO_FILTER: Rule 2's filtering off: every subrange whose
 *     maximum delegate reaches tau (Rule 1) is concatenated whole, not only
 *     its keys above tau; the candidate workspace grows to n.
 *   DRTOPK_ABLATE_SKIP_LAST_DIGIT: the first top-k stops one 8-bit digit
 *     early (Sec. 3.3): tau = the k-th largest delegate with its low byte
 *     cleared, a lower threshold; the candidate workspace grows to n.
 * beta = 1 is Rules 1 + 2 alone (no Rule 3). alpha / beta as for
 * drtopk_topk_ex; stats optional (HOST; synchronizes `stream` when given).
 * Never served from the graph cache.
 */
#define DRTOPK_ABLATE_NO_FILTER 1
#define DRTOPK_ABLATE_SKIP_LAST_DIGIT 2
drtopk_status drtopk_topk_ablate(const void* keys, drtopk_dtype dtype, int64_t n, int64_t k,
                                 int alpha, int beta, int flags, void* out_keys,
                                 int32_t* out_idx, drtopk_stats* stats, void* stream);

/*
 * The delegate pass alone (Sec. 3.1, 3.3, 4.1), exposed as a stage. For
 * each subrange i of 2^alpha keys (the last may be shorter) writes its beta
 * largest keys, order-mapped, to d_keys[i*beta + j] (descending, ties by
 * smaller index) and their int32 positions in keys to d_idx[i*beta + j].
 * A subrange with fewer than beta keys pads with key 0 and index -1.
 * d_keys, d_idx: device, ceil(n / 2^alpha) * beta entries.
 */
drtopk_status drtopk_delegates(const void* keys, drtopk_dtype dtype,
                               int64_t n, int alpha, int beta,
                               uint32_t* d_keys, int32_t* d_idx,
                               void* stream);

/*
 * k-selection without any allocation (the paper has no counterpart; this
 * entry point exists for callers that may not allocate device memory while
 * serving queries, e.g. pipelines that forbid allocation after start-up or
 * processes whose device memory is wholly owned by another allocator).
 * Same arguments and result as drtopk_kth, but the workspace is a fixed
 * 64 MiB array inside this library (a file-scope __device__ array): every
 * GPU that loads the library holds it until the process exits, and no
 * cudaMalloc, cudaMallocAsync or cudaFree is called.
 *   - Limit: the query's workspace (delegate keys and segments, the
 *     candidates above the threshold and their survivors) must fit in
 *     64 MiB; otherwise the call returns DRTOPK_ERR_NOMEM and launches
 *     nothing. For n = 2^30 this admits k up to about 4096.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture on the device.
 *   - All calls on a device share the array, which keeps the previous call's
 *     contents (the call clears what must start at zero). Calls that overlap
 *     on the GPU (different streams or threads without ordering between
 *     them) race on the array and give wrong results: order them.
 *   - Device-side errors of these calls are reported by drtopk_sync_status
 *     (the call itself cannot read them back without allocating).
 */
drtopk_status drtopk_kth_noalloc(const void* keys, drtopk_dtype dtype,
                                 int64_t n, int64_t k, void* out_kth,
                                 void* stream);

/*
 * top-k of a HOST array: copies keys (host, pinned or pageable) to the
 * device, computes what drtopk_topk computes and copies the results back to
 * host out_keys / out_idx. Synchronous: returns when the host outputs are
 * written. The keys travel in pieces of whole subranges (about 128 MB) on a
 * copy stream of the library; the delegate pass of each piece runs on
 * `stream` as soon as that piece has landed, while the later pieces are
 * still in flight, and the rest of the query follows the last piece. The
 * device copy goes to a staging buffer the library keeps per device, grown
 * to the largest call so far (n * 4 + 2 k * 4 bytes, 256-byte aligned
 * parts) and held until the process exits. Calls on one device are
 * serialised on that buffer. With pageable host memory the copies do not
 * overlap the kernels.
 */
drtopk_status drtopk_topk_host(const void* keys, drtopk_dtype dtype,
                               int64_t n, int64_t k, void* out_keys,
                               int32_t* out_idx, void* stream);

/*
 * ---------------------------------------------------------------- batched --
 * Many independent top-k queries over rows of one concatenated array, all
 * in ONE persistent kernel launch (the paper applies the method to one
 * vector per call; the batched form runs the same steps per row: delegate
 * pass Sec. 3.1/3.3, threshold Rule 2 Sec. 3.2, filter Rules 2-3, second
 * top-k Sec. 4.1, with the k-th key and ties as in drtopk_topk). One CTA
 * takes one row at a time, largest rows first; every intermediate (the
 * delegate vector, the candidates up to 4096) stays in shared memory.
 *
 * Rows: row r is keys[row_off[r] .. row_off[r+1]) (row_off: rows+1 int64,
 * row_off[0] >= 0), with 1 <= length <= 2^24 and k_r = ks[r] (int32) in
 * [1, min(length, 4096)]. row_off and ks may be host or device pointers
 * (a device array is copied to the host to plan the launch: synchronous). The outputs of row r
 * are out_keys / out_idx[o_r .. o_r + k_r) with o_r = k_0 + ... + k_{r-1}
 * (packed in row order), sorted by (key descending, index ascending); an
 * index is the position within the row. keys (device) must be 4-byte
 * aligned; rows may start at any element (a row's bulk copies may read the
 * bytes of its first 16-byte block before its first key, never past it).
 *
 * Per-row parameters: rows of at most 4096 keys are selected directly (no
 * delegates: the row is held on chip and radix-selected). Longer rows take
 * (alpha, beta) from the tuning table entry of (floor(log2 n_r),
 * floor(log2 k_r)) when one is set (drtopk_tune_set,
 * drtopk_autotune_batched; alpha = 1 there means the direct select), else
 * the direct select when the row fits on chip (direct_max_onchip of
 * drtopk_batch_limits) and 2 * ceil(n_r / 32) < 2k_r (even one subrange per
 * 32 keys gives too few delegates), else alpha by Rule 4 / Eq. 9 and
 * beta = 2, lowered while fewer than 2k_r delegates would exist. alpha is
 * then raised to at least 5 and until beta * ceil(n_r / 2^alpha) <=
 * max_delegates (the delegates fit on chip).
 */
typedef struct drtopk_batch_plan drtopk_batch_plan;

/* Limits of the batched path (host only; any pointer may be NULL):
 * max_k = 4096, max_row = 2^24 keys, direct_max = 4096 (rows up to this
 * length always skip the delegates), direct_max_onchip = longest row the
 * direct select can hold on chip, max_delegates = delegate slots per row
 * kept on chip, onchip_candidates = candidates kept on chip before
 * spilling to the plan's device scratch. */
drtopk_status drtopk_batch_limits(int32_t* max_k, int64_t* max_row, int32_t* direct_max,
                                  int32_t* direct_max_onchip, int32_t* max_delegates,
                                  int32_t* onchip_candidates);

/*
 * Builds a reusable plan for a fixed row layout: per-row parameters, the
 * processing order and a device scratch for candidates that exceed shared
 * memory (sized by the bound |{x > tau}| < floor((k-1)/beta) 2^alpha + k of
 * every row). alpha / beta > 0 force the parameters of every row longer
 * than 4096 keys (alpha in [5, 16], beta in [1, 4]; the on-chip clamp still
 * applies; alpha = 1 selects directly every row that fits on chip); 0 picks
 * them as described above. Allocates device memory;
 * synchronous. *out receives the plan (release with
 * drtopk_batch_plan_destroy).
 */
drtopk_status drtopk_batch_plan_create(drtopk_dtype dtype, const int64_t* row_off,
                                       const int32_t* ks, int32_t rows, int alpha,
                                       int beta, drtopk_batch_plan** out);

/*
 * Runs the plan on `stream`: one memset and one kernel launch, no host
 * synchronization and no allocation, so the call may be captured in a CUDA
 * graph. keys: device, at least row_off[rows] elements; out_keys / out_idx:
 * device, sum(ks) entries each. Device-side errors are read by
 * drtopk_batch_plan_status. Calls that share a plan must be ordered.
 */
drtopk_status drtopk_batch_plan_run(drtopk_batch_plan* plan, const void* keys,
                                    void* out_keys, int32_t* out_idx, void* stream);

/* Synchronizes `stream` and returns the device error status of the last
 * run of the plan (DRTOPK_ERR_TIMEOUT when a bounded wait gave up). */
drtopk_status drtopk_batch_plan_status(drtopk_batch_plan* plan, void* stream);

/* (alpha, beta) the plan uses for each row, in row order (HOST arrays of
 * `rows` entries; alpha 0 marks a direct select). */
drtopk_status drtopk_batch_plan_params(const drtopk_batch_plan* plan, int32_t* alpha,
                                       int32_t* beta);

/*
 * Device cycles (clock64 of the first thread of each CTA, summed over CTAs
 * and over runs since the last reset) spent in each step of the batched
 * kernel. Rows with delegates: out[0] delegate pass, [1] threshold select,
 * [2] filter, [3] second select (or sort of all candidates), [4] tie
 * ranking, [5] final sort and output. Directly selected rows: [6] load,
 * [7] select, [8] collection, [9] sort and output. out: HOST, 10 entries.
 * reset != 0 clears the counters. Synchronizes `stream`.
 */
#define DRTOPK_BATCH_PHASES 10
drtopk_status drtopk_batch_plan_phase_cycles(drtopk_batch_plan* plan, uint64_t* out,
                                             int reset, void* stream);

/* Synchronizes the device and frees the plan. */
drtopk_status drtopk_batch_plan_destroy(drtopk_batch_plan* plan);

/* One-shot batched top-k: plan, run, status, destroy. Synchronous. */
drtopk_status drtopk_topk_batched(const void* keys, drtopk_dtype dtype,
                                  const int64_t* row_off, const int32_t* ks,
                                  int32_t rows, void* out_keys, int32_t* out_idx,
                                  void* stream);

/*
 * The per-shape tuning table of the batched path (process-wide), indexed by
 * log2n in [10, 31] and log2k in [0, 12]. alpha = 0 (the initial state)
 * means the default choice; set alpha in [5, 16] with beta in [1, 4], or
 * alpha = 1 for the direct select. Host only.
 */
drtopk_status drtopk_tune_get(int32_t log2n, int32_t log2k, int* alpha, int* beta);
drtopk_status drtopk_tune_set(int32_t log2n, int32_t log2k, int alpha, int beta);

/*
 * Autotuner (Sec. 4.2 picks alpha by a model; this measures instead): for
 * every log2n in [min_log2n, max_log2n] (10..24) and every power-of-two k
 * up to min(4096, n / 2), times the batched kernel on rows_per_shape rows of
 * 2^log2n hashed keys for alpha in [Rule 4 - 3, Rule 4 + 2] (within [5, 16])
 * and beta in {1, 2, 3, 4}, and stores the fastest pair in the table.
 * Allocates 2^max_log2n * rows_per_shape keys; synchronous.
 */
drtopk_status drtopk_autotune_batched(drtopk_dtype dtype, int32_t min_log2n,
                                      int32_t max_log2n, int32_t rows_per_shape,
                                      void* stream);

/*
 * ----------------------------------------------------------------- server --
 * Continuous batching of top-k requests (no counterpart in the paper, which
 * answers one query per call). A scheduler thread admits submitted requests
 * in arrival order while the device-resident state of the admitted ones fits
 * the HBM budget: for each request its keys (4n bytes), outputs (8k bytes)
 * and, for a single query, the workspace drtopk_plan reports; plus the
 * server's own buffers (fixed_bytes of the statistics, about 0.6 GB for 152
 * SMs). Admitted requests with n <= batch_max_n (default 2^20), k <= 4096
 * and candidates within the batched scratch are coalesced, per dtype, into
 * batched launches (drtopk_topk_batched's kernel, up to 4096 rows, two
 * launches in flight); the others run as single queries, round-robin over
 * four streams, so that large and small work overlap. Results are those of
 * drtopk_topk on the same arguments, bit for bit.
 *
 * Ownership: the caller owns keys (device, 4-byte aligned), out_keys and
 * out_idx (device, k entries each); keys must stay alive and unmodified and
 * the outputs untouched until the ticket completes. Submit, poll and wait
 * may be called from any host thread.
 */
typedef struct drtopk_server drtopk_server;

/* flags of drtopk_server_create_ex */
#define DRTOPK_SERVER_PLAIN 1 /* no batching: every request is one plain
                                 single-query launch sequence on one stream,
                                 in arrival order (the baseline) */

typedef struct {
  uint64_t submitted, completed, failed;
  uint64_t batches;          /* batched launches */
  uint64_t batched_requests; /* requests served by them */
  uint64_t single_queries;   /* requests served as single queries */
  uint64_t peak_bytes;       /* largest admitted state + fixed_bytes */
  uint64_t in_use_bytes;     /* admitted state now + fixed_bytes */
  uint64_t fixed_bytes;      /* the server's own device buffers */
} drtopk_server_stats;

/* Creates a server on `device` (starts its scheduler thread). Returns
 * DRTOPK_ERR_BUDGET when the budget does not exceed the server's own
 * buffers. batch_max_n: largest n sent to batched launches (0: 2^20). */
drtopk_status drtopk_server_create(size_t hbm_budget_bytes, int device, drtopk_server** out);
drtopk_status drtopk_server_create_ex(size_t hbm_budget_bytes, int device, int flags,
                                      int64_t batch_max_n, drtopk_server** out);

/* Queues a top-k request (1 <= k <= n <= 2^31 - 1). *ticket identifies it.
 * DRTOPK_ERR_BUDGET when the request alone exceeds the budget. Never
 * blocks on the GPU. */
drtopk_status drtopk_server_submit(drtopk_server* srv, const void* keys, drtopk_dtype dtype,
                                   int64_t n, int64_t k, void* out_keys, int32_t* out_idx,
                                   uint64_t* ticket);

/* DRTOPK_PENDING while the request runs; else its final status (DRTOPK_OK
 * when the outputs are written), after which the ticket is forgotten (a
 * later poll returns DRTOPK_ERR_INVALID). _ex also returns the latency from
 * submission to completion seen by the scheduler, in microseconds. */
drtopk_status drtopk_server_poll(drtopk_server* srv, uint64_t ticket);
drtopk_status drtopk_server_poll_ex(drtopk_server* srv, uint64_t ticket, double* latency_us);

/* Blocks until the request completes; then as drtopk_server_poll_ex. */
drtopk_status drtopk_server_wait(drtopk_server* srv, uint64_t ticket, double* latency_us);

drtopk_status drtopk_server_get_stats(drtopk_server* srv, drtopk_server_stats* out);

/* Host only: the bytes a request counts against the budget and whether it
 * would be batched (flags and batch_max_n as for drtopk_server_create_ex). */
drtopk_status drtopk_server_footprint(drtopk_dtype dtype, int64_t n, int64_t k, int flags,
                                      int64_t batch_max_n, size_t* bytes, int* batched);

/* Finishes every submitted request, stops the scheduler and frees the
 * server. Tickets not yet polled are forgotten. */
drtopk_status drtopk_server_destroy(drtopk_server* srv);

/* Stage timing (CUDA events recorded on the launching stream around each
 * stage while profiling is on). Stages: 0 delegate pass, 1 threshold
 * select, 2 filter, 3 tie ranking, 4 second top-k, 5 output sort. */
#define DRTOPK_NUM_STAGES 6
typedef struct {
  double ms[DRTOPK_NUM_STAGES];       /* summed device time per stage */
  int64_t launches[DRTOPK_NUM_STAGES]; /* queries that ran the stage */
} drtopk_profile;

/* Start collecting stage times (clears previous data). Host only. */
drtopk_status drtopk_profile_begin(void);
/* Stop collecting; synchronizes the recorded events and fills *out. */
drtopk_status drtopk_profile_end(drtopk_profile* out);

/* Number of kernels this library has launched since it was loaded. */
uint64_t drtopk_launch_count(void);

/* Number of device or pinned-host allocations this library has made since
 * it was loaded (each workspace taken from its stream-ordered pool counts,
 * as do memory pools, staging buffers, graph-cache workspaces, batched
 * plans and server buffers). Host only. */
uint64_t drtopk_alloc_count(void);

#ifdef __cplusplus
}
#endif

#endif /* DRTOPK_H */
