// Host-side launchers of the drtopk kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace drtopk {

// Counts every kernel this library launches (drtopk_launch_count).
void note_launch(int n = 1);

// Delegate pass (delegate.cu). fuse_hist: also histogram the first digit of
// the threshold select and resolve it in the last block.
cudaError_t launch_delegates(const Work& w, const void* keys, bool fuse_hist, int sms,
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

// Number of 2048-subrange blocks of the tie scans (select.cu).
int64_t tie_blocks(int64_t S);

// Resolves exact delegate positions for drtopk_delegates (select.cu).
cudaError_t launch_resolve_delegates(const Work& w, const void* keys, int32_t* d_idx,
                                     cudaStream_t s);

}  // namespace drtopk
