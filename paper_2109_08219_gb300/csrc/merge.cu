// Exchange step of the distributed form (Sec. 4.4, "Distributed Dr. Top-k"):
// every GPU computes the top-k of its own contiguous shard; the primary GPU
// gathers the lists and computes the final top-k over them. The final top-k
// runs the single-query path over the concatenated lists; this file maps
// its output positions back to global indices.
#include "common.cuh"
#include "launch.h"

namespace drtopk {
namespace {

// Thread j: position pos[j] in the concatenated lists -> its part p (the
// last part whose first position is <= pos) -> global index
// part_base[p] + idx[pos].
__global__ void merge_gather_kernel(MergeParts mp, const int32_t* pos, const int32_t* idx,
                                    int64_t k, int64_t* out_gidx) {
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < k;
       j += int64_t(gridDim.x) * blockDim.x) {
    const int64_t q = pos[j];
    int lo = 0, hi = mp.parts - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (mp.off[mid] <= q) lo = mid;
      else hi = mid - 1;
    }
    out_gidx[j] = mp.base[lo] + static_cast<int64_t>(idx[q]);
  }
}

}  // namespace

cudaError_t launch_merge_gather(const MergeParts& mp, const int32_t* pos, const int32_t* idx,
                                int64_t k, int64_t* out_gidx, int sms, cudaStream_t s) {
  const int64_t want = (k + 255) / 256;
  const int grid = static_cast<int>(want < int64_t(sms) * 8 ? (want > 0 ? want : 1) : int64_t(sms) * 8);
  merge_gather_kernel<<<grid, 256, 0, s>>>(mp, pos, idx, k, out_gidx);
  note_launch();
  return cudaGetLastError();
}

}  // namespace drtopk
