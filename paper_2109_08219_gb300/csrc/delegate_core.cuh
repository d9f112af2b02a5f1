// Per-thread top-beta building blocks shared by the delegate pass of the
// single-query path and of the batched path (internal).
#pragma once

#include "common.cuh"

namespace drtopk {

template <int B>
struct Pow2 {
  static constexpr int v = (B <= 1) ? 1 : (B <= 2) ? 2 : 4;
};

// value-only insertion into a descending list m[0..B)
template <int B>
__device__ __forceinline__ void insert_val(uint32_t (&m)[B], uint32_t x) {
#pragma unroll
  for (int j = B - 1; j >= 1; --j) m[j] = max(m[j], min(m[j - 1], x));
  m[0] = max(m[0], x);
}

template <int DT, int B>
__device__ __forceinline__ void insert4(uint32_t (&m)[B], uint4 v) {
  insert_val<B>(m, map_key<DT>(v.x));
  insert_val<B>(m, map_key<DT>(v.y));
  insert_val<B>(m, map_key<DT>(v.z));
  insert_val<B>(m, map_key<DT>(v.w));
}

// Bitonic merge of two descending lists of P composites; result descending
// in a (the top P of the union).
template <int P>
__device__ __forceinline__ void merge_desc(uint64_t (&a)[P], const uint64_t (&b)[P]) {
#pragma unroll
  for (int i = 0; i < P; ++i) a[i] = max(a[i], b[P - 1 - i]);
  // a is bitonic; sort descending with half-cleaners
#pragma unroll
  for (int h = P / 2; h >= 1; h >>= 1) {
#pragma unroll
    for (int i = 0; i < P; ++i) {
      if ((i & h) == 0) {
        const uint64_t x = a[i], y = a[i + h];
        a[i] = max(x, y);
        a[i + h] = min(x, y);
      }
    }
  }
}

template <int P>
__device__ __forceinline__ void shfl_merge(uint64_t (&a)[P], int xor_off) {
  uint64_t b[P];
#pragma unroll
  for (int i = 0; i < P; ++i) b[i] = __shfl_xor_sync(0xFFFFFFFFu, a[i], xor_off);
  merge_desc<P>(a, b);
}

// Scalar-key variant for shared-memory data of arbitrary alignment.
template <int DT, int B>
__device__ __forceinline__ void insert1(uint32_t (&m)[B], uint32_t raw) {
  insert_val<B>(m, map_key<DT>(raw));
}

}  // namespace drtopk
