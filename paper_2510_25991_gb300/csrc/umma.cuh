// umma.cuh -- shared-memory operand layout of the tcgen05 tensor-core kernels.
//
// Canonical K-major layout without swizzle: core matrices of 8 rows x 16 bytes (4 TF32
// values); core matrix (row group g, K group kk) of a rows x K operand starts at byte
// g * (K * 32) + kk * 128, i.e. leading byte offset (K direction) 128 and stride byte offset
// (row direction) 32 K.
#pragma once
#include <cstdint>

namespace ddst {

__host__ __device__ __forceinline__ uint32_t umma_off(int row, int k, int K) {
  return (uint32_t)((row >> 3) * (K * 32) + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// Round to TF32 (nearest, ties away): the 3xTF32 split x = hi + lo uses hi = rna(x),
// lo = rna(x - hi).
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Writes the TF32 hi/lo split of (-diag(scale) X)^T in the K-major operand layout: operand row
// r, K index c holds -scale[c] * X(c, r); X is M x M row-major in shared memory with leading
// dimension ld, scale a global vector of M values (NULL: the copy is zero).
__device__ __forceinline__ void store_umma_split_T(const float* __restrict__ X, int ld, int M,
                                                   const float* __restrict__ scale,
                                                   float* __restrict__ hi,
                                                   float* __restrict__ lo) {
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
    const int r = e / M, c = e - r * M;
    const float v = scale ? -scale[c] * X[c * ld + r] : 0.f;
    const float h = tf32_rna(v);
    const uint32_t o = umma_off(r, c, M) >> 2;
    hi[o] = h;
    lo[o] = tf32_rna(v - h);
  }
}

}  // namespace ddst
