// splittile.cuh -- 128 x 128 operand tiles pre-split into TF32 parts for the tcgen05 kernels
// (large-block Gauss-Jordan panels, batched dense products).
#pragma once
#include "umma.cuh"

namespace ddst {

constexpr int BT = 128;  // panel width and output tile edge

// ---------------------------------------------------------------------------------------------
// Operand tiles of the tensor-core steps are stored once, already split into TF32 parts
// (hi = rna(x), lo = rna(x - hi)) in the canonical K-major layout, chunk-major: element (r, k) of
// a 128 x 128 tile (r: output row, k: contraction index) sits at float offset
//     (k / 16) * 2048 + umma_off(r, k % 16, 16) / 4
// of the hi part, and 16384 floats further in the lo part.  One 16-wide K chunk of one part is a
// contiguous 8 KB block, so the MMA kernels load their operands with plain bulk copies.
// ---------------------------------------------------------------------------------------------
constexpr int SPLIT_TILE = 2 * BT * BT;  // floats of one split tile (hi + lo)

__device__ __forceinline__ int split_off(int r, int k) {
  return (k >> 4) * 2048 + (int)(umma_off(r, k & 15, 16) >> 2);
}

// Element (r, k) read from shared memory at src[r * ldr + k * ldk].
__device__ __forceinline__ void store_split_tile(const float* __restrict__ src, int ldr, int ldk,
                                                 float* __restrict__ dst) {
  for (int e = threadIdx.x; e < BT * (BT / 4); e += blockDim.x) {
    const int r = e % BT, k = 4 * (e / BT);
    float x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = src[r * ldr + (k + u) * ldk];
    float4 h, l;
    h.x = tf32_rna(x[0]); l.x = tf32_rna(x[0] - h.x);
    h.y = tf32_rna(x[1]); l.y = tf32_rna(x[1] - h.y);
    h.z = tf32_rna(x[2]); l.z = tf32_rna(x[2] - h.z);
    h.w = tf32_rna(x[3]); l.w = tf32_rna(x[3] - h.w);
    const int o = split_off(r, k);
    *reinterpret_cast<float4*>(dst + o) = h;
    *reinterpret_cast<float4*>(dst + BT * BT + o) = l;
  }
}


}  // namespace ddst
