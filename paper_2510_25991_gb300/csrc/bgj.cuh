// bgj.cuh -- blocked Gauss-Jordan inversion of a small dense block in shared memory (no
// pivoting), shared by the pivot sweeps of the single-CTA factorization and by the pivot-block
// step of the large-block factorization.
#pragma once
#include "common.cuh"

namespace ddst {

// ---------------------------------------------------------------------------------------------
// Blocked Gauss-Jordan inversion in shared memory (block pivots of 16): the 16 x 16 pivot
// block is inverted by warp 0 (warp-synchronous, no pivoting), then the pivot row panel
// R = P^{-1} X(q, :), the column panel C = X(:, q) and the trailing update
// X(i, j) -= C(i, :) R(:, j), X(i, q) = -C(i, :) P^{-1} run on all threads as small GEMMs.
// Three block barriers per 16 pivots.  X has leading dimension LD = M + 4 (16-byte rows).
// The trailing update runs over 4 x 4 patches distributed round-robin over the threads, with
// 16-byte shared-memory loads of the column panel (kept transposed) and the row panel.
// ---------------------------------------------------------------------------------------------
template <typename T, int M>
struct BGJ {
  static constexpr int LD = M + 4;
  static constexpr int NB = 16;
  // column panel, stored transposed (NB rows of LD): C(i, t) at Cp[t * LD + i]
  static constexpr size_t CP = (size_t)NB * LD;
  static constexpr size_t smem_elems = (size_t)M * LD + CP + (size_t)NB * LD;
};

// Four consecutive elements from 16-byte-aligned shared memory.
__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 f = *reinterpret_cast<const float4*>(p);
  v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

template <typename T, int M>
__device__ __forceinline__ void bgj_invert(T* __restrict__ X, T* __restrict__ Cp,
                                           T* __restrict__ Rp, const T* __restrict__ thr,
                                           DevStatus* st, int slab, int block) {
  using G = BGJ<T, M>;
  constexpr int LD = G::LD, NB = G::NB;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  for (int q0 = 0; q0 < M; q0 += NB) {
    // (a) warp 0 inverts the pivot block in registers: lane owns row lane/2, columns
    //     8*(lane&1)..+7; pivot rows and entries travel by warp shuffles (no barriers).
    if (warp == 0) {
      const int r = lane >> 1, h = lane & 1;
      T* P = X + q0 * LD + q0;
      T v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = P[r * LD + 8 * h + e];
      for (int pp = 0; pp < NB; ++pp) {
        T prow[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) prow[e] = __shfl_sync(0xffffffffu, v[e], 2 * pp + h);
        const int sel = pp & 7;
        const T lo4 = (sel & 2) ? ((sel & 1) ? v[3] : v[2]) : ((sel & 1) ? v[1] : v[0]);
        const T hi4 = (sel & 2) ? ((sel & 1) ? v[7] : v[6]) : ((sel & 1) ? v[5] : v[4]);
        const T pe = (sel & 4) ? hi4 : lo4;
        T piv = __shfl_sync(0xffffffffu, pe, 2 * pp + (pp >> 3));
        const T fv = __shfl_sync(0xffffffffu, pe, 2 * r + (pp >> 3));
        const T lim = thr[q0 + pp];
        if (!(fabs(piv) > lim)) {
          if (lane == 0) set_status(st, ST_SINGULAR, slab, block);
          piv = (piv < T(0)) ? -lim : lim;
          if (lim == T(0)) piv = T(1);
        }
        const T inv = T(1) / piv;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int c = 8 * h + e;
          const T ps = (c == pp ? T(1) : prow[e]) * inv;
          v[e] = (r == pp) ? ps : ((c == pp ? T(0) : v[e]) - fv * ps);
        }
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) P[r * LD + 8 * h + e] = v[e];
    }
    __syncthreads();
    // (b) column panel C = X(:, q) (old values; block rows unused; stored transposed) and row
    //     panel R = P^{-1} X(q, :)
    for (int e = tid; e < M * NB; e += blockDim.x) {
      const int i = e / NB, t = e - i * NB;
      Cp[t * LD + i] = X[i * LD + q0 + t];
    }
    for (int e = tid; e < NB * (M / 4); e += blockDim.x) {  // four columns per thread
      const int t = e / (M / 4), j = 4 * (e - t * (M / 4));
      T acc[4] = {T(0), T(0), T(0), T(0)};
      if (j < q0 || j >= q0 + NB) {
#pragma unroll
        for (int s2 = 0; s2 < NB; ++s2) {
          const T pv = X[(q0 + t) * LD + q0 + s2];
          T xv[4];
          ld4(X + (q0 + s2) * LD + j, xv);
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u] = fma(pv, xv[u], acc[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) Rp[t * LD + j + u] = acc[u];
    }
    __syncthreads();
    // (c) trailing update on 4 x 4 patches (patch index -> rows 4*pi.., columns 4*pj..)
    for (int pidx = tid; pidx < (M / 4) * (M / 4); pidx += blockDim.x) {
      {
        const int i0 = (pidx / (M / 4)) * 4, j0 = (pidx % (M / 4)) * 4;
        const bool in_i = (i0 >= q0 && i0 < q0 + NB), in_j = (j0 >= q0 && j0 < q0 + NB);
        if (in_i && in_j) continue;
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
        if (in_i) {
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) X[(i0 + a) * LD + j0 + b] = Rp[(i0 + a - q0) * LD + j0 + b];
          continue;
        }
        // rows outside the pivot block: need C(i, :) and either R(:, j) or P^{-1}(:, j)
#pragma unroll
        for (int t = 0; t < NB; ++t) {
          T cv[4], rv[4];
          ld4(Cp + t * LD + i0, cv);
          ld4(in_j ? (X + (q0 + t) * LD + j0) : (Rp + t * LD + j0), rv);
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(cv[a], rv[b], acc[a][b]);
        }
        if (in_j) {
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) X[(i0 + a) * LD + j0 + b] = -acc[a][b];
        } else {
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) X[(i0 + a) * LD + j0 + b] -= acc[a][b];
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace ddst
