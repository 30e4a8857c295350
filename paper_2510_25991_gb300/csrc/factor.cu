// factor.cu -- two-sided block factorization of every double-slab operator A_j(I_j, I_j).
//
// The paper factors each local stiffness matrix by a sparse LU (Sec. 2.5, Alg. 2, "factorize
// A_j(I_j,I_j) = L_j U_j", pivoting omitted).  Here every double slab is ordered along y into
// nb blocks of m = (2w-1)(n-1)^(dim-2) unknowns, which makes A_j block tridiagonal:
//     L_k x_{k-1} + D_k x_k + U_k x_{k+1},   L_k = diag(ell_k), U_k = diag(ups_k).
// Two block-LU sweeps are computed concurrently (one CTA per slab and direction):
//   forward pivots   Sigma_1 = D_1,   Sigma_k  = D_k - L_k Sigma_{k-1}^{-1} U_{k-1}
//   backward pivots  Lambda_nb = D_nb, Lambda_k = D_k - U_k Lambda_{k+1}^{-1} L_{k+1}
// and their explicit inverses F_k = Sigma_k^{-1}, B_k = Lambda_k^{-1} are stored, each also
// transposed (thread-per-row products in the single-RHS sweeps need both orientations).  A third,
// fully parallel pass stores the diagonal blocks of the inverse,
//     G_k = (A_j^{-1})_{kk} = (Sigma_k + Lambda_k - D_k)^{-1},
// which lets multi-right-hand-side solves start from any block and single solves run their
// two sweeps at the same time.  No pivoting (as in the paper); a pivot below
// 1e3 * eps * |D_k(p,p)| reports DDST_ERR_SINGULAR with the slab and block.
#include "kernels.cuh"

namespace ddst {

// Entry (r, c) of the diagonal block D_k from the stencil pack held in shared memory
// (cxr/tr, cxc/tc: x offset and z index of row r and column c, precomputed by the caller).
template <typename T>
__device__ __forceinline__ T dblock(const T* __restrict__ pk, int M, int m, int r, int c, int cxr,
                                    int tr, int cxc, int tc) {
  if (r == c) return pk[PK_DIAG * M + r];
  if (r >= m || c >= m) return T(0);
  if (tr == tc) {
    if (cxc == cxr - 1) return pk[PK_WEST * M + r];
    if (cxc == cxr + 1) return pk[PK_EAST * M + r];
  }
  if (cxr == cxc) {
    if (tc == tr - 1) return pk[PK_ZLO * M + r];
    if (tc == tr + 1) return pk[PK_ZHI * M + r];
  }
  return T(0);
}

// In-place Gauss-Jordan inversion of an M x M matrix held in registers by 256 threads
// (16 x 16 thread grid, RP x RP patch each).  One barrier per pivot (double-buffered pivot
// row/column).  Pivot magnitude check against thr[] (per row, shared memory).
template <typename T, int M>
__device__ __forceinline__ void gj_invert(T (&x)[M / 16][M / 16], int ty, int tx,
                                          T* __restrict__ s_row, T* __restrict__ s_col,
                                          const T* __restrict__ thr, DevStatus* st, int slab,
                                          int block) {
  constexpr int RP = M / 16;
  for (int p = 0; p < M; ++p) {
    const int buf = (p & 1) * M;
    const int owner = p / RP, pi = p - owner * RP;
    if (ty == owner) {
#pragma unroll
      for (int rr = 0; rr < RP; ++rr)
        if (rr == pi) {
#pragma unroll
          for (int cc = 0; cc < RP; ++cc) s_row[buf + tx * RP + cc] = x[rr][cc];
        }
    }
    if (tx == owner) {
#pragma unroll
      for (int cc = 0; cc < RP; ++cc)
        if (cc == pi) {
#pragma unroll
          for (int rr = 0; rr < RP; ++rr) s_col[buf + ty * RP + rr] = x[rr][cc];
        }
    }
    __syncthreads();
    T piv = s_row[buf + p];
    const T lim = thr[p];
    if (!(fabs(piv) > lim)) {  // also catches NaN
      if (threadIdx.x == 0) set_status(st, ST_SINGULAR, slab, block);
      piv = (piv < T(0)) ? -lim : lim;
      if (lim == T(0)) piv = T(1);
    }
    const T inv = T(1) / piv;
    T prow[RP], fcol[RP];
#pragma unroll
    for (int cc = 0; cc < RP; ++cc) {
      const int c = tx * RP + cc;
      prow[cc] = (c == p ? T(1) : s_row[buf + c]) * inv;
    }
#pragma unroll
    for (int rr = 0; rr < RP; ++rr) fcol[rr] = s_col[buf + ty * RP + rr];
#pragma unroll
    for (int rr = 0; rr < RP; ++rr) {
      const int r = ty * RP + rr;
#pragma unroll
      for (int cc = 0; cc < RP; ++cc) {
        const int c = tx * RP + cc;
        if (r == p)
          x[rr][cc] = prow[cc];
        else
          x[rr][cc] = (c == p ? T(0) : x[rr][cc]) - fcol[rr] * prow[cc];
      }
    }
  }
  __syncthreads();
}

// Forward (blockIdx.y == 0) or backward (== 1) pivot sweep of one slab (blockIdx.x indexes
// slab_ids, the slabs of this block-size class).
template <typename T, int M>
__global__ void __launch_bounds__(256) k_factor(const SlabDesc* __restrict__ slabs,
                                                const int* __restrict__ slab_ids,
                                                const T* __restrict__ pack, T* __restrict__ F,
                                                T* __restrict__ B, T* __restrict__ Ft,
                                                T* __restrict__ Bt, DevStatus* st) {
  constexpr int RP = M / 16;
  const int sid = slab_ids[blockIdx.x];
  const SlabDesc s = slabs[sid];
  const int dir = blockIdx.y;
  __shared__ T s_pk[PK_NFIELDS * M];
  __shared__ T s_cpl[M];
  __shared__ T s_row[2 * M], s_col[2 * M], s_thr[M];
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  T x[RP][RP];
#pragma unroll
  for (int rr = 0; rr < RP; ++rr)
#pragma unroll
    for (int cc = 0; cc < RP; ++cc) x[rr][cc] = T(0);
  T* out = (dir == 0 ? F : B) + s.fac_off;
  T* outT = (dir == 0 ? Ft : Bt) + s.fac_off;
  const int rowfield = dir == 0 ? PK_SOUTH : PK_NORTH;
  int cxr[RP], trr[RP], cxc[RP], tcc[RP];
#pragma unroll
  for (int q = 0; q < RP; ++q) {
    const int r = ty * RP + q, c = tx * RP + q;
    cxr[q] = r / s.p; trr[q] = r - cxr[q] * s.p;
    cxc[q] = c / s.p; tcc[q] = c - cxc[q] * s.p;
  }
  for (int step = 0; step < s.nb; ++step) {
    const int k = dir == 0 ? step + 1 : s.nb - step;
    const T* pk = pack + s.pack_off + (int64_t)(k - 1) * PK_NFIELDS * M;
    for (int i = threadIdx.x; i < PK_NFIELDS * M; i += blockDim.x) s_pk[i] = pk[i];
    if (step > 0) {
      const int kp = dir == 0 ? k - 1 : k + 1;
      const T* pp = pack + s.pack_off + (int64_t)(kp - 1) * PK_NFIELDS * M;
      for (int i = threadIdx.x; i < M; i += blockDim.x)
        s_cpl[i] = pp[(dir == 0 ? PK_NORTH : PK_SOUTH) * M + i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < M; i += blockDim.x)
      s_thr[i] = T(1e3) * Eps<T>::v * fabs(s_pk[PK_DIAG * M + i]);
#pragma unroll
    for (int rr = 0; rr < RP; ++rr) {
      const int r = ty * RP + rr;
      const T rs = s_pk[rowfield * M + r];
#pragma unroll
      for (int cc = 0; cc < RP; ++cc) {
        const int c = tx * RP + cc;
        const T d = dblock<T>(s_pk, M, s.m, r, c, cxr[rr], trr[rr], cxc[cc], tcc[cc]);
        x[rr][cc] = step > 0 ? d - rs * x[rr][cc] * s_cpl[c] : d;
      }
    }
    __syncthreads();
    gj_invert<T, M>(x, ty, tx, s_row, s_col, s_thr, st, sid, k);
    T* ob = out + (int64_t)(k - 1) * M * M;
    T* obT = outT + (int64_t)(k - 1) * M * M;
#pragma unroll
    for (int rr = 0; rr < RP; ++rr) {
      const int r = ty * RP + rr;
#pragma unroll
      for (int cc = 0; cc < RP; ++cc) {
        ob[r * M + tx * RP + cc] = x[rr][cc];
        obT[(tx * RP + cc) * M + r] = x[rr][cc];
      }
    }
  }
}

// Diagonal blocks of the inverse: G_k = (D_k - L_k F_{k-1} U_{k-1} - U_k B_{k+1} L_{k+1})^{-1}.
// grid = (nb, slabs of the class).
template <typename T, int M>
__global__ void __launch_bounds__(256) k_center(const SlabDesc* __restrict__ slabs,
                                                const int* __restrict__ slab_ids,
                                                const T* __restrict__ pack,
                                                const T* __restrict__ F, const T* __restrict__ B,
                                                T* __restrict__ G, DevStatus* st) {
  constexpr int RP = M / 16;
  const int sid = slab_ids[blockIdx.y];
  const SlabDesc s = slabs[sid];
  const int k = blockIdx.x + 1;
  if (k > s.nb) return;
  __shared__ T s_pk[PK_NFIELDS * M];
  __shared__ T s_up[M], s_ln[M];  // ups_{k-1} (cols of forward term), ell_{k+1} (backward term)
  __shared__ T s_row[2 * M], s_col[2 * M], s_thr[M];
  const T* pk = pack + s.pack_off + (int64_t)(k - 1) * PK_NFIELDS * M;
  for (int i = threadIdx.x; i < PK_NFIELDS * M; i += blockDim.x) s_pk[i] = pk[i];
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    s_up[i] = k > 1 ? pack[s.pack_off + (int64_t)(k - 2) * PK_NFIELDS * M + PK_NORTH * M + i] : T(0);
    s_ln[i] = k < s.nb ? pack[s.pack_off + (int64_t)k * PK_NFIELDS * M + PK_SOUTH * M + i] : T(0);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < M; i += blockDim.x)
    s_thr[i] = T(1e3) * Eps<T>::v * fabs(s_pk[PK_DIAG * M + i]);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  int cxr[RP], trr[RP], cxc[RP], tcc[RP];
#pragma unroll
  for (int q = 0; q < RP; ++q) {
    const int r = ty * RP + q, c = tx * RP + q;
    cxr[q] = r / s.p; trr[q] = r - cxr[q] * s.p;
    cxc[q] = c / s.p; tcc[q] = c - cxc[q] * s.p;
  }
  const T* Fp = F + s.fac_off + (int64_t)(k - 2) * M * M;  // F_{k-1}
  const T* Bn = B + s.fac_off + (int64_t)k * M * M;        // B_{k+1}
  T x[RP][RP];
#pragma unroll
  for (int rr = 0; rr < RP; ++rr) {
    const int r = ty * RP + rr;
    const T ell = s_pk[PK_SOUTH * M + r], ups = s_pk[PK_NORTH * M + r];
#pragma unroll
    for (int cc = 0; cc < RP; ++cc) {
      const int c = tx * RP + cc;
      T v = dblock<T>(s_pk, M, s.m, r, c, cxr[rr], trr[rr], cxc[cc], tcc[cc]);
      if (k > 1) v -= ell * Fp[r * M + c] * s_up[c];
      if (k < s.nb) v -= ups * Bn[r * M + c] * s_ln[c];
      x[rr][cc] = v;
    }
  }
  __syncthreads();
  gj_invert<T, M>(x, ty, tx, s_row, s_col, s_thr, st, sid, k);
  T* ob = G + s.fac_off + (int64_t)(k - 1) * M * M;
#pragma unroll
  for (int rr = 0; rr < RP; ++rr) {
    const int r = ty * RP + rr;
#pragma unroll
    for (int cc = 0; cc < RP; ++cc) ob[r * M + tx * RP + cc] = x[rr][cc];
  }
}

template <typename T, int M>
void launch_factor_M(const SlabDesc* d_slabs, const int* d_ids, int nids, int max_nb,
                     const T* pack, T* F, T* B, T* G, T* Ft, T* Bt, DevStatus* st,
                     cudaStream_t s) {
  if (nids == 0) return;
  note_launch();
  k_factor<T, M><<<dim3(nids, 2), 256, 0, s>>>(d_slabs, d_ids, pack, F, B, Ft, Bt, st);
  note_launch();
  k_center<T, M><<<dim3(max_nb, nids), 256, 0, s>>>(d_slabs, d_ids, pack, F, B, G, st);
}

template <typename T>
void launch_factor(int M, const SlabDesc* d_slabs, const int* d_ids, int nids, int max_nb,
                   const T* pack, T* F, T* B, T* G, T* Ft, T* Bt, DevStatus* st, cudaStream_t s) {
  switch (M) {
    case 32: launch_factor_M<T, 32>(d_slabs, d_ids, nids, max_nb, pack, F, B, G, Ft, Bt, st, s); break;
    case 64: launch_factor_M<T, 64>(d_slabs, d_ids, nids, max_nb, pack, F, B, G, Ft, Bt, st, s); break;
    case 128: launch_factor_M<T, 128>(d_slabs, d_ids, nids, max_nb, pack, F, B, G, Ft, Bt, st, s); break;
    default: break;
  }
}

template void launch_factor<float>(int, const SlabDesc*, const int*, int, int, const float*,
                                   float*, float*, float*, float*, float*, DevStatus*,
                                   cudaStream_t);
template void launch_factor<double>(int, const SlabDesc*, const int*, int, int, const double*,
                                    double*, double*, double*, double*, double*, DevStatus*,
                                    cudaStream_t);

}  // namespace ddst
