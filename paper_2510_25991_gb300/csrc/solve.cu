// solve.cu -- single-right-hand-side local solves with the two-sided factorization.
//
// Local Dirichlet solves on every double slab are needed for the equivalent loads
// fhat_j = R_{C_j} A_j^{-1} b (Sec. 2.2, Eq. (equilib1)), for the volume reconstruction from
// interface traces, and (transposed) for the adjoint.  With forward pivots Sigma_k (inverse F_k),
// backward pivots Lambda_k (inverse B_k) and G_k = (Sigma_k + Lambda_k - D_k)^{-1}:
//   top-down   bf_1 = b_1,   bf_k = b_k - L_k F_{k-1} bf_{k-1}
//   bottom-up  bb_nb = b_nb, bb_k = b_k - U_k B_{k+1} bb_{k+1}
//   x_k = G_k (bf_k + bb_k - b_k)                       (all k in parallel)
// For A^T the couplings swap (L_k^T = U_{k-1}-position, diagonal) and every block is transposed:
//   bf_k = b_k - diag(ups_{k-1}) F_{k-1}^T bf_{k-1},  bb_k = b_k - diag(ell_{k+1}) B_{k+1}^T bb_{k+1},
//   x_k = G_k^T (bf_k + bb_k - b_k).
// The two sweeps of a slab run concurrently in two CTAs; each streams its factor blocks
// through a ring of bulk (TMA) copies.
#include "kernels.cuh"

namespace ddst {

// One sweep of one slab (blockIdx.y = 0: top-down with F, 1: bottom-up with B).  The product
// y = A v is formed as y[r] = sum_c W[c][r] v[c] with W = A^T row-major (thread per row, no
// bank conflicts): W = F^T, B^T for A^{-1} sweeps and W = F, B for A^{-T} sweeps.  Each ring
// stage carries the factor block, the right-hand-side block and the coupling vector of one step
// (three bulk copies on one mbarrier); the ring is deep enough to keep ~NST steps in flight.
// 4 M threads: thread t handles row t % M over the column quarter t / M (a warp shares one
// quarter, so the shared-memory reads of W are conflict-free); the quarters' partial sums are
// combined in shared memory before the row update.
template <typename T, int M, int NST>
__global__ void __launch_bounds__(4 * M) k_solve_sweep(const SlabDesc* __restrict__ slabs,
                                                   const int* __restrict__ ids,
                                                   const T* __restrict__ Wf,
                                                   const T* __restrict__ Wb,
                                                   const T* __restrict__ pack,
                                                   const T* __restrict__ b, T* __restrict__ bf,
                                                   T* __restrict__ bb, int transpose,
                                                   DevStatus* st) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sW = reinterpret_cast<T*>(smem_raw);   // [NST][M*M]
  T* sB = sW + NST * M * M;                 // [NST][M] right-hand-side block
  T* sC = sB + NST * M;                     // [NST][M] coupling vector
  T* sv = sC + NST * M;                     // [M] current vector
  T* red = sv + M;                          // [4][M] partial sums of the column quarters
  uint64_t* bar = reinterpret_cast<uint64_t*>(red + 4 * M);
  __shared__ int s_abort;
  const int sid = ids[blockIdx.x];
  const SlabDesc s = slabs[sid];
  const bool down = blockIdx.y == 0;
  const T* Fac = (down ? Wf : Wb) + s.fac_off;
  T* out = (down ? bf : bb) + s.loc_off;
  const T* rhs = b + s.loc_off;
  const int nb = s.nb;
  const int r = threadIdx.x % M, part = threadIdx.x / M;
  int issued = 0, consumed = 0;
  auto blk_of = [&](int step) { return down ? step + 1 : nb - step; };
  // coupling: non-transposed top-down ell_k (SOUTH of k), bottom-up ups_k (NORTH of k);
  // transposed top-down ups_{k-1} (NORTH of k-1), bottom-up ell_{k+1} (SOUTH of k+1).
  auto issue = [&](int step) {
    ++issued;
    const int k = blk_of(step);
    const int fidx = down ? k - 2 : k;
    int cfield, cblk;
    if (!transpose) { cfield = down ? PK_SOUTH : PK_NORTH; cblk = k; }
    else { cfield = down ? PK_NORTH : PK_SOUTH; cblk = down ? k - 1 : k + 1; }
    const int stage = (step - 1) % NST;
    mbar_arrive_expect_tx(&bar[stage], (M * M + 2 * M) * sizeof(T));
    bulk_g2s(sW + stage * M * M, Fac + (int64_t)fidx * M * M, M * M * sizeof(T), &bar[stage]);
    bulk_g2s(sB + stage * M, rhs + (int64_t)(k - 1) * M, M * sizeof(T), &bar[stage]);
    bulk_g2s(sC + stage * M, pack + s.pack_off + (int64_t)(cblk - 1) * PK_NFIELDS * M + cfield * M,
             M * sizeof(T), &bar[stage]);
  };
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int q = 0; q < NST; ++q) mbar_init(&bar[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 1; q <= NST && q < nb; ++q) issue(q);
  if (part == 0) {
    const int k = blk_of(0);
    const T v = rhs[(int64_t)(k - 1) * M + r];
    sv[r] = v;
    out[(int64_t)(k - 1) * M + r] = v;
  }
  __syncthreads();
  for (int step = 1; step < nb; ++step) {
    const int k = blk_of(step);
    const int stage = (step - 1) % NST;
    if (!mbar_wait(&bar[stage], ((step - 1) / NST) & 1, st, sid, k)) s_abort = 1;
    consumed = step;
    const T* W = sW + stage * M * M;
    T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
    const int c0 = part * (M / 4);
#pragma unroll
    for (int c = c0; c < c0 + M / 4; c += 4) {
      a0 = fma(W[c * M + r], sv[c], a0);
      a1 = fma(W[(c + 1) * M + r], sv[c + 1], a1);
      a2 = fma(W[(c + 2) * M + r], sv[c + 2], a2);
      a3 = fma(W[(c + 3) * M + r], sv[c + 3], a3);
    }
    red[part * M + r] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    if (s_abort) break;
    if (part == 0) {
      const T v = sB[stage * M + r] -
                  sC[stage * M + r] * ((red[r] + red[M + r]) + (red[2 * M + r] + red[3 * M + r]));
      sv[r] = v;
      out[(int64_t)(k - 1) * M + r] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0 && step + NST < nb) {
      fence_proxy_async();
      issue(step + NST);
    }
  }
  if (threadIdx.x == 0)
    for (int q = consumed + 1; q <= issued; ++q)
      mbar_wait(&bar[(q - 1) % NST], ((q - 1) / NST) & 1, st, sid, -1);
}

// x_k = G_k (bf_k + bb_k - b_k)  (or G_k^T (...)).  grid = (nb, nslab-of-class).
// mode 0: full block written to x (slab-local); mode 1: only the central rows, written as FP64
// into the interface vector iface at the slab's offset.
template <typename T, int M>
__global__ void __launch_bounds__(128) k_solve_combine(const SlabDesc* __restrict__ slabs,
                                                       const int* __restrict__ ids,
                                                       const T* __restrict__ G,
                                                       const T* __restrict__ b,
                                                       const T* __restrict__ bf,
                                                       const T* __restrict__ bb,
                                                       T* __restrict__ x, double* __restrict__ iface,
                                                       int transpose, int mode) {
  const SlabDesc s = slabs[ids[blockIdx.y]];
  const int k = blockIdx.x + 1;
  if (k > s.nb) return;
  __shared__ T sv[M];
  const int64_t o = s.loc_off + (int64_t)(k - 1) * M;
  for (int c = threadIdx.x; c < M; c += blockDim.x) sv[c] = bf[o + c] + bb[o + c] - b[o + c];
  __syncthreads();
  const T* Gk = G + s.fac_off + (int64_t)(k - 1) * M * M;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (mode == 0) {
    if (!transpose) {  // a warp takes 4 consecutive rows per round (M/8 loads in flight per lane)
      for (int r0 = warp * 4; r0 < M; r0 += 16) {
        T p[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          p[u] = T(0);
#pragma unroll
          for (int c = lane; c < M; c += 32) p[u] += Gk[(r0 + u) * M + c] * sv[c];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const T v = warp_sum(p[u]);
          if (lane == 0) x[o + r0 + u] = v;
        }
      }
    } else {
      for (int r = threadIdx.x; r < M; r += blockDim.x) {
        T acc = T(0);
        for (int c = 0; c < M; ++c) acc += Gk[c * M + r] * sv[c];
        x[o + r] = acc;
      }
    }
  } else {
    // central rows C_t = (w-1)p + t, t = 0..p-1 (non-transposed only)
    for (int t = warp; t < s.p; t += 4) {
      const int r = (s.w - 1) * s.p + t;
      T part = T(0);
      for (int c = lane; c < M; c += 32) part += Gk[r * M + c] * sv[c];
      part = warp_sum(part);
      if (lane == 0) iface[s.if_off + (int64_t)(k - 1) * s.p + t] = static_cast<double>(part);
    }
  }
}

template <typename T, int M, int NST>
static void run_solve(const SlabDesc* d_slabs, const int* d_ids, int nids, int max_nb,
                      const T* F, const T* B, const T* Ft, const T* Bt, const T* G,
                      const T* pack, const T* b, T* bf, T* bb, T* x, double* iface,
                      int transpose, int mode, DevStatus* st, cudaStream_t s) {
  const size_t smem = (size_t)NST * (M * M + 2 * M) * sizeof(T) + 5 * M * sizeof(T) + NST * 8;
  raise_smem_limit(reinterpret_cast<const void*>(&k_solve_sweep<T, M, NST>), smem);
  // A^{-1} sweeps multiply by F, B: pass their transposes (thread-per-row form); A^{-T} sweeps
  // multiply by F^T, B^T: pass F, B.
  const T* Wf = transpose ? F : Ft;
  const T* Wb = transpose ? B : Bt;
  note_launch();
  k_solve_sweep<T, M, NST><<<dim3(nids, 2), 4 * M, smem, s>>>(d_slabs, d_ids, Wf, Wb, pack, b, bf, bb,
                                                         transpose, st);
  note_launch();
  k_solve_combine<T, M><<<dim3(max_nb, nids), 128, 0, s>>>(d_slabs, d_ids, G, b, bf, bb, x, iface,
                                                          transpose, mode);
}

template <typename T>
void launch_local_solve(int M, const SlabDesc* d_slabs, const int* d_ids, int nids, int max_nb,
                        const T* F, const T* B, const T* Ft, const T* Bt, const T* G,
                        const T* pack, const T* b, T* bf, T* bb, T* x, double* iface,
                        int transpose, int mode, DevStatus* st, cudaStream_t s) {
  if (nids == 0) return;
  // ring depth: ~200 KB of stages in flight per slab sweep
  constexpr bool F32 = sizeof(T) == 4;
  switch (M) {
    case 32: run_solve<T, 32, F32 ? 24 : 16>(d_slabs, d_ids, nids, max_nb, F, B, Ft, Bt, G, pack, b, bf, bb, x, iface, transpose, mode, st, s); break;
    case 64: run_solve<T, 64, F32 ? 11 : 5>(d_slabs, d_ids, nids, max_nb, F, B, Ft, Bt, G, pack, b, bf, bb, x, iface, transpose, mode, st, s); break;
    case 128: run_solve<T, 128, F32 ? 3 : 1>(d_slabs, d_ids, nids, max_nb, F, B, Ft, Bt, G, pack, b, bf, bb, x, iface, transpose, mode, st, s); break;
    default: break;
  }
}

template void launch_local_solve<float>(int, const SlabDesc*, const int*, int, int, const float*,
                                        const float*, const float*, const float*, const float*,
                                        const float*, const float*, float*, float*, float*,
                                        double*, int, int, DevStatus*, cudaStream_t);
template void launch_local_solve<double>(int, const SlabDesc*, const int*, int, int,
                                         const double*, const double*, const double*,
                                         const double*, const double*, const double*,
                                         const double*, double*, double*, double*, double*, int,
                                         int, DevStatus*, cudaStream_t);

}  // namespace ddst
