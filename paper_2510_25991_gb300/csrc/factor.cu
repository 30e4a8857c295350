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
#include "bgj.cuh"
#include "kernels.cuh"
#include "umma.cuh"

namespace ddst {

// X (shared, leading dimension LD) += D_k: the diagonal and the x / z couplings of row r sit in
// the stencil pack pk at p and 1 entries off the diagonal (x and z neighbours of the node), one
// thread per row instead of a lookup per entry of the block.
template <typename T>
__device__ __forceinline__ void add_dblock(T* __restrict__ X, int LD, const T* __restrict__ pk,
                                           int M, int m, int p) {
  for (int r = threadIdx.x; r < M; r += blockDim.x) {
    T* row = X + r * LD;
    row[r] += pk[PK_DIAG * M + r];
    if (r >= m) continue;
    const int cx = r / p, t = r - cx * p;
    if (cx >= 1) row[r - p] += pk[PK_WEST * M + r];
    if (r + p < m) row[r + p] += pk[PK_EAST * M + r];
    if (t >= 1) row[r - 1] += pk[PK_ZLO * M + r];
    if (t + 1 < p) row[r + 1] += pk[PK_ZHI * M + r];
  }
}

// Writes X (shared, LD) as a row-major M x M block to `dst` (4 consecutive entries per thread)
// and, if dstT, its transpose.
template <typename T, int M>
__device__ __forceinline__ void store_block(const T* __restrict__ X, T* __restrict__ dst,
                                            T* __restrict__ dstT) {
  constexpr int LD = BGJ<T, M>::LD;
  for (int e = threadIdx.x; e < M * (M / 4); e += blockDim.x) {
    const int i = e / (M / 4), j = 4 * (e - i * (M / 4));
#pragma unroll
    for (int u = 0; u < 4; ++u) dst[i * M + j + u] = X[i * LD + j + u];
  }
  if (dstT)
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
      const int i = e / M, j = e - i * M;
      dstT[e] = X[j * LD + i];
    }
}

// One chunk of a forward (dir 0) or backward (dir 1) pivot sweep.  Rows are visited from
// `start` through `last` (ascending for dir 0, descending for dir 1); inverses are stored for the
// rows from `first` on.  A chunk whose start is not the slab's end row begins with
// Sigma_start = D_start (its warm-up rows): the pivot recurrence forgets its initial value
// exponentially (about exp(-pi/w) per row for slab width w), so after the warm-up the pivots
// agree with the sequential ones to rounding.  The warm-up's last inverse is written to the
// check slot `chk` and compared with the previous chunk's stored inverse of the same row by
// k_factor_verify; the host falls back to the exact sequential sweep if any check fails.  The
// stencil pack of the next row is prefetched by a bulk copy while the current one is inverted.
// Each chunk's recurrence is latency-bound (one block row at a time), so throughput comes from
// concurrent chunks: the FP32 kernel runs 128-thread CTAs, 6 resident per SM (shared memory).
template <typename T> struct FactorOcc {
  static constexpr int threads = 256, min_blocks = 1;
};
template <> struct FactorOcc<float> {
  static constexpr int threads = 128, min_blocks = 6;
};

template <typename T, int M>
__global__ void __launch_bounds__(FactorOcc<T>::threads, FactorOcc<T>::min_blocks) k_factor(const SlabDesc* __restrict__ slabs,
                                                const FacChunk* __restrict__ chunks,
                                                const T* __restrict__ pack, T* __restrict__ F,
                                                T* __restrict__ B, T* __restrict__ Ft,
                                                T* __restrict__ Bt, T* __restrict__ chk,
                                                float* __restrict__ Uhi, float* __restrict__ Ulo,
                                                int64_t umma_elems, DevStatus* st) {
  using G = BGJ<T, M>;
  constexpr int LD = G::LD;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* X = reinterpret_cast<T*>(smem_raw);
  T* Cp = X + M * LD;
  T* Rp = Cp + G::CP;
  T* pk = Rp + G::NB * LD;              // [3][PK_NFIELDS * M]: ring (previous, current, next)
  T* thr = pk + 3 * PK_NFIELDS * M;     // [M]
  uint64_t* bar = reinterpret_cast<uint64_t*>(thr + M);  // [3]
  const FacChunk ch = chunks[blockIdx.x];
  const int sid = ch.slab;
  const SlabDesc s = slabs[sid];
  const int dir = ch.dir;
  // Uhi/Ulo hold the forward copies in [0, umma_half) and the backward ones behind them
  const int64_t umma_half = umma_elems;
  const int sgn = dir == 0 ? 1 : -1;
  const int len = (ch.last - ch.start) * sgn + 1;
  T* out = (dir == 0 ? F : B) + s.fac_off;
  T* outT = (dir == 0 ? Ft : Bt) + s.fac_off;
  const int rowfield = dir == 0 ? PK_SOUTH : PK_NORTH;   // ell_k (fwd) or ups_k (bwd)
  const int colfield = dir == 0 ? PK_NORTH : PK_SOUTH;   // ups_{k-1} (fwd) or ell_{k+1} (bwd)
  const uint32_t pbytes = PK_NFIELDS * M * sizeof(T);
  auto blk = [&](int step) { return ch.start + sgn * step; };
  auto issue = [&](int step) {
    const int k = blk(step);
    mbar_arrive_expect_tx(&bar[step % 3], pbytes);
    bulk_g2s(pk + (step % 3) * PK_NFIELDS * M, pack + s.pack_off + (int64_t)(k - 1) * PK_NFIELDS * M,
             pbytes, &bar[step % 3]);
  };
  if (threadIdx.x == 0) {
    for (int q = 0; q < 3; ++q) mbar_init(&bar[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) issue(0);
  int waited = 0, issued = 1;
  bool ok = true;
  for (int step = 0; step < len; ++step) {
    const int k = blk(step);
    if (!mbar_wait(&bar[step % 3], (step / 3) & 1, st, sid, k)) ok = false;
    waited = step + 1;
    __syncthreads();
    if (!ok) break;
    if (threadIdx.x == 0 && step + 1 < len) {
      fence_proxy_async();
      issue(step + 1);
      ++issued;
    }
    const T* cur = pk + (step % 3) * PK_NFIELDS * M;
    const T* prv = pk + ((step + 2) % 3) * PK_NFIELDS * M;   // previous row (step - 1)
    for (int i = threadIdx.x; i < M; i += blockDim.x) thr[i] = T(1e3) * Eps<T>::v * fabs(cur[PK_DIAG * M + i]);
    // Sigma_k = D_k - diag(ell_k) F_{k-1} diag(ups_{k-1})   (backward: ups_k, B_{k+1}, ell_{k+1})
    for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
      const int r = e / M, c = e - r * M;
      X[r * LD + c] = step > 0 ? -(cur[rowfield * M + r] * X[r * LD + c] * prv[colfield * M + c]) : T(0);
    }
    __syncthreads();
    add_dblock<T>(X, LD, cur, M, s.m, s.p);
    __syncthreads();
    bgj_invert<T, M>(X, Cp, Rp, thr, st, sid, k);
    if ((k - ch.first) * sgn >= 0) {
      store_block<T, M>(X, out + (int64_t)(k - 1) * M * M, outT + (int64_t)(k - 1) * M * M);
      if constexpr (sizeof(T) == 4) {
        // tensor-core operand copy of the transfer-build step (transposed, TF32 hi/lo, K-major):
        // forward -diag(ell_{k+1}) F_k, backward -diag(ups_{k-1}) B_k, so that a sweep step of
        // Alg. 1 is the plain product Y_next^T = Y^T (scaled copy).  The copies of F_nb and B_1
        // are never used and are written as zeros.
        if (Uhi) {
          const int kn = k + sgn;  // the block whose coupling scales this inverse
          const float* scl = (kn >= 1 && kn <= s.nb)
                                 ? reinterpret_cast<const float*>(pack) + s.pack_off +
                                       (int64_t)(kn - 1) * PK_NFIELDS * M + rowfield * M
                                 : nullptr;
          store_umma_split_T<M>(reinterpret_cast<const float*>(X), LD, scl,
                             Uhi + (dir == 0 ? 0 : umma_half) + s.fac_off + (int64_t)(k - 1) * M * M,
                             Ulo + (dir == 0 ? 0 : umma_half) + s.fac_off + (int64_t)(k - 1) * M * M);
        }
      }
    }
    else if (ch.chk >= 0 && k == ch.first - sgn)
      store_block<T, M>(X, chk + (int64_t)ch.chk * M * M, nullptr);
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = waited; q < issued; ++q) mbar_wait(&bar[q % 3], (q / 3) & 1, st, sid, -1);
}

// Convergence check of the warm-started chunks: relative max difference between a chunk's
// warm-up inverse and the previous chunk's stored inverse of the same row.  One CTA per chunk.
template <typename T, int M>
__global__ void k_factor_verify(const SlabDesc* __restrict__ slabs,
                                const FacChunk* __restrict__ chunks, const T* __restrict__ F,
                                const T* __restrict__ B, const T* __restrict__ chk,
                                float* __restrict__ diff) {
  const FacChunk ch = chunks[blockIdx.x];
  if (ch.chk < 0) {
    if (threadIdx.x == 0) diff[blockIdx.x] = 0.f;
    return;
  }
  const SlabDesc s = slabs[ch.slab];
  const int row = ch.first - (ch.dir == 0 ? 1 : -1);
  const T* ref = (ch.dir == 0 ? F : B) + s.fac_off + (int64_t)(row - 1) * M * M;
  const T* got = chk + (int64_t)ch.chk * M * M;
  float md = 0.f, mr = 0.f;
  // live m x m block only: the padded diagonal of an inverse is 1, far above its h^2-sized
  // entries, and would hide any difference in them
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
    const int r = e / M, c = e - r * M;
    if (r >= s.m || c >= s.m) continue;
    md = fmaxf(md, (float)fabs(ref[e] - got[e]));
    mr = fmaxf(mr, (float)fabs(ref[e]));
  }
  __shared__ float sd[256], sr[256];
  sd[threadIdx.x] = md;
  sr[threadIdx.x] = mr;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sd[threadIdx.x] = fmaxf(sd[threadIdx.x], sd[threadIdx.x + o]);
      sr[threadIdx.x] = fmaxf(sr[threadIdx.x], sr[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) diff[blockIdx.x] = sr[0] > 0.f ? sd[0] / sr[0] : 0.f;
}

// Diagonal blocks of the inverse: G_k = (D_k - L_k F_{k-1} U_{k-1} - U_k B_{k+1} L_{k+1})^{-1}.
// grid = (nb, slabs of the class).
template <typename T, int M>
__global__ void __launch_bounds__(256) k_center(const SlabDesc* __restrict__ slabs,
                                                const int* __restrict__ slab_ids,
                                                const T* __restrict__ pack,
                                                const T* __restrict__ F, const T* __restrict__ B,
                                                T* __restrict__ Gout, DevStatus* st) {
  using G = BGJ<T, M>;
  constexpr int LD = G::LD;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* X = reinterpret_cast<T*>(smem_raw);
  T* Cp = X + M * LD;
  T* Rp = Cp + G::CP;
  T* pk = Rp + G::NB * LD;          // [PK_NFIELDS * M]
  T* thr = pk + PK_NFIELDS * M;     // [M]
  T* up = thr + M;                  // ups_{k-1}
  T* ln = up + M;                   // ell_{k+1}
  const int sid = slab_ids[blockIdx.y];
  const SlabDesc s = slabs[sid];
  const int k = blockIdx.x + 1;
  if (k > s.nb) return;
  const T* pkg = pack + s.pack_off + (int64_t)(k - 1) * PK_NFIELDS * M;
  for (int i = threadIdx.x; i < PK_NFIELDS * M; i += blockDim.x) pk[i] = pkg[i];
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    up[i] = k > 1 ? pack[s.pack_off + (int64_t)(k - 2) * PK_NFIELDS * M + PK_NORTH * M + i] : T(0);
    ln[i] = k < s.nb ? pack[s.pack_off + (int64_t)k * PK_NFIELDS * M + PK_SOUTH * M + i] : T(0);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < M; i += blockDim.x) thr[i] = T(1e3) * Eps<T>::v * fabs(pk[PK_DIAG * M + i]);
  const T* Fp = F + s.fac_off + (int64_t)(k - 2) * M * M;  // F_{k-1}
  const T* Bn = B + s.fac_off + (int64_t)k * M * M;        // B_{k+1}
  for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
    const int r = e / M, c = e - r * M;
    T v = T(0);
    if (k > 1) v -= pk[PK_SOUTH * M + r] * Fp[e] * up[c];
    if (k < s.nb) v -= pk[PK_NORTH * M + r] * Bn[e] * ln[c];
    X[r * LD + c] = v;
  }
  __syncthreads();
  add_dblock<T>(X, LD, pk, M, s.m, s.p);
  __syncthreads();
  bgj_invert<T, M>(X, Cp, Rp, thr, st, sid, k);
  store_block<T, M>(X, Gout + s.fac_off + (int64_t)(k - 1) * M * M, nullptr);
}

template <typename T, int M>
static size_t factor_smem() {
  return BGJ<T, M>::smem_elems * sizeof(T) + (3 * PK_NFIELDS * M + M) * sizeof(T) + 24;
}

template <typename T, int M>
void launch_factor_M(const SlabDesc* d_slabs, const FacChunk* d_chunks, int nchunks,
                     const int* d_ids, int nids, int max_nb, const T* pack, T* F, T* B, T* G,
                     T* Ft, T* Bt, T* chk, float* diff, float* Uhi, float* Ulo,
                     int64_t umma_elems, int phase, DevStatus* st, cudaStream_t s) {
  using Gc = BGJ<T, M>;
  const size_t sm_f = factor_smem<T, M>();
  const size_t sm_c = Gc::smem_elems * sizeof(T) + (PK_NFIELDS * M + 3 * M) * sizeof(T);
  raise_smem_limit(reinterpret_cast<const void*>(&k_factor<T, M>), sm_f);
  raise_smem_limit(reinterpret_cast<const void*>(&k_center<T, M>), sm_c);
  if (phase == 0) {  // pivot sweeps + convergence check of warm-started chunks
    if (nchunks == 0) return;
    note_launch();
    k_factor<T, M><<<nchunks, FactorOcc<T>::threads, sm_f, s>>>(d_slabs, d_chunks, pack, F, B, Ft, Bt, chk, Uhi, Ulo,
                                              umma_elems, st);
    note_launch();
    k_factor_verify<T, M><<<nchunks, 256, 0, s>>>(d_slabs, d_chunks, F, B, chk, diff);
  } else {           // diagonal blocks of the inverse
    if (nids == 0) return;
    note_launch();
    k_center<T, M><<<dim3(max_nb, nids), 256, sm_c, s>>>(d_slabs, d_ids, pack, F, B, G, st);
  }
}

template <typename T>
void launch_factor(int M, int phase, const SlabDesc* d_slabs, const FacChunk* d_chunks,
                   int nchunks, const int* d_ids, int nids, int max_nb, const T* pack, T* F,
                   T* B, T* G, T* Ft, T* Bt, T* chk, float* diff, float* Uhi, float* Ulo,
                   int64_t umma_elems, DevStatus* st, cudaStream_t s) {
  switch (M) {
    case 32: launch_factor_M<T, 32>(d_slabs, d_chunks, nchunks, d_ids, nids, max_nb, pack, F, B, G, Ft, Bt, chk, diff, Uhi, Ulo, umma_elems, phase, st, s); break;
    case 64: launch_factor_M<T, 64>(d_slabs, d_chunks, nchunks, d_ids, nids, max_nb, pack, F, B, G, Ft, Bt, chk, diff, Uhi, Ulo, umma_elems, phase, st, s); break;
    case 128: launch_factor_M<T, 128>(d_slabs, d_chunks, nchunks, d_ids, nids, max_nb, pack, F, B, G, Ft, Bt, chk, diff, nullptr, nullptr, 0, phase, st, s); break;
    default: break;
  }
}

// Resident factor CTAs per SM for block size M (drives the chunk count).
template <typename T>
int factor_ctas_per_sm(int M) {
  int n = 0;
  switch (M) {
    case 32: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_factor<T, 32>, FactorOcc<T>::threads, factor_smem<T, 32>()); break;
    case 64: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_factor<T, 64>, FactorOcc<T>::threads, factor_smem<T, 64>()); break;
    case 128: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_factor<T, 128>, FactorOcc<T>::threads, factor_smem<T, 128>()); break;
    default: break;
  }
  cudaGetLastError();
  return n > 0 ? n : 1;
}

template void launch_factor<float>(int, int, const SlabDesc*, const FacChunk*, int, const int*,
                                   int, int, const float*, float*, float*, float*, float*,
                                   float*, float*, float*, float*, float*, int64_t, DevStatus*,
                                   cudaStream_t);
template void launch_factor<double>(int, int, const SlabDesc*, const FacChunk*, int, const int*,
                                    int, int, const double*, double*, double*, double*, double*,
                                    double*, double*, float*, float*, float*, int64_t, DevStatus*,
                                    cudaStream_t);
template int factor_ctas_per_sm<float>(int);
template int factor_ctas_per_sm<double>(int);

}  // namespace ddst
