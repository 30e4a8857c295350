// bigblock.cu -- factorization and local solves of double slabs whose dense blocks are large
// (m > 128: every 3D double slab of a fine grid, and 2D slabs wider than 64 cells).
//
// Alg. 2 of the paper factors each local operator A_j(I_j, I_j) once (Sec. 2.5).  Ordered along y,
// A_j is block tridiagonal with dense diagonal blocks D_k of size m = (2w-1)(n-1)^(dim-2) and
// diagonal couplings L_k = diag(ell_k), U_k = diag(ups_k).  Here the one-sided block LU
//     Sigma_1 = D_1,   Sigma_k = D_k - L_k Sigma_{k-1}^{-1} U_{k-1},   F_k = Sigma_k^{-1}
// is computed with all slabs of a block-size class advancing together, one block row k at a time.
// Each F_k is formed in place: Sigma_k is written into the slot of F_k and inverted there by a
// blocked Gauss-Jordan elimination with 128-wide panels (no pivoting, as in the paper).  Per panel
// q (rows/columns Q = 128q .. 128q+127):
//   pivot    P = X(Q,Q), P^{-1} by the shared-memory Gauss-Jordan kernel; copies C = X(:,Q) and
//            X(Q,:)^T are kept for the next two steps
//   row      R = P^{-1} X(Q,:)  (stored transposed, R^T, and written back into X(Q,:));  R(:,Q) =
//            P^{-1}, so that the update below also produces the column panel
//   update   X(I,J) = X(I,J) - C(I,:) R(:,J) for I != Q, J != Q;  X(I,Q) = -C(I,:) P^{-1}
// The row and update steps are dense products with K = 128: tcgen05 tensor-core kernels in the
// FP32 path (3xTF32 with FP32 accumulation in tensor memory, or plain TF32 in the TF32 mode), FMA
// kernels in FP64 (and as an FP32 reference).  The local solves of a slab stream its F_k (forward and backward block sweeps,
// one batched matrix-vector product per block row); A_j^{-T} uses the same factors transposed.
#include "bgj.cuh"
#include "kernels.cuh"
#include "splittile.cuh"
#include "umma.cuh"

namespace ddst {

// ---------------------------------------------------------------------------------------------
// Sigma_k = D_k - diag(ell_k) F_{k-1} diag(ups_{k-1}), written into the slot of F_k.
// grid = (chunks, slabs of the class).
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_big_sigma(const SlabDesc* __restrict__ slabs,
                                                   const int* __restrict__ ids,
                                                   const T* __restrict__ pack, T* __restrict__ F,
                                                   int k) {
  const SlabDesc s = slabs[ids[blockIdx.y]];
  if (k > s.nb) return;
  const int M = s.M;
  T* X = F + s.fac_off + (int64_t)(k - 1) * M * M;
  const T* Xp = F + s.fac_off + (int64_t)(k - 2) * M * M;  // used only for k > 1
  const T* pk = pack + s.pack_off + (int64_t)(k - 1) * PK_NFIELDS * M;
  const T* pkp = pack + s.pack_off + (int64_t)(k - 2) * PK_NFIELDS * M;
  const int64_t total = (int64_t)M * M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / M), c = (int)(e - (int64_t)r * M);
    T v = T(0);
    if (r == c) {
      v = pk[PK_DIAG * M + r];
    } else if (r < s.m && c < s.m) {
      // x neighbours sit p entries away (same z), z neighbours one entry away (same x column)
      if (c == r - s.p) v = pk[PK_WEST * M + r];
      else if (c == r + s.p) v = pk[PK_EAST * M + r];
      else if (s.p > 1 && c == r - 1 && r % s.p != 0) v = pk[PK_ZLO * M + r];
      else if (s.p > 1 && c == r + 1 && r % s.p != s.p - 1) v = pk[PK_ZHI * M + r];
    }
    if (k > 1) v -= pk[PK_SOUTH * M + r] * Xp[e] * pkp[PK_NORTH * M + c];
    X[e] = v;
  }
}

// ---------------------------------------------------------------------------------------------
// Pivot step of panel q.  grid = (M/128, slabs).  CTA q inverts P = X(Q,Q) in shared memory
// (singular-pivot check against 1e3 eps |D_k|) and writes X(Q,Q) = P^{-1}; every other CTA b
// copies the tiles X(B,Q) and X(Q,B) of the column and row panels (on the tensor-core path only
// for the first panel of a block row: later panels' tiles are written split by the update and row
// steps of the panel before, and the launch has one CTA per slab).  Work buffers are per slab of
// the class.  FMA path (plain row-major): C = X(:,Q) (M x 128), XqT = X(Q,:)^T (M x 128),
// Pinv = P^{-1} (128 x 128), RT(Q rows) = P^{-T}.  Tensor-core path (SPLIT, split tiles): the
// same operands as split tiles, C tile b = X(B,Q), XqT tile b = X(Q,B)^T, Pinv = P^{-1} and RT
// tile q = P^{-T}, and C tile q = P.
// ---------------------------------------------------------------------------------------------
template <typename T, bool SPLIT>
__global__ void __launch_bounds__(512) k_big_pivot(const SlabDesc* __restrict__ slabs,
                                                   const int* __restrict__ ids,
                                                   const T* __restrict__ pack, T* __restrict__ F,
                                                   int k, int q, T* __restrict__ Cb,
                                                   T* __restrict__ XqT, T* __restrict__ RT,
                                                   T* __restrict__ Pinv, DevStatus* st) {
  using G = BGJ<T, BT>;
  constexpr int LD = G::LD;
  constexpr int LS = BT + 1;  // staging tiles: conflict-free row and column reads
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* Xs = reinterpret_cast<T*>(smem_raw);
  const int sid = ids[blockIdx.y];
  const SlabDesc s = slabs[sid];
  if (k > s.nb) return;
  const int M = s.M, nP = M / BT;
  T* X = F + s.fac_off + (int64_t)(k - 1) * M * M;
  // a grid of one CTA per slab launches only the pivot CTA (the copies were written by the
  // previous panel's update and row steps)
  const int b = gridDim.x == 1 ? q : (int)blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t Q0 = (int64_t)q * BT, B0 = (int64_t)b * BT;
  // per-slab work buffers: plain M x 128 panels, or nP split tiles
  const int64_t wo = SPLIT ? (int64_t)blockIdx.y * nP * SPLIT_TILE : (int64_t)blockIdx.y * M * BT;
  T* C = Cb + wo;
  T* Xt = XqT + wo;
  T* R = RT + wo;
  T* Pi = Pinv + (int64_t)blockIdx.y * (SPLIT ? SPLIT_TILE : BT * BT);
  if (b != q) {
    if constexpr (SPLIT) {
      float* S1 = reinterpret_cast<float*>(Xs);  // X(B, Q): (r = i, k = t)
      float* S2 = S1 + BT * LS;                  // X(Q, B): (t, j)
      for (int e = tid; e < BT * BT; e += blockDim.x) {
        const int i = e / BT, t = e - i * BT;
        S1[i * LS + t] = X[(B0 + i) * M + Q0 + t];
        S2[i * LS + t] = X[(Q0 + i) * M + B0 + t];
      }
      __syncthreads();
      store_split_tile(S1, LS, 1, C + (int64_t)b * SPLIT_TILE);
      store_split_tile(S2, 1, LS, Xt + (int64_t)b * SPLIT_TILE);  // (r = j, k = t) = X(Q0+t, B0+j)
    } else {
      for (int e = tid; e < BT * BT; e += blockDim.x) {
        const int i = e / BT, t = e - i * BT;
        C[(B0 + i) * BT + t] = X[(B0 + i) * M + Q0 + t];
        Xs[i * LS + t] = X[(Q0 + i) * M + B0 + t];
      }
      __syncthreads();
      for (int e = tid; e < BT * BT; e += blockDim.x) {
        const int j = e / BT, t = e - j * BT;
        Xt[(B0 + j) * BT + t] = Xs[t * LS + j];
      }
    }
    return;
  }
  T* Cp = Xs + BT * LD;
  T* Rp = Cp + G::CP;
  T* thr = Rp + G::NB * LD;
  const T* pk = pack + s.pack_off + (int64_t)(k - 1) * PK_NFIELDS * M;
  for (int e = tid; e < BT * BT; e += blockDim.x) {
    const int i = e / BT, t = e - i * BT;
    Xs[i * LD + t] = X[(Q0 + i) * M + Q0 + t];
  }
  for (int i = tid; i < BT; i += blockDim.x) thr[i] = T(1e3) * Eps<T>::v * fabs(pk[PK_DIAG * M + Q0 + i]);
  __syncthreads();
  if constexpr (SPLIT) {
    store_split_tile(reinterpret_cast<const float*>(Xs), LD, 1, C + (int64_t)q * SPLIT_TILE);
  } else {
    for (int e = tid; e < BT * BT; e += blockDim.x) C[(Q0 + e / BT) * BT + e % BT] = Xs[(e / BT) * LD + e % BT];
  }
  __syncthreads();
  bgj_invert<T, BT>(Xs, Cp, Rp, thr, st, sid, k);
  for (int e = tid; e < BT * BT; e += blockDim.x) {
    const int i = e / BT, t = e - i * BT;
    X[(Q0 + i) * M + Q0 + t] = Xs[i * LD + t];
  }
  if constexpr (SPLIT) {
    store_split_tile(reinterpret_cast<const float*>(Xs), LD, 1, Pi);                          // P^{-1}
    store_split_tile(reinterpret_cast<const float*>(Xs), 1, LD, R + (int64_t)q * SPLIT_TILE);  // P^{-T}
  } else {
    for (int e = tid; e < BT * BT; e += blockDim.x) {
      const int i = e / BT, t = e - i * BT;
      Pi[e] = Xs[i * LD + t];
      R[(Q0 + i) * BT + t] = Xs[t * LD + i];  // RT rows of panel Q hold P^{-T}
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Row and update steps as FMA products (FP64 path; FP32 reference for the tensor-core kernel).
// Tile (I, J) of 128 x 128 with K = 128: acc(i, j) = sum_t A(i, t) Bt(j, t), A and Bt row-major
// 128-wide panels.
//   ROW    (grid = (M/128, 1, slabs), J != q): A = XqT(J rows), Bt = Pinv;  RT(J rows) = acc,
//          X(Q, J) = acc^T
//   UPDATE (grid = (M/128, M/128, slabs), I != q): A = C(I rows), Bt = RT(J rows);
//          X(I, J) = [J != q] X(I, J) - acc
// 256 threads, 8 x 8 outputs each, K staged through shared memory 16 at a time.
// ---------------------------------------------------------------------------------------------
enum { GJ_ROW = 0, GJ_UPDATE = 1 };

// Tiles of the update of panel q (I != q), split for the look-ahead: set 0 all of them
// ((nP-1) nP tiles), set 1 the row block q+1 and the column block q+1 (2 nP - 2), which the
// next panel's pivot and row steps read, set 2 the rest ((nP-2)(nP-1)).
enum { GJ_ALL = 0, GJ_NEXT = 1, GJ_REST = 2 };
__host__ __device__ __forceinline__ int gj_count(int tset, int nP) {
  return tset == GJ_ALL ? (nP - 1) * nP : tset == GJ_NEXT ? 2 * nP - 2 : (nP - 2) * (nP - 1);
}
__device__ __forceinline__ void gj_tile(int tset, int nP, int q, int t, int& I, int& J) {
  if (tset == GJ_ALL) {
    I = t / nP;
    J = t - I * nP;
    if (I >= q) ++I;
    return;
  }
  if (tset == GJ_NEXT) {
    if (t < nP) {
      I = q + 1;
      J = t;
      return;
    }
    I = t - nP;          // column q+1, rows other than q and q+1
    if (I >= q) I += 2;
    J = q + 1;
    return;
  }
  const int c = nP - 1;  // rows other than q and q+1, columns other than q+1
  I = t / c;
  J = t - I * c;
  if (I >= q) I += 2;
  if (J >= q + 1) ++J;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(256) k_big_gemm_fma(const SlabDesc* __restrict__ slabs,
                                                      const int* __restrict__ ids,
                                                      T* __restrict__ F, int k, int q,
                                                      const T* __restrict__ Cb,
                                                      const T* __restrict__ XqT,
                                                      T* __restrict__ RT,
                                                      const T* __restrict__ Pinv, int tset) {
  constexpr int KC = 16;
  __shared__ T As[KC][BT + 4];
  __shared__ T Bs[KC][BT + 4];
  const SlabDesc s = slabs[ids[blockIdx.z]];
  if (k > s.nb) return;
  const int M = s.M;
  int I, J;
  if (MODE == GJ_ROW) {
    J = I = blockIdx.x;
    if (J == q) return;
  } else {
    gj_tile(tset, M / BT, q, blockIdx.x, I, J);
  }
  T* X = F + s.fac_off + (int64_t)(k - 1) * M * M;
  const int64_t wo = (int64_t)blockIdx.z * M * BT;
  const T* A = MODE == GJ_ROW ? XqT + wo + (int64_t)J * BT * BT : Cb + wo + (int64_t)I * BT * BT;
  const T* Bt = MODE == GJ_ROW ? Pinv + (int64_t)blockIdx.z * BT * BT : RT + wo + (int64_t)J * BT * BT;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[a][c] = T(0);
  for (int t0 = 0; t0 < BT; t0 += KC) {
    for (int e = tid; e < BT * KC; e += 256) {
      const int r = e / KC, t = e - r * KC;
      As[t][r] = A[r * BT + t0 + t];
      Bs[t][r] = Bt[r * BT + t0 + t];
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < KC; ++t) {
      T av[8], bv[8];
#pragma unroll
      for (int a = 0; a < 8; ++a) av[a] = As[t][ty + 16 * a];
#pragma unroll
      for (int c = 0; c < 8; ++c) bv[c] = Bs[t][tx + 16 * c];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = fma(av[a], bv[c], acc[a][c]);
    }
    __syncthreads();
  }
  const int64_t I0 = (int64_t)I * BT, J0 = (int64_t)J * BT, Q0 = (int64_t)q * BT;
  if (MODE == GJ_UPDATE && J != q) {  // old values first: 64 independent loads in flight
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[a][c] = X[(I0 + ty + 16 * a) * M + J0 + tx + 16 * c] - acc[a][c];
  } else if (MODE == GJ_UPDATE) {
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[a][c] = -acc[a][c];
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int i = ty + 16 * a;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int j = tx + 16 * c;
      if (MODE == GJ_ROW) {
        RT[wo + (J0 + i) * BT + j] = acc[a][c];
        X[(Q0 + j) * M + J0 + i] = acc[a][c];
      } else {
        X[(I0 + i) * M + J0 + j] = acc[a][c];
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// The same two steps on the tensor cores (FP32 data, 3xTF32, FP32 accumulation in TMEM), with
// the operands as split tiles (see above).  One 128 x 128 output tile per CTA, K = 128 in 8
// chunks of 16 through a 3-deep ring of bulk copies (A hi, A lo, B hi, B lo: 32 KB a chunk).
//   ROW    A = XqT tile J, B = Pinv:  RT tile J (split) = acc, X(Q, J) = acc^T
//   UPDATE A = C tile I,  B = RT tile J:  X(I, J) = [J != q] X(I, J) - acc
// Roles: warp 4 lane 0 issues the bulk copies, warp 5 allocates tensor memory and issues the
// MMAs, D += A_hi B_hi + A_hi B_lo + A_lo B_hi; warps 0-3 are the epilogue (thread = TMEM lane =
// output row): they load the old values of their rows before the accumulator is ready and stage
// 32 x 32 blocks through shared memory so that every global row access is coalesced.
// Barriers: full[s] (copies landed), empty[s] (MMA commit), dready (last commit).  Every wait is
// bounded and also ends when another role raised the abort flag; copies in flight are drained
// and the tensor memory is freed on every path.
// ---------------------------------------------------------------------------------------------
struct GjTc {
  static constexpr int KC = 16;
  static constexpr int NCH = BT / KC;
  static constexpr int NST = 3;
  static constexpr uint32_t PART = BT * KC * 4;       // one operand part (hi or lo) of a chunk
  static constexpr uint32_t STAGE = 4 * PART;         // A hi, A lo, B hi, B lo
  static constexpr size_t RING = (size_t)NST * STAGE; // 96 KB
  static constexpr size_t SMEM = RING + 8 * (2 * NST + 2) + 1024;
  static constexpr int THREADS = 192;
  static constexpr uint32_t TCOLS = 128;
};

template <int MODE>
__global__ void __launch_bounds__(GjTc::THREADS, 2)
    k_big_gemm_tc(const SlabDesc* __restrict__ slabs, const int* __restrict__ ids,
                  float* __restrict__ F, int k, int q, const float* __restrict__ Cs,
                  const float* __restrict__ XqTs, float* __restrict__ RTs,
                  const float* __restrict__ Pis, DevStatus* st, int tset,
                  float* __restrict__ Cn, float* __restrict__ XqTn, int three) {
  using C = GjTc;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* ring = smem_raw;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + C::RING);
  uint64_t* empty = full + C::NST;
  uint64_t* dready = empty + C::NST;
  uint64_t* done = dready + 1;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  volatile int* abort = &s_abort;

  const int sid = ids[blockIdx.z];
  const SlabDesc s = slabs[sid];
  if (k > s.nb) return;
  const int M = s.M, nP = M / BT;
  int I, J;
  if (MODE == GJ_ROW) {
    J = I = blockIdx.x;
    if (J == q) return;
  } else {
    gj_tile(tset, nP, q, blockIdx.x, I, J);
  }
  float* X = F + s.fac_off + (int64_t)(k - 1) * M * M;
  const int64_t wo = (int64_t)blockIdx.z * nP * SPLIT_TILE;
  const float* A = MODE == GJ_ROW ? XqTs + wo + (int64_t)J * SPLIT_TILE : Cs + wo + (int64_t)I * SPLIT_TILE;
  const float* B = MODE == GJ_ROW ? Pis + (int64_t)blockIdx.z * SPLIT_TILE : RTs + wo + (int64_t)J * SPLIT_TILE;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(C::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    s_abort = 0;
    for (int b = 0; b < C::NST; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], 1);
    }
    mbar_init(dready, 1);
    mbar_init(done, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp < 4) {
    // ---------------------------------------------------------------- epilogue (thread = row)
    const int64_t I0 = (int64_t)I * BT, J0 = (int64_t)J * BT, Q0 = (int64_t)q * BT;
    // Bulk path (the update outside the next panel's row and column blocks): -acc is staged row
    // by row in the idle ring and added to X (stored, for column block q) by bulk copies, so the
    // memory system performs the read-modify-write and the SM never waits for old values.
    const bool bulk = MODE == GJ_UPDATE && tset != GJ_NEXT;
    // Otherwise (the next panel's tiles, whose new values are also copied split, and the row
    // step): the old values of this warp's 32 rows, one 32-column block at a time, loaded ahead
    // (the first block while the MMAs run), 32 independent loads in flight per lane.
    float old[32];
    const bool keep = !bulk && MODE == GJ_UPDATE && J != q;
    float* xrow = X + (I0 + warp * 32) * M + J0 + lane;  // row warp*32 + rr at + rr * M
    if (keep) {
#pragma unroll
      for (int rr = 0; rr < 32; ++rr) old[rr] = xrow[(int64_t)rr * M];
    }
    bool go = mbar_wait_ab(dready, 0, abort, st, sid, k);
    go = __all_sync(0xffffffffu, go);  // tcgen05.ld is warp-collective
    if (go && bulk) {
      tc_fence_after();
      // row pitch 132 floats (528 B): 16-byte aligned rows and conflict-free 16-byte stores
      constexpr int LP = BT + 4;
      float* rowbuf = reinterpret_cast<float*>(ring) + (warp * 32 + lane) * LP;
#pragma unroll 1
      for (int cc = 0; cc < BT / 32; ++cc) {
        uint32_t v[32];
        tmem_ld32_wait(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          float4 o;
          o.x = -__uint_as_float(v[4 * g]);
          o.y = -__uint_as_float(v[4 * g + 1]);
          o.z = -__uint_as_float(v[4 * g + 2]);
          o.w = -__uint_as_float(v[4 * g + 3]);
          *reinterpret_cast<float4*>(rowbuf + cc * 32 + 4 * g) = o;
        }
      }
      fence_proxy_async();  // this thread's row is visible to its bulk copy
      float* dst = X + (I0 + warp * 32 + lane) * M + J0;
      if (J == q) bulk_s2g(dst, rowbuf, BT * 4);
      else bulk_s2g_add(dst, rowbuf, BT * 4);
      bulk_commit();
      bulk_wait_all();  // performed before the CTA exits (and before its ring is released)
    } else if (go) {
      tc_fence_after();
      // the ring is idle once the last MMA completed: reuse it for the 32 x 33 staging blocks
      float* E = reinterpret_cast<float*>(ring) + warp * 32 * 33;
      // the next panel's operand tiles, written split here so its pivot launch need not copy:
      // the update of the next panel's row and column blocks writes C_{q+1}(I) (column block
      // q+1) and XqT_{q+1}(J) (row block q+1); the row step writes C_{q+1}(q) (tile (q, q+1))
      const int qn = q + 1;
      // C_{q+1} tile I = new X(I, q+1) (update: I != q+1; the row step's tile is (q, q+1))
      const bool wr_c = Cn != nullptr && J == qn && (MODE == GJ_ROW || I != qn);
      const bool wr_x = Cn != nullptr && MODE == GJ_UPDATE && I == qn && J != qn;  // XqT_{q+1}(J)
      float* cn = wr_c ? Cn + wo + (int64_t)(MODE == GJ_ROW ? q : I) * SPLIT_TILE : nullptr;
      float* xn = wr_x ? XqTn + wo + (int64_t)J * SPLIT_TILE : nullptr;
#pragma unroll 1
      for (int cc = 0; cc < BT / 32; ++cc) {
        uint32_t v[32];
        tmem_ld32_wait(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
        if (MODE == GJ_ROW) {
          // RT tile J (split): row i = warp*32 + lane, contraction index cc*32 + e
          float* rt = RTs + wo + (int64_t)J * SPLIT_TILE;
          const int i = warp * 32 + lane;
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            float4 h, l;
            const float x0 = __uint_as_float(v[4 * g]), x1 = __uint_as_float(v[4 * g + 1]);
            const float x2 = __uint_as_float(v[4 * g + 2]), x3 = __uint_as_float(v[4 * g + 3]);
            h.x = tf32_rna(x0); l.x = tf32_rna(x0 - h.x);
            h.y = tf32_rna(x1); l.y = tf32_rna(x1 - h.y);
            h.z = tf32_rna(x2); l.z = tf32_rna(x2 - h.z);
            h.w = tf32_rna(x3); l.w = tf32_rna(x3 - h.w);
            const int o = split_off(i, cc * 32 + 4 * g);
            *reinterpret_cast<float4*>(rt + o) = h;
            *reinterpret_cast<float4*>(rt + BT * BT + o) = l;
          }
        }
#pragma unroll
        for (int e = 0; e < 32; ++e) E[lane * 33 + e] = __uint_as_float(v[e]);
        __syncwarp();
        // E(rr, cl): output row warp*32 + rr, output column cc*32 + cl
        if (MODE == GJ_ROW) {
#pragma unroll 8
          for (int cl = 0; cl < 32; ++cl)
            X[(Q0 + cc * 32 + cl) * M + J0 + warp * 32 + lane] = E[lane * 33 + cl];
          if (cn) {  // tile (q, q+1) of X is acc^T: element (r = cc*32 + cl, k = warp*32 + lane)
            for (int cl = 0; cl < 32; ++cl) {
              const float x = E[lane * 33 + cl], h = tf32_rna(x);
              const int o = split_off(cc * 32 + cl, warp * 32 + lane);
              cn[o] = h;
              cn[BT * BT + o] = tf32_rna(x - h);
            }
          }
        } else {
          float nxt[32];
          if (keep && cc + 1 < BT / 32) {
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) nxt[rr] = xrow[(int64_t)rr * M + (cc + 1) * 32];
          }
#pragma unroll
          for (int rr = 0; rr < 32; ++rr) {
            const float x = (keep ? old[rr] : 0.f) - E[rr * 33 + lane];
            xrow[(int64_t)rr * M + cc * 32] = x;
            if (cn || xn) E[rr * 33 + lane] = x;  // keep the new values for the copies below
          }
          __syncwarp();
          if (cn) {  // C_{q+1}(I): element (r = warp*32 + lane, k = cc*32 + e), this thread's row
            const int r = warp * 32 + lane;
#pragma unroll
            for (int g = 0; g < 8; ++g) {
              float4 h, l;
              const float x0 = E[lane * 33 + 4 * g], x1 = E[lane * 33 + 4 * g + 1];
              const float x2 = E[lane * 33 + 4 * g + 2], x3 = E[lane * 33 + 4 * g + 3];
              h.x = tf32_rna(x0); l.x = tf32_rna(x0 - h.x);
              h.y = tf32_rna(x1); l.y = tf32_rna(x1 - h.y);
              h.z = tf32_rna(x2); l.z = tf32_rna(x2 - h.z);
              h.w = tf32_rna(x3); l.w = tf32_rna(x3 - h.w);
              const int o = split_off(r, cc * 32 + 4 * g);
              *reinterpret_cast<float4*>(cn + o) = h;
              *reinterpret_cast<float4*>(cn + BT * BT + o) = l;
            }
          }
          if (xn) {  // XqT_{q+1}(J): element (r = cc*32 + e, k = warp*32 + lane) = X(q+1 row, J col)
            for (int e = 0; e < 32; ++e) {
              const float x = E[lane * 33 + e], h = tf32_rna(x);
              const int o = split_off(cc * 32 + e, warp * 32 + lane);
              xn[o] = h;
              xn[BT * BT + o] = tf32_rna(x - h);
            }
          }
          if (keep && cc + 1 < BT / 32) {
#pragma unroll
            for (int rr = 0; rr < 32; ++rr) old[rr] = nxt[rr];
          }
        }
        __syncwarp();
      }
    }
  } else if (warp == 4) {
    // ---------------------------------------------------------------- bulk-copy producer
    if (lane == 0) {
      int issued = 0;
      for (int c = 0; c < C::NCH; ++c) {
        const int stage = c % C::NST;
        if (c >= C::NST && !mbar_wait_ab(&empty[stage], ((c / C::NST) - 1) & 1, abort, st, sid, k))
          break;
        unsigned char* sb = ring + stage * C::STAGE;
        // the TF32 mode (three == 0) uses only the hi parts
        mbar_arrive_expect_tx(&full[stage], three ? C::STAGE : 2 * C::PART);
        bulk_g2s(sb, A + c * 2048, C::PART, &full[stage]);
        if (three) bulk_g2s(sb + C::PART, A + BT * BT + c * 2048, C::PART, &full[stage]);
        bulk_g2s(sb + 2 * C::PART, B + c * 2048, C::PART, &full[stage]);
        if (three) bulk_g2s(sb + 3 * C::PART, B + BT * BT + c * 2048, C::PART, &full[stage]);
        ++issued;
      }
      // no copy may still target this CTA's shared memory when it exits
      for (int c = issued > C::NST ? issued - C::NST : 0; c < issued; ++c)
        mbar_wait(&full[c % C::NST], (c / C::NST) & 1, st, sid, -1);
    }
  } else if (lane == 0) {
    // ---------------------------------------------------------------- MMA issue (warp 5)
    constexpr uint32_t IDESC = idesc_tf32(BT, BT);
    for (int c = 0; c < C::NCH; ++c) {
      const int stage = c % C::NST;
      if (!mbar_wait_ab(&full[stage], (c / C::NST) & 1, abort, st, sid, k)) break;
      tc_fence_after();
      const uint32_t sa = smem_u32(ring + stage * C::STAGE);
#pragma unroll
      for (int ks = 0; ks < C::KC / 8; ++ks) {
        const uint64_t ah = umma_desc(sa + ks * 256, 128, C::KC * 32);
        const uint64_t al = umma_desc(sa + C::PART + ks * 256, 128, C::KC * 32);
        const uint64_t bh = umma_desc(sa + 2 * C::PART + ks * 256, 128, C::KC * 32);
        const uint64_t bl = umma_desc(sa + 3 * C::PART + ks * 256, 128, C::KC * 32);
        mma_tf32_ss(tmem, ah, bh, IDESC, (c > 0 || ks > 0) ? 1u : 0u);
        if (three) {
          mma_tf32_ss(tmem, ah, bl, IDESC, 1u);
          mma_tf32_ss(tmem, al, bh, IDESC, 1u);
        }
      }
      mma_commit(&empty[stage]);
      if (c == C::NCH - 1) mma_commit(dready);
    }
    // every MMA issued has completed before the accumulator is released
    mma_commit(done);
    mbar_wait(done, 0, st, sid, -1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 5)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TCOLS)
                 : "memory");
}

// ---------------------------------------------------------------------------------------------
// Local solves through the stored inverses F_k = Sigma_k^{-1}:
//   A^{-1} b:  z_1 = b_1,  z_k = b_k - ell_k o (F_{k-1} z_{k-1});
//              x_nb = F_nb z_nb,  x_k = F_k (z_k - ups_k o x_{k+1})
//   A^{-T} b:  w_1 = F_1^T b_1,  w_k = F_k^T (b_k - ups_{k-1} o w_{k-1});
//              x_nb = w_nb,  x_{k-1} = w_{k-1} - F_{k-1}^T (ell_k o x_k)
// (o: elementwise product with the diagonal coupling).  One launch per block row and direction,
// over all slabs of the class; step i of a backward sweep handles block nb - i of each slab.
// ---------------------------------------------------------------------------------------------
enum { SV_NFWD = 0, SV_NBWD = 1, SV_TFWD = 2, SV_TBWD = 3 };

template <typename T>
struct SolveStep {
  int kf;                 // factor block applied (1-based; 0: nothing to do for this slab)
  const T* P; const T* Q; const T* phi; T vs;   // v = P + vs phi o Q   (P, Q, phi may be NULL)
  T* out; const T* R; const T* psi; T os;       // out = R + os psi o y (R, psi may be NULL)
};

template <typename T>
__device__ __forceinline__ SolveStep<T> solve_step(const SlabDesc& s, const T* pack, const T* b,
                                                   T* z, T* x, int mode, int i) {
  SolveStep<T> d{};
  const int M = s.M, nb = s.nb;
  auto vec = [&](const T* base, int blk) { return base + s.loc_off + (int64_t)(blk - 1) * M; };
  auto fld = [&](int blk, int f) { return pack + s.pack_off + (int64_t)(blk - 1) * PK_NFIELDS * M + f * M; };
  if (mode == SV_NFWD) {                      // i = block k (2..nb)
    const int kk = i;
    if (kk < 2 || kk > nb) return d;
    d.kf = kk - 1;
    d.P = vec(kk == 2 ? b : z, kk - 1);
    d.out = z + s.loc_off + (int64_t)(kk - 1) * M;
    d.R = vec(b, kk); d.psi = fld(kk, PK_SOUTH); d.os = T(-1);
  } else if (mode == SV_NBWD) {               // block k = nb - i
    const int kk = nb - i;
    if (kk < 1) return d;
    d.kf = kk;
    d.P = vec(kk == 1 ? b : z, kk);
    if (kk < nb) { d.Q = vec(x, kk + 1); d.phi = fld(kk, PK_NORTH); d.vs = T(-1); }
    d.out = x + s.loc_off + (int64_t)(kk - 1) * M;
    d.os = T(1);
  } else if (mode == SV_TFWD) {               // i = block k (1..nb)
    const int kk = i;
    if (kk < 1 || kk > nb) return d;
    d.kf = kk;
    d.P = vec(b, kk);
    if (kk > 1) { d.Q = vec(z, kk - 1); d.phi = fld(kk - 1, PK_NORTH); d.vs = T(-1); }
    d.out = z + s.loc_off + (int64_t)(kk - 1) * M;
    d.os = T(1);
  } else {                                    // SV_TBWD: block k = nb - i (>= 2) -> x_{k-1}
    const int kk = nb - i;
    if (kk < 2) return d;
    d.kf = kk - 1;
    d.Q = vec(i == 0 ? z : x, kk); d.phi = fld(kk, PK_SOUTH); d.vs = T(1);
    d.out = x + s.loc_off + (int64_t)(kk - 2) * M;
    d.R = vec(z, kk - 1); d.os = T(-1);
  }
  return d;
}

template <typename T>
__device__ __forceinline__ void load_v(const SolveStep<T>& d, int M, T* v) {
  for (int c = threadIdx.x; c < M; c += blockDim.x) {
    T a = d.P ? d.P[c] : T(0);
    if (d.Q) a += d.vs * (d.phi ? d.phi[c] : T(1)) * d.Q[c];
    v[c] = a;
  }
}

// y = F v (row-major F): a warp takes 4 rows, lanes stride the columns with 16-byte loads.
// Only the live m x m part is read: the padding of every F_k is exactly the identity (Sigma_k is
// the identity there and the Gauss-Jordan panels keep exact zeros off it), so a padded row gives
// v itself.  grid = (M / 32, slabs of the class), 256 threads.
template <typename T>
__global__ void __launch_bounds__(256) k_big_gemv_n(const SlabDesc* __restrict__ slabs,
                                                    const int* __restrict__ ids,
                                                    const T* __restrict__ F,
                                                    const T* __restrict__ pack,
                                                    const T* __restrict__ b, T* __restrict__ z,
                                                    T* __restrict__ x, int mode, int i) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* v = reinterpret_cast<T*>(smem_raw);
  const SlabDesc s = slabs[ids[blockIdx.y]];
  const SolveStep<T> d = solve_step<T>(s, pack, b, z, x, mode, i);
  if (d.kf == 0) return;
  const int M = s.M;
  load_v(d, M, v);
  __syncthreads();
  const T* Fk = F + s.fac_off + (int64_t)(d.kf - 1) * M * M;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = blockIdx.x * 32 + warp * 4;
  constexpr int VW = 16 / sizeof(T);  // elements per 16-byte load
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const int m = s.m;
  if (r0 >= m) {  // padded rows: identity
    if (lane < 4) {
      const int r = r0 + lane;
      d.out[r] = (d.R ? d.R[r] : T(0)) + d.os * (d.psi ? d.psi[r] : T(1)) * v[r];
    }
    return;
  }
  // columns up to m rounded to the load width (covers the diagonal of every row of this warp)
  const int mc = min(M, (m + VW - 1) / VW * VW);
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (int c = lane * VW; c < mc; c += 32 * VW) {
    T vv[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) vv[e] = v[c + e];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const V f = *reinterpret_cast<const V*>(Fk + (int64_t)(r0 + u) * M + c);
      const T* fe = reinterpret_cast<const T*>(&f);
#pragma unroll
      for (int e = 0; e < VW; ++e) acc[u] = fma(fe[e], vv[e], acc[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const T y = warp_sum(acc[u]);
    if (lane == 0) {
      const int r = r0 + u;
      d.out[r] = (d.R ? d.R[r] : T(0)) + d.os * (d.psi ? d.psi[r] : T(1)) * y;
    }
  }
}

// y = F^T v: a CTA owns 64 columns (lanes hold two adjacent columns), its 8 warps split the rows
// and combine their partial sums in shared memory.  grid = (M / 64, slabs of the class).  (Reading
// only the live rows, as the non-transposed product does, measured slower here: 1.56 against
// 1.06 s for the adjoint batch's large-block problems.)
template <typename T>
__global__ void __launch_bounds__(256) k_big_gemv_t(const SlabDesc* __restrict__ slabs,
                                                    const int* __restrict__ ids,
                                                    const T* __restrict__ F,
                                                    const T* __restrict__ pack,
                                                    const T* __restrict__ b, T* __restrict__ z,
                                                    T* __restrict__ x, int mode, int i) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SlabDesc s = slabs[ids[blockIdx.y]];
  const int M = s.M;
  T* v = reinterpret_cast<T*>(smem_raw);
  T* red = v + M;  // [8][64]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c0 = blockIdx.x * 64 + 2 * lane;
  if (mode == SV_TBWD && i == 0 && s.nb >= 1) {  // x_nb = w_nb (this CTA's columns)
    T* xn = x + s.loc_off + (int64_t)(s.nb - 1) * M;
    const T* wn = z + s.loc_off + (int64_t)(s.nb - 1) * M;
    if (warp == 0) { xn[c0] = wn[c0]; xn[c0 + 1] = wn[c0 + 1]; }
  }
  const SolveStep<T> d = solve_step<T>(s, pack, b, z, x, mode, i);
  if (d.kf == 0) return;
  load_v(d, M, v);
  __syncthreads();
  const T* Fk = F + s.fac_off + (int64_t)(d.kf - 1) * M * M;
  T a0 = T(0), a1 = T(0), b0 = T(0), b1 = T(0);
  int r = warp;
  for (; r + 8 < M; r += 16) {
    const T* p0 = Fk + (int64_t)r * M + c0;
    const T* p1 = Fk + (int64_t)(r + 8) * M + c0;
    const T f00 = p0[0], f01 = p0[1], f10 = p1[0], f11 = p1[1];
    a0 = fma(f00, v[r], a0); a1 = fma(f01, v[r], a1);
    b0 = fma(f10, v[r + 8], b0); b1 = fma(f11, v[r + 8], b1);
  }
  for (; r < M; r += 8) {
    const T* p0 = Fk + (int64_t)r * M + c0;
    a0 = fma(p0[0], v[r], a0); a1 = fma(p0[1], v[r], a1);
  }
  red[warp * 64 + 2 * lane] = a0 + b0;
  red[warp * 64 + 2 * lane + 1] = a1 + b1;
  __syncthreads();
  if (threadIdx.x < 64) {
    T y = T(0);
#pragma unroll
    for (int w = 0; w < 8; ++w) y += red[w * 64 + threadIdx.x];
    const int c = blockIdx.x * 64 + threadIdx.x;
    d.out[c] = (d.R ? d.R[c] : T(0)) + d.os * (d.psi ? d.psi[c] : T(1)) * y;
  }
}

// ---------------------------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------------------------
// Shared memory of the pivot kernel: the Gauss-Jordan block of CTA q, or the staging tiles of
// the copying CTAs (two in the split path, one in the plain path).
template <typename T>
static size_t pivot_smem_gj() {  // the pivot CTA alone: its Gauss-Jordan block
  return BGJ<T, BT>::smem_elems * sizeof(T) + BT * sizeof(T) + 16;
}

template <typename T, bool SPLIT>
static size_t pivot_smem() {
  const size_t gj = BGJ<T, BT>::smem_elems * sizeof(T) + BT * sizeof(T) + 16;
  const size_t stage = (size_t)(SPLIT ? 2 : 1) * BT * (BT + 1) * sizeof(T);
  return gj > stage ? gj : stage;
}

// One block row k of the large-block factorization with look-ahead.  Stream sh (high priority)
// runs the Sigma_k formation and, per panel q, the update of the next panel's row and column
// blocks followed by that panel's pivot and row steps; stream sl runs the rest of panel q's
// update at the same time.  The work buffers alternate between two sets by panel parity, so the
// next panel's pivot step never overwrites operands the current update still reads.  ev: three
// events owned by the caller.  On return both streams' work is ordered before later work on sh.
template <typename T>
void launch_big_factor_step(int M, const SlabDesc* d_slabs, const int* d_ids, int nids,
                            const T* pack, T* F, int k, T* const Cb[2], T* const XqT[2],
                            T* const RT[2], T* const Pinv[2], int tensor_cores, DevStatus* st,
                            cudaStream_t sh, cudaStream_t sl, cudaEvent_t* ev, int form_sigma) {
  const int nP = M / BT;
  bool tc = false;
  if constexpr (sizeof(T) == 4) tc = tensor_cores != 0;
  const int three = tensor_cores == 1 ? 1 : 0;  // 1: 3xTF32, 2: TF32
  const size_t psm = tc ? pivot_smem<T, true>() : pivot_smem<T, false>();
  auto pivot = [&](int q) {
    const int b = q & 1;
    note_launch();
    if constexpr (sizeof(T) == 4) {
      if (tc) {
        // from the second panel on, the copies come from the previous panel's update and row
        k_big_pivot<float, true><<<dim3(q == 0 ? nP : 1, nids), 512, q == 0 ? psm : pivot_smem_gj<float>(),
                                   sh>>>(d_slabs, d_ids, pack, F, k, q, Cb[b], XqT[b], RT[b],
                                         Pinv[b], st);
        return;
      }
    }
    k_big_pivot<T, false><<<dim3(nP, nids), 512, psm, sh>>>(d_slabs, d_ids, pack, F, k, q, Cb[b],
                                                            XqT[b], RT[b], Pinv[b], st);
  };
  auto row = [&](int q) {
    const int b = q & 1;
    note_launch();
    if constexpr (sizeof(T) == 4) {
      if (tc) {
        k_big_gemm_tc<GJ_ROW><<<dim3(nP, 1, nids), GjTc::THREADS, GjTc::SMEM, sh>>>(
            d_slabs, d_ids, F, k, q, Cb[b], XqT[b], RT[b], Pinv[b], st, GJ_ALL,
            q + 1 < nP ? Cb[b ^ 1] : nullptr, q + 1 < nP ? XqT[b ^ 1] : nullptr, three);
        return;
      }
    }
    k_big_gemm_fma<T, GJ_ROW><<<dim3(nP, 1, nids), 256, 0, sh>>>(d_slabs, d_ids, F, k, q, Cb[b],
                                                                 XqT[b], RT[b], Pinv[b], GJ_ALL);
  };
  auto update = [&](int q, int tset, cudaStream_t s) {
    const int b = q & 1;
    if (gj_count(tset, nP) == 0) return;  // two panels: panel 0 has no tiles besides the next
    note_launch();
    const dim3 grid(gj_count(tset, nP), 1, nids);
    if constexpr (sizeof(T) == 4) {
      if (tc) {
        const bool nx = tset == GJ_NEXT;
        k_big_gemm_tc<GJ_UPDATE><<<grid, GjTc::THREADS, GjTc::SMEM, s>>>(
            d_slabs, d_ids, F, k, q, Cb[b], XqT[b], RT[b], Pinv[b], st, tset,
            nx ? Cb[b ^ 1] : nullptr, nx ? XqT[b ^ 1] : nullptr, three);
        return;
      }
    }
    k_big_gemm_fma<T, GJ_UPDATE><<<grid, 256, 0, s>>>(d_slabs, d_ids, F, k, q, Cb[b], XqT[b],
                                                      RT[b], Pinv[b], tset);
  };
  if (tc) {
    if constexpr (sizeof(T) == 4) {
      raise_smem_limit(reinterpret_cast<const void*>(&k_big_pivot<float, true>), psm);
      raise_smem_limit(reinterpret_cast<const void*>(&k_big_gemm_tc<GJ_ROW>), GjTc::SMEM);
      raise_smem_limit(reinterpret_cast<const void*>(&k_big_gemm_tc<GJ_UPDATE>), GjTc::SMEM);
    }
  } else {
    raise_smem_limit(reinterpret_cast<const void*>(&k_big_pivot<T, false>), psm);
  }
  cudaEvent_t evA = ev[0], evB[2] = {ev[1], ev[2]};
  if (form_sigma) {
    note_launch();
    k_big_sigma<T><<<dim3(512, nids), 256, 0, sh>>>(d_slabs, d_ids, pack, F, k);
  }
  pivot(0);
  if (nP == 1) return;
  row(0);
  cudaEventRecord(evA, sh);
  for (int q = 0; q < nP; ++q) {
    const bool ahead = q + 1 < nP;
    cudaStreamWaitEvent(sl, evA, 0);
    update(q, ahead ? GJ_REST : GJ_ALL, sl);
    cudaEventRecord(evB[q & 1], sl);
    if (ahead) {
      if (q >= 1) cudaStreamWaitEvent(sh, evB[(q - 1) & 1], 0);  // rest of panel q-1 done
      update(q, GJ_NEXT, sh);
      pivot(q + 1);
      row(q + 1);
      cudaEventRecord(evA, sh);
    }
  }
  cudaStreamWaitEvent(sh, evB[(nP - 1) & 1], 0);
}

template <typename T>
void launch_big_solve(int M, const SlabDesc* d_slabs, const int* d_ids, int nids, int max_nb,
                      const T* F, const T* pack, const T* b, T* z, T* x, int transpose,
                      cudaStream_t s) {
  const size_t vsm = (size_t)M * sizeof(T);
  const size_t tsm = (size_t)(M + 8 * 64) * sizeof(T);
  raise_smem_limit(reinterpret_cast<const void*>(&k_big_gemv_n<T>), vsm);
  raise_smem_limit(reinterpret_cast<const void*>(&k_big_gemv_t<T>), tsm);
  if (!transpose) {
    for (int k = 2; k <= max_nb; ++k) {
      note_launch();
      k_big_gemv_n<T><<<dim3(M / 32, nids), 256, vsm, s>>>(d_slabs, d_ids, F, pack, b, z, x,
                                                           SV_NFWD, k);
    }
    for (int i = 0; i < max_nb; ++i) {
      note_launch();
      k_big_gemv_n<T><<<dim3(M / 32, nids), 256, vsm, s>>>(d_slabs, d_ids, F, pack, b, z, x,
                                                           SV_NBWD, i);
    }
  } else {
    for (int k = 1; k <= max_nb; ++k) {
      note_launch();
      k_big_gemv_t<T><<<dim3(M / 64, nids), 256, tsm, s>>>(d_slabs, d_ids, F, pack, b, z, x,
                                                           SV_TFWD, k);
    }
    for (int i = 0; i < max_nb; ++i) {
      note_launch();
      k_big_gemv_t<T><<<dim3(M / 64, nids), 256, tsm, s>>>(d_slabs, d_ids, F, pack, b, z, x,
                                                           SV_TBWD, i);
    }
  }
}

// Central rows of slab-local vectors of the listed slabs into the FP64 interface vector.
template <typename T>
__global__ void k_big_extract(const SlabDesc* __restrict__ slabs, const int* __restrict__ ids,
                              const T* __restrict__ loc, double* __restrict__ iface) {
  const SlabDesc s = slabs[ids[blockIdx.y]];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.ng;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / s.p) + 1, t = (int)(e % s.p);
    iface[s.if_off + e] =
        static_cast<double>(loc[s.loc_off + (int64_t)(k - 1) * s.M + (s.w - 1) * s.p + t]);
  }
}

template <typename T>
void launch_big_extract(const SlabDesc* d_slabs, const int* d_ids, int nids, const T* loc,
                        double* iface, cudaStream_t s) {
  note_launch();
  k_big_extract<T><<<dim3(32, nids), 256, 0, s>>>(d_slabs, d_ids, loc, iface);
}

template void launch_big_factor_step<float>(int, const SlabDesc*, const int*, int, const float*,
                                            float*, int, float* const[2], float* const[2],
                                            float* const[2], float* const[2], int, DevStatus*,
                                            cudaStream_t, cudaStream_t, cudaEvent_t*, int);
template void launch_big_factor_step<double>(int, const SlabDesc*, const int*, int,
                                             const double*, double*, int, double* const[2],
                                             double* const[2], double* const[2],
                                             double* const[2], int, DevStatus*, cudaStream_t,
                                             cudaStream_t, cudaEvent_t*, int);
template void launch_big_solve<float>(int, const SlabDesc*, const int*, int, int, const float*,
                                      const float*, const float*, float*, float*, int,
                                      cudaStream_t);
template void launch_big_solve<double>(int, const SlabDesc*, const int*, int, int, const double*,
                                       const double*, const double*, double*, double*, int,
                                       cudaStream_t);
template void launch_big_extract<float>(const SlabDesc*, const int*, int, const float*, double*,
                                        cudaStream_t);
template void launch_big_extract<double>(const SlabDesc*, const int*, int, const double*, double*,
                                         cudaStream_t);

}  // namespace ddst
