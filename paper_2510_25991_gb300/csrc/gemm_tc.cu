// gemm_tc.cu -- batched dense products of square blocks for the direct interface solver.
//
// The block cyclic reduction of the equilibrium system (Sec. 1, Eq. (modelS); the direct
// solvers of Sec. 4) eliminates half of the interface blocks per level; every elimination is a
// handful of products C = alpha A B (+ C) of dense n_Gamma x n_Gamma blocks (padded to a
// multiple of 128).  FP32 blocks run on the tcgen05 tensor cores: the operands are first packed
// into pre-split 128 x 128 TF32 tiles (the layout of splittile.cuh), so the product kernel only
// issues bulk copies and MMAs; the accumulator lives in tensor memory and leaves through bulk
// stores or bulk reduce-adds of staged rows.  FP64 blocks (and an FP32 reference) use FMA.
#include "kernels.cuh"
#include "splittile.cuh"
#include "umma.cuh"

namespace ddst {

// ---------------------------------------------------------------------------------------------
// Packing.  grid = (nT * nT source tiles, tasks), 256 threads.  trans = 0 (an A operand): tile
// (I, kt) of the packed matrix holds element (r, k) = src(128 I + r, 128 kt + k); trans = 1 (a B
// operand, packed as B^T): tile (J, kt) holds (r, k) = src(128 kt + k, 128 J + r).  Tiles of
// one row I (or J) are consecutive in kt.
// ---------------------------------------------------------------------------------------------
constexpr int PK_LS = BT + 1;
constexpr size_t PACK_SMEM = sizeof(float) * BT * PK_LS;

__global__ void __launch_bounds__(256) k_pack_split(const PackTask* __restrict__ tasks, int nT) {
  extern __shared__ float S[];
  const PackTask t = tasks[blockIdx.y];
  const int ti = blockIdx.x / nT, tj = blockIdx.x - ti * nT;
  const int64_t ld = (int64_t)nT * BT;
  const float* src = t.src + (int64_t)ti * BT * ld + (int64_t)tj * BT;
  for (int e = threadIdx.x; e < BT * (BT / 4); e += blockDim.x) {
    const int i = e / (BT / 4), c = 4 * (e - i * (BT / 4));
    const float4 v = *reinterpret_cast<const float4*>(src + i * ld + c);
    float* d = S + i * PK_LS + c;
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
  }
  __syncthreads();
  if (!t.trans) store_split_tile(S, PK_LS, 1, t.dst + ((int64_t)ti * nT + tj) * SPLIT_TILE);
  else store_split_tile(S, 1, PK_LS, t.dst + ((int64_t)tj * nT + ti) * SPLIT_TILE);
}

// ---------------------------------------------------------------------------------------------
// C = alpha A B (accumulate = 0) or C += alpha A B (accumulate = 1), C row-major with leading
// dimension 128 nT.  grid = (nT * nT output tiles, tasks); one 128 x 128 tile per CTA, K = 128 nT
// streamed in 16-wide chunks through a 3-stage ring of bulk copies (A hi/lo, B hi/lo), three
// MMAs per chunk (3xTF32: hi hi + hi lo + lo hi) or one (three = 0, TF32).  Warps 0-3: epilogue
// (thread = output row); warp 4: copies; warp 5: TMEM and MMAs.  Waits are bounded; copies in
// flight are drained and the tensor memory freed on every path.
// ---------------------------------------------------------------------------------------------
struct GmTc {
  static constexpr int KC = 16;
  static constexpr int NST = 3;
  static constexpr uint32_t PART = BT * KC * 4;
  static constexpr uint32_t STAGE = 4 * PART;
  static constexpr size_t RING = (size_t)NST * STAGE;  // 96 KB; the epilogue stages rows here
  static constexpr size_t SMEM = RING + 8 * (2 * NST + 2) + 1024;
  static constexpr int THREADS = 192;
  static constexpr uint32_t TCOLS = 128;
};

__global__ void __launch_bounds__(GmTc::THREADS, 2)
    k_gemm_tc(const GemmTask* __restrict__ tasks, int nT, DevStatus* st, int three) {
  using C = GmTc;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* ring = smem_raw;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + C::RING);
  uint64_t* empty = full + C::NST;
  uint64_t* dready = empty + C::NST;
  uint64_t* done = dready + 1;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  volatile int* abort = &s_abort;

  const int task = blockIdx.y;
  const GemmTask t = tasks[task];
  const int I = blockIdx.x / nT, J = blockIdx.x - I * nT;
  const int nch = nT * (BT / C::KC);
  const float* A = t.A + (int64_t)I * nT * SPLIT_TILE;
  const float* B = t.B + (int64_t)J * nT * SPLIT_TILE;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int kTag = -3;  // block field of a timeout record from this kernel

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
    bool go = mbar_wait_ab(dready, 0, abort, st, task, kTag);
    go = __all_sync(0xffffffffu, go);  // tcgen05.ld is warp-collective
    if (go) {
      tc_fence_after();
      constexpr int LP = BT + 4;  // 528-byte rows: 16-byte aligned, conflict-free stores
      float* rowbuf = reinterpret_cast<float*>(ring) + (warp * 32 + lane) * LP;
#pragma unroll 1
      for (int cc = 0; cc < BT / 32; ++cc) {
        uint32_t v[32];
        tmem_ld32_wait(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), v);
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          float4 o;
          o.x = t.alpha * __uint_as_float(v[4 * g]);
          o.y = t.alpha * __uint_as_float(v[4 * g + 1]);
          o.z = t.alpha * __uint_as_float(v[4 * g + 2]);
          o.w = t.alpha * __uint_as_float(v[4 * g + 3]);
          *reinterpret_cast<float4*>(rowbuf + cc * 32 + 4 * g) = o;
        }
      }
      fence_proxy_async();
      float* dst = t.C + ((int64_t)I * BT + warp * 32 + lane) * ((int64_t)nT * BT) + (int64_t)J * BT;
      if (t.accumulate) bulk_s2g_add(dst, rowbuf, BT * 4);
      else bulk_s2g(dst, rowbuf, BT * 4);
      bulk_commit();
      bulk_wait_all();
    }
  } else if (warp == 4) {
    // ---------------------------------------------------------------- bulk-copy producer
    if (lane == 0) {
      int issued = 0;
      for (int c = 0; c < nch; ++c) {
        const int stage = c % C::NST;
        if (c >= C::NST &&
            !mbar_wait_ab(&empty[stage], ((c / C::NST) - 1) & 1, abort, st, task, kTag))
          break;
        unsigned char* sb = ring + stage * C::STAGE;
        const int64_t off = (int64_t)(c >> 3) * SPLIT_TILE + (c & 7) * 2048;
        mbar_arrive_expect_tx(&full[stage], three ? C::STAGE : 2 * C::PART);
        bulk_g2s(sb, A + off, C::PART, &full[stage]);
        if (three) bulk_g2s(sb + C::PART, A + off + BT * BT, C::PART, &full[stage]);
        bulk_g2s(sb + 2 * C::PART, B + off, C::PART, &full[stage]);
        if (three) bulk_g2s(sb + 3 * C::PART, B + off + BT * BT, C::PART, &full[stage]);
        ++issued;
      }
      for (int c = issued > C::NST ? issued - C::NST : 0; c < issued; ++c)
        mbar_wait(&full[c % C::NST], (c / C::NST) & 1, st, task, -1);
    }
  } else if (lane == 0) {
    // ---------------------------------------------------------------- MMA issue (warp 5)
    constexpr uint32_t IDESC = idesc_tf32(BT, BT);
    for (int c = 0; c < nch; ++c) {
      const int stage = c % C::NST;
      if (!mbar_wait_ab(&full[stage], (c / C::NST) & 1, abort, st, task, kTag)) break;
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
      if (c == nch - 1) mma_commit(dready);
    }
    mma_commit(done);
    mbar_wait(done, 0, st, task, -1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 5)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TCOLS)
                 : "memory");
}

// ---------------------------------------------------------------------------------------------
// FMA product on plain row-major blocks (FP64 path; FP32 reference for the tensor-core kernel):
// C = alpha A B (+ C).  grid = (nT * nT tiles, tasks), 256 threads, 8 x 8 outputs per thread, K
// staged through shared memory 16 at a time.
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_fma(const GemmTaskT<T>* __restrict__ tasks, int nT) {
  constexpr int KC = 16;
  __shared__ T As[KC][BT + 4];
  __shared__ T Bs[KC][BT + 4];
  const GemmTaskT<T> t = tasks[blockIdx.y];
  const int I = blockIdx.x / nT, J = blockIdx.x - I * nT;
  const int64_t ld = (int64_t)nT * BT;
  const T* A = t.A + (int64_t)I * BT * ld;
  const T* B = t.B + (int64_t)J * BT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[8][8] = {};
  for (int k0 = 0; k0 < ld; k0 += KC) {
    for (int e = threadIdx.x; e < KC * BT; e += blockDim.x) {
      const int r = e / KC, kk = e - r * KC;  // A(r, k0 + kk)
      As[kk][r] = A[r * ld + k0 + kk];
      const int kb = e / BT, c = e - kb * BT;  // B(k0 + kb, c)
      Bs[kb][c] = B[(k0 + kb) * ld + c];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      T a[8], b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[kk][ty * 8 + i];
#pragma unroll
      for (int j = 0; j < 8; ++j) b[j] = Bs[kk][tx * 8 + j];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  T* Cp = t.C + ((int64_t)I * BT + ty * 8) * ld + (int64_t)J * BT + tx * 8;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      T* c = Cp + (int64_t)i * ld + j;
      *c = t.alpha * acc[i][j] + (t.accumulate ? *c : T(0));
    }
}

void launch_pack_split(const PackTask* d_tasks, int ntasks, int nT, cudaStream_t st) {
  if (ntasks <= 0) return;
  raise_smem_limit(reinterpret_cast<const void*>(&k_pack_split), PACK_SMEM);
  note_launch();
  k_pack_split<<<dim3(nT * nT, ntasks), 256, PACK_SMEM, st>>>(d_tasks, nT);
}

void launch_gemm_tc(const GemmTask* d_tasks, int ntasks, int nT, int three, DevStatus* dst,
                    cudaStream_t st) {
  if (ntasks <= 0) return;
  raise_smem_limit(reinterpret_cast<const void*>(&k_gemm_tc), GmTc::SMEM);
  note_launch();
  k_gemm_tc<<<dim3(nT * nT, ntasks), GmTc::THREADS, GmTc::SMEM, st>>>(d_tasks, nT, dst, three);
}

template <typename T>
void launch_gemm_fma(const GemmTaskT<T>* d_tasks, int ntasks, int nT, cudaStream_t st) {
  if (ntasks <= 0) return;
  note_launch();
  k_gemm_fma<T><<<dim3(nT * nT, ntasks), 256, 0, st>>>(d_tasks, nT);
}

template void launch_gemm_fma<float>(const GemmTaskT<float>*, int, int, cudaStream_t);
template void launch_gemm_fma<double>(const GemmTaskT<double>*, int, int, cudaStream_t);

}  // namespace ddst
