// common.cuh -- shared device-side definitions of the GB300 DD library.
//
// Geometry (slabs normal to x, blocks ordered along y):
//   double slab j (1-based) of a problem with n cells and slab width w holds the interior
//   x-planes i = (j-1)w+1 .. (j+1)w-1.  It is ordered as nb = n-1 blocks along y; block k
//   (1-based) holds the local unknowns c = cx * p + t, cx = 0..2w-2 (x offset), t = 0..p-1
//   (z index - 1 in 3D, p = n-1; p = 1 in 2D).  m = (2w-1) p; blocks are padded to M >= m
//   with identity rows/columns.  Global interior index of (cx, k, t):
//   ((i-1)(n-1) + (k-1)) p + t with i = (j-1)w+1+cx.
//   The interface Gamma_j is the plane cx = w-1; its index (k, t) -> (k-1) p + t.
//
// The block-tridiagonal local operator A_j(I_j, I_j) (Sec. 2.2, Eq. (defS); Alg. 2) has
// diagonal blocks D_k and diagonal couplings L_k = diag(ell_k) (to block k-1) and
// U_k = diag(ups_k) (to block k+1).
#pragma once
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace ddst {

// Process-wide count of kernels launched by the library (reported by ddst_kernel_launches).
std::atomic<long long>& launch_counter();
inline void note_launch(int n = 1) { launch_counter().fetch_add(n, std::memory_order_relaxed); }
// Raises the dynamic shared-memory limit of kernel `func` on the current device to at least
// `bytes` (never lowers it; nothing to do up to the 48 KiB default).  Thread-safe: one limit
// per (device, kernel), kept under a lock, so a smaller request on another thread cannot undo
// a larger one.  Returns the error of the attribute call (cudaSuccess when none was needed).
cudaError_t raise_smem_limit(const void* func, size_t bytes);

// Stencil pack fields, stored per (slab, block) as [field][M] in the working precision.
enum PackField { PK_DIAG = 0, PK_WEST = 1, PK_EAST = 2, PK_SOUTH = 3, PK_NORTH = 4,
                 PK_ZLO = 5, PK_ZHI = 6, PK_NFIELDS = 7 };

struct ProbDesc {
  int dim;
  int n;            // cells per side
  int w;            // slab width (cells)
  int nds;          // number of double slabs = n/w - 1
  int p;            // (n-1)^(dim-2)
  int m;            // (2w-1) p
  int M;            // padded block size
  int nb;           // n - 1
  int64_t ng;       // interface size nb * p
  int64_t nint;     // interior unknowns (n-1)^dim
  int64_t nnode;    // nodes (n+1)^dim
  int64_t vol_off;  // offset of this problem in concatenated interior vectors
  int64_t node_off; // offset in concatenated nodal vectors
  int64_t if_off;   // offset in concatenated interface vectors
  int slab0;        // index of the problem's first slab in the global slab list
  int has_c;
  double h;
  double b[3];
};

struct SlabDesc {
  int prob;         // problem index
  int j;            // 1-based slab index within the problem
  int M;            // padded block size
  int m;
  int nb;
  int p;
  int w;
  int n;
  int64_t ng;
  int64_t fac_off;  // element offset of this slab's [nb][M][M] blocks (F, B, G arrays)
  int64_t pack_off; // element offset of [nb][PK_NFIELDS][M]
  int64_t loc_off;  // element offset of slab-local vectors [nb][M]
  int64_t sp_off;   // element offset of dense S_{j,j-1} (column-major ng x ng), -1 if none
  int64_t sn_off;   // element offset of dense S_{j,j+1}, -1 if none
  int64_t vol_off;  // problem's interior-vector offset
  int64_t node_off; // problem's nodal-vector offset
  int64_t if_off;   // offset of Gamma_j in the concatenated interface vector
};

// Device-side status written by kernels (first error wins).
struct DevStatus {
  int code;   // 0 ok, else a ddst_status value
  int slab;
  int block;
  int aux;
};

enum { ST_SINGULAR = 4, ST_TIMEOUT = 6 };

__device__ __forceinline__ void set_status(DevStatus* st, int code, int slab, int block) {
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->slab = slab;
    st->block = block;
  }
}

template <typename T> struct Eps;
template <> struct Eps<float> { static constexpr float v = 1.1920929e-07f; };
template <> struct Eps<double> { static constexpr double v = 2.220446049250313e-16; };

// ---------------------------------------------------------------------------------------
// Warp reductions
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------------------
// mbarrier + bulk-copy (TMA, untiled) helpers.  Every wait is bounded: after ~2 s of
// clock64 cycles the waiting thread reports ST_TIMEOUT and gives up.
// ---------------------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start before the kernel ahead of it in the stream has finished; pdl_wait() returns once that
// kernel has completed and its memory operations are visible (immediately for a plain launch),
// and pdl_release() lets the kernel behind this one be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Bulk global -> shared copy completing on an mbarrier.  dst/src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false (and records ST_TIMEOUT) if the phase never completes.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, DevStatus* st,
                                          int slab, int block) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > 4000000000LL) {
      set_status(st, ST_TIMEOUT, slab, block);
      return false;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Index helpers
// ---------------------------------------------------------------------------------------
// Global interior index of slab-local unknown (cx, k, t) of slab j.
__device__ __forceinline__ int64_t vol_index(const SlabDesc& s, int cx, int k, int t) {
  const int i = (s.j - 1) * s.w + 1 + cx;
  return ((int64_t)(i - 1) * (s.n - 1) + (k - 1)) * s.p + t;
}

}  // namespace ddst
