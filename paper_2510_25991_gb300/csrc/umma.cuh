// umma.cuh -- shared-memory operand layout of the tcgen05 tensor-core kernels.
//
// Canonical K-major layout without swizzle: core matrices of 8 rows x 16 bytes (4 TF32
// values); core matrix (row group g, K group kk) of a rows x K operand starts at byte
// g * (K * 32) + kk * 128, i.e. leading byte offset (K direction) 128 and stride byte offset
// (row direction) 32 K.
#pragma once
#include <cstdint>

#include "common.cuh"

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
// dimension ld, scale a global vector of M values (NULL: the copy is zero).  Each thread writes
// four consecutive K entries of one row (one 16-byte store per part); consecutive threads take
// consecutive rows, so the shared-memory reads X(c, r) are conflict-free.
template <int M>
__device__ __forceinline__ void store_umma_split_T(const float* __restrict__ X, int ld,
                                                   const float* __restrict__ scale,
                                                   float* __restrict__ hi,
                                                   float* __restrict__ lo) {
  for (int e = threadIdx.x; e < M * (M / 4); e += blockDim.x) {
    const int r = e % M, c = 4 * (e / M);
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = scale ? -scale[c + u] * X[(c + u) * ld + r] : 0.f;
    float4 h, l;
    h.x = tf32_rna(v[0]); l.x = tf32_rna(v[0] - h.x);
    h.y = tf32_rna(v[1]); l.y = tf32_rna(v[1] - h.y);
    h.z = tf32_rna(v[2]); l.z = tf32_rna(v[2] - h.z);
    h.w = tf32_rna(v[3]); l.w = tf32_rna(v[3] - h.w);
    const uint32_t o = umma_off(r, c, M) >> 2;
    *reinterpret_cast<float4*>(hi + o) = h;
    *reinterpret_cast<float4*>(lo + o) = l;
  }
}

// ---------------------------------------------------------------------------------------
// tcgen05 helpers (inline PTX): shared-memory descriptors, instruction descriptor, MMA issue,
// commits, fences and tensor-memory loads/stores.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; no swizzle, base offset 0
  return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also returns (false) once *abort is set by another role.  budget: clock
// cycles before the wait gives up (records ST_TIMEOUT and raises *abort); 4e9 is about 2 s.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort,
                                             DevStatus* st, int slab, int block,
                                             long long budget = 4000000000LL) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > budget) {
      set_status(st, ST_TIMEOUT, slab, block);
      *abort = 1;
      return false;
    }
  }
}

// D (tmem) = A (tmem, 128 lanes x 8 columns) * B (shared-memory descriptor) [+ D].
__device__ __forceinline__ void mma_tf32_tmem_a(uint32_t tmem_d, uint32_t tmem_a, uint64_t b,
                                                uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

// Loads from tensor memory complete (tcgen05.wait::ld) inside the same asm statement, so no
// use of the destination registers can be scheduled before the wait.
// MB consecutive 32-bit columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld32_wait(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld64_wait(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
}

// Two single columns a and b of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld1x2_wait(uint32_t ta, uint32_t tb, uint32_t& ra,
                                                uint32_t& rb) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%2];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%1}, [%3];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(ra), "=r"(rb)
      : "r"(ta), "r"(tb)
      : "memory");
}

// 16 consecutive 32-bit columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// 3xTF32 split x = hi + lo with hi = rna_tf32(x), lo = rna_tf32(x - hi): both parts are exact
// TF32 values, so the tensor core (which keeps only the upper 19 bits of an operand) reads them
// unchanged, and the dropped lo * lo product stays below 2^-22 |x y|.
__device__ __forceinline__ void tf32_split(uint32_t x, uint32_t& hi, uint32_t& lo) {
  const float h = tf32_rna(__uint_as_float(x));
  hi = __float_as_uint(h);
  lo = __float_as_uint(tf32_rna(__uint_as_float(x) - h));
}


// D (tmem) = A (shared-memory descriptor) * B (shared-memory descriptor) [+ D].
__device__ __forceinline__ void mma_tf32_ss(uint32_t tmem_d, uint64_t a, uint64_t b,
                                            uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

// Bulk shared -> global copies of the async proxy: plain store or element-wise FP32 add at the
// destination (performed by the memory system, so the issuing thread never reads the old
// values).  Both addresses 16-byte aligned, bytes a multiple of 16; the shared-memory source
// must be made visible to the async proxy first (fence.proxy.async).
__device__ __forceinline__ void bulk_s2g(float* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_s2g_add(float* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(
                   dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until every committed bulk group of this thread has completed (its writes performed).
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

}  // namespace ddst
