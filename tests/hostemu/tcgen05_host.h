// Host model of the tcgen05 tensor-core instructions that the library's kernels use, written
// from the public PTX ISA description, for CPU tests of those kernels' index arithmetic, operand
// layouts and synchronisation (include after cuda_host_shim.h and mbarrier_host.h):
// * tensor memory: 128 lanes x 512 columns of 32-bit words for the CTA that runs; an address is
//   lane << 16 | column; alloc returns column 0 and accesses outside the allocation abort;
// * shared-memory matrix descriptors: start address >> 4 in bits 0..13, leading byte offset
//   >> 4 in bits 16..29, stride byte offset >> 4 in bits 32..45; no swizzle, K-major operands:
//   element (row, k) of a core matrix grid sits at start + (row / 8) SBO + (k / 4) LBO +
//   (row % 8) 16 + (k % 4) 4 bytes;
// * the instruction descriptor's shape: N >> 3 in bits 17..22, M >> 4 in bits 24..28;
// * kind::tf32, K = 8 per instruction: each operand keeps its upper 19 bits (TF32), products and
//   sums in FP32, D = A B^T (+ D) in lanes 0..M-1, columns d .. d + N - 1; the MMA completes at
//   once, so a commit arrives on its mbarrier at once;
// * shared-memory addresses are byte offsets from the CTA's dynamic shared memory
//   (host_smem_base).
#pragma once
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

inline unsigned char* host_smem_base = nullptr;
inline uint32_t host_tmem[128][512];
inline int host_tmem_cols = 0;

inline void host_tc_fail(const char* what) {
  std::fprintf(stderr, "tcgen05 model: %s\n", what);
  std::abort();
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  const unsigned char* q = static_cast<const unsigned char*>(p);
  if (!host_smem_base || q < host_smem_base) host_tc_fail("address outside shared memory");
  return static_cast<uint32_t>(q - host_smem_base);
}

inline float __uint_as_float(uint32_t u) { float f; std::memcpy(&f, &u, 4); return f; }
inline uint32_t __float_as_uint(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }

inline float tf32_rna(float x) {  // cvt.rna.tf32.f32: 10-bit significand, nearest, ties away
  uint32_t u = __float_as_uint(x);
  u = (u + 0x1000u) & ~0x1fffu;
  return __uint_as_float(u);
}

// alloc / relinquish / dealloc are warp-collective: lane 0 acts
inline void host_tmem_alloc(uint32_t* dst, uint32_t cols) {
  if ((threadIdx.x & 31) != 0) return;
  if (host_tmem_cols != 0) host_tc_fail("second allocation");
  if (cols < 32 || cols > 512 || (cols & (cols - 1))) host_tc_fail("column count");
  host_tmem_cols = (int)cols;
  for (auto& lane : host_tmem)
    for (auto& w : lane) w = 0x7fc00000u;  // NaN: reads of unwritten columns show
  *dst = 0;
}
inline void host_tmem_relinquish() {}
inline void host_tmem_dealloc(uint32_t taddr, uint32_t cols) {
  if ((threadIdx.x & 31) != 0) return;
  if (taddr != 0 || (int)cols != host_tmem_cols) host_tc_fail("dealloc of another allocation");
  host_tmem_cols = 0;
}

inline uint32_t& host_tmem_at(uint32_t taddr, int dl, int dc) {
  const int lane = (int)(taddr >> 16) + dl, col = (int)(taddr & 0xffffu) + dc;
  if (lane < 0 || lane >= 128 || col < 0 || col >= host_tmem_cols) host_tc_fail("tensor memory access");
  return host_tmem[lane][col];
}

inline float host_desc_elem(uint64_t d, int row, int k) {
  const uint32_t start = (uint32_t)(d & 0x3fffu) << 4;
  const uint32_t lbo = (uint32_t)((d >> 16) & 0x3fffu) << 4;
  const uint32_t sbo = (uint32_t)((d >> 32) & 0x3fffu) << 4;
  const uint32_t off = start + (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 2) * lbo +
                       (uint32_t)(row & 7) * 16 + (uint32_t)(k & 3) * 4;
  float v;
  std::memcpy(&v, host_smem_base + off, 4);
  return v;
}

inline float host_tf32(float x) { return __uint_as_float(__float_as_uint(x) & ~0x1fffu); }

template <typename GetA>
inline void host_mma(uint32_t tmem_d, GetA a, uint64_t b, uint32_t idesc, uint32_t accum) {
  const int N = (int)((idesc >> 17) & 0x3fu) << 3, M = (int)((idesc >> 24) & 0x1fu) << 4;
  if (M != 128 || N < 8 || N > 256) host_tc_fail("shape");
  float As[128][8], Bs[256][8];
  for (int m = 0; m < M; ++m)
    for (int k = 0; k < 8; ++k) As[m][k] = host_tf32(a(m, k));
  for (int n = 0; n < N; ++n)
    for (int k = 0; k < 8; ++k) Bs[n][k] = host_tf32(host_desc_elem(b, n, k));
  for (int m = 0; m < M; ++m)
    for (int n = 0; n < N; ++n) {
      uint32_t& d = host_tmem_at(tmem_d, m, n);
      float acc = accum ? __uint_as_float(d) : 0.f;
      for (int k = 0; k < 8; ++k) acc += As[m][k] * Bs[n][k];
      d = __float_as_uint(acc);
    }
}

inline void mma_tf32_ss(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
  host_mma(tmem_d, [&](int m, int k) { return host_desc_elem(a, m, k); }, b, idesc, accum);
}
inline void mma_tf32_tmem_a(uint32_t tmem_d, uint32_t tmem_a, uint64_t b, uint32_t idesc,
                            uint32_t accum) {
  host_mma(tmem_d, [&](int m, int k) { return __uint_as_float(host_tmem_at(tmem_a, m, k)); }, b,
           idesc, accum);
}

inline void mma_commit(uint64_t* bar) { host_mbar_arrive(bar); }
inline void mbar_arrive1(uint64_t* bar) { host_mbar_arrive(bar); }
inline void tc_fence_before() { std::atomic_thread_fence(std::memory_order_seq_cst); }
inline void tc_fence_after() { std::atomic_thread_fence(std::memory_order_seq_cst); }

// 32x32b loads and stores: thread i of the warp takes lane (address lane) + i
template <int N>
inline void host_tmem_ld(uint32_t taddr, uint32_t (&r)[N]) {
  for (int j = 0; j < N; ++j) r[j] = host_tmem_at(taddr, threadIdx.x & 31, j);
}
inline void tmem_ld32_wait(uint32_t taddr, uint32_t (&r)[32]) { host_tmem_ld(taddr, r); }
inline void tmem_ld64_wait(uint32_t taddr, uint32_t (&r)[64]) { host_tmem_ld(taddr, r); }
inline void tmem_ld1x2_wait(uint32_t ta, uint32_t tb, uint32_t& ra, uint32_t& rb) {
  ra = host_tmem_at(ta, threadIdx.x & 31, 0);
  rb = host_tmem_at(tb, threadIdx.x & 31, 0);
}
inline void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  for (int j = 0; j < 16; ++j) host_tmem_at(taddr, threadIdx.x & 31, j) = r[j];
}
inline void tmem_wait_st() { std::atomic_thread_fence(std::memory_order_seq_cst); }

// bulk shared -> global stores (plain, or element-wise FP32 add), complete at once
inline void host_bulk_check(const void* g, const void* s, uint32_t bytes) {
  if (((uintptr_t)g | (uintptr_t)s) % 16 != 0 || bytes % 16 != 0) host_tc_fail("bulk store alignment");
}
inline void bulk_s2g(float* dst, const void* src, uint32_t bytes) {
  host_bulk_check(dst, src, bytes);
  std::memcpy(dst, src, bytes);
}
inline void bulk_s2g_add(float* dst, const void* src, uint32_t bytes) {
  host_bulk_check(dst, src, bytes);
  const float* s = static_cast<const float*>(src);
  for (uint32_t i = 0; i < bytes / 4; ++i) dst[i] += s[i];
}
inline void bulk_commit() {}
inline void bulk_wait_all() {}
