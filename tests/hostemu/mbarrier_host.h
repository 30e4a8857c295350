// Host model of the shared-memory mbarrier and the bulk (TMA, untiled) global -> shared copy,
// as the library's kernels use them: one arrival per phase (mbarrier.init with count 1), made
// by the thread that issues the phase's copies with the expected byte count, or by a plain
// arrival (a tensor-core commit).  The 64-bit
// barrier word holds the number of completed phases (bits 0..31), the transaction bytes still
// outstanding (bits 32..62) and whether the phase's arrival has happened (bit 63).  A copy is a
// memcpy that then counts its bytes off; the phase completes when none are outstanding.  The
// copy checks what the hardware requires of it: 16-byte aligned addresses, a size that is a
// multiple of 16 bytes, and no more bytes than the arrival announced.
#pragma once
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <thread>

inline void host_mbar_init(uint64_t* bar, uint32_t count) {
  if (count != 1) { std::fprintf(stderr, "mbarrier model: count %u\n", count); std::abort(); }
  std::atomic_ref<uint64_t>(*bar).store(0);
}

inline void host_mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  std::atomic_ref<uint64_t> a(*bar);
  const uint64_t v = a.load();
  if (v >> 63) { std::fprintf(stderr, "mbarrier model: second arrival in one phase\n"); std::abort(); }
  a.store(v | (1ull << 63) | ((uint64_t)bytes << 32));
}

inline void host_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  if (((uintptr_t)dst | (uintptr_t)src) % 16 != 0 || bytes % 16 != 0) {
    std::fprintf(stderr, "bulk copy: unaligned (dst %p, src %p, %u bytes)\n", dst, src, bytes);
    std::abort();
  }
  std::memcpy(dst, src, bytes);
  std::atomic_ref<uint64_t> a(*bar);
  uint64_t v = a.load();
  const uint64_t pend = (v >> 32) & 0x7fffffffull;
  if (!(v >> 63) || pend < bytes) {
    std::fprintf(stderr, "mbarrier model: %u bytes arrive, %llu announced\n", bytes,
                 (unsigned long long)pend);
    std::abort();
  }
  v = pend == bytes ? (v & 0xffffffffull) + 1 : (v & ~(0x7fffffffull << 32)) | ((pend - bytes) << 32);
  a.store(v, std::memory_order_release);
}

// A plain arrival (mbarrier.arrive, or a tensor-core commit): completes the phase unless copies
// announced by an expect-tx are still outstanding.
inline void host_mbar_arrive(uint64_t* bar) {
  std::atomic_ref<uint64_t> a(*bar);
  const uint64_t v = a.load();
  if (v >> 63) { std::fprintf(stderr, "mbarrier model: second arrival in one phase\n"); std::abort(); }
  const uint64_t pend = (v >> 32) & 0x7fffffffull;
  a.store(pend == 0 ? (v & 0xffffffffull) + 1 : v | (1ull << 63), std::memory_order_release);
}

// True once the phase of the given parity has completed.
inline bool host_mbar_try_wait(uint64_t* bar, uint32_t parity) {
  return (std::atomic_ref<uint64_t>(*bar).load(std::memory_order_acquire) & 1) != parity;
}

// Bounded wait: false when the phase has not completed after a long spin.
inline bool host_mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long it = 0; it < 200000000L; ++it) {
    if (host_mbar_try_wait(bar, parity)) return true;
    std::this_thread::yield();
  }
  return false;
}
