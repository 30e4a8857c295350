// Host model of the shared-memory mbarrier and the bulk (TMA, untiled) global -> shared copy,
// as the library's kernels use them.  A phase completes once its expected arrivals (the count
// given at init) have arrived and the transaction bytes announced by expect-tx arrivals have
// all landed; the next phase then expects the same count again.  The 64-bit barrier word holds
// the number of completed phases (bits 0..15), the arrivals still expected (bits 16..31) and
// the transaction bytes outstanding (bits 32..62); the count of every barrier is kept in a
// table beside it.  A copy is a memcpy that then counts its bytes off.  The model checks what
// the hardware requires: 16-byte aligned copy addresses and sizes, no arrival beyond the count,
// no more bytes than announced.
#pragma once
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>

inline std::mutex g_mbar_mu;
inline std::map<const uint64_t*, uint32_t> g_mbar_count;

inline void host_mbar_fail(const char* what) {
  std::fprintf(stderr, "mbarrier model: %s\n", what);
  std::abort();
}

inline void host_mbar_init(uint64_t* bar, uint32_t count) {
  if (count == 0 || count > 0xffffu) host_mbar_fail("count");
  {
    std::lock_guard<std::mutex> lk(g_mbar_mu);
    g_mbar_count[bar] = count;
  }
  std::atomic_ref<uint64_t>(*bar).store((uint64_t)count << 16);
}

inline uint32_t host_mbar_count(const uint64_t* bar) {
  std::lock_guard<std::mutex> lk(g_mbar_mu);
  auto it = g_mbar_count.find(bar);
  if (it == g_mbar_count.end()) host_mbar_fail("barrier used before init");
  return it->second;
}

// Applies `arrivals` arrivals and `tx` transaction bytes (announced: tx > 0; landed: tx < 0).
inline void host_mbar_update(uint64_t* bar, uint32_t arrivals, int64_t tx) {
  const uint32_t count = host_mbar_count(bar);
  std::atomic_ref<uint64_t> a(*bar);
  uint64_t v = a.load();
  for (;;) {
    const uint64_t done = v & 0xffffu, left = (v >> 16) & 0xffffu;
    const int64_t pend = (int64_t)((v >> 32) & 0x7fffffffull) + tx;
    if (arrivals > left) host_mbar_fail("arrival beyond the count");
    if (pend < 0) host_mbar_fail("more bytes landed than announced");
    const uint64_t nleft = left - arrivals;
    const uint64_t nv = (nleft == 0 && pend == 0)
                            ? ((done + 1) & 0xffffu) | ((uint64_t)count << 16)
                            : done | (nleft << 16) | ((uint64_t)pend << 32);
    if (a.compare_exchange_weak(v, nv, std::memory_order_acq_rel)) return;
  }
}

inline void host_mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  host_mbar_update(bar, 1, (int64_t)bytes);
}

// A plain arrival (mbarrier.arrive, or a tensor-core commit).
inline void host_mbar_arrive(uint64_t* bar) { host_mbar_update(bar, 1, 0); }

inline void host_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  if (((uintptr_t)dst | (uintptr_t)src) % 16 != 0 || bytes % 16 != 0) {
    std::fprintf(stderr, "bulk copy: unaligned (dst %p, src %p, %u bytes)\n", dst, src, bytes);
    std::abort();
  }
  std::memcpy(dst, src, bytes);
  host_mbar_update(bar, 0, -(int64_t)bytes);
}

// True once the phase of the given parity has completed.
inline bool host_mbar_try_wait(uint64_t* bar, uint32_t parity) {
  return (std::atomic_ref<uint64_t>(*bar).load(std::memory_order_acquire) & 1) != parity;
}

// Bounded wait: false when the phase has not completed after a long spin.
inline bool host_mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long it = 0; it < 20000000L; ++it) {
    if (host_mbar_try_wait(bar, parity)) return true;
    std::this_thread::yield();
  }
  return false;
}
