// Host emulation of the CUDA features used by the HBS kernels, for CPU tests of their index
// arithmetic and synchronisation: one CTA at a time, one OS thread per CUDA thread,
// std::barrier for __syncthreads, counter-based warp synchronisation and an exchange buffer for
// shuffles.  Block-scope
// __shared__ variables become function statics (shared by the threads of the CTA that runs).
#pragma once
#include <algorithm>
#include <atomic>
#include <barrier>
#include <condition_variable>
#include <mutex>
#include <cmath>
#include <cstdint>
#include <functional>
#include <thread>
#include <vector>

#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __launch_bounds__(...)
#define __restrict__
#define __shared__ static
#define __align__(x) __attribute__((aligned(x)))

struct alignas(16) float4 { float x, y, z, w; };
struct alignas(16) uint4 { unsigned x, y, z, w; };
struct alignas(16) double2 { double x, y; };

struct HostDim3 { unsigned x = 0, y = 0, z = 0; };
inline thread_local HostDim3 threadIdx, blockIdx;
inline HostDim3 blockDim{256, 1, 1}, gridDim{1, 1, 1};
inline std::barrier<>* g_cta_barrier = nullptr;
// Warp-level synchronisation over the lanes of a mask (the whole warp, or a group of lanes
// that always synchronise together): per-lane arrival counters, one set per mask kind, so that
// groups that loop a different number of times never wait for one another.
inline std::atomic<int64_t> g_arrive[2][32][32];
inline double g_exchange[32][32];

inline void __syncthreads() { g_cta_barrier->arrive_and_wait(); }
inline void __syncwarp(unsigned mask = 0xffffffffu) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, kind = mask == 0xffffffffu ? 0 : 1;
  const int64_t my = ++g_arrive[kind][w][l];
  for (int m = 0; m < 32; ++m)
    if (mask & (1u << m))
      while (g_arrive[kind][w][m].load() < my) std::this_thread::yield();
}
template <typename T>
inline T __shfl_xor_sync(unsigned mask, T v, int lane_mask) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  g_exchange[w][l] = static_cast<double>(v);
  __syncwarp(mask);
  const T r = static_cast<T>(g_exchange[w][l ^ lane_mask]);
  __syncwarp(mask);
  return r;
}
template <typename T>
inline T __shfl_sync(unsigned mask, T v, int src_lane) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  g_exchange[w][l] = static_cast<double>(v);
  __syncwarp(mask);
  const T r = static_cast<T>(g_exchange[w][src_lane & 31]);
  __syncwarp(mask);
  return r;
}
inline int __all_sync(unsigned mask, int pred) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  g_exchange[w][l] = pred ? 1.0 : 0.0;
  __syncwarp(mask);
  int all = 1;
  for (int m = 0; m < 32; ++m)
    if ((mask & (1u << m)) && g_exchange[w][m] == 0.0) all = 0;
  __syncwarp(mask);
  return all;
}
inline int __any_sync(unsigned mask, int pred) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  g_exchange[w][l] = pred ? 1.0 : 0.0;
  __syncwarp(mask);
  int any = 0;
  for (int m = 0; m < 32; ++m)
    if ((mask & (1u << m)) && g_exchange[w][m] != 0.0) any = 1;
  __syncwarp(mask);
  return any;
}
template <typename T>
inline T __ldcg(const T* p) { return *p; }
// CTAs run one after another here, so device-scope atomics and fences only need to be atomic
inline unsigned atomicAdd(unsigned* p, unsigned v) { return std::atomic_ref<unsigned>(*p).fetch_add(v); }
inline int atomicAdd(int* p, int v) { return std::atomic_ref<int>(*p).fetch_add(v); }
inline double atomicAdd(double* p, double v) { return std::atomic_ref<double>(*p).fetch_add(v); }
inline int atomicCAS(int* p, int cmp, int val) {
  std::atomic_ref<int>(*p).compare_exchange_strong(cmp, val);
  return cmp;
}
inline void __threadfence() { std::atomic_thread_fence(std::memory_order_seq_cst); }
// Host stand-ins for the device intrinsics of the random-number generators: the high half of a
// 32 x 32-bit product and cos / sin of pi x through the C library.
inline uint32_t __umulhi(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }
inline double cospi(double x) { return std::cos(M_PI * x); }
inline float cospif(float x) { return (float)std::cos(M_PI * (double)x); }
inline void sincospif(float x, float* s, float* c) {
  *s = (float)std::sin(M_PI * (double)x);
  *c = (float)std::cos(M_PI * (double)x);
}
using std::fma;
using std::max;
using std::min;

template <typename T>
inline T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Worker threads kept across launches (creating a few hundred threads per launch dominated
// the run time of long launch sequences): run(n, f) calls f(t) on workers 0..n-1 and returns
// when all of them have finished.
struct HostThreadPool {
  std::mutex mu;
  std::condition_variable wake, done;
  std::vector<std::thread> workers;
  std::function<void(unsigned)> job;
  uint64_t generation = 0;
  unsigned active = 0, remaining = 0;
  bool stop = false;
  void worker(unsigned id) {
    uint64_t seen = 0;
    for (;;) {
      std::function<void(unsigned)> f;
      {
        std::unique_lock<std::mutex> lk(mu);
        wake.wait(lk, [&] { return stop || generation != seen; });
        if (stop) return;
        seen = generation;
        if (id >= active) continue;
        f = job;
      }
      f(id);
      std::lock_guard<std::mutex> lk(mu);
      if (--remaining == 0) done.notify_all();
    }
  }
  void run(unsigned n, std::function<void(unsigned)> f) {
    while (workers.size() < n) {
      const unsigned id = (unsigned)workers.size();
      workers.emplace_back([this, id] { worker(id); });
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      job = std::move(f);
      active = n;
      remaining = n;
      ++generation;
    }
    wake.notify_all();
    std::unique_lock<std::mutex> lk(mu);
    done.wait(lk, [&] { return remaining == 0; });
  }
  ~HostThreadPool() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    wake.notify_all();
    for (auto& t : workers) t.join();
  }
};
inline HostThreadPool g_host_pool;

// Runs `body` for every CTA of a (gx, gy, gz) grid of (bx, by)-thread CTAs, one CTA after
// another: bx * by threads (threadIdx.x = t % bx, threadIdx.y = t / bx) walk the CTAs together,
// with a barrier at the end of each CTA (a kernel's early return only skips to it).
inline void host_run_grid(unsigned gx, unsigned gy, unsigned bx, unsigned by,
                          const std::function<void()>& body, unsigned gz = 1) {
  const unsigned threads = bx * by;
  blockDim.x = bx;
  blockDim.y = by;
  gridDim.x = gx;
  gridDim.y = gy;
  gridDim.z = gz;
  for (auto& k : g_arrive)
    for (auto& w : k)
      for (auto& c : w) c.store(0);
  std::barrier<> cta(threads), end(threads);
  g_cta_barrier = &cta;
  g_host_pool.run(threads, [&body, &end, bx, gx, gy, gz](unsigned t) {
    threadIdx.x = t % bx;
    threadIdx.y = t / bx;
    for (unsigned zz = 0; zz < gz; ++zz)
      for (unsigned yy = 0; yy < gy; ++yy)
        for (unsigned xx = 0; xx < gx; ++xx) {
          blockIdx.x = xx;
          blockIdx.y = yy;
          blockIdx.z = zz;
          body();
          end.arrive_and_wait();
        }
  });
}

inline void host_launch2(unsigned gx, unsigned gy, unsigned threads,
                         const std::function<void()>& body) {
  host_run_grid(gx, gy, threads, 1, body);
}

inline void host_launch2d(unsigned gx, unsigned gy, unsigned bx, unsigned by,
                          const std::function<void()>& body) {
  host_run_grid(gx, gy, bx, by, body);
}

inline void host_launch3(unsigned gx, unsigned gy, unsigned gz, unsigned threads,
                         const std::function<void()>& body) {
  host_run_grid(gx, gy, threads, 1, body, gz);
}

inline void host_launch(unsigned grid, unsigned threads, const std::function<void()>& body) {
  host_run_grid(grid, 1, threads, 1, body);
}
