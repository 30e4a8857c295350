// Host emulation of the CUDA features used by the HBS apply kernels, for CPU tests of their
// index arithmetic and synchronisation: one CTA at a time, one OS thread per CUDA thread,
// std::barrier for __syncthreads and a per-warp exchange buffer for shuffles.  Block-scope
// __shared__ variables become function statics (shared by the threads of the CTA that runs).
#pragma once
#include <algorithm>
#include <barrier>
#include <cmath>
#include <cstdint>
#include <functional>
#include <thread>
#include <vector>

#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __launch_bounds__(x)
#define __restrict__
#define __shared__ static

struct HostDim3 { unsigned x = 0, y = 0, z = 0; };
inline thread_local HostDim3 threadIdx, blockIdx;
inline HostDim3 blockDim{256, 1, 1};
inline std::barrier<>* g_cta_barrier = nullptr;
inline std::barrier<>* g_warp_barrier[32];
inline double g_exchange[32][32];

inline void __syncthreads() { g_cta_barrier->arrive_and_wait(); }
inline void __syncwarp(unsigned = 0xffffffffu) { g_warp_barrier[threadIdx.x >> 5]->arrive_and_wait(); }
template <typename T>
inline T __shfl_xor_sync(unsigned, T v, int lane_mask) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  g_exchange[w][l] = static_cast<double>(v);
  g_warp_barrier[w]->arrive_and_wait();
  const T r = static_cast<T>(g_exchange[w][l ^ lane_mask]);
  g_warp_barrier[w]->arrive_and_wait();
  return r;
}
template <typename T>
inline T __ldcg(const T* p) { return *p; }
using std::fma;
using std::max;
using std::min;

template <typename T>
inline T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Runs `body` for every CTA of a one-dimensional grid of `threads`-thread CTAs.
inline void host_launch(unsigned grid, unsigned threads, const std::function<void()>& body) {
  blockDim.x = threads;
  for (unsigned b = 0; b < grid; ++b) {
    std::barrier<> cta(threads);
    g_cta_barrier = &cta;
    for (unsigned w = 0; w < (threads + 31) / 32; ++w) g_warp_barrier[w] = new std::barrier<>(32);
    std::vector<std::thread> ts;
    for (unsigned t = 0; t < threads; ++t)
      ts.emplace_back([&body, t, b] { threadIdx.x = t; blockIdx.x = b; body(); });
    for (auto& t : ts) t.join();
    for (unsigned w = 0; w < (threads + 31) / 32; ++w) delete g_warp_barrier[w];
  }
}
