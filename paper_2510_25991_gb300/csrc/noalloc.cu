// noalloc.cu -- allocation-free FP64 residual of the finite-difference system.
//
// Every other entry point of this library allocates device memory (cudaMalloc) for its
// context and work buffers.  Some callers cannot allow that: code that runs while a memory
// budget is locked, allocators that forbid new device allocations, or host threads that must
// not take the driver's allocation locks.  ddst_residual_noalloc serves them: it computes
// r = b(f, g) - A u and the norms ||r||_2, ||b||_2 for caller-owned device arrays, and its only
// scratch -- one FP64 partial sum per 256 interior unknowns and per norm -- is the file-scope
// device array below.  That array exists once per GPU that loads the library and stays
// allocated until the process exits.
#include <mutex>
#include <string>

#include "../../include/ddst.h"
#include "kernels.cuh"

namespace ddst {

constexpr int kNoallocThreads = 256;
constexpr int64_t kNoallocMaxBlocks = 65536;  // 16,777,216 interior unknowns at most
// Two partial sums per CTA: ||r||^2 in [0, kNoallocMaxBlocks), ||b||^2 behind it (1 MiB).
static __device__ __align__(256) double g_noalloc_partials[2 * kNoallocMaxBlocks];

__device__ __forceinline__ int64_t na_node(int dim, int n, int x, int y, int z) {
  const int64_t s = n + 1;
  return dim == 2 ? (int64_t)x * s + y : ((int64_t)x * s + y) * s + z;
}

// One interior node per thread: b_p = f_p - sum_{boundary q} coef_pq g_q, r_p = b_p - (A u)_p
// with the same face-average stencil as the solver's refinement residual; per-CTA partial
// sums of r^2 and b^2 go to part[blockIdx.x] and part[kNoallocMaxBlocks + blockIdx.x].
__global__ void __launch_bounds__(kNoallocThreads)
    k_residual_noalloc(int dim, int n, double b0, double b1, double b2,
                       const double* __restrict__ a, const double* __restrict__ c,
                       const double* __restrict__ f, const double* __restrict__ g,
                       const double* __restrict__ u, double* __restrict__ r,
                       double* __restrict__ part, int64_t nint) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double bc[3] = {b0, b1, b2};
  const double h = 1.0 / n, h2 = 1.0 / (h * h), h2b = 0.5 / h;
  double rr = 0.0, bb = 0.0;
  if (q < nint) {
    int x, y, z;
    int64_t str[3];
    if (dim == 2) {
      x = (int)(q / (n - 1)) + 1; y = (int)(q % (n - 1)) + 1; z = 0;
      str[0] = n - 1; str[1] = 1; str[2] = 0;
    } else {
      const int64_t nn = (int64_t)(n - 1) * (n - 1);
      x = (int)(q / nn) + 1; y = (int)((q / (n - 1)) % (n - 1)) + 1; z = (int)(q % (n - 1)) + 1;
      str[0] = nn; str[1] = n - 1; str[2] = 1;
    }
    const int64_t pn = na_node(dim, n, x, y, z);
    const double ap = a[pn];
    double rhs = f[q];
    double diag = c ? c[pn] : 0.0, off = 0.0;
    for (int d = 0; d < dim; ++d) {
      for (int s = -1; s <= 1; s += 2) {
        int xx = x, yy = y, zz = z;
        if (d == 0) xx += s; else if (d == 1) yy += s; else zz += s;
        const int coord = d == 0 ? xx : (d == 1 ? yy : zz);
        const int64_t qn = na_node(dim, n, xx, yy, zz);
        const double af = 0.5 * (ap + a[qn]);
        const double coef = -af * h2 + s * bc[d] * h2b;
        diag += af * h2;
        if (coord == 0 || coord == n) rhs -= coef * g[qn];
        else off += coef * u[q + s * str[d]];
      }
    }
    const double rv = rhs - (diag * u[q] + off);
    r[q] = rv;
    rr = rv * rv;
    bb = rhs * rhs;
  }
  __shared__ double red[2][kNoallocThreads / 32];
  rr = warp_sum(rr);
  bb = warp_sum(bb);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = rr;
    red[1][threadIdx.x >> 5] = bb;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double v0 = threadIdx.x < (kNoallocThreads / 32) ? red[0][threadIdx.x] : 0.0;
    double v1 = threadIdx.x < (kNoallocThreads / 32) ? red[1][threadIdx.x] : 0.0;
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    if (threadIdx.x == 0) {
      part[blockIdx.x] = v0;
      part[kNoallocMaxBlocks + blockIdx.x] = v1;
    }
  }
}

// norms[0] = sqrt(sum part[0..np)), norms[1] = sqrt(sum part[max..max+np)).  One CTA.
__global__ void k_norms_noalloc(const double* __restrict__ part, int np, double* __restrict__ norms) {
  double v0 = 0.0, v1 = 0.0;
  for (int e = threadIdx.x; e < np; e += blockDim.x) {
    v0 += part[e];
    v1 += part[kNoallocMaxBlocks + e];
  }
  __shared__ double red[2][32];
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = v0;
    red[1][threadIdx.x >> 5] = v1;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double a0 = threadIdx.x < (blockDim.x >> 5) ? red[0][threadIdx.x] : 0.0;
    double a1 = threadIdx.x < (blockDim.x >> 5) ? red[1][threadIdx.x] : 0.0;
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    if (threadIdx.x == 0) {
      norms[0] = sqrt(a0);
      norms[1] = sqrt(a1);
    }
  }
}

void set_global_error(const std::string& m);  // message for ddst_last_error(NULL), api.cu

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {nullptr};  // device address of g_noalloc_partials, per device

// Memory the kernels may read on device dev: device memory of dev itself, or managed memory.
// Device memory of another GPU is refused (without peer access a load from it would fault).
bool on_device(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice && at.device == dev) ||
         at.type == cudaMemoryTypeManaged;
}
}  // namespace

}  // namespace ddst

extern "C" ddst_status ddst_residual_noalloc(const ddst_grid* grid, const ddst_coeffs* coeffs,
                                             const double* f, const double* g, const double* u,
                                             double* r, double* norms, void* stream) {
  using namespace ddst;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  auto bad = [](ddst_status s, const std::string& m) {
    set_global_error(m);
    return s;
  };
  if (!grid || !coeffs) return bad(DDST_ERR_INVALID_ARG, "grid or coeffs is NULL");
  if (grid->dim != 2 && grid->dim != 3) return bad(DDST_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (grid->n < 2 || grid->n > 65536) return bad(DDST_ERR_INVALID_ARG, "n out of range");
  const int dim = grid->dim, n = (int)grid->n;
  int64_t nint = 1;
  for (int d = 0; d < dim; ++d) nint *= (n - 1);
  const int64_t nblk = (nint + kNoallocThreads - 1) / kNoallocThreads;
  if (nblk > kNoallocMaxBlocks)
    return bad(DDST_ERR_INVALID_ARG, "ddst_residual_noalloc handles at most " +
                                         std::to_string(kNoallocMaxBlocks * kNoallocThreads) +
                                         " interior unknowns; this grid has " +
                                         std::to_string(nint));
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return bad(DDST_ERR_CUDA, "cudaGetDevice failed");
  }
  if (!on_device(coeffs->a, dev) || !on_device(f, dev) || !on_device(g, dev) ||
      !on_device(u, dev) || !on_device(r, dev) || !on_device(norms, dev) ||
      (coeffs->c && !on_device(coeffs->c, dev)))
    return bad(DDST_ERR_INVALID_ARG,
               "ddst_residual_noalloc takes device arrays of the current device only (it stages "
               "nothing)");
  if (!g_noalloc_ptr[dev]) {
    // host code may not use the array's name as an address: ask the runtime for it, once per
    // device, with that device current
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return bad(DDST_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const double* b = coeffs->b;
  note_launch();
  k_residual_noalloc<<<(unsigned)nblk, kNoallocThreads, 0, st>>>(
      dim, n, b[0], dim > 1 ? b[1] : 0.0, dim > 2 ? b[2] : 0.0, coeffs->a, coeffs->c, f, g, u, r,
      g_noalloc_ptr[dev], nint);
  note_launch();
  k_norms_noalloc<<<1, 1024, 0, st>>>(g_noalloc_ptr[dev], (int)nblk, norms);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bad(DDST_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return DDST_OK;
}
