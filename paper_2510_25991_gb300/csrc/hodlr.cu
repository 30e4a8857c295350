// hodlr.cu -- weak-admissibility hierarchical compression of the transfer operators.
//
// Sec. 2.4 of the paper: every S_{j,j'} is stored on a cluster tree shared by its source and
// target interface (the interfaces are discretized isomorphically); with weak admissibility
// every off-diagonal block of every level is low rank and only the diagonal leaves are dense.
// The paper uses nested (HBS) bases built by the randomized scheme of its reference [fastHBS];
// this library stores the non-nested HODLR variant.  Each off-diagonal block B is compressed
// by randomized sampling (Gaussian test matrix, Alg. 1's sampling step applied to the formed
// block):
//   1. Y = B Omega, Omega ~ N(0,1)^{q x s}, s = k_max + oversample (Philox4x32-10 counters,
//      Box-Muller with the CUDA math library's logf/sincospif).
//   2. Columns of Y orthonormalized in order by classical Gram-Schmidt applied twice; a column
//      is kept only if its residual norm exceeds tol * ||S_{j,j'}||_2 (rank detection: the
//      residual of a Gaussian sample estimates ||(I - Q Q^T) B||_F), at most k_max columns.
//   3. V = B^T Q, so that B ~ Q V^T.
// ||S_{j,j'}||_2 is estimated by power iteration on S^T S.  Balanced bisection tree: node t of
// level l spans [(t ng) >> l, ((t+1) ng) >> l); depth L = min{L : ceil(ng / 2^L) <= leaf}.
#include <algorithm>
#include <cmath>
#include <cstring>

#include <map>

#include "hodlr.cuh"
#include "kernels.cuh"

namespace ddst {

// ---------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter-based generator.
// ---------------------------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += W0;
    k1 += W1;
  }
  return c;
}

__device__ __forceinline__ float u01(uint32_t v) {  // (0, 1)
  return ((v >> 8) + 0.5f) * (1.0f / 16777216.0f);
}

// Four standard normal numbers for counter (a, b, c).
__device__ __forceinline__ void gauss4(uint32_t a, uint32_t b, uint32_t c, uint64_t seed,
                                       float out[4]) {
  const U4 r = philox4x32_10(U4{a, b, c, 0x5eedu}, (uint32_t)seed, (uint32_t)(seed >> 32));
  float s0, c0, s1, c1;
  const float r0 = sqrtf(-2.0f * logf(u01(r.x)));
  const float r1 = sqrtf(-2.0f * logf(u01(r.z)));
  sincospif(2.0f * u01(r.y), &s0, &c0);
  sincospif(2.0f * u01(r.w), &s1, &c1);
  out[0] = r0 * c0;
  out[1] = r0 * s0;
  out[2] = r1 * c1;
  out[3] = r1 * s1;
}

struct SBlk {         // one dense S block
  int64_t off;        // column-major ng x ng in S
  int64_t ng;
};

// Work item of the tiled kernels: (block, first row or column of the tile).
struct HItem {
  int blk;
  int64_t lo;
};

// ---------------------------------------------------------------------------------------------
// Norm estimate: power iteration on S^T S for every S block (batched GEMV).
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_sblk_gemv(const SBlk* __restrict__ sb, const T* __restrict__ S,
                            const double* __restrict__ x, double* __restrict__ y,
                            int64_t stride) {
  const SBlk b = sb[blockIdx.y];
  const double* xv = x + blockIdx.y * stride;
  double* yv = y + blockIdx.y * stride;
  const T* M = S + b.off;
  {  // y += S(:, chunk) x(chunk): thread per row, 128 columns per CTA (y zeroed)
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.z * 128;
    if (row >= b.ng || c0 >= b.ng) return;
    const int64_t c1 = min(b.ng, c0 + 128);
    double acc = 0.0;
    for (int64_t cb = c0; cb < c1; cb += 32) {  // four independent chains per 32 columns
      T p[4] = {T(0), T(0), T(0), T(0)};
      const int64_t ce = min(c1, cb + 32);
      int64_t c = cb;
      for (; c + 3 < ce; c += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u] = fma(M[(c + u) * b.ng + row], static_cast<T>(xv[c + u]), p[u]);
      }
      for (; c < ce; ++c) p[0] = fma(M[c * b.ng + row], static_cast<T>(xv[c]), p[0]);
      acc += (double)((p[0] + p[1]) + (p[2] + p[3]));
    }
    atomicAdd(&yv[row], acc);
  }
}

// y = S^T x for every S block: the columns are streamed through 32-row shared-memory tiles (a
// CTA owns 128 columns; each warp loads 16 coalesced column segments per tile) and x's 32 tile
// rows are staged beside them, so the kernel is not bound by per-column reads of x through L1
// (a warp per column reading x through L1 was).  grid = (ceil(ng/128), blocks), 256 threads.
template <typename T>
__global__ void __launch_bounds__(256) k_sblk_gemv_t(const SBlk* __restrict__ sb,
                                                     const T* __restrict__ S,
                                                     const double* __restrict__ x,
                                                     double* __restrict__ y, int64_t stride) {
  __shared__ T tile[128 * 33];
  __shared__ T xs[32];
  __shared__ double red[256];
  const SBlk b = sb[blockIdx.y];
  const int64_t ng = b.ng, c0 = (int64_t)blockIdx.x * 128;
  if (c0 >= ng) return;  // uniform over the CTA
  const double* xv = x + blockIdx.y * stride;
  const T* M = S + b.off;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cl = tid & 127, half = tid >> 7;
  double acc = 0.0;
  for (int64_t r0 = 0; r0 < ng; r0 += 32) {
    const int64_t r = r0 + lane;
#pragma unroll
    for (int cc = 0; cc < 16; ++cc) {
      const int64_t c = c0 + warp * 16 + cc;
      tile[(warp * 16 + cc) * 33 + lane] = (c < ng && r < ng) ? M[c * ng + r] : T(0);
    }
    if (tid < 32) xs[tid] = r0 + tid < ng ? static_cast<T>(xv[r0 + tid]) : T(0);
    __syncthreads();
    T p = T(0);
#pragma unroll
    for (int i = 0; i < 16; ++i) p = fma(tile[cl * 33 + half * 16 + i], xs[half * 16 + i], p);
    acc += static_cast<double>(p);
    __syncthreads();
  }
  red[tid] = acc;
  __syncthreads();
  const int64_t c = c0 + cl;
  if (half == 0 && c < ng) y[blockIdx.y * stride + c] = red[tid] + red[tid + 128];
}

// x_b <- y_b / ||y_b||, nrm[b] = ||y_b||  (one CTA per block)
__global__ void k_sblk_normalize(const SBlk* __restrict__ sb, double* __restrict__ x,
                                 const double* __restrict__ y, int64_t stride,
                                 double* __restrict__ nrm) {
  const SBlk b = sb[blockIdx.x];
  const double* yv = y + blockIdx.x * stride;
  double* xv = x + blockIdx.x * stride;
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < b.ng; e += blockDim.x) acc += yv[e] * yv[e];
  __shared__ double red[32];
  __shared__ double tot;
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) tot = sqrt(t);
  }
  __syncthreads();
  const double inv = tot > 0.0 ? 1.0 / tot : 0.0;
  for (int64_t e = threadIdx.x; e < b.ng; e += blockDim.x) xv[e] = yv[e] * inv;
  if (threadIdx.x == 0) nrm[blockIdx.x] = tot;
}

__global__ void k_sblk_init(const SBlk* __restrict__ sb, double* __restrict__ x, int64_t stride,
                            uint64_t seed) {
  const SBlk b = sb[blockIdx.x];
  double* xv = x + blockIdx.x * stride;
  for (int64_t e = threadIdx.x; e < b.ng; e += blockDim.x) {
    float g[4];
    gauss4((uint32_t)e, (uint32_t)blockIdx.x, 0xabcdu, seed, g);
    xv[e] = g[0];
  }
}

// ---------------------------------------------------------------------------------------------
// Compression kernels
// ---------------------------------------------------------------------------------------------
struct HDev {        // per off-diagonal block, device view for compression
  int64_t s_off;     // element offset of B(0,0) in S (column-major, leading dim ng)
  int64_t ng;
  int64_t p, q;      // rows, cols
  int s;             // sample capacity
  int sblk;
  int64_t u_off, v_off;
};

// Omega (q x s, column-major) into the V slot.
template <typename T>
__global__ void k_gen_omega(const HDev* __restrict__ hb, T* __restrict__ UV, uint64_t seed) {
  const HDev b = hb[blockIdx.y];
  const int64_t total = b.q * ((b.s + 3) / 4);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e % b.q;
    const int jg = (int)(e / b.q);
    float g[4];
    gauss4((uint32_t)c, (uint32_t)jg, (uint32_t)blockIdx.y, seed, g);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = 4 * jg + u;
      if (j < b.s) UV[b.v_off + (int64_t)j * b.q + c] = static_cast<T>(g[u]);
    }
  }
}

// Y = B Omega for a tile of 64 rows (all s samples).  256 threads: 16 row groups (4 rows) x
// 16 sample groups (SC/16 samples).  Column chunks of 32 staged in shared memory.
template <typename T, int SC>
__global__ void __launch_bounds__(256) k_sketch(const HItem* __restrict__ items,
                                                const HDev* __restrict__ hb,
                                                const T* __restrict__ S, T* __restrict__ UV) {
  constexpr int CPT = SC / 16;
  const HItem it = items[blockIdx.x];
  const HDev b = hb[it.blk];
  __shared__ T sB[32][64 + 1];
  __shared__ T sO[32][SC + 1];
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
  T acc[4][CPT];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[a][c] = T(0);
  const T* Bp = S + b.s_off + it.lo;  // B(row, col) at Bp[col * ng + row - lo]
  const T* Om = UV + b.v_off;         // Omega(col, j) at Om[j * q + col]
  for (int64_t c0 = 0; c0 < b.q; c0 += 32) {
    for (int e = threadIdx.x; e < 32 * 64; e += 256) {
      const int cc = e >> 6, rr = e & 63;
      const int64_t col = c0 + cc, row = it.lo + rr;
      sB[cc][rr] = (col < b.q && row < b.p) ? Bp[col * b.ng + rr] : T(0);
    }
    for (int e = threadIdx.x; e < 32 * SC; e += 256) {
      const int j = e / 32, cc = e % 32;
      const int64_t col = c0 + cc;
      sO[cc][j] = (col < b.q && j < b.s) ? Om[(int64_t)j * b.q + col] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int cc = 0; cc < 32; ++cc) {
      T bv[4], ov[CPT];
#pragma unroll
      for (int a = 0; a < 4; ++a) bv[a] = sB[cc][tr * 4 + a];
#pragma unroll
      for (int c = 0; c < CPT; ++c) ov[c] = sO[cc][tc * CPT + c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[a][c] = fma(bv[a], ov[c], acc[a][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t row = it.lo + tr * 4 + a;
    if (row >= b.p) continue;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int j = tc * CPT + c;
      if (j < b.s) UV[b.u_off + (int64_t)j * b.p + row] = acc[a][c];
    }
  }
}

// In-place CGS2 orthonormalization of the sketch columns with rank detection (one CTA per
// block).  Column j is kept (appended as Q[:, r]) when its residual norm exceeds thr and the
// working precision can still orthogonalize it: a residual below ~1e3 eps of the sample's own
// norm is rounding noise, so it is rejected (this floors the effective tolerance at about
// 1e3 eps_T relative to the block).  A third pass runs when the second one still removed
// more than 30% of the norm ("twice is enough" test).  The scan stops after `run` consecutive
// rejected samples: the stopping rule of the adaptive randomized range finder (Halko, Martinsson
// & Tropp 2011, Sec. 4.4), with the oversampling as the run length.
template <typename T>
__global__ void __launch_bounds__(512) k_range_cgs2(const HDev* __restrict__ hb,
                                                    T* __restrict__ UV,
                                                    const double* __restrict__ snorm, double tol,
                                                    int kmax, int run, int* __restrict__ rank_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const HDev b = hb[blockIdx.x];
  T* y = reinterpret_cast<T*>(smem_raw);  // p values
  __shared__ T h[256];
  __shared__ double red[32];
  __shared__ double s_nu;
  T* Q = UV + b.u_off;
  const double thr = tol * snorm[b.sblk];
  const int nw = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  auto norm_y = [&]() -> double {
    T part = T(0);
    for (int64_t i = threadIdx.x; i < b.p; i += blockDim.x) part = fma(y[i], y[i], part);
    const double acc = warp_sum((double)part);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      double t = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
      t = warp_sum(t);
      if (threadIdx.x == 0) s_nu = sqrt(t);
    }
    __syncthreads();
    const double v = s_nu;
    __syncthreads();
    return v;
  };
  int r = 0, rejected = 0;
  for (int j = 0; j < b.s && rejected < run; ++j) {
    for (int64_t i = threadIdx.x; i < b.p; i += blockDim.x) y[i] = Q[(int64_t)j * b.p + i];
    __syncthreads();
    const double n0 = norm_y();
    double prev = n0, cur = n0;
    for (int pass = 0; pass < 3 && r > 0; ++pass) {
      for (int c = warp; c < r; c += nw) {
        T part = T(0);
        for (int64_t i = lane; i < b.p; i += 32) part = fma(Q[(int64_t)c * b.p + i], y[i], part);
        const double acc = warp_sum((double)part);
        if (lane == 0) h[c] = static_cast<T>(acc);
      }
      __syncthreads();
      for (int64_t i = threadIdx.x; i < b.p; i += blockDim.x) {
        T acc = T(0);
        for (int c = 0; c < r; ++c) acc = fma(Q[(int64_t)c * b.p + i], h[c], acc);
        y[i] -= acc;
      }
      __syncthreads();
      prev = cur;
      cur = norm_y();
      if (pass >= 1 && cur >= 0.7 * prev) break;
    }
    const double nu = cur;
    const double floor_ = 1e3 * (double)Eps<T>::v * n0;
    if (nu > thr && nu > floor_ && r < kmax && r < 256) {
      const T inv = static_cast<T>(1.0 / nu);
      for (int64_t i = threadIdx.x; i < b.p; i += blockDim.x) Q[(int64_t)r * b.p + i] = y[i] * inv;
      ++r;
      rejected = 0;
    } else {
      ++rejected;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) rank_out[blockIdx.x] = r;
}

// V = B^T Q (q x r) for a tile of 64 columns of B.  Row chunks of 32 staged in shared memory.
template <typename T, int SC>
__global__ void __launch_bounds__(256) k_project(const HItem* __restrict__ items,
                                                 const HDev* __restrict__ hb,
                                                 const int* __restrict__ rank,
                                                 const T* __restrict__ S, T* __restrict__ UV) {
  constexpr int CPT = SC / 16;
  const HItem it = items[blockIdx.x];
  const HDev b = hb[it.blk];
  const int r = rank[it.blk];
  if (r == 0) return;
  __shared__ T sB[64][32 + 1];   // [col][row]
  __shared__ T sQ[32][SC + 1];   // [row][j]
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
  T acc[4][CPT];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[a][c] = T(0);
  const T* Q = UV + b.u_off;
  for (int64_t r0 = 0; r0 < b.p; r0 += 32) {
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
      const int cc = e >> 5, rr = e & 31;
      const int64_t col = it.lo + cc, row = r0 + rr;
      sB[cc][rr] = (col < b.q && row < b.p) ? S[b.s_off + col * b.ng + row] : T(0);
    }
    for (int e = threadIdx.x; e < 32 * SC; e += 256) {
      const int j = e / 32, rr = e % 32;
      const int64_t row = r0 + rr;
      sQ[rr][j] = (row < b.p && j < r) ? Q[(int64_t)j * b.p + row] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < 32; ++rr) {
      T bv[4], qv[CPT];
#pragma unroll
      for (int a = 0; a < 4; ++a) bv[a] = sB[tr * 4 + a][rr];
#pragma unroll
      for (int c = 0; c < CPT; ++c) qv[c] = sQ[rr][tc * CPT + c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[a][c] = fma(bv[a], qv[c], acc[a][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t col = it.lo + tr * 4 + a;
    if (col >= b.q) continue;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int j = tc * CPT + c;
      if (j < r) UV[b.v_off + (int64_t)j * b.q + col] = acc[a][c];
    }
  }
}

// Dense leaves: copy S(lo:lo+len, lo:lo+len) of every leaf (rows len..ld of each column zero).
template <typename T>
__global__ void k_copy_leaves(const HLeaf* __restrict__ lv, const int64_t* __restrict__ soff,
                              const int64_t* __restrict__ sng, const T* __restrict__ S,
                              T* __restrict__ D) {
  const HLeaf L = lv[blockIdx.y];
  const int64_t ng = sng[L.sblk], off = soff[L.sblk];
  const int64_t total = L.ld * L.len;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / L.ld, rr = e % L.ld;
    D[L.d_off + e] = rr < L.len ? S[off + (L.lo + c) * ng + L.lo + rr] : T(0);
  }
}

// ---------------------------------------------------------------------------------------------
// Application: y = x - K x (or x - K^T x) in two kernels.
//   k_h_inner : t_b = W_in^T x for every low-rank block b (W_in = V; U when transposed);
//   k_h_owner : one CTA per output-owner item (interface, leaf row range): the dense leaves and
//               the low-rank blocks (W_out t_b, W_out = U; V when transposed) of the S blocks
//               that write these rows, then y = x - sum, written once (no accumulator, no
//               atomics), or y = sum alone (K x) when asked.
// ---------------------------------------------------------------------------------------------
// One warp per low-rank block: t_b = W_in^T x_in over all rank columns, eight columns at a time,
// rows unrolled by four (32 loads in flight per lane), one warp reduction per column.  All
// blocks fit in one wave, so the time is that of the longest (top-level) block.
template <typename T>
__global__ void __launch_bounds__(256) k_h_inner(const HBlock* __restrict__ bl, int nblk,
                                                 const T* __restrict__ UV,
                                                 const double* __restrict__ x0,
                                                 double* __restrict__ t, int transpose,
                                                 const int* kdev, int64_t kstride) {
  // the owner kernel may start now: its dense-leaf part does not read t (programmatic launch)
  pdl_release();
  const int wi = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (wi >= nblk) return;
  const HBlock& b = bl[wi];
  const int rank = b.rank;
  if (rank == 0) return;
  const double* x = x0 + (kdev ? (int64_t)(*kdev - 1) * kstride : 0);
  const int len = (int)(transpose ? b.nrows : b.ncols);
  const double* xv = x + (transpose ? b.out_if + b.row0 : b.in_if + b.col0);
  const T* W = UV + (transpose ? b.u_off : b.v_off);
  for (int c0 = 0; c0 < rank; c0 += 8) {
    const int nc = min(8, rank - c0);
    const T* Wc = W + (int64_t)c0 * len;
    T acc[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) acc[g] = T(0);
    int r = lane;
    for (; r + 96 < len; r += 128) {
      T xr[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) xr[u] = static_cast<T>(xv[r + 32 * u]);
#pragma unroll
      for (int g = 0; g < 8; ++g)
        if (g < nc) {
          const T* wg = Wc + (int64_t)g * len + r;
          acc[g] = fma(wg[0], xr[0], fma(wg[32], xr[1], fma(wg[64], xr[2], fma(wg[96], xr[3], acc[g]))));
        }
    }
    for (; r < len; r += 32) {
      const T xr = static_cast<T>(xv[r]);
#pragma unroll
      for (int g = 0; g < 8; ++g)
        if (g < nc) acc[g] = fma(Wc[(int64_t)g * len + r], xr, acc[g]);
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const double v = warp_sum((double)acc[g]);
      if (lane == 0 && g < nc) t[b.t_off + c0 + g] = v;
    }
  }
}

// Dense leaves are column-major with a leading dimension that is a multiple of 4, so every
// column starts on a 16-byte boundary and is read with 16-byte vectors.
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ void vec_fma(const typename Vec16<T>::type& m, T x, T* a);
template <>
__device__ __forceinline__ void vec_fma<float>(const float4& m, float x, float* a) {
  a[0] = fma(m.x, x, a[0]); a[1] = fma(m.y, x, a[1]); a[2] = fma(m.z, x, a[2]); a[3] = fma(m.w, x, a[3]);
}
template <>
__device__ __forceinline__ void vec_fma<double>(const double2& m, double x, double* a) {
  a[0] = fma(m.x, x, a[0]); a[1] = fma(m.y, x, a[1]);
}
template <typename T>
__device__ __forceinline__ T vec_dot(const typename Vec16<T>::type& m, const T* x);
template <>
__device__ __forceinline__ float vec_dot<float>(const float4& m, const float* x) {
  return m.x * x[0] + m.y * x[1] + m.z * x[2] + m.w * x[3];
}
template <>
__device__ __forceinline__ double vec_dot<double>(const double2& m, const double* x) {
  return m.x * x[0] + m.y * x[1];
}

constexpr int OWN_T = 128;  // threads of an owner CTA: 9 resident per SM, one wave at 2048^2

template <typename T>
__global__ void __launch_bounds__(OWN_T) k_h_owner(const HOwn* __restrict__ items,
                                                 const HBlock* __restrict__ bl,
                                                 const HLeaf* __restrict__ lv,
                                                 const T* __restrict__ UV,
                                                 const T* __restrict__ D,
                                                 const double* __restrict__ t,
                                                 const double* __restrict__ x0,
                                                 double* __restrict__ y, int transpose,
                                                 int konly, const int* kdev, int64_t kstride) {
  using V = typename Vec16<T>::type;
  constexpr int VEC = Vec16<T>::n;
  const double* x = x0 + (kdev ? (int64_t)(*kdev - 1) * kstride : 0);
  const HOwn* it = items + blockIdx.x;
  const int len = it->len, nsrc = it->nsrc;  // len <= 256
  __shared__ __align__(16) T sx[2 * 256];
  __shared__ T red[256 * 4];
  __shared__ double outv[256];
  // low-rank blocks over these rows, per (source, level): W_out offset of row lo, its leading
  // dimension, rank, and t_b (first HOWN_TCAP entries) staged once
  constexpr int NSL = 2 * HOWN_MAXL;
  __shared__ int64_t s_woff[NSL], s_nr[NSL];
  __shared__ int s_rank[NSL];
  __shared__ T s_t[NSL * HOWN_TCAP];
  for (int r = threadIdx.x; r < len; r += blockDim.x) outv[r] = 0.0;
  for (int q = threadIdx.x; q < NSL; q += blockDim.x) {
    const int s = q / HOWN_MAXL, l = q % HOWN_MAXL;
    const int hb = s < nsrc ? it->hb[s][l] : -1;
    s_rank[q] = 0;
    if (hb >= 0) {
      const HBlock& B = bl[hb];
      s_rank[q] = B.rank;
      s_nr[q] = transpose ? B.ncols : B.nrows;
      s_woff[q] = (transpose ? B.v_off : B.u_off) + it->lo - (transpose ? B.col0 : B.row0);
    }
  }
  // dense leaves of both sources over these rows (same tree, so same ld), one pass
  const int ld = nsrc > 0 ? (int)lv[it->leaf[0]].ld : 0;
  const T* M0 = nsrc > 0 ? D + lv[it->leaf[0]].d_off : nullptr;
  const T* M1 = nsrc > 1 ? D + lv[it->leaf[1]].d_off : nullptr;
  for (int q = 0; q < nsrc; ++q) {
    const HLeaf L = lv[it->leaf[q]];
    const double* xv = x + (transpose ? L.out_if : L.in_if) + L.lo;
    for (int e = threadIdx.x; e < ld; e += blockDim.x)
      sx[q * 256 + e] = e < len ? static_cast<T>(xv[e]) : T(0);
  }
  __syncthreads();
  if (nsrc > 0) {
    if (!transpose) {  // D x: thread = (vector of VEC rows, column group)
      const int nvr = ld / VEC;
      const int rv = nvr <= 32 ? 32 : (nvr <= 64 ? 64 : 128);
      const int groups = OWN_T / rv;  // >= 1 (nvr <= 128 for len <= 256)
      const int r = threadIdx.x % rv, g = threadIdx.x / rv;
      T a[VEC];
#pragma unroll
      for (int q = 0; q < VEC; ++q) a[q] = T(0);
      if (r < nvr) {
        const int ldv = ld / VEC;
        const V* c0p = reinterpret_cast<const V*>(M0) + r;
        const V* c1p = reinterpret_cast<const V*>(M1 ? M1 : M0) + r;
        const T* sx1 = sx + (M1 ? 256 : 0);
        const T f1 = M1 ? T(1) : T(0);
        int c = g;
        for (; c + 3 * groups < len; c += 4 * groups) {  // eight 16-byte loads in flight
          V m[8];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            m[u] = c0p[(int64_t)(c + u * groups) * ldv];
            m[4 + u] = c1p[(int64_t)(c + u * groups) * ldv];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            vec_fma<T>(m[u], sx[c + u * groups], a);
            vec_fma<T>(m[4 + u], f1 * sx1[c + u * groups], a);
          }
        }
        for (; c < len; c += groups) {
          vec_fma<T>(c0p[(int64_t)c * ldv], sx[c], a);
          vec_fma<T>(c1p[(int64_t)c * ldv], f1 * sx1[c], a);
        }
      }
#pragma unroll
      for (int q = 0; q < VEC; ++q) red[g * (rv * VEC) + r * VEC + q] = a[q];
      __syncthreads();
      for (int row = threadIdx.x; row < len; row += blockDim.x) {
        double tot = 0.0;
        for (int q = 0; q < groups; ++q) tot += (double)red[q * (rv * VEC) + row];
        outv[row] += tot;
      }
    } else {  // D^T x: warp per column, both leaves
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      const int nvr = ld / VEC;
      for (int c = warp; c < len; c += OWN_T / 32) {
        const V* col0 = reinterpret_cast<const V*>(M0 + (int64_t)c * ld);
        T part = T(0);
        for (int v = lane; v < nvr; v += 32) part += vec_dot<T>(col0[v], sx + v * VEC);
        if (M1) {
          const V* col1 = reinterpret_cast<const V*>(M1 + (int64_t)c * ld);
          for (int v = lane; v < nvr; v += 32) part += vec_dot<T>(col1[v], sx + 256 + v * VEC);
        }
        const double sm = warp_sum((double)part);
        if (lane == 0) outv[c] += sm;
      }
    }
  }
  // the low-rank part needs t from k_h_inner: when launched as its programmatic dependent, this
  // kernel ran the dense part concurrently and waits here for the inner kernel's results
  pdl_wait();
  for (int e = threadIdx.x; e < NSL * HOWN_TCAP; e += blockDim.x) {
    const int q = e / HOWN_TCAP, c = e % HOWN_TCAP;
    const int s = q / HOWN_MAXL, l = q % HOWN_MAXL;
    const int hb = s < nsrc ? it->hb[s][l] : -1;
    if (hb >= 0 && c < bl[hb].rank) s_t[e] = static_cast<T>(t[bl[hb].t_off + c]);
  }
  __syncthreads();
  // W_out(rows, :) t_b of every low-rank block, one row per thread: the first eight columns of
  // a block are loaded together (one latency round per block), further columns in a tail loop
  for (int r = threadIdx.x; r < len; r += blockDim.x) {
    double a = 0.0;
    for (int q = 0; q < NSL; ++q) {
      const int rank = s_rank[q];
      if (rank == 0) continue;
      const T* W = UV + s_woff[q] + r;
      const int64_t nr = s_nr[q];
      const T* tq = s_t + q * HOWN_TCAP;
      T wv[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) wv[c] = c < rank ? W[(int64_t)c * nr] : T(0);
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < 8; ++c) acc = fma(wv[c], c < rank ? tq[c] : T(0), acc);
      for (int c = 8; c < rank; ++c) {
        T tc;
        if (c < HOWN_TCAP) {
          tc = tq[c];
        } else {
          const int hb = it->hb[q / HOWN_MAXL][q % HOWN_MAXL];
          tc = static_cast<T>(t[bl[hb].t_off + c]);
        }
        acc = fma(W[(int64_t)c * nr], tc, acc);
      }
      a += (double)acc;
    }
    outv[r] += a;
  }
  __syncthreads();
  const int64_t o = it->out + it->lo;
  for (int r = threadIdx.x; r < len; r += blockDim.x) y[o + r] = konly ? outv[r] : x[o + r] - outv[r];
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
void HodlrSet::clear() { release(); }

void HodlrSet::release() {
  for (void* p : {UV, D, (void*)t, (void*)d_blocks, (void*)d_leaves, (void*)d_own,
                  (void*)d_own_T})
    if (p) cudaFree(p);
  UV = D = nullptr;
  t = nullptr;
  d_blocks = nullptr;
  d_leaves = nullptr;
  d_own = d_own_T = nullptr;
  blocks.clear();
  leaves.clear();
  built = false;
  bytes = 0;
  max_rank = 0;
  n_own = n_own_T = 0;
}

static int levels_for(int64_t ng, int leaf) {
  int L = 0;
  while ((ng + (1LL << L) - 1) / (1LL << L) > leaf) ++L;
  return L;
}

template <typename T>
static void launch_sketch(int SC, const HItem* it, int n, const HDev* hb, const T* S, T* UV,
                          cudaStream_t st) {
  if (n == 0) return;
  switch (SC) {
    case 32: note_launch(); k_sketch<T, 32><<<n, 256, 0, st>>>(it, hb, S, UV); break;
    case 64: note_launch(); k_sketch<T, 64><<<n, 256, 0, st>>>(it, hb, S, UV); break;
    case 96: note_launch(); k_sketch<T, 96><<<n, 256, 0, st>>>(it, hb, S, UV); break;
    default: note_launch(); k_sketch<T, 128><<<n, 256, 0, st>>>(it, hb, S, UV); break;
  }
}

template <typename T>
static void launch_project(int SC, const HItem* it, int n, const HDev* hb, const int* rank,
                           const T* S, T* UV, cudaStream_t st) {
  if (n == 0) return;
  switch (SC) {
    case 16: note_launch(); k_project<T, 16><<<n, 256, 0, st>>>(it, hb, rank, S, UV); break;
    case 32: note_launch(); k_project<T, 32><<<n, 256, 0, st>>>(it, hb, rank, S, UV); break;
    case 64: note_launch(); k_project<T, 64><<<n, 256, 0, st>>>(it, hb, rank, S, UV); break;
    case 96: note_launch(); k_project<T, 96><<<n, 256, 0, st>>>(it, hb, rank, S, UV); break;
    default: note_launch(); k_project<T, 128><<<n, 256, 0, st>>>(it, hb, rank, S, UV); break;
  }
}

template <typename T>
int hodlr_build(HodlrSet& H, const HodlrParams& hp, const std::vector<SlabDesc>& slabs,
                const std::vector<ProbDesc>& probs, const SlabDesc* /*d_slabs*/, const T* S,
                cudaStream_t st, std::string& msg) {
  H.release();
  H.esz = sizeof(T);
  const int kmax = std::max(1, std::min(hp.k_max, 128));
  const int s_req = std::min(128, kmax + std::max(0, hp.oversample));
  const int leaf = std::max(8, std::min(256, hp.leaf));
  // S blocks
  std::vector<SBlk> sb;
  std::vector<int> sb_slab, sb_side;
  for (size_t si = 0; si < slabs.size(); ++si) {
    const SlabDesc& s = slabs[si];
    if (s.sp_off >= 0) { sb.push_back({s.sp_off, s.ng}); sb_slab.push_back((int)si); sb_side.push_back(-1); }
    if (s.sn_off >= 0) { sb.push_back({s.sn_off, s.ng}); sb_slab.push_back((int)si); sb_side.push_back(1); }
  }
  const int nsb = (int)sb.size();
  H.sblk_slab = sb_slab;
  H.sblk_side = sb_side;
  H.sblk_L.assign(nsb, 0);
  if (nsb == 0) { H.built = true; return 0; }
  int64_t max_ng = 0;
  for (auto& b : sb) max_ng = std::max(max_ng, b.ng);
  // blocks and leaves
  std::vector<HDev> hd;
  std::vector<int> sb_fb(nsb + 1), sb_fl(nsb);  // first block / first leaf of every S block
  int64_t uv = 0, dl = 0, tl = 0;
  for (int b = 0; b < nsb; ++b) {
    const SlabDesc& s = slabs[sb_slab[b]];
    const int64_t ng = sb[b].ng;
    const int L = levels_for(ng, leaf);
    if (L > HOWN_MAXL) { msg = "cluster tree deeper than 12 levels (raise leaf_size)"; return 3; }
    H.sblk_L[b] = L;
    sb_fb[b] = (int)H.blocks.size();
    sb_fl[b] = (int)H.leaves.size();
    const int64_t in_if = s.if_off + (sb_side[b] < 0 ? -ng : ng), out_if = s.if_off;
    for (int lev = 1; lev <= L; ++lev) {
      for (int64_t t = 0; t < (1LL << (lev - 1)); ++t) {
        const int64_t lo1 = ((2 * t) * ng) >> lev, hi1 = ((2 * t + 1) * ng) >> lev;
        const int64_t lo2 = hi1, hi2 = ((2 * t + 2) * ng) >> lev;
        const int64_t rr[2][4] = {{lo1, hi1, lo2, hi2}, {lo2, hi2, lo1, hi1}};
        for (int e = 0; e < 2; ++e) {
          HBlock k{};
          k.sblk = b;
          k.level = lev;
          k.row0 = rr[e][0]; k.nrows = rr[e][1] - rr[e][0];
          k.col0 = rr[e][2]; k.ncols = rr[e][3] - rr[e][2];
          const int sc = (int)std::min<int64_t>(s_req, std::min(k.nrows, k.ncols));
          k.u_off = uv; uv += k.nrows * sc;
          k.v_off = uv; uv += k.ncols * sc;
          k.t_off = tl; tl += sc;
          k.in_if = in_if; k.out_if = out_if;
          k.rank = sc;  // capacity until compressed
          H.blocks.push_back(k);
          HDev d{};
          d.s_off = sb[b].off + k.col0 * ng + k.row0;
          d.ng = ng; d.p = k.nrows; d.q = k.ncols; d.s = sc; d.sblk = b;
          d.u_off = k.u_off; d.v_off = k.v_off;
          hd.push_back(d);
        }
      }
    }
    for (int64_t t = 0; t < (1LL << L); ++t) {
      HLeaf lf{};
      lf.sblk = b;
      lf.lo = (t * ng) >> L;
      lf.len = (((t + 1) * ng) >> L) - lf.lo;
      lf.ld = (lf.len + 3) / 4 * 4;
      lf.d_off = dl; dl += lf.ld * lf.len;
      lf.in_if = in_if; lf.out_if = out_if;
      H.leaves.push_back(lf);
    }
  }
  const int nblk = (int)H.blocks.size();
  sb_fb[nsb] = nblk;
  // device memory
  auto al = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes < 16 ? 16 : bytes) != cudaSuccess) { cudaGetLastError(); return false; }
    return true;
  };
  SBlk* d_sb = nullptr; double *d_x = nullptr, *d_y = nullptr, *d_nrm = nullptr;
  HDev* d_hd = nullptr; HItem *d_items = nullptr; int* d_rank = nullptr;
  int64_t *d_soff = nullptr, *d_sng = nullptr;
  const int64_t stride = max_ng;
  bool ok = al(&H.UV, sizeof(T) * uv) && al(&H.D, sizeof(T) * dl) && al((void**)&H.t, sizeof(double) * tl) &&
            al((void**)&H.d_blocks, sizeof(HBlock) * nblk) &&
            al((void**)&H.d_leaves, sizeof(HLeaf) * H.leaves.size()) &&
            al((void**)&d_sb, sizeof(SBlk) * nsb) && al((void**)&d_x, sizeof(double) * stride * nsb) &&
            al((void**)&d_y, sizeof(double) * stride * nsb) && al((void**)&d_nrm, sizeof(double) * nsb) &&
            al((void**)&d_hd, sizeof(HDev) * nblk) && al((void**)&d_rank, sizeof(int) * nblk) &&
            al((void**)&d_soff, sizeof(int64_t) * nsb) && al((void**)&d_sng, sizeof(int64_t) * nsb);
  auto cleanup = [&]() {
    for (void* p : {(void*)d_sb, (void*)d_x, (void*)d_y, (void*)d_nrm, (void*)d_hd, (void*)d_items,
                    (void*)d_rank, (void*)d_soff, (void*)d_sng})
      if (p) cudaFree(p);
  };
  if (!ok) { cleanup(); H.release(); msg = "out of device memory"; return 2; }
  std::vector<int64_t> soff(nsb), sng(nsb);
  for (int b = 0; b < nsb; ++b) { soff[b] = sb[b].off; sng[b] = sb[b].ng; }
  cudaMemcpyAsync(d_sb, sb.data(), sizeof(SBlk) * nsb, cudaMemcpyHostToDevice, st);
  // a tree without low-rank levels (n_Gamma <= leaf) has only dense leaves: no sketch below
  if (nblk > 0) cudaMemcpyAsync(d_hd, hd.data(), sizeof(HDev) * nblk, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_soff, soff.data(), sizeof(int64_t) * nsb, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_sng, sng.data(), sizeof(int64_t) * nsb, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(H.d_leaves, H.leaves.data(), sizeof(HLeaf) * H.leaves.size(), cudaMemcpyHostToDevice, st);
  // ||S||_2 by power iteration on S^T S (2 steps; an underestimate only lowers the truncation
  // threshold, i.e. errs towards higher ranks)
  note_launch();
  k_sblk_init<<<nsb, 256, 0, st>>>(d_sb, d_x, stride, hp.seed ^ 0x9e3779b97f4a7c15ull);
  const unsigned gr = (unsigned)((max_ng + 255) / 256);
  const unsigned gz = (unsigned)((max_ng + 127) / 128);
  for (int itp = 0; itp < 2; ++itp) {
    cudaMemsetAsync(d_y, 0, sizeof(double) * stride * nsb, st);
    note_launch(3);
    k_sblk_gemv<T><<<dim3(gr, nsb, gz), 256, 0, st>>>(d_sb, S, d_x, d_y, stride);
    k_sblk_gemv_t<T><<<dim3(gz, nsb), 256, 0, st>>>(d_sb, S, d_y, d_x, stride);
    k_sblk_normalize<<<nsb, 256, 0, st>>>(d_sb, d_x, d_x, stride, d_nrm);
  }
  // d_nrm now holds ||S^T S x|| ~ sigma_max^2
  // sketches
  int SC = 32;
  while (SC < s_req) SC += 32;
  std::vector<HItem> items;
  for (int b = 0; b < nblk; ++b)
    for (int64_t lo = 0; lo < hd[b].p; lo += 64) items.push_back({b, lo});
  std::vector<HItem> pitems;
  for (int b = 0; b < nblk; ++b)
    for (int64_t lo = 0; lo < hd[b].q; lo += 64) pitems.push_back({b, lo});
  const size_t nit = std::max(items.size(), pitems.size());
  if (!al((void**)&d_items, sizeof(HItem) * nit)) { cleanup(); H.release(); msg = "oom"; return 2; }
  if (nblk > 0) {
    note_launch();
    k_gen_omega<T><<<dim3(32, nblk), 256, 0, st>>>(d_hd, (T*)H.UV, hp.seed);
    cudaMemcpyAsync(d_items, items.data(), sizeof(HItem) * items.size(), cudaMemcpyHostToDevice, st);
    launch_sketch<T>(SC, d_items, (int)items.size(), d_hd, S, (T*)H.UV, st);
  }
  // sigma estimate: sqrt of the Rayleigh quotient norm
  std::vector<double> nrm(nsb);
  cudaMemcpyAsync(nrm.data(), d_nrm, sizeof(double) * nsb, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  for (auto& v : nrm) v = std::sqrt(std::max(v, 0.0));
  cudaMemcpyAsync(d_nrm, nrm.data(), sizeof(double) * nsb, cudaMemcpyHostToDevice, st);
  if (nblk > 0) {
    int64_t maxp = 0;
    for (auto& d : hd) maxp = std::max(maxp, d.p);
    const size_t smem = sizeof(T) * maxp;
    raise_smem_limit(reinterpret_cast<const void*>(&k_range_cgs2<T>), smem);
    note_launch();
    k_range_cgs2<T><<<nblk, 512, smem, st>>>(d_hd, (T*)H.UV, d_nrm, hp.tol, kmax,
                                             std::max(1, hp.oversample), d_rank);
  }
  // the projection is instantiated for the largest detected rank, not the sample capacity
  std::vector<int> ranks(nblk);
  if (nblk > 0) {
    cudaMemcpyAsync(ranks.data(), d_rank, sizeof(int) * nblk, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    int maxr = 0;
    for (int v : ranks) maxr = std::max(maxr, v);
    const int SCp = maxr <= 16 ? 16 : (maxr <= 32 ? 32 : (maxr <= 64 ? 64 : (maxr <= 96 ? 96 : 128)));
    cudaMemcpyAsync(d_items, pitems.data(), sizeof(HItem) * pitems.size(), cudaMemcpyHostToDevice, st);
    if (maxr > 0) launch_project<T>(SCp, d_items, (int)pitems.size(), d_hd, d_rank, S, (T*)H.UV, st);
  }
  note_launch();
  k_copy_leaves<T><<<dim3(16, (unsigned)H.leaves.size()), 256, 0, st>>>(H.d_leaves, d_soff, d_sng, S,
                                                                       (T*)H.D);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  cleanup();
  if (e != cudaSuccess) { msg = cudaGetErrorString(e); H.release(); return 1; }
  int64_t used = 0;
  for (int b = 0; b < nblk; ++b) {
    H.blocks[b].rank = ranks[b];
    H.max_rank = std::max(H.max_rank, ranks[b]);
    used += (H.blocks[b].nrows + H.blocks[b].ncols) * ranks[b];
  }
  H.bytes = (used + dl) * (int64_t)sizeof(T);
  H.t_len = tl;
  if (nblk > 0)
    cudaMemcpyAsync(H.d_blocks, H.blocks.data(), sizeof(HBlock) * nblk, cudaMemcpyHostToDevice, st);
  // output-owner items: one per (interface, leaf row range), for the plain and transposed apply
  std::vector<HOwn> own[2];
  {
    std::map<int64_t, std::vector<int>> by_if[2];  // S blocks writing an interface: out_if / in_if
    for (int b = 0; b < nsb; ++b) {
      by_if[0][H.leaves[sb_fl[b]].out_if].push_back(b);
      by_if[1][H.leaves[sb_fl[b]].in_if].push_back(b);
    }
    const std::vector<int> none;
    for (const ProbDesc& P : probs) {
      const int L = levels_for(P.ng, leaf);
      for (int j = 0; j < P.nds; ++j) {
        const int64_t iface = P.if_off + (int64_t)j * P.ng;
        for (int tr = 0; tr < 2; ++tr) {
          const auto f = by_if[tr].find(iface);
          const std::vector<int>& src = f == by_if[tr].end() ? none : f->second;
          if (src.size() > 2) { msg = "more than two S blocks write one interface"; H.release(); return 1; }
          for (int64_t tt = 0; tt < (1LL << L); ++tt) {
            HOwn o{};
            o.out = iface;
            o.lo = (tt * P.ng) >> L;
            o.len = (int)((((tt + 1) * P.ng) >> L) - o.lo);
            o.nsrc = (int)src.size();
            for (int q = 0; q < o.nsrc; ++q) {
              const int b = src[q];
              o.leaf[q] = sb_fl[b] + (int)tt;
              for (int l = 0; l < HOWN_MAXL; ++l) o.hb[q][l] = -1;
              for (int bi = sb_fb[b]; bi < sb_fb[b + 1]; ++bi) {
                const HBlock& B = H.blocks[bi];
                const int64_t a0 = tr ? B.col0 : B.row0, an = tr ? B.ncols : B.nrows;
                if (B.rank > 0 && o.lo >= a0 && o.lo < a0 + an) o.hb[q][B.level - 1] = bi;
              }
            }
            own[tr].push_back(o);
          }
        }
      }
    }
  }
  H.n_own = (int)own[0].size();
  H.n_own_T = (int)own[1].size();
  if (!al((void**)&H.d_own, sizeof(HOwn) * std::max<size_t>(1, own[0].size())) ||
      !al((void**)&H.d_own_T, sizeof(HOwn) * std::max<size_t>(1, own[1].size()))) {
    H.release(); msg = "oom"; return 2;
  }
  for (int tr = 0; tr < 2; ++tr)
    if (!own[tr].empty())
      cudaMemcpyAsync(tr ? H.d_own_T : H.d_own, own[tr].data(), sizeof(HOwn) * own[tr].size(),
                      cudaMemcpyHostToDevice, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { msg = cudaGetErrorString(e); H.release(); return 1; }
  H.built = true;
  return 0;
}

template <typename T>
void hodlr_apply(HodlrSet& H, const SlabDesc*, const ProbDesc*, int, const double* x, double* y,
                 int transpose, cudaStream_t st, const int* kdev, int64_t kstride) {
  const int konly = transpose >> 1;  // bit 1: y = K x (or K^T x) instead of (I - K) x
  transpose &= 1;
  if (!H.blocks.empty()) {
    note_launch();
    const int nblk = (int)H.blocks.size();
    k_h_inner<T><<<(nblk + 7) / 8, 256, 0, st>>>(H.d_blocks, nblk, (const T*)H.UV, x, H.t,
                                                 transpose, kdev, kstride);
  }
  const int no = transpose ? H.n_own_T : H.n_own;
  if (no > 0) {
    // programmatic dependent of k_h_inner: the dense leaves stream while the inner products run
    note_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(no);
    cfg.blockDim = dim3(OWN_T);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = H.blocks.empty() ? 0 : 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_h_owner<T>, (const HOwn*)(transpose ? H.d_own_T : H.d_own),
                       (const HBlock*)H.d_blocks, (const HLeaf*)H.d_leaves, (const T*)H.UV,
                       (const T*)H.D, (const double*)H.t, x, y, transpose, konly, kdev, kstride);
  }
}

int hodlr_expand(HodlrSet& H, int slab, int side, size_t esz, double* out, cudaStream_t st) {
  int sbk = -1;
  for (size_t b = 0; b < H.sblk_slab.size(); ++b)
    if (H.sblk_slab[b] == slab && H.sblk_side[b] == side) sbk = (int)b;
  if (sbk < 0) return 1;
  auto fetch = [&](const void* base, int64_t off, int64_t n, std::vector<double>& dst) {
    dst.resize(n);
    if (esz == 8) {
      cudaMemcpyAsync(dst.data(), (const double*)base + off, sizeof(double) * n,
                      cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
    } else {
      std::vector<float> tmp(n);
      cudaMemcpyAsync(tmp.data(), (const float*)base + off, sizeof(float) * n,
                      cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      for (int64_t e = 0; e < n; ++e) dst[e] = tmp[e];
    }
  };
  int64_t ng = 0;
  for (auto& lf : H.leaves)
    if (lf.sblk == sbk) ng = std::max(ng, lf.lo + lf.len);
  std::fill(out, out + ng * ng, 0.0);
  std::vector<double> U, V, Dm;
  for (auto& b : H.blocks) {
    if (b.sblk != sbk || b.rank == 0) continue;
    fetch(H.UV, b.u_off, b.nrows * b.rank, U);
    fetch(H.UV, b.v_off, b.ncols * b.rank, V);
    for (int64_t c = 0; c < b.ncols; ++c)
      for (int64_t r = 0; r < b.nrows; ++r) {
        double a = 0.0;
        for (int k = 0; k < b.rank; ++k) a += U[k * b.nrows + r] * V[k * b.ncols + c];
        out[(b.col0 + c) * ng + b.row0 + r] = a;
      }
  }
  for (auto& lf : H.leaves) {
    if (lf.sblk != sbk) continue;
    fetch(H.D, lf.d_off, lf.ld * lf.len, Dm);
    for (int64_t c = 0; c < lf.len; ++c)
      for (int64_t r = 0; r < lf.len; ++r) out[(lf.lo + c) * ng + lf.lo + r] = Dm[c * lf.ld + r];
  }
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template int hodlr_build<float>(HodlrSet&, const HodlrParams&, const std::vector<SlabDesc>&,
                                const std::vector<ProbDesc>&, const SlabDesc*, const float*,
                                cudaStream_t, std::string&);
template int hodlr_build<double>(HodlrSet&, const HodlrParams&, const std::vector<SlabDesc>&,
                                 const std::vector<ProbDesc>&, const SlabDesc*, const double*,
                                 cudaStream_t, std::string&);
template void hodlr_apply<float>(HodlrSet&, const SlabDesc*, const ProbDesc*, int, const double*,
                                 double*, int, cudaStream_t, const int*, int64_t);
template void hodlr_apply<double>(HodlrSet&, const SlabDesc*, const ProbDesc*, int, const double*,
                                  double*, int, cudaStream_t, const int*, int64_t);

}  // namespace ddst
