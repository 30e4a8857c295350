// krylov.cu -- interface operator application and the GMRES building blocks.
//
// The equilibrium system (I - K) u = fhat (Sec. 1, Eq. (modelS); Sec. 2.2, Eq. (equilib2)):
// block row j reads  u_j - S_{j,j-1} u_{j-1} - S_{j,j+1} u_{j+1}.  It is solved by unrestarted
// GMRES (Sec. 5): Arnoldi with classical Gram-Schmidt applied twice, Givens rotations, x0 = 0.
// Krylov vectors are FP64; the operator's blocks are stored in the working precision T and
// multiplied in T with FP64 accumulation every 32 terms.
#include "kernels.cuh"

namespace ddst {

// y_j = x_j - S_{j,j-1} x_{j-1} - S_{j,j+1} x_{j+1} (konly: y_j = S_{j,j-1} x_{j-1} + S_{j,j+1}
// x_{j+1}, i.e. y = K x); S column-major.  grid = (row tiles of 128, slabs); 256 threads = 128
// rows x 2 interleaved halves of the sources.
template <typename T>
__global__ void __launch_bounds__(256) k_apply_dense(const SlabDesc* __restrict__ slabs,
                                                     const ProbDesc* __restrict__ probs,
                                                     const T* __restrict__ S,
                                                     const double* __restrict__ x0,
                                                     double* __restrict__ y, const int* kdev,
                                                     int64_t kstride, int konly) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const double* x = x0 + (kdev ? (int64_t)(*kdev - 1) * kstride : 0);
  const SlabDesc s = slabs[blockIdx.y];
  const ProbDesc P = probs[s.prob];
  const int64_t ng = s.ng;
  if ((int64_t)blockIdx.x * 128 >= ng) return;
  T* xp = reinterpret_cast<T*>(smem_raw);
  T* xn = xp + ng;
  __shared__ double red[256];
  const bool hp = s.j >= 2, hn = s.j <= P.nds - 1;
  for (int64_t e = threadIdx.x; e < ng; e += blockDim.x) {
    xp[e] = hp ? static_cast<T>(x[s.if_off - ng + e]) : T(0);
    xn[e] = hn ? static_cast<T>(x[s.if_off + ng + e]) : T(0);
  }
  __syncthreads();
  const int64_t row = (int64_t)blockIdx.x * 128 + (threadIdx.x & 127);
  const int half = threadIdx.x >> 7;
  double acc = 0.0;
  if (row < ng) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int64_t off = side == 0 ? s.sp_off : s.sn_off;
      if (off < 0) continue;
      const T* col = S + off + row;
      const T* xs = side == 0 ? xp : xn;
      int64_t src = half;
      while (src < ng) {
        T p0 = T(0), p1 = T(0), p2 = T(0), p3 = T(0);
        const int64_t stop = min(ng, src + 64);
        for (; src + 6 < stop; src += 8) {
          p0 = fma(col[src * ng], xs[src], p0);
          p1 = fma(col[(src + 2) * ng], xs[src + 2], p1);
          p2 = fma(col[(src + 4) * ng], xs[src + 4], p2);
          p3 = fma(col[(src + 6) * ng], xs[src + 6], p3);
        }
        for (; src < stop; src += 2) p0 = fma(col[src * ng], xs[src], p0);
        acc += static_cast<double>(p0) + static_cast<double>(p1) + static_cast<double>(p2) +
               static_cast<double>(p3);
      }
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (half == 0 && row < ng)
    y[s.if_off + row] = konly ? red[threadIdx.x] + red[threadIdx.x + 128]
                              : x[s.if_off + row] - (red[threadIdx.x] + red[threadIdx.x + 128]);
}

// y_j = x_j - S_{j+1,j}^T x_{j+1} - S_{j-1,j}^T x_{j-1} (konly: y = K^T x).  S is stored by
// columns, so (S^T x)_c is a dot product down column c.  A CTA owns 128 output points (columns)
// and streams its columns through shared memory in 32-row tiles: warp w loads 16 columns of a
// tile, one coalesced 32-row segment each (16 independent loads in flight per warp), and the 256
// threads (128 columns x 2 row halves) then take 16 terms each from the transposed tile, partial
// sums in the working precision added into FP64 per tile.  The neighbouring traces are staged
// once in shared memory.  grid = (ceil(ng/128), slabs), 256 threads, dynamic shared memory
// 2 max_ng + 128 x 33 elements.  (A warp per column reading the traces from global memory was
// bound by the L1 request queue at a tenth of the forward apply's bandwidth.)
template <typename T>
__global__ void __launch_bounds__(256) k_apply_dense_T(const SlabDesc* __restrict__ slabs,
                                                       const ProbDesc* __restrict__ probs,
                                                       const T* __restrict__ S,
                                                       const double* __restrict__ x0,
                                                       double* __restrict__ y, const int* kdev,
                                                       int64_t kstride, int konly,
                                                       int64_t max_ng) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const double* x = x0 + (kdev ? (int64_t)(*kdev - 1) * kstride : 0);
  const int sidx = blockIdx.y;
  const SlabDesc& s = slabs[sidx];
  const int64_t ng = s.ng, if_off = s.if_off;
  const int64_t c0 = (int64_t)blockIdx.x * 128;
  if (c0 >= ng) return;  // uniform over the CTA
  const int j = s.j, nds = probs[s.prob].nds;
  // slab j+1 maps Gamma_j -> Gamma_{j+1} through its S_{j+1,j}; a neighbour without explicit
  // blocks (a class applied matrix-free, offset -1) contributes nothing here
  const int64_t offs[2] = {j <= nds - 1 ? slabs[sidx + 1].sp_off : -1,
                           j >= 2 ? slabs[sidx - 1].sn_off : -1};
  T* xs0 = reinterpret_cast<T*>(smem_raw);  // Gamma_{j+1}
  T* xs1 = xs0 + max_ng;                     // Gamma_{j-1}
  T* tile = xs1 + max_ng;                    // [128][33]: column, row within the tile
  for (int64_t e = threadIdx.x; e < ng; e += blockDim.x) {
    xs0[e] = offs[0] >= 0 ? static_cast<T>(x[if_off + ng + e]) : T(0);
    xs1[e] = offs[1] >= 0 ? static_cast<T>(x[if_off - ng + e]) : T(0);
  }
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int cl = tid & 127, half = tid >> 7;
  double acc = 0.0;
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    const int64_t off = offs[side];
    if (off < 0) continue;  // uniform
    const T* xs = side == 0 ? xs0 : xs1;
#pragma unroll 1
    for (int64_t r0 = 0; r0 < ng; r0 += 32) {
      __syncthreads();  // the staged traces (first pass) / the previous tile's readers
      const int64_t r = r0 + lane;
#pragma unroll
      for (int cc = 0; cc < 16; ++cc) {
        const int64_t c = c0 + warp * 16 + cc;
        tile[(warp * 16 + cc) * 33 + lane] = (c < ng && r < ng) ? S[off + c * ng + r] : T(0);
      }
      __syncthreads();
      T p = T(0);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int rr = half * 16 + i;
        p = fma(tile[cl * 33 + rr], r0 + rr < ng ? xs[r0 + rr] : T(0), p);
      }
      acc += static_cast<double>(p);
    }
  }
  __syncthreads();
  double* red = reinterpret_cast<double*>(tile);  // 256 doubles fit in the tile's space
  red[tid] = acc;
  __syncthreads();
  const int64_t c = c0 + cl;
  if (half == 0 && c < ng) {
    const double v = red[tid] + red[tid + 128];
    y[if_off + c] = konly ? v : x[if_off + c] - v;
  }
}

// GMRES solution from the Krylov basis: x = sum_{i<k} y[i] V[i]
__global__ void k_combine_basis(const double* __restrict__ V, double* __restrict__ x,
                                const double* __restrict__ h, int k, int64_t n) {
  extern __shared__ double sh[];
  for (int i = threadIdx.x; i < k; i += blockDim.x) sh[i] = h[i];
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    int i = 0;
    for (; i + 3 < k; i += 4) {
      acc += sh[i] * V[(int64_t)i * n + e] + sh[i + 1] * V[(int64_t)(i + 1) * n + e] +
             sh[i + 2] * V[(int64_t)(i + 2) * n + e] + sh[i + 3] * V[(int64_t)(i + 3) * n + e];
    }
    for (; i < k; ++i) acc += sh[i] * V[(int64_t)i * n + e];
    x[e] = acc;
  }
}

// out = x / sqrt(nrm2[0]) and gv[0] = sqrt(nrm2[0])  (start of Arnoldi)
__global__ void k_normalize_start(const double* __restrict__ x, const double* __restrict__ nrm2,
                                  double* __restrict__ out, int64_t n) {
  const double nr = sqrt(nrm2[0]);
  const double a = nr > 0.0 ? 1.0 / nr : 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = a * x[e];
}

// Back substitution R y = g (R column-major upper triangle, kk x kk).  One CTA.
__global__ void k_trisolve(const double* __restrict__ H, int ldh, const double* __restrict__ gv,
                           int kk, double* __restrict__ y) {
  extern __shared__ double rhs[];
  for (int i = threadIdx.x; i < kk; i += blockDim.x) rhs[i] = gv[i];
  __syncthreads();
  for (int i = kk - 1; i >= 0; --i) {
    const double* col = H + (int64_t)i * ldh;
    const double yi = rhs[i] / col[i];
    __syncthreads();
    for (int l = threadIdx.x; l < i; l += blockDim.x) rhs[l] -= col[l] * yi;
    if (threadIdx.x == 0) y[i] = yi;
    __syncthreads();
  }
}

// ---- Arnoldi step with device-resident state (graph-capturable) ---------------------------
// State: *kdev = k basis vectors V[0..k) exist; w = (I - K) V[k-1] has just been formed.  One
// step is classical Gram-Schmidt with selective reorthogonalization (a second pass only when the
// first one cancels more than half of ||w||^2: Kahan-Parlett, "twice is enough"), the Givens
// update of the least-squares problem and the normalization V[k] = w / ||w||:
//   dots   : P1[i][c] = V[i] . w over chunk c (i < k), P1[k][c] = |w|^2 over chunk c
//   update : h1 = sum_c P1;  w -= V h1;  second pass needed iff |w|^2 - |h1|^2 < |w|^2 / 2
//            (flag kdev[1]); then P2[i][c] = V[i] . w, or Pn[c] = |w|^2 if no second pass
//   update : if the flag is set, h2 = sum_c P2;  w -= V h2;  Pn[c] = |w|^2; else h2 = 0
//   finish : V[k] = w / sqrt(sum_c Pn); the last CTA to finish applies the Givens rotations to
//            the new column of the Hessenberg matrix of (I - K) and advances *kdev.
// The Arnoldi process runs on K itself (w = K V[k-1]): K and I - K span the same Krylov spaces,
// and (I - K) V_k = V_{k+1} (I~ - Hbar_K) with I~ the identity padded by a zero row, so column
// k-1 of the (I - K) matrix is e_{k-1} - (h1 + h2) with subdiagonal -||w||.  On K the first
// Gram-Schmidt pass rarely cancels half of ||w|| (on I - K it always would, through the
// V[k-1] component), so the second pass is mostly skipped.
// Partial sums are stored per chunk (i-major, coalesced for the readers) and reduced by each
// consumer CTA: no two CTAs update the same address.
constexpr int ARN_T = 256, ARN_E = 4, ARN_CHUNK = ARN_T * ARN_E, ARN_G = 8;

// sh[i] = sum_c P[i * nchunk + c] for i < k (every thread of the CTA takes part).  A warp sums
// two rows per round; each lane issues its loads of a 128-chunk window together (predicated,
// independent), so a round costs one L2 latency for up to 128 chunks.
__device__ __forceinline__ void arn_reduce(const double* __restrict__ P, int nchunk, int k,
                                           double* __restrict__ sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int W = ARN_T / 32;
  for (int i = warp; i < k; i += 2 * W) {
    const int i2 = i + W;
    const double* r1 = P + (int64_t)i * nchunk;
    const double* r2 = P + (int64_t)(i2 < k ? i2 : i) * nchunk;
    double a[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) a[q] = 0.0;
    for (int c0 = 0; c0 < nchunk; c0 += 128) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = c0 + q * 32 + lane;
        a[q] += c < nchunk ? r1[c] : 0.0;
        a[4 + q] += c < nchunk ? r2[c] : 0.0;
      }
    }
    const double s1 = warp_sum((a[0] + a[1]) + (a[2] + a[3]));
    const double s2 = warp_sum((a[4] + a[5]) + (a[6] + a[7]));
    if (lane == 0) {
      sh[i] = s1;
      if (i2 < k) sh[i2] = s2;
    }
  }
  __syncthreads();
}

// P[i * nchunk + blockIdx.x] = V[i] . wv over this CTA's chunk, for i < k, ARN_G vectors at once.
__device__ __forceinline__ void arn_chunk_dots(const double* __restrict__ V, int64_t n, int k,
                                               int64_t base, const double (&wv)[ARN_E],
                                               double* __restrict__ P, int nchunk) {
  __shared__ double red[2][ARN_T / 32][ARN_G];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int buf = 0;
  for (int i0 = 0; i0 < k; i0 += ARN_G, buf ^= 1) {
    double acc[ARN_G];
#pragma unroll
    for (int g = 0; g < ARN_G; ++g) acc[g] = 0.0;
#pragma unroll
    for (int g = 0; g < ARN_G; ++g) {
      if (i0 + g < k) {
        const double* v = V + (int64_t)(i0 + g) * n;
#pragma unroll
        for (int e = 0; e < ARN_E; ++e) {
          const int64_t idx = base + e * ARN_T + threadIdx.x;
          if (idx < n) acc[g] = fma(v[idx], wv[e], acc[g]);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < ARN_G; ++g) {
      const double t = warp_sum(acc[g]);
      if (lane == 0) red[buf][warp][g] = t;
    }
    __syncthreads();
    if (threadIdx.x < ARN_G && i0 + threadIdx.x < k) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < ARN_T / 32; ++q) t += red[buf][q][threadIdx.x];
      P[(int64_t)(i0 + threadIdx.x) * nchunk + blockIdx.x] = t;
    }
  }
}

__device__ __forceinline__ void arn_load_chunk(const double* __restrict__ w, int64_t n,
                                               int64_t base, double (&wv)[ARN_E]) {
#pragma unroll
  for (int e = 0; e < ARN_E; ++e) {
    const int64_t idx = base + e * ARN_T + threadIdx.x;
    wv[e] = idx < n ? w[idx] : 0.0;
  }
}

// wv -= sum_{i<k} h[i] V[i] over this CTA's chunk, ARN_G vectors at once.
__device__ __forceinline__ void arn_chunk_update(const double* __restrict__ V, int64_t n, int k,
                                                 int64_t base, const double* __restrict__ h,
                                                 double (&wv)[ARN_E]) {
  for (int i0 = 0; i0 < k; i0 += ARN_G) {
    double vv[ARN_G][ARN_E];
#pragma unroll
    for (int g = 0; g < ARN_G; ++g) {
      const double* v = V + (int64_t)(i0 + g) * n;
#pragma unroll
      for (int e = 0; e < ARN_E; ++e) {
        const int64_t idx = base + e * ARN_T + threadIdx.x;
        vv[g][e] = (i0 + g < k && idx < n) ? v[idx] : 0.0;
      }
    }
#pragma unroll
    for (int g = 0; g < ARN_G; ++g) {
      const double hg = i0 + g < k ? h[i0 + g] : 0.0;
#pragma unroll
      for (int e = 0; e < ARN_E; ++e) wv[e] = fma(-hg, vv[g][e], wv[e]);
    }
  }
}

// First-pass dots: the chunk of w is staged in shared memory and each warp takes whole basis
// vectors (warp q: vectors q, q + 8, ...), 32 loads in flight per lane and one warp reduction
// per vector, no block barrier inside the loop.
__global__ void __launch_bounds__(ARN_T) k_arn_dots(const double* __restrict__ V,
                                                    const double* __restrict__ w, int64_t n,
                                                    const int* __restrict__ kdev,
                                                    double* __restrict__ P1, int nchunk) {
  __shared__ double sw[ARN_CHUNK];
  const int k = *kdev;
  const int64_t base = (int64_t)blockIdx.x * ARN_CHUNK;
  double wv[ARN_E];
  arn_load_chunk(w, n, base, wv);
#pragma unroll
  for (int e = 0; e < ARN_E; ++e) sw[e * ARN_T + threadIdx.x] = wv[e];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t len = n - base < ARN_CHUNK ? n - base : ARN_CHUNK;
  for (int i = warp; i < k; i += ARN_T / 32) {
    const double* v = V + (int64_t)i * n + base;
    double acc = 0.0;
    if (len == ARN_CHUNK) {
      double a4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int e = 0; e < ARN_CHUNK / 32; ++e)
        a4[e & 3] = fma(v[e * 32 + lane], sw[e * 32 + lane], a4[e & 3]);
      acc = (a4[0] + a4[1]) + (a4[2] + a4[3]);
    } else {
      for (int64_t e = lane; e < len; e += 32) acc = fma(v[e], sw[e], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) P1[(int64_t)i * nchunk + blockIdx.x] = acc;
  }
  double acc = 0.0;  // |w|^2 over the chunk, row k of P1
#pragma unroll
  for (int e = 0; e < ARN_E; ++e) acc = fma(wv[e], wv[e], acc);
  __shared__ double red[ARN_T / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < ARN_T / 32 ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) P1[(int64_t)k * nchunk + blockIdx.x] = t;
  }
}

// h = sum_c Pin (CTA 0 also stores it in hout); w -= V h; then P2 = V . w or Pn[c] = |w|^2 over
// the chunk.  first = 1: the first pass, which also decides (identically in every CTA) whether
// a second pass is needed and publishes that in kdev[1]; first = 0: the second pass, skipped
// (h = 0) when kdev[1] is clear.
__global__ void __launch_bounds__(ARN_T) k_arn_update(const double* __restrict__ V,
                                                      double* __restrict__ w, int64_t n,
                                                      int* __restrict__ kdev,
                                                      const double* __restrict__ Pin,
                                                      double* __restrict__ hout,
                                                      double* __restrict__ Pout,
                                                      double* __restrict__ Pn, int nchunk,
                                                      int first) {
  __shared__ double sh[1024 + 1];
  const int k = *kdev;
  if (!first && kdev[1] == 0) {  // no second pass: h2 = 0, Pn already holds |w|^2
    if (blockIdx.x == 0)
      for (int i = threadIdx.x; i < k; i += ARN_T) hout[i] = 0.0;
    return;
  }
  arn_reduce(Pin, nchunk, first ? k + 1 : k, sh);
  bool dots = false;
  if (first) {
    double hn = 0.0;
    for (int i = 0; i < k; ++i) hn = fma(sh[i], sh[i], hn);
    dots = sh[k] - hn < 0.5 * sh[k];  // lost more than half of |w|^2: reorthogonalize
    if (blockIdx.x == 0 && threadIdx.x == 0) kdev[1] = dots ? 1 : 0;
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < k; i += ARN_T) hout[i] = sh[i];
  const int64_t base = (int64_t)blockIdx.x * ARN_CHUNK;
  double wv[ARN_E];
  arn_load_chunk(w, n, base, wv);
  arn_chunk_update(V, n, k, base, sh, wv);
#pragma unroll
  for (int e = 0; e < ARN_E; ++e) {
    const int64_t idx = base + e * ARN_T + threadIdx.x;
    if (idx < n) w[idx] = wv[e];
  }
  if (dots) {
    arn_chunk_dots(V, n, k, base, wv, Pout, nchunk);
  } else {
    double acc = 0.0;
#pragma unroll
    for (int e = 0; e < ARN_E; ++e) acc = fma(wv[e], wv[e], acc);
    __shared__ double red[ARN_T / 32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      double t = threadIdx.x < ARN_T / 32 ? red[threadIdx.x] : 0.0;
      t = warp_sum(t);
      if (threadIdx.x == 0) Pn[blockIdx.x] = t;
    }
  }
}

// V[k] = w / ||w|| over this CTA's chunk (0 at breakdown).  The last CTA to get here (atomic
// ticket after a fence; nothing waits) applies the previous Givens rotations to the new column
// e_{k-1} - (h1 + h2) (subdiagonal -||w||), forms the new one, records the residual estimate
// and advances *kdev.
__global__ void __launch_bounds__(ARN_T) k_arn_finish(double* __restrict__ V,
                                                      const double* __restrict__ w, int64_t n,
                                                      int* __restrict__ kdev,
                                                      const double* __restrict__ Pn, int nchunk,
                                                      const double* __restrict__ h1,
                                                      const double* __restrict__ h2,
                                                      double* __restrict__ H, int ldh,
                                                      double* __restrict__ cs,
                                                      double* __restrict__ sn,
                                                      double* __restrict__ gv,
                                                      const double* __restrict__ beta,
                                                      double* __restrict__ resid, int kmax,
                                                      unsigned* __restrict__ ticket) {
  __shared__ double s_hn2;
  __shared__ bool s_last;
  const int k = *kdev;
  if (threadIdx.x < 32) {
    double a = 0.0;
    for (int c = threadIdx.x; c < nchunk; c += 32) a += Pn[c];
    a = warp_sum(a);
    if (threadIdx.x == 0) s_hn2 = a;
  }
  __syncthreads();
  const double sub = sqrt(fmax(s_hn2, 0.0));
  const double inv = sub > 0.0 ? 1.0 / sub : 0.0;
  const int64_t base = (int64_t)blockIdx.x * ARN_CHUNK;
  double* out = V + (int64_t)k * n;
#pragma unroll
  for (int e = 0; e < ARN_E; ++e) {
    const int64_t idx = base + e * ARN_T + threadIdx.x;
    if (idx < n) out[idx] = inv * w[idx];
  }
  __threadfence();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  // Givens update of column j = k - 1 (single CTA)
  __shared__ double col[1024], c_s[1024], s_s[1024];
  const int j = k - 1;
  for (int i = threadIdx.x; i <= j; i += ARN_T) col[i] = (i == j ? 1.0 : 0.0) - (h1[i] + h2[i]);
  for (int i = threadIdx.x; i < j; i += ARN_T) {
    c_s[i] = cs[i];
    s_s[i] = sn[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < j; ++i) {
      const double t = c_s[i] * col[i] + s_s[i] * col[i + 1];
      col[i + 1] = -s_s[i] * col[i] + c_s[i] * col[i + 1];
      col[i] = t;
    }
    const double a = col[j], b = -sub;
    const double den = hypot(a, b);
    double c = 1.0, s = 0.0;
    if (den > 0.0) { c = a / den; s = b / den; }
    cs[j] = c;
    sn[j] = s;
    col[j] = den;
    gv[j + 1] = -s * gv[j];
    gv[j] = c * gv[j];
    resid[j] = fabs(gv[j + 1]) / beta[0];
    if (k < kmax) *kdev = k + 1;
    *ticket = 0u;
  }
  __syncthreads();
  double* hc = H + (int64_t)j * ldh;
  for (int i = threadIdx.x; i <= j; i += ARN_T) hc[i] = col[i];
}

int arnoldi_chunks(int64_t n) { return (int)((n + ARN_CHUNK - 1) / ARN_CHUNK); }

void launch_arnoldi_step(double* V, double* w, int64_t n, int* kdev, double* h1, double* h2,
                         double* part, unsigned* ticket, double* H, int ldh, double* cs,
                         double* sn, double* gv, const double* beta, double* resid, int kmax,
                         cudaStream_t st) {
  const int nchunk = arnoldi_chunks(n);
  double* P1 = part;
  double* P2 = part + (int64_t)(kmax + 1) * nchunk;
  double* Pn = part + 2 * (int64_t)(kmax + 1) * nchunk;
  note_launch(4);
  k_arn_dots<<<nchunk, ARN_T, 0, st>>>(V, w, n, kdev, P1, nchunk);
  k_arn_update<<<nchunk, ARN_T, 0, st>>>(V, w, n, kdev, P1, h1, P2, Pn, nchunk, 1);
  k_arn_update<<<nchunk, ARN_T, 0, st>>>(V, w, n, kdev, P2, h2, nullptr, Pn, nchunk, 0);
  k_arn_finish<<<nchunk, ARN_T, 0, st>>>(V, w, n, kdev, Pn, nchunk, h1, h2, H, ldh, cs, sn, gv,
                                         beta, resid, kmax, ticket);
}

// ------------------------------------------------------------------------------------------
template <typename T>
void launch_apply_dense(const SlabDesc* d_slabs, const ProbDesc* d_probs, int nslab,
                        int64_t max_ng, const T* S, const double* x, double* y, int transpose,
                        cudaStream_t st, const int* kdev, int64_t kstride) {
  const int konly = transpose >> 1;  // bit 1: y = K x (or K^T x) instead of (I - K) x
  transpose &= 1;
  if (!transpose) {
    const size_t smem = 2 * max_ng * sizeof(T);
    raise_smem_limit(reinterpret_cast<const void*>(&k_apply_dense<T>), smem);
    note_launch();
    k_apply_dense<T><<<dim3((unsigned)((max_ng + 127) / 128), nslab), 256, smem, st>>>(
        d_slabs, d_probs, S, x, y, kdev, kstride, konly);
  } else {
    note_launch();
    const size_t smT = (2 * (size_t)max_ng + 128 * 33) * sizeof(T);
    raise_smem_limit(reinterpret_cast<const void*>(&k_apply_dense_T<T>), smT);
    k_apply_dense_T<T><<<dim3((unsigned)((max_ng + 127) / 128), nslab), 256, smT, st>>>(
        d_slabs, d_probs, S, x, y, kdev, kstride, konly, max_ng);
  }
}

template void launch_apply_dense<float>(const SlabDesc*, const ProbDesc*, int, int64_t,
                                        const float*, const double*, double*, int, cudaStream_t,
                                        const int*, int64_t);
template void launch_apply_dense<double>(const SlabDesc*, const ProbDesc*, int, int64_t,
                                         const double*, const double*, double*, int,
                                         cudaStream_t, const int*, int64_t);

void launch_combine_basis(const double* V, const double* y, int k, int64_t n, double* x,
                          cudaStream_t st) {
  note_launch();
  k_combine_basis<<<1024, 256, k * sizeof(double), st>>>(V, x, y, k, n);
}

void launch_normalize_start(const double* x, const double* nrm2, double* out, int64_t n,
                            cudaStream_t st) {
  note_launch();
  k_normalize_start<<<1024, 256, 0, st>>>(x, nrm2, out, n);
}

void launch_trisolve(const double* H, int ldh, const double* gv, int kk, double* y,
                     cudaStream_t st) {
  note_launch();
  k_trisolve<<<1, 256, kk * sizeof(double), st>>>(H, ldh, gv, kk, y);
}

}  // namespace ddst
