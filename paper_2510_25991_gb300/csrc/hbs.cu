// hbs.cu -- nested-basis HBS compression of the transfer operators from random samples, and the
// telescoping apply (Sec. 2.4; Alg. 1: s = 3k + q Gaussian samples Y = S Omega, Z = S^T Psi).
//
// Compression, level by level from the leaves of the bisection tree shared by rows and columns:
//   k_hbs_gen    : Gaussian test matrices Omega, Psi (counter-based, per block; FP32 arithmetic
//                  for FP32 samples)
//   k_hbs_sample : Y = S Omega and Z = S^T Psi (64-row tiles, 32-column chunks in shared memory)
//   k_hbs_node   : one CTA per tree node.  In shared memory: Householder QR of Omega_t^T applied
//                  to Y_t^T (its trailing rows are Y_t P with P an orthonormal null-space basis
//                  of Omega_t, the leading ones Y_t Q_1 for the pseudo-inverse); U = the
//                  leading k columns of the column-pivoted QR of Y_t P; the same for V from
//                  (Psi_t, Z_t); D = (I - U U^T) Y_t Omega_t^+ + U U^T ((I - V V^T) Z_t
//                  Psi_t^+)^T; the reduced samples V^T Omega_t, U^T Psi_t, U^T (Y_t - D Omega_t)
//                  and V^T (Z_t - D^T Psi_t) written as the parent's rows.  The root keeps
//                  D_0 = Y_0 Omega_0^+.
// Apply (three launches; the tree is cut three levels above the leaves): k_hbs_up (one CTA per
// subtree below the cut: V^T x of its leaves and inner nodes), k_hbs_top (one CTA per block: the
// levels above the cut up, the root, and down), k_hbs_down (one CTA per subtree of an output
// interface: y of its inner nodes, then D x + U g of its leaves for both blocks writing there,
// combined into (I - K) x or K x).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <utility>

#include "hbs.cuh"

namespace ddst {

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Standard normal number for counter (block, which, index) by the Box-Muller transform of two
// 53-bit uniforms from the splitmix64 finalizer.
__device__ __forceinline__ double gauss_at(uint64_t seed, int blk, int which, int64_t e) {
  const uint64_t base = mix64(seed ^ mix64(((uint64_t)(uint32_t)blk << 2) | (uint64_t)which));
  const uint64_t a = mix64(base + 2 * (uint64_t)e), b = mix64(base + 2 * (uint64_t)e + 1);
  const double u1 = ((double)(a >> 11) + 1.0) * (1.0 / 9007199254740992.0);  // (0, 1]
  const double u2 = (double)(b >> 11) * (1.0 / 9007199254740992.0);          // [0, 1)
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// The same in single precision (24-bit uniforms, FP32 logarithm and cosine) for FP32 samples.
__device__ __forceinline__ float gauss_at_f(uint64_t seed, int blk, int which, int64_t e) {
  const uint64_t base = mix64(seed ^ mix64(((uint64_t)(uint32_t)blk << 2) | (uint64_t)which));
  const uint64_t a = mix64(base + 2 * (uint64_t)e), b = mix64(base + 2 * (uint64_t)e + 1);
  const float u1 = ((float)(a >> 40) + 1.0f) * (1.0f / 16777216.0f);  // (0, 1]
  const float u2 = (float)(b >> 40) * (1.0f / 16777216.0f);           // [0, 1)
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

template <typename T>
__device__ __forceinline__ T gauss_t(uint64_t seed, int blk, int which, int64_t e) {
  if constexpr (sizeof(T) == 4) return gauss_at_f(seed, blk, which, e);
  else return static_cast<T>(gauss_at(seed, blk, which, e));
}

struct SampBlk {     // one block of the sampling step
  const void* S;     // column-major ng x ng
  int64_t ng;
  int64_t row0;      // first row of the block in the leaf-level sample arrays
};

struct SampItem {
  int blk;
  int64_t lo;
};

}  // namespace

// Omega and Psi of every block (rows row0 .. row0 + ng - 1, row-major, s per row).
template <typename T>
__global__ void k_hbs_gen(const SampBlk* __restrict__ sb, T* __restrict__ Om, T* __restrict__ Ps,
                          int s, uint64_t seed) {
  const SampBlk b = sb[blockIdx.y];
  const int64_t tot = b.ng * s;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    Om[b.row0 * s + e] = gauss_t<T>(seed, blockIdx.y, 0, e);
    Ps[b.row0 * s + e] = gauss_t<T>(seed, blockIdx.y, 1, e);
  }
}

template <typename T>
__global__ void k_hbs_cvt(const double* __restrict__ src, T* __restrict__ dst, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = static_cast<T>(src[e]);
}

// Y = S Omega (trans 0) or Z = S^T Psi (trans 1) for a tile of 64 rows and all s samples.
// 256 threads: 16 row groups of 4 rows x 16 sample groups of CPT samples (s <= 16 CPT); the
// columns of S are staged 32 at a time together with the matching rows of the test matrix.
template <typename T, int CPT>
__global__ void __launch_bounds__(256) k_hbs_sample(const SampItem* __restrict__ items,
                                                    const SampBlk* __restrict__ sb,
                                                    const T* __restrict__ G, T* __restrict__ Y,
                                                    int s, int trans) {
  __shared__ T As[32][64 + 1];
  __shared__ T Bs[32][16 * CPT];
  const SampItem it = items[blockIdx.x];
  const SampBlk b = sb[it.blk];
  const T* S = static_cast<const T*>(b.S);
  const int64_t ng = b.ng, lo = it.lo;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][CPT];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc[i][j] = T(0);
  for (int64_t c0 = 0; c0 < ng; c0 += 32) {
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
      int r, cc;
      if (!trans) { r = e & 63; cc = e >> 6; } else { cc = e & 31; r = e >> 5; }
      const int64_t gr = lo + r, gc = c0 + cc;
      T v = T(0);
      if (gr < ng && gc < ng) v = trans ? S[gr * ng + gc] : S[gc * ng + gr];
      As[cc][r] = v;
    }
    for (int e = threadIdx.x; e < 32 * 16 * CPT; e += 256) {
      const int cc = e / (16 * CPT), j = e - cc * (16 * CPT);
      const int64_t gc = c0 + cc;
      Bs[cc][j] = (gc < ng && j < s) ? G[(b.row0 + gc) * s + j] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int cc = 0; cc < 32; ++cc) {
      T a[4], bv[CPT];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[cc][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < CPT; ++j) bv[j] = Bs[cc][tx * CPT + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < CPT; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = lo + ty * 4 + i;
    if (gr >= ng) continue;
#pragma unroll
    for (int j = 0; j < CPT; ++j) {
      const int jj = tx * CPT + j;
      if (jj < s) Y[(b.row0 + gr) * s + jj] = acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Node compression
// ---------------------------------------------------------------------------------------------
// Shared-memory layout of k_hbs_node (elements of T), for row sets of up to nm rows:
//   W  s x 2nm  (column-major, ld s): [Omega_t^T | Y_t^T], later the reloaded samples
//   G  nm x s   Y_t P (column-major, ld n) for the pivoted QR
//   U, V  nm x k;  X1, X2, D  nm x nm;  T1, T2  k x nm;  T3  k x k;  tau, tauG 64;  nrm s
struct NodeLayout {
  int64_t W, G, U, V, X1, X2, D, T1, T2, T3, tau, tauG, nrm, total;
  __host__ __device__ NodeLayout(int nm, int s, int k) {
    int64_t o = 0;
    W = o; o += (int64_t)s * 2 * nm;
    G = o; o += (int64_t)nm * s;
    U = o; o += (int64_t)nm * k;
    V = o; o += (int64_t)nm * k;
    X1 = o; o += (int64_t)nm * nm;
    X2 = o; o += (int64_t)nm * nm;
    D = o; o += (int64_t)nm * nm;
    T1 = o; o += (int64_t)k * nm;
    T2 = o; o += (int64_t)k * nm;
    T3 = o; o += (int64_t)k * k;
    tau = o; o += 64;
    tauG = o; o += 64;
    nrm = o; o += s;
    total = o;
  }
};

size_t hbs_node_smem(int n_max, int s, int k, size_t esz) {
  return (size_t)NodeLayout(n_max, s, k).total * esz + 16;
}

// Householder reflector of column x[0..m) in place (LAPACK convention: beta = -sign(alpha)
// ||x||, v = x / (alpha - beta) below the first entry, tau = (beta - alpha) / beta; tau = 0 when
// x[1..m) is zero).  Run by one warp; returns tau to every lane.
template <typename T>
__device__ T house_warp(T* x, int m) {
  const int lane = threadIdx.x & 31;
  T ss = T(0);
  for (int i = 1 + lane; i < m; i += 32) ss += x[i] * x[i];
  ss = warp_sum(ss);
  const T alpha = x[0];
  if (ss == T(0)) return T(0);
  const T nrm = sqrt(alpha * alpha + ss);
  const T beta = alpha >= T(0) ? -nrm : nrm;
  const T scale = T(1) / (alpha - beta);
  __syncwarp();
  for (int i = 1 + lane; i < m; i += 32) x[i] *= scale;
  __syncwarp();
  if (lane == 0) x[0] = beta;
  __syncwarp();
  return (beta - alpha) / beta;
}

// Applies H = I - tau [1; v] [1; v]^T (v below the first entry of `v`, length m) to columns
// c0 .. ncol-1 of A (leading dimension lda; each column's segment starts at A + c lda, aligned
// with v).  Four threads per column (a quarter of the rows each, combined by shuffles within the
// group), every column at once.
template <typename T>
__device__ void house_apply_cols(const T* v, T tau, T* A, int64_t lda, int c0, int ncol, int m) {
  const int sub = threadIdx.x & 3;
  const unsigned gmask = 0xFu << (threadIdx.x & 28);
  for (int c = c0 + (threadIdx.x >> 2); c < ncol; c += blockDim.x >> 2) {
    T* col = A + (int64_t)c * lda;
    T w = T(0);
    for (int i = 1 + sub; i < m; i += 4) w += v[i] * col[i];
    w += __shfl_xor_sync(gmask, w, 1);
    w += __shfl_xor_sync(gmask, w, 2);
    w = (w + col[0]) * tau;
    __syncwarp(gmask);
    for (int i = 1 + sub; i < m; i += 4) col[i] -= w * v[i];
    if (sub == 0) col[0] -= w;
  }
}

// Squared norms of rows j .. n-1 of columns c0 .. ncol-1 of A (leading dimension lda).
template <typename T>
__device__ void col_norms(const T* A, int64_t lda, int j, int n, int c0, int ncol, T* nrm) {
  const int sub = threadIdx.x & 3;
  const unsigned gmask = 0xFu << (threadIdx.x & 28);
  for (int c = c0 + (threadIdx.x >> 2); c < ncol; c += blockDim.x >> 2) {
    const T* col = A + (int64_t)c * lda;
    T ss = T(0);
    for (int i = j + sub; i < n; i += 4) ss += col[i] * col[i];
    ss += __shfl_xor_sync(gmask, ss, 1);
    ss += __shfl_xor_sync(gmask, ss, 2);
    if (sub == 0) nrm[c] = ss;
  }
}

// Householder QR of the first n columns of W (s x ncol, ld s), every reflector applied to the
// other columns as it is formed.  R ends in the upper triangle of the first n columns.
template <typename T>
__device__ void qr_front(T* W, int s, int n, int ncol, T* tau) {
  const int warp = threadIdx.x >> 5;
  for (int j = 0; j < n; ++j) {
    if (warp == 0) {
      const T t = house_warp(W + (int64_t)j * s + j, s - j);
      if ((threadIdx.x & 31) == 0) tau[j] = t;
    }
    __syncthreads();
    const T t = tau[j];
    if (t != T(0)) house_apply_cols(W + (int64_t)j * s + j, t, W + j, s, j + 1, ncol, s - j);
    __syncthreads();
  }
}

// One side of a node: W = [A_t^T | B_t^T] (A the test rows, B the samples, n x s each) after
// qr_front.  X (n x n, column-major) = B_t A_t^+ = (B_t Q_1) R^{-T}, solved row by row of B_t.
template <typename T>
__device__ void pinv_product(const T* W, int s, int n, T* X) {
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    const T* w = W + (int64_t)(n + a) * s;  // (Q^T B_t^T)(:, a): rows 0..n-1 = (B_t Q_1)(a, :)
    for (int i = n - 1; i >= 0; --i) {
      T acc = w[i];
      for (int j = i + 1; j < n; ++j) acc -= W[(int64_t)j * s + i] * X[(int64_t)j * n + a];
      X[(int64_t)i * n + a] = acc / W[(int64_t)i * s + i];
    }
  }
}

// Leading k columns of the orthogonal factor of the column-pivoted QR of G (n x r, ld n), into
// Q (n x k, ld n).  Pivot: the largest remaining partial column norm (first on ties).
template <typename T>
__device__ void qrcp_basis(T* G, int n, int r, int k, T* tau, T* nrm, T* Q) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ int piv;
  for (int j = 0; j < k; ++j) {
    col_norms(G, n, j, n, j, r, nrm);
    __syncthreads();
    if (threadIdx.x == 0) {
      int p = j;
      for (int c = j + 1; c < r; ++c)
        if (nrm[c] > nrm[p]) p = c;
      piv = p;
    }
    __syncthreads();
    const int p = piv;
    if (p != j)
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const T t = G[(int64_t)j * n + i];
        G[(int64_t)j * n + i] = G[(int64_t)p * n + i];
        G[(int64_t)p * n + i] = t;
      }
    __syncthreads();
    if (warp == 0) {
      const T t = house_warp(G + (int64_t)j * n + j, n - j);
      if (lane == 0) tau[j] = t;
    }
    __syncthreads();
    const T t = tau[j];
    if (t != T(0)) house_apply_cols(G + (int64_t)j * n + j, t, G + j, n, j + 1, r, n - j);
    __syncthreads();
  }
  // Q = H_0 ... H_{k-1} [I_k; 0]
  for (int e = threadIdx.x; e < n * k; e += blockDim.x) {
    const int i = e % n, c = e / n;
    Q[e] = i == c ? T(1) : T(0);
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const T t = tau[j];
    if (t != T(0)) house_apply_cols(G + (int64_t)j * n + j, t, Q + j, n, 0, k, n - j);
    __syncthreads();
  }
}

// Loads [A_t^T | B_t^T] into W (column c < n: row c of A_t; c >= n: row c - n of B_t).
template <typename T>
__device__ void load_side(T* W, const T* A, const T* B, int64_t row, int n, int s) {
  for (int e = threadIdx.x; e < 2 * n * s; e += blockDim.x) {
    const int c = e / s, i = e - c * s;
    W[e] = c < n ? A[(row + c) * s + i] : B[(row + c - n) * s + i];
  }
}

// One CTA per node of the current level (list of node indices).  Inputs at this level: the
// samples Y, Z and test rows Om, Ps (row-major, s per row); outputs: the factors and the k
// reduced rows of each of the four in the next level's arrays.
template <typename T>
__global__ void __launch_bounds__(256) k_hbs_node(const HbsNode* __restrict__ nodes,
                                                  const int* __restrict__ list,
                                                  const T* __restrict__ Yc, const T* __restrict__ Zc,
                                                  const T* __restrict__ Oc, const T* __restrict__ Pc,
                                                  T* __restrict__ Yn, T* __restrict__ Zn,
                                                  T* __restrict__ On, T* __restrict__ Pn,
                                                  T* __restrict__ F, int k, int s, int nm) {
  extern __shared__ __align__(16) unsigned char hbs_smem[];
  T* sm = reinterpret_cast<T*>(hbs_smem);
  const NodeLayout ly(nm, s, k);
  const HbsNode nd = nodes[list[blockIdx.x]];
  const int n = nd.n;
  T *W = sm + ly.W, *G = sm + ly.G, *U = sm + ly.U, *V = sm + ly.V, *X1 = sm + ly.X1,
    *X2 = sm + ly.X2, *D = sm + ly.D, *T1 = sm + ly.T1, *T2 = sm + ly.T2, *T3 = sm + ly.T3,
    *tau = sm + ly.tau, *tauG = sm + ly.tauG, *nrm = sm + ly.nrm;
  const bool root = nd.level == 0;
  const int r = s - n;
  for (int side = 0; side < (root ? 1 : 2); ++side) {
    load_side(W, side ? Pc : Oc, side ? Zc : Yc, nd.in_row, n, s);
    __syncthreads();
    qr_front(W, s, n, 2 * n, tau);
    pinv_product(W, s, n, side ? X2 : X1);
    if (!root) {
      // G = (trailing rows of Q^T B^T)^T = B_t P
      for (int e = threadIdx.x; e < n * r; e += blockDim.x) {
        const int a = e % n, j = e / n;
        G[e] = W[(int64_t)(n + a) * s + n + j];
      }
      __syncthreads();
      qrcp_basis(G, n, r, k, tauG, nrm, side ? V : U);
    }
    __syncthreads();
  }
  if (root) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) F[nd.d_off + e] = X1[e];
    return;
  }
  // D = X1 + U (T2 - T3 V^T - T1), T1 = U^T X1, T2 = U^T X2^T, T3 = T2 V
  for (int e = threadIdx.x; e < k * n; e += blockDim.x) {
    const int p = e % k, c = e / k;
    T t1 = T(0), t2 = T(0);
    for (int a = 0; a < n; ++a) {
      const T u = U[(int64_t)p * n + a];
      t1 += u * X1[(int64_t)c * n + a];
      t2 += u * X2[(int64_t)a * n + c];
    }
    T1[e] = t1;
    T2[e] = t2;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int p = e % k, q = e / k;
    T t = T(0);
    for (int c = 0; c < n; ++c) t += T2[(int64_t)c * k + p] * V[(int64_t)q * n + c];
    T3[e] = t;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < k * n; e += blockDim.x) {
    const int p = e % k, c = e / k;
    T t = T2[e] - T1[e];
    for (int q = 0; q < k; ++q) t -= T3[(int64_t)q * k + p] * V[(int64_t)q * n + c];
    T1[e] = t;  // T1 now holds T2 - T3 V^T - T1
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int a = e % n, c = e / n;
    T t = X1[e];
    for (int p = 0; p < k; ++p) t += U[(int64_t)p * n + a] * T1[(int64_t)c * k + p];
    D[e] = t;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * k; e += blockDim.x) {
    F[nd.u_off + e] = U[e];
    F[nd.v_off + e] = V[e];
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) F[nd.d_off + e] = D[e];
  // reduced samples: rows of this node in W (row-major n x s each: A at 0, B at n s)
  for (int side = 0; side < 2; ++side) {
    const T* A = side ? Pc : Oc;
    const T* B = side ? Zc : Yc;
    T* An = side ? Pn : On;
    T* Bn = side ? Zn : Yn;
    const T* Wl = side ? U : V;  // test rows reduce with the other side's basis
    const T* Wr = side ? V : U;
    __syncthreads();
    for (int e = threadIdx.x; e < n * s; e += blockDim.x) {
      W[e] = A[nd.in_row * s + e];
      W[(int64_t)n * s + e] = B[nd.in_row * s + e];
    }
    __syncthreads();
    // E = B_t - D A_t (side 0) or B_t - D^T A_t (side 1), in place over B_t
    for (int e = threadIdx.x; e < n * s; e += blockDim.x) {
      const int a = e / s, j = e - a * s;
      T t = W[(int64_t)n * s + e];
      for (int c = 0; c < n; ++c)
        t -= (side ? D[(int64_t)a * n + c] : D[(int64_t)c * n + a]) * W[(int64_t)c * s + j];
      G[e] = t;  // staged: W's B rows are still read by other threads
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k * s; e += blockDim.x) {
      const int p = e / s, j = e - p * s;
      T ta = T(0), tb = T(0);
      for (int a = 0; a < n; ++a) {
        ta += Wl[(int64_t)p * n + a] * W[(int64_t)a * s + j];
        tb += Wr[(int64_t)p * n + a] * G[(int64_t)a * s + j];
      }
      An[(nd.out_row + p) * s + j] = ta;
      Bn[(nd.out_row + p) * s + j] = tb;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Apply
// ---------------------------------------------------------------------------------------------
// The tree of a block with L >= 1 levels is cut at level ls = max(1, L - 3): one CTA owns the
// subtree of each node of level ls (at most 8 leaves, 512 rows, all its inner nodes), so the
// upward and downward passes inside a subtree run in shared memory; k_hbs_top does the few
// levels above ls for a whole block.
__host__ __device__ __forceinline__ int hbs_cut_level(int L) { return L > 3 ? L - 3 : 1; }

// out[p] = W(:, p)^T v for the k columns of W (n x k, column-major, n <= 64) by one warp, in
// the operators' precision (GB300 runs FP64 arithmetic at a small fraction of FP32); the loads
// of eight columns are issued before their reductions.  Lane 0 stores the results: out_s in
// shared memory (working precision), out_g in global memory (FP64).
template <typename T>
__device__ __forceinline__ void warp_cols_dot(const T* __restrict__ W, int n, int k, const T* v,
                                              T* out_s, double* out_g) {
  const int lane = threadIdx.x & 31;
  for (int p0 = 0; p0 < k; p0 += 8) {
    T acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int p = p0 + u;
      acc[u] = T(0);
      if (p < k) {
        const T* col = W + (int64_t)p * n;
        if (lane < n) acc[u] = fma(col[lane], v[lane], acc[u]);
        if (lane + 32 < n) acc[u] = fma(col[lane + 32], v[lane + 32], acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const T r = warp_sum(acc[u]);
      const int p = p0 + u;
      if (lane == 0 && p < k) { out_s[p] = r; out_g[p] = (double)r; }
    }
  }
}

// Upward pass inside one subtree (item: block, subtree root node): x_hat = V^T x of its leaves,
// then of its inner nodes level by level (U^T transposed), kept in shared memory and written to
// the block's x_hat scratch.  256 threads, a warp per node.
template <typename T>
__global__ void __launch_bounds__(256) k_hbs_up(const HbsLeafItem* __restrict__ items,
                                                const HbsBlock* __restrict__ bl,
                                                const HbsNode* __restrict__ nodes,
                                                const T* __restrict__ F,
                                                const double* __restrict__ x0,
                                                double* __restrict__ scratch, int transpose,
                                                int k, const int* kdev, int64_t kstride) {
  __shared__ T xs[512];
  __shared__ T xl[4][8][64];  // [level - ls][node][2k inputs of the next level up]
  const HbsLeafItem it = items[blockIdx.x];
  const HbsBlock b = bl[it.blk];
  const HbsNode rt = nodes[it.node];
  const int L = b.L, ls = rt.level, m = L - ls, warp = threadIdx.x >> 5;
  const int64_t hi = ((int64_t)(rt.t + 1) * b.ng) >> ls;
  const int len = (int)(hi - rt.lo);
  const double* x = x0 + (kdev ? (int64_t)(*kdev - 1) * kstride : 0) +
                    (transpose ? b.out_if : b.in_if) + rt.lo;
  for (int r = threadIdx.x; r < len; r += blockDim.x) xs[r] = static_cast<T>(x[r]);
  __syncthreads();
  double* xh = scratch + b.xh_off;
  for (int j = warp; j < (1 << m); j += 8) {  // leaves
    const int a = (1 << L) - 1 + rt.t * (1 << m) + j;
    const HbsNode& nd = nodes[b.node0 + a];
    // x_hat of child j lands in its parent's input vector: rows (j & 1) k of slot j >> 1
    T* dst = m > 0 ? &xl[m - 1][j >> 1][(j & 1) * k] : &xl[3][0][0];
    warp_cols_dot(F + (transpose ? nd.u_off : nd.v_off), nd.n, k, xs + (nd.lo - rt.lo), dst,
                  xh + (int64_t)a * k);
  }
  __syncthreads();
  for (int d = m - 1; d >= 0; --d) {  // inner nodes of the subtree, level ls + d
    const int lev = ls + d;
    for (int j = warp; j < (1 << d); j += 8) {
      const int a = (1 << lev) - 1 + rt.t * (1 << d) + j;
      const HbsNode& nd = nodes[b.node0 + a];
      T* dst = d > 0 ? &xl[d - 1][j >> 1][(j & 1) * k] : &xl[3][0][0];
      warp_cols_dot(F + (transpose ? nd.u_off : nd.v_off), 2 * k, k, xl[d][j], dst,
                    xh + (int64_t)a * k);
    }
    __syncthreads();
  }
}

// The levels above the cut for one block: x_hat of levels ls-1 .. 1, the root's y_0 = D_0 x_0,
// and y_a = D_a x_a + U_a g of levels 1 .. ls-1 (transposed: U^T, D^T, V).  Products in the
// operators' precision from vectors staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_hbs_top(const HbsBlock* __restrict__ bl,
                                                 const HbsNode* __restrict__ nodes,
                                                 const T* __restrict__ F,
                                                 double* __restrict__ scratch, int transpose,
                                                 int k) {
  __shared__ T vin[1024];  // inputs of up to 1024 / 2k nodes of one level (2k each)
  __shared__ T gin[512];   // their parents' y at their rows (k each)
  const HbsBlock b = bl[blockIdx.x];
  if (b.L == 0) return;
  const int ls = hbs_cut_level(b.L), k2 = 2 * k, CH = 1024 / k2;
  double* xh = scratch + b.xh_off;
  double* yh = scratch + b.yh_off;
  for (int lev = ls - 1; lev >= 0; --lev) {  // up; level 0 is the root's y_0 = D_0 x_0
    const int first = (1 << lev) - 1, cnt = 1 << lev;
    for (int c0 = 0; c0 < cnt; c0 += CH) {
      const int nc = min(CH, cnt - c0);
      for (int e = threadIdx.x; e < nc * k2; e += blockDim.x)  // children of the chunk, contiguous
        vin[e] = static_cast<T>(xh[(int64_t)(2 * (first + c0) + 1) * k + e]);
      __syncthreads();
      if (lev > 0) {
        for (int e = threadIdx.x; e < nc * k; e += blockDim.x) {
          const int jn = e / k, p = e % k, i = first + c0 + jn;
          const HbsNode& nd = nodes[b.node0 + i];
          const T* W = F + (int64_t)(transpose ? nd.u_off : nd.v_off) + (int64_t)p * k2;
          T acc = T(0);
#pragma unroll 8
          for (int a = 0; a < k2; ++a) acc = fma(W[a], vin[jn * k2 + a], acc);
          xh[(int64_t)i * k + p] = (double)acc;
        }
      } else {
        const T* D0 = F + nodes[b.node0].d_off;
        for (int a = threadIdx.x; a < k2; a += blockDim.x) {
          T acc = T(0);
#pragma unroll 8
          for (int c = 0; c < k2; ++c)
            acc = fma(transpose ? D0[(int64_t)a * k2 + c] : D0[(int64_t)c * k2 + a], vin[c], acc);
          yh[a] = (double)acc;
        }
      }
      __syncthreads();
    }
  }
  for (int lev = 1; lev <= ls - 1; ++lev) {  // down
    const int first = (1 << lev) - 1, cnt = 1 << lev;
    for (int c0 = 0; c0 < cnt; c0 += CH) {
      const int nc = min(CH, cnt - c0);
      for (int e = threadIdx.x; e < nc * k2; e += blockDim.x)
        vin[e] = static_cast<T>(xh[(int64_t)(2 * (first + c0) + 1) * k + e]);
      for (int e = threadIdx.x; e < nc * k; e += blockDim.x) {
        const int i = first + c0 + e / k, p = e % k;
        gin[e] = static_cast<T>(yh[(int64_t)((i - 1) / 2) * k2 + ((i - 1) & 1) * k + p]);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < nc * k2; e += blockDim.x) {
        const int jn = e / k2, row = e % k2, i = first + c0 + jn;
        const HbsNode& nd = nodes[b.node0 + i];
        const T* Dm = F + nd.d_off;
        const T* W2 = F + (transpose ? nd.v_off : nd.u_off);
        T acc = T(0);
#pragma unroll 8
        for (int c = 0; c < k2; ++c)
          acc = fma(transpose ? Dm[(int64_t)row * k2 + c] : Dm[(int64_t)c * k2 + row],
                    vin[jn * k2 + c], acc);
#pragma unroll 8
        for (int p = 0; p < k; ++p) acc = fma(W2[(int64_t)p * k2 + row], gin[jn * k + p], acc);
        yh[(int64_t)i * k2 + row] = (double)acc;
      }
      __syncthreads();
    }
  }
}

// Downward pass inside one subtree and the output (item: the rows of one subtree of one output
// interface; up to two blocks write there, taken one after the other): y_a = D_a x_a + U_a g of
// the subtree's inner nodes level by level in shared memory (g: the parent's y at the rows of a;
// for the subtree root from the block's y_hat), then D x + U g of its leaves; y = x - sum (or the
// sum with konly).  Transposed: D^T and V.  Products in the operators' precision; the sums of
// the two blocks and the output in FP64.  256 threads.
template <typename T>
__global__ void __launch_bounds__(256) k_hbs_down(const HbsOwn* __restrict__ items,
                                                  const HbsBlock* __restrict__ bl,
                                                  const HbsNode* __restrict__ nodes,
                                                  const T* __restrict__ F,
                                                  const double* __restrict__ scratch,
                                                  const double* __restrict__ x0,
                                                  double* __restrict__ y, int transpose, int konly,
                                                  int k, int lcap, const int* kdev,
                                                  int64_t kstride) {
  __shared__ T xs[512];
  __shared__ double outv[512];
  __shared__ T xa[4][64];     // inputs x_a of the nodes of one inner level
  __shared__ T yv[2][4][64];  // y of the nodes of the current and the previous level
  __shared__ T groot[32];
  const double* x = x0 + (kdev ? (int64_t)(*kdev - 1) * kstride : 0);
  const HbsOwn it = items[blockIdx.x];
  const int len = it.len, k2 = 2 * k;
  for (int r = threadIdx.x; r < len; r += blockDim.x) outv[r] = 0.0;
  for (int q = 0; q < it.nsrc; ++q) {
    const HbsBlock b = bl[it.blk[q]];
    const HbsNode rt = nodes[it.node[q]];
    const int L = b.L, ls = rt.level, m = L - ls;
    const double* xin = x + (transpose ? b.out_if : b.in_if) + it.lo;
    __syncthreads();  // the previous source's readers of xs, yv are done
    for (int r = threadIdx.x; r < len; r += blockDim.x) xs[r] = static_cast<T>(xin[r]);
    if (L > 0) {
      const int ir = it.node[q] - b.node0;
      for (int p = threadIdx.x; p < k; p += blockDim.x)
        groot[p] = static_cast<T>(
            scratch[b.yh_off + (int64_t)((ir - 1) / 2) * k2 + ((ir - 1) & 1) * k + p]);
    }
    __syncthreads();
    int cur = 0;
    for (int d = 0; d < m; ++d) {  // inner nodes of the subtree at level ls + d
      const int lev = ls + d, nl = 1 << d;
      for (int e = threadIdx.x; e < nl * k2; e += blockDim.x) {
        const int j = e / k2, c = e % k2;
        const int a = (1 << lev) - 1 + rt.t * nl + j;
        xa[j][c] = static_cast<T>(scratch[b.xh_off + (int64_t)(2 * a + 1) * k + c]);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < nl * k2; e += blockDim.x) {
        const int j = e / k2, row = e % k2;
        const int a = (1 << lev) - 1 + rt.t * nl + j;
        const HbsNode& nd = nodes[b.node0 + a];
        const T* Dm = F + nd.d_off;
        const T* W2 = F + (transpose ? nd.v_off : nd.u_off);
        const T* g = d == 0 ? groot : &yv[cur ^ 1][j >> 1][(j & 1) * k];
        T acc = T(0);
#pragma unroll 8
        for (int c = 0; c < k2; ++c)
          acc = fma(transpose ? Dm[(int64_t)row * k2 + c] : Dm[(int64_t)c * k2 + row], xa[j][c], acc);
#pragma unroll 8
        for (int p = 0; p < k; ++p) acc = fma(W2[(int64_t)p * k2 + row], g[p], acc);
        yv[cur][j][row] = acc;
      }
      __syncthreads();
      cur ^= 1;
    }
    // leaves (level L): thread per (leaf, row), lcap (the leaf size bound) rows per leaf
    for (int e = threadIdx.x; e < (1 << m) * lcap; e += blockDim.x) {
      const int j = e / lcap, rr = e - j * lcap;
      const int a = (1 << L) - 1 + rt.t * (1 << m) + j;
      const HbsNode& nd = nodes[b.node0 + a];
      const int n = nd.n;
      if (rr >= n) continue;
      const int off = (int)(nd.lo - it.lo);
      const T* Dm = F + nd.d_off;
      T acc = T(0);
      if (!transpose) {
#pragma unroll 8
        for (int c = 0; c < n; ++c) acc = fma(Dm[(int64_t)c * n + rr], xs[off + c], acc);
      } else {
#pragma unroll 8
        for (int c = 0; c < n; ++c) acc = fma(Dm[(int64_t)rr * n + c], xs[off + c], acc);
      }
      if (L > 0) {
        const T* W2 = F + (transpose ? nd.v_off : nd.u_off);
        const T* g = m == 0 ? groot : &yv[cur ^ 1][j >> 1][(j & 1) * k];
#pragma unroll 8
        for (int p = 0; p < k; ++p) acc = fma(W2[(int64_t)p * n + rr], g[p], acc);
      }
      outv[off + rr] += (double)acc;
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < len; r += blockDim.x) {
    const int64_t o = it.out + it.lo + r;
    y[o] = konly ? outv[r] : x[o] - outv[r];
  }
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
void HbsSet::release() {
  for (void* p : {F, (void*)scratch, (void*)d_nodes, (void*)d_blocks, (void*)d_own,
                  (void*)d_own_T, (void*)d_leaf_items})
    if (p) cudaFree(p);
  F = nullptr; scratch = nullptr; d_nodes = nullptr; d_blocks = nullptr; d_own = nullptr;
  d_own_T = nullptr; d_leaf_items = nullptr;
  nodes.clear(); blocks.clear(); blk_slab.clear(); blk_side.clear(); bare.clear();
  n_own = n_own_T = n_leaf_items = 0;
  max_L = 0;
  f_elems = bytes = 0;
  built = false;
}

namespace {

int tree_levels(int64_t ng, int leaf) {  // smallest L with ceil(ng / 2^L) <= leaf
  int L = 0;
  while ((ng + (int64_t(1) << L) - 1) / (int64_t(1) << L) > leaf) ++L;
  return L;
}

// Output items: blocks grouped by the interface they write (their source interface when
// transposed), one item per leaf of that interface.
std::vector<HbsOwn> make_owners(const HbsSet& H, bool transpose) {
  std::map<int64_t, std::vector<int>> by_out;
  for (size_t b = 0; b < H.blocks.size(); ++b)
    by_out[transpose ? H.blocks[b].in_if : H.blocks[b].out_if].push_back((int)b);
  std::vector<HbsOwn> out;
  for (auto& kv : by_out) {
    const auto& bs = kv.second;
    for (size_t g = 0; g < bs.size(); g += 2) {  // at most two blocks per item
      const HbsBlock& b0 = H.blocks[bs[g]];
      const int ls = b0.L == 0 ? 0 : hbs_cut_level(b0.L);
      for (int t = 0; t < (1 << ls); ++t) {  // one item per subtree below the cut
        HbsOwn o{};
        o.out = kv.first;
        o.nsrc = (g + 1 < bs.size()) ? 2 : 1;
        for (int q = 0; q < o.nsrc; ++q) {
          o.blk[q] = bs[g + q];
          o.node[q] = H.blocks[bs[g + q]].node0 + (1 << ls) - 1 + t;
        }
        const HbsNode& nd = H.nodes[o.node[0]];
        o.lo = nd.lo;
        o.len = (int)((((int64_t)(t + 1) * b0.ng) >> ls) - nd.lo);
        out.push_back(o);
      }
    }
  }
  for (const auto& bi : H.bare)  // no block writes there: y = x (or 0 for K x)
    for (int64_t lo = 0; lo < bi.second; lo += 64) {
      HbsOwn o{};
      o.out = bi.first;
      o.lo = lo;
      o.len = (int)std::min<int64_t>(64, bi.second - lo);
      o.nsrc = 0;
      out.push_back(o);
    }
  return out;
}

}  // namespace

template <typename T>
int hbs_build(HbsSet& H, const std::vector<HbsInput>& in,
              const std::vector<std::pair<int64_t, int64_t>>& bare, int k, int s, int leaf,
              uint64_t seed, cudaStream_t st, std::string& msg) {
  H.release();
  H.bare = bare;
  const int nb = (int)in.size();
  if (nb == 0) { msg = "no blocks"; return 3; }
  if (k < 1 || k > 32 || s < 3 * k || s > 96 || leaf < 1 || leaf > 64) {
    msg = "rank must be 1..32 with 3k <= samples <= 96 and a leaf size of 1..64";
    return 3;
  }
  H.k = k; H.s = s; H.leaf = leaf; H.esz = sizeof(T);
  int64_t fo = 0, so = 0, rows0 = 0;
  int nmax = 0, Lmax = 0;
  std::vector<int64_t> row0(nb);
  for (int b = 0; b < nb; ++b) {
    const int64_t ng = in[b].ng;
    if (ng < 1) { msg = "empty block"; H.release(); return 3; }
    const int L = tree_levels(ng, leaf);
    if (L > 20) { msg = "tree too deep"; H.release(); return 3; }
    Lmax = std::max(Lmax, L);
    HbsBlock hb{};
    hb.ng = ng; hb.L = L; hb.node0 = (int)H.nodes.size();
    hb.in_if = in[b].in_if; hb.out_if = in[b].out_if;
    hb.xh_off = so; so += ((int64_t(2) << L) - 1) * k;
    hb.yh_off = so; so += std::max<int64_t>(1, (int64_t(1) << L) - 1) * 2 * k;
    for (int lev = 0; lev <= L; ++lev)
      for (int t = 0; t < (1 << lev); ++t) {
        HbsNode nd{};
        nd.blk = b; nd.level = lev; nd.t = t;
        nd.lo = (int64_t(t) * ng) >> lev;
        nd.n = lev == L ? (int)(((int64_t(t + 1) * ng) >> lev) - nd.lo) : 2 * k;
        nd.u_off = nd.v_off = -1;
        if (lev > 0) {
          if (nd.n < k) {
            msg = "a leaf holds fewer indices than the rank (raise the leaf size)";
            H.release();
            return 3;
          }
          if (nd.n + k > s) {
            msg = "a node's rows plus the rank exceed the sample count";
            H.release();
            return 3;
          }
          nd.u_off = fo; fo += (int64_t)nd.n * k;
          nd.v_off = fo; fo += (int64_t)nd.n * k;
        } else if (nd.n > s) {
          msg = "the root's rows exceed the sample count";
          H.release();
          return 3;
        }
        nd.d_off = fo; fo += (int64_t)nd.n * nd.n;
        nmax = std::max(nmax, nd.n);
        H.nodes.push_back(nd);
      }
    row0[b] = rows0;
    rows0 += ng;
    H.blocks.push_back(hb);
    H.blk_slab.push_back(in[b].slab);
    H.blk_side.push_back(in[b].side);
  }
  if (nmax > 64) { msg = "row sets above 64"; H.release(); return 3; }
  const size_t smem = hbs_node_smem(nmax, s, k, sizeof(T));
  if (smem > 227 * 1024) { msg = "node workspace above the shared-memory limit"; H.release(); return 3; }
  // row offsets of every node's samples, level by level from the leaves (d = steps from them)
  std::vector<std::vector<int>> steps(Lmax + 1);
  for (int b = 0; b < nb; ++b) {
    const HbsBlock& hb = H.blocks[b];
    for (int lev = hb.L; lev >= 0; --lev)
      for (int t = 0; t < (1 << lev); ++t) steps[hb.L - lev].push_back(hb.node0 + (1 << lev) - 1 + t);
  }
  for (int d = 0; d <= Lmax; ++d) {
    int64_t nxt = 0;
    for (int id : steps[d]) {
      HbsNode& nd = H.nodes[id];
      const HbsBlock& hb = H.blocks[nd.blk];
      if (d == 0) nd.in_row = row0[nd.blk] + nd.lo;
      if (nd.level > 0) {
        nd.out_row = nxt;
        nxt += k;
        if (nd.t % 2 == 0) {  // the parent's rows start at its first child's reduced rows
          HbsNode& par = H.nodes[hb.node0 + (1 << (nd.level - 1)) - 1 + nd.t / 2];
          par.in_row = nd.out_row;
        }
      }
    }
  }
  H.max_L = Lmax;
  H.f_elems = fo;
  H.bytes = fo * (int64_t)sizeof(T);
  auto al = [&](void** p, size_t bytes) { return cudaMalloc(p, std::max<size_t>(bytes, 16)) == cudaSuccess; };
  T* arr[8] = {};
  SampBlk* d_sb = nullptr;
  SampItem* d_items = nullptr;
  int* d_list = nullptr;
  double* d_stage = nullptr;
  auto cleanup = [&]() {
    for (T* p : arr) if (p) cudaFree(p);
    for (void* p : {(void*)d_sb, (void*)d_items, (void*)d_list, (void*)d_stage}) if (p) cudaFree(p);
  };
  bool ok = al(&H.F, sizeof(T) * fo) && al((void**)&H.scratch, sizeof(double) * so) &&
            al((void**)&H.d_nodes, sizeof(HbsNode) * H.nodes.size()) &&
            al((void**)&H.d_blocks, sizeof(HbsBlock) * nb) &&
            al((void**)&d_sb, sizeof(SampBlk) * nb) &&
            al((void**)&d_list, sizeof(int) * H.nodes.size());
  // the reduced rows of a level (k per node) can outnumber the leaf rows when leaf < 2k
  int64_t rows_max = rows0, red = 0;
  for (int b = 0; b < nb; ++b) red += (int64_t(1) << H.blocks[b].L) * k;
  rows_max = std::max(rows_max, red);
  for (int a = 0; a < 8 && ok; ++a) ok = al((void**)&arr[a], sizeof(T) * rows_max * s);
  if (!ok) { cleanup(); H.release(); msg = "out of device memory"; return 2; }
  T *Yc = arr[0], *Zc = arr[1], *Oc = arr[2], *Pc = arr[3];
  T *Yn = arr[4], *Zn = arr[5], *On = arr[6], *Pn = arr[7];
  cudaMemcpyAsync(H.d_nodes, H.nodes.data(), sizeof(HbsNode) * H.nodes.size(),
                  cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(H.d_blocks, H.blocks.data(), sizeof(HbsBlock) * nb, cudaMemcpyHostToDevice, st);
  std::vector<SampBlk> sb(nb);
  std::vector<SampItem> items;
  for (int b = 0; b < nb; ++b) {
    sb[b] = SampBlk{in[b].S, in[b].ng, row0[b]};
    for (int64_t lo = 0; lo < in[b].ng; lo += 64) items.push_back(SampItem{b, lo});
  }
  cudaMemcpyAsync(d_sb, sb.data(), sizeof(SampBlk) * nb, cudaMemcpyHostToDevice, st);
  if (!al((void**)&d_items, sizeof(SampItem) * items.size())) {
    cleanup(); H.release(); msg = "out of device memory"; return 2;
  }
  cudaMemcpyAsync(d_items, items.data(), sizeof(SampItem) * items.size(), cudaMemcpyHostToDevice, st);
  // test matrices: given (FP64, converted) or drawn on the device
  bool given = false;
  for (int b = 0; b < nb; ++b) given = given || in[b].omega || in[b].psi;
  if (given) {
    int64_t maxe = 0;
    for (int b = 0; b < nb; ++b) maxe = std::max(maxe, in[b].ng * s);
    if (!al((void**)&d_stage, sizeof(double) * maxe)) {
      cleanup(); H.release(); msg = "out of device memory"; return 2;
    }
    for (int b = 0; b < nb; ++b)
      for (int w = 0; w < 2; ++w) {
        const double* src = w ? in[b].psi : in[b].omega;
        if (!src) { cleanup(); H.release(); msg = "omega and psi are given for every block or none"; return 3; }
        cudaMemcpyAsync(d_stage, src, sizeof(double) * in[b].ng * s, cudaMemcpyHostToDevice, st);
        note_launch();
        k_hbs_cvt<T><<<256, 256, 0, st>>>(d_stage, (w ? Pc : Oc) + row0[b] * s, in[b].ng * s);
      }
    cudaStreamSynchronize(st);  // the host arrays are the caller's
  } else {
    note_launch();
    k_hbs_gen<T><<<dim3(64, nb), 256, 0, st>>>(d_sb, Oc, Pc, s, seed);
  }
  note_launch(2);
  const unsigned nit = (unsigned)items.size();
  if (s <= 32) {
    k_hbs_sample<T, 2><<<nit, 256, 0, st>>>(d_items, d_sb, Oc, Yc, s, 0);
    k_hbs_sample<T, 2><<<nit, 256, 0, st>>>(d_items, d_sb, Pc, Zc, s, 1);
  } else if (s <= 64) {
    k_hbs_sample<T, 4><<<nit, 256, 0, st>>>(d_items, d_sb, Oc, Yc, s, 0);
    k_hbs_sample<T, 4><<<nit, 256, 0, st>>>(d_items, d_sb, Pc, Zc, s, 1);
  } else {
    k_hbs_sample<T, 6><<<nit, 256, 0, st>>>(d_items, d_sb, Oc, Yc, s, 0);
    k_hbs_sample<T, 6><<<nit, 256, 0, st>>>(d_items, d_sb, Pc, Zc, s, 1);
  }
  cudaError_t e = raise_smem_limit((const void*)k_hbs_node<T>, smem);
  if (e != cudaSuccess) { cleanup(); H.release(); msg = cudaGetErrorString(e); return 1; }
  std::vector<int> lists;
  for (int d = 0; d <= Lmax; ++d) lists.insert(lists.end(), steps[d].begin(), steps[d].end());
  cudaMemcpyAsync(d_list, lists.data(), sizeof(int) * lists.size(), cudaMemcpyHostToDevice, st);
  size_t pos = 0;
  for (int d = 0; d <= Lmax; ++d) {
    const int cnt = (int)steps[d].size();
    if (cnt > 0) {
      note_launch();
      k_hbs_node<T><<<cnt, 256, smem, st>>>(H.d_nodes, d_list + pos, Yc, Zc, Oc, Pc, Yn, Zn, On,
                                            Pn, (T*)H.F, k, s, nmax);
    }
    pos += cnt;
    std::swap(Yc, Yn); std::swap(Zc, Zn); std::swap(Oc, On); std::swap(Pc, Pn);
  }
  // apply items
  std::vector<HbsLeafItem> li;  // upward-pass items: the subtrees below the cut
  for (int b = 0; b < nb; ++b) {
    const HbsBlock& hb = H.blocks[b];
    if (hb.L == 0) continue;
    const int ls = hbs_cut_level(hb.L);
    for (int t = 0; t < (1 << ls); ++t) li.push_back(HbsLeafItem{b, hb.node0 + (1 << ls) - 1 + t});
  }
  const std::vector<HbsOwn> own = make_owners(H, false), ownT = make_owners(H, true);
  ok = al((void**)&H.d_leaf_items, sizeof(HbsLeafItem) * li.size()) &&
       al((void**)&H.d_own, sizeof(HbsOwn) * own.size()) &&
       al((void**)&H.d_own_T, sizeof(HbsOwn) * ownT.size());
  if (!ok) { cleanup(); H.release(); msg = "out of device memory"; return 2; }
  if (!li.empty())
    cudaMemcpyAsync(H.d_leaf_items, li.data(), sizeof(HbsLeafItem) * li.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(H.d_own, own.data(), sizeof(HbsOwn) * own.size(), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(H.d_own_T, ownT.data(), sizeof(HbsOwn) * ownT.size(), cudaMemcpyHostToDevice, st);
  H.n_leaf_items = (int)li.size();
  H.n_own = (int)own.size();
  H.n_own_T = (int)ownT.size();
  e = cudaStreamSynchronize(st);
  cleanup();
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) { H.release(); msg = cudaGetErrorString(e); return 1; }
  H.built = true;
  return 0;
}

template <typename T>
void hbs_apply(HbsSet& H, const double* x, double* y, int transpose, cudaStream_t st,
               const int* kdev, int64_t kstride) {
  const int konly = transpose >> 1;
  transpose &= 1;
  if (H.n_leaf_items > 0) {
    note_launch(2);
    k_hbs_up<T><<<H.n_leaf_items, 256, 0, st>>>(H.d_leaf_items, H.d_blocks, H.d_nodes,
                                                (const T*)H.F, x, H.scratch, transpose, H.k, kdev,
                                                kstride);
    k_hbs_top<T><<<(unsigned)H.blocks.size(), 256, 0, st>>>(H.d_blocks, H.d_nodes, (const T*)H.F,
                                                            H.scratch, transpose, H.k);
  }
  const int no = transpose ? H.n_own_T : H.n_own;
  if (no > 0) {
    note_launch();
    k_hbs_down<T><<<no, 256, 0, st>>>(transpose ? H.d_own_T : H.d_own, H.d_blocks, H.d_nodes,
                                      (const T*)H.F, H.scratch, x, y, transpose, konly, H.k,
                                      H.leaf, kdev, kstride);
  }
}

int hbs_expand(HbsSet& H, int b, double* out, cudaStream_t st) {
  if (b < 0 || b >= (int)H.blocks.size()) return 1;
  const HbsBlock& hb = H.blocks[b];
  const int k = H.k, L = hb.L;
  const int64_t ng = hb.ng;
  auto fetch = [&](int64_t off, int64_t n, std::vector<double>& dst) {
    dst.resize(n);
    if (H.esz == 8) {
      cudaMemcpyAsync(dst.data(), (const double*)H.F + off, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
    } else {
      std::vector<float> tmp(n);
      cudaMemcpyAsync(tmp.data(), (const float*)H.F + off, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      for (int64_t e = 0; e < n; ++e) dst[e] = tmp[e];
    }
  };
  // A_0 = D_0; A_l = U_l A_{l-1} V_l^T + D_l (block-diagonal U_l, V_l, D_l), column-major
  const HbsNode& root = H.nodes[hb.node0];
  std::vector<double> A, Um, Vm, Dm;
  fetch(root.d_off, (int64_t)root.n * root.n, A);
  int64_t dim = root.n;
  for (int lev = 1; lev <= L; ++lev) {
    const int cnt = 1 << lev;
    std::vector<int64_t> off(cnt + 1, 0);
    for (int t = 0; t < cnt; ++t) off[t + 1] = off[t] + H.nodes[hb.node0 + cnt - 1 + t].n;
    const int64_t nd = off[cnt];
    std::vector<double> B((size_t)(dim * nd), 0.0);  // A_{l-1} V^T: dim x nd
    std::vector<double> C((size_t)(nd * nd), 0.0);
    for (int t = 0; t < cnt; ++t) {
      const HbsNode& no = H.nodes[hb.node0 + cnt - 1 + t];
      fetch(no.v_off, (int64_t)no.n * k, Vm);
      for (int64_t c = 0; c < no.n; ++c)
        for (int64_t r = 0; r < dim; ++r) {
          double a = 0.0;
          for (int q = 0; q < k; ++q) a += A[(t * k + q) * dim + r] * Vm[q * no.n + c];
          B[(off[t] + c) * dim + r] = a;
        }
    }
    for (int t = 0; t < cnt; ++t) {
      const HbsNode& no = H.nodes[hb.node0 + cnt - 1 + t];
      fetch(no.u_off, (int64_t)no.n * k, Um);
      fetch(no.d_off, (int64_t)no.n * no.n, Dm);
      for (int64_t c = 0; c < nd; ++c)
        for (int64_t r = 0; r < no.n; ++r) {
          double a = 0.0;
          for (int p = 0; p < k; ++p) a += Um[p * no.n + r] * B[c * dim + t * k + p];
          C[c * nd + off[t] + r] = a;
        }
      for (int64_t c = 0; c < no.n; ++c)
        for (int64_t r = 0; r < no.n; ++r) C[(off[t] + c) * nd + off[t] + r] += Dm[c * no.n + r];
    }
    A.swap(C);
    dim = nd;
  }
  if (dim != ng) return 1;
  std::copy(A.begin(), A.end(), out);
  return 0;
}

template int hbs_build<float>(HbsSet&, const std::vector<HbsInput>&,
                              const std::vector<std::pair<int64_t, int64_t>>&, int, int, int,
                              uint64_t, cudaStream_t, std::string&);
template int hbs_build<double>(HbsSet&, const std::vector<HbsInput>&,
                               const std::vector<std::pair<int64_t, int64_t>>&, int, int, int,
                               uint64_t, cudaStream_t, std::string&);
template void hbs_apply<float>(HbsSet&, const double*, double*, int, cudaStream_t, const int*, int64_t);
template void hbs_apply<double>(HbsSet&, const double*, double*, int, cudaStream_t, const int*,
                                int64_t);

}  // namespace ddst
