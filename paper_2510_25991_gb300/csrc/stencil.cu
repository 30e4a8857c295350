// stencil.cu -- finite-difference operator generation and FP64 global-grid kernels.
//
// Discretization of Sec. 1, Eq. (basic) with the five-point (2D, Sec. 2.1) / seven-point (3D,
// Sec. 5.2) stencil:  (A u)_p = sum_faces a_pq (u_p - u_q)/h^2
//                              + sum_d b_d (u_{p+e_d} - u_{p-e_d})/(2h) + c_p u_p,
// a_pq = (a_p + a_q)/2.  Dirichlet neighbours move to the right-hand side.
#include "kernels.cuh"

namespace ddst {

__device__ __forceinline__ int64_t node_index(int dim, int n, int x, int y, int z) {
  const int64_t s = n + 1;
  return dim == 2 ? (int64_t)x * s + y : ((int64_t)x * s + y) * s + z;
}

// Stencil pack of every (slab, block): diag, west, east, south (ell), north (ups), zlo, zhi.
// One CTA per (slab, block); threads over local unknowns.  Coefficients in FP64, stored as T.
template <typename T>
__global__ void k_stencil_pack(const SlabDesc* __restrict__ slabs,
                               const ProbDesc* __restrict__ probs,
                               const double* __restrict__ a_all,
                               const double* __restrict__ c_all, T* __restrict__ pack) {
  const SlabDesc s = slabs[blockIdx.y];
  const int k = blockIdx.x + 1;
  if (k > s.nb) return;
  const ProbDesc P = probs[s.prob];
  const double* a = a_all + s.node_off;
  const double* cc = P.has_c ? c_all + s.node_off : nullptr;
  const double h2 = 1.0 / (P.h * P.h);
  const double h2b = 0.5 / P.h;
  T* out = pack + s.pack_off + (int64_t)(k - 1) * PK_NFIELDS * s.M;
  for (int c = threadIdx.x; c < s.M; c += blockDim.x) {
    double f[PK_NFIELDS] = {1.0, 0, 0, 0, 0, 0, 0};
    if (c < s.m) {
      const int cx = c / s.p, t = c % s.p;
      const int x = (s.j - 1) * s.w + 1 + cx, y = k, z = t + 1;
      const double ap = a[node_index(P.dim, s.n, x, y, z)];
      const double axm = 0.5 * (ap + a[node_index(P.dim, s.n, x - 1, y, z)]);
      const double axp = 0.5 * (ap + a[node_index(P.dim, s.n, x + 1, y, z)]);
      const double aym = 0.5 * (ap + a[node_index(P.dim, s.n, x, y - 1, z)]);
      const double ayp = 0.5 * (ap + a[node_index(P.dim, s.n, x, y + 1, z)]);
      double diag = (axm + axp + aym + ayp) * h2;
      double zlo = 0.0, zhi = 0.0;
      if (P.dim == 3) {
        const double azm = 0.5 * (ap + a[node_index(P.dim, s.n, x, y, z - 1)]);
        const double azp = 0.5 * (ap + a[node_index(P.dim, s.n, x, y, z + 1)]);
        diag += (azm + azp) * h2;
        if (t > 0) zlo = -azm * h2 - P.b[2] * h2b;
        if (t < s.p - 1) zhi = -azp * h2 + P.b[2] * h2b;
      }
      if (cc) diag += cc[node_index(P.dim, s.n, x, y, z)];
      f[PK_DIAG] = diag;
      f[PK_WEST] = -axm * h2 - P.b[0] * h2b;   // cx == 0: coupling to x-plane (j-1)w
      f[PK_EAST] = -axp * h2 + P.b[0] * h2b;   // cx == 2w-2: coupling to x-plane (j+1)w
      f[PK_SOUTH] = (k > 1) ? -aym * h2 - P.b[1] * h2b : 0.0;
      f[PK_NORTH] = (k < s.nb) ? -ayp * h2 + P.b[1] * h2b : 0.0;
      f[PK_ZLO] = zlo;
      f[PK_ZHI] = zhi;
    }
#pragma unroll
    for (int q = 0; q < PK_NFIELDS; ++q) out[q * s.M + c] = static_cast<T>(f[q]);
  }
}

// b = f + (Dirichlet neighbour terms), FP64, all problems (grid.y = problem).
// transpose = 1 builds nothing different for b (only A changes); kept for symmetry.
__global__ void k_rhs(const ProbDesc* __restrict__ probs, const double* __restrict__ a_all,
                      const double* __restrict__ f_all, const double* __restrict__ g_all,
                      double* __restrict__ b_all) {
  const ProbDesc P = probs[blockIdx.y];
  const double* a = a_all + P.node_off;
  const double* g = g_all + P.node_off;
  const int n = P.n;
  const double h2 = 1.0 / (P.h * P.h), h2b = 0.5 / P.h;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P.nint;
       q += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    if (P.dim == 2) {
      x = (int)(q / (n - 1)) + 1; y = (int)(q % (n - 1)) + 1; z = 0;
    } else {
      const int64_t nn = (int64_t)(n - 1) * (n - 1);
      x = (int)(q / nn) + 1; y = (int)((q / (n - 1)) % (n - 1)) + 1; z = (int)(q % (n - 1)) + 1;
    }
    const double ap = a[node_index(P.dim, n, x, y, z)];
    double acc = f_all[P.vol_off + q];
    const int nd = P.dim;
    for (int d = 0; d < nd; ++d) {
      for (int s = -1; s <= 1; s += 2) {
        int xx = x, yy = y, zz = z;
        if (d == 0) xx += s; else if (d == 1) yy += s; else zz += s;
        const int coord = d == 0 ? xx : (d == 1 ? yy : zz);
        if (coord == 0 || coord == n) {
          const int64_t qi = node_index(P.dim, n, xx, yy, zz);
          const double af = 0.5 * (ap + a[qi]);
          const double coef = -af * h2 + s * P.b[d] * h2b;
          acc -= coef * g[qi];
        }
      }
    }
    b_all[P.vol_off + q] = acc;
  }
}

// r = b - A u (transpose = 0) or r = b - A^T u (transpose = 1), FP64, interior part of A.
// Optionally accumulates ||r||^2 partial sums per CTA into part[blockIdx.y * gridDim.x + bx].
__global__ void k_residual(const ProbDesc* __restrict__ probs, const double* __restrict__ a_all,
                           const double* __restrict__ c_all, const double* __restrict__ b_all,
                           const double* __restrict__ u_all, double* __restrict__ r_all,
                           int transpose, double* __restrict__ part) {
  const ProbDesc P = probs[blockIdx.y];
  const double* a = a_all + P.node_off;
  const double* cc = P.has_c ? c_all + P.node_off : nullptr;
  const double* u = u_all + P.vol_off;
  const int n = P.n;
  const double h2 = 1.0 / (P.h * P.h), h2b = 0.5 / P.h;
  const double sg = transpose ? -1.0 : 1.0;
  double local = 0.0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P.nint;
       q += (int64_t)gridDim.x * blockDim.x) {
    int x, y, z;
    int64_t str[3];
    if (P.dim == 2) {
      x = (int)(q / (n - 1)) + 1; y = (int)(q % (n - 1)) + 1; z = 0;
      str[0] = n - 1; str[1] = 1; str[2] = 0;
    } else {
      const int64_t nn = (int64_t)(n - 1) * (n - 1);
      x = (int)(q / nn) + 1; y = (int)((q / (n - 1)) % (n - 1)) + 1; z = (int)(q % (n - 1)) + 1;
      str[0] = nn; str[1] = n - 1; str[2] = 1;
    }
    const double ap = a[node_index(P.dim, n, x, y, z)];
    const double up = u[q];
    double diag = cc ? cc[node_index(P.dim, n, x, y, z)] : 0.0;
    double off = 0.0;
    for (int d = 0; d < P.dim; ++d) {
      for (int s = -1; s <= 1; s += 2) {
        int xx = x, yy = y, zz = z;
        if (d == 0) xx += s; else if (d == 1) yy += s; else zz += s;
        const int coord = d == 0 ? xx : (d == 1 ? yy : zz);
        const double af = 0.5 * (ap + a[node_index(P.dim, n, xx, yy, zz)]);
        diag += af * h2;
        if (coord != 0 && coord != n) {
          const double coef = -af * h2 + sg * s * P.b[d] * h2b;
          off += coef * u[q + s * str[d]];
        }
      }
    }
    const double rv = b_all[P.vol_off + q] - (diag * up + off);
    r_all[P.vol_off + q] = rv;
    local += rv * rv;
  }
  if (part) {
    __shared__ double red[32];
    local = warp_sum(local);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x < 32) {
      double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
      v = warp_sum(v);
      if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = v;
    }
  }
}

// Slab-local gather: loc[k][c] = vol[global(cx, k, t)] (zero in padding), FP64 -> T.
template <typename T>
__global__ void k_gather(const SlabDesc* __restrict__ slabs, const double* __restrict__ vol,
                         T* __restrict__ loc) {
  const SlabDesc s = slabs[blockIdx.y];
  const int64_t total = (int64_t)s.nb * s.M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / s.M) + 1, c = (int)(e % s.M);
    T v = T(0);
    if (c < s.m) v = static_cast<T>(vol[s.vol_off + vol_index(s, c / s.p, k, c % s.p)]);
    loc[s.loc_off + e] = v;
  }
}

// Slab-local scatter of a volume solution: slab j owns x-planes cx = 0..w-1 (its left half and
// Gamma_j); the last slab of a problem also owns cx = w..2w-2.  mode 0: vol = x; 1: vol += x.
template <typename T>
__global__ void k_scatter(const SlabDesc* __restrict__ slabs, const ProbDesc* __restrict__ probs,
                          const T* __restrict__ loc, double* __restrict__ vol, int mode) {
  const SlabDesc s = slabs[blockIdx.y];
  const ProbDesc P = probs[s.prob];
  const int ncx = (s.j == P.nds) ? 2 * s.w - 1 : s.w;
  const int64_t total = (int64_t)s.nb * ncx * s.p;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e % s.p);
    const int cx = (int)((e / s.p) % ncx);
    const int k = (int)(e / ((int64_t)s.p * ncx)) + 1;
    const double v = static_cast<double>(loc[s.loc_off + (int64_t)(k - 1) * s.M + cx * s.p + t]);
    const int64_t gi = s.vol_off + vol_index(s, cx, k, t);
    vol[gi] = mode ? vol[gi] + v : v;
  }
}

// Interface values of slab-local vectors: out[(k-1)p + t] = loc[k][C_t] (C_t = (w-1)p + t).
template <typename T>
__global__ void k_extract_center(const SlabDesc* __restrict__ slabs, const T* __restrict__ loc,
                                 double* __restrict__ iface) {
  const SlabDesc s = slabs[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.ng;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / s.p) + 1, t = (int)(e % s.p);
    iface[s.if_off + e] =
        static_cast<double>(loc[s.loc_off + (int64_t)(k - 1) * s.M + (s.w - 1) * s.p + t]);
  }
}

// Adds the Dirichlet data of the neighbouring interfaces to slab-local right-hand sides:
// loc[k][W_t] -= beta_{k,t} uG_{j-1}[(k,t)], loc[k][E_t] -= gamma_{k,t} uG_{j+1}[(k,t)]
// (interior interfaces only; physical boundary data is already part of b).
template <typename T>
__global__ void k_add_iface_dirichlet(const SlabDesc* __restrict__ slabs,
                                      const ProbDesc* __restrict__ probs,
                                      const T* __restrict__ pack, const double* __restrict__ uG,
                                      T* __restrict__ loc) {
  const SlabDesc s = slabs[blockIdx.y];
  const ProbDesc P = probs[s.prob];
  const int64_t stride_if = s.ng;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.ng;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / s.p) + 1, t = (int)(e % s.p);
    const T* pk = pack + s.pack_off + (int64_t)(k - 1) * PK_NFIELDS * s.M;
    T* row = loc + s.loc_off + (int64_t)(k - 1) * s.M;
    if (s.j >= 2) {
      const double beta = static_cast<double>(pk[PK_WEST * s.M + t]);
      row[t] = static_cast<T>(static_cast<double>(row[t]) - beta * uG[s.if_off - stride_if + e]);
    }
    if (s.j <= P.nds - 1) {
      const int cE = (2 * s.w - 2) * s.p + t;
      const double gam = static_cast<double>(pk[PK_EAST * s.M + cE]);
      row[cE] = static_cast<T>(static_cast<double>(row[cE]) - gam * uG[s.if_off + stride_if + e]);
    }
  }
}

// Adjoint counterpart of k_add_iface_dirichlet: the interface data u_{j-1}, u_{j+1} enters the
// local right-hand side through -beta / -gamma, so its transpose maps a slab-local vector z to
// interface contributions out_{j-1} -= beta z[W], out_{j+1} -= gamma z[E] (atomic: neighbours
// of two slabs write the same interface).
template <typename T>
__global__ void k_iface_dirichlet_T(const SlabDesc* __restrict__ slabs,
                                    const ProbDesc* __restrict__ probs,
                                    const T* __restrict__ pack, const T* __restrict__ loc,
                                    double* __restrict__ out) {
  const SlabDesc s = slabs[blockIdx.y];
  const ProbDesc P = probs[s.prob];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.ng;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / s.p) + 1, t = (int)(e % s.p);
    const T* pk = pack + s.pack_off + (int64_t)(k - 1) * PK_NFIELDS * s.M;
    const T* row = loc + s.loc_off + (int64_t)(k - 1) * s.M;
    if (s.j >= 2) {
      const double beta = static_cast<double>(pk[PK_WEST * s.M + t]);
      atomicAdd(&out[s.if_off - s.ng + e], -beta * static_cast<double>(row[t]));
    }
    if (s.j <= P.nds - 1) {
      const int cE = (2 * s.w - 2) * s.p + t;
      const double gam = static_cast<double>(pk[PK_EAST * s.M + cE]);
      atomicAdd(&out[s.if_off + s.ng + e], -gam * static_cast<double>(row[cE]));
    }
  }
}

// Transpose of the center extraction: loc[k][C_t] += iface[(k,t)] (loc pre-zeroed by caller).
template <typename T>
__global__ void k_inject_center(const SlabDesc* __restrict__ slabs, const double* __restrict__ iface,
                                T* __restrict__ loc) {
  const SlabDesc s = slabs[blockIdx.y];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.ng;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / s.p) + 1, t = (int)(e % s.p);
    T* row = loc + s.loc_off + (int64_t)(k - 1) * s.M;
    row[(s.w - 1) * s.p + t] += static_cast<T>(iface[s.if_off + e]);
  }
}

// Transpose of the slab-local gather restricted to the owned planes (adjoint of k_scatter):
// loc[k][c] = vol[...] for owned cx, 0 elsewhere.
template <typename T>
__global__ void k_gather_owned(const SlabDesc* __restrict__ slabs,
                               const ProbDesc* __restrict__ probs, const double* __restrict__ vol,
                               T* __restrict__ loc) {
  const SlabDesc s = slabs[blockIdx.y];
  const ProbDesc P = probs[s.prob];
  const int ncx = (s.j == P.nds) ? 2 * s.w - 1 : s.w;
  const int64_t total = (int64_t)s.nb * s.M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / s.M) + 1, c = (int)(e % s.M);
    T v = T(0);
    if (c < s.m && c / s.p < ncx) v = static_cast<T>(vol[s.vol_off + vol_index(s, c / s.p, k, c % s.p)]);
    loc[s.loc_off + e] = v;
  }
}

// Transpose of k_gather: vol[global] += loc[k][c] over all slab-local unknowns (atomic, since
// neighbouring double slabs overlap).
template <typename T>
__global__ void k_gather_T(const SlabDesc* __restrict__ slabs, const T* __restrict__ loc,
                           double* __restrict__ vol) {
  const SlabDesc s = slabs[blockIdx.y];
  const int64_t total = (int64_t)s.nb * s.M;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / s.M) + 1, c = (int)(e % s.M);
    if (c < s.m)
      atomicAdd(&vol[s.vol_off + vol_index(s, c / s.p, k, c % s.p)],
                static_cast<double>(loc[s.loc_off + e]));
  }
}

// Partial sums of x.y over n elements (grid-stride); part[blockIdx.x].
__global__ void k_dot_partial(const double* __restrict__ x, const double* __restrict__ y,
                              int64_t n, double* __restrict__ part) {
  double v = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    v += x[e] * y[e];
  __shared__ double red[32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}

// Per-problem sums of squares, first stage: part[q * gridDim.x + b] for problem q = blockIdx.y
// over its interior unknowns x[vol_off, vol_off + nint).
__global__ void k_prob_sqnorm_partial(const ProbDesc* __restrict__ probs, const double* __restrict__ x,
                                      double* __restrict__ part) {
  const int64_t off = probs[blockIdx.y].vol_off, n = probs[blockIdx.y].nint;
  double v = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    v += x[off + e] * x[off + e];
  __shared__ double red[32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

// Sum of np partials into out[0]; with several CTAs, CTA c sums part[c np, (c + 1) np) into out[c].
__global__ void k_sum_partials(const double* __restrict__ part, int np, double* __restrict__ out) {
  part += (int64_t)blockIdx.x * np;
  double v = 0.0;
  for (int e = threadIdx.x; e < np; e += blockDim.x) v += part[e];
  __shared__ double red[32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
  }
}

// IMEX right-hand side of one backward-Euler step (Sec. 6, Example 1, Eq. (convdiff)):
// f = u / dt - v . grad_h u at every interior node, central differences, u = 0 on boundary
// nodes.  vel: component d of every problem's nodal velocity at vel + d tot_nodes.
// grid = (chunks, problems).
__global__ void k_imex_rhs(const ProbDesc* __restrict__ probs, const double* __restrict__ u,
                           const double* __restrict__ vel, int64_t tot_nodes, double inv_dt,
                           double* __restrict__ f) {
  const ProbDesc P = probs[blockIdx.y];
  const int nb = P.n - 1, nn = P.n + 1;
  const double inv2h = 0.5 * P.n;
  const double* U = u + P.vol_off;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < P.nint;
       e += (int64_t)gridDim.x * blockDim.x) {
    int c[3] = {0, 0, 0};  // 1-based interior coordinates, x slowest
    int64_t r = e, node = 0, sint = 1;
    int64_t s_int[3];
    for (int d = P.dim - 1; d >= 0; --d) {
      c[d] = (int)(r % nb) + 1;
      r /= nb;
      s_int[d] = sint;
      sint *= nb;
    }
    for (int d = 0; d < P.dim; ++d) node = node * nn + c[d];
    double val = U[e] * inv_dt;
    for (int d = 0; d < P.dim; ++d) {
      const double up = c[d] < nb ? U[e + s_int[d]] : 0.0;
      const double dn = c[d] > 1 ? U[e - s_int[d]] : 0.0;
      val -= vel[d * tot_nodes + P.node_off + node] * (up - dn) * inv2h;
    }
    f[P.vol_off + e] = val;
  }
}

// y = a*x + y  (FP64)
__global__ void k_axpy(int64_t n, double a, const double* __restrict__ x, double* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] += a * x[e];
}

// ------------------------------------------------------------------------------------------
// Host launchers
// ------------------------------------------------------------------------------------------
template <typename T>
void launch_stencil_pack(const SlabDesc* d_slabs, int nslab, int max_nb, const ProbDesc* d_probs,
                         const double* a, const double* c, T* pack, cudaStream_t st) {
  dim3 grid(max_nb, nslab);
  note_launch();
  k_stencil_pack<T><<<grid, 128, 0, st>>>(d_slabs, d_probs, a, c, pack);
}

void launch_rhs(const ProbDesc* d_probs, int nprob, const double* a, const double* f,
                const double* g, double* b, cudaStream_t st) {
  note_launch();
  k_rhs<<<dim3(512, nprob), 256, 0, st>>>(d_probs, a, f, g, b);
}

void launch_residual(const ProbDesc* d_probs, int nprob, const double* a, const double* c,
                     const double* b, const double* u, double* r, int transpose, double* part,
                     int nblk, cudaStream_t st) {
  note_launch();
  k_residual<<<dim3(nblk, nprob), 256, 0, st>>>(d_probs, a, c, b, u, r, transpose, part);
}

template <typename T>
void launch_gather(const SlabDesc* d_slabs, int nslab, const double* vol, T* loc, cudaStream_t st) {
  note_launch();
  k_gather<T><<<dim3(64, nslab), 256, 0, st>>>(d_slabs, vol, loc);
}

template <typename T>
void launch_gather_owned(const SlabDesc* d_slabs, const ProbDesc* d_probs, int nslab,
                         const double* vol, T* loc, cudaStream_t st) {
  note_launch();
  k_gather_owned<T><<<dim3(64, nslab), 256, 0, st>>>(d_slabs, d_probs, vol, loc);
}

template <typename T>
void launch_gather_T(const SlabDesc* d_slabs, int nslab, const T* loc, double* vol,
                     cudaStream_t st) {
  note_launch();
  k_gather_T<T><<<dim3(64, nslab), 256, 0, st>>>(d_slabs, loc, vol);
}

template <typename T>
void launch_scatter(const SlabDesc* d_slabs, const ProbDesc* d_probs, int nslab, const T* loc,
                    double* vol, int mode, cudaStream_t st) {
  note_launch();
  k_scatter<T><<<dim3(64, nslab), 256, 0, st>>>(d_slabs, d_probs, loc, vol, mode);
}

template <typename T>
void launch_extract_center(const SlabDesc* d_slabs, int nslab, const T* loc, double* iface,
                           cudaStream_t st) {
  note_launch();
  k_extract_center<T><<<dim3(16, nslab), 256, 0, st>>>(d_slabs, loc, iface);
}

template <typename T>
void launch_inject_center(const SlabDesc* d_slabs, int nslab, const double* iface, T* loc,
                          cudaStream_t st) {
  note_launch();
  k_inject_center<T><<<dim3(16, nslab), 256, 0, st>>>(d_slabs, iface, loc);
}

template <typename T>
void launch_add_iface_dirichlet(const SlabDesc* d_slabs, const ProbDesc* d_probs, int nslab,
                                const T* pack, const double* uG, T* loc, cudaStream_t st) {
  note_launch();
  k_add_iface_dirichlet<T><<<dim3(16, nslab), 256, 0, st>>>(d_slabs, d_probs, pack, uG, loc);
}

template <typename T>
void launch_iface_dirichlet_T(const SlabDesc* d_slabs, const ProbDesc* d_probs, int nslab,
                              const T* pack, const T* loc, double* out, cudaStream_t st) {
  note_launch();
  k_iface_dirichlet_T<T><<<dim3(16, nslab), 256, 0, st>>>(d_slabs, d_probs, pack, loc, out);
}

void launch_dot(const double* x, const double* y, int64_t n, double* part, int nblk,
                double* out, cudaStream_t st) {
  note_launch();
  k_dot_partial<<<nblk, 256, 0, st>>>(x, y, n, part);
  note_launch();
  k_sum_partials<<<1, 256, 0, st>>>(part, nblk, out);
}

void launch_prob_sqnorms(const ProbDesc* d_probs, int nprob, const double* x, double* part,
                         int nblk, double* out, cudaStream_t st) {
  note_launch();
  k_prob_sqnorm_partial<<<dim3(nblk, nprob), 256, 0, st>>>(d_probs, x, part);
  note_launch();
  k_sum_partials<<<nprob, 256, 0, st>>>(part, nblk, out);
}

void launch_imex_rhs(const ProbDesc* d_probs, int nprob, const double* u, const double* vel,
                     int64_t tot_nodes, double inv_dt, double* f, cudaStream_t st) {
  note_launch();
  k_imex_rhs<<<dim3(256, nprob), 256, 0, st>>>(d_probs, u, vel, tot_nodes, inv_dt, f);
}

void launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t st) {
  note_launch();
  k_axpy<<<1024, 256, 0, st>>>(n, a, x, y);
}

#define INST(T)                                                                                  \
  template void launch_stencil_pack<T>(const SlabDesc*, int, int, const ProbDesc*, const double*, \
                                       const double*, T*, cudaStream_t);                         \
  template void launch_gather<T>(const SlabDesc*, int, const double*, T*, cudaStream_t);         \
  template void launch_gather_owned<T>(const SlabDesc*, const ProbDesc*, int, const double*, T*, \
                                       cudaStream_t);                                            \
  template void launch_gather_T<T>(const SlabDesc*, int, const T*, double*, cudaStream_t);       \
  template void launch_scatter<T>(const SlabDesc*, const ProbDesc*, int, const T*, double*, int, \
                                  cudaStream_t);                                                 \
  template void launch_extract_center<T>(const SlabDesc*, int, const T*, double*, cudaStream_t); \
  template void launch_inject_center<T>(const SlabDesc*, int, const double*, T*, cudaStream_t);  \
  template void launch_add_iface_dirichlet<T>(const SlabDesc*, const ProbDesc*, int, const T*,   \
                                              const double*, T*, cudaStream_t);                  \
  template void launch_iface_dirichlet_T<T>(const SlabDesc*, const ProbDesc*, int, const T*,     \
                                            const T*, double*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace ddst
