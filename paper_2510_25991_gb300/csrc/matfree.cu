// matfree.cu -- the interface operator K applied through local solves, with no explicit S.
//
// Sec. 2.2, Eq. (defS): S_{j,j'} = -R_{C_j} A_j(I_j,I_j)^{-1} A(I_j, J_{j,j'}).  Block row j of
// K x is therefore one Dirichlet solve on the double slab Psi_j whose right-hand side carries
// the neighbouring traces x_{j-1}, x_{j+1} through the x couplings of its first and last local
// planes, read back on the central plane Gamma_j.  The transpose runs the other way: x_j enters
// at the central plane, the transposed local solve follows, and the boundary planes feed
// Gamma_{j-1} and Gamma_{j+1}.  This is the paper's matrix-free application of S (Sec. 2.5 and
// the LU/HBS comparison of Sec. 5.1): no transfer operator is formed or stored, and every
// application streams the local factors once.  The kernels here build the right-hand sides and
// the result; the local solves are those of solve.cu / bigblock.cu.
//
// x may be indexed by a device-resident Krylov basis count (x_eff = x + (*kdev - 1) kstride),
// so that one GMRES step including this operator is captured once as a CUDA graph.
#include "kernels.cuh"

namespace ddst {

__device__ __forceinline__ const double* eff(const double* x, const int* kdev, int64_t kstride) {
  return kdev ? x + (int64_t)(*kdev - 1) * kstride : x;
}

// loc (zeroed by the caller) gets the Dirichlet data of the neighbouring interfaces:
// loc[k][W_t] = -beta_{k,t} x_{j-1}(k,t),  loc[k][E_t] = -gamma_{k,t} x_{j+1}(k,t).
// grid = (chunks, listed slabs).
template <typename T>
__global__ void k_mf_rhs(const SlabDesc* __restrict__ slabs, const int* __restrict__ ids,
                         const ProbDesc* __restrict__ probs, const T* __restrict__ pack,
                         const double* __restrict__ x0, const int* __restrict__ kdev,
                         int64_t kstride, T* __restrict__ loc) {
  const SlabDesc s = slabs[ids[blockIdx.y]];
  const ProbDesc P = probs[s.prob];
  const double* x = eff(x0, kdev, kstride);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.ng;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / s.p) + 1, t = (int)(e % s.p);
    const T* pk = pack + s.pack_off + (int64_t)(k - 1) * PK_NFIELDS * s.M;
    T* row = loc + s.loc_off + (int64_t)(k - 1) * s.M;
    if (s.j >= 2)
      row[t] = static_cast<T>(-static_cast<double>(pk[PK_WEST * s.M + t]) * x[s.if_off - s.ng + e]);
    if (s.j <= P.nds - 1) {
      const int cE = (2 * s.w - 2) * s.p + t;
      row[cE] = static_cast<T>(-static_cast<double>(pk[PK_EAST * s.M + cE]) * x[s.if_off + s.ng + e]);
    }
  }
}

// loc (zeroed by the caller) gets x_j on the central plane: loc[k][C_t] = x_j(k,t).
template <typename T>
__global__ void k_mf_inject(const SlabDesc* __restrict__ slabs, const int* __restrict__ ids,
                            const double* __restrict__ x0, const int* __restrict__ kdev,
                            int64_t kstride, T* __restrict__ loc) {
  const SlabDesc s = slabs[ids[blockIdx.y]];
  const double* x = eff(x0, kdev, kstride);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.ng;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / s.p) + 1, t = (int)(e % s.p);
    loc[s.loc_off + (int64_t)(k - 1) * s.M + (s.w - 1) * s.p + t] = static_cast<T>(x[s.if_off + e]);
  }
}

// Transposed Dirichlet coupling: the data x_{j-1}, x_{j+1} enters slab j's right-hand side
// through -beta / -gamma, so z (slab-local) feeds out_{j-1} -= beta z[W], out_{j+1} -= gamma z[E]
// (atomic: two slabs feed each interface).
template <typename T>
__global__ void k_mf_dirichlet_T(const SlabDesc* __restrict__ slabs, const int* __restrict__ ids,
                                 const ProbDesc* __restrict__ probs, const T* __restrict__ pack,
                                 const T* __restrict__ loc, double* __restrict__ out) {
  const SlabDesc s = slabs[ids[blockIdx.y]];
  const ProbDesc P = probs[s.prob];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.ng;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / s.p) + 1, t = (int)(e % s.p);
    const T* pk = pack + s.pack_off + (int64_t)(k - 1) * PK_NFIELDS * s.M;
    const T* row = loc + s.loc_off + (int64_t)(k - 1) * s.M;
    if (s.j >= 2)
      atomicAdd(&out[s.if_off - s.ng + e],
                -static_cast<double>(pk[PK_WEST * s.M + t]) * static_cast<double>(row[t]));
    if (s.j <= P.nds - 1) {
      const int cE = (2 * s.w - 2) * s.p + t;
      atomicAdd(&out[s.if_off + s.ng + e],
                -static_cast<double>(pk[PK_EAST * s.M + cE]) * static_cast<double>(row[cE]));
    }
  }
}

// On the interface Gamma_j of every listed slab: y = x - Kx (konly = 0) or y = Kx (konly = 1).
__global__ void k_mf_combine(const SlabDesc* __restrict__ slabs, const int* __restrict__ ids,
                             const double* __restrict__ x0, const int* __restrict__ kdev,
                             int64_t kstride, const double* __restrict__ kx, double* __restrict__ y,
                             int konly) {
  const SlabDesc s = slabs[ids[blockIdx.y]];
  const double* x = eff(x0, kdev, kstride);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.ng;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = s.if_off + e;
    y[i] = konly ? kx[i] : x[i] - kx[i];
  }
}

template <typename T>
void launch_mf_rhs(const SlabDesc* d_slabs, const int* d_ids, int nids, const ProbDesc* d_probs,
                   const T* pack, const double* x, const int* kdev, int64_t kstride, T* loc,
                   cudaStream_t st) {
  note_launch();
  k_mf_rhs<T><<<dim3(32, nids), 256, 0, st>>>(d_slabs, d_ids, d_probs, pack, x, kdev, kstride, loc);
}

template <typename T>
void launch_mf_inject(const SlabDesc* d_slabs, const int* d_ids, int nids, const double* x,
                      const int* kdev, int64_t kstride, T* loc, cudaStream_t st) {
  note_launch();
  k_mf_inject<T><<<dim3(32, nids), 256, 0, st>>>(d_slabs, d_ids, x, kdev, kstride, loc);
}

template <typename T>
void launch_mf_dirichlet_T(const SlabDesc* d_slabs, const int* d_ids, int nids,
                           const ProbDesc* d_probs, const T* pack, const T* loc, double* out,
                           cudaStream_t st) {
  note_launch();
  k_mf_dirichlet_T<T><<<dim3(32, nids), 256, 0, st>>>(d_slabs, d_ids, d_probs, pack, loc, out);
}

void launch_mf_combine(const SlabDesc* d_slabs, const int* d_ids, int nids, const double* x,
                       const int* kdev, int64_t kstride, const double* kx, double* y, int konly,
                       cudaStream_t st) {
  note_launch();
  k_mf_combine<<<dim3(32, nids), 256, 0, st>>>(d_slabs, d_ids, x, kdev, kstride, kx, y, konly);
}

#define INST(T)                                                                                  \
  template void launch_mf_rhs<T>(const SlabDesc*, const int*, int, const ProbDesc*, const T*,    \
                                 const double*, const int*, int64_t, T*, cudaStream_t);          \
  template void launch_mf_inject<T>(const SlabDesc*, const int*, int, const double*, const int*, \
                                    int64_t, T*, cudaStream_t);                                  \
  template void launch_mf_dirichlet_T<T>(const SlabDesc*, const int*, int, const ProbDesc*,      \
                                         const T*, const T*, double*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace ddst
