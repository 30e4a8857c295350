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
template <typename T>
__global__ void k_mf_rhs(const SlabDesc* __restrict__ slabs, const ProbDesc* __restrict__ probs,
                         const T* __restrict__ pack, const double* __restrict__ x0,
                         const int* __restrict__ kdev, int64_t kstride, T* __restrict__ loc) {
  const SlabDesc s = slabs[blockIdx.y];
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
__global__ void k_mf_inject(const SlabDesc* __restrict__ slabs, const double* __restrict__ x0,
                            const int* __restrict__ kdev, int64_t kstride, T* __restrict__ loc) {
  const SlabDesc s = slabs[blockIdx.y];
  const double* x = eff(x0, kdev, kstride);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < s.ng;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / s.p) + 1, t = (int)(e % s.p);
    loc[s.loc_off + (int64_t)(k - 1) * s.M + (s.w - 1) * s.p + t] = static_cast<T>(x[s.if_off + e]);
  }
}

// y = x - Kx (konly = 0) or y = Kx (konly = 1).
__global__ void k_mf_combine(int64_t n, const double* __restrict__ x0, const int* __restrict__ kdev,
                             int64_t kstride, const double* __restrict__ kx, double* __restrict__ y,
                             int konly) {
  const double* x = eff(x0, kdev, kstride);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = konly ? kx[e] : x[e] - kx[e];
}

template <typename T>
void launch_mf_rhs(const SlabDesc* d_slabs, const ProbDesc* d_probs, int nslab, const T* pack,
                   const double* x, const int* kdev, int64_t kstride, T* loc, cudaStream_t st) {
  note_launch();
  k_mf_rhs<T><<<dim3(32, nslab), 256, 0, st>>>(d_slabs, d_probs, pack, x, kdev, kstride, loc);
}

template <typename T>
void launch_mf_inject(const SlabDesc* d_slabs, int nslab, const double* x, const int* kdev,
                      int64_t kstride, T* loc, cudaStream_t st) {
  note_launch();
  k_mf_inject<T><<<dim3(32, nslab), 256, 0, st>>>(d_slabs, x, kdev, kstride, loc);
}

void launch_mf_combine(int64_t n, const double* x, const int* kdev, int64_t kstride,
                       const double* kx, double* y, int konly, cudaStream_t st) {
  note_launch();
  k_mf_combine<<<256, 256, 0, st>>>(n, x, kdev, kstride, kx, y, konly);
}

template void launch_mf_rhs<float>(const SlabDesc*, const ProbDesc*, int, const float*,
                                   const double*, const int*, int64_t, float*, cudaStream_t);
template void launch_mf_rhs<double>(const SlabDesc*, const ProbDesc*, int, const double*,
                                    const double*, const int*, int64_t, double*, cudaStream_t);
template void launch_mf_inject<float>(const SlabDesc*, int, const double*, const int*, int64_t,
                                      float*, cudaStream_t);
template void launch_mf_inject<double>(const SlabDesc*, int, const double*, const int*, int64_t,
                                       double*, cudaStream_t);

}  // namespace ddst
