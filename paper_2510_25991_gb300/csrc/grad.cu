// grad.cu -- gradient assembly of the discrete adjoint.
//
// With lambda = A^{-T} dL/du for the FD system A(a) u = b(a, f, g) of Sec. 1, Eq. (basic):
//   dL/df_p = lambda_p                                         (interior nodes)
//   dL/dg_q = sum_{interior p ~ q} lambda_p (a_pq/h^2 - s b_d/(2h)),  q = p + s e_d on the boundary
//   dL/da_pq = -(lambda_p - lambda_q)(u_p - u_q)/h^2 per face (u_q = g_q, lambda_q = 0 on the
//              boundary), and nodal dL/da_node = 1/2 sum of the faces at the node
//              (a_pq = (a_p + a_q)/2).
#include "kernels.cuh"

namespace ddst {

__device__ __forceinline__ int64_t nidx(int dim, int n, int x, int y, int z) {
  const int64_t s = n + 1;
  return dim == 2 ? (int64_t)x * s + y : ((int64_t)x * s + y) * s + z;
}

// grid.y = problem.  dLdg and dLda must be zeroed by the caller (nodal, concatenated).
__global__ void k_gradients(const ProbDesc* __restrict__ probs, const double* __restrict__ a_all,
                            const double* __restrict__ g_all, const double* __restrict__ u_all,
                            const double* __restrict__ lam_all, double* __restrict__ dLdg,
                            double* __restrict__ dLda) {
  const ProbDesc P = probs[blockIdx.y];
  const int n = P.n;
  const double* a = a_all + P.node_off;
  const double* g = g_all + P.node_off;
  const double* u = u_all + P.vol_off;
  const double* lam = lam_all + P.vol_off;
  const double h2 = 1.0 / (P.h * P.h), h2b = 0.5 / P.h;
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
    const int64_t pn = nidx(P.dim, n, x, y, z);
    const double lp = lam[q], up = u[q], ap = a[pn];
    for (int d = 0; d < P.dim; ++d) {
      for (int s = -1; s <= 1; s += 2) {
        int xx = x, yy = y, zz = z;
        if (d == 0) xx += s; else if (d == 1) yy += s; else zz += s;
        const int coord = d == 0 ? xx : (d == 1 ? yy : zz);
        const int64_t qn = nidx(P.dim, n, xx, yy, zz);
        const bool bnd = coord == 0 || coord == n;
        if (bnd) {
          const double af = 0.5 * (ap + a[qn]);
          if (dLdg) atomicAdd(&dLdg[P.node_off + qn], lp * (af * h2 - s * P.b[d] * h2b));
          if (dLda) {
            const double df = -(lp - 0.0) * (up - g[qn]) * h2;
            atomicAdd(&dLda[P.node_off + pn], 0.5 * df);
            atomicAdd(&dLda[P.node_off + qn], 0.5 * df);
          }
        } else if (s == 1 && dLda) {
          const int64_t qi = q + str[d];
          const double df = -(lp - lam[qi]) * (up - u[qi]) * h2;
          atomicAdd(&dLda[P.node_off + pn], 0.5 * df);
          atomicAdd(&dLda[P.node_off + qn], 0.5 * df);
        }
      }
    }
  }
}

void launch_gradients(const ProbDesc* d_probs, int nprob, const double* a, const double* g,
                      const double* u, const double* lam, double* dLdg, double* dLda,
                      cudaStream_t st) {
  note_launch();
  k_gradients<<<dim3(512, nprob), 256, 0, st>>>(d_probs, a, g, u, lam, dLdg, dLda);
}

}  // namespace ddst
