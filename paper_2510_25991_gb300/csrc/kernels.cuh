// kernels.cuh -- host-side launchers of the device kernels (all stream-ordered, no sync).
#pragma once
#include "common.cuh"

namespace ddst {

// One CTA of the multi-right-hand-side sweep that forms S explicitly (sweep.cu).
struct TileDesc {
  int slab;    // global slab index
  int q0;      // first central source point of the tile
  int nq;      // number of sources in the tile (<= tile width)
  int dir;     // 0 = upward sweep (blocks kstart..1), 1 = downward (kstart..nb)
  int kstart;  // first block of the sweep
  int len;     // number of blocks visited
};

// stencil.cu
template <typename T>
void launch_stencil_pack(const SlabDesc* d_slabs, int nslab, int max_nb, const ProbDesc* d_probs,
                         const double* a, const double* c, T* pack, cudaStream_t st);
void launch_rhs(const ProbDesc* d_probs, int nprob, const double* a, const double* f,
                const double* g, double* b, cudaStream_t st);
void launch_residual(const ProbDesc* d_probs, int nprob, const double* a, const double* c,
                     const double* b, const double* u, double* r, int transpose, double* part,
                     int nblk, cudaStream_t st);
template <typename T>
void launch_gather(const SlabDesc* d_slabs, int nslab, const double* vol, T* loc, cudaStream_t st);
template <typename T>
void launch_gather_owned(const SlabDesc* d_slabs, const ProbDesc* d_probs, int nslab,
                         const double* vol, T* loc, cudaStream_t st);
template <typename T>
void launch_gather_T(const SlabDesc* d_slabs, int nslab, const T* loc, double* vol,
                     cudaStream_t st);
template <typename T>
void launch_scatter(const SlabDesc* d_slabs, const ProbDesc* d_probs, int nslab, const T* loc,
                    double* vol, int mode, cudaStream_t st);
template <typename T>
void launch_extract_center(const SlabDesc* d_slabs, int nslab, const T* loc, double* iface,
                           cudaStream_t st);
template <typename T>
void launch_inject_center(const SlabDesc* d_slabs, int nslab, const double* iface, T* loc,
                          cudaStream_t st);
template <typename T>
void launch_add_iface_dirichlet(const SlabDesc* d_slabs, const ProbDesc* d_probs, int nslab,
                                const T* pack, const double* uG, T* loc, cudaStream_t st);
template <typename T>
void launch_iface_dirichlet_T(const SlabDesc* d_slabs, const ProbDesc* d_probs, int nslab,
                              const T* pack, const T* loc, double* out, cudaStream_t st);
void launch_dot(const double* x, const double* y, int64_t n, double* part, int nblk, double* out,
                cudaStream_t st);
// out[q] = sum of squares of x over problem q's interior unknowns (part: nprob * nblk doubles).
void launch_prob_sqnorms(const ProbDesc* d_probs, int nprob, const double* x, double* part,
                         int nblk, double* out, cudaStream_t st);
void launch_axpy(int64_t n, double a, const double* x, double* y, cudaStream_t st);
// f = u / dt - v . grad_h u on every problem's interior (u = 0 on the boundary nodes); vel holds
// component d of the nodal velocity of every problem at vel + d tot_nodes.
void launch_imex_rhs(const ProbDesc* d_probs, int nprob, const double* u, const double* vel,
                     int64_t tot_nodes, double inv_dt, double* f, cudaStream_t st);

// One CTA of the pivot sweeps (factor.cu): rows start..last of one slab and direction, inverses
// stored from `first` on, warm-up inverse of row first-1 (first+1 backward) into check slot chk.
struct FacChunk {
  int slab;
  int dir;     // 0 forward (F), 1 backward (B)
  int start;   // first row visited (1-based)
  int first;   // first row whose inverse is stored
  int last;    // last row visited
  int chk;     // check slot, -1 when the chunk starts at the slab's end row (exact)
};

// factor.cu: phase 0 = pivot sweeps F, B (+ transposes) and chunk verification (diff[chunk]);
// phase 1 = diagonal inverse blocks G.  One block-size class per call.
// Uhi/Ulo (FP32 only, may be NULL): tensor-core operand copies of F^T (first umma_elems
// elements) and B^T (next umma_elems), TF32 hi/lo split, K-major operand layout (umma.cuh).
template <typename T>
void launch_factor(int M, int phase, const SlabDesc* d_slabs, const FacChunk* d_chunks,
                   int nchunks, const int* d_ids, int nids, int max_nb, const T* pack, T* F,
                   T* B, T* G, T* Ft, T* Bt, T* chk, float* diff, float* Uhi, float* Ulo,
                   int64_t umma_elems, DevStatus* st, cudaStream_t s);
template <typename T>
int factor_ctas_per_sm(int M);

// sweep.cu: explicit transfer operators
template <typename T>
int sbuild_tile_cols(int M);
template <typename T>
void launch_sbuild(int M, const SlabDesc* d_slabs, const TileDesc* d_tiles, int ntiles,
                   const T* F, const T* B, const T* G, const T* pack, T* S, DevStatus* st,
                   cudaStream_t s);

// sweep_tc.cu: explicit transfer operators on tcgen05 (FP32 data, 3xTF32), M in {32, 64};
// budget: clock cycles before a pipeline wait of a role gives up (ST_TIMEOUT); three: 3xTF32 (1)
// or TF32 (0)
void launch_sbuild_tc(int M, const SlabDesc* d_slabs, const TileDesc* d_tiles, int ntiles,
                      const float* Fhi, const float* Flo, const float* Bhi, const float* Blo,
                      const float* G, const float* pack, float* S, DevStatus* st,
                      long long budget, int three, cudaStream_t s);
int sbuild_tc_tile_cols();  // sources per CTA of the tensor-core transfer build

// solve.cu: single-RHS local solves (mode 0: full block into x; mode 1: central rows -> iface)
template <typename T>
// F, B row-major inverses; Ft, Bt their transposes.
void launch_local_solve(int M, const SlabDesc* d_slabs, const int* d_ids, int nids, int max_nb,
                        const T* F, const T* B, const T* Ft, const T* Bt, const T* G,
                        const T* pack, const T* b, T* bf, T* bb, T* x, double* iface,
                        int transpose, int mode, DevStatus* st, cudaStream_t s);

// krylov.cu
// x may be indexed by a device-resident basis count: x_eff = x + (*kdev - 1) * kstride.
// transpose: bit 0 = transposed operator, bit 1 = y = K x instead of (I - K) x.
template <typename T>
void launch_apply_dense(const SlabDesc* d_slabs, const ProbDesc* d_probs, int nslab,
                        int64_t max_ng, const T* S, const double* x, double* y, int transpose,
                        cudaStream_t st, const int* kdev = nullptr, int64_t kstride = 0);
// One Arnoldi step (CGS2) with device-resident state; graph-capturable (arguments fixed).
void launch_arnoldi_step(double* V, double* w, int64_t n, int* kdev, double* h1, double* h2,
                         double* part, unsigned* ticket, double* H, int ldh, double* cs,
                         double* sn, double* gv, const double* beta, double* resid, int kmax,
                         cudaStream_t st);
int arnoldi_chunks(int64_t n);  // chunks of the Arnoldi kernels (partial sums per chunk)
void launch_combine_basis(const double* V, const double* y, int k, int64_t n, double* x,
                          cudaStream_t st);
void launch_normalize_start(const double* x, const double* nrm2, double* out, int64_t n,
                            cudaStream_t st);
void launch_trisolve(const double* H, int ldh, const double* gv, int kk, double* y,
                     cudaStream_t st);

// bigblock.cu: large dense blocks (M a multiple of 128).  One block row k of the one-sided block
// LU of every slab in the class (Sigma_k formed in the slot of F_k, inverted there by 128-wide
// Gauss-Jordan panels with look-ahead on two streams: sh high priority, sl the bulk updates; ev
// three events).  Two sets of work buffers (alternating by panel parity), each Cb, XqT, RT
// (nids x M x 128, twice that when split for the tensor cores) and Pinv (nids x 128 x 128, or
// twice).  tensor_cores: 0 FMA, 1 tcgen05 3xTF32, 2 tcgen05 TF32.  form_sigma = 0 skips the
// Schur complement and inverts the block already in the slot of F_k (the pivot floor is then
// 1e3 eps |pack diagonal|).  All work is ordered before later work on sh.
template <typename T>
void launch_big_factor_step(int M, const SlabDesc* d_slabs, const int* d_ids, int nids,
                            const T* pack, T* F, int k, T* const Cb[2], T* const XqT[2],
                            T* const RT[2], T* const Pinv[2], int tensor_cores, DevStatus* st,
                            cudaStream_t sh, cudaStream_t sl, cudaEvent_t* ev, int form_sigma = 1);
// Local solve x = A^{-1} b (transpose 0) or A^{-T} b (transpose 1) of every slab of the class;
// z is a slab-local temporary.
template <typename T>
void launch_big_solve(int M, const SlabDesc* d_slabs, const int* d_ids, int nids, int max_nb,
                      const T* F, const T* pack, const T* b, T* z, T* x, int transpose,
                      cudaStream_t s);
template <typename T>
void launch_big_extract(const SlabDesc* d_slabs, const int* d_ids, int nids, const T* loc,
                        double* iface, cudaStream_t s);

// gemm_tc.cu: batched products of square blocks of edge 128 nT (row-major, leading dimension
// 128 nT).  Packing writes pre-split TF32 tiles: trans 0 for an A operand, 1 for a B operand
// (packed as B^T); a packed block takes 2 (128 nT)^2 floats.
struct PackTask {
  const float* src;
  float* dst;
  int trans;
};
struct GemmTask {  // C = alpha A B (+ C when accumulate), A and B packed
  const float* A;
  const float* B;
  float* C;
  float alpha;
  int accumulate;
};
template <typename T>
struct GemmTaskT {  // the same on plain row-major blocks (FMA kernel)
  const T* A;
  const T* B;
  T* C;
  T alpha;
  int accumulate;
};
void launch_pack_split(const PackTask* d_tasks, int ntasks, int nT, cudaStream_t st);
// three: 1 3xTF32, 0 TF32.  Timeouts of the bounded waits are recorded in *dst.
void launch_gemm_tc(const GemmTask* d_tasks, int ntasks, int nT, int three, DevStatus* dst,
                    cudaStream_t st);
template <typename T>
void launch_gemm_fma(const GemmTaskT<T>* d_tasks, int ntasks, int nT, cudaStream_t st);

// bcr.cu: products of interface blocks with FP64 vectors for the direct interface solve.
// Task: y = x0 + coef sum over its terms of op(M_t) v_t (op = transpose or not, M_t blocks of
// leading dimension ldm, vectors of length n; NULL terms and a NULL x0 count as zero).  x0 may
// alias y; the v_t may not.
template <typename T>
struct BlockMv {
  double* y;
  const double* x0;
  double coef;
  const T* M[2];
  const double* v[2];
};
template <typename T>
void launch_block_mv(const BlockMv<T>* d_tasks, int ntasks, int n, int ldm, int transpose,
                     cudaStream_t st);

// matfree.cu: the interface operator through local solves, over the listed slabs (x indexed by
// kdev as above)
template <typename T>
void launch_mf_rhs(const SlabDesc* d_slabs, const int* d_ids, int nids, const ProbDesc* d_probs,
                   const T* pack, const double* x, const int* kdev, int64_t kstride, T* loc,
                   cudaStream_t st);
template <typename T>
void launch_mf_inject(const SlabDesc* d_slabs, const int* d_ids, int nids, const double* x,
                      const int* kdev, int64_t kstride, T* loc, cudaStream_t st);
template <typename T>
void launch_mf_dirichlet_T(const SlabDesc* d_slabs, const int* d_ids, int nids,
                           const ProbDesc* d_probs, const T* pack, const T* loc, double* out,
                           cudaStream_t st);
void launch_mf_combine(const SlabDesc* d_slabs, const int* d_ids, int nids, const double* x,
                       const int* kdev, int64_t kstride, const double* kx, double* y, int konly,
                       cudaStream_t st);

// grad.cu: dL/dg and dL/da from lambda and u (nodal outputs accumulated; zero them first)
void launch_gradients(const ProbDesc* d_probs, int nprob, const double* a, const double* g,
                      const double* u, const double* lam, double* dLdg, double* dLda,
                      cudaStream_t st);

}  // namespace ddst
