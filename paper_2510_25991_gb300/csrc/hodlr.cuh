// hodlr.cuh -- weak-admissibility hierarchical (HODLR) form of the transfer operators.
#pragma once
#include <string>
#include <vector>

#include "common.cuh"

namespace ddst {

struct HodlrParams {
  double tol;      // relative truncation tolerance (w.r.t. ||S_{j,j'}||_2)
  int k_max;       // rank cap
  int oversample;  // extra samples
  int leaf;        // leaf size
  uint64_t seed;   // sketch seed
};

// One low-rank off-diagonal block (device offsets in elements of the working precision).
struct HBlock {
  int sblk;        // S block id: 2 * slab + (side > 0)
  int level;
  int64_t row0, nrows, col0, ncols;
  int rank;
  int64_t u_off;   // U: nrows x rank, column-major
  int64_t v_off;   // V: ncols x rank, column-major (block ~ U V^T)
  int64_t t_off;   // scratch offset for V^T x
  int64_t in_if, out_if;  // interface offsets of source / target vectors
};

struct HLeaf {
  int sblk;
  int64_t lo, len;
  int64_t ld;      // leading dimension: len rounded up to a multiple of 4 (zero rows below len)
  int64_t d_off;   // dense leaf, column-major ld x len
  int64_t in_if, out_if;
};

// Output-owner work item of the apply: rows [lo, lo + len) of one interface (a leaf range of
// the shared cluster tree).  Up to two S blocks write there (S_{j,j-1} and S_{j,j+1} onto
// Gamma_j; transposed: S_{j+1,j}^T and S_{j-1,j}^T); for each, its dense leaf over these rows
// and, per tree level, the low-rank block whose output range holds them (-1: none / rank 0).
constexpr int HOWN_MAXL = 12;
constexpr int HOWN_TCAP = 16;  // t_b entries per block staged in shared memory by the apply
struct HOwn {
  int64_t out;                 // interface offset of the output rows
  int64_t lo;                  // first row within the interface
  int len;                     // number of rows (<= 256)
  int nsrc;                    // contributing S blocks (0..2)
  int leaf[2];
  int hb[2][HOWN_MAXL];
};

struct HodlrSet {
  bool built = false;
  size_t esz = 4;
  void* UV = nullptr;      // factors
  void* D = nullptr;       // dense leaves
  double* t = nullptr;     // V^T x (U^T x when transposed) per low-rank block (FP64)
  HBlock* d_blocks = nullptr;
  HLeaf* d_leaves = nullptr;
  std::vector<HBlock> blocks;
  std::vector<HLeaf> leaves;
  HOwn* d_own = nullptr;      // output-owner items of the apply
  HOwn* d_own_T = nullptr;    // ... of the transposed apply
  int n_own = 0, n_own_T = 0;
  int64_t t_len = 0;
  int64_t bytes = 0;
  int max_rank = 0;
  std::vector<int> sblk_L;     // tree depth per S block
  std::vector<int> sblk_slab;  // slab of each S block
  std::vector<int> sblk_side;  // -1: S_{j,j-1}, +1: S_{j,j+1}
  void clear();
  void release();
};

// Compresses every dense S block; returns 0 on success, 1 on CUDA error, 2 on OOM, 3 when the
// cluster tree would be deeper than HOWN_MAXL levels (an argument error).
template <typename T>
int hodlr_build(HodlrSet& H, const HodlrParams& hp, const std::vector<SlabDesc>& slabs,
                const std::vector<ProbDesc>& probs, const SlabDesc* d_slabs, const T* S,
                cudaStream_t st, std::string& msg);

// y = (I - K) x (transpose bit 0 clear) or (I - K)^T x with the HODLR blocks; with bit 1 set,
// y = K x (or K^T x).  When kdev is given the input is x + (*kdev - 1) * kstride
// (device-resident Krylov index, graph-capturable).
template <typename T>
void hodlr_apply(HodlrSet& H, const SlabDesc* d_slabs, const ProbDesc* d_probs, int nslab,
                 const double* x, double* y, int transpose, cudaStream_t st,
                 const int* kdev = nullptr, int64_t kstride = 0);

// Dense column-major expansion of S block (slab, side) into host memory `out` (ng*ng doubles).
int hodlr_expand(HodlrSet& H, int slab, int side, size_t esz, double* out, cudaStream_t st);

}  // namespace ddst
