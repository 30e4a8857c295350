// hbs.cuh -- nested-basis HBS form of the transfer operators, compressed from random samples
// (Sec. 2.4; Alg. 1 draws s = 3k + q Gaussian samples Y = S Omega, Z = S^T Psi).
#pragma once
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"

namespace ddst {

// One tree node of one block, in heap order per block (root 0, children of i at 2i+1, 2i+2).
// Levels 1..L carry U (n x k), V (n x k) and D (n x n), column-major; the root (level 0) carries
// D_0 only (2k x 2k, or the whole block when the tree has one level).
struct HbsNode {
  int blk;          // block id
  int level;
  int n;            // rows of the node's row set (leaves: index count; inner nodes and root: 2k)
  int t;            // index within its level
  int64_t lo;       // first index of the node's range in the bisection tree (t ng >> level)
  int64_t in_row;   // compression: first sample row of the node in the current level buffer
  int64_t out_row;  // compression: first of its k reduced rows in the next level's buffer
  int64_t u_off, v_off, d_off;  // factor offsets (elements); -1 where absent
};

// Per block: tree shape and apply scratch.  x_hat holds V^T x (U^T x transposed) of every node
// at levels 1..L (k entries at xh_off + heap index * k), y_hat the downward vectors of the root
// and the inner nodes (2k entries at yh_off + heap index * 2k), both FP64.
struct HbsBlock {
  int64_t ng;
  int L;
  int node0;        // first node (heap index 0) in the node array
  int64_t xh_off;   // x_hat scratch offset (FP64 entries)
  int64_t yh_off;   // y_hat scratch offset
  int64_t in_if, out_if;  // interface offsets of the source and target vectors (0 and 0 alone)
};

// Output item of the apply: the rows of one subtree of one output interface (node: the
// subtree's root; the whole block when its tree has one level); up to two blocks
// write there (S_{j,j-1} and S_{j,j+1} onto Gamma_j; transposed: S_{j+1,j}^T and S_{j-1,j}^T).
struct HbsOwn {
  int64_t out;      // interface offset of the output rows (+ lo)
  int64_t lo;
  int len;
  int nsrc;
  int blk[2];
  int node[2];      // subtree root node (absolute index)
};

struct HbsLeafItem {  // up-pass item: one subtree of one block
  int blk;
  int node;          // absolute index of the subtree's root node
};

struct HbsSet {
  bool built = false;
  size_t esz = 4;
  int k = 0, s = 0, leaf = 0;
  int max_L = 0;                // deepest tree over the blocks
  void* F = nullptr;            // factors (element type of the context)
  double* scratch = nullptr;    // x_hat and y_hat
  HbsNode* d_nodes = nullptr;
  HbsBlock* d_blocks = nullptr;
  HbsOwn* d_own = nullptr;
  HbsOwn* d_own_T = nullptr;
  HbsLeafItem* d_leaf_items = nullptr;
  int n_leaf_items = 0;
  std::vector<HbsNode> nodes;
  std::vector<HbsBlock> blocks;
  int n_own = 0, n_own_T = 0;
  int64_t f_elems = 0;
  int64_t bytes = 0;
  std::vector<int> blk_slab, blk_side;  // context blocks: slab and side (-1 / +1)
  std::vector<std::pair<int64_t, int64_t>> bare;  // interfaces no block writes: (offset, length)
  void release();
};

// Input of one block: S column-major (S[c * ng + r]) and, optionally, the test matrices
// (row-major ng x s FP64 host arrays; NULL: drawn on the device from the seed).  A standalone
// block has in_if = out_if = 0, and the apply with bit 1 set then gives y = S_H x.
struct HbsInput {
  const void* S;
  int64_t ng;
  const double* omega;
  const double* psi;
  int64_t in_if, out_if;
  int slab, side;
};

// Shared-memory bytes of the node kernel for row sets of up to n_max rows.
size_t hbs_node_smem(int n_max, int s, int k, size_t esz);

// Compresses every block (`bare`: interfaces that no block writes, where K = 0, given as
// (offset, length)); returns 0 on success, 1 on CUDA error, 2 on OOM, 3 on a bad argument
// (k < 1, a node's rows + k above s, shared memory above the per-CTA limit).
template <typename T>
int hbs_build(HbsSet& H, const std::vector<HbsInput>& in,
              const std::vector<std::pair<int64_t, int64_t>>& bare, int k, int s, int leaf,
              uint64_t seed, cudaStream_t st, std::string& msg);

// Apply: y = (I - K) x or (I - K)^T x (bit 0), y = K x or K^T x with bit 1 set.  With
// kdev the input is x + (*kdev - 1) * kstride (graph-capturable Krylov index).
template <typename T>
void hbs_apply(HbsSet& H, const double* x, double* y, int transpose, cudaStream_t st,
               const int* kdev = nullptr, int64_t kstride = 0);

// Dense column-major expansion of block b into host memory (ng * ng doubles).
int hbs_expand(HbsSet& H, int b, double* out, cudaStream_t st);

}  // namespace ddst
