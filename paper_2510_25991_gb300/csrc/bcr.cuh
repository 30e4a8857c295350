// bcr.cuh -- direct solver of the equilibrium system by block cyclic reduction (host side).
#pragma once
#include <cuda_runtime.h>

#include <functional>
#include <vector>

#include "kernels.cuh"

namespace ddst {

// One level of the reduction: the blocks at odd positions of the current list are eliminated.
struct BcrLevel {
  std::vector<int> odd, even;      // block ids (interface j - 1)
  std::vector<int> oleft, oright;  // per odd block: the neighbouring even blocks (right: -1)
  std::vector<int> eleft, eright;  // per even block: the neighbouring odd blocks (-1: none)
  std::vector<int> pslot, qslot;   // per even block: slots of P_j, Q_j (-1: none)
};

// One problem's factored system (I - K) u = fhat with N_ds blocks of n_Gamma unknowns, stored
// padded to NG = 128 nT: D holds the inverses of the eliminated diagonal blocks, L and U each
// block's couplings at the level it was eliminated, PQ the products P_j = L_j D_left^{-1} and
// Q_j = U_j D_right^{-1} of the blocks that stayed.
struct BcrSystem {
  int nds = 0, NG = 0, nT = 0, npq = 0, last = 0;
  int64_t ng = 0;
  size_t esz = 0;
  void *D = nullptr, *L = nullptr, *U = nullptr, *PQ = nullptr;
  std::vector<BcrLevel> levels;
  // device task lists of the solves (built for one pair of solve buffers)
  const double* tasks_x = nullptr;
  void* d_tasks = nullptr;
  std::vector<std::pair<int, int>> runs[2];  // per direction: (first task, count) per launch
  std::vector<int> run_trans[2];              // per launch: transposed product
};

// What the factorization needs from its context.
struct BcrEnv {
  std::function<cudaError_t(void**, size_t)> alloc;
  std::function<void(void*&)> release;
  cudaStream_t st = nullptr, sh = nullptr, sl = nullptr;
  cudaEvent_t* ev = nullptr;  // 5 events: 3 for the panel look-ahead, 2 to join the streams
  DevStatus* d_st = nullptr;
  int tensor_cores = 0;       // 0 FMA, 1 3xTF32, 2 TF32 (FP32 only)
};

// Factors one problem's system from its explicit transfer blocks: S (element type T, row-major
// n_Gamma x n_Gamma blocks) with S_{j,j-1} at sp_off[j - 1] and S_{j,j+1} at sn_off[j - 1]
// (-1: none).  Returns a CUDA error, or cudaSuccess after the work is enqueued on env.st.
template <typename T>
cudaError_t bcr_factor(BcrSystem& B, const T* S, const std::vector<int64_t>& sp_off,
                       const std::vector<int64_t>& sn_off, int nds, int64_t ng,
                       const BcrEnv& env);

// x := (I - K)^{-1} x, or (I - K)^{-T} x (transpose), for one problem: x and tmp are its
// N_ds n_Gamma FP64 interface values.  The task lists are rebuilt when x changes.
template <typename T>
cudaError_t bcr_solve(BcrSystem& B, double* x, double* tmp, int transpose, const BcrEnv& env);

void bcr_free(BcrSystem& B, const BcrEnv& env);

}  // namespace ddst
