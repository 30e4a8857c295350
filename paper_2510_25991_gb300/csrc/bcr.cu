// bcr.cu -- direct solve of the equilibrium system (I - K) u = fhat by block cyclic reduction.
//
// The equilibrium system of Sec. 1, Eq. (modelS) (Sec. 2.2, Eq. (equilib2)) is block
// tridiagonal with identity diagonal blocks and the transfer blocks -S_{j,j-1}, -S_{j,j+1} off
// it; Sec. 4 (direct solvers) proposes block tridiagonal elimination for it as the remedy when
// GMRES iteration counts grow (H -> 0, oscillatory problems).  Here it is eliminated by block
// cyclic reduction: each level removes the blocks at odd positions of the remaining list, all of
// them at once, with block j (even position, odd neighbours a = left, c = right) updated by
//     P_j = L_j D_a^{-1},  Q_j = U_j D_c^{-1},
//     D_j -= P_j U_a + Q_j L_c,   L_j <- -P_j L_a,   U_j <- -Q_j U_c,
// so a level is one batched inversion of the eliminated diagonal blocks (the large-block
// Gauss-Jordan panels of bigblock.cu) and batched dense products (gemm_tc.cu: tcgen05 3xTF32 in
// FP32, FMA in FP64).  The solve replays the levels: forward, r_j -= P_j r_a + Q_j r_c; the last
// block, u = D^{-1} r; backward, u_i = D_i^{-1} (r_i - L_i u_left - U_i u_right).  The transposed
// system uses the same factors transposed (forward z_i = D_i^{-T} s_i, s_j -= L_c^T z_c +
// U_a^T z_a; backward y_i = z_i - P_right^T y_right - Q_left^T y_left).
#include <algorithm>

#include "bcr.cuh"
#include "common.cuh"
#include "splittile.cuh"

namespace ddst {

// ---------------------------------------------------------------------------------------------
// Initial blocks: dst (NG x NG, row-major, padded) = sign * src on the top-left n x n, zero
// elsewhere, where src holds the transfer block column by column (the transfer build writes one
// source point's column at a time); identity when src is NULL (the diagonal blocks, padding
// included).  32 x 32 tiles transposed through shared memory, grid = (NG/32, NG/32), 32 x 8.
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_bcr_init(const T* __restrict__ src, int64_t n,
                                                  T* __restrict__ dst, int NG, T sign) {
  __shared__ T tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (src) {
    for (int k = ty; k < 32; k += 8) {  // src column c0 + k, rows r0 + tx (coalesced)
      const int64_t c = c0 + k, r = r0 + tx;
      tile[k][tx] = (r < n && c < n) ? src[c * n + r] : T(0);
    }
    __syncthreads();
  }
  for (int k = ty; k < 32; k += 8) {  // dst row r0 + k, columns c0 + tx (coalesced)
    const int64_t r = r0 + k, c = c0 + tx;
    dst[r * NG + c] = src ? sign * tile[tx][k] : (r == c ? T(1) : T(0));
  }
}

// ---------------------------------------------------------------------------------------------
// Block products with FP64 vectors.  Task: y = x0 + coef sum_t op(M_t) v_t over rows r < n (x0
// NULL: zero).  Not transposed: a warp per row, grid = (ceil(n / 8), tasks), 256 threads, the
// task's vectors staged in shared memory.  Transposed: a CTA per 32 columns, the 8 warps split
// the rows and reduce through shared memory.
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_block_mv_n(const BlockMv<T>* __restrict__ tasks, int n,
                                                    int ldm, int staged) {
  extern __shared__ double vs[];  // 2 n when staged
  const BlockMv<T> t = tasks[blockIdx.y];
  if (staged) {
    for (int e = threadIdx.x; e < 2 * n; e += blockDim.x) {
      const int s = e / n, k = e - s * n;
      vs[e] = t.v[s] ? t.v[s][k] : 0.0;
    }
    __syncthreads();
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * 8 + warp;
  if (r >= n) return;
  double acc = 0.0;
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    if (!t.M[s]) continue;
    const T* row = t.M[s] + (int64_t)r * ldm;
    const double* v = staged ? vs + s * n : t.v[s];
    for (int k = lane; k < n; k += 32) acc += static_cast<double>(row[k]) * v[k];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) t.y[r] = (t.x0 ? t.x0[r] : 0.0) + t.coef * acc;
}

template <typename T>
__global__ void __launch_bounds__(256) k_block_mv_t(const BlockMv<T>* __restrict__ tasks, int n,
                                                    int ldm) {
  __shared__ double red[8][33];
  const BlockMv<T> t = tasks[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * 32 + lane;
  double acc = 0.0;
  if (c < n) {
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (!t.M[s]) continue;
      const T* col = t.M[s] + c;
      const double* v = t.v[s];
      for (int k = warp; k < n; k += 8) acc += static_cast<double>(col[(int64_t)k * ldm]) * v[k];
    }
  }
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && c < n) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += red[w][lane];
    t.y[c] = (t.x0 ? t.x0[c] : 0.0) + t.coef * s;
  }
}

template <typename T>
void launch_block_mv(const BlockMv<T>* d_tasks, int ntasks, int n, int ldm, int transpose,
                     cudaStream_t st) {
  if (ntasks <= 0) return;
  note_launch();
  if (!transpose) {
    const int staged = n <= 8192 ? 1 : 0;  // 128 KB of shared memory at most
    const size_t sm = staged ? sizeof(double) * 2 * n : 0;
    raise_smem_limit(reinterpret_cast<const void*>(&k_block_mv_n<T>), sm);
    k_block_mv_n<T><<<dim3((n + 7) / 8, ntasks), 256, sm, st>>>(d_tasks, n, ldm, staged);
  } else {
    k_block_mv_t<T><<<dim3((n + 31) / 32, ntasks), 256, 0, st>>>(d_tasks, n, ldm);
  }
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
namespace {

struct Scratch {  // device buffers that live for one factorization
  std::vector<void*> bufs;
  const BcrEnv* env;
  ~Scratch() {
    for (void*& p : bufs) env->release(p);
  }
  cudaError_t get(void** p, size_t bytes) {
    const cudaError_t e = env->alloc(p, bytes);
    if (e == cudaSuccess) bufs.push_back(*p);
    return e;
  }
};

template <typename T>
cudaError_t upload(Scratch& sc, const std::vector<T>& h, T** d, cudaStream_t st) {
  if (h.empty()) { *d = nullptr; return cudaSuccess; }
  cudaError_t e = sc.get(reinterpret_cast<void**>(d), sizeof(T) * h.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(*d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);  // h is a host temporary
}

}  // namespace

template <typename T>
cudaError_t bcr_factor(BcrSystem& B, const T* S, const std::vector<int64_t>& sp_off,
                       const std::vector<int64_t>& sn_off, int nds, int64_t ng,
                       const BcrEnv& env) {
  cudaStream_t st = env.st;
  B.nds = nds;
  B.ng = ng;
  B.NG = (int)((ng + BT - 1) / BT) * BT;
  B.nT = B.NG / BT;
  B.esz = sizeof(T);
  const int NG = B.NG, nT = B.nT;
  const size_t blk = (size_t)NG * NG;
  // level structure
  B.levels.clear();
  std::vector<int> cur(nds);
  for (int j = 0; j < nds; ++j) cur[j] = j;
  int npq = 0, max_odd = 1, max_even = 0;
  while (cur.size() > 1) {
    BcrLevel lv;
    const int m = (int)cur.size();
    for (int p = 0; p < m; ++p) {
      if (p & 1) {
        lv.odd.push_back(cur[p]);
        lv.oleft.push_back(cur[p - 1]);
        lv.oright.push_back(p + 1 < m ? cur[p + 1] : -1);
      } else {
        lv.even.push_back(cur[p]);
        lv.eleft.push_back(p >= 1 ? cur[p - 1] : -1);
        lv.eright.push_back(p + 1 < m ? cur[p + 1] : -1);
        lv.pslot.push_back(p >= 1 ? npq++ : -1);
        lv.qslot.push_back(p + 1 < m ? npq++ : -1);
      }
    }
    max_odd = std::max(max_odd, (int)lv.odd.size());
    max_even = std::max(max_even, (int)lv.even.size());
    cur = lv.even;
    B.levels.push_back(std::move(lv));
  }
  B.last = cur[0];
  B.npq = npq;
  cudaError_t e;
  if ((e = env.alloc(&B.D, sizeof(T) * blk * nds)) != cudaSuccess) return e;
  if ((e = env.alloc(&B.L, sizeof(T) * blk * nds)) != cudaSuccess) return e;
  if ((e = env.alloc(&B.U, sizeof(T) * blk * nds)) != cudaSuccess) return e;
  if (npq > 0 && (e = env.alloc(&B.PQ, sizeof(T) * blk * npq)) != cudaSuccess) return e;
  T* D = (T*)B.D;
  T* L = (T*)B.L;
  T* U = (T*)B.U;
  T* PQ = (T*)B.PQ;
  auto blkp = [&](T* base, int j) { return base + (size_t)j * blk; };
  const dim3 ig(NG / 32, NG / 32), ib(32, 8);
  for (int j = 0; j < nds; ++j) {
    note_launch();
    k_bcr_init<T><<<ig, ib, 0, st>>>(nullptr, ng, blkp(D, j), NG, T(1));
    note_launch();
    k_bcr_init<T><<<ig, ib, 0, st>>>(sp_off[j] >= 0 ? S + sp_off[j] : nullptr, ng, blkp(L, j),
                                     NG, T(-1));
    note_launch();
    k_bcr_init<T><<<ig, ib, 0, st>>>(sn_off[j] >= 0 ? S + sn_off[j] : nullptr, ng, blkp(U, j),
                                     NG, T(-1));
  }
  // a block without a neighbour on one side has no coupling there: zero it (not identity)
  if (sp_off[0] < 0 && (e = cudaMemsetAsync(blkp(L, 0), 0, sizeof(T) * blk, st)) != cudaSuccess) return e;
  if (sn_off[nds - 1] < 0 &&
      (e = cudaMemsetAsync(blkp(U, nds - 1), 0, sizeof(T) * blk, st)) != cudaSuccess) return e;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  Scratch sc{{}, &env};
  // inversions: every block is a one-block "slab" of edge NG whose pivot floor is 1e3 eps
  std::vector<SlabDesc> vs(nds);
  for (int j = 0; j < nds; ++j) {
    SlabDesc s{};
    s.prob = 0; s.j = j + 1; s.M = NG; s.m = (int)ng; s.nb = 1; s.p = 1; s.w = 1; s.n = 0;
    s.ng = ng; s.fac_off = (int64_t)j * (int64_t)blk; s.pack_off = 0; s.loc_off = 0;
    s.sp_off = -1; s.sn_off = -1;
    vs[j] = s;
  }
  SlabDesc* d_vs = nullptr;
  if ((e = upload(sc, vs, &d_vs, st)) != cudaSuccess) return e;
  std::vector<T> ones((size_t)PK_NFIELDS * NG, T(0));
  for (int i = 0; i < NG; ++i) ones[(size_t)PK_DIAG * NG + i] = T(1);
  T* d_ones = nullptr;
  if ((e = upload(sc, ones, &d_ones, st)) != cudaSuccess) return e;
  const bool split = sizeof(T) == 4 && env.tensor_cores != 0;
  T *Cb[2], *XqT[2], *RT[2], *Pinv[2];
  const size_t panel = 2 * sizeof(T) * (size_t)max_odd * NG * BT;
  for (int b = 0; b < 2; ++b) {
    if ((e = sc.get(reinterpret_cast<void**>(&Cb[b]), panel)) != cudaSuccess) return e;
    if ((e = sc.get(reinterpret_cast<void**>(&XqT[b]), panel)) != cudaSuccess) return e;
    if ((e = sc.get(reinterpret_cast<void**>(&RT[b]), panel)) != cudaSuccess) return e;
    if ((e = sc.get(reinterpret_cast<void**>(&Pinv[b]), 2 * sizeof(T) * (size_t)max_odd * BT * BT)) != cudaSuccess)
      return e;
  }
  auto invert = [&](const std::vector<int>& ids) -> cudaError_t {
    int* d_ids = nullptr;
    cudaError_t e2 = upload(sc, ids, &d_ids, st);
    if (e2 != cudaSuccess) return e2;
    if ((e2 = cudaEventRecord(env.ev[3], st)) != cudaSuccess) return e2;
    if ((e2 = cudaStreamWaitEvent(env.sh, env.ev[3], 0)) != cudaSuccess) return e2;
    launch_big_factor_step<T>(NG, d_vs, d_ids, (int)ids.size(), d_ones, D, 1, Cb, XqT, RT, Pinv,
                              env.tensor_cores, env.d_st, env.sh, env.sl, env.ev, 0);
    if ((e2 = cudaGetLastError()) != cudaSuccess) return e2;
    if ((e2 = cudaEventRecord(env.ev[4], env.sh)) != cudaSuccess) return e2;
    return cudaStreamWaitEvent(st, env.ev[4], 0);
  };
  // packed operands (tensor-core path): A slots 2 per even block, B slots 3 per odd block
  float *Apk = nullptr, *Bpk = nullptr;
  const size_t pblk = 2 * blk;  // floats of one packed block (hi + lo)
  if (split) {
    if ((e = sc.get(reinterpret_cast<void**>(&Apk), sizeof(float) * pblk * 2 * std::max(max_even, 1))) != cudaSuccess)
      return e;
    if ((e = sc.get(reinterpret_cast<void**>(&Bpk), sizeof(float) * pblk * 3 * max_odd)) != cudaSuccess)
      return e;
  }
  for (const BcrLevel& lv : B.levels) {
    if ((e = invert(lv.odd)) != cudaSuccess) return e;
    const int ne = (int)lv.even.size(), no = (int)lv.odd.size();
    std::vector<int> opos(nds, -1);  // odd block id -> position in this level's odd list
    for (int o = 0; o < no; ++o) opos[lv.odd[o]] = o;
    if constexpr (sizeof(T) == 4) {
      if (split) {
        float* Df = reinterpret_cast<float*>(D);
        float* Lf = reinterpret_cast<float*>(L);
        float* Uf = reinterpret_cast<float*>(U);
        float* PQf = reinterpret_cast<float*>(PQ);
        auto aslot = [&](int ei, int w) { return Apk + pblk * (size_t)(2 * ei + w); };
        auto bslot = [&](int o, int w) { return Bpk + pblk * (size_t)(3 * o + w); };
        const int three = env.tensor_cores == 1 ? 1 : 0;
        std::vector<PackTask> pk;
        for (int ei = 0; ei < ne; ++ei) {
          const int j = lv.even[ei];
          if (lv.eleft[ei] >= 0) pk.push_back({Lf + (size_t)j * blk, aslot(ei, 0), 0});
          if (lv.eright[ei] >= 0) pk.push_back({Uf + (size_t)j * blk, aslot(ei, 1), 0});
        }
        for (int o = 0; o < no; ++o) {
          const int i = lv.odd[o];
          pk.push_back({Df + (size_t)i * blk, bslot(o, 0), 1});
          pk.push_back({Lf + (size_t)i * blk, bslot(o, 1), 1});
          if (lv.oright[o] >= 0) pk.push_back({Uf + (size_t)i * blk, bslot(o, 2), 1});
        }
        PackTask* d_pk = nullptr;
        if ((e = upload(sc, pk, &d_pk, st)) != cudaSuccess) return e;
        launch_pack_split(d_pk, (int)pk.size(), nT, st);
        std::vector<GemmTask> g1, g2;
        std::vector<PackTask> pk2;
        for (int ei = 0; ei < ne; ++ei) {
          const int j = lv.even[ei], a = lv.eleft[ei], c = lv.eright[ei];
          if (a >= 0) {
            float* P = PQf + (size_t)lv.pslot[ei] * blk;
            g1.push_back({aslot(ei, 0), bslot(opos[a], 0), P, 1.f, 0});
            pk2.push_back({P, aslot(ei, 0), 0});
            g2.push_back({aslot(ei, 0), bslot(opos[a], 2), Df + (size_t)j * blk, -1.f, 1});
            g2.push_back({aslot(ei, 0), bslot(opos[a], 1), Lf + (size_t)j * blk, -1.f, 0});
          }
          if (c >= 0) {
            float* Q = PQf + (size_t)lv.qslot[ei] * blk;
            g1.push_back({aslot(ei, 1), bslot(opos[c], 0), Q, 1.f, 0});
            pk2.push_back({Q, aslot(ei, 1), 0});
            g2.push_back({aslot(ei, 1), bslot(opos[c], 1), Df + (size_t)j * blk, -1.f, 1});
            if (lv.oright[opos[c]] >= 0)
              g2.push_back({aslot(ei, 1), bslot(opos[c], 2), Uf + (size_t)j * blk, -1.f, 0});
          }
        }
        GemmTask *d_g1 = nullptr, *d_g2 = nullptr;
        PackTask* d_pk2 = nullptr;
        if ((e = upload(sc, g1, &d_g1, st)) != cudaSuccess) return e;
        if ((e = upload(sc, pk2, &d_pk2, st)) != cudaSuccess) return e;
        if ((e = upload(sc, g2, &d_g2, st)) != cudaSuccess) return e;
        launch_gemm_tc(d_g1, (int)g1.size(), nT, three, env.d_st, st);
        launch_pack_split(d_pk2, (int)pk2.size(), nT, st);
        launch_gemm_tc(d_g2, (int)g2.size(), nT, three, env.d_st, st);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        continue;
      }
    }
    // FMA products on the plain blocks; the two updates of D_j go to separate launches
    std::vector<GemmTaskT<T>> g1, g2, g3;
    for (int ei = 0; ei < ne; ++ei) {
      const int j = lv.even[ei], a = lv.eleft[ei], c = lv.eright[ei];
      if (a >= 0) {
        T* P = PQ + (size_t)lv.pslot[ei] * blk;
        g1.push_back({blkp(L, j), blkp(D, a), P, T(1), 0});
        g2.push_back({P, blkp(U, a), blkp(D, j), T(-1), 1});
        g2.push_back({P, blkp(L, a), blkp(L, j), T(-1), 0});
      }
      if (c >= 0) {
        T* Q = PQ + (size_t)lv.qslot[ei] * blk;
        g1.push_back({blkp(U, j), blkp(D, c), Q, T(1), 0});
        g3.push_back({Q, blkp(L, c), blkp(D, j), T(-1), 1});
        if (lv.oright[opos[c]] >= 0) g2.push_back({Q, blkp(U, c), blkp(U, j), T(-1), 0});
      }
    }
    GemmTaskT<T> *d_g1 = nullptr, *d_g2 = nullptr, *d_g3 = nullptr;
    if ((e = upload(sc, g1, &d_g1, st)) != cudaSuccess) return e;
    if ((e = upload(sc, g2, &d_g2, st)) != cudaSuccess) return e;
    if ((e = upload(sc, g3, &d_g3, st)) != cudaSuccess) return e;
    launch_gemm_fma<T>(d_g1, (int)g1.size(), nT, st);
    launch_gemm_fma<T>(d_g2, (int)g2.size(), nT, st);
    launch_gemm_fma<T>(d_g3, (int)g3.size(), nT, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = invert(std::vector<int>{B.last})) != cudaSuccess) return e;
  // the scratch is released when this returns: finish the work that reads it first
  return cudaStreamSynchronize(st);
}

template <typename T>
static cudaError_t bcr_build_tasks(BcrSystem& B, double* x, double* tmp, const BcrEnv& env) {
  const int64_t ng = B.ng;
  const size_t blk = (size_t)B.NG * B.NG;
  const T* D = (const T*)B.D;
  const T* L = (const T*)B.L;
  const T* U = (const T*)B.U;
  const T* PQ = (const T*)B.PQ;
  auto X = [&](int j) { return x + (int64_t)j * ng; };
  auto Tm = [&](int j) { return tmp + (int64_t)j * ng; };
  auto Db = [&](int j) { return D + (size_t)j * blk; };
  auto Lb = [&](int j) { return L + (size_t)j * blk; };
  auto Ub = [&](int j) { return U + (size_t)j * blk; };
  auto Pb = [&](int slot) { return slot >= 0 ? PQ + (size_t)slot * blk : nullptr; };
  std::vector<BlockMv<T>> tasks;
  for (int dir = 0; dir < 2; ++dir) {
    B.runs[dir].clear();
    B.run_trans[dir].clear();
  }
  auto run = [&](int dir, int trans, std::vector<BlockMv<T>> ts) {
    if (ts.empty()) return;
    B.runs[dir].push_back({(int)tasks.size(), (int)ts.size()});
    B.run_trans[dir].push_back(trans);
    tasks.insert(tasks.end(), ts.begin(), ts.end());
  };
  auto mv = [](double* y, const double* x0, double coef, const T* M0, const double* v0,
               const T* M1, const double* v1) {
    BlockMv<T> t{};
    t.y = y; t.x0 = x0; t.coef = coef;
    t.M[0] = M0; t.v[0] = v0; t.M[1] = M1; t.v[1] = v1;
    return t;
  };
  const int nl = (int)B.levels.size();
  // (I - K)^{-1}
  for (const BcrLevel& lv : B.levels) {
    std::vector<BlockMv<T>> ts;
    for (size_t ei = 0; ei < lv.even.size(); ++ei) {
      const int j = lv.even[ei], a = lv.eleft[ei], c = lv.eright[ei];
      ts.push_back(mv(X(j), X(j), -1.0, Pb(lv.pslot[ei]), a >= 0 ? X(a) : nullptr,
                      Pb(lv.qslot[ei]), c >= 0 ? X(c) : nullptr));
    }
    run(0, 0, ts);
  }
  run(0, 0, {mv(Tm(B.last), X(B.last), 0.0, nullptr, nullptr, nullptr, nullptr)});
  run(0, 0, {mv(X(B.last), nullptr, 1.0, Db(B.last), Tm(B.last), nullptr, nullptr)});
  for (int l = nl - 1; l >= 0; --l) {
    const BcrLevel& lv = B.levels[l];
    std::vector<BlockMv<T>> ts1, ts2;
    for (size_t o = 0; o < lv.odd.size(); ++o) {
      const int i = lv.odd[o], a = lv.oleft[o], c = lv.oright[o];
      ts1.push_back(mv(Tm(i), X(i), -1.0, Lb(i), X(a), c >= 0 ? Ub(i) : nullptr,
                       c >= 0 ? X(c) : nullptr));
      ts2.push_back(mv(X(i), nullptr, 1.0, Db(i), Tm(i), nullptr, nullptr));
    }
    run(0, 0, ts1);
    run(0, 0, ts2);
  }
  // (I - K)^{-T}
  for (const BcrLevel& lv : B.levels) {
    std::vector<BlockMv<T>> ts1, ts2;
    for (size_t o = 0; o < lv.odd.size(); ++o) {
      const int i = lv.odd[o];
      ts1.push_back(mv(Tm(i), nullptr, 1.0, Db(i), X(i), nullptr, nullptr));  // z_i
    }
    for (size_t ei = 0; ei < lv.even.size(); ++ei) {
      const int j = lv.even[ei], a = lv.eleft[ei], c = lv.eright[ei];
      // s_j -= L_c^T z_c + U_a^T z_a
      ts2.push_back(mv(X(j), X(j), -1.0, c >= 0 ? Lb(c) : nullptr, c >= 0 ? Tm(c) : nullptr,
                       a >= 0 ? Ub(a) : nullptr, a >= 0 ? Tm(a) : nullptr));
    }
    run(1, 1, ts1);
    run(1, 1, ts2);
  }
  run(1, 0, {mv(Tm(B.last), X(B.last), 0.0, nullptr, nullptr, nullptr, nullptr)});
  run(1, 1, {mv(X(B.last), nullptr, 1.0, Db(B.last), Tm(B.last), nullptr, nullptr)});
  for (int l = nl - 1; l >= 0; --l) {
    const BcrLevel& lv = B.levels[l];
    // even block -> its P / Q slot at this level
    std::vector<BlockMv<T>> ts;
    for (size_t o = 0; o < lv.odd.size(); ++o) {
      const int i = lv.odd[o], el = lv.oleft[o], er = lv.oright[o];
      // P of the even block right of i (its left odd is i), Q of the even block left of i
      const T* Pr = nullptr;
      const T* Ql = nullptr;
      for (size_t ei = 0; ei < lv.even.size(); ++ei) {
        if (lv.even[ei] == er) Pr = Pb(lv.pslot[ei]);
        if (lv.even[ei] == el) Ql = Pb(lv.qslot[ei]);
      }
      ts.push_back(mv(X(i), Tm(i), -1.0, Pr, er >= 0 ? X(er) : nullptr, Ql, X(el)));
    }
    run(1, 1, ts);
  }
  if (B.d_tasks) env.release(B.d_tasks);
  cudaError_t e = env.alloc(&B.d_tasks, sizeof(BlockMv<T>) * tasks.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(B.d_tasks, tasks.data(), sizeof(BlockMv<T>) * tasks.size(),
                      cudaMemcpyHostToDevice, env.st);
  if (e != cudaSuccess) return e;
  B.tasks_x = x;
  return cudaStreamSynchronize(env.st);  // tasks is a host temporary
}

template <typename T>
cudaError_t bcr_solve(BcrSystem& B, double* x, double* tmp, int transpose, const BcrEnv& env) {
  if (B.tasks_x != x || !B.d_tasks) {
    const cudaError_t e = bcr_build_tasks<T>(B, x, tmp, env);
    if (e != cudaSuccess) return e;
  }
  const int dir = transpose ? 1 : 0;
  const BlockMv<T>* t = (const BlockMv<T>*)B.d_tasks;
  for (size_t r = 0; r < B.runs[dir].size(); ++r)
    launch_block_mv<T>(t + B.runs[dir][r].first, B.runs[dir][r].second, (int)B.ng, B.NG,
                       B.run_trans[dir][r], env.st);
  return cudaGetLastError();
}

void bcr_free(BcrSystem& B, const BcrEnv& env) {
  env.release(B.D);
  env.release(B.L);
  env.release(B.U);
  env.release(B.PQ);
  env.release(B.d_tasks);
  B.tasks_x = nullptr;
  B.levels.clear();
}

template cudaError_t bcr_factor<float>(BcrSystem&, const float*, const std::vector<int64_t>&,
                                       const std::vector<int64_t>&, int, int64_t, const BcrEnv&);
template cudaError_t bcr_factor<double>(BcrSystem&, const double*, const std::vector<int64_t>&,
                                        const std::vector<int64_t>&, int, int64_t, const BcrEnv&);
template cudaError_t bcr_solve<float>(BcrSystem&, double*, double*, int, const BcrEnv&);
template cudaError_t bcr_solve<double>(BcrSystem&, double*, double*, int, const BcrEnv&);
template void launch_block_mv<float>(const BlockMv<float>*, int, int, int, int, cudaStream_t);
template void launch_block_mv<double>(const BlockMv<double>*, int, int, int, int, cudaStream_t);

}  // namespace ddst
