// sweep.cu -- explicit formation of the solution-transfer operators S_{j,j-1}, S_{j,j+1}.
//
// Sec. 2.2, Eq. (defS) / Sec. 2.5:  S_{j,j'} = -R_{C_j} A_j(I_j,I_j)^{-1} A_j(I_j, J_{j,j'}).
// A_j(I_j, J_{j,j-1}) has one nonzero per boundary point: the west coupling beta of the
// adjacent unknown (cx = 0); likewise gamma (east, cx = 2w-2) for J_{j,j+1}.  Hence
//     S_{j,j-1}[q, (i,t)] = -beta_{i,t}  Y^(q)_i[W_t],   S_{j,j+1}[q, (i,t)] = -gamma_{i,t} Y^(q)_i[E_t],
// where Y^(q) = A_j^{-T} e_{C(q)} is the transposed solve with a unit source at central point q.
// One transposed solve per central point therefore yields a full row of both operators (Alg. 1
// with the identity as test matrix applied from the left).
//
// The columns Y^(q) of A_j^{-T} are generated from the two-sided factorization (factor.cu):
//     Y_{k0} = G_{k0}^T e_C,
//     Y_{i-1} = -F_{i-1}^T diag(ell_i) Y_i      (i <= k0, upward sweep)
//     Y_{i+1} = -B_{i+1}^T diag(ups_i) Y_i      (i >= k0, downward sweep)
// A CTA owns R consecutive sources q of one slab and one direction; each step is one
// (M x M) x (M x R) product.  The factor block of the next steps streams in through a ring of
// bulk (TMA) copies completing on mbarriers; the panel lives in shared memory.
// Storage of S: column-major n_Gamma x n_Gamma (element (q, src) at src * n_Gamma + q).
#include "kernels.cuh"

namespace ddst {

template <typename T, int N>
__device__ __forceinline__ void lds(T (&d)[N], const T* __restrict__ s) {
  if constexpr ((N * sizeof(T)) % 16 == 0) {
    const uint4* v = reinterpret_cast<const uint4*>(s);
#pragma unroll
    for (int q = 0; q < (int)(N * sizeof(T) / 16); ++q) {
      uint4 u = v[q];
      T tmp[16 / sizeof(T)];
      memcpy(tmp, &u, 16);
#pragma unroll
      for (int e = 0; e < (int)(16 / sizeof(T)); ++e) d[q * (16 / sizeof(T)) + e] = tmp[e];
    }
  } else {
#pragma unroll
    for (int e = 0; e < N; ++e) d[e] = s[e];
  }
}

template <typename T, int N>
__device__ __forceinline__ void sts(T* __restrict__ s, const T (&d)[N]) {
  if constexpr ((N * sizeof(T)) % 16 == 0) {
    uint4* v = reinterpret_cast<uint4*>(s);
#pragma unroll
    for (int q = 0; q < (int)(N * sizeof(T) / 16); ++q) {
      T tmp[16 / sizeof(T)];
#pragma unroll
      for (int e = 0; e < (int)(16 / sizeof(T)); ++e) tmp[e] = d[q * (16 / sizeof(T)) + e];
      uint4 u;
      memcpy(&u, tmp, 16);
      v[q] = u;
    }
  } else {
#pragma unroll
    for (int e = 0; e < N; ++e) s[e] = d[e];
  }
}

template <typename T, int M, int R, int NST>
struct SweepCfg {
  static constexpr int THREADS = 128;
  static constexpr int RPT = M / 4;     // rows per thread (one warp per quarter of rows)
  static constexpr int CPT = R / 32;    // columns per lane
  static constexpr size_t SMEM =
      (size_t)NST * (M * M + PK_NFIELDS * M) * sizeof(T) + 2ull * M * R * sizeof(T) + NST * 8;
};

template <typename T, int M, int R, int NST>
__global__ void __launch_bounds__(128) k_sbuild(const SlabDesc* __restrict__ slabs,
                                                const TileDesc* __restrict__ tiles,
                                                const T* __restrict__ F, const T* __restrict__ B,
                                                const T* __restrict__ G,
                                                const T* __restrict__ pack, T* __restrict__ S,
                                                DevStatus* st) {
  using C = SweepCfg<T, M, R, NST>;
  constexpr int RPT = C::RPT, CPT = C::CPT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* sF = reinterpret_cast<T*>(smem_raw);
  T* sPk = sF + NST * M * M;
  T* sP = sPk + NST * PK_NFIELDS * M;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sP + 2 * M * R);
  __shared__ int s_abort;

  const TileDesc td = tiles[blockIdx.x];
  const SlabDesc s = slabs[td.slab];
  const bool up = td.dir == 0;
  const T* Fac = (up ? F : B) + s.fac_off;
  const int len = td.len;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = warp * RPT, c0 = lane * CPT;
  const int64_t ng = s.ng;
  const int eastlo = (2 * s.w - 2) * s.p;

  int k0[CPT], t0[CPT];
  bool act[CPT];
#pragma unroll
  for (int cc = 0; cc < CPT; ++cc) {
    const int col = c0 + cc;
    act[cc] = col < td.nq;
    const int q = td.q0 + col;
    k0[cc] = q / s.p + 1;
    t0[cc] = q - (k0[cc] - 1) * s.p;
  }

  int issued = 0;  // bulk-copy stages issued (thread 0 only)
  auto issue = [&](int stp) {
    ++issued;
    const int stage = stp % NST;
    const int i = up ? td.kstart - stp : td.kstart + stp;
    const bool has_f = up ? (i >= 2) : (i <= s.nb - 1);
    const uint32_t bpk = PK_NFIELDS * M * sizeof(T);
    const uint32_t bf = M * M * sizeof(T);
    mbar_arrive_expect_tx(&bar[stage], bpk + (has_f ? bf : 0u));
    bulk_g2s(sPk + stage * PK_NFIELDS * M, pack + s.pack_off + (int64_t)(i - 1) * PK_NFIELDS * M,
             bpk, &bar[stage]);
    if (has_f) {
      const int fidx = up ? i - 2 : i;  // F_{i-1} or B_{i+1} (0-based block index)
      bulk_g2s(sF + stage * M * M, Fac + (int64_t)fidx * M * M, bf, &bar[stage]);
    }
  };

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int q = 0; q < NST; ++q) mbar_init(&bar[q], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 0; q < NST && q < len; ++q) issue(q);

  T acc[RPT][CPT];
#pragma unroll
  for (int rr = 0; rr < RPT; ++rr)
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) acc[rr][cc] = T(0);

  int consumed = 0;  // number of stages waited for
  for (int step = 0; step < len; ++step) {
    const int i = up ? td.kstart - step : td.kstart + step;
    const int stage = step % NST;
    // inject the sources whose central point lies in block i: Y_i = G_i^T e_{C_t0}
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
      if (act[cc] && k0[cc] == i) {
        const T* grow = G + s.fac_off + (int64_t)(i - 1) * M * M + (int64_t)((s.w - 1) * s.p + t0[cc]) * M;
#pragma unroll
        for (int rr = 0; rr < RPT; ++rr) acc[rr][cc] = grow[r0 + rr];
      }
    }
    if (!mbar_wait(&bar[stage], (step / NST) & 1, st, td.slab, i)) s_abort = 1;
    consumed = step + 1;
    const T* pk = sPk + stage * PK_NFIELDS * M;
    // outputs of block i: rows W_t (cx = 0) and E_t (cx = 2w-2)
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const int r = r0 + rr;
      if (r < s.p && s.sp_off >= 0) {
        const T coef = -pk[PK_WEST * M + r];
        T* dst = S + s.sp_off + ((int64_t)(i - 1) * s.p + r) * ng + td.q0;
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc)
          if (act[cc] && (up ? (k0[cc] >= i) : (k0[cc] < i))) dst[c0 + cc] = coef * acc[rr][cc];
      }
      if (r >= eastlo && r < s.m && s.sn_off >= 0) {
        const T coef = -pk[PK_EAST * M + r];
        T* dst = S + s.sn_off + ((int64_t)(i - 1) * s.p + (r - eastlo)) * ng + td.q0;
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc)
          if (act[cc] && (up ? (k0[cc] >= i) : (k0[cc] < i))) dst[c0 + cc] = coef * acc[rr][cc];
      }
    }
    if (step == len - 1) break;
    // scaled panel -diag(ell_i) Y_i (up) or -diag(ups_i) Y_i (down) into shared memory
    T* buf = sP + (step & 1) * M * R;
    const int rf = up ? PK_SOUTH : PK_NORTH;
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr) {
      const T sc = -pk[rf * M + r0 + rr];
      T v[CPT];
#pragma unroll
      for (int cc = 0; cc < CPT; ++cc) v[cc] = sc * acc[rr][cc];
      sts<T, CPT>(buf + (r0 + rr) * R + c0, v);
    }
    __syncthreads();
    if (s_abort) break;
    if (threadIdx.x == 0 && step >= 1 && step - 1 + NST < len) {
      fence_proxy_async();
      issue(step - 1 + NST);
    }
    // Y_{next} = A * panel with A[r][c] = F[c][r]
    const T* A = sF + stage * M * M;
#pragma unroll
    for (int rr = 0; rr < RPT; ++rr)
#pragma unroll
      for (int cc = 0; cc < CPT; ++cc) acc[rr][cc] = T(0);
#pragma unroll 4
    for (int c = 0; c < M; ++c) {
      T a[RPT], b[CPT];
      lds<T, RPT>(a, A + c * M + r0);
      lds<T, CPT>(b, buf + c * R + c0);
#pragma unroll
      for (int rr = 0; rr < RPT; ++rr)
#pragma unroll
        for (int cc = 0; cc < CPT; ++cc) acc[rr][cc] = fma(a[rr], b[cc], acc[rr][cc]);
    }
  }
  // Never leave with a bulk copy in flight into this CTA's shared memory (bounded wait).
  if (threadIdx.x == 0)
    for (int q = consumed; q < issued; ++q) mbar_wait(&bar[q % NST], (q / NST) & 1, st, td.slab, -1);
}

template <typename T, int M, int R, int NST>
static void run_sbuild(const SlabDesc* d_slabs, const TileDesc* d_tiles, int ntiles, const T* F,
                       const T* B, const T* G, const T* pack, T* S, DevStatus* st,
                       cudaStream_t s) {
  using C = SweepCfg<T, M, R, NST>;
  raise_smem_limit(reinterpret_cast<const void*>(&k_sbuild<T, M, R, NST>), C::SMEM);
  note_launch();
  k_sbuild<T, M, R, NST><<<ntiles, C::THREADS, C::SMEM, s>>>(d_slabs, d_tiles, F, B, G, pack, S, st);
}

template <typename T>
int sbuild_tile_cols(int M) {
  if (sizeof(T) == 4) return M == 128 ? 64 : 128;
  return M == 128 ? 32 : 64;
}

template <>
void launch_sbuild<float>(int M, const SlabDesc* d_slabs, const TileDesc* d_tiles, int ntiles,
                          const float* F, const float* B, const float* G, const float* pack,
                          float* S, DevStatus* st, cudaStream_t s) {
  if (ntiles == 0) return;
  switch (M) {
    case 32: run_sbuild<float, 32, 128, 3>(d_slabs, d_tiles, ntiles, F, B, G, pack, S, st, s); break;
    case 64: run_sbuild<float, 64, 128, 2>(d_slabs, d_tiles, ntiles, F, B, G, pack, S, st, s); break;
    case 128: run_sbuild<float, 128, 64, 2>(d_slabs, d_tiles, ntiles, F, B, G, pack, S, st, s); break;
    default: break;
  }
}

template <>
void launch_sbuild<double>(int M, const SlabDesc* d_slabs, const TileDesc* d_tiles, int ntiles,
                           const double* F, const double* B, const double* G,
                           const double* pack, double* S, DevStatus* st, cudaStream_t s) {
  if (ntiles == 0) return;
  switch (M) {
    case 32: run_sbuild<double, 32, 64, 2>(d_slabs, d_tiles, ntiles, F, B, G, pack, S, st, s); break;
    case 64: run_sbuild<double, 64, 64, 2>(d_slabs, d_tiles, ntiles, F, B, G, pack, S, st, s); break;
    default: break;
  }
}

template int sbuild_tile_cols<float>(int);
template int sbuild_tile_cols<double>(int);

}  // namespace ddst
