// sweep_tc.cu -- explicit transfer operators on the tensor cores (tcgen05, 3xTF32).
//
// Same recurrences as sweep.cu (Sec. 2.2, Eq. (defS); Alg. 1 with the identity as test matrix):
//     Y_{k0} = G_{k0}^T e_C,  Y_{i-1} = -F_{i-1}^T diag(ell_i) Y_i (up),
//     Y_{i+1} = -B_{i+1}^T diag(ups_i) Y_i (down),
// for 256 sources of one slab and one direction at once.  The factor kernel stores the coupling
// folded into a tensor-core copy of every inverse, Ft_{i-1} = -diag(ell_i) F_{i-1} (up) and
// Bt_{i+1} = -diag(ups_i) B_{i+1} (down), already transposed into the K-major operand layout and
// split into TF32 hi/lo parts.  A sweep step is then the plain product
//     Y_next^T (128 x MB) = Y^T (128 x MB) * Ft   per tile of 128 sources,
// with the sources as the MMA's M dimension and the block rows as N (and K).
//
// Tensor memory per tile: two accumulators D0/D1 (MB columns each) and a lo column block.  The
// epilogue of step s reads Y^T from D[s % 2] (or the G row of a source injected at this block),
// stores the two S entries the block contributes, and splits Y^T in place into TF32 parts:
// hi = rna(y) back into D[s % 2], lo = rna(y - hi) into the lo block.  The MMAs of step s read
// A_hi from D[s % 2] and A_lo from the lo block and write D[(s + 1) % 2]:
//     D_next = A_hi B_hi + A_hi B_lo + A_lo B_hi   (3xTF32, Ootomo & Yokota 2022),
// or D_next = A_hi B_hi alone in the TF32 mode (its lo copies are then not loaded).
//
// A CTA holds two tiles that visit the same blocks in lockstep, so one factor stream feeds both,
// and the tensor core works on one tile while the other tile's epilogue runs.  Roles:
//   warps 0-3 / 4-7 : epilogue of tile 0 / 1 (thread = TMEM lane = source column);
//   warp 8          : bulk-copy producer (Ft hi/lo, stencil pack, G rows of injected sources);
//   warp 9          : TMEM allocation and MMA issue.
// Barriers: full[st] (copy landed), empty[st] (MMAs and epilogues done with the stage),
// dready[u] (tile u's accumulator complete), aready[u] (tile u's A operand stored).  Every wait is
// bounded and also gives up once another role has raised the CTA's abort flag.
//
// Shared-memory operand layout (canonical K-major, no swizzle): core matrices of 8 rows x 16 B,
// core matrix (row group g, k group kk) at byte g * (K * 32) + kk * 128; LBO (K direction) =
// 128 B, SBO (row direction) = 32 K B.  The MMA for K slice s (8 elements) starts at + s * 256 B.
#include "kernels.cuh"
#include "umma.cuh"

namespace ddst {

template <int MB>
struct TcCfg {
  static constexpr int TILE = 128;                            // sources per tile (MMA M)
  static constexpr int NT = 2;                                // tiles per CTA
  static constexpr int NST = 4;                               // ring stages
  static constexpr uint32_t FBLK = MB * MB * 4;               // one factor part (hi or lo)
  static constexpr uint32_t PKB = PK_NFIELDS * MB * 4;        // stencil pack of one block
  static constexpr uint32_t GSLOT = 4096;                     // p G rows of the injected sources
  static constexpr uint32_t STAGE = 2 * FBLK + PKB + GSLOT;
  static constexpr int THREADS = NT * TILE + 64;
  static constexpr int TCOLS = NT * 3 * MB <= 256 ? 256 : 512;
  static constexpr size_t RING = (size_t)NST * STAGE;
  static constexpr size_t BARS = 8 * (2 * NST + 2 * NT + 1);
  // at most 512 / TCOLS CTAs may share an SM's tensor memory: pad shared memory to enforce it
  static constexpr size_t MIN_SMEM = TCOLS == 512 ? 120 * 1024 : 80 * 1024;
  static constexpr size_t SMEM = RING + BARS > MIN_SMEM ? RING + BARS : MIN_SMEM;
};

template <int MB>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[MB]) {
  if constexpr (MB == 32) tmem_ld32_wait(taddr, r);
  else tmem_ld64_wait(taddr, r);
}

template <int MB>
__global__ void __launch_bounds__(TcCfg<MB>::THREADS, 1)
    k_sbuild_tc(const SlabDesc* __restrict__ slabs, const TileDesc* __restrict__ tiles,
                const float* __restrict__ Fhi, const float* __restrict__ Flo,
                const float* __restrict__ Bhi, const float* __restrict__ Blo,
                const float* __restrict__ G, const float* __restrict__ pack,
                float* __restrict__ S, DevStatus* st, long long budget, int three) {
  using C = TcCfg<MB>;
  constexpr int NST = C::NST, NT = C::NT;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* ring = smem_raw;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + C::RING);
  uint64_t* empty = full + NST;
  uint64_t* dready = empty + NST;
  uint64_t* aready = dready + NT;
  uint64_t* done = aready + NT;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  volatile int* abort = &s_abort;

  const TileDesc td = tiles[blockIdx.x];
  const SlabDesc s = slabs[td.slab];
  const bool up = td.dir == 0;
  const int len = td.len;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nlive = (td.nq + C::TILE - 1) / C::TILE;           // 1 or 2 tiles with sources
  const bool g_in_ring = (uint32_t)s.p * MB * 4 <= C::GSLOT;
  auto blk = [&](int stp) { return up ? td.kstart - stp : td.kstart + stp; };

  if (warp == 9) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"((uint32_t)C::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    s_abort = 0;
    for (int b = 0; b < NST; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], 1 + 4 * nlive);
    }
    for (int u = 0; u < NT; ++u) {
      mbar_init(&dready[u], 1);
      mbar_init(&aready[u], 4);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 8) {
    // ------------------------------------------------------------------ producer
    if (lane == 0) {
      const float* Fh = (up ? Fhi : Bhi) + s.fac_off;
      const float* Fl = (up ? Flo : Blo) + s.fac_off;
      int issued = 0;
      for (int stp = 0; stp < len; ++stp) {
        const int stage = stp % NST;
        if (stp >= NST && !mbar_wait_ab(&empty[stage], ((stp / NST) - 1) & 1, abort, st, td.slab, blk(stp), budget))
          break;
        const int i = blk(stp);
        const bool has_f = stp < len - 1;
        // sources of this CTA injected at block i: q in [(i-1) p, i p) and [q0, q0 + nq)
        const int64_t qa = (int64_t)(i - 1) * s.p, qb = qa + s.p;
        const bool has_g = g_in_ring && qa < td.q0 + td.nq && qb > td.q0;
        const uint32_t gbytes = (uint32_t)s.p * MB * 4;
        unsigned char* sb = ring + stage * C::STAGE;
        // 1xTF32 (three == 0) reads only the hi part of the factor copy
        mbar_arrive_expect_tx(&full[stage], C::PKB + (has_f ? (three ? 2 : 1) * C::FBLK : 0u) +
                                                (has_g ? gbytes : 0u));
        bulk_g2s(sb + 2 * C::FBLK, pack + s.pack_off + (int64_t)(i - 1) * PK_NFIELDS * MB, C::PKB,
                 &full[stage]);
        if (has_f) {
          const int fidx = up ? i - 2 : i;
          bulk_g2s(sb, Fh + (int64_t)fidx * MB * MB, C::FBLK, &full[stage]);
          if (three) bulk_g2s(sb + C::FBLK, Fl + (int64_t)fidx * MB * MB, C::FBLK, &full[stage]);
        }
        if (has_g)
          bulk_g2s(sb + 2 * C::FBLK + C::PKB,
                   G + s.fac_off + (int64_t)(i - 1) * MB * MB + (int64_t)(s.w - 1) * s.p * MB,
                   gbytes, &full[stage]);
        ++issued;
      }
      // no copy may still target this CTA's shared memory when it exits
      for (int stp = issued > NST ? issued - NST : 0; stp < issued; ++stp)
        mbar_wait(&full[stp % NST], (stp / NST) & 1, st, td.slab, -1);
    }
  } else if (warp == 9) {
    // ------------------------------------------------------------------ MMA issue
    if (lane == 0) {
      constexpr uint32_t IDESC = idesc_tf32(C::TILE, MB);
      for (int stp = 0; stp < len - 1; ++stp) {
        const int stage = stp % NST;
        const int i = blk(stp);
        if (!mbar_wait_ab(&full[stage], (stp / NST) & 1, abort, st, td.slab, i, budget)) break;
        const unsigned char* fb = ring + stage * C::STAGE;
        const uint32_t b_hi = smem_u32(fb), b_lo = smem_u32(fb + C::FBLK);
        bool ok = true;
        for (int u = 0; u < nlive; ++u) {
          if (!mbar_wait_ab(&aready[u], stp & 1, abort, st, td.slab, i, budget)) { ok = false; break; }
          tc_fence_after();
          const uint32_t base = tmem + (uint32_t)(u * 3 * MB);
          const uint32_t a_hi = base + (uint32_t)((stp & 1) * MB);
          const uint32_t d = base + (uint32_t)(((stp + 1) & 1) * MB);
          const uint32_t a_lo = base + 2 * MB;
#pragma unroll
          for (int ks = 0; ks < MB / 8; ++ks) {
            const uint64_t dbh = umma_desc(b_hi + ks * 256, 128, MB * 32);
            const uint64_t dbl = umma_desc(b_lo + ks * 256, 128, MB * 32);
            mma_tf32_tmem_a(d, a_hi + ks * 8, dbh, IDESC, ks > 0 ? 1u : 0u);
            if (three) {
              mma_tf32_tmem_a(d, a_hi + ks * 8, dbl, IDESC, 1u);
              mma_tf32_tmem_a(d, a_lo + ks * 8, dbh, IDESC, 1u);
            }
          }
          mma_commit(&dready[u]);
        }
        if (!ok) break;
        mma_commit(&empty[stage]);
      }
      // every MMA issued has completed before the accumulators are released
      mma_commit(done);
      mbar_wait(done, 0, st, td.slab, -1);
    }
  } else if (warp / 4 < nlive) {
    // ------------------------------------------------------------------ epilogue of tile u
    const int u = warp / 4;
    const int lt = tid - u * C::TILE;
    const uint32_t base = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(u * 3 * MB);
    const bool act = lt < td.nq - u * C::TILE;
    const int q = td.q0 + u * C::TILE + lt;
    const int k0 = q / s.p + 1, t0 = q - (k0 - 1) * s.p;
    const int64_t ng = s.ng;
    const int eastlo = (2 * s.w - 2) * s.p;
    for (int stp = 0; stp < len; ++stp) {
      const int stage = stp % NST;
      const int i = blk(stp);
      if (!mbar_wait_ab(&full[stage], (stp / NST) & 1, abort, st, td.slab, i, budget)) break;
      if (stp > 0) {
        if (!mbar_wait_ab(&dready[u], (stp - 1) & 1, abort, st, td.slab, i, budget)) break;
        tc_fence_after();
      }
      const uint32_t dcur = base + (uint32_t)((stp & 1) * MB);
      const unsigned char* sb = ring + stage * C::STAGE;
      const float* pk = reinterpret_cast<const float*>(sb + 2 * C::FBLK);
      const bool inj = act && k0 == i;  // Y_i = G_i^T e_{C_t0}: row (w-1)p + t0 of G_i
      const float* grow = !inj ? nullptr
                          : g_in_ring
                              ? reinterpret_cast<const float*>(sb + 2 * C::FBLK + C::PKB) + t0 * MB
                              : G + s.fac_off + (int64_t)(i - 1) * MB * MB +
                                    (int64_t)((s.w - 1) * s.p + t0) * MB;
      // the two S entries of block i for the sources this direction owns, from Y_i in FP32
      // (the accumulator D[s % 2] before it is split, or the injected G row)
      const bool own = act && (up ? (k0 >= i) : (k0 < i));
      if (__any_sync(0xffffffffu, own)) {
        for (int t = 0; t < s.p; ++t) {
          uint32_t rw = 0u, re = 0u;
          if (stp > 0) tmem_ld1x2_wait(dcur + (uint32_t)t, dcur + (uint32_t)(eastlo + t), rw, re);
          float yw = __uint_as_float(rw), ye = __uint_as_float(re);
          if (inj) {
            yw = grow[t];
            ye = grow[eastlo + t];
          }
          if (own) {
            if (s.sp_off >= 0)
              S[s.sp_off + ((int64_t)(i - 1) * s.p + t) * ng + q] = -pk[PK_WEST * MB + t] * yw;
            if (s.sn_off >= 0)
              S[s.sn_off + ((int64_t)(i - 1) * s.p + t) * ng + q] = -pk[PK_EAST * MB + eastlo + t] * ye;
          }
        }
      }
      if (stp < len - 1) {
        // A operand of this step: Y_i^T split into TF32 hi (into D[s % 2]) and lo parts
        uint32_t v[MB];
        if (stp > 0) {
          tmem_ld_cols<MB>(dcur, v);
        } else {
#pragma unroll
          for (int c = 0; c < MB; ++c) v[c] = 0u;  // nothing injected yet: Y = 0
        }
        if (inj) {
#pragma unroll
          for (int c = 0; c < MB; ++c) v[c] = __float_as_uint(grow[c]);
        }
#pragma unroll
        for (int c16 = 0; c16 < MB; c16 += 16) {
          uint32_t hi[16], lo[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) tf32_split(v[c16 + e], hi[e], lo[e]);
          tmem_st16(dcur + (uint32_t)c16, hi);
          tmem_st16(base + (uint32_t)(2 * MB + c16), lo);
        }
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive1(&aready[u]);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive1(&empty[stage]);  // pack and G rows of this stage consumed
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 9)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)C::TCOLS)
                 : "memory");
}

template <int MB>
static void run_tc(const SlabDesc* d_slabs, const TileDesc* d_tiles, int ntiles,
                   const float* Fhi, const float* Flo, const float* Bhi, const float* Blo,
                   const float* G, const float* pack, float* S, DevStatus* st, long long budget,
                   int three, cudaStream_t s) {
  using C = TcCfg<MB>;
  raise_smem_limit(reinterpret_cast<const void*>(&k_sbuild_tc<MB>), C::SMEM);
  note_launch();
  k_sbuild_tc<MB><<<ntiles, C::THREADS, C::SMEM, s>>>(d_slabs, d_tiles, Fhi, Flo, Bhi, Blo, G,
                                                      pack, S, st, budget, three);
}

void launch_sbuild_tc(int M, const SlabDesc* d_slabs, const TileDesc* d_tiles, int ntiles,
                      const float* Fhi, const float* Flo, const float* Bhi, const float* Blo,
                      const float* G, const float* pack, float* S, DevStatus* st,
                      long long budget, int three, cudaStream_t s) {
  if (ntiles == 0) return;
  switch (M) {
    case 32: run_tc<32>(d_slabs, d_tiles, ntiles, Fhi, Flo, Bhi, Blo, G, pack, S, st, budget, three, s); break;
    case 64: run_tc<64>(d_slabs, d_tiles, ntiles, Fhi, Flo, Bhi, Blo, G, pack, S, st, budget, three, s); break;
    default: break;
  }
}

int sbuild_tc_tile_cols() { return TcCfg<64>::NT * TcCfg<64>::TILE; }

}  // namespace ddst
