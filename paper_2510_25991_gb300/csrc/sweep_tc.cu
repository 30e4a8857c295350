// sweep_tc.cu -- explicit transfer operators on the tensor cores (tcgen05, 3xTF32).
//
// Same recurrences as sweep.cu (Sec. 2.2, Eq. (defS); Alg. 1 with the identity as test matrix):
//     Y_{k0} = G_{k0}^T e_C,  Y_{i-1} = -F_{i-1}^T diag(ell_i) Y_i (up),
//     Y_{i+1} = -B_{i+1}^T diag(ups_i) Y_i (down),
// for a tile of R = 128 sources at once.  Each step is computed transposed,
//     Y_next^T (128 x MB) = P^T (128 x MB) * F (MB x MB),   P = -diag(ell_i) Y_i,
// so the 128 sources form the MMA's M dimension and the block rows its N dimension:
//   * A operand: the panel P^T in shared memory (K-major), rewritten every step by the epilogue;
//   * B operand: F^T (or B^T) of the step, stored by the factor kernel in the same K-major
//     layout and already split into TF32 hi/lo parts, streamed in by bulk copies;
//   * accumulator: 128 TMEM lanes x MB columns (FP32).  Thread t of the 4 warps owns TMEM lane t,
//     i.e. source column t: one tcgen05.ld returns its whole column for the epilogue.
// 3xTF32: A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi with x_hi = rna_tf32(x), x_lo = rna_tf32(x - x_hi)
// (split-operand emulation of FP32 products, Ootomo & Yokota 2022).
//
// Shared-memory operand layout (canonical K-major, no swizzle): core matrices of 8 rows x 16 B,
// core matrix (row group g, k group kk) at byte g * (K * 32) + kk * 128; LBO (K direction) =
// 128 B, SBO (row direction) = 32 K B.  The MMA for K slice s (8 elements) starts at + s * 256 B.
#include "kernels.cuh"
#include "umma.cuh"

namespace ddst {

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; no swizzle, base offset 0
  return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int MB>
struct TcCfg {
  static constexpr int R = 128;                               // sources per CTA (MMA M)
  static constexpr int NST = 3;                               // factor ring stages
  static constexpr uint32_t PANEL = R * MB * 4;               // bytes of one panel part
  static constexpr uint32_t FBLK = MB * MB * 4;               // bytes of one factor part
  static constexpr uint32_t PKB = PK_NFIELDS * MB * 4;        // bytes of one pack
  static constexpr uint32_t STAGE = 2 * FBLK + PKB;
  static constexpr size_t SMEM = 2 * (size_t)PANEL + NST * (size_t)STAGE + 8 * 2 * NST;
  static constexpr int TCOLS = MB < 32 ? 32 : MB;             // TMEM columns (power of two)
};

template <int MB>
__global__ void __launch_bounds__(128) k_sbuild_tc(const SlabDesc* __restrict__ slabs,
                                                   const TileDesc* __restrict__ tiles,
                                                   const float* __restrict__ Fhi,
                                                   const float* __restrict__ Flo,
                                                   const float* __restrict__ Bhi,
                                                   const float* __restrict__ Blo,
                                                   const float* __restrict__ G,
                                                   const float* __restrict__ pack,
                                                   float* __restrict__ S, DevStatus* st) {
  using C = TcCfg<MB>;
  constexpr int R = C::R, NST = C::NST;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* pan_hi = smem_raw;
  unsigned char* pan_lo = pan_hi + C::PANEL;
  unsigned char* stages = pan_lo + C::PANEL;
  uint64_t* bar = reinterpret_cast<uint64_t*>(stages + NST * C::STAGE);  // [NST] loads, [NST] mma
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;

  const TileDesc td = tiles[blockIdx.x];
  const SlabDesc s = slabs[td.slab];
  const bool up = td.dir == 0;
  const float* Fh = (up ? Fhi : Bhi) + s.fac_off;
  const float* Fl = (up ? Flo : Blo) + s.fac_off;
  const int len = td.len;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t ng = s.ng;
  const int eastlo = (2 * s.w - 2) * s.p;
  // this thread's source column
  const bool act = tid < td.nq;
  const int q = td.q0 + tid;
  const int k0 = q / s.p + 1, t0 = q - (k0 - 1) * s.p;
  uint64_t* mbar = bar + NST;

  int issued = 0;
  auto issue = [&](int stp) {
    ++issued;
    const int stage = stp % NST;
    const int i = up ? td.kstart - stp : td.kstart + stp;
    const bool has_f = up ? (i >= 2) : (i <= s.nb - 1);
    unsigned char* sb = stages + stage * C::STAGE;
    mbar_arrive_expect_tx(&bar[stage], C::PKB + (has_f ? 2 * C::FBLK : 0u));
    bulk_g2s(sb + 2 * C::FBLK, pack + s.pack_off + (int64_t)(i - 1) * PK_NFIELDS * MB, C::PKB,
             &bar[stage]);
    if (has_f) {
      const int fidx = up ? i - 2 : i;
      bulk_g2s(sb, Fh + (int64_t)fidx * MB * MB, C::FBLK, &bar[stage]);
      bulk_g2s(sb + C::FBLK, Fl + (int64_t)fidx * MB * MB, C::FBLK, &bar[stage]);
    }
  };

  if (warp == 0) {  // TMEM accumulator: 128 lanes x TCOLS FP32 columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"((uint32_t)C::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    s_abort = 0;
    for (int b = 0; b < 2 * NST; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  if (tid == 0)
    for (int stp = 0; stp < NST && stp < len; ++stp) issue(stp);

  float y[MB];
#pragma unroll
  for (int r = 0; r < MB; ++r) y[r] = 0.f;
  constexpr uint32_t IDESC = idesc_tf32(R, MB);
  int consumed = 0, mma_issued = 0, mma_waited = 0;
  for (int step = 0; step < len; ++step) {
    const int i = up ? td.kstart - step : td.kstart + step;
    const int stage = step % NST;
    if (act && k0 == i) {  // inject Y_i = G_i^T e_{C_t0} for this source
      const float* grow = G + s.fac_off + (int64_t)(i - 1) * MB * MB + (int64_t)((s.w - 1) * s.p + t0) * MB;
#pragma unroll
      for (int r = 0; r < MB; ++r) y[r] = grow[r];
    }
    if (!mbar_wait(&bar[stage], (step / NST) & 1, st, td.slab, i)) s_abort = 1;
    consumed = step + 1;
    const float* pk = reinterpret_cast<const float*>(stages + stage * C::STAGE + 2 * C::FBLK);
    // outputs of block i (rows W_t, E_t) for the sources this sweep direction owns
    if (act && (up ? (k0 >= i) : (k0 < i))) {
#pragma unroll
      for (int r = 0; r < MB; ++r) {
        if (r < s.p && s.sp_off >= 0)
          S[s.sp_off + ((int64_t)(i - 1) * s.p + r) * ng + q] = -pk[PK_WEST * MB + r] * y[r];
        if (r >= eastlo && r < s.m && s.sn_off >= 0)
          S[s.sn_off + ((int64_t)(i - 1) * s.p + (r - eastlo)) * ng + q] = -pk[PK_EAST * MB + r] * y[r];
      }
    }
    if (step == len - 1) break;
    // panel P^T (row = this source, K = block row): -diag(ell_i) Y_i (up) / -diag(ups_i) Y_i
    {
      const int rf = up ? PK_SOUTH : PK_NORTH;
#pragma unroll
      for (int r4 = 0; r4 < MB; r4 += 4) {
        float4 hi, lo;
        float* h = &hi.x;
        float* l = &lo.x;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float v = -pk[rf * MB + r4 + e] * y[r4 + e];
          h[e] = tf32_rna(v);
          l[e] = tf32_rna(v - h[e]);
        }
        const uint32_t off = umma_off(tid, r4, MB);
        *reinterpret_cast<float4*>(pan_hi + off) = hi;
        *reinterpret_cast<float4*>(pan_lo + off) = lo;
      }
    }
    fence_proxy_async();  // generic-proxy panel stores -> visible to the tensor core (async proxy)
    tc_fence_before();
    __syncthreads();
    if (s_abort) break;
    if (tid == 0) {
      tc_fence_after();
      const unsigned char* fb = stages + stage * C::STAGE;
      const uint32_t a_hi = smem_u32(pan_hi), a_lo = smem_u32(pan_lo);
      const uint32_t b_hi = smem_u32(fb), b_lo = smem_u32(fb + C::FBLK);
      const uint32_t sbo_a = MB * 32, sbo_b = MB * 32;
#pragma unroll
      for (int ks = 0; ks < MB / 8; ++ks) {
        const uint64_t dah = umma_desc(a_hi + ks * 256, 128, sbo_a);
        const uint64_t dal = umma_desc(a_lo + ks * 256, 128, sbo_a);
        const uint64_t dbh = umma_desc(b_hi + ks * 256, 128, sbo_b);
        const uint64_t dbl = umma_desc(b_lo + ks * 256, 128, sbo_b);
        mma_tf32(tmem, dah, dbh, IDESC, ks > 0 ? 1u : 0u);
        mma_tf32(tmem, dah, dbl, IDESC, 1u);
        mma_tf32(tmem, dal, dbh, IDESC, 1u);
      }
      mma_commit(&mbar[step & 1]);
    }
    ++mma_issued;
    // the ring stage of the previous step is free (its MMAs completed): prefetch 2 steps ahead
    if (tid == 0 && step >= 1 && step - 1 + NST < len) {
      fence_proxy_async();
      issue(step - 1 + NST);
    }
    if (mbar_wait(&mbar[step & 1], (step >> 1) & 1, st, td.slab, i))
      mma_waited = mma_issued;
    else
      s_abort = 1;  // every thread leaves together at the next barrier
    tc_fence_after();
    // Y_{next} column for this source: TMEM lane = tid (warp quadrant 32 * warp)
#pragma unroll
    for (int c16 = 0; c16 < MB; c16 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c16, v);
      tmem_wait_ld();
#pragma unroll
      for (int e = 0; e < 16; ++e) y[c16 + e] = v[e];
    }
    tc_fence_before();
  }
  // drain: no bulk copy or MMA may still target this CTA's shared memory / TMEM
  if (tid == 0) {
    for (int stp = consumed; stp < issued; ++stp)
      mbar_wait(&bar[stp % NST], (stp / NST) & 1, st, td.slab, -1);
    if (mma_waited < mma_issued)
      mbar_wait(&mbar[(mma_issued - 1) & 1], ((mma_issued - 1) >> 1) & 1, st, td.slab, -1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)C::TCOLS)
                 : "memory");
}

// ---------------------------------------------------------------------------------------------
// Two-tile ping-pong version: A operand in tensor memory, warp-specialised.
//
// A CTA takes 256 sources of one slab and one sweep direction as two 128-source tiles that visit
// the same blocks in lockstep, so one factor stream feeds both.  Per tile, TMEM holds the
// accumulator D (MB columns) and the panel P^T split into TF32 hi and lo parts (MB columns each);
// the MMA reads A from TMEM ([a_tmem] form) and B (F hi/lo) from the shared-memory ring.  While
// the tensor core works on one tile, the other tile's epilogue warps read their accumulator,
// write S, and store the next panel.  Roles:
//   warps 0-3 / 4-7 : epilogue of tile 0 / 1 (thread = TMEM lane = source column);
//   warp 8          : bulk-copy producer (F hi/lo, stencil pack, G rows of injecting sources);
//   warp 9          : TMEM allocation and MMA issue.
// Barriers: full[st] (copy landed), empty[st] (MMAs and epilogues done with the stage),
// dready[u] (tile u's accumulator complete), aready[u] (tile u's panel stored).  Every wait is
// bounded and also gives up once another role has raised the CTA's abort flag.
// ---------------------------------------------------------------------------------------------
template <int MB>
struct Tc2Cfg {
  static constexpr int TILE = 128;                            // sources per tile (MMA M)
  static constexpr int NT = 2;                                // tiles per CTA
  static constexpr int NST = 4;                               // ring stages
  static constexpr uint32_t FBLK = MB * MB * 4;               // one factor part (hi or lo)
  static constexpr uint32_t PKB = PK_NFIELDS * MB * 4;        // stencil pack of one block
  static constexpr uint32_t GSLOT = 4096;                     // p G rows of the injecting sources
  static constexpr uint32_t STAGE = 2 * FBLK + PKB + GSLOT;
  static constexpr int THREADS = NT * TILE + 64;
  static constexpr int TCOLS = NT * 3 * MB <= 256 ? 256 : 512;
  static constexpr size_t RING = (size_t)NST * STAGE;
  static constexpr size_t BARS = 8 * (2 * NST + 2 * NT + 1);
  // at most 512 / TCOLS CTAs may share an SM's tensor memory: pad shared memory to enforce it
  static constexpr size_t MIN_SMEM = TCOLS == 512 ? 120 * 1024 : 80 * 1024;
  static constexpr size_t SMEM = RING + BARS > MIN_SMEM ? RING + BARS : MIN_SMEM;
};

__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also returns (false) once *abort is set by another role.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort,
                                             DevStatus* st, int slab, int block) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > 4000000000LL) {
      set_status(st, ST_TIMEOUT, slab, block);
      *abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void mma_tf32_tmem_a(uint32_t tmem_d, uint32_t tmem_a, uint64_t b,
                                                uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}

// 16 consecutive 32-bit columns of this warp's 32 TMEM lanes (one lane per thread).
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

template <int MB>
__global__ void __launch_bounds__(Tc2Cfg<MB>::THREADS, 1)
    k_sbuild_tc2(const SlabDesc* __restrict__ slabs, const TileDesc* __restrict__ tiles,
                 const float* __restrict__ Fhi, const float* __restrict__ Flo,
                 const float* __restrict__ Bhi, const float* __restrict__ Blo,
                 const float* __restrict__ G, const float* __restrict__ pack,
                 float* __restrict__ S, DevStatus* st) {
  using C = Tc2Cfg<MB>;
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
        if (stp >= NST && !mbar_wait_ab(&empty[stage], ((stp / NST) - 1) & 1, abort, st, td.slab, blk(stp)))
          break;
        const int i = blk(stp);
        const bool has_f = stp < len - 1;
        // sources of this CTA injected at block i: q in [(i-1) p, i p) and [q0, q0 + nq)
        const int64_t qa = (int64_t)(i - 1) * s.p, qb = qa + s.p;
        const bool has_g = g_in_ring && qa < td.q0 + td.nq && qb > td.q0;
        const uint32_t gbytes = (uint32_t)s.p * MB * 4;
        unsigned char* sb = ring + stage * C::STAGE;
        mbar_arrive_expect_tx(&full[stage], C::PKB + (has_f ? 2 * C::FBLK : 0u) + (has_g ? gbytes : 0u));
        bulk_g2s(sb + 2 * C::FBLK, pack + s.pack_off + (int64_t)(i - 1) * PK_NFIELDS * MB, C::PKB,
                 &full[stage]);
        if (has_f) {
          const int fidx = up ? i - 2 : i;
          bulk_g2s(sb, Fh + (int64_t)fidx * MB * MB, C::FBLK, &full[stage]);
          bulk_g2s(sb + C::FBLK, Fl + (int64_t)fidx * MB * MB, C::FBLK, &full[stage]);
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
        if (!mbar_wait_ab(&full[stage], (stp / NST) & 1, abort, st, td.slab, i)) break;
        const unsigned char* fb = ring + stage * C::STAGE;
        const uint32_t b_hi = smem_u32(fb), b_lo = smem_u32(fb + C::FBLK);
        bool ok = true;
        for (int u = 0; u < nlive; ++u) {
          if (!mbar_wait_ab(&aready[u], stp & 1, abort, st, td.slab, i)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(u * 3 * MB);
          const uint32_t a_hi = d + MB, a_lo = d + 2 * MB;
#pragma unroll
          for (int ks = 0; ks < MB / 8; ++ks) {
            const uint64_t dbh = umma_desc(b_hi + ks * 256, 128, MB * 32);
            const uint64_t dbl = umma_desc(b_lo + ks * 256, 128, MB * 32);
            mma_tf32_tmem_a(d, a_hi + ks * 8, dbh, IDESC, ks > 0 ? 1u : 0u);
            mma_tf32_tmem_a(d, a_hi + ks * 8, dbl, IDESC, 1u);
            mma_tf32_tmem_a(d, a_lo + ks * 8, dbh, IDESC, 1u);
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
    const uint32_t lane_addr = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t d_col = tmem + lane_addr + (uint32_t)(u * 3 * MB);
    const bool act = lt < td.nq - u * C::TILE;
    const int q = td.q0 + u * C::TILE + lt;
    const int k0 = q / s.p + 1, t0 = q - (k0 - 1) * s.p;
    const int64_t ng = s.ng;
    const int eastlo = (2 * s.w - 2) * s.p;
    const int rf = up ? PK_SOUTH : PK_NORTH;
    float y[MB];
#pragma unroll
    for (int r = 0; r < MB; ++r) y[r] = 0.f;
    for (int stp = 0; stp < len; ++stp) {
      const int stage = stp % NST;
      const int i = blk(stp);
      if (!mbar_wait_ab(&full[stage], (stp / NST) & 1, abort, st, td.slab, i)) break;
      if (stp > 0) {
        if (!mbar_wait_ab(&dready[u], (stp - 1) & 1, abort, st, td.slab, i)) break;
        tc_fence_after();
#pragma unroll
        for (int c16 = 0; c16 < MB; c16 += 16) {
          float v[16];
          tmem_ld16(d_col + (uint32_t)c16, v);
#pragma unroll
          for (int e = 0; e < 16; ++e) y[c16 + e] = v[e];
        }
        tmem_wait_ld();
      }
      const unsigned char* sb = ring + stage * C::STAGE;
      const float* pk = reinterpret_cast<const float*>(sb + 2 * C::FBLK);
      if (act && k0 == i) {  // inject Y_i = G_i^T e_{C_t0} (row (w-1)p + t0 of G_i)
        const float* grow = g_in_ring
                                ? reinterpret_cast<const float*>(sb + 2 * C::FBLK + C::PKB) + t0 * MB
                                : G + s.fac_off + (int64_t)(i - 1) * MB * MB +
                                      (int64_t)((s.w - 1) * s.p + t0) * MB;
#pragma unroll
        for (int r = 0; r < MB; ++r) y[r] = grow[r];
      }
      if (act && (up ? (k0 >= i) : (k0 < i))) {
#pragma unroll
        for (int r = 0; r < MB; ++r) {
          if (r < s.p && s.sp_off >= 0)
            S[s.sp_off + ((int64_t)(i - 1) * s.p + r) * ng + q] = -pk[PK_WEST * MB + r] * y[r];
          if (r >= eastlo && r < s.m && s.sn_off >= 0)
            S[s.sn_off + ((int64_t)(i - 1) * s.p + (r - eastlo)) * ng + q] = -pk[PK_EAST * MB + r] * y[r];
        }
      }
      if (stp < len - 1) {
        // panel row of this source: P^T = (-diag(ell_i) Y_i)^T (up) or (-diag(ups_i) Y_i)^T
#pragma unroll
        for (int c16 = 0; c16 < MB; c16 += 16) {
          uint32_t hi[16], lo[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float v = -pk[rf * MB + c16 + e] * y[c16 + e];
            const float h = tf32_rna(v);
            hi[e] = __float_as_uint(h);
            lo[e] = __float_as_uint(tf32_rna(v - h));
          }
          tmem_st16(d_col + (uint32_t)(MB + c16), hi);
          tmem_st16(d_col + (uint32_t)(2 * MB + c16), lo);
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
static void run_tc2(const SlabDesc* d_slabs, const TileDesc* d_tiles, int ntiles,
                    const float* Fhi, const float* Flo, const float* Bhi, const float* Blo,
                    const float* G, const float* pack, float* S, DevStatus* st, cudaStream_t s) {
  using C = Tc2Cfg<MB>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_sbuild_tc2<MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    attr = true;
  }
  note_launch();
  k_sbuild_tc2<MB><<<ntiles, C::THREADS, C::SMEM, s>>>(d_slabs, d_tiles, Fhi, Flo, Bhi, Blo, G,
                                                       pack, S, st);
}

template <int MB>
static void run_tc(const SlabDesc* d_slabs, const TileDesc* d_tiles, int ntiles,
                   const float* Fhi, const float* Flo, const float* Bhi, const float* Blo,
                   const float* G, const float* pack, float* S, DevStatus* st, cudaStream_t s) {
  using C = TcCfg<MB>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_sbuild_tc<MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    attr = true;
  }
  note_launch();
  k_sbuild_tc<MB><<<ntiles, 128, C::SMEM, s>>>(d_slabs, d_tiles, Fhi, Flo, Bhi, Blo, G, pack, S, st);
}

void launch_sbuild_tc(int version, int M, const SlabDesc* d_slabs, const TileDesc* d_tiles,
                      int ntiles, const float* Fhi, const float* Flo, const float* Bhi,
                      const float* Blo, const float* G, const float* pack, float* S,
                      DevStatus* st, cudaStream_t s) {
  if (ntiles == 0) return;
  if (version == 2) {
    switch (M) {
      case 32: run_tc<32>(d_slabs, d_tiles, ntiles, Fhi, Flo, Bhi, Blo, G, pack, S, st, s); break;
      case 64: run_tc<64>(d_slabs, d_tiles, ntiles, Fhi, Flo, Bhi, Blo, G, pack, S, st, s); break;
      default: break;
    }
    return;
  }
  switch (M) {
    case 32: run_tc2<32>(d_slabs, d_tiles, ntiles, Fhi, Flo, Bhi, Blo, G, pack, S, st, s); break;
    case 64: run_tc2<64>(d_slabs, d_tiles, ntiles, Fhi, Flo, Bhi, Blo, G, pack, S, st, s); break;
    default: break;
  }
}

int sbuild_tc_tile_cols(int version) { return version == 2 ? TcCfg<64>::R : 2 * Tc2Cfg<64>::TILE; }

}  // namespace ddst
