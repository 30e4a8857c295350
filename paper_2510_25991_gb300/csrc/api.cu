// api.cu -- host orchestration behind the C ABI of include/ddst.h.
//
// Pipeline (Alg. 2 of the paper, per double slab, batched over all slabs of all problems):
//   ddst_setup            stencil pack (local discretization) + two-sided block factorization
//   ddst_build_transfer   explicit S_{j,j-1}, S_{j,j+1} by multi-RHS transposed solves (Alg. 1)
//   ddst_compress         HODLR compression of every S block (Sec. 2.4)
//   ddst_solve            fhat (Sec. 2.2, Eq. (equilib1)), GMRES on (I - K) u = fhat (Sec. 5),
//                         volume reconstruction, FP64 residual refinement
//   ddst_solve_adjoint    the same chain transposed, then gradient assembly
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ddst.h"
#include "bcr.cuh"
#include "hbs.cuh"
#include "hodlr.cuh"
#include "kernels.cuh"

using namespace ddst;

namespace {
// Message of the last error raised without a context (ddst_last_error(NULL)); one per thread,
// so concurrent setups on different threads do not overwrite each other's message.
thread_local std::string g_setup_error;
}  // namespace

namespace ddst {
void set_global_error(const std::string& m) { g_setup_error = m; }

std::atomic<long long>& launch_counter() {
  static std::atomic<long long> c{0};
  return c;
}

cudaError_t raise_smem_limit(const void* func, size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> limit;
  int dev = 0;
  const cudaError_t ed = cudaGetDevice(&dev);
  if (ed != cudaSuccess) return ed;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[{dev, func}];
  if (bytes <= cur) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}
}  // namespace ddst

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// CTAs per problem in the refinement's per-problem norms: about 1024 in all (at least 8 and at
// most 256 per problem), so a single large problem streams its vectors at full bandwidth
int norm_blocks(int nprob) { return std::max(8, std::min(256, 1024 / std::max(nprob, 1))); }

}  // namespace

// A dense operator compressed on its own into HBS form (the standalone entry points).
struct ddst_hbs {
  ddst::HbsSet H;
  int prec = 0;
  int64_t ng = 0;
  cudaStream_t st = nullptr;
  void* S = nullptr;
  double* x = nullptr;
  double* y = nullptr;
};

struct ddst_ctx {
  int nprob = 0;
  int prec = DDST_MIXED;
  cudaStream_t stream = nullptr;
  ddst_options opt{};
  std::vector<ProbDesc> probs;
  std::vector<SlabDesc> slabs;
  std::map<int, std::vector<int>> cls;     // M -> slab ids
  std::map<int, int*> d_cls;               // M -> device id array
  std::map<int, int> cls_maxnb;
  ProbDesc* d_probs = nullptr;
  SlabDesc* d_slabs = nullptr;
  DevStatus* d_st = nullptr;
  int max_nb = 0;
  int64_t max_ng = 0;
  int64_t tot_nodes = 0, tot_vol = 0, tot_if = 0, tot_loc = 0, fac_elems = 0, pack_elems = 0,
          s_elems = 0;
  size_t esz = 4;  // sizeof working precision
  // device buffers
  double *d_a = nullptr, *d_c = nullptr;
  void *F = nullptr, *B = nullptr, *G = nullptr, *Ft = nullptr, *Bt = nullptr, *pack = nullptr,
       *S = nullptr;
  void *loc_b = nullptr, *loc_bf = nullptr, *loc_bb = nullptr, *loc_x = nullptr;
  double *d_f = nullptr, *d_g = nullptr, *d_b = nullptr, *d_u = nullptr, *d_r = nullptr,
         *d_e = nullptr, *d_lam = nullptr, *d_ga = nullptr, *d_gn = nullptr, *d_an = nullptr;
  double *if_fh = nullptr, *if_u = nullptr, *if_w = nullptr, *if_tmp = nullptr;
  double *V = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *gv = nullptr,
         *resid = nullptr, *part = nullptr, *scal = nullptr,
         *ysol = nullptr;
  double *pn_part = nullptr, *pn = nullptr;  // per-problem norms of the refinement (2 nprob each)
  int ldh = 0;
  int nchunk = 0;
  HodlrSet hodlr;  // compressed operators (when compressed)
  HbsSet hbs;      // nested-basis operators (when compressed into HBS form)
  int state = 0;   // 1 factored, 2 transfer formed, 3 HODLR, 4 HBS
  bool have_solution = false;
  std::vector<void*> owned;
  std::string err;
  float t_factor = 0.f, t_transfer = 0.f, t_compress = 0.f;
  int factor_chunks = 1;
  double factor_check = 0.0;
  bool use_tc = false;            // FP32 transfer build on tcgen05
  cudaStream_t cap_stream = nullptr;     // internal stream for graph capture
  // one GMRES step, captured per (transposed, operator group): index 2 transpose + group
  cudaGraphExec_t arn_graph[4] = {nullptr, nullptr, nullptr, nullptr};
  int arn_graph_state[4] = {0, 0, 0, 0};  // operator state the graphs were captured for
  // A context whose problems are partly explicit and partly matrix-free keeps the two operator
  // groups' interfaces contiguous (explicit problems first) and runs one GMRES per group, so the
  // explicit problems do not pay a local solve per iteration for as long as the matrix-free ones
  // iterate (and the other way round).  grp_off / grp_n: interface range of each group.
  bool grouped = false;
  int64_t grp_off[2] = {0, 0}, grp_n[2] = {0, 0};
  int* d_k = nullptr;                    // device-resident Krylov basis count
  double* arn_part = nullptr;            // Arnoldi partial sums: 2 (maxit+1) + 1 rows of chunks
  unsigned* arn_ticket = nullptr;        // last-CTA ticket of the Arnoldi finish kernel
  double *h1 = nullptr, *h2 = nullptr, *d_beta = nullptr;
  float *Uhi = nullptr, *Ulo = nullptr;  // tensor-core operand copies of F^T | B^T
  // large-block classes (M > 128, or > 64 in FP64): one-sided factors in Fbig, work buffers
  std::map<int, bool> big;               // M -> factored by the large-block kernels
  int64_t fac_big_elems = 0;
  void* Fbig = nullptr;
  struct BigWork { void *C[2] = {}, *XqT[2] = {}, *RT[2] = {}, *Pinv[2] = {}; };  // two sets
  std::map<int, BigWork> bigw;
  int big_tc = 0;                        // large-block updates: 0 FMA, 1 tcgen05 3xTF32, 2 TF32
  bool tf32 = false;                     // DDST_MIXED_TF32: one TF32 product per tensor-core step
  // look-ahead of the large-block factorization: panel steps on a high-priority stream, the bulk
  // updates on a second one
  cudaStream_t s_hi = nullptr, s_lo = nullptr;
  cudaEvent_t big_ev[5] = {};
  // matrix-free interface operator (no explicit S): its own slab-local buffers, so that an
  // application inside GMRES leaves the DD solve's vectors untouched
  // matfree: every class is applied matrix-free; mf_any: at least one (large-block classes in
  // an otherwise explicit context); mf_cls: per class
  bool matfree = false, mf_any = false;
  std::map<int, bool> mf_cls;
  int* d_mf_ids = nullptr;               // slabs of the matrix-free classes
  int n_mf_ids = 0;
  void *mf_b = nullptr, *mf_z = nullptr, *mf_z2 = nullptr, *mf_x = nullptr;
  double* if_kx = nullptr;
  double* d_vel = nullptr;               // marching: nodal velocity components of every problem
  long long arn_graph_launches[4] = {0, 0, 0, 0};  // kernels per replay of each captured step
  bool solve_bufs_ready = false;
  // direct interface solver (interface_solver = 1): block cyclic reduction of every problem's
  // equilibrium system, formed from the explicit S at the first solve after build_transfer
  std::vector<BcrSystem> bcr;
  bool bcr_ready = false;
  float t_bcr = 0.f;
  bool factors_valid = false;            // local factors present (recompute_factors releases them)
};

namespace {

ddst_status fail(ddst_ctx* c, ddst_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf; else g_setup_error = buf;
  return s;
}

ddst_status cuda_fail(ddst_ctx* c, cudaError_t e, const char* what) {
  return fail(c, e == cudaErrorMemoryAllocation ? DDST_ERR_OOM : DDST_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define CK(expr)                                                 \
  do {                                                           \
    cudaError_t _e = (expr);                                     \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #expr);     \
  } while (0)

// Allocation-failure injection for tests of the out-of-memory path: with the environment
// variable DDST_FAIL_ALLOC=k, the k-th device allocation of the library made after the variable
// was set (or changed) fails as cudaErrorMemoryAllocation without calling cudaMalloc.
bool inject_alloc_failure() {
  static std::mutex mu;
  static std::string last;
  static long count = 0;
  const char* v = getenv("DDST_FAIL_ALLOC");
  std::lock_guard<std::mutex> lock(mu);
  if (!v || !*v) {
    last.clear();
    count = 0;
    return false;
  }
  if (last != v) {
    last = v;
    count = 0;
  }
  return ++count == atol(v);
}

// Bounded-wait budget of the pipelined tensor-core kernels' role waits, in clock cycles: 4e9
// (about 2 s), or DDST_WAIT_CYCLES when set (a testing hook that makes a wait expire).
long long pipeline_wait_budget() {
  const char* v = getenv("DDST_WAIT_CYCLES");
  const long long c = v ? atoll(v) : 0;
  return c > 0 ? c : 4000000000LL;
}

template <typename P>
cudaError_t dalloc(ddst_ctx* ctx, P** out, size_t bytes) {
  if (inject_alloc_failure()) return cudaErrorMemoryAllocation;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes < 16 ? 16 : bytes);
  if (e != cudaSuccess) { cudaGetLastError(); return e; }
  ctx->owned.push_back(p);
  *out = reinterpret_cast<P*>(p);
  return cudaSuccess;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Copy n doubles from a host or device pointer into device memory dst (stream-ordered).
cudaError_t stage_in(double* dst, const double* src, size_t n, cudaStream_t st) {
  return cudaMemcpyAsync(dst, src, n * sizeof(double),
                         is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
}

cudaError_t stage_out(double* dst, const double* src, size_t n, cudaStream_t st) {
  return cudaMemcpyAsync(dst, src, n * sizeof(double),
                         is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
}

ddst_status check_status(ddst_ctx* ctx, ddst_info* info) {
  DevStatus h;
  CK(cudaMemcpyAsync(&h, ctx->d_st, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (h.code == 0) return DDST_OK;
  CK(cudaMemsetAsync(ctx->d_st, 0, sizeof(DevStatus), ctx->stream));
  if (info) {
    info->fail_slab = h.slab;
    info->fail_block = h.block;
  }
  if (h.code == ST_SINGULAR)
    return fail(ctx, DDST_ERR_SINGULAR, "singular pivot in slab %d (block %d)", h.slab, h.block);
  if (h.code == ST_TIMEOUT)
    return fail(ctx, DDST_ERR_TIMEOUT, "bounded device wait expired (slab %d, block %d)", h.slab,
                h.block);
  return fail(ctx, DDST_ERR_CUDA, "device status %d", h.code);
}

// Padded block size: 32, 64 or 128 for the single-CTA kernels, else a multiple of 128 (at most
// 8192) for the large-block kernels.
int pad_M(int m) {
  if (m <= 32) return 32;
  if (m <= 64) return 64;
  if (m <= 128) return 128;
  return m <= 8192 ? ((m + 127) / 128) * 128 : -1;
}

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
  float stop() {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

void drop_graphs(ddst_ctx* ctx) {
  for (int q = 0; q < 4; ++q) {
    if (ctx->arn_graph[q]) cudaGraphExecDestroy(ctx->arn_graph[q]);
    ctx->arn_graph[q] = nullptr;
    ctx->arn_graph_state[q] = 0;
  }
}

// --------------------------------------------------------------------------------------------
// Factorization: pivot sweeps in warm-started chunks (verified), exact fallback, diagonal blocks
// --------------------------------------------------------------------------------------------
template <typename T>
ddst_status factor_all(ddst_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const bool f32 = sizeof(T) == 4;
  const double tol = f32 ? 1e-5 : 1e-11;
  auto plan = [&](int M, const std::vector<int>& ids, bool exact, std::vector<FacChunk>& out,
                  int& nslots) {
    const int conc = factor_ctas_per_sm<T>(M) * nsm;
    const int per_sd = std::max(1, conc / std::max(1, 2 * (int)ids.size()));
    for (int sid : ids) {
      const SlabDesc& s = ctx->slabs[sid];
      const int W = ctx->opt.factor_warmup > 0 ? ctx->opt.factor_warmup : (f32 ? 4 : 10) * s.w;
      int nch = 1;
      if (!exact) {
        if (ctx->opt.factor_chunks > 1) nch = ctx->opt.factor_chunks;
        else if (ctx->opt.factor_chunks == 0 && s.nb >= 4 * W) nch = per_sd;
        nch = std::max(1, std::min(nch, s.nb / 2));
      }
      const int C = (s.nb + nch - 1) / nch;
      for (int dir = 0; dir < 2; ++dir) {
        for (int c = 0; c < nch; ++c) {
          FacChunk f{};
          f.slab = sid;
          f.dir = dir;
          if (dir == 0) {
            f.first = c * C + 1;
            f.last = std::min(s.nb, (c + 1) * C);
            f.start = std::max(1, f.first - W);
            f.chk = f.start == 1 ? -1 : nslots++;
          } else {
            f.first = s.nb - c * C;
            f.last = std::max(1, s.nb - (c + 1) * C + 1);
            f.start = std::min(s.nb, f.first + W);
            f.chk = f.start == s.nb ? -1 : nslots++;
          }
          if ((f.last - f.first) * (dir == 0 ? 1 : -1) < 0) continue;
          out.push_back(f);
        }
      }
    }
    std::stable_sort(out.begin(), out.end(), [](const FacChunk& a, const FacChunk& b) {
      return std::abs(a.last - a.start) > std::abs(b.last - b.start);
    });
  };
  auto run_sweeps = [&](bool exact, double& worst, int& chunks_used) -> ddst_status {
    worst = 0.0;
    chunks_used = 1;
    for (auto& kv : ctx->cls) {
      if (ctx->big[kv.first]) continue;
      std::vector<FacChunk> ch;
      int nslots = 0;
      plan(kv.first, kv.second, exact, ch, nslots);
      chunks_used = std::max<int>(chunks_used, (int)(ch.size() / (2 * kv.second.size())));
      FacChunk* d_ch = nullptr;
      T* d_chk = nullptr;
      float* d_diff = nullptr;
      CK(cudaMallocAsync(&d_ch, sizeof(FacChunk) * ch.size(), st));
      CK(cudaMallocAsync(&d_chk, sizeof(T) * (size_t)std::max(1, nslots) * kv.first * kv.first, st));
      CK(cudaMallocAsync(&d_diff, sizeof(float) * ch.size(), st));
      CK(cudaMemcpyAsync(d_ch, ch.data(), sizeof(FacChunk) * ch.size(), cudaMemcpyHostToDevice, st));
      launch_factor<T>(kv.first, 0, ctx->d_slabs, d_ch, (int)ch.size(), ctx->d_cls[kv.first],
                       (int)kv.second.size(), ctx->cls_maxnb[kv.first], (T*)ctx->pack, (T*)ctx->F,
                       (T*)ctx->B, (T*)ctx->G, (T*)ctx->Ft, (T*)ctx->Bt, d_chk, d_diff,
                       ctx->use_tc ? ctx->Uhi : nullptr, ctx->use_tc ? ctx->Ulo : nullptr,
                       ctx->fac_elems, ctx->d_st, st);
      CK(cudaGetLastError());
      std::vector<float> diff(ch.size());
      CK(cudaMemcpyAsync(diff.data(), d_diff, sizeof(float) * ch.size(), cudaMemcpyDeviceToHost, st));
      CK(cudaFreeAsync(d_ch, st));
      CK(cudaFreeAsync(d_chk, st));
      CK(cudaFreeAsync(d_diff, st));
      CK(cudaStreamSynchronize(st));
      for (float d : diff) worst = (d == d) ? std::max(worst, (double)d) : HUGE_VAL;  // NaN fails
    }
    return DDST_OK;
  };
  double worst = 0.0;
  int used = 1;
  ddst_status s = run_sweeps(ctx->opt.factor_chunks == 1, worst, used);
  if (s != DDST_OK) return s;
  if (!(worst <= tol)) {  // a warm-up did not converge (or produced NaN): exact sweeps
    ctx->factor_check = worst;
    double w2 = 0.0;
    s = run_sweeps(true, w2, used);
    if (s != DDST_OK) return s;
    used = 1;
  } else {
    ctx->factor_check = worst;
  }
  ctx->factor_chunks = used;
  for (auto& kv : ctx->cls) {
    if (ctx->big[kv.first]) continue;
    launch_factor<T>(kv.first, 1, ctx->d_slabs, nullptr, 0, ctx->d_cls[kv.first],
                     (int)kv.second.size(), ctx->cls_maxnb[kv.first], (T*)ctx->pack, (T*)ctx->F,
                     (T*)ctx->B, (T*)ctx->G, (T*)ctx->Ft, (T*)ctx->Bt, nullptr, nullptr, nullptr,
                     nullptr, 0, ctx->d_st, st);
  }
  CK(cudaGetLastError());
  // large blocks: one-sided block LU, every slab of a class one block row at a time, on the
  // look-ahead streams, joined back into the context stream at the end
  if (ctx->s_hi) {
    CK(cudaEventRecord(ctx->big_ev[3], st));
    CK(cudaStreamWaitEvent(ctx->s_hi, ctx->big_ev[3], 0));
    for (auto& kv : ctx->cls) {
      if (!ctx->big[kv.first]) continue;
      ddst_ctx::BigWork& bw = ctx->bigw[kv.first];
      T* C[2] = {(T*)bw.C[0], (T*)bw.C[1]};
      T* XqT[2] = {(T*)bw.XqT[0], (T*)bw.XqT[1]};
      T* RT[2] = {(T*)bw.RT[0], (T*)bw.RT[1]};
      T* Pinv[2] = {(T*)bw.Pinv[0], (T*)bw.Pinv[1]};
      for (int k = 1; k <= ctx->cls_maxnb[kv.first]; ++k) {
        launch_big_factor_step<T>(kv.first, ctx->d_slabs, ctx->d_cls[kv.first],
                                  (int)kv.second.size(), (const T*)ctx->pack, (T*)ctx->Fbig, k, C,
                                  XqT, RT, Pinv, ctx->big_tc, ctx->d_st, ctx->s_hi, ctx->s_lo,
                                  ctx->big_ev);
        CK(cudaGetLastError());
      }
    }
    CK(cudaEventRecord(ctx->big_ev[4], ctx->s_hi));
    CK(cudaStreamWaitEvent(st, ctx->big_ev[4], 0));
  }
  return DDST_OK;
}

// --------------------------------------------------------------------------------------------
// Factor storage: allocated at setup, and (recompute_factors) released once the transfer
// operators exist and recomputed for every solve
// --------------------------------------------------------------------------------------------
void dfree(ddst_ctx* ctx, void*& p) {
  if (!p) return;
  auto it = std::find(ctx->owned.begin(), ctx->owned.end(), p);
  if (it != ctx->owned.end()) ctx->owned.erase(it);
  cudaFree(p);
  p = nullptr;
}

cudaError_t alloc_factors(ddst_ctx* ctx) {
  const size_t es = ctx->esz;
  cudaError_t e;
#define AF(ptr, bytes) if ((e = dalloc(ctx, &(ptr), (bytes))) != cudaSuccess) return e;
  AF(ctx->F, es * ctx->fac_elems);
  AF(ctx->B, es * ctx->fac_elems);
  AF(ctx->G, es * ctx->fac_elems);
  AF(ctx->Ft, es * ctx->fac_elems);
  AF(ctx->Bt, es * ctx->fac_elems);
  if (ctx->use_tc) {
    AF(ctx->Uhi, sizeof(float) * 2 * ctx->fac_elems);
    AF(ctx->Ulo, sizeof(float) * 2 * ctx->fac_elems);
  }
  if (ctx->fac_big_elems > 0) AF(ctx->Fbig, es * ctx->fac_big_elems);
  for (auto& kv : ctx->cls) {
    if (!ctx->big[kv.first]) continue;
    // panels of 128 columns per slab: plain (FMA path) or split into TF32 hi/lo parts
    // (tensor-core path), hence twice the plain size
    ddst_ctx::BigWork& bw = ctx->bigw[kv.first];
    const size_t panel = 2 * es * kv.second.size() * (size_t)kv.first * 128;
    for (int b = 0; b < 2; ++b) {
      AF(bw.C[b], panel);
      AF(bw.XqT[b], panel);
      AF(bw.RT[b], panel);
      AF(bw.Pinv[b], 2 * es * kv.second.size() * 128 * 128);
    }
  }
#undef AF
  ctx->factors_valid = false;
  return cudaSuccess;
}

void release_factors(ddst_ctx* ctx) {
  cudaStreamSynchronize(ctx->stream);
  void** arrays[] = {&ctx->F, &ctx->B, &ctx->G, &ctx->Ft, &ctx->Bt, &ctx->Fbig,
                     reinterpret_cast<void**>(&ctx->Uhi), reinterpret_cast<void**>(&ctx->Ulo)};
  for (void** a : arrays) dfree(ctx, *a);
  for (auto& kv : ctx->bigw)
    for (int b = 0; b < 2; ++b) {
      dfree(ctx, kv.second.C[b]);
      dfree(ctx, kv.second.XqT[b]);
      dfree(ctx, kv.second.RT[b]);
      dfree(ctx, kv.second.Pinv[b]);
    }
  ctx->factors_valid = false;
}

// --------------------------------------------------------------------------------------------
// Setup
// --------------------------------------------------------------------------------------------
ddst_status setup_impl(int nprob, const ddst_grid* grids, const ddst_coeffs* coeffs,
                       const int* widths, const ddst_options* opt, void* stream, ddst_ctx** out) {
  if (!out) return fail(nullptr, DDST_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nprob <= 0 || !grids || !coeffs || !widths)
    return fail(nullptr, DDST_ERR_INVALID_ARG, "bad problem list");
  ddst_ctx* ctx = new ddst_ctx();
  ctx->nprob = nprob;
  ctx->stream = reinterpret_cast<cudaStream_t>(stream);
  if (opt) ctx->opt = *opt; else ddst_options_default(&ctx->opt);
  ctx->opt.autotune_cache = nullptr;  // read by the setup wrapper only; not kept
  ctx->prec = ctx->opt.precision == DDST_FP64 ? DDST_FP64 : DDST_MIXED;
  ctx->tf32 = ctx->opt.precision == DDST_MIXED_TF32;
  ctx->esz = ctx->prec == DDST_FP64 ? 8 : 4;
  const bool auto_tol = !(ctx->opt.gmres_tol > 0.0);  // picked once the operator kind is known
  int64_t node_off = 0, vol_off = 0, if_off = 0, fac_off = 0, fac_big_off = 0, pack_off = 0,
          loc_off = 0, s_off = 0;
  // Operator groups: with automatic explicit_S, problems whose blocks exceed the single-CTA
  // kernels are applied matrix-free and the others explicitly.  Their interfaces are laid out
  // group by group (explicit first), so that each group's GMRES works on a contiguous range.
  // (Arguments are checked in the loop below; an invalid problem only gets a placeholder here.)
  std::vector<int> grp(nprob, 0);
  std::vector<int64_t> if_len(nprob, 0), if_base(nprob, 0);
  {
    bool any_b = false, all_b = true;
    for (int q = 0; q < nprob; ++q) {
      const ddst_grid& gr = grids[q];
      const int w = widths[q];
      bool big = false;
      if ((gr.dim == 2 || gr.dim == 3) && w >= 1 && gr.n >= 4 && gr.n <= (1 << 20) &&
          gr.n % w == 0 && gr.n / w >= 2) {
        const int64_t pp = gr.dim == 2 ? 1 : gr.n - 1;
        const int64_t m = (2 * (int64_t)w - 1) * pp;
        const int M = m <= 8192 ? pad_M((int)m) : -1;
        big = M < 0 || M > 128 || (ctx->prec == DDST_FP64 && M > 64);
        if_len[q] = (gr.n / w - 1) * (gr.dim == 2 ? gr.n - 1 : (gr.n - 1) * (gr.n - 1));
      }
      grp[q] = big ? 1 : 0;
      any_b = any_b || big;
      all_b = all_b && big;
    }
    ctx->grouped = ctx->opt.explicit_S < 0 && any_b && !all_b;
    int64_t o = 0;
    for (int g = 0; g < 2; ++g) {
      ctx->grp_off[g] = o;
      for (int q = 0; q < nprob; ++q)
        if ((ctx->grouped ? grp[q] : 0) == g) {
          if_base[q] = o;
          o += if_len[q];
        }
      ctx->grp_n[g] = o - ctx->grp_off[g];
    }
  }
  for (int q = 0; q < nprob; ++q) {
    const ddst_grid& gr = grids[q];
    const int w = widths[q];
    if (gr.dim != 2 && gr.dim != 3) { ddst_destroy(ctx); return fail(nullptr, DDST_ERR_INVALID_ARG, "dim must be 2 or 3"); }
    if (gr.n < 4 || gr.n > (1 << 20) || w < 1 || gr.n % w != 0 || gr.n / w < 2) {
      ddst_destroy(ctx);
      return fail(nullptr, DDST_ERR_INVALID_ARG, "problem %d: need n %% w == 0 and n/w >= 2", q);
    }
    if (!coeffs[q].a) { ddst_destroy(ctx); return fail(nullptr, DDST_ERR_INVALID_ARG, "problem %d: a is NULL", q); }
    ProbDesc P{};
    P.dim = gr.dim;
    P.n = (int)gr.n;
    P.w = w;
    P.nds = P.n / w - 1;
    P.p = gr.dim == 2 ? 1 : P.n - 1;
    P.m = (2 * w - 1) * P.p;
    P.M = pad_M(P.m);
    if (P.M < 0) {
      ddst_destroy(ctx);
      return fail(nullptr, DDST_ERR_INVALID_ARG,
                  "problem %d: block size (2w-1)(n-1)^(dim-2) = %d exceeds 8192", q, P.m);
    }
    // blocks above the single-CTA kernels' reach (128 in FP32, 64 in FP64) go to the
    // large-block kernels, padded to a multiple of 128
    const bool isbig = P.M > 128 || (ctx->prec == DDST_FP64 && P.M > 64);
    if (isbig) P.M = ((P.m + 127) / 128) * 128;
    ctx->big[P.M] = isbig;
    P.nb = P.n - 1;
    P.ng = (int64_t)P.nb * P.p;
    P.nint = 1;
    P.nnode = 1;
    for (int d = 0; d < gr.dim; ++d) { P.nint *= (P.n - 1); P.nnode *= (P.n + 1); }
    P.vol_off = vol_off;
    P.node_off = node_off;
    P.if_off = if_base[q];
    P.slab0 = (int)ctx->slabs.size();
    P.has_c = coeffs[q].c != nullptr;
    P.h = 1.0 / P.n;
    for (int d = 0; d < 3; ++d) P.b[d] = d < gr.dim ? coeffs[q].b[d] : 0.0;
    for (int j = 1; j <= P.nds; ++j) {
      SlabDesc s{};
      s.prob = q; s.j = j; s.M = P.M; s.m = P.m; s.nb = P.nb; s.p = P.p; s.w = w; s.n = P.n;
      s.ng = P.ng;
      if (isbig) { s.fac_off = fac_big_off; fac_big_off += (int64_t)P.nb * P.M * P.M; }
      else { s.fac_off = fac_off; fac_off += (int64_t)P.nb * P.M * P.M; }
      s.pack_off = pack_off; pack_off += (int64_t)P.nb * PK_NFIELDS * P.M;
      s.loc_off = loc_off; loc_off += (int64_t)P.nb * P.M;
      s.sp_off = -1; s.sn_off = -1;  // large-block slabs never form S
      if (j >= 2 && !isbig) { s.sp_off = s_off; s_off += P.ng * P.ng; }
      if (j <= P.nds - 1 && !isbig) { s.sn_off = s_off; s_off += P.ng * P.ng; }
      s.vol_off = vol_off; s.node_off = node_off;
      s.if_off = P.if_off + (int64_t)(j - 1) * P.ng;
      ctx->cls[P.M].push_back((int)ctx->slabs.size());
      ctx->cls_maxnb[P.M] = std::max(ctx->cls_maxnb[P.M], P.nb);
      ctx->slabs.push_back(s);
    }
    ctx->max_nb = std::max(ctx->max_nb, P.nb);
    ctx->max_ng = std::max(ctx->max_ng, P.ng);
    node_off += P.nnode;
    vol_off += P.nint;
    if_off += (int64_t)P.nds * P.ng;
    ctx->probs.push_back(P);
  }
  ctx->tot_nodes = node_off; ctx->tot_vol = vol_off; ctx->tot_if = if_off;
  ctx->tot_loc = loc_off; ctx->fac_elems = fac_off; ctx->pack_elems = pack_off; ctx->s_elems = s_off;
  ctx->fac_big_elems = fac_big_off;
  bool any_big = false;
  for (auto& kv : ctx->big) any_big = any_big || kv.second;
  if (ctx->opt.explicit_S == 1 && any_big) {
    ddst_destroy(ctx);
    return fail(nullptr, DDST_ERR_INVALID_ARG,
                "explicit transfer operators need blocks of at most 128 (64 in FP64) unknowns; "
                "use explicit_S = 0 or -1 (matrix-free) for larger blocks");
  }
  bool all_big = true;
  for (auto& kv : ctx->big) all_big = all_big && kv.second;
  ctx->matfree = ctx->opt.explicit_S == 0 || (ctx->opt.explicit_S < 0 && all_big);
  ctx->mf_any = ctx->matfree || any_big;
  std::vector<int> mf_ids;
  for (auto& kv : ctx->cls) {
    ctx->mf_cls[kv.first] = ctx->matfree || ctx->big[kv.first];
    if (ctx->mf_cls[kv.first]) mf_ids.insert(mf_ids.end(), kv.second.begin(), kv.second.end());
  }
  ctx->n_mf_ids = (int)mf_ids.size();
  // automatic inner tolerance: the FP64 DD solve is accurate, so a tight inner tolerance
  // finishes in one or two refinement steps.  The FP32 DD solve is only an approximate inverse
  // inside the FP64 refinement: with explicit operators (a 120 us iteration against a few ms of
  // local solves per refinement step) 1e-3 balances iterations against steps; with matrix-free
  // operators every iteration is itself a local solve, and 1e-2 is cheaper (both measured on
  // the 2048^2 and 127^3 workloads).
  if (auto_tol) ctx->opt.gmres_tol = ctx->prec == DDST_FP64 ? 1e-10 : (ctx->mf_any ? 1e-2 : 1e-3);
  ctx->big_tc = ctx->prec == DDST_MIXED && ctx->opt.tensor_cores != 0 ? (ctx->tf32 ? 2 : 1) : 0;
  const int nslab = (int)ctx->slabs.size();
  const size_t es = ctx->esz;
  cudaError_t e;
#define AL(ptr, bytes)                                                        \
  if ((e = dalloc(ctx, &(ptr), (bytes))) != cudaSuccess) {                    \
    ddst_status s_ = cuda_fail(nullptr, e, "cudaMalloc " #ptr);               \
    ddst_destroy(ctx);                                                        \
    return s_;                                                                \
  }
  AL(ctx->d_probs, sizeof(ProbDesc) * nprob);
  AL(ctx->d_slabs, sizeof(SlabDesc) * nslab);
  AL(ctx->d_st, sizeof(DevStatus));
  AL(ctx->d_a, sizeof(double) * ctx->tot_nodes);
  AL(ctx->d_c, sizeof(double) * ctx->tot_nodes);
  AL(ctx->pack, es * ctx->pack_elems);
  AL(ctx->loc_b, es * ctx->tot_loc);
  AL(ctx->loc_bf, es * ctx->tot_loc);
  AL(ctx->loc_bb, es * ctx->tot_loc);
  AL(ctx->loc_x, es * ctx->tot_loc);
  for (auto& kv : ctx->cls) {
    int* d = nullptr;
    AL(d, sizeof(int) * kv.second.size());
    ctx->d_cls[kv.first] = d;
  }
  if (any_big) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if ((e = cudaStreamCreateWithPriority(&ctx->s_hi, cudaStreamNonBlocking, hi)) != cudaSuccess ||
        (e = cudaStreamCreateWithPriority(&ctx->s_lo, cudaStreamNonBlocking, lo)) != cudaSuccess) {
      ddst_status s_ = cuda_fail(nullptr, e, "stream create");
      ddst_destroy(ctx);
      return s_;
    }
    for (cudaEvent_t& ev : ctx->big_ev)
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
        ddst_status s_ = cuda_fail(nullptr, e, "event create");
        ddst_destroy(ctx);
        return s_;
      }
  }
  if (ctx->mf_any) {
    AL(ctx->mf_b, es * ctx->tot_loc);
    AL(ctx->mf_z, es * ctx->tot_loc);
    AL(ctx->mf_z2, es * ctx->tot_loc);
    AL(ctx->mf_x, es * ctx->tot_loc);
    AL(ctx->if_kx, sizeof(double) * ctx->tot_if);
    AL(ctx->d_mf_ids, sizeof(int) * mf_ids.size());
  }
  // tensor-core transfer build: explicit classes only, all of them with blocks <= 64
  ctx->use_tc = ctx->prec == DDST_MIXED && ctx->opt.tensor_cores != 0 && !ctx->matfree;
  for (auto& kv : ctx->cls)
    if (!ctx->mf_cls[kv.first] && kv.first > 64) ctx->use_tc = false;
#undef AL
  if ((e = alloc_factors(ctx)) != cudaSuccess) {
    ddst_status s_ = cuda_fail(nullptr, e, "cudaMalloc factors");
    ddst_destroy(ctx);
    return s_;
  }
  cudaStream_t st = ctx->stream;
  auto bail = [&](cudaError_t err, const char* what) {
    ddst_status s_ = cuda_fail(nullptr, err, what);
    ddst_destroy(ctx);
    return s_;
  };
  if ((e = cudaMemcpyAsync(ctx->d_probs, ctx->probs.data(), sizeof(ProbDesc) * nprob,
                           cudaMemcpyHostToDevice, st)) != cudaSuccess) return bail(e, "copy probs");
  if ((e = cudaMemcpyAsync(ctx->d_slabs, ctx->slabs.data(), sizeof(SlabDesc) * nslab,
                           cudaMemcpyHostToDevice, st)) != cudaSuccess) return bail(e, "copy slabs");
  for (auto& kv : ctx->cls)
    if ((e = cudaMemcpyAsync(ctx->d_cls[kv.first], kv.second.data(), sizeof(int) * kv.second.size(),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess) return bail(e, "copy ids");
  if (ctx->mf_any && !mf_ids.empty() &&
      (e = cudaMemcpyAsync(ctx->d_mf_ids, mf_ids.data(), sizeof(int) * mf_ids.size(),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess) return bail(e, "copy ids");
  cudaMemsetAsync(ctx->d_st, 0, sizeof(DevStatus), st);
  cudaMemsetAsync(ctx->d_c, 0, sizeof(double) * ctx->tot_nodes, st);
  for (int q = 0; q < nprob; ++q) {
    const ProbDesc& P = ctx->probs[q];
    if ((e = stage_in(ctx->d_a + P.node_off, coeffs[q].a, P.nnode, st)) != cudaSuccess) return bail(e, "copy a");
    if (coeffs[q].c)
      if ((e = stage_in(ctx->d_c + P.node_off, coeffs[q].c, P.nnode, st)) != cudaSuccess) return bail(e, "copy c");
  }
  Timer tm(st);
  ddst_status fs;
  if (ctx->prec == DDST_FP64) {
    launch_stencil_pack<double>(ctx->d_slabs, nslab, ctx->max_nb, ctx->d_probs, ctx->d_a, ctx->d_c,
                                (double*)ctx->pack, st);
    fs = factor_all<double>(ctx);
  } else {
    launch_stencil_pack<float>(ctx->d_slabs, nslab, ctx->max_nb, ctx->d_probs, ctx->d_a, ctx->d_c,
                               (float*)ctx->pack, st);
    fs = factor_all<float>(ctx);
  }
  if (fs != DDST_OK) {
    g_setup_error = ctx->err;
    ddst_destroy(ctx);
    return fs;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return bail(e, "factor launch");
  ctx->t_factor = tm.stop();
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return bail(e, "factor");
  ddst_status s = check_status(ctx, nullptr);
  if (s != DDST_OK) {
    g_setup_error = ctx->err;
    ddst_destroy(ctx);
    return s;
  }
  ctx->factors_valid = true;
  ctx->state = 1;
  *out = ctx;
  return DDST_OK;
}

// Local factors for a solve: recomputed (allocated and factored again) when recompute_factors
// released them; the factorization time counts towards the solve.
template <typename T>
ddst_status ensure_factors(ddst_ctx* ctx) {
  if (ctx->factors_valid) return DDST_OK;
  cudaError_t e = alloc_factors(ctx);
  if (e != cudaSuccess) {
    release_factors(ctx);
    return cuda_fail(ctx, e, "cudaMalloc factors (recompute_factors)");
  }
  ddst_status fs = factor_all<T>(ctx);
  if (fs != DDST_OK) return fs;
  CK(cudaStreamSynchronize(ctx->stream));
  fs = check_status(ctx, nullptr);
  if (fs != DDST_OK) return fs;
  ctx->factors_valid = true;
  return DDST_OK;
}

void maybe_release_factors(ddst_ctx* ctx) {
  if (ctx->opt.recompute_factors == 1 && ctx->state >= 2) release_factors(ctx);
}

// --------------------------------------------------------------------------------------------
// Transfer operators
// --------------------------------------------------------------------------------------------
void drop_bcr(ddst_ctx* ctx);

template <typename T>
ddst_status build_transfer_impl(ddst_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  drop_bcr(ctx);  // formed again from the new operators when next needed
  if (ctx->matfree) {  // S is applied through the local factors: nothing to form
    ctx->t_transfer = 0.f;
    ctx->hodlr.clear();
    ctx->hbs.release();
    drop_graphs(ctx);
    ctx->state = 2;
    return DDST_OK;
  }
  if (!ctx->S) {
    cudaError_t e = dalloc(ctx, &ctx->S, sizeof(T) * ctx->s_elems);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc S");
  }
  Timer tm(st);
  for (auto& kv : ctx->cls) {
    const int M = kv.first;
    if (ctx->mf_cls[M]) continue;  // applied matrix-free
    const int R = (sizeof(T) == 4 && ctx->use_tc) ? sbuild_tc_tile_cols()
                                                  : sbuild_tile_cols<T>(M);
    std::vector<TileDesc> tiles;
    for (int sid : kv.second) {
      const SlabDesc& s = ctx->slabs[sid];
      if (s.sp_off < 0 && s.sn_off < 0) continue;
      for (int64_t q0 = 0; q0 < s.ng; q0 += R) {
        const int nq = (int)std::min<int64_t>(R, s.ng - q0);
        TileDesc up{sid, (int)q0, nq, 0, (int)((q0 + nq - 1) / s.p) + 1, 0};
        up.len = up.kstart;
        TileDesc dn{sid, (int)q0, nq, 1, (int)(q0 / s.p) + 1, 0};
        dn.len = s.nb - dn.kstart + 1;
        tiles.push_back(up);
        tiles.push_back(dn);
      }
    }
    std::stable_sort(tiles.begin(), tiles.end(),
                     [](const TileDesc& a, const TileDesc& b) { return a.len > b.len; });
    if (tiles.empty()) continue;
    TileDesc* d_tiles = nullptr;
    cudaError_t e = cudaMallocAsync(&d_tiles, sizeof(TileDesc) * tiles.size(), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMallocAsync tiles");
    CK(cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(TileDesc) * tiles.size(),
                       cudaMemcpyHostToDevice, st));
    if constexpr (sizeof(T) == 4) {
      if (ctx->use_tc)
        launch_sbuild_tc(M, ctx->d_slabs, d_tiles, (int)tiles.size(), ctx->Uhi, ctx->Ulo,
                         ctx->Uhi + ctx->fac_elems, ctx->Ulo + ctx->fac_elems, (const float*)ctx->G,
                         (const float*)ctx->pack, (float*)ctx->S, ctx->d_st,
                         pipeline_wait_budget(), ctx->tf32 ? 0 : 1, st);
      else
        launch_sbuild<T>(M, ctx->d_slabs, d_tiles, (int)tiles.size(), (const T*)ctx->F,
                         (const T*)ctx->B, (const T*)ctx->G, (const T*)ctx->pack, (T*)ctx->S,
                         ctx->d_st, st);
    } else {
      launch_sbuild<T>(M, ctx->d_slabs, d_tiles, (int)tiles.size(), (const T*)ctx->F,
                       (const T*)ctx->B, (const T*)ctx->G, (const T*)ctx->pack, (T*)ctx->S,
                       ctx->d_st, st);
    }
    CK(cudaGetLastError());
    CK(cudaFreeAsync(d_tiles, st));
  }
  ctx->t_transfer = tm.stop();
  CK(cudaStreamSynchronize(st));
  ddst_status s = check_status(ctx, nullptr);
  if (s != DDST_OK) return s;
  ctx->hodlr.clear();
  ctx->hbs.release();
  drop_graphs(ctx);
  ctx->state = 2;
  return DDST_OK;
}

// --------------------------------------------------------------------------------------------
// Solve
// --------------------------------------------------------------------------------------------
ddst_status ensure_solve_buffers(ddst_ctx* ctx) {
  // set only once every buffer exists: a failed allocation leaves the context able to retry
  if (ctx->solve_bufs_ready) return DDST_OK;
  ctx->opt.gmres_max_iter = std::max(1, std::min(ctx->opt.gmres_max_iter, 1000));
  const int maxit = ctx->opt.gmres_max_iter;
  ctx->ldh = maxit + 1;
  ctx->nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(256, (ctx->tot_if + 4095) / 4096));
  cudaError_t e;
#define AL(ptr, bytes) if ((e = dalloc(ctx, &(ptr), (bytes))) != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc " #ptr);
  AL(ctx->d_f, sizeof(double) * ctx->tot_vol);
  AL(ctx->d_g, sizeof(double) * ctx->tot_nodes);
  AL(ctx->d_b, sizeof(double) * ctx->tot_vol);
  AL(ctx->d_u, sizeof(double) * ctx->tot_vol);
  AL(ctx->d_r, sizeof(double) * ctx->tot_vol);
  AL(ctx->d_e, sizeof(double) * ctx->tot_vol);
  AL(ctx->d_lam, sizeof(double) * ctx->tot_vol);
  AL(ctx->d_ga, sizeof(double) * ctx->tot_vol);
  AL(ctx->d_gn, sizeof(double) * ctx->tot_nodes);
  AL(ctx->d_an, sizeof(double) * ctx->tot_nodes);
  AL(ctx->if_fh, sizeof(double) * ctx->tot_if);
  AL(ctx->if_u, sizeof(double) * ctx->tot_if);
  AL(ctx->if_w, sizeof(double) * ctx->tot_if);
  AL(ctx->if_tmp, sizeof(double) * ctx->tot_if);
  AL(ctx->V, sizeof(double) * ctx->tot_if * (size_t)(maxit + 1));
  AL(ctx->H, sizeof(double) * (size_t)ctx->ldh * (maxit + 1));
  AL(ctx->cs, sizeof(double) * (maxit + 1));
  AL(ctx->sn, sizeof(double) * (maxit + 1));
  AL(ctx->gv, sizeof(double) * (maxit + 2));
  AL(ctx->resid, sizeof(double) * (maxit + 1));
  AL(ctx->part, sizeof(double) * (size_t)(maxit + 1) * std::max(ctx->nchunk, 1024));
  AL(ctx->scal, sizeof(double) * 16);
  AL(ctx->pn_part, sizeof(double) * 2 * (size_t)ctx->nprob * norm_blocks(ctx->nprob));
  AL(ctx->pn, sizeof(double) * 2 * (size_t)ctx->nprob);
  AL(ctx->ysol, sizeof(double) * (maxit + 1));
  AL(ctx->d_k, sizeof(int) * 4);
  AL(ctx->h1, sizeof(double) * (maxit + 1));
  AL(ctx->h2, sizeof(double) * (maxit + 1));
  AL(ctx->d_beta, sizeof(double) * 2);
  AL(ctx->arn_part, sizeof(double) * (size_t)(2 * (maxit + 1) + 1) * arnoldi_chunks(ctx->tot_if));
  AL(ctx->arn_ticket, sizeof(unsigned) * 4);
  if ((e = cudaMemsetAsync(ctx->arn_ticket, 0, sizeof(unsigned) * 4, ctx->stream)) != cudaSuccess)
    return cuda_fail(ctx, e, "memset ticket");
#undef AL
  ctx->solve_bufs_ready = true;
  return DDST_OK;
}

// Local Dirichlet solves of every double slab, all block-size classes: x = A_j^{-1} b
// (transpose: A_j^{-T} b).  mode 0 writes x slab-locally; mode 1 (not transposed) writes the
// central rows, R_C x, into the FP64 interface vector iface.  z1, z2: slab-local temporaries.
template <typename T>
void local_solves(ddst_ctx* ctx, const T* b, T* z1, T* z2, T* x, double* iface, int transpose,
                  int mode, cudaStream_t st, bool only_mf = false) {
  for (auto& kv : ctx->cls) {
    const int M = kv.first, nids = (int)kv.second.size();
    if (only_mf && !ctx->mf_cls[M]) continue;
    if (ctx->big[M]) {
      launch_big_solve<T>(M, ctx->d_slabs, ctx->d_cls[M], nids, ctx->cls_maxnb[M],
                          (const T*)ctx->Fbig, (const T*)ctx->pack, b, z1, x, transpose, st);
      if (mode == 1) launch_big_extract<T>(ctx->d_slabs, ctx->d_cls[M], nids, x, iface, st);
    } else {
      launch_local_solve<T>(M, ctx->d_slabs, ctx->d_cls[M], nids, ctx->cls_maxnb[M], (T*)ctx->F,
                            (T*)ctx->B, (T*)ctx->Ft, (T*)ctx->Bt, (T*)ctx->G, (T*)ctx->pack, b, z1,
                            z2, x, iface, transpose, mode, ctx->d_st, st);
    }
  }
}

// y = (I - K) x, or K x (bit 1 of mode), or the transposes (bit 0), with K applied through local
// solves (Sec. 2.2, Eq. (defS)): K x = R_C A_j^{-1} (-A(I_j, J) x_J) per double slab;
// K^T x = -A(J, I_j) A_j^{-T} R_C^T x_j.  Covers the interfaces of the matrix-free classes only
// (a problem's slabs are all in one class, so K never couples them to an explicit class); uses
// the matrix-free buffers only.
template <typename T>
void apply_matfree(ddst_ctx* ctx, const double* x, double* y, int mode, cudaStream_t st,
                   const int* kdev, int64_t kstride) {
  if (ctx->n_mf_ids == 0) return;
  T* b = (T*)ctx->mf_b;
  cudaMemsetAsync(b, 0, ctx->esz * ctx->tot_loc, st);
  if (!(mode & 1)) {
    launch_mf_rhs<T>(ctx->d_slabs, ctx->d_mf_ids, ctx->n_mf_ids, ctx->d_probs, (const T*)ctx->pack,
                     x, kdev, kstride, b, st);
    local_solves<T>(ctx, b, (T*)ctx->mf_z, (T*)ctx->mf_z2, (T*)ctx->mf_x, ctx->if_kx, 0, 1, st, true);
  } else {
    launch_mf_inject<T>(ctx->d_slabs, ctx->d_mf_ids, ctx->n_mf_ids, x, kdev, kstride, b, st);
    local_solves<T>(ctx, b, (T*)ctx->mf_z, (T*)ctx->mf_z2, (T*)ctx->mf_x, nullptr, 1, 0, st, true);
    cudaMemsetAsync(ctx->if_kx, 0, sizeof(double) * ctx->tot_if, st);
    launch_mf_dirichlet_T<T>(ctx->d_slabs, ctx->d_mf_ids, ctx->n_mf_ids, ctx->d_probs,
                             (const T*)ctx->pack, (const T*)ctx->mf_x, ctx->if_kx, st);
  }
  launch_mf_combine(ctx->d_slabs, ctx->d_mf_ids, ctx->n_mf_ids, x, kdev, kstride, ctx->if_kx, y,
                    (mode & 2) ? 1 : 0, st);
}

// group: -1 every problem; 0 the explicit operators only; 1 the matrix-free ones only (a
// grouped context's per-group GMRES).  x and y are indexed by absolute interface offsets.
template <typename T>
void apply_interface_T(ddst_ctx* ctx, const double* x, double* y, int transpose,
                       cudaStream_t st = nullptr, const int* kdev = nullptr, int64_t kstride = 0,
                       int group = -1) {
  if (!st) st = ctx->stream;
  if (ctx->matfree || group == 1) {
    apply_matfree<T>(ctx, x, y, transpose, st, kdev, kstride);
    return;
  }
  // explicit operators (their apply also writes the matrix-free classes' interfaces, as if K
  // were zero there), then the matrix-free classes overwrite their own interfaces
  if (ctx->state == 4)
    hbs_apply<T>(ctx->hbs, x, y, transpose, st, kdev, kstride);
  else if (ctx->state == 3)
    hodlr_apply<T>(ctx->hodlr, ctx->d_slabs, ctx->d_probs, (int)ctx->slabs.size(), x, y, transpose,
                   st, kdev, kstride);
  else
    launch_apply_dense<T>(ctx->d_slabs, ctx->d_probs, (int)ctx->slabs.size(), ctx->max_ng,
                          (const T*)ctx->S, x, y, transpose, st, kdev, kstride);
  if (ctx->mf_any && group < 0) apply_matfree<T>(ctx, x, y, transpose, st, kdev, kstride);
}

// One GMRES step (operator application + Arnoldi CGS2 + Givens + normalization) captured as a
// CUDA graph on the internal stream; replayed on the context stream.
// group -1 (one GMRES over every problem) or a grouped context's operator group, whose GMRES
// vectors hold its interface range [grp_off, grp_off + grp_n) only.
template <typename T>
ddst_status arnoldi_graph(ddst_ctx* ctx, int transpose, int group, cudaGraphExec_t* out) {
  const int key = (transpose ? 2 : 0) + (group > 0 ? 1 : 0);
  if (ctx->arn_graph[key] && ctx->arn_graph_state[key] == ctx->state) {
    *out = ctx->arn_graph[key];
    return DDST_OK;
  }
  if (ctx->arn_graph[key]) {
    cudaGraphExecDestroy(ctx->arn_graph[key]);
    ctx->arn_graph[key] = nullptr;
  }
  if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  const int64_t n = group < 0 ? ctx->tot_if : ctx->grp_n[group];
  const int64_t off = group < 0 ? 0 : ctx->grp_off[group];
  const int maxit = std::max(1, ctx->opt.gmres_max_iter);
  cudaGraph_t g = nullptr;
  const long long l0 = launch_counter().load();
  CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
  // Arnoldi on K (bit 1 of the mode): same Krylov space as I - K, see launch_arnoldi_step.  The
  // operator kernels index by absolute interface offsets: the basis and w are passed shifted by
  // the group's offset (entries outside the group are neither read for it nor kept)
  apply_interface_T<T>(ctx, ctx->V - off, ctx->if_w - off, transpose | 2, ctx->cap_stream,
                       ctx->d_k, n, group);
  launch_arnoldi_step(ctx->V, ctx->if_w, n, ctx->d_k, ctx->h1, ctx->h2, ctx->arn_part,
                      ctx->arn_ticket, ctx->H, ctx->ldh, ctx->cs, ctx->sn, ctx->gv, ctx->d_beta,
                      ctx->resid, maxit, ctx->cap_stream);
  const cudaError_t ec = cudaStreamEndCapture(ctx->cap_stream, &g);
  // launches recorded during capture run only when the graph is replayed: count them there
  ctx->arn_graph_launches[key] = launch_counter().load() - l0;
  launch_counter().fetch_sub(ctx->arn_graph_launches[key]);
  if (ec != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(ctx, ec, "graph capture");
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return cuda_fail(ctx, ei, "graph instantiate");
  ctx->arn_graph[key] = ex;
  ctx->arn_graph_state[key] = ctx->state;
  *out = ex;
  return DDST_OK;
}

double host_scalar(ddst_ctx* ctx, const double* d) {
  double h = 0.0;
  cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  return h;
}

// --------------------------------------------------------------------------------------------
// Direct interface solver: block cyclic reduction of (I - K) from the explicit S (bcr.cu)
// --------------------------------------------------------------------------------------------
BcrEnv bcr_env(ddst_ctx* ctx) {
  BcrEnv env;
  env.alloc = [ctx](void** p, size_t b) { return dalloc(ctx, p, b); };
  env.release = [ctx](void*& p) { dfree(ctx, p); };
  env.st = ctx->stream;
  env.sh = ctx->s_hi;
  env.sl = ctx->s_lo;
  env.ev = ctx->big_ev;
  env.d_st = ctx->d_st;
  env.tensor_cores = ctx->prec == DDST_MIXED && ctx->opt.tensor_cores != 0 ? (ctx->tf32 ? 2 : 1) : 0;
  return env;
}

void drop_bcr(ddst_ctx* ctx) {
  if (ctx->bcr.empty()) return;
  cudaStreamSynchronize(ctx->stream);
  const BcrEnv env = bcr_env(ctx);
  for (BcrSystem& b : ctx->bcr) bcr_free(b, env);
  ctx->bcr.clear();
  ctx->bcr_ready = false;
}

// The panel look-ahead streams and events (created at setup when a class has large blocks).
cudaError_t ensure_side_streams(ddst_ctx* ctx) {
  cudaError_t e;
  if (!ctx->s_hi) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if ((e = cudaStreamCreateWithPriority(&ctx->s_hi, cudaStreamNonBlocking, hi)) != cudaSuccess) return e;
    if ((e = cudaStreamCreateWithPriority(&ctx->s_lo, cudaStreamNonBlocking, lo)) != cudaSuccess) return e;
  }
  for (cudaEvent_t& ev : ctx->big_ev)
    if (!ev && (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return e;
  return cudaSuccess;
}

template <typename T>
ddst_status ensure_bcr(ddst_ctx* ctx) {
  if (ctx->bcr_ready) return DDST_OK;
  if (ctx->state < 2) return fail(ctx, DDST_ERR_STATE, "ddst_build_transfer has not completed");
  if (ctx->mf_any)
    return fail(ctx, DDST_ERR_NOT_IMPLEMENTED,
                "the direct interface solve eliminates the explicit transfer operators; this "
                "context applies some matrix-free (explicit_S = 0, or blocks larger than 128)");
  for (const ProbDesc& P : ctx->probs)
    if (P.ng > 8192)
      return fail(ctx, DDST_ERR_NOT_IMPLEMENTED,
                  "direct interface solve: interfaces of %lld points exceed 8192",
                  (long long)P.ng);
  cudaError_t e = ensure_side_streams(ctx);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream create");
  drop_bcr(ctx);
  Timer tm(ctx->stream);
  const BcrEnv env = bcr_env(ctx);
  ctx->bcr.resize(ctx->nprob);
  for (int q = 0; q < ctx->nprob; ++q) {
    const ProbDesc& P = ctx->probs[q];
    std::vector<int64_t> sp(P.nds), sn(P.nds);
    for (int j = 0; j < P.nds; ++j) {
      sp[j] = ctx->slabs[P.slab0 + j].sp_off;
      sn[j] = ctx->slabs[P.slab0 + j].sn_off;
    }
    e = bcr_factor<T>(ctx->bcr[q], (const T*)ctx->S, sp, sn, P.nds, P.ng, env);
    if (e != cudaSuccess) {
      drop_bcr(ctx);
      return e == cudaErrorMemoryAllocation ? cuda_fail(ctx, e, "cudaMalloc (direct interface solver)")
                                            : cuda_fail(ctx, e, "direct interface factorization");
    }
  }
  ctx->t_bcr = tm.stop();
  ddst_status s = check_status(ctx, nullptr);
  if (s != DDST_OK) {
    drop_bcr(ctx);
    const std::string m = ctx->err;
    return fail(ctx, s, "direct interface factorization: %s (slab = interface block, 0-based)",
                m.c_str());
  }
  ctx->bcr_ready = true;
  return DDST_OK;
}

// x = (I - K)^{-1} rhs (or ^{-T}) for every problem through the factored systems.
template <typename T>
ddst_status direct_interface_solve(ddst_ctx* ctx, const double* rhs, double* x, int transpose) {
  ddst_status s = ensure_bcr<T>(ctx);
  if (s != DDST_OK) return s;
  const BcrEnv env = bcr_env(ctx);
  if (rhs != x) CK(cudaMemcpyAsync(x, rhs, sizeof(double) * ctx->tot_if, cudaMemcpyDeviceToDevice, ctx->stream));
  for (int q = 0; q < ctx->nprob; ++q) {
    const ProbDesc& P = ctx->probs[q];
    const cudaError_t e = bcr_solve<T>(ctx->bcr[q], x + P.if_off, ctx->if_tmp + P.if_off, transpose, env);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "direct interface solve");
  }
  return DDST_OK;
}

// GMRES on (I - K) x = rhs (or its transpose), x0 = 0, over one operator group's interface
// range (group -1: all of it; rhs and x point at the range's start).  Returns iterations; sets
// *relres.
template <typename T>
ddst_status gmres_range(ddst_ctx* ctx, const double* rhs, double* x, double tol, int transpose,
                        int group, int* iters, double* relres) {
  cudaStream_t st = ctx->stream;
  const int64_t n = group < 0 ? ctx->tot_if : ctx->grp_n[group];
  const int maxit = std::max(1, ctx->opt.gmres_max_iter);
  // host convergence checks: every iteration when a matrix-free application (local solves on
  // every slab) costs far more than the check's synchronization, else every 8
  const bool mf = group < 0 ? ctx->mf_any : group == 1;
  const int check = ctx->opt.check_every > 0 ? ctx->opt.check_every : (mf ? 1 : 8);
  launch_dot(rhs, rhs, n, ctx->part, 256, ctx->scal, st);
  const double beta = std::sqrt(host_scalar(ctx, ctx->scal));
  *iters = 0;
  *relres = 0.0;
  if (!(beta > 0.0)) {
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    return DDST_OK;
  }
  launch_normalize_start(rhs, ctx->scal, ctx->V, n, st);
  CK(cudaMemsetAsync(ctx->gv, 0, sizeof(double) * (maxit + 2), st));
  CK(cudaMemcpyAsync(ctx->gv, &beta, sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->d_beta, &beta, sizeof(double), cudaMemcpyHostToDevice, st));
  const int one = 1;
  CK(cudaMemcpyAsync(ctx->d_k, &one, sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(ctx->h1, 0, sizeof(double) * (maxit + 1), st));
  CK(cudaMemsetAsync(ctx->h2, 0, sizeof(double) * (maxit + 1), st));
  CK(cudaMemsetAsync(ctx->scal + 1, 0, sizeof(double), st));
  cudaGraphExec_t graph = nullptr;
  ddst_status gs = arnoldi_graph<T>(ctx, transpose, group, &graph);
  if (gs != DDST_OK) return gs;
  std::vector<double> hres(maxit + 1);
  int kk = -1;
  int k = 0;
  for (k = 1; k <= maxit; ++k) {
    CK(cudaGraphLaunch(graph, st));
    note_launch((int)ctx->arn_graph_launches[(transpose ? 2 : 0) + (group > 0 ? 1 : 0)]);
    if (k % check == 0 || k == maxit) {
      CK(cudaMemcpyAsync(hres.data(), ctx->resid, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      CK(cudaGetLastError());
      for (int i = std::max(0, k - check); i < k; ++i)
        if (hres[i] <= tol || hres[i] == 0.0) { kk = i + 1; break; }
      if (kk > 0) break;
    }
  }
  if (kk < 0) kk = maxit;
  launch_trisolve(ctx->H, ctx->ldh, ctx->gv, kk, ctx->ysol, st);
  launch_combine_basis(ctx->V, ctx->ysol, kk, n, x, st);
  CK(cudaGetLastError());
  *iters = kk;
  *relres = hres[kk - 1];
  if (hres[kk - 1] > tol && hres[kk - 1] != 0.0)
    return fail(ctx, DDST_ERR_NOT_CONVERGED, "GMRES: relative residual %.3e after %d iterations",
                hres[kk - 1], kk);
  return DDST_OK;
}

// GMRES on the whole interface system: one Krylov space, or one per operator group in a
// grouped context (the groups never couple).  Iterations and residual: the larger over groups.
template <typename T>
ddst_status gmres_impl(ddst_ctx* ctx, const double* rhs, double* x, double tol, int transpose,
                       int* iters, double* relres) {
  if (!ctx->grouped) return gmres_range<T>(ctx, rhs, x, tol, transpose, -1, iters, relres);
  *iters = 0;
  *relres = 0.0;
  ddst_status worst = DDST_OK;
  for (int g = 0; g < 2; ++g) {
    if (ctx->grp_n[g] == 0) continue;
    int it = 0;
    double rr = 0.0;
    const ddst_status s = gmres_range<T>(ctx, rhs + ctx->grp_off[g], x + ctx->grp_off[g], tol,
                                         transpose, g, &it, &rr);
    if (s != DDST_OK && s != DDST_ERR_NOT_CONVERGED) return s;
    if (s != DDST_OK) worst = s;
    *iters = std::max(*iters, it);
    *relres = std::max(*relres, rr);
  }
  if (worst != DDST_OK)
    return fail(ctx, worst, "GMRES: relative residual %.3e after %d iterations", *relres, *iters);
  return DDST_OK;
}

// A-posteriori error of a contracting fixed-point iteration: if every step reduces the error by
// a factor rho < 1, the error after applying the correction delta_k is at most
// rho / (1 - rho) ||delta_k||.  rho is estimated by the larger of the last two ratios
// ||delta_k|| / ||delta_{k-1}|| and used as observed: a slow contraction (rho near 1) enlarges
// the bound accordingly, and rho >= 1 (no contraction seen) gives no bound at all (infinity),
// unless the correction itself is at the FP64 rounding level of the residual (relative size below
// 1e-14), where the corrections are rounding noise and their size is the only error measure left.
// The first correction (from zero) has no estimate and counts in full.  After two corrections the
// one ratio seen is that of the first DD solve on the whole right-hand side, which resolves it
// better than later solves resolve the residual (that residual lies where the inner GMRES and the
// low-precision factors are weakest), so it underestimates the later contraction: the bound is
// then the last correction itself (rho taken as at least 1/2).  Returns the bound relative to
// ||x|| given the correction norms so far (hist) and ||x||.
double refine_error_estimate(const std::vector<double>& hist, double xn) {
  const size_t k = hist.size();
  if (k == 0 || !(xn > 0.0)) return 0.0;
  const double rel = hist[k - 1] / xn;
  if (k < 2) return rel;
  double rho = hist[k - 2] > 0.0 ? hist[k - 1] / hist[k - 2] : 1.0;
  if (k >= 3 && hist[k - 3] > 0.0) rho = std::max(rho, hist[k - 2] / hist[k - 3]);
  if (rel <= 1e-14) return rel;
  if (!(rho < 1.0)) return HUGE_VAL;
  if (k == 2) rho = std::max(rho, 0.5);
  return rel * rho / (1.0 - rho);
}

// One refinement step's bookkeeping for a batch: appends each problem's correction norm
// ||e_q|| to hist[q] and returns the largest of the problems' bounds, each relative to its own
// ||x_q||.  A bound over the concatenated batch would let a problem with a small solution hide
// behind one with a large solution (the interface GMRES also stops on the batch's residual), so
// the stopping test holds problem by problem.  One host synchronisation.
double refine_batch_estimate(ddst_ctx* ctx, const double* e, const double* x,
                             std::vector<std::vector<double>>& hist, double* rho) {
  const int np = ctx->nprob;
  cudaStream_t st = ctx->stream;
  const int nb = norm_blocks(np);
  launch_prob_sqnorms(ctx->d_probs, np, e, ctx->pn_part, nb, ctx->pn, st);
  launch_prob_sqnorms(ctx->d_probs, np, x, ctx->pn_part + (size_t)np * nb, nb, ctx->pn + np, st);
  std::vector<double> h(2 * (size_t)np);
  cudaMemcpyAsync(h.data(), ctx->pn, sizeof(double) * 2 * np, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  hist.resize(np);
  double est = 0.0;
  for (int q = 0; q < np; ++q) {
    hist[q].push_back(std::sqrt(h[q]));
    const double xn = std::sqrt(h[np + q]);
    est = std::max(est, refine_error_estimate(hist[q], xn));
    const size_t k = hist[q].size();  // observed contraction, rounding-level corrections aside
    if (k >= 2 && hist[q][k - 2] > 0.0 && xn > 0.0 && hist[q][k - 1] > 1e-14 * xn)
      *rho = std::max(*rho, hist[q][k - 1] / hist[q][k - 2]);
  }
  return est;
}

// One application of the DD solve map (Alg. 2 + GMRES + reconstruction):
// rhs volume vector r (FP64) -> volume correction e (FP64); traces written into ctx->if_u.
template <typename T>
ddst_status dd_apply(ddst_ctx* ctx, const double* r, double* e, int* iters, double* relres,
                     double tol) {
  cudaStream_t st = ctx->stream;
  const int nslab = (int)ctx->slabs.size();
  T* lb = (T*)ctx->loc_b;
  // equivalent loads fhat_j = R_C A_j^{-1} r|Psi_j  (Sec. 2.2, Eq. (equilib1))
  launch_gather<T>(ctx->d_slabs, nslab, r, lb, st);
  local_solves<T>(ctx, lb, (T*)ctx->loc_bf, (T*)ctx->loc_bb, (T*)ctx->loc_x, ctx->if_fh, 0, 1, st);
  CK(cudaGetLastError());
  // interface solve (I - K) u_Gamma = fhat: GMRES, or the block cyclic reduction
  ddst_status s;
  if (ctx->opt.interface_solver == 1) {
    s = direct_interface_solve<T>(ctx, ctx->if_fh, ctx->if_u, 0);
    *iters = 0;
    *relres = 0.0;
  } else {
    s = gmres_impl<T>(ctx, ctx->if_fh, ctx->if_u, tol, 0, iters, relres);
  }
  if (s != DDST_OK && s != DDST_ERR_NOT_CONVERGED) return s;
  // volume reconstruction: local Dirichlet solves with the traces on Gamma_{j-1}, Gamma_{j+1}
  launch_add_iface_dirichlet<T>(ctx->d_slabs, ctx->d_probs, nslab, (T*)ctx->pack, ctx->if_u, lb, st);
  local_solves<T>(ctx, lb, (T*)ctx->loc_bf, (T*)ctx->loc_bb, (T*)ctx->loc_x, nullptr, 0, 0, st);
  launch_scatter<T>(ctx->d_slabs, ctx->d_probs, nslab, (T*)ctx->loc_x, e, 0, st);
  CK(cudaGetLastError());
  return s;
}

double vec_norm(ddst_ctx* ctx, const double* x, int64_t n, int slot) {
  launch_dot(x, x, n, ctx->part, 256, ctx->scal + slot, ctx->stream);
  return std::sqrt(host_scalar(ctx, ctx->scal + slot));
}

// Result of one forward solve on the device-resident d_f, d_g (solution in d_u).
struct SolveStats {
  int total_it = 0, first_it = 0, nref = 0;
  double est = 0.0, relres = 0.0, rho = 0.0;
  ddst_status result = DDST_OK;
};

// The forward solve on the staged data: right-hand side b(f, g), DD solve, FP64 refinement
// until every problem's error bound is below refine_tol (Alg. 2, Eq. (equilib1), Eq. (modelS)).
// x0 = 0 (warm = false) or the current d_u (warm = true: the refinement then starts from it).
template <typename T>
ddst_status solve_core(ddst_ctx* ctx, bool warm, SolveStats* ss) {
  cudaStream_t st = ctx->stream;
  ddst_status s;
  const int64_t N = ctx->tot_vol;
  launch_rhs(ctx->d_probs, ctx->nprob, ctx->d_a, ctx->d_f, ctx->d_g, ctx->d_b, st);
  if (!warm) CK(cudaMemsetAsync(ctx->d_u, 0, sizeof(double) * N, st));
  const double bnorm = vec_norm(ctx, ctx->d_b, N, 3);
  const double tol = ctx->opt.gmres_tol;
  std::vector<std::vector<double>> dnorm;
  const int rmax = std::max(0, ctx->opt.refine_max);
  for (int it = 0; it <= rmax; ++it) {
    const double* rhs = ctx->d_b;
    if (it > 0 || warm) {
      launch_residual(ctx->d_probs, ctx->nprob, ctx->d_a, ctx->d_c, ctx->d_b, ctx->d_u, ctx->d_r, 0,
                      nullptr, 512, st);
      rhs = ctx->d_r;
    }
    int its = 0;
    double rr = 0.0;
    s = dd_apply<T>(ctx, rhs, ctx->d_e, &its, &rr, tol);
    if (s != DDST_OK && s != DDST_ERR_NOT_CONVERGED) return s;
    if (it == 0) ss->first_it = its;
    ss->total_it += its;
    ++ss->nref;
    launch_axpy(N, 1.0, ctx->d_e, ctx->d_u, st);
    ss->est = refine_batch_estimate(ctx, ctx->d_e, ctx->d_u, dnorm, &ss->rho);
    if (rmax == 0) {  // plain DD solve: its accuracy is the interface GMRES's
      if (s == DDST_ERR_NOT_CONVERGED) ss->result = s;
      break;
    }
    if (ss->est <= ctx->opt.refine_tol) break;
    if (it == rmax) ss->result = DDST_ERR_NOT_CONVERGED;
  }
  launch_residual(ctx->d_probs, ctx->nprob, ctx->d_a, ctx->d_c, ctx->d_b, ctx->d_u, ctx->d_r, 0,
                  nullptr, 512, st);
  ss->relres = bnorm > 0.0 ? vec_norm(ctx, ctx->d_r, N, 6) / bnorm : 0.0;
  return DDST_OK;
}

void fill_info(ddst_ctx* ctx, const SolveStats& ss, float ms, ddst_info* info) {
  if (!info) return;
  info->gmres_iters = ss.total_it;
  info->gmres_iters_first = ss.first_it;
  info->refine_iters = ss.nref;
  info->rel_residual = ss.relres;
  info->est_rel_error = ss.est;
  info->refine_rho = ss.rho;
  info->t_direct = ctx->t_bcr;
  info->t_factor = ctx->t_factor;
  info->t_transfer = ctx->t_transfer;
  info->t_compress = ctx->t_compress;
  info->t_solve = ms;
  info->bytes_factors = (int64_t)((5 + (ctx->use_tc ? 4 : 0)) * ctx->fac_elems +
                                  ctx->fac_big_elems + ctx->pack_elems) * (int64_t)ctx->esz;
  info->bytes_transfer = ctx->matfree ? 0
                         : ctx->state == 3 ? ctx->hodlr.bytes
                         : ctx->state == 4 ? ctx->hbs.bytes : ctx->s_elems * (int64_t)ctx->esz;
  info->max_rank = ctx->state == 3 ? ctx->hodlr.max_rank : ctx->state == 4 ? ctx->hbs.k : 0;
  info->fail_slab = -1;
  info->fail_block = -1;
  info->factor_chunks = ctx->factor_chunks;
  info->factor_check = ctx->factor_check;
}

template <typename T>
ddst_status solve_impl(ddst_ctx* ctx, const double* const* f, const double* const* g,
                       double* const* u, ddst_info* info) {
  cudaStream_t st = ctx->stream;
  ddst_status s = ensure_solve_buffers(ctx);
  if (s != DDST_OK) return s;
  Timer tfac(st);
  s = ensure_factors<T>(ctx);
  if (s != DDST_OK) return s;
  const float recompute_ms = tfac.stop();
  for (int q = 0; q < ctx->nprob; ++q) {
    const ProbDesc& P = ctx->probs[q];
    if (!f[q] || !g[q] || !u[q]) return fail(ctx, DDST_ERR_INVALID_ARG, "NULL array for problem %d", q);
    CK(stage_in(ctx->d_f + P.vol_off, f[q], P.nint, st));
    CK(stage_in(ctx->d_g + P.node_off, g[q], P.nnode, st));
  }
  Timer tm(st);
  SolveStats ss;
  s = solve_core<T>(ctx, false, &ss);
  if (s != DDST_OK) return s;
  const float ms = tm.stop();
  for (int q = 0; q < ctx->nprob; ++q) {
    const ProbDesc& P = ctx->probs[q];
    CK(stage_out(u[q], ctx->d_u + P.vol_off, P.nint, st));
  }
  CK(cudaStreamSynchronize(st));
  ddst_status ds = check_status(ctx, info);
  if (ds != DDST_OK) return ds;
  ctx->have_solution = true;
  fill_info(ctx, ss, ms + recompute_ms, info);
  maybe_release_factors(ctx);
  if (ss.result != DDST_OK)
    return fail(ctx, ss.result, "refinement stopped at estimated relative error %.3e", ss.est);
  return DDST_OK;
}

// IMEX backward-Euler marching (Sec. 6, Example 1, Eq. (convdiff)): every step solves the
// context's operator (the caller sets it up with reaction c = 1/dt) for the right-hand side
// f = U_n / dt - v . grad_h U_n (central differences, U_n = 0 on the boundary) with zero Dirichlet
// data, reusing the factors, the transfer operators and (interface_solver = 1) the factored
// equilibrium system.  The refinement of step n + 1 starts from U_n.
template <typename T>
ddst_status march_impl(ddst_ctx* ctx, int nsteps, double dt, const double* const* vel,
                       const double* const* u0, double* const* u, ddst_info* info) {
  cudaStream_t st = ctx->stream;
  ddst_status s = ensure_solve_buffers(ctx);
  if (s != DDST_OK) return s;
  s = ensure_factors<T>(ctx);
  if (s != DDST_OK) return s;
  if (!ctx->d_vel) {  // component-major: component d of every problem's nodes at d tot_nodes
    cudaError_t e = dalloc(ctx, &ctx->d_vel, sizeof(double) * 3 * ctx->tot_nodes);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMalloc velocity");
  }
  for (int q = 0; q < ctx->nprob; ++q) {
    const ProbDesc& P = ctx->probs[q];
    if (!vel[q] || !u0[q] || !u[q]) return fail(ctx, DDST_ERR_INVALID_ARG, "NULL array for problem %d", q);
    for (int d = 0; d < P.dim; ++d)
      CK(stage_in(ctx->d_vel + d * ctx->tot_nodes + P.node_off, vel[q] + (int64_t)d * P.nnode,
                  P.nnode, st));
    CK(stage_in(ctx->d_u + P.vol_off, u0[q], P.nint, st));
  }
  CK(cudaMemsetAsync(ctx->d_g, 0, sizeof(double) * ctx->tot_nodes, st));
  Timer tm(st);
  SolveStats tot;
  for (int n = 0; n < nsteps; ++n) {
    launch_imex_rhs(ctx->d_probs, ctx->nprob, ctx->d_u, ctx->d_vel, ctx->tot_nodes, 1.0 / dt,
                    ctx->d_f, st);
    SolveStats ss;
    s = solve_core<T>(ctx, true, &ss);
    if (s != DDST_OK) return s;
    tot.total_it += ss.total_it;
    tot.nref += ss.nref;
    if (n == 0) tot.first_it = ss.first_it;
    tot.est = std::max(tot.est, ss.est);
    tot.rho = std::max(tot.rho, ss.rho);
    tot.relres = std::max(tot.relres, ss.relres);
    if (ss.result != DDST_OK) { tot.result = ss.result; break; }
  }
  const float ms = tm.stop();
  for (int q = 0; q < ctx->nprob; ++q) {
    const ProbDesc& P = ctx->probs[q];
    CK(stage_out(u[q], ctx->d_u + P.vol_off, P.nint, st));
  }
  CK(cudaStreamSynchronize(st));
  ddst_status ds = check_status(ctx, info);
  if (ds != DDST_OK) return ds;
  fill_info(ctx, tot, ms, info);
  maybe_release_factors(ctx);
  if (tot.result != DDST_OK)
    return fail(ctx, tot.result, "a step's refinement stopped at estimated relative error %.3e",
                tot.est);
  return DDST_OK;
}


// Transposed DD map e = M^T r, where M is the forward DD solve map (dd_apply):
//   M = P A^{-1} G - P A^{-1} D (I - K)^{-1} R A^{-1} G
//   M^T r = G^T A^{-T} (P^T r + R^T mu),  mu = -(I - K)^{-T} D^T A^{-T} P^T r
// (G: slab gather, P: owned-plane scatter, R: central rows, D: Dirichlet data of the
// neighbouring interfaces).  Transposed local solves run through the same factors.
template <typename T>
ddst_status dd_apply_T(ddst_ctx* ctx, const double* r, double* e, int* iters, double* relres,
                       double tol) {
  cudaStream_t st = ctx->stream;
  const int nslab = (int)ctx->slabs.size();
  T* lb = (T*)ctx->loc_b;
  launch_gather_owned<T>(ctx->d_slabs, ctx->d_probs, nslab, r, lb, st);
  local_solves<T>(ctx, lb, (T*)ctx->loc_bf, (T*)ctx->loc_bb, (T*)ctx->loc_x, nullptr, 1, 0, st);
  CK(cudaMemsetAsync(ctx->if_fh, 0, sizeof(double) * ctx->tot_if, st));
  launch_iface_dirichlet_T<T>(ctx->d_slabs, ctx->d_probs, nslab, (T*)ctx->pack, (T*)ctx->loc_x,
                              ctx->if_fh, st);
  CK(cudaGetLastError());
  ddst_status s;
  if (ctx->opt.interface_solver == 1) {
    s = direct_interface_solve<T>(ctx, ctx->if_fh, ctx->if_u, 1);
    *iters = 0;
    *relres = 0.0;
  } else {
    s = gmres_impl<T>(ctx, ctx->if_fh, ctx->if_u, tol, 1, iters, relres);
  }
  if (s != DDST_OK && s != DDST_ERR_NOT_CONVERGED) return s;
  launch_inject_center<T>(ctx->d_slabs, nslab, ctx->if_u, lb, st);
  local_solves<T>(ctx, lb, (T*)ctx->loc_bf, (T*)ctx->loc_bb, (T*)ctx->loc_x, nullptr, 1, 0, st);
  CK(cudaMemsetAsync(e, 0, sizeof(double) * ctx->tot_vol, st));
  launch_gather_T<T>(ctx->d_slabs, nslab, (T*)ctx->loc_x, e, st);
  CK(cudaGetLastError());
  return s;
}

template <typename T>
ddst_status solve_adjoint_impl(ddst_ctx* ctx, const double* const* dLdu, double* const* dLdf,
                               double* const* dLdg, double* const* dLda, ddst_info* info) {
  cudaStream_t st = ctx->stream;
  const int64_t N = ctx->tot_vol;
  Timer tfac(st);
  ddst_status sf = ensure_factors<T>(ctx);
  if (sf != DDST_OK) return sf;
  const float recompute_ms = tfac.stop();
  for (int q = 0; q < ctx->nprob; ++q) {
    const ProbDesc& P = ctx->probs[q];
    if (!dLdu[q]) return fail(ctx, DDST_ERR_INVALID_ARG, "dL/du is NULL for problem %d", q);
    CK(stage_in(ctx->d_ga + P.vol_off, dLdu[q], P.nint, st));
  }
  Timer tm(st);
  CK(cudaMemsetAsync(ctx->d_lam, 0, sizeof(double) * N, st));
  const double gnorm = vec_norm(ctx, ctx->d_ga, N, 3);
  int total_it = 0, first_it = 0, nref = 0;
  double est = 0.0, rho = 0.0;
  std::vector<std::vector<double>> dnorm;
  ddst_status result = DDST_OK, s;
  const int rmax = std::max(0, ctx->opt.refine_max);
  for (int it = 0; it <= rmax; ++it) {
    const double* rhs = ctx->d_ga;
    if (it > 0) {
      launch_residual(ctx->d_probs, ctx->nprob, ctx->d_a, ctx->d_c, ctx->d_ga, ctx->d_lam,
                      ctx->d_r, 1, nullptr, 512, st);
      rhs = ctx->d_r;
    }
    int its = 0;
    double rr = 0.0;
    s = dd_apply_T<T>(ctx, rhs, ctx->d_e, &its, &rr, ctx->opt.gmres_tol);
    if (s != DDST_OK && s != DDST_ERR_NOT_CONVERGED) return s;
    if (it == 0) first_it = its;
    total_it += its;
    ++nref;
    launch_axpy(N, 1.0, ctx->d_e, ctx->d_lam, st);
    est = refine_batch_estimate(ctx, ctx->d_e, ctx->d_lam, dnorm, &rho);
    if (rmax == 0) {
      if (s == DDST_ERR_NOT_CONVERGED) result = s;
      break;
    }
    if (est <= ctx->opt.refine_tol) break;
    if (it == rmax) result = DDST_ERR_NOT_CONVERGED;
  }
  launch_residual(ctx->d_probs, ctx->nprob, ctx->d_a, ctx->d_c, ctx->d_ga, ctx->d_lam, ctx->d_r, 1,
                  nullptr, 512, st);
  const double relres = gnorm > 0.0 ? vec_norm(ctx, ctx->d_r, N, 6) / gnorm : 0.0;
  CK(cudaMemsetAsync(ctx->d_gn, 0, sizeof(double) * ctx->tot_nodes, st));
  CK(cudaMemsetAsync(ctx->d_an, 0, sizeof(double) * ctx->tot_nodes, st));
  launch_gradients(ctx->d_probs, ctx->nprob, ctx->d_a, ctx->d_g, ctx->d_u, ctx->d_lam, ctx->d_gn,
                   ctx->d_an, st);
  CK(cudaGetLastError());
  const float ms = tm.stop();
  for (int q = 0; q < ctx->nprob; ++q) {
    const ProbDesc& P = ctx->probs[q];
    if (dLdf && dLdf[q]) CK(stage_out(dLdf[q], ctx->d_lam + P.vol_off, P.nint, st));
    if (dLdg && dLdg[q]) CK(stage_out(dLdg[q], ctx->d_gn + P.node_off, P.nnode, st));
    if (dLda && dLda[q]) CK(stage_out(dLda[q], ctx->d_an + P.node_off, P.nnode, st));
  }
  CK(cudaStreamSynchronize(st));
  ddst_status ds = check_status(ctx, info);
  if (ds != DDST_OK) return ds;
  if (info) {
    info->gmres_iters = total_it;
    info->gmres_iters_first = first_it;
    info->refine_iters = nref;
    info->rel_residual = relres;
    info->est_rel_error = est;
    info->refine_rho = rho;
    info->t_direct = ctx->t_bcr;
    info->t_solve = ms;
    info->t_factor = ctx->t_factor;
    info->t_transfer = ctx->t_transfer;
    info->t_compress = ctx->t_compress;
    info->max_rank = ctx->state == 3 ? ctx->hodlr.max_rank : ctx->state == 4 ? ctx->hbs.k : 0;
    info->fail_slab = info->fail_block = -1;
  }
  if (info) info->t_solve += recompute_ms;
  maybe_release_factors(ctx);
  if (result != DDST_OK)
    return fail(ctx, result, "adjoint refinement stopped at estimated relative error %.3e", est);
  return DDST_OK;
}

// DDST_AUTO: the FP32 factorization first; if one of its pivots falls below the FP32 floor
// (an indefinite local operator whose leading block minors pass near zero), the FP64
// factorization, whose floor is nine orders of magnitude lower.  Other errors return as they are.
ddst_status setup_precision(int nprob, const ddst_grid* grids, const ddst_coeffs* coeffs,
                            const int* widths, const ddst_options* opt, void* stream,
                            ddst_ctx** out) {
  ddst_options o;
  if (opt) o = *opt; else ddst_options_default(&o);
  if (o.precision != DDST_FP64 && o.precision != DDST_MIXED && o.precision != DDST_AUTO &&
      o.precision != DDST_MIXED_TF32) {
    if (out) *out = nullptr;
    return fail(nullptr, DDST_ERR_INVALID_ARG,
                "precision must be DDST_FP64, DDST_MIXED, DDST_MIXED_TF32 or DDST_AUTO");
  }
  if (o.autotune_cache && *o.autotune_cache) {  // tuned knobs for this device and these shapes
    char key[8192];
    int found = 0;
    if (ddst_autotune_key(nprob, grids, coeffs, widths, o.precision, key, sizeof(key)) == DDST_OK)
      ddst_autotune_lookup(o.autotune_cache, key, &o, &found);
  }
  if (o.precision != DDST_AUTO) return setup_impl(nprob, grids, coeffs, widths, &o, stream, out);
  o.precision = DDST_MIXED;
  const ddst_status s = setup_impl(nprob, grids, coeffs, widths, &o, stream, out);
  if (s != DDST_ERR_SINGULAR) return s;
  const std::string first = g_setup_error;
  o.precision = DDST_FP64;
  const ddst_status s2 = setup_impl(nprob, grids, coeffs, widths, &o, stream, out);
  if (s2 == DDST_ERR_INVALID_ARG) {  // blocks too large for the FP64 kernels: report the pivot
    g_setup_error = first;
    return s;
  }
  return s2;
}

}  // namespace

// ============================================================================================
// C ABI
// ============================================================================================
extern "C" {

void ddst_options_default(ddst_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->precision = DDST_MIXED;
  opt->gmres_tol = 0.0;  // automatic (see the header)
  opt->gmres_max_iter = 1000;
  opt->refine_tol = 1e-9;
  opt->refine_max = 8;
  opt->k_max = 64;
  opt->oversample = 10;
  opt->leaf_size = 128;
  opt->seed = 1234;
  opt->check_every = 0;
  opt->factor_chunks = 0;
  opt->factor_warmup = 0;
  opt->tensor_cores = -1;
  opt->explicit_S = -1;
  opt->recompute_factors = 0;
  opt->autotune_cache = nullptr;
  opt->interface_solver = -1;
}

ddst_status ddst_setup(const ddst_grid* grid, const ddst_coeffs* coeffs, int slab_width,
                       const ddst_options* opt, void* stream, ddst_ctx** out) {
  return setup_precision(1, grid, coeffs, &slab_width, opt, stream, out);
}

ddst_status ddst_setup_batch(int nprob, const ddst_grid* grids, const ddst_coeffs* coeffs,
                             const int* slab_widths, const ddst_options* opt, void* stream,
                             ddst_ctx** out) {
  return setup_precision(nprob, grids, coeffs, slab_widths, opt, stream, out);
}

ddst_status ddst_get_precision(const ddst_ctx* ctx, int* precision) {
  if (!ctx || !precision) return fail(nullptr, DDST_ERR_INVALID_ARG, "ctx or precision is NULL");
  *precision = ctx->tf32 ? DDST_MIXED_TF32 : ctx->prec;
  return DDST_OK;
}

ddst_status ddst_get_options(const ddst_ctx* ctx, ddst_options* opt) {
  if (!ctx || !opt) return fail(nullptr, DDST_ERR_INVALID_ARG, "ctx or opt is NULL");
  *opt = ctx->opt;
  opt->precision = ctx->tf32 ? DDST_MIXED_TF32 : ctx->prec;
  if (opt->tensor_cores < 0) opt->tensor_cores = 1;
  if (opt->check_every == 0) opt->check_every = ctx->mf_any ? 1 : 8;
  if (opt->interface_solver < 0) opt->interface_solver = 0;
  opt->autotune_cache = nullptr;  // read during setup only
  return DDST_OK;
}

ddst_status ddst_build_transfer(ddst_ctx* ctx) {
  if (!ctx) return fail(nullptr, DDST_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->state < 1) return fail(ctx, DDST_ERR_STATE, "ddst_setup has not completed");
  ddst_status s = ctx->prec == DDST_FP64 ? ensure_factors<double>(ctx) : ensure_factors<float>(ctx);
  if (s != DDST_OK) return s;
  s = ctx->prec == DDST_FP64 ? build_transfer_impl<double>(ctx) : build_transfer_impl<float>(ctx);
  if (s == DDST_OK) maybe_release_factors(ctx);
  return s;
}

ddst_status ddst_compress(ddst_ctx* ctx, double tol) {
  if (!ctx) return fail(nullptr, DDST_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->state < 2) return fail(ctx, DDST_ERR_STATE, "ddst_build_transfer has not completed");
  if (ctx->matfree && tol > 0.0)
    return fail(ctx, DDST_ERR_NOT_IMPLEMENTED,
                "compression samples the explicit transfer operators; this context applies them "
                "matrix-free (explicit_S = 0, or blocks larger than 128)");
  drop_graphs(ctx);
  ctx->hbs.release();
  if (!(tol > 0.0)) {
    ctx->hodlr.clear();
    ctx->state = 2;
    return DDST_OK;
  }
  Timer tm(ctx->stream);
  HodlrParams hp{tol, ctx->opt.k_max, ctx->opt.oversample, ctx->opt.leaf_size, ctx->opt.seed};
  std::string msg;
  int rc = ctx->prec == DDST_FP64
               ? hodlr_build<double>(ctx->hodlr, hp, ctx->slabs, ctx->probs, ctx->d_slabs,
                                     (const double*)ctx->S, ctx->stream, msg)
               : hodlr_build<float>(ctx->hodlr, hp, ctx->slabs, ctx->probs, ctx->d_slabs,
                                    (const float*)ctx->S, ctx->stream, msg);
  ctx->t_compress = tm.stop();
  if (rc != 0)
    return fail(ctx, rc == 2 ? DDST_ERR_OOM : rc == 3 ? DDST_ERR_INVALID_ARG : DDST_ERR_CUDA,
                "compress: %s", msg.c_str());
  ctx->state = 3;
  return DDST_OK;
}

ddst_status ddst_compress_hbs(ddst_ctx* ctx, int rank, int oversample) {
  if (!ctx) return fail(nullptr, DDST_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->state < 2) return fail(ctx, DDST_ERR_STATE, "ddst_build_transfer has not completed");
  if (ctx->matfree || ctx->mf_any)
    return fail(ctx, DDST_ERR_NOT_IMPLEMENTED,
                "HBS compression samples the explicit transfer operators; this context applies "
                "some of them matrix-free");
  if (rank < 1 || rank > 32 || oversample < 0 || 3 * rank + oversample > 96)
    return fail(ctx, DDST_ERR_INVALID_ARG,
                "rank %d, oversample %d: need 1 <= rank <= 32 and 3 rank + oversample <= 96", rank,
                oversample);
  drop_graphs(ctx);
  ctx->hodlr.clear();
  ctx->hbs.release();
  ctx->state = 2;
  std::vector<HbsInput> in;
  for (size_t si = 0; si < ctx->slabs.size(); ++si) {
    const SlabDesc& s = ctx->slabs[si];
    const ProbDesc& P = ctx->probs[s.prob];
    for (int side = -1; side <= 1; side += 2) {
      const int64_t off = side < 0 ? s.sp_off : s.sn_off;
      if (off < 0) continue;
      in.push_back(HbsInput{(const char*)ctx->S + off * (int64_t)ctx->esz, P.ng, nullptr, nullptr,
                            s.if_off + side * P.ng, s.if_off, (int)si, side});
    }
  }
  std::vector<std::pair<int64_t, int64_t>> bare;  // a single interface: K = 0 there
  for (int q = 0; q < ctx->nprob; ++q)
    if (ctx->probs[q].nds == 1) bare.push_back({ctx->probs[q].if_off, ctx->probs[q].ng});
  Timer tm(ctx->stream);
  std::string msg;
  const int s = 3 * rank + oversample;
  int rc = in.empty() ? 0
           : ctx->prec == DDST_FP64
               ? hbs_build<double>(ctx->hbs, in, bare, rank, s, 2 * rank, ctx->opt.seed, ctx->stream, msg)
               : hbs_build<float>(ctx->hbs, in, bare, rank, s, 2 * rank, ctx->opt.seed, ctx->stream, msg);
  ctx->t_compress = tm.stop();
  if (rc != 0)
    return fail(ctx, rc == 2 ? DDST_ERR_OOM : rc == 3 ? DDST_ERR_INVALID_ARG : DDST_ERR_CUDA,
                "compress_hbs: %s", msg.c_str());
  if (in.empty()) return fail(ctx, DDST_ERR_INVALID_ARG, "compress_hbs: no transfer operators");
  ctx->state = 4;
  return DDST_OK;
}

ddst_status ddst_hbs_create(const double* S, int64_t ng, int rank, int nsamples, int leaf,
                            const double* omega, const double* psi, int precision,
                            ddst_hbs** out) {
  if (!out) return fail(nullptr, DDST_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!S || ng < 1) return fail(nullptr, DDST_ERR_INVALID_ARG, "S is NULL or ng < 1");
  if ((omega == nullptr) != (psi == nullptr))
    return fail(nullptr, DDST_ERR_INVALID_ARG, "omega and psi are both given or both NULL");
  if (precision != DDST_FP64 && precision != DDST_MIXED)
    return fail(nullptr, DDST_ERR_INVALID_ARG, "precision must be DDST_FP64 or DDST_MIXED");
  if (is_device_ptr(S) || (omega && (is_device_ptr(omega) || is_device_ptr(psi))))
    return fail(nullptr, DDST_ERR_INVALID_ARG, "S, omega and psi are host arrays");
  ddst_hbs* h = new ddst_hbs();
  h->prec = precision;
  h->ng = ng;
  const size_t esz = precision == DDST_FP64 ? 8 : 4;
  const size_t nbytes = esz * (size_t)(ng * ng);
  cudaError_t e = cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&h->S, nbytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->x, sizeof(double) * ng);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->y, sizeof(double) * ng);
  if (e != cudaSuccess) {
    ddst_hbs_destroy(h);
    return fail(nullptr, e == cudaErrorMemoryAllocation ? DDST_ERR_OOM : DDST_ERR_CUDA, "%s",
                cudaGetErrorString(e));
  }
  // row-major FP64 input -> column-major working precision
  std::vector<double> cm64;
  std::vector<float> cm32;
  if (esz == 8) cm64.resize((size_t)(ng * ng)); else cm32.resize((size_t)(ng * ng));
  for (int64_t r = 0; r < ng; ++r)
    for (int64_t c = 0; c < ng; ++c) {
      const double v = S[r * ng + c];
      if (esz == 8) cm64[c * ng + r] = v; else cm32[c * ng + r] = (float)v;
    }
  e = cudaMemcpyAsync(h->S, esz == 8 ? (const void*)cm64.data() : (const void*)cm32.data(), nbytes,
                      cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) {
    ddst_hbs_destroy(h);
    return fail(nullptr, DDST_ERR_CUDA, "%s", cudaGetErrorString(e));
  }
  std::vector<HbsInput> in{HbsInput{h->S, ng, omega, psi, 0, 0, 0, 0}};
  std::string msg;
  const int rc = esz == 8
                     ? hbs_build<double>(h->H, in, {}, rank, nsamples, leaf, 1234, h->st, msg)
                     : hbs_build<float>(h->H, in, {}, rank, nsamples, leaf, 1234, h->st, msg);
  if (rc != 0) {
    ddst_hbs_destroy(h);
    return fail(nullptr, rc == 2 ? DDST_ERR_OOM : rc == 3 ? DDST_ERR_INVALID_ARG : DDST_ERR_CUDA,
                "hbs_create: %s", msg.c_str());
  }
  *out = h;
  return DDST_OK;
}

ddst_status ddst_hbs_apply(ddst_hbs* h, const double* x, double* y, int transpose) {
  if (!h || !x || !y) return fail(nullptr, DDST_ERR_INVALID_ARG, "NULL argument");
  const size_t nb = sizeof(double) * (size_t)h->ng;
  const bool dx = is_device_ptr(x), dy = is_device_ptr(y);
  cudaError_t e = cudaMemcpyAsync(h->x, x, nb, dx ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  h->st);
  if (e != cudaSuccess) return fail(nullptr, DDST_ERR_CUDA, "%s", cudaGetErrorString(e));
  if (h->prec == DDST_FP64)
    hbs_apply<double>(h->H, h->x, h->y, (transpose ? 1 : 0) | 2, h->st);
  else
    hbs_apply<float>(h->H, h->x, h->y, (transpose ? 1 : 0) | 2, h->st);
  e = cudaMemcpyAsync(y, h->y, nb, dy ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, DDST_ERR_CUDA, "%s", cudaGetErrorString(e));
  return DDST_OK;
}

ddst_status ddst_hbs_expand(ddst_hbs* h, double* out) {
  if (!h || !out) return fail(nullptr, DDST_ERR_INVALID_ARG, "NULL argument");
  if (is_device_ptr(out)) return fail(nullptr, DDST_ERR_INVALID_ARG, "out is a host array");
  const int64_t ng = h->ng;
  std::vector<double> cm((size_t)(ng * ng));
  if (hbs_expand(h->H, 0, cm.data(), h->st)) return fail(nullptr, DDST_ERR_CUDA, "expand failed");
  for (int64_t c = 0; c < ng; ++c)
    for (int64_t r = 0; r < ng; ++r) out[r * ng + c] = cm[c * ng + r];
  return DDST_OK;
}

ddst_status ddst_hbs_stats(const ddst_hbs* h, int* levels, int64_t* entries) {
  if (!h) return fail(nullptr, DDST_ERR_INVALID_ARG, "NULL handle");
  if (levels) *levels = h->H.blocks.empty() ? 0 : h->H.blocks[0].L;
  if (entries) *entries = h->H.f_elems;
  return DDST_OK;
}

void ddst_hbs_destroy(ddst_hbs* h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  h->H.release();
  for (void* p : {h->S, (void*)h->x, (void*)h->y})
    if (p) cudaFree(p);
  if (h->st) cudaStreamDestroy(h->st);
  delete h;
}

ddst_status ddst_solve_batch(ddst_ctx* ctx, const double* const* f, const double* const* g,
                             double* const* u, ddst_info* info) {
  if (!ctx) return fail(nullptr, DDST_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->state < 2) return fail(ctx, DDST_ERR_STATE, "transfer operators not built");
  if (!f || !g || !u) return fail(ctx, DDST_ERR_INVALID_ARG, "NULL pointer array");
  if (info) { memset(info, 0, sizeof(*info)); info->fail_slab = info->fail_block = -1; }
  return ctx->prec == DDST_FP64 ? solve_impl<double>(ctx, f, g, u, info)
                                : solve_impl<float>(ctx, f, g, u, info);
}

ddst_status ddst_march(ddst_ctx* ctx, int nsteps, double dt, const double* const* vel,
                       const double* const* u0, double* const* u, ddst_info* info) {
  if (!ctx) return fail(nullptr, DDST_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->state < 2) return fail(ctx, DDST_ERR_STATE, "transfer operators not built");
  if (nsteps < 0 || !(dt > 0.0)) return fail(ctx, DDST_ERR_INVALID_ARG, "need nsteps >= 0, dt > 0");
  if (!vel || !u0 || !u) return fail(ctx, DDST_ERR_INVALID_ARG, "NULL pointer array");
  if (info) { memset(info, 0, sizeof(*info)); info->fail_slab = info->fail_block = -1; }
  return ctx->prec == DDST_FP64 ? march_impl<double>(ctx, nsteps, dt, vel, u0, u, info)
                                : march_impl<float>(ctx, nsteps, dt, vel, u0, u, info);
}

ddst_status ddst_solve(ddst_ctx* ctx, const double* f, const double* g, double* u,
                       ddst_info* info) {
  if (ctx && ctx->nprob != 1) return fail(ctx, DDST_ERR_STATE, "batched context: use ddst_solve_batch");
  return ddst_solve_batch(ctx, &f, &g, &u, info);
}

ddst_status ddst_solve_adjoint_batch(ddst_ctx* ctx, const double* const* dL_du,
                                     double* const* dL_df, double* const* dL_dg,
                                     double* const* dL_da, ddst_info* info) {
  if (!ctx) return fail(nullptr, DDST_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->have_solution) return fail(ctx, DDST_ERR_STATE, "ddst_solve has not completed");
  if (!dL_du) return fail(ctx, DDST_ERR_INVALID_ARG, "dL/du array is NULL");
  if (info) { memset(info, 0, sizeof(*info)); info->fail_slab = info->fail_block = -1; }
  return ctx->prec == DDST_FP64 ? solve_adjoint_impl<double>(ctx, dL_du, dL_df, dL_dg, dL_da, info)
                                : solve_adjoint_impl<float>(ctx, dL_du, dL_df, dL_dg, dL_da, info);
}

ddst_status ddst_solve_adjoint(ddst_ctx* ctx, const double* dL_du, double* dL_df, double* dL_dg,
                               double* dL_da, ddst_info* info) {
  if (ctx && ctx->nprob != 1) return fail(ctx, DDST_ERR_STATE, "batched context: use ddst_solve_adjoint_batch");
  return ddst_solve_adjoint_batch(ctx, &dL_du, &dL_df, &dL_dg, &dL_da, info);
}

ddst_status ddst_interface_trace(ddst_ctx* ctx, int prob, double* uG) {
  if (!ctx) return fail(nullptr, DDST_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->have_solution) return fail(ctx, DDST_ERR_STATE, "no solution yet");
  if (prob < 0 || prob >= ctx->nprob || !uG) return fail(ctx, DDST_ERR_INVALID_ARG, "bad argument");
  const ProbDesc& P = ctx->probs[prob];
  // traces of the final solution: read Gamma_j planes of u
  std::vector<double> hu(P.nint);
  CK(cudaMemcpyAsync(hu.data(), ctx->d_u + P.vol_off, sizeof(double) * P.nint,
                     cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  std::vector<double> out((size_t)P.nds * P.ng);
  const int64_t plane = P.ng;
  for (int j = 1; j <= P.nds; ++j) {
    const int i = j * P.w;
    memcpy(&out[(size_t)(j - 1) * P.ng], &hu[(size_t)(i - 1) * plane], sizeof(double) * P.ng);
  }
  CK(cudaMemcpyAsync(uG, out.data(), sizeof(double) * out.size(),
                     is_device_ptr(uG) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return DDST_OK;
}

ddst_status ddst_get_transfer(ddst_ctx* ctx, int prob, int j, int side, double* out) {
  if (!ctx) return fail(nullptr, DDST_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->state < 2) return fail(ctx, DDST_ERR_STATE, "transfer operators not built");
  if (prob < 0 || prob >= ctx->nprob || !out || (side != -1 && side != 1))
    return fail(ctx, DDST_ERR_INVALID_ARG, "bad argument");
  const ProbDesc& P = ctx->probs[prob];
  if (j < 1 || j > P.nds) return fail(ctx, DDST_ERR_INVALID_ARG, "slab index out of range");
  if (ctx->mf_cls[P.M])
    return fail(ctx, DDST_ERR_NOT_IMPLEMENTED,
                "problem %d applies its transfer operators matrix-free: none is formed", prob);
  const SlabDesc& s = ctx->slabs[P.slab0 + j - 1];
  const int64_t off = side < 0 ? s.sp_off : s.sn_off;
  if (off < 0) return fail(ctx, DDST_ERR_INVALID_ARG, "slab %d has no neighbour on that side", j);
  const int64_t ng = P.ng;
  std::vector<double> cm((size_t)(ng * ng));
  if (ctx->state == 3) {
    int rc = hodlr_expand(ctx->hodlr, P.slab0 + j - 1, side, ctx->esz, cm.data(), ctx->stream);
    if (rc) return fail(ctx, DDST_ERR_CUDA, "expand failed");
  } else if (ctx->state == 4) {
    int b = -1;
    for (size_t q = 0; q < ctx->hbs.blk_slab.size(); ++q)
      if (ctx->hbs.blk_slab[q] == P.slab0 + j - 1 && ctx->hbs.blk_side[q] == side) b = (int)q;
    if (b < 0 || hbs_expand(ctx->hbs, b, cm.data(), ctx->stream))
      return fail(ctx, DDST_ERR_CUDA, "expand failed");
  } else if (ctx->esz == 8) {
    CK(cudaMemcpyAsync(cm.data(), (double*)ctx->S + off, sizeof(double) * ng * ng,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  } else {
    std::vector<float> tmp((size_t)(ng * ng));
    CK(cudaMemcpyAsync(tmp.data(), (float*)ctx->S + off, sizeof(float) * ng * ng,
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (size_t e = 0; e < tmp.size(); ++e) cm[e] = tmp[e];
  }
  std::vector<double> rm((size_t)(ng * ng));
  for (int64_t c = 0; c < ng; ++c)
    for (int64_t r = 0; r < ng; ++r) rm[r * ng + c] = cm[c * ng + r];
  CK(cudaMemcpyAsync(out, rm.data(), sizeof(double) * rm.size(),
                     is_device_ptr(out) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return DDST_OK;
}

ddst_status ddst_apply_interface(ddst_ctx* ctx, int prob, const double* x, double* y,
                                 int transpose) {
  if (!ctx) return fail(nullptr, DDST_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->state < 2) return fail(ctx, DDST_ERR_STATE, "transfer operators not built");
  if (prob < 0 || prob >= ctx->nprob || !x || !y) return fail(ctx, DDST_ERR_INVALID_ARG, "bad argument");
  ddst_status s = ensure_solve_buffers(ctx);
  if (s != DDST_OK) return s;
  if (ctx->mf_any) {  // matrix-free operators apply through the local factors
    s = ctx->prec == DDST_FP64 ? ensure_factors<double>(ctx) : ensure_factors<float>(ctx);
    if (s != DDST_OK) return s;
  }
  const ProbDesc& P = ctx->probs[prob];
  const int64_t len = (int64_t)P.nds * P.ng;
  CK(cudaMemsetAsync(ctx->if_tmp, 0, sizeof(double) * ctx->tot_if, ctx->stream));
  CK(stage_in(ctx->if_tmp + P.if_off, x, len, ctx->stream));
  if (ctx->prec == DDST_FP64) apply_interface_T<double>(ctx, ctx->if_tmp, ctx->if_w, transpose != 0);
  else apply_interface_T<float>(ctx, ctx->if_tmp, ctx->if_w, transpose != 0);
  CK(cudaGetLastError());
  CK(stage_out(y, ctx->if_w + P.if_off, len, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return DDST_OK;
}

ddst_status ddst_solve_interface(ddst_ctx* ctx, int prob, const double* rhs, double* x,
                                 int transpose) {
  if (!ctx) return fail(nullptr, DDST_ERR_INVALID_ARG, "ctx is NULL");
  if (prob < 0 || prob >= ctx->nprob) return fail(ctx, DDST_ERR_INVALID_ARG, "bad problem index");
  if (!rhs || !x) return fail(ctx, DDST_ERR_INVALID_ARG, "rhs or x is NULL");
  if (ctx->state < 2) return fail(ctx, DDST_ERR_STATE, "transfer operators not built");
  ddst_status s = ensure_solve_buffers(ctx);
  if (s != DDST_OK) return s;
  const ProbDesc& P = ctx->probs[prob];
  const size_t len = (size_t)P.nds * P.ng;
  CK(cudaMemsetAsync(ctx->if_u, 0, sizeof(double) * ctx->tot_if, ctx->stream));
  CK(stage_in(ctx->if_u + P.if_off, rhs, len, ctx->stream));
  s = ctx->prec == DDST_FP64 ? direct_interface_solve<double>(ctx, ctx->if_u, ctx->if_u, transpose != 0)
                             : direct_interface_solve<float>(ctx, ctx->if_u, ctx->if_u, transpose != 0);
  if (s != DDST_OK) return s;
  CK(stage_out(x, ctx->if_u + P.if_off, len, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx, nullptr);
}

ddst_status ddst_time_apply(ddst_ctx* ctx, int transpose, int reps, float* ms) {
  if (!ctx || !ms || reps < 1) return fail(ctx, DDST_ERR_INVALID_ARG, "bad argument");
  if (ctx->state < 2) return fail(ctx, DDST_ERR_STATE, "transfer operators not built");
  ddst_status s = ensure_solve_buffers(ctx);
  if (s != DDST_OK) return s;
  if (ctx->mf_any) {
    s = ctx->prec == DDST_FP64 ? ensure_factors<double>(ctx) : ensure_factors<float>(ctx);
    if (s != DDST_OK) return s;
  }
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(ctx->if_tmp, 0, sizeof(double) * ctx->tot_if, st));
  auto one = [&]() {
    if (ctx->prec == DDST_FP64) apply_interface_T<double>(ctx, ctx->if_tmp, ctx->if_w, transpose != 0, st);
    else apply_interface_T<float>(ctx, ctx->if_tmp, ctx->if_w, transpose != 0, st);
  };
  one();  // warm
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, st));
  for (int r = 0; r < reps; ++r) one();
  CK(cudaEventRecord(e1, st));
  CK(cudaEventSynchronize(e1));
  float t = 0.f;
  CK(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CK(cudaGetLastError());
  *ms = t / reps;
  return DDST_OK;
}

ddst_status ddst_query(const ddst_ctx* ctx, int prob, int* n_ds, int64_t* n_gamma, int* max_rank) {
  if (!ctx) return fail(nullptr, DDST_ERR_INVALID_ARG, "ctx is NULL");
  if (prob < 0 || prob >= ctx->nprob)
    return fail(nullptr, DDST_ERR_INVALID_ARG, "prob %d outside [0, %d)", prob, ctx->nprob);
  const ProbDesc& P = ctx->probs[prob];
  if (n_ds) *n_ds = P.nds;
  if (n_gamma) *n_gamma = P.ng;
  if (max_rank)
    *max_rank = ctx->state == 3 ? ctx->hodlr.max_rank : ctx->state == 4 ? ctx->hbs.k : 0;
  return DDST_OK;
}

int64_t ddst_kernel_launches(void) { return (int64_t)launch_counter().load(); }

const char* ddst_last_error(const ddst_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_setup_error.c_str();
}

void ddst_destroy(ddst_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto& g : ctx->arn_graph)
    if (g) cudaGraphExecDestroy(g);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->s_hi) { cudaStreamSynchronize(ctx->s_hi); cudaStreamDestroy(ctx->s_hi); }
  if (ctx->s_lo) { cudaStreamSynchronize(ctx->s_lo); cudaStreamDestroy(ctx->s_lo); }
  for (cudaEvent_t ev : ctx->big_ev)
    if (ev) cudaEventDestroy(ev);
  ctx->hodlr.release();
  ctx->hbs.release();
  for (void* p : ctx->owned) cudaFree(p);
  delete ctx;
}

}  // extern "C"
