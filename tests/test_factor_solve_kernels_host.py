"""The two-sided block factorization, the single-right-hand-side local solves and the explicit
transfer build (`csrc/factor.cu`, `csrc/solve.cu`, `csrc/sweep.cu`, with the blocked Gauss-Jordan
inversion of `csrc/bgj.cuh`), compiled for the host and run with one OS thread per CUDA thread
under AddressSanitizer (`tests/hostemu/cuda_host_shim.h`).  The bulk copies and mbarriers of
these kernels run on a host model (`tests/hostemu/mbarrier_host.h`) that also checks the copies'
16-byte alignment and byte counts.

Every double-slab operator A_j(I_j, I_j) is the oracle's assembled matrix (O1) restricted to the
index set I_j of O2, in the kernels' block order (y blocks, x offset, z).  Against its plain
definitions:
* F_k = Sigma_k^{-1} is the last diagonal block of the inverse of the leading k x k block
  submatrix, B_k = Lambda_k^{-1} the first diagonal block of the inverse of the trailing one, and
  G_k the k-th diagonal block of A_j^{-1}; padded rows and columns are the identity;
* the local solves equal A_j^{-1} b and A_j^{-T} b, and their central rows Gamma_j;
* the transfer build gives O3's S_{j,j-1} and S_{j,j+1} (Sec. 2.2, Eq. (defS)), every entry
  written once;
* chunked pivot sweeps with warm-up rows give the sequential pivots and a small convergence
  check, and too short a warm-up makes the check report a large difference;
* the FP32 factorization's tensor-core operand copies hold the TF32 hi/lo split of
  -diag(ell_{k+1}) F_k (forward) and -diag(ups_{k-1}) B_k (backward), transposed, in the K-major
  operand layout;
* the tensor-core transfer build (`csrc/sweep_tc.cu`, on the tcgen05 model of
  `tests/hostemu/tcgen05_host.h`) from those copies gives O3's operators, every entry written,
  in 3xTF32 and in TF32.
In FP64 and FP32, for block sizes 32 and 64, in 2D with convection and in 3D.
"""
import os
import re
import shutil
import struct
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import ddst_inputs as I
from oracle import ddst_oracle as O
from test_tc_kernels_host import _host_tmem_calls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_25991_gb300", "csrc")
# AddressSanitizer by default; DDST_HOST_SANITIZER=thread runs the same tests under
# ThreadSanitizer, which reports accesses of two threads that no barrier orders
SANITIZE = "-fsanitize=" + os.environ.get("DDST_HOST_SANITIZER", "address")

# Host stand-ins for the inline-PTX helpers on the mbarrier / bulk-copy model (TF32 rounding and
# the tensor-core instructions come from the tcgen05 model).
HOST_HELPERS = r'''
inline void mbar_init(uint64_t* bar, uint32_t count) { host_mbar_init(bar, count); }
inline void fence_mbar_init() {}
inline void fence_proxy_async() { std::atomic_thread_fence(std::memory_order_seq_cst); }
inline void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) { host_mbar_arrive_expect_tx(bar, bytes); }
inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) { host_bulk_g2s(dst, src, bytes, bar); }
inline bool mbar_wait(uint64_t* bar, uint32_t parity, DevStatus* st, int slab, int block) {
  if (host_mbar_wait(bar, parity)) return true;
  set_status(st, ST_TIMEOUT, slab, block);
  return false;
}
inline bool mbar_wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort, DevStatus* st,
                         int slab, int block, long long budget = 0) {
  (void)budget;
  for (long it = 0; it < 20000000L; ++it) {
    if (host_mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
    std::this_thread::yield();
  }
  set_status(st, ST_TIMEOUT, slab, block);
  *abort = 1;
  return false;
}
'''

MAIN = r'''
#include <fstream>
#include <limits>
using namespace ddst;

template <typename T> struct Cfg;
template <> struct Cfg<double> { static constexpr int nst32 = 16, nst64 = 5, r32 = 64, r64 = 64, s32 = 2, s64 = 2; };
template <> struct Cfg<float> { static constexpr int nst32 = 24, nst64 = 11, r32 = 128, r64 = 128, s32 = 3, s64 = 2; };

template <typename V> static void put(std::ofstream& o, const V& v) {
  for (auto e : v) { const double d = (double)e; o.write((const char*)&d, 8); }
}

template <typename T, int M>
int run(std::ifstream& f, std::ofstream& o, const int64_t* h, const double* dd) {
  const int dim = (int)h[0], n = (int)h[1], w = (int)h[2], has_c = (int)h[4];
  const int64_t nnode = h[5];
  const int nchunks = (int)h[7], full = (int)h[8];
  ProbDesc P{};
  P.dim = dim; P.n = n; P.w = w; P.nds = n / w - 1; P.has_c = has_c; P.M = M;
  P.h = dd[0]; P.b[0] = dd[1]; P.b[1] = dd[2]; P.b[2] = dd[3];
  const int p = dim == 2 ? 1 : n - 1, m = (2 * w - 1) * p, nb = n - 1, nds = P.nds;
  const int64_t ng = (int64_t)nb * p, nint = (int64_t)nb * nb * p, nloc = (int64_t)nds * nb * M;
  P.p = p; P.m = m; P.nb = nb; P.nint = nint; P.ng = ng; P.nnode = nnode;
  std::vector<SlabDesc> slabs(nds);
  int64_t s_off = 0;
  for (int q = 0; q < nds; ++q) {
    SlabDesc s{};
    s.prob = 0; s.j = q + 1; s.M = M; s.m = m; s.nb = nb; s.p = p; s.w = w; s.n = n; s.ng = ng;
    s.fac_off = (int64_t)q * nb * M * M; s.pack_off = (int64_t)q * nb * PK_NFIELDS * M;
    s.loc_off = (int64_t)q * nb * M; s.if_off = (int64_t)q * ng;
    s.sp_off = -1; s.sn_off = -1;
    if (s.j >= 2) { s.sp_off = s_off; s_off += ng * ng; }
    if (s.j <= nds - 1) { s.sn_off = s_off; s_off += ng * ng; }
    slabs[q] = s;
  }
  std::vector<double> A(nnode), C(nnode), b64(nloc);
  f.read((char*)A.data(), 8 * nnode); f.read((char*)C.data(), 8 * nnode);
  std::vector<FacChunk> ch(nchunks);
  int nslots = 0;
  for (auto& c : ch) {
    int32_t v[6]; f.read((char*)v, 24);
    c.slab = v[0]; c.dir = v[1]; c.start = v[2]; c.first = v[3]; c.last = v[4]; c.chk = v[5];
    nslots = std::max(nslots, c.chk + 1);
  }
  f.read((char*)b64.data(), 8 * nloc);
  std::vector<T> pack((int64_t)nds * nb * PK_NFIELDS * M, T(0)), b(b64.begin(), b64.end());
  host_launch2(nb, nds, 128, [&] { k_stencil_pack<T>(slabs.data(), &P, A.data(), C.data(), pack.data()); });

  // pivot sweeps and their convergence check
  const int64_t nfac = (int64_t)nds * nb * M * M;
  std::vector<T> F(nfac, T(0)), B(nfac, T(0)), Ft(nfac, T(0)), Bt(nfac, T(0)), G(nfac, T(0));
  std::vector<T> chk((int64_t)std::max(1, nslots) * M * M, T(0));
  std::vector<float> diff(nchunks, -1.f), Uhi, Ulo;
  if (sizeof(T) == 4) { Uhi.assign(2 * nfac, -1.f); Ulo.assign(2 * nfac, -1.f); }
  DevStatus stt{};
  {
    const size_t sm = BGJ<T, M>::smem_elems * sizeof(T) + (3 * PK_NFIELDS * M + M) * sizeof(T) + 24;
    std::vector<unsigned char> dyn(sm);
    host_dynamic_smem = dyn.data();
    host_launch(nchunks, FactorOcc<T>::threads, [&] {
      k_factor<T, M>(slabs.data(), ch.data(), pack.data(), F.data(), B.data(), Ft.data(), Bt.data(),
                     chk.data(), Uhi.empty() ? nullptr : Uhi.data(), Ulo.empty() ? nullptr : Ulo.data(),
                     nfac, &stt);
    });
    host_launch(nchunks, 256, [&] {
      k_factor_verify<T, M>(slabs.data(), ch.data(), F.data(), B.data(), chk.data(), diff.data());
    });
  }
  put(o, F); put(o, B); put(o, Ft); put(o, Bt); put(o, diff);
  if (sizeof(T) == 4) { put(o, Uhi); put(o, Ulo); }
  if (!full) { const double code = stt.code; o.write((const char*)&code, 8); return 0; }

  // diagonal blocks of the inverse
  std::vector<int> ids(nds);
  for (int q = 0; q < nds; ++q) ids[q] = q;
  {
    const size_t sm = BGJ<T, M>::smem_elems * sizeof(T) + (PK_NFIELDS * M + 3 * M) * sizeof(T);
    std::vector<unsigned char> dyn(sm);
    host_dynamic_smem = dyn.data();
    host_launch2(nb, nds, 256, [&] {
      k_center<T, M>(slabs.data(), ids.data(), pack.data(), F.data(), B.data(), G.data(), &stt);
    });
  }
  put(o, G);

  // local solves: A^{-1} b (full blocks and central rows) and A^{-T} b
  constexpr int NST = M == 32 ? Cfg<T>::nst32 : Cfg<T>::nst64;
  auto solve = [&](int transpose, int mode, std::vector<T>& x, std::vector<double>& iface) {
    std::vector<T> bf(nloc, T(0)), bb(nloc, T(0));
    const size_t sm = (size_t)NST * (M * M + 2 * M) * sizeof(T) + 5 * M * sizeof(T) + NST * 8;
    std::vector<unsigned char> dyn(sm);
    host_dynamic_smem = dyn.data();
    host_launch2(nds, 2, 4 * M, [&] {
      k_solve_sweep<T, M, NST>(slabs.data(), ids.data(), transpose ? F.data() : Ft.data(),
                               transpose ? B.data() : Bt.data(), pack.data(), b.data(), bf.data(),
                               bb.data(), transpose, &stt);
    });
    host_launch2(nb, nds, 128, [&] {
      k_solve_combine<T, M>(slabs.data(), ids.data(), G.data(), b.data(), bf.data(), bb.data(),
                            x.data(), iface.data(), transpose, mode);
    });
  };
  std::vector<T> x(nloc, T(0)), xT(nloc, T(0)), xdummy(nloc, T(0));
  std::vector<double> iface(nds * ng, std::numeric_limits<double>::quiet_NaN()), idummy(1);
  solve(0, 0, x, idummy);
  solve(1, 0, xT, idummy);
  solve(0, 1, xdummy, iface);
  put(o, x); put(o, xT); put(o, iface);

  // explicit transfer operators, tiles as the library plans them
  constexpr int R = M == 32 ? Cfg<T>::r32 : Cfg<T>::r64;
  constexpr int SN = M == 32 ? Cfg<T>::s32 : Cfg<T>::s64;
  std::vector<TileDesc> tiles;
  for (int sid = 0; sid < nds; ++sid)
    for (int64_t q0 = 0; q0 < ng; q0 += R) {
      const int nq = (int)std::min<int64_t>(R, ng - q0);
      TileDesc up{sid, (int)q0, nq, 0, (int)((q0 + nq - 1) / p) + 1, 0};
      up.len = up.kstart;
      TileDesc dn{sid, (int)q0, nq, 1, (int)(q0 / p) + 1, 0};
      dn.len = nb - dn.kstart + 1;
      tiles.push_back(up);
      tiles.push_back(dn);
    }
  std::vector<T> S(s_off, std::numeric_limits<T>::quiet_NaN());
  {
    using Cs = SweepCfg<T, M, R, SN>;
    std::vector<unsigned char> dyn(Cs::SMEM);
    host_dynamic_smem = dyn.data();
    host_launch((unsigned)tiles.size(), 128, [&] {
      k_sbuild<T, M, R, SN>(slabs.data(), tiles.data(), F.data(), B.data(), G.data(), pack.data(),
                           S.data(), &stt);
    });
  }
  put(o, S);
  if constexpr (sizeof(T) == 4) {
    // the same operators on the tensor cores, from the factor kernel's TF32 operand copies
    using Ct = TcCfg<M>;
    const int Rt = Ct::NT * Ct::TILE;
    std::vector<TileDesc> tt;
    for (int sid = 0; sid < nds; ++sid)
      for (int64_t q0 = 0; q0 < ng; q0 += Rt) {
        const int nq = (int)std::min<int64_t>(Rt, ng - q0);
        TileDesc up{sid, (int)q0, nq, 0, (int)((q0 + nq - 1) / p) + 1, 0};
        up.len = up.kstart;
        TileDesc dn{sid, (int)q0, nq, 1, (int)(q0 / p) + 1, 0};
        dn.len = nb - dn.kstart + 1;
        tt.push_back(up);
        tt.push_back(dn);
      }
    unsigned char* sm = static_cast<unsigned char*>(std::aligned_alloc(1024, (Ct::SMEM + 1023) / 1024 * 1024));
    host_smem_base = sm;
    for (int three = 1; three >= 0; --three) {
      std::vector<float> Stc(s_off, std::numeric_limits<float>::quiet_NaN());
      host_launch((unsigned)tt.size(), Ct::THREADS, [&] {
        k_sbuild_tc<M>(slabs.data(), tt.data(), Uhi.data(), Ulo.data(), Uhi.data() + nfac,
                       Ulo.data() + nfac, G.data(), pack.data(), Stc.data(), &stt, 4000000000LL, three);
      });
      put(o, Stc);
    }
    std::free(sm);
  }
  const double code = stt.code;
  o.write((const char*)&code, 8);
  return 0;
}

int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  std::ofstream o(argv[2], std::ios::binary);
  int64_t h[10]; double d[4];
  f.read((char*)h, 80); f.read((char*)d, 32);
  const int M = (int)h[3], esz = (int)h[6];
  if (esz == 8) return M == 32 ? run<double, 32>(f, o, h, d) : run<double, 64>(f, o, h, d);
  return M == 32 ? run<float, 32>(f, o, h, d) : run<float, 64>(f, o, h, d);
}
'''


def _between(src, start, end):
    i = src.index(start)
    return src[i:src.index(end, i)]


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    rd = lambda name: open(os.path.join(CSRC, name)).read()
    common, kern, bgj, umma = rd("common.cuh"), rd("kernels.cuh"), rd("bgj.cuh"), rd("umma.cuh")
    st, fac, sol, swp = rd("stencil.cu"), rd("factor.cu"), rd("solve.cu"), rd("sweep.cu")
    grab = lambda pat, src: re.search(pat, src, re.S).group(0)
    parts = [
        grab(r"enum PackField \{.*?\};", common),
        grab(r"struct ProbDesc \{.*?\n\};", common),
        grab(r"struct SlabDesc \{.*?\n\};", common),
        grab(r"struct DevStatus \{.*?\n\};", common),
        grab(r"enum \{ ST_SINGULAR.*?\};", common),
        grab(r"__device__ __forceinline__ void set_status\(.*?\n\}", common),
        _between(common, "template <typename T> struct Eps;", "// -----"),
        grab(r"__device__ __forceinline__ int64_t vol_index\(.*?\n\}", common),
        grab(r"struct TileDesc \{.*?\n\};", kern),
        grab(r"struct FacChunk \{.*?\n\};", kern),
        HOST_HELPERS,
        grab(r"__host__ __device__ __forceinline__ uint32_t umma_off\(.*?\n\}", umma),
        _between(umma, "template <int M>\n__device__ __forceinline__ void store_umma_split_T(",
                 "// -----"),
        grab(r"__device__ __forceinline__ uint64_t umma_desc\(.*?\n\}", umma),
        grab(r"__host__ __device__ constexpr uint32_t idesc_tf32\(.*?\n\}", umma),
        grab(r"__device__ __forceinline__ void tf32_split\(.*?\n\}", umma),
        _between(bgj, "template <typename T, int M>\nstruct BGJ {", "}  // namespace ddst"),
        _between(st, "__device__ __forceinline__ int64_t node_index(",
                 "// b = f + (Dirichlet neighbour terms)"),
        _between(fac, "// X (shared, leading dimension LD) += D_k",
                 "template <typename T, int M>\nstatic size_t factor_smem()"),
        _between(sol, "// One sweep of one slab",
                 "template <typename T, int M, int NST>\nstatic void run_solve("),
        _between(swp, "template <typename T, int N>\n__device__ __forceinline__ void lds(",
                 "template <typename T, int M, int R, int NST>\nstatic void run_sbuild("),
    ]
    tc = _between(rd("sweep_tc.cu"), "template <int MB>\nstruct TcCfg {",
                  "template <int MB>\nstatic void run_tc(")
    tc = tc.replace("extern __shared__ __align__(1024) unsigned char smem_raw[];",
                    "unsigned char* smem_raw = host_smem_base;")
    parts.append(_host_tmem_calls(tc))
    body = "\n".join(parts)
    dyn = "extern __shared__ __align__(128) unsigned char smem_raw[];"
    assert body.count(dyn) == 4
    body = body.replace(dyn, "unsigned char* smem_raw = host_dynamic_smem;")
    code = ('#include "cuda_host_shim.h"\n#include "mbarrier_host.h"\n#include "tcgen05_host.h"\n#include <cstring>\n'
            "static unsigned char* host_dynamic_smem = nullptr;\nnamespace ddst {\n" + body +
            "\n}  // namespace ddst\n" + MAIN)
    d = tmp_path_factory.mktemp("factor_host")
    (d / "factor_host.cpp").write_text(code)
    exe = d / "factor_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "factor_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    return d, exe


def _pad_M(m):
    return 32 if m <= 32 else 64


def _exact_chunks(nds, nb, slabs=None):
    out = []
    for s in (range(nds) if slabs is None else slabs):
        out.append((s, 0, 1, 1, nb, -1))
        out.append((s, 1, nb, nb, 1, -1))
    return out


def _warm_chunks(slabs, nb, nch, W):
    """Chunks of the pivot sweeps with W warm-up rows, as the library plans them."""
    out, slots = [], 0
    C = (nb + nch - 1) // nch
    for s in slabs:
        for d in range(2):
            for c in range(nch):
                if d == 0:
                    first, last = c * C + 1, min(nb, (c + 1) * C)
                    start = max(1, first - W)
                    chk = -1 if start == 1 else slots
                else:
                    first, last = nb - c * C, max(1, nb - (c + 1) * C + 1)
                    start = min(nb, first + W)
                    chk = -1 if start == nb else slots
                slots += chk >= 0
                out.append((s, d, start, first, last, chk))
    return out


def _run(harness, name, n, w, esz, chunks, full, over=None, tag=""):
    d, exe = harness
    prob = I.make_problem(name, n=n, w=w, **(over or {}))
    dim = prob["dim"]
    p = 1 if dim == 2 else n - 1
    m, nb, nds = (2 * w - 1) * p, n - 1, n // w - 1
    M = _pad_M(m)
    ng = nb * p
    nloc, nfac = nds * nb * M, nds * nb * M * M
    has_c = prob.get("c") is not None
    bb = list(prob["b"]) + [0.0] * (3 - len(prob["b"]))
    nnode = (n + 1) ** dim
    rng = np.random.default_rng(n * 10 + w)
    b = np.zeros((nds, nb, M))
    b[:, :, :m] = rng.standard_normal((nds, nb, m))
    path = d / f"fac_{name}_{n}_{w}_{esz}{tag}.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("10q", dim, n, w, M, int(has_c), nnode, esz, len(chunks), full, 0))
        f.write(struct.pack("4d", 1.0 / n, *bb))
        f.write(np.asarray(prob["a"], dtype=np.float64).ravel().tobytes())
        f.write((np.asarray(prob["c"], dtype=np.float64).ravel() if has_c else np.zeros(nnode)).tobytes())
        for c in chunks:
            f.write(struct.pack("6i", *c))
        f.write(b.tobytes())
    out = path.with_suffix(".out")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    raw = np.fromfile(out, dtype=np.float64)
    res, pos = {}, 0
    sizes = [("F", nfac), ("B", nfac), ("Ft", nfac), ("Bt", nfac), ("diff", len(chunks))]
    if esz == 4:
        sizes += [("Uhi", 2 * nfac), ("Ulo", 2 * nfac)]
    if full:
        sizes += [("G", nfac), ("x", nloc), ("xT", nloc), ("iface", nds * ng),
                  ("S", 2 * (nds - 1) * ng * ng)]
        if esz == 4:
            sizes += [("S_tc3", 2 * (nds - 1) * ng * ng), ("S_tc1", 2 * (nds - 1) * ng * ng)]
    for key, cnt in sizes:
        res[key] = raw[pos:pos + cnt]
        pos += cnt
    res["code"] = raw[pos]
    assert pos + 1 == raw.size
    for key in ("F", "B", "Ft", "Bt", "G"):
        if key in res:
            res[key] = res[key].reshape(nds, nb, M, M)
    for key in ("x", "xT"):
        if key in res:
            res[key] = res[key].reshape(nds, nb, M)
    A = sp.csr_matrix(O.assemble(prob)[0])
    geo = O.slab_geometry(dim, n, w)
    ctx = dict(prob=prob, A=A, geo=geo, dim=dim, p=p, m=m, nb=nb, nds=nds, M=M, ng=ng, b=b)
    return res, ctx


def _local_matrix(ctx, j):
    """A_j(I_j, I_j) in the kernels' block order: y block k, then x offset cx, then z."""
    w2 = 2 * ctx["geo"].w - 1
    Ij = np.asarray(ctx["geo"].I[j]).reshape(w2, ctx["nb"], ctx["p"]).transpose(1, 0, 2).ravel()
    return ctx["A"][Ij][:, Ij].toarray()


def _ref_pivot_inverses(Aj, nb, m):
    Fr = [np.linalg.inv(Aj[:k * m, :k * m])[-m:, -m:] for k in range(1, nb + 1)]
    Br = [np.linalg.inv(Aj[(k - 1) * m:, (k - 1) * m:])[:m, :m] for k in range(1, nb + 1)]
    Ai = np.linalg.inv(Aj)
    Gr = [Ai[(k - 1) * m:k * m, (k - 1) * m:k * m] for k in range(1, nb + 1)]
    return Fr, Br, Gr


def _check_block(got, want, m, tol):
    M = got.shape[-1]
    scale = np.abs(want).max()
    err = np.abs(got[:m, :m] - want).max() / scale
    assert err <= tol, err
    pad = got.copy()
    pad[:m, :m] = 0.0
    assert np.array_equal(pad, np.diag(np.r_[np.zeros(m), np.ones(M - m)]))
    return err


def _umma_index(r, c, K):
    """Float index of operand row r, K index c in the K-major no-swizzle layout: core matrices of
    8 rows x 4 TF32 values (16 bytes a row), consecutive along K every 128 bytes, row groups of 8
    every 32 K bytes."""
    return (r >> 3) * (K * 8) + (c >> 2) * 32 + (r & 7) * 4 + (c & 3)


def _check_tc_copies(res, ctx, j, Aj):
    """FP32: the TF32 hi/lo split of -diag(ell_{k+1}) F_k and -diag(ups_{k-1}) B_k, transposed."""
    m, nb, M = ctx["m"], ctx["nb"], ctx["M"]
    nfac = ctx["nds"] * nb * M * M
    idx = np.array([[_umma_index(r, c, M) for c in range(M)] for r in range(M)])
    for d, X, key in ((0, res["F"], "F"), (1, res["B"], "B")):
        for k in range(1, nb + 1):
            base = d * nfac + (j * nb + k - 1) * M * M
            hi = res["Uhi"][base:base + M * M][idx]      # [r, c]
            lo = res["Ulo"][base:base + M * M][idx]
            for v in (hi, lo):                            # TF32: 13 low significand bits zero
                bits = v.astype(np.float32).view(np.uint32)
                assert np.all(bits & 0x1FFF == 0)
            kn = k + 1 if d == 0 else k - 1
            want = np.zeros((M, M))
            if 1 <= kn <= nb:
                # ell_{k+1} = L_{k+1}(c, c) couples block k+1 to block k; ups_{k-1} = U_{k-1}(c, c)
                cpl = np.diag(Aj[(kn - 1) * m:kn * m, (k - 1) * m:k * m])
                want[:, :m] = (-cpl[:, None] * X[j, k - 1, :m, :]).T   # operand (r, c) = -s_c X(c, r)
            assert np.all(np.abs(hi + lo - want) <= 2.0 ** -21 * np.abs(want) + 1e-30), (key, k)


CASES = [("convdiff2d", 32, 4, 8, None), ("convdiff2d", 32, 4, 4, None),
         ("vardiff3d", 8, 2, 8, {"b": (1.0, -0.5, 2.0)}), ("vardiff3d", 12, 3, 8, None),
         ("vardiff3d", 12, 3, 4, {"b": (0.5, 1.0, -1.0)})]


@pytest.mark.parametrize("name,n,w,esz,over", CASES)
def test_factor_solve_and_transfer_build_on_the_host(harness, name, n, w, esz, over):
    nds, nb = n // w - 1, n - 1
    res, ctx = _run(harness, name, n, w, esz, _exact_chunks(nds, nb), 1, over)
    assert res["code"] == 0.0
    m, M, ng, p = ctx["m"], ctx["M"], ctx["ng"], ctx["p"]
    u = 2.0 ** -53 if esz == 8 else 2.0 ** -24
    # blocks: Gauss-Jordan on well-conditioned M-matrix blocks, a few dozen roundings
    tol_blk = 64 * u
    assert np.all(res["diff"] == 0.0)          # no warm-started chunks
    Sp, Sn = O.transfer_blocks(ctx["A"], ctx["geo"], O.factor_local(ctx["A"], ctx["geo"]))
    S = res["S"]
    assert not np.isnan(S).any()               # every entry written by one of the two sweeps
    s_off = 0
    for j in range(nds):
        Aj = _local_matrix(ctx, j)
        Fr, Br, Gr = _ref_pivot_inverses(Aj, nb, m)
        for k in range(nb):
            _check_block(res["F"][j, k], Fr[k], m, tol_blk)
            _check_block(res["B"][j, k], Br[k], m, tol_blk)
            _check_block(res["G"][j, k], Gr[k], m, tol_blk)
            assert np.array_equal(res["Ft"][j, k], res["F"][j, k].T)
            assert np.array_equal(res["Bt"][j, k], res["B"][j, k].T)
        if esz == 4:
            _check_tc_copies(res, ctx, j, Aj)
        # solves: backward error of a stable solve, cond(A_j) u
        tol = 8 * np.linalg.cond(Aj) * u
        bj = ctx["b"][j, :, :m].ravel()
        for key, Am in (("x", Aj), ("xT", Aj.T)):
            want = np.linalg.solve(Am, bj)
            got = res[key][j]
            assert np.abs(got[:, :m].ravel() - want).max() <= tol * np.abs(want).max(), key
            assert np.all(got[:, m:] == 0.0)
        centre = np.linalg.solve(Aj, bj).reshape(nb, m)[:, (w - 1) * p:w * p].ravel()
        got = res["iface"][j * ng:(j + 1) * ng]
        assert np.abs(got - centre).max() <= tol * np.abs(centre).max()
        # transfer operators, column-major n_Gamma x n_Gamma
        for Sref in (Sp[j], Sn[j]):
            if Sref is None:
                continue
            blk = S[s_off:s_off + ng * ng].reshape(ng, ng).T
            assert np.abs(blk - Sref).max() <= tol * np.abs(Sref).max()
            if esz == 4:
                # the tensor-core build from the TF32 operand copies: 3xTF32 to FP32 accuracy;
                # one TF32 product per step rounds an operand to 11 bits once per block row
                for key, tl in (("S_tc3", tol), ("S_tc1", nb * 2.0 ** -11)):
                    bt = res[key][s_off:s_off + ng * ng].reshape(ng, ng).T
                    assert np.abs(bt - Sref).max() <= tl * np.abs(Sref).max(), key
            s_off += ng * ng
    assert s_off == S.size
    if esz == 4:
        assert not np.isnan(res["S_tc3"]).any() and not np.isnan(res["S_tc1"]).any()


@pytest.mark.parametrize("W", [20, 4])
def test_warm_started_pivot_chunks_on_the_host(harness, W):
    """Chunks of the pivot sweeps that start W rows early from Sigma = D (2D, w = 2: the pivot
    recurrence forgets its start by about exp(-pi / w) per row).  With 20 warm-up rows the
    stored inverses are the sequential ones and the convergence check is at rounding level;
    with 4 the check reports the difference, and the library then reruns the sweeps exactly."""
    n, w, nb, slabs = 64, 2, 63, [0, 15, 30]
    chunks = _warm_chunks(slabs, nb, 2, W)
    assert sum(c[5] >= 0 for c in chunks) == 2 * len(slabs)
    res, ctx = _run(harness, "convdiff2d", n, w, 8, chunks, 0, tag=f"_W{W}")
    assert res["code"] == 0.0
    m = ctx["m"]
    worst = 0.0
    for j in slabs:
        Fr, Br, _ = _ref_pivot_inverses(_local_matrix(ctx, j), nb, m)
        for k in range(nb):
            for X, R in ((res["F"][j, k], Fr[k]), (res["B"][j, k], Br[k])):
                worst = max(worst, np.abs(X[:m, :m] - R).max() / np.abs(R).max())
    warm = np.array([res["diff"][q] for q, c in enumerate(chunks) if c[5] >= 0])
    assert np.all(res["diff"][[c[5] < 0 for c in chunks]] == 0.0)
    if W == 20:
        assert worst <= 1e-13 and warm.max() <= 1e-12
    else:
        assert warm.min() > 1e-5 and worst > 1e-6   # the check sees what the sweep got wrong
