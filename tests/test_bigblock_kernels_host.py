"""The large-block factorization and local solves of `csrc/bigblock.cu` (double slabs with
m > 128 unknowns per block row), compiled for the host and run with one OS thread per
CUDA thread under AddressSanitizer (`tests/hostemu/cuda_host_shim.h`):
* `k_big_sigma`, `k_big_pivot`, `k_big_gemm_fma` (row and update steps of the 128-wide panel
  Gauss-Jordan inversion, with the look-ahead split of the update): F_k = Sigma_k^{-1} of the
  one-sided block LU Sigma_k = D_k - L_k Sigma_{k-1}^{-1} U_{k-1} of the oracle's local operator
  (O1 restricted to I_j), with three 128-wide panels (M = 384, FP64) and two (M = 256, FP32);
* the look-ahead: the update of panel q runs on a second stream beside the next panel's pivot
  and row steps, so two orders of the same launches are legal (the second stream finishing each
  update before the next panel starts, and the first stream running ahead).  Both give the same
  factors bit for bit;
* `k_big_gemv_n`, `k_big_gemv_t`, `k_big_extract`: A_j^{-1} b, A_j^{-T} b and the central rows,
  against a sparse direct solve;
* the tensor-core operand copies of the first pivot step (`k_big_pivot` with split tiles, FP32):
  TF32 hi/lo parts of X(B, Q), X(Q, B)^T, P, P^{-1} and P^{-T} in the chunked K-major layout;
* the FP32 factorization with the panel products on the tensor cores (`k_big_gemm_tc` on the
  tcgen05 model of `tests/hostemu/tcgen05_host.h`), 3xTF32 and TF32.
In FP64 and FP32.
"""
import os
import re
import shutil
import struct
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import ddst_inputs as I
from oracle import ddst_oracle as O
from test_tc_kernels_host import MBAR_HELPERS, _host_tmem_calls

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_25991_gb300", "csrc")
# AddressSanitizer by default; DDST_HOST_SANITIZER=thread runs the same tests under
# ThreadSanitizer, which reports accesses of two threads that no barrier orders
SANITIZE = "-fsanitize=" + os.environ.get("DDST_HOST_SANITIZER", "address")

MAIN = r'''
#include <fstream>
using namespace ddst;
template <typename V> static void put(std::ofstream& o, const V& v) {
  for (auto e : v) { const double d = (double)e; o.write((const char*)&d, 8); }
}
template <typename T, int MODE>
void gemm(unsigned gx, int nids, const SlabDesc* sl, const int* ids, T* F, int k, int q,
          const T* C, const T* X, T* R, const T* P, int tset) {
  host_launch3(gx, 1, nids, 256, [&] { k_big_gemm_fma<T, MODE>(sl, ids, F, k, q, C, X, R, P, tset); });
}
template <typename T>
int run(std::ifstream& f, std::ofstream& o, const int64_t* h, const double* dd) {
  const int dim = (int)h[0], n = (int)h[1], w = (int)h[2], M = (int)h[3], has_c = (int)h[4];
  const int64_t nnode = h[5];
  const int nids = (int)h[7], sched = (int)h[8];
  ProbDesc P{};
  P.dim = dim; P.n = n; P.w = w; P.nds = n / w - 1; P.has_c = has_c; P.M = M;
  P.h = dd[0]; P.b[0] = dd[1]; P.b[1] = dd[2]; P.b[2] = dd[3];
  const int p = dim == 2 ? 1 : n - 1, m = (2 * w - 1) * p, nb = n - 1, nds = P.nds, nP = M / BT;
  const int64_t ng = (int64_t)nb * p, nint = (int64_t)nb * nb * p, nloc = (int64_t)nds * nb * M;
  P.p = p; P.m = m; P.nb = nb; P.nint = nint; P.ng = ng; P.nnode = nnode;
  std::vector<SlabDesc> slabs(nds);
  for (int q = 0; q < nds; ++q) {
    SlabDesc s{};
    s.prob = 0; s.j = q + 1; s.M = M; s.m = m; s.nb = nb; s.p = p; s.w = w; s.n = n; s.ng = ng;
    s.fac_off = (int64_t)q * nb * M * M; s.pack_off = (int64_t)q * nb * PK_NFIELDS * M;
    s.loc_off = (int64_t)q * nb * M; s.if_off = (int64_t)q * ng; s.sp_off = -1; s.sn_off = -1;
    slabs[q] = s;
  }
  std::vector<double> A(nnode), C(nnode), b64(nloc);
  f.read((char*)A.data(), 8 * nnode); f.read((char*)C.data(), 8 * nnode);
  std::vector<int> ids(nids);
  for (auto& v : ids) { int32_t t; f.read((char*)&t, 4); v = t; }
  f.read((char*)b64.data(), 8 * nloc);
  std::vector<T> pack((int64_t)nds * nb * PK_NFIELDS * M, T(0)), b(b64.begin(), b64.end());
  host_launch2(nb, nds, 128, [&] { k_stencil_pack<T>(slabs.data(), &P, A.data(), C.data(), pack.data()); });
  const int64_t nfac = (int64_t)nds * nb * M * M;
  std::vector<T> F(nfac, T(0));
  DevStatus stt{};
  const SlabDesc* sl = slabs.data();
  const int* id = ids.data();

  // FP32: the split-tile operand copies of the first pivot step on Sigma_1 = D_1
  if constexpr (sizeof(T) == 4) {
    std::vector<float> F1(nfac, 0.f), Cs(nids * nP * SPLIT_TILE, -1.f), Xs(Cs.size(), -1.f),
        Rs(Cs.size(), -1.f), Ps(nids * SPLIT_TILE, -1.f);
    host_launch2(4, nids, 256, [&] { k_big_sigma<float>(sl, id, pack.data(), F1.data(), 1); });
    put(o, F1);
    const size_t gj = BGJ<float, BT>::smem_elems * 4 + BT * 4 + 16, stage = 2 * BT * (BT + 1) * 4;
    std::vector<unsigned char> dyn(gj > stage ? gj : stage);
    host_dynamic_smem = dyn.data();
    host_launch2(nP, nids, 512, [&] {
      k_big_pivot<float, true>(sl, id, pack.data(), F1.data(), 1, 0, Cs.data(), Xs.data(), Rs.data(), Ps.data(), &stt);
    });
    put(o, F1); put(o, Cs); put(o, Xs); put(o, Rs); put(o, Ps);
  }

  std::vector<T> Cb[2], XqT[2], RT[2], Pinv[2];
  for (int e = 0; e < 2; ++e) {
    Cb[e].assign((int64_t)nids * M * BT, T(0)); XqT[e] = Cb[e]; RT[e] = Cb[e];
    Pinv[e].assign((int64_t)nids * BT * BT, T(0));
  }
  const size_t gj = BGJ<T, BT>::smem_elems * sizeof(T) + BT * sizeof(T) + 16;
  const size_t stage = (size_t)BT * (BT + 1) * sizeof(T);
  std::vector<unsigned char> pdyn(gj > stage ? gj : stage);
  std::function<void(int, int)> pivot = [&](int k, int q) {
    const int e = q & 1;
    host_dynamic_smem = pdyn.data();
    host_launch2(nP, nids, 512, [&] {
      k_big_pivot<T, false>(sl, id, pack.data(), F.data(), k, q, Cb[e].data(), XqT[e].data(),
                            RT[e].data(), Pinv[e].data(), &stt);
    });
  };
  std::function<void(int, int)> row = [&](int k, int q) {
    const int e = q & 1;
    gemm<T, GJ_ROW>(nP, nids, sl, id, F.data(), k, q, Cb[e].data(), XqT[e].data(), RT[e].data(), Pinv[e].data(), GJ_ALL);
  };
  std::function<void(int, int, int)> update = [&](int k, int q, int tset) {
    const int e = q & 1;
    const int cnt = gj_count(tset, nP);
    if (cnt == 0) return;
    gemm<T, GJ_UPDATE>(cnt, nids, sl, id, F.data(), k, q, Cb[e].data(), XqT[e].data(), RT[e].data(), Pinv[e].data(), tset);
  };
  // tensor-core path (FP32): split-tile work buffers; from the second panel on, the pivot copies
  // come from the previous panel's update and row steps
  const int tc = (int)h[9], three = tc == 1 ? 1 : 0;
  std::vector<float> Cs2[2], Xs2[2], Rs2[2], Ps2[2];
  unsigned char* tsm = nullptr;
  if constexpr (sizeof(T) == 4) {
    if (tc) {
      for (int e = 0; e < 2; ++e) {
        Cs2[e].assign((int64_t)nids * nP * SPLIT_TILE, 0.f); Xs2[e] = Cs2[e]; Rs2[e] = Cs2[e];
        Ps2[e].assign((int64_t)nids * SPLIT_TILE, 0.f);
      }
      tsm = static_cast<unsigned char*>(std::aligned_alloc(1024, (GjTc::SMEM + 1023) / 1024 * 1024));
      const size_t stage2 = 2 * (size_t)BT * (BT + 1) * 4;
      if (pdyn.size() < stage2) pdyn.resize(stage2);
      pivot = [&](int k, int q) {
        const int e = q & 1;
        host_dynamic_smem = pdyn.data();
        host_launch2(q == 0 ? nP : 1, nids, 512, [&] {
          k_big_pivot<float, true>(sl, id, pack.data(), F.data(), k, q, Cs2[e].data(), Xs2[e].data(),
                                   Rs2[e].data(), Ps2[e].data(), &stt);
        });
      };
      row = [&](int k, int q) {
        const int e = q & 1;
        const bool nx = q + 1 < nP;
        host_smem_base = tsm;
        host_launch3(nP, 1, nids, GjTc::THREADS, [&] {
          k_big_gemm_tc<GJ_ROW>(sl, id, F.data(), k, q, Cs2[e].data(), Xs2[e].data(), Rs2[e].data(),
                                Ps2[e].data(), &stt, GJ_ALL, nx ? Cs2[e ^ 1].data() : nullptr,
                                nx ? Xs2[e ^ 1].data() : nullptr, three);
        });
      };
      update = [&](int k, int q, int tset) {
        const int e = q & 1;
        const int cnt = gj_count(tset, nP);
        if (cnt == 0) return;
        const bool nx = tset == GJ_NEXT;
        host_smem_base = tsm;
        host_launch3(cnt, 1, nids, GjTc::THREADS, [&] {
          k_big_gemm_tc<GJ_UPDATE>(sl, id, F.data(), k, q, Cs2[e].data(), Xs2[e].data(), Rs2[e].data(),
                                   Ps2[e].data(), &stt, tset, nx ? Cs2[e ^ 1].data() : nullptr,
                                   nx ? Xs2[e ^ 1].data() : nullptr, three);
        });
      };
    }
  }
  for (int k = 1; k <= nb; ++k) {
    host_launch2(4, nids, 256, [&] { k_big_sigma<T>(sl, id, pack.data(), F.data(), k); });
    pivot(k, 0);
    if (nP == 1) continue;
    row(k, 0);
    for (int q = 0; q < nP; ++q) {
      const bool ahead = q + 1 < nP;
      if (sched == 0) update(k, q, ahead ? GJ_REST : GJ_ALL);   // second stream keeps up
      if (ahead) {
        update(k, q, GJ_NEXT);
        pivot(k, q + 1);
        row(k, q + 1);
      }
      if (sched == 1) update(k, q, ahead ? GJ_REST : GJ_ALL);   // first stream runs ahead
    }
  }
  put(o, F);
  if (tsm) std::free(tsm);

  // local solves of the listed slabs
  std::vector<T> z(nloc, T(0)), x(nloc, T(0)), xT(nloc, T(0));
  std::vector<unsigned char> vdyn((size_t)(M + 8 * 64) * sizeof(T));
  host_dynamic_smem = vdyn.data();
  for (int k = 2; k <= nb; ++k)
    host_launch2(M / 32, nids, 256, [&] { k_big_gemv_n<T>(sl, id, F.data(), pack.data(), b.data(), z.data(), x.data(), SV_NFWD, k); });
  for (int i = 0; i < nb; ++i)
    host_launch2(M / 32, nids, 256, [&] { k_big_gemv_n<T>(sl, id, F.data(), pack.data(), b.data(), z.data(), x.data(), SV_NBWD, i); });
  std::fill(z.begin(), z.end(), T(0));
  for (int k = 1; k <= nb; ++k)
    host_launch2(M / 64, nids, 256, [&] { k_big_gemv_t<T>(sl, id, F.data(), pack.data(), b.data(), z.data(), xT.data(), SV_TFWD, k); });
  for (int i = 0; i < nb; ++i)
    host_launch2(M / 64, nids, 256, [&] { k_big_gemv_t<T>(sl, id, F.data(), pack.data(), b.data(), z.data(), xT.data(), SV_TBWD, i); });
  std::vector<double> iface(nds * ng, 0.0);
  host_launch2(3, nids, 64, [&] { k_big_extract<T>(sl, id, x.data(), iface.data()); });
  put(o, x); put(o, xT); put(o, iface);
  const double code = stt.code;
  o.write((const char*)&code, 8);
  return 0;
}
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  std::ofstream o(argv[2], std::ios::binary);
  int64_t h[10]; double d[4];
  f.read((char*)h, 80); f.read((char*)d, 32);
  return h[6] == 8 ? run<double>(f, o, h, d) : run<float>(f, o, h, d);
}
'''


def _between(src, start, end):
    i = src.index(start)
    return src[i:src.index(end, i + len(start))]


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    rd = lambda name: open(os.path.join(CSRC, name)).read()
    common, bgj, umma, split = rd("common.cuh"), rd("bgj.cuh"), rd("umma.cuh"), rd("splittile.cuh")
    st, big = rd("stencil.cu"), rd("bigblock.cu")
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
        MBAR_HELPERS,
        grab(r"__host__ __device__ __forceinline__ uint32_t umma_off\(.*?\n\}", umma),
        grab(r"__device__ __forceinline__ uint64_t umma_desc\(.*?\n\}", umma),
        grab(r"__host__ __device__ constexpr uint32_t idesc_tf32\(.*?\n\}", umma),
        _between(split, "constexpr int BT = 128;", "}  // namespace ddst"),
        _between(bgj, "template <typename T, int M>\nstruct BGJ {", "}  // namespace ddst"),
        _between(st, "__device__ __forceinline__ int64_t node_index(",
                 "// b = f + (Dirichlet neighbour terms)"),
        _between(big, "template <typename T>\n__global__ void __launch_bounds__(256) k_big_sigma(",
                 "struct GjTc {"),
        _between(big, "struct GjTc {", "// Local solves through the stored inverses"),
        _between(big, "enum { SV_NFWD = 0", "// Host launchers"),
        _between(big, "// Central rows of slab-local vectors",
                 "template <typename T>\nvoid launch_big_extract("),
    ]
    body = "\n".join(parts)
    body = _host_tmem_calls(body.replace("extern __shared__ __align__(1024) unsigned char smem_raw[];",
                                         "unsigned char* smem_raw = host_smem_base;"))
    for dyn in ("extern __shared__ __align__(128) unsigned char smem_raw[];",
                "extern __shared__ __align__(16) unsigned char smem_raw[];"):
        assert dyn in body
        body = body.replace(dyn, "unsigned char* smem_raw = host_dynamic_smem;")
    code = ('#include "cuda_host_shim.h"\n#include "mbarrier_host.h"\n#include "tcgen05_host.h"\n'
            '#include <cstring>\n#include <type_traits>\n'
            "static unsigned char* host_dynamic_smem = nullptr;\nnamespace ddst {\n" + body +
            "\n}  // namespace ddst\n" + MAIN)
    d = tmp_path_factory.mktemp("bigblock_host")
    (d / "big_host.cpp").write_text(code)
    exe = d / "big_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "big_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    return d, exe


# 3D problems: (n, w, listed slabs).  n = 21, w = 7: m = 13 * 20 = 260 unknowns per block row,
# M = 384 (three 128-wide panels: the look-ahead has a rest of the update to run beside the next
# panel), the second of two slabs; n = 20, w = 5: m = 171, M = 256 (two panels), the first and
# last of three slabs (per-slab work buffers, a gap in the slab list).
CFG64 = (21, 7, (1,))
CFG32 = (20, 5, (0, 2))


def _run(harness, esz, sched, cfg, tc=0):
    d, exe = harness
    N, W, IDS = cfg
    prob = I.make_problem("vardiff3d", n=N, w=W, b=(1.0, -0.5, 0.75))
    p, nb, nds = N - 1, N - 1, N // W - 1
    m = (2 * W - 1) * p
    M = (m + 127) // 128 * 128
    ng, nloc, nfac = nb * p, nds * nb * M, nds * nb * M * M
    nnode = (N + 1) ** 3
    rng = np.random.default_rng(17)
    b = np.zeros((nds, nb, M))
    b[:, :, :m] = rng.standard_normal((nds, nb, m))
    path = d / f"big_{esz}_{sched}_{tc}.bin"
    with open(path, "wb") as f:
        has_c = prob.get("c") is not None
        f.write(struct.pack("10q", 3, N, W, M, int(has_c), nnode, esz, len(IDS), sched, tc))
        f.write(struct.pack("4d", 1.0 / N, *prob["b"]))
        f.write(np.asarray(prob["a"], dtype=np.float64).ravel().tobytes())
        f.write((np.asarray(prob["c"], dtype=np.float64).ravel() if has_c else np.zeros(nnode)).tobytes())
        f.write(struct.pack(f"{len(IDS)}i", *IDS))
        f.write(b.tobytes())
    out = path.with_suffix(".out")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stderr[-3000:]
    raw = np.fromfile(out, dtype=np.float64)
    res, pos = {}, 0
    nP, st = M // 128, 2 * 128 * 128
    sizes = []
    if esz == 4:
        sizes = [("Sig1", nfac), ("Piv1", nfac), ("Cs", len(IDS) * nP * st), ("Xs", len(IDS) * nP * st),
                 ("Rs", len(IDS) * nP * st), ("Ps", len(IDS) * st)]
    sizes += [("F", nfac), ("x", nloc), ("xT", nloc), ("iface", nds * ng)]
    for key, cnt in sizes:
        res[key] = raw[pos:pos + cnt]
        pos += cnt
    res["code"] = raw[pos]
    assert pos + 1 == raw.size
    for key in ("Sig1", "Piv1", "F"):
        if key in res:
            res[key] = res[key].reshape(nds, nb, M, M)
    for key in ("x", "xT"):
        res[key] = res[key].reshape(nds, nb, M)
    A = sp.csr_matrix(O.assemble(prob)[0])
    geo = O.slab_geometry(3, N, W)
    return res, dict(A=A, geo=geo, p=p, m=m, M=M, nb=nb, nds=nds, ng=ng, b=b, nP=nP, w=W, ids=IDS)


def _local(ctx, j):
    w2 = 2 * ctx["w"] - 1
    Ij = np.asarray(ctx["geo"].I[j]).reshape(w2, ctx["nb"], ctx["p"]).transpose(1, 0, 2).ravel()
    return sp.csr_matrix(ctx["A"][Ij][:, Ij])


def _one_sided_lu(Aj, nb, m):
    """F_k = Sigma_k^{-1}, Sigma_1 = D_1, Sigma_k = D_k - L_k Sigma_{k-1}^{-1} U_{k-1}."""
    blk = lambda a, c: Aj[a * m:(a + 1) * m, c * m:(c + 1) * m].toarray()
    F = []
    for k in range(nb):
        S = blk(k, k)
        if k:
            S = S - blk(k, k - 1) @ F[-1] @ blk(k - 1, k)
        F.append(np.linalg.inv(S))
    return F


@pytest.fixture(scope="module")
def fp64_runs(harness):
    with ThreadPoolExecutor(max_workers=2) as ex:   # two host processes side by side
        return list(ex.map(lambda sched: _run(harness, 8, sched, CFG64), (0, 1)))


def test_lookahead_orders_give_the_same_factors(fp64_runs):
    (r0, _), (r1, _) = fp64_runs
    assert r0["code"] == 0.0 and r1["code"] == 0.0
    assert np.array_equal(r0["F"], r1["F"])


@pytest.mark.parametrize("esz", [8, 4])
def test_large_block_factor_and_solves_on_the_host(harness, fp64_runs, esz):
    res, ctx = fp64_runs[0] if esz == 8 else _run(harness, 4, 0, CFG32)
    IDS, W = ctx["ids"], ctx["w"]
    assert res["code"] == 0.0
    m, M, nb, nds, ng, p = ctx["m"], ctx["M"], ctx["nb"], ctx["nds"], ctx["ng"], ctx["p"]
    u = 2.0 ** -53 if esz == 8 else 2.0 ** -24
    pad = np.diag(np.r_[np.zeros(m), np.ones(M - m)])
    for j in range(nds):
        if j not in IDS:                  # slabs not listed stay untouched
            assert not res["F"][j].any() and not res["x"][j].any() and not res["xT"][j].any()
            continue
        Aj = _local(ctx, j)
        Fr = _one_sided_lu(Aj, nb, m)
        for k in range(nb):
            got = res["F"][j, k]
            assert np.abs(got[:m, :m] - Fr[k]).max() <= 256 * u * np.abs(Fr[k]).max()
            rest = got.copy()
            rest[:m, :m] = 0.0
            assert np.array_equal(rest, pad)          # the padding is exactly the identity
        bj = ctx["b"][j, :, :m].ravel()
        # 1-norm condition number, estimated (Higham and Tisseur's block estimator)
        lu = spla.splu(sp.csc_matrix(Aj))
        inv = spla.LinearOperator(Aj.shape, matvec=lu.solve, rmatvec=lambda v: lu.solve(v, trans="T"),
                                  dtype=np.float64)
        cond = spla.onenormest(sp.csc_matrix(Aj)) * spla.onenormest(inv)
        for key, Am in (("x", Aj), ("xT", Aj.T.tocsr())):
            want = spla.spsolve(sp.csc_matrix(Am), bj)
            got = res[key][j]
            assert np.abs(got[:, :m].ravel() - want).max() <= 8 * cond * u * np.abs(want).max(), key
            assert np.all(got[:, m:] == 0.0)
        centre = res["x"][j][:, (W - 1) * p:W * p].ravel()
        assert np.array_equal(res["iface"][j * ng:(j + 1) * ng], centre)
    if esz == 4:
        _check_split_pivot(res, ctx)


def _split_index(r, k):
    """Float offset of element (r, k) of a split tile: 16-wide K chunks of 2048 floats, each in
    the K-major core-matrix layout (8 rows x 4 values, row groups every 128 floats)."""
    c = k % 16
    return (k // 16) * 2048 + (r >> 3) * 128 + (c >> 2) * 32 + (r & 7) * 4 + (c & 3)


def _decode(tile):
    idx = np.array([[_split_index(r, k) for k in range(128)] for r in range(128)])
    hi, lo = tile[:128 * 128][idx], tile[128 * 128:][idx]
    for v in (hi, lo):
        assert np.all(v.astype(np.float32).view(np.uint32) & 0x1FFF == 0)   # TF32 parts
    return hi + lo


def _check_split_pivot(res, ctx):
    """First pivot step (k = 1, panel 0) with split tiles: C tile b = X(B, 0), C tile 0 = P,
    XqT tile b = X(0, B)^T, Pinv = P^{-1}, RT tile 0 = P^{-T}, with X = Sigma_1 = D_1."""
    m, M, nb, nP = ctx["m"], ctx["M"], ctx["nb"], ctx["nP"]
    st = 2 * 128 * 128
    close = lambda got, want: np.all(np.abs(got - want) <= 2.0 ** -21 * np.abs(want))
    for y, j in enumerate(ctx["ids"]):
        Aj = _local(ctx, j)
        D1 = np.eye(M)
        D1[:m, :m] = Aj[:m, :m].toarray()
        X = res["Sig1"][j, 0]
        assert np.array_equal(X, D1.astype(np.float32).astype(np.float64))
        Pinv = res["Piv1"][j, 0][:128, :128]
        assert np.abs(Pinv - np.linalg.inv(X[:128, :128])).max() <= 1e-4 * np.abs(Pinv).max()
        for bb in range(nP):
            C = _decode(res["Cs"][(y * nP + bb) * st:(y * nP + bb + 1) * st])
            assert close(C, X[128 * bb:128 * (bb + 1), :128])
            if bb:
                Xt = _decode(res["Xs"][(y * nP + bb) * st:(y * nP + bb + 1) * st])
                assert close(Xt, X[:128, 128 * bb:128 * (bb + 1)].T)
        assert close(_decode(res["Ps"][y * st:(y + 1) * st]), Pinv)
        assert close(_decode(res["Rs"][y * nP * st:(y * nP + 1) * st]), Pinv.T)


@pytest.mark.parametrize("tc", [1, 2])
def test_large_block_tensor_core_factor_on_the_host(harness, tc):
    """The FP32 factorization with the row and update products on the tensor cores
    (`k_big_gemm_tc` on the tcgen05 model of `tests/hostemu/tcgen05_host.h`; 1: 3xTF32, 2: one
    TF32 product), its split-tile pivot copies and the next panel's operand tiles written by the
    update and row steps: F_k against the one-sided block LU, the padding exactly the identity,
    and (3xTF32) the solves against a sparse direct solve."""
    res, ctx = _run(harness, 4, 0, CFG32, tc)
    assert res["code"] == 0.0
    m, M, nb, nP = ctx["m"], ctx["M"], ctx["nb"], ctx["nP"]
    # 3xTF32: FP32 accuracy; TF32: one 11-bit operand rounding per panel product
    tol = 256 * 2.0 ** -24 if tc == 1 else 4 * nP * 2.0 ** -11
    pad = np.diag(np.r_[np.zeros(m), np.ones(M - m)])
    for j in ctx["ids"]:
        Aj = _local(ctx, j)
        Fr = _one_sided_lu(Aj, nb, m)
        for k in range(nb):
            got = res["F"][j, k]
            assert np.abs(got[:m, :m] - Fr[k]).max() <= tol * np.abs(Fr[k]).max()
            rest = got.copy()
            rest[:m, :m] = 0.0
            assert np.array_equal(rest, pad)
        if tc == 1:
            bj = ctx["b"][j, :, :m].ravel()
            lu = spla.splu(sp.csc_matrix(Aj))
            inv = spla.LinearOperator(Aj.shape, matvec=lu.solve,
                                      rmatvec=lambda v: lu.solve(v, trans="T"), dtype=np.float64)
            cond = spla.onenormest(sp.csc_matrix(Aj)) * spla.onenormest(inv)
            want = lu.solve(bj)
            assert np.abs(res["x"][j][:, :m].ravel() - want).max() <= 8 * cond * 2.0 ** -24 * np.abs(want).max()


def test_tensor_core_lookahead_orders_give_the_same_factors(harness):
    """Three panels (M = 384) on the tensor-core model, 3xTF32: the next panel's operand tiles
    are written by the update of its row and column blocks and by the row step, into the other
    parity's buffers, while the rest of the current panel's update still reads this parity's.
    Both legal orders give the same factors bit for bit, and they are the block LU's."""
    with ThreadPoolExecutor(max_workers=2) as ex:
        (r0, ctx), (r1, _) = ex.map(lambda sched: _run(harness, 4, sched, CFG64, 1), (0, 1))
    assert r0["code"] == 0.0 and r1["code"] == 0.0 and ctx["nP"] == 3
    assert np.array_equal(r0["F"], r1["F"])
    m, nb = ctx["m"], ctx["nb"]
    Fr = _one_sided_lu(_local(ctx, 1), nb, m)
    for k in range(nb):
        assert np.abs(r0["F"][1, k, :m, :m] - Fr[k]).max() <= 256 * 2.0 ** -24 * np.abs(Fr[k]).max()
