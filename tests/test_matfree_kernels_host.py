"""The matrix-free interface kernels of `csrc/matfree.cu`, compiled for the host and run with one
OS thread per CUDA thread under AddressSanitizer (`tests/hostemu/cuda_host_shim.h`).

Block row j of K x is one Dirichlet solve on the double slab Psi_j, read back on Gamma_j
(Sec. 2.2, Eq. (defS): S_{j,j'} = -R_{C_j} A_j(I_j,I_j)^{-1} A(I_j, J_{j,j'})); K^T x runs the
other way.  The test runs the library's kernels around the local solves and does the solves
itself, densely, on the oracle's assembled matrix (O1) in the slab-local order that the
library's gather kernel produces:
* `k_mf_rhs`: the neighbouring traces enter the local right-hand side;
* `k_mf_inject` and `k_mf_dirichlet_T`: x_j at the central plane, and the transposed coupling
  of the boundary planes onto Gamma_{j-1} and Gamma_{j+1};
* `k_mf_combine`: y = x - K x or y = K x on every interface.
K x and K^T x must equal the oracle's K (O3, O4) on a 2D convection problem and a 3D problem,
with the input taken through a device-side Krylov index (x + (k - 1) stride) and the slabs
listed in reverse order.
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

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_25991_gb300", "csrc")
# AddressSanitizer by default; DDST_HOST_SANITIZER=thread runs the same tests under
# ThreadSanitizer, which reports accesses of two threads that no barrier orders
SANITIZE = "-fsanitize=" + os.environ.get("DDST_HOST_SANITIZER", "address")

MAIN = r'''
#include <cstring>
#include <fstream>
#include <string>
using namespace ddst;
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  const bool post = std::string(argv[3]) == "post";
  int64_t h[6]; double d[4]; f.read((char*)h, 48); f.read((char*)d, 32);
  const int dim = (int)h[0], n = (int)h[1], w = (int)h[2], M = (int)h[3], has_c = (int)h[4];
  const int64_t nnode = h[5];
  ProbDesc P{}; P.dim = dim; P.n = n; P.w = w; P.nds = n / w - 1; P.has_c = has_c;
  P.h = d[0]; P.b[0] = d[1]; P.b[1] = d[2]; P.b[2] = d[3];
  const int p = dim == 2 ? 1 : n - 1, m = (2 * w - 1) * p, nb = n - 1, nds = P.nds;
  const int64_t ng = (int64_t)nb * p, nint = (int64_t)nb * nb * p, nloc = (int64_t)nds * nb * M;
  const int64_t nif = (int64_t)nds * ng;
  P.nint = nint; P.ng = ng;
  std::vector<SlabDesc> slabs(nds);
  for (int q = 0; q < nds; ++q) {
    SlabDesc s{};
    s.prob = 0; s.j = q + 1; s.M = M; s.m = m; s.nb = nb; s.p = p; s.w = w; s.n = n; s.ng = ng;
    s.pack_off = (int64_t)q * nb * PK_NFIELDS * M; s.loc_off = (int64_t)q * nb * M;
    s.vol_off = 0; s.node_off = 0; s.if_off = (int64_t)q * ng;
    slabs[q] = s;
  }
  std::vector<int> ids(nds);
  for (int q = 0; q < nds; ++q) ids[q] = nds - 1 - q;      // listed in reverse order
  const int kdev = 2;                                      // x = x0 + (kdev - 1) nif
  std::vector<double> A(nnode), C(nnode), x0(2 * nif);
  f.read((char*)A.data(), 8 * nnode); f.read((char*)C.data(), 8 * nnode);
  f.read((char*)x0.data(), 8 * 2 * nif);
  std::vector<double> pack((int64_t)nds * nb * PK_NFIELDS * M);
  host_launch2(nb, nds, 128, [&] { k_stencil_pack<double>(slabs.data(), &P, A.data(), C.data(), pack.data()); });
  std::ofstream o(argv[2], std::ios::binary);
  auto L = [&](std::function<void()> fn) { host_launch2(3, nds, 64, fn); };
  if (!post) {
    std::vector<double> vol(nint), gmap(nloc, -1.0), rhs(nloc, 0.0), inj(nloc, 0.0);
    for (int64_t e = 0; e < nint; ++e) vol[e] = (double)e;
    L([&] { k_gather<double>(slabs.data(), vol.data(), gmap.data()); });
    L([&] { k_mf_rhs<double>(slabs.data(), ids.data(), &P, pack.data(), x0.data(), &kdev, nif, rhs.data()); });
    L([&] { k_mf_inject<double>(slabs.data(), ids.data(), x0.data(), &kdev, nif, inj.data()); });
    for (auto* v : {&gmap, &rhs, &inj}) o.write((const char*)v->data(), 8 * v->size());
  } else {
    std::vector<double> zT(nloc), kx(nif), ktx(nif, 0.0), y0(nif, -7.0), y1(nif, -7.0), y2(nif, -7.0);
    f.read((char*)zT.data(), 8 * nloc); f.read((char*)kx.data(), 8 * nif);
    L([&] { k_mf_dirichlet_T<double>(slabs.data(), ids.data(), &P, pack.data(), zT.data(), ktx.data()); });
    L([&] { k_mf_combine(slabs.data(), ids.data(), x0.data(), &kdev, nif, kx.data(), y0.data(), 0); });
    L([&] { k_mf_combine(slabs.data(), ids.data(), x0.data(), &kdev, nif, kx.data(), y1.data(), 1); });
    L([&] { k_mf_combine(slabs.data(), ids.data(), x0.data(), &kdev, nif, ktx.data(), y2.data(), 0); });
    for (auto* v : {&ktx, &y0, &y1, &y2}) o.write((const char*)v->data(), 8 * v->size());
  }
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    st = open(os.path.join(CSRC, "stencil.cu")).read()
    mf = open(os.path.join(CSRC, "matfree.cu")).read()
    common = open(os.path.join(CSRC, "common.cuh")).read()
    structs = [re.search(r"struct %s \{.*?\n\};" % nme, common, re.S).group(0)
               for nme in ("ProbDesc", "SlabDesc")]
    enum = re.search(r"enum PackField \{.*?\};", common, re.S).group(0)
    vidx = re.search(r"__device__ __forceinline__ int64_t vol_index\(.*?\n\}", common, re.S).group(0)
    pack = st[st.index("__device__ __forceinline__ int64_t node_index("):
              st.index("// b = f + (Dirichlet neighbour terms)")]
    gather = st[st.index("// Slab-local gather:"):st.index("// Partial sums of x.y over n elements")]
    kern = mf[mf.index("__device__ __forceinline__ const double* eff("):
              mf.index("template <typename T>\nvoid launch_mf_rhs(")]
    d = tmp_path_factory.mktemp("matfree_host")
    code = ('#include "cuda_host_shim.h"\n#include <functional>\nnamespace ddst {\n' + enum + "\n" +
            "\n".join(structs) + "\n" + vidx + "\n" + pack + "\n" + gather + "\n" + kern +
            "\n}  // namespace ddst\n" + MAIN)
    (d / "mf_host.cpp").write_text(code)
    exe = d / "mf_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "mf_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


def _run(exe, path, mode):
    out = path.with_suffix("." + mode)
    r = subprocess.run([str(exe), str(path), str(out), mode], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.fromfile(out, dtype=np.float64)


@pytest.mark.parametrize("name,n,w", [("convdiff2d", 24, 4), ("vardiff3d", 8, 2)])
def test_matfree_kernels_on_the_host(harness, name, n, w):
    d, exe = harness
    over = {"b": (1.5, -1.0, 0.5)} if name == "vardiff3d" else {}
    prob = I.make_problem(name, n=n, w=w, **over)
    dim = prob["dim"]
    p = 1 if dim == 2 else n - 1
    m, nb = (2 * w - 1) * p, n - 1
    M = ((m + 31) // 32) * 32 + (32 if m % 32 == 0 else 0)
    geo = O.slab_geometry(dim, n, w)
    nds, ng = geo.nds, geo.ngamma
    nif, nloc = nds * ng, nds * nb * M
    rng = np.random.default_rng(7 * n)
    x0 = rng.standard_normal(2 * nif)
    x = x0[nif:]
    has_c = prob.get("c") is not None
    bb = list(prob["b"]) + [0.0] * (3 - len(prob["b"]))
    nnode = (n + 1) ** dim
    head = (struct.pack("6q", dim, n, w, M, int(has_c), nnode) + struct.pack("4d", 1.0 / n, *bb) +
            np.asarray(prob["a"], dtype=np.float64).ravel().tobytes() +
            (np.asarray(prob["c"], dtype=np.float64).ravel() if has_c else np.zeros(nnode)).tobytes() +
            x0.tobytes())
    path = d / f"mf_{name}.bin"
    path.write_bytes(head)
    gmap, rhs, inj = np.split(_run(exe, path, "pre"), [nloc, 2 * nloc])
    gmap, rhs, inj = (v.reshape(nds, nb, M) for v in (gmap, rhs, inj))

    A = sp.csr_matrix(O.assemble(prob)[0])
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo))
    K = np.eye(nif) - O.interface_matrix(Sp, Sn, ng)

    centre = (np.arange(nb)[:, None] * m + (w - 1) * p + np.arange(p)[None, :]).ravel()
    kx = np.zeros(nif)
    zT = np.zeros((nds, nb, M))
    for j in range(nds):
        gm = gmap[j, :, :m].ravel().astype(np.int64)
        assert np.array_equal(np.sort(gm), np.sort(geo.I[j]))
        Aj = A[gm][:, gm].toarray()
        z = np.linalg.solve(Aj, rhs[j, :, :m].ravel())
        kx[j * ng:(j + 1) * ng] = z[centre]
        assert np.all(inj[j, :, m:] == 0.0) and np.all(rhs[j, :, m:] == 0.0)
        zT[j, :, :m] = np.linalg.solve(Aj.T, inj[j, :, :m].ravel()).reshape(nb, m)
    scale = np.abs(x).max()
    assert np.abs(kx - K @ x).max() <= 1e-10 * scale

    path.write_bytes(head + zT.tobytes() + kx.tobytes())
    ktx, y0, y1, y2 = np.split(_run(exe, path, "post"), [nif, 2 * nif, 3 * nif])
    assert np.abs(ktx - K.T @ x).max() <= 1e-10 * scale
    assert np.array_equal(y0, x - kx)
    assert np.array_equal(y1, kx)
    assert np.abs(y2 - (x - K.T @ x)).max() <= 1e-10 * scale
