"""The local operator of every double slab (a1: A_j(I_j, I_j) of Sec. 2.2, Eq. (defS), ordered
along y as block-tridiagonal with diagonal couplings, Alg. 2): `k_stencil_pack` of
`csrc/stencil.cu`, compiled for the host and run with one OS thread per CUDA thread under
AddressSanitizer (`tests/hostemu/cuda_host_shim.h`).  Every entry its pack encodes (diagonal,
x, y and z couplings, and the couplings to the neighbouring interfaces) must equal the oracle's
assembled matrix (O1) at the same global unknowns; padding rows hold the identity."""
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
NF = 7  # diag, west, east, south, north, zlo, zhi

MAIN = r'''
#include <fstream>
using namespace ddst;
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  int64_t h[6]; double d[4]; f.read((char*)h, 48); f.read((char*)d, 32);
  const int dim = (int)h[0], n = (int)h[1], w = (int)h[2], M = (int)h[3], has_c = (int)h[4];
  const int64_t nnode = h[5];
  ProbDesc P{}; P.dim = dim; P.n = n; P.w = w; P.nds = n / w - 1; P.has_c = has_c;
  P.h = d[0]; P.b[0] = d[1]; P.b[1] = d[2]; P.b[2] = d[3];
  const int p = dim == 2 ? 1 : n - 1, m = (2 * w - 1) * p, nb = n - 1;
  std::vector<SlabDesc> slabs(P.nds);
  for (int q = 0; q < P.nds; ++q) {
    SlabDesc s{};
    s.prob = 0; s.j = q + 1; s.M = M; s.m = m; s.nb = nb; s.p = p; s.w = w; s.n = n;
    s.pack_off = (int64_t)q * nb * NFIELDS * M; s.node_off = 0;
    slabs[q] = s;
  }
  std::vector<double> A(nnode), C(nnode), pack((int64_t)P.nds * nb * NFIELDS * M, -99.0);
  f.read((char*)A.data(), 8 * nnode); f.read((char*)C.data(), 8 * nnode);
  host_launch2(nb, P.nds, 128, [&] { k_stencil_pack<double>(slabs.data(), &P, A.data(), C.data(), pack.data()); });
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)pack.data(), 8 * pack.size());
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "stencil.cu")).read()
    common = open(os.path.join(CSRC, "common.cuh")).read()
    structs = [re.search(r"struct %s \{.*?\n\};" % nme, common, re.S).group(0)
               for nme in ("ProbDesc", "SlabDesc")]
    enum = re.search(r"enum PackField \{.*?\};", common, re.S).group(0)
    i = src.index("__device__ __forceinline__ int64_t node_index(")
    j = src.index("// b = f + (Dirichlet neighbour terms)")
    d = tmp_path_factory.mktemp("pack_host")
    code = ('#include "cuda_host_shim.h"\nnamespace ddst {\n' + enum + "\n" + "\n".join(structs) +
            "\n" + src[i:j] + "\n}  // namespace ddst\nconstexpr int NFIELDS = ddst::PK_NFIELDS;\n" + MAIN)
    (d / "pack_host.cpp").write_text(code)
    exe = d / "pack_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "pack_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


@pytest.mark.parametrize("name,n,w,over", [("convdiff2d", 16, 4, {}), ("helmholtz2d", 12, 3, {}),
                                           ("vardiff3d", 8, 2, {"b": (1.5, -2.0, 3.0)})])
def test_stencil_pack_on_the_host_matches_the_oracle(harness, name, n, w, over):
    d, exe = harness
    prob = I.make_problem(name, n=n, w=w, **over)
    dim = prob["dim"]
    p = 1 if dim == 2 else n - 1
    m, nb, nds = (2 * w - 1) * p, n - 1, n // w - 1
    M = ((m + 31) // 32) * 32 + (32 if m % 32 == 0 else 0)  # padding rows included
    has_c = prob.get("c") is not None
    bb = list(prob["b"]) + [0.0] * (3 - len(prob["b"]))
    nnode = (n + 1) ** dim
    path = d / f"pack_{name}.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("6q", dim, n, w, M, int(has_c), nnode) + struct.pack("4d", 1.0 / n, *bb))
        f.write(np.asarray(prob["a"], dtype=np.float64).ravel().tobytes())
        f.write((np.asarray(prob["c"], dtype=np.float64).ravel() if has_c else np.zeros(nnode)).tobytes())
    out = d / (path.name + ".out")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    pack = np.fromfile(out, dtype=np.float64).reshape(nds, nb, NF, M)
    A = sp.csr_matrix(O.assemble(prob)[0])
    scale = abs(A).max()

    def gidx(j, cx, k, t):  # global interior index of local unknown (cx, k, t) of slab j
        i = (j - 1) * w + 1 + cx
        return ((i - 1) * (n - 1) + (k - 1)) * p + t

    for j in range(1, nds + 1):
        for k in range(1, nb + 1):
            f = pack[j - 1, k - 1]
            assert np.all(f[0, m:] == 1.0) and np.all(f[1:, m:] == 0.0)  # identity padding
            for c in range(m):
                cx, t = divmod(c, p)
                g = gidx(j, cx, k, t)
                want = {0: A[g, g]}
                # x couplings: inside the slab, or to the neighbouring interface planes
                if cx > 0 or j > 1:
                    want[1] = A[g, gidx(j, cx - 1, k, t)]
                if cx < 2 * w - 2 or j < nds:
                    want[2] = A[g, gidx(j, cx + 1, k, t)]
                want[3] = A[g, gidx(j, cx, k - 1, t)] if k > 1 else 0.0
                want[4] = A[g, gidx(j, cx, k + 1, t)] if k < nb else 0.0
                if dim == 3:
                    want[5] = A[g, g - 1] if t > 0 else 0.0
                    want[6] = A[g, g + 1] if t < p - 1 else 0.0
                else:
                    want[5] = want[6] = 0.0
                for q, v in want.items():
                    assert abs(f[q, c] - v) <= 1e-12 * scale, (j, k, c, q, f[q, c], v)
