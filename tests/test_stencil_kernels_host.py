"""The FP64 global-grid kernels that the refinement's accuracy rests on (Sec. 1, Eq. (basic);
five-point stencil Sec. 2.1, seven-point Sec. 5.2): `k_rhs` (b = f + the Dirichlet neighbour
terms) and `k_residual` (r = b - A u or b - A^T u, with per-CTA partial sums of ||r||^2),
compiled for the host from `csrc/stencil.cu` and run with one OS thread per CUDA thread under
AddressSanitizer (`tests/hostemu/cuda_host_shim.h`) on a batch of problems of different sizes
and dimensions, against the oracle's assembled system (O1)."""
import os
import re
import shutil
import struct
import subprocess

import numpy as np
import pytest

import ddst_inputs as I
from oracle import ddst_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_25991_gb300", "csrc")
# AddressSanitizer by default; DDST_HOST_SANITIZER=thread runs the same tests under
# ThreadSanitizer, which reports accesses of two threads that no barrier orders
SANITIZE = "-fsanitize=" + os.environ.get("DDST_HOST_SANITIZER", "address")

MAIN = r'''
#include <fstream>
using namespace ddst;
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  int64_t h[4]; f.read((char*)h, 32);
  const int nprob = (int)h[0], transpose = (int)h[1]; const int64_t nvol = h[2], nnode = h[3];
  std::vector<ProbDesc> probs(nprob);
  for (auto& P : probs) {
    int64_t a[8]; double d[4]; f.read((char*)a, 64); f.read((char*)d, 32);
    P = ProbDesc{};
    P.dim = (int)a[0]; P.n = (int)a[1]; P.nint = a[2]; P.nnode = a[3]; P.vol_off = a[4];
    P.node_off = a[5]; P.has_c = (int)a[6];
    P.h = d[0]; P.b[0] = d[1]; P.b[1] = d[2]; P.b[2] = d[3];
  }
  std::vector<double> A(nnode), C(nnode), G(nnode), Fv(nvol), U(nvol), B(nvol, 0.0), R(nvol, 0.0);
  f.read((char*)A.data(), 8 * nnode); f.read((char*)C.data(), 8 * nnode); f.read((char*)G.data(), 8 * nnode);
  f.read((char*)Fv.data(), 8 * nvol); f.read((char*)U.data(), 8 * nvol);
  const unsigned nblk = 3;
  std::vector<double> part(nblk * nprob, 0.0);
  host_launch2(nblk, nprob, 256, [&] { k_rhs(probs.data(), A.data(), Fv.data(), G.data(), B.data()); });
  host_launch2(nblk, nprob, 256, [&] { k_residual(probs.data(), A.data(), C.data(), B.data(), U.data(), R.data(), transpose, part.data()); });
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)B.data(), 8 * nvol); o.write((const char*)R.data(), 8 * nvol);
  o.write((const char*)part.data(), 8 * nblk * nprob);
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
    prob = re.search(r"struct ProbDesc \{.*?\n\};", common, re.S).group(0)
    i = src.index("__device__ __forceinline__ int64_t node_index(")
    j = src.index("// Stencil pack of every (slab, block)")
    k0 = src.index("// b = f + (Dirichlet neighbour terms)")
    k1 = src.index("// Slab-local gather:")
    d = tmp_path_factory.mktemp("stencil_host")
    code = ('#include "cuda_host_shim.h"\nnamespace ddst {\n' + prob + "\n" + src[i:j] + "\n" +
            src[k0:k1] + "\n}  // namespace ddst\n" + MAIN)
    (d / "stencil_host.cpp").write_text(code)
    exe = d / "stencil_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "stencil_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


@pytest.mark.parametrize("transpose", [0, 1])
def test_rhs_and_residual_on_the_host_match_the_oracle(harness, transpose):
    d, exe = harness
    probs = [I.make_problem("convdiff2d", n=24, w=6), I.make_problem("helmholtz2d", n=16, w=4),
             I.make_problem("vardiff3d", n=10, w=2)]
    rng = np.random.default_rng(9 + transpose)
    hdr, A_, C_, G_, F_, U_ = b"", [], [], [], [], []
    vol_off = node_off = 0
    offs = []
    for p in probs:
        dim, n = p["dim"], p["n"]
        nint, nnode = (n - 1) ** dim, (n + 1) ** dim
        bb = list(p["b"]) + [0.0] * (3 - len(p["b"]))
        hdr += struct.pack("8q", dim, n, nint, nnode, vol_off, node_off, 1 if p.get("c") is not None else 0, 0)
        hdr += struct.pack("4d", 1.0 / n, *bb)
        A_.append(np.asarray(p["a"]).ravel())
        C_.append(np.asarray(p["c"]).ravel() if p.get("c") is not None else np.zeros(nnode))
        G_.append(np.asarray(p["g"]).ravel())
        F_.append(np.asarray(p["f"]).ravel())
        U_.append(rng.standard_normal(nint))
        offs.append((vol_off, nint))
        vol_off += nint
        node_off += nnode
    path = d / f"case_{transpose}.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("4q", len(probs), transpose, vol_off, node_off) + hdr)
        for arrs in (A_, C_, G_, F_, U_):
            f.write(np.concatenate(arrs).astype(np.float64).tobytes())
    out = d / (path.name + ".out")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    raw = np.fromfile(out, dtype=np.float64)
    B, R, part = raw[:vol_off], raw[vol_off:2 * vol_off], raw[2 * vol_off:].reshape(len(probs), -1)
    for q, (p, (o, nint)) in enumerate(zip(probs, offs)):
        A, b = O.assemble(p)
        assert np.abs(B[o:o + nint] - b).max() <= 1e-12 * np.abs(b).max()
        Am = A.T if transpose else A
        want = b - Am @ U_[q]
        assert np.abs(R[o:o + nint] - want).max() <= 1e-11 * np.abs(want).max()
        assert abs(part[q].sum() - want @ want) <= 1e-10 * (want @ want)
