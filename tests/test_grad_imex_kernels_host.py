"""Two global-grid kernels with oracle counterparts, compiled for the host and run with one OS
thread per CUDA thread under AddressSanitizer (`tests/hostemu/cuda_host_shim.h`) on a batch of
a 2D convection, a 2D Helmholtz and a 3D problem:
* `k_gradients` (`csrc/grad.cu`): dL/dg and nodal dL/da of the discrete adjoint from u and
  lambda, accumulated with atomics, against O7's `gradients`;
* `k_imex_rhs` (`csrc/stencil.cu`): the explicit right-hand side U_n/dt - v . grad_h U_n of one
  backward-Euler step (Sec. 6, Example 1), against O8's `imex_rhs`."""
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
  int64_t h[3]; f.read((char*)h, 24);
  const int nprob = (int)h[0]; const int64_t nvol = h[1], nnode = h[2];
  double inv_dt; f.read((char*)&inv_dt, 8);
  std::vector<ProbDesc> probs(nprob);
  for (auto& P : probs) {
    int64_t a[6]; double d[4]; f.read((char*)a, 48); f.read((char*)d, 32);
    P = ProbDesc{};
    P.dim = (int)a[0]; P.n = (int)a[1]; P.nint = a[2]; P.nnode = a[3]; P.vol_off = a[4]; P.node_off = a[5];
    P.h = d[0]; P.b[0] = d[1]; P.b[1] = d[2]; P.b[2] = d[3];
  }
  std::vector<double> A(nnode), G(nnode), U(nvol), L(nvol), vel(3 * nnode), dg(nnode, 0.0), da(nnode, 0.0), fr(nvol, 0.0);
  f.read((char*)A.data(), 8 * nnode); f.read((char*)G.data(), 8 * nnode);
  f.read((char*)U.data(), 8 * nvol); f.read((char*)L.data(), 8 * nvol); f.read((char*)vel.data(), 8 * 3 * nnode);
  host_launch2(3, nprob, 256, [&] { k_gradients(probs.data(), A.data(), G.data(), U.data(), L.data(), dg.data(), da.data()); });
  host_launch2(3, nprob, 256, [&] { k_imex_rhs(probs.data(), U.data(), vel.data(), nnode, inv_dt, fr.data()); });
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)dg.data(), 8 * nnode); o.write((const char*)da.data(), 8 * nnode);
  o.write((const char*)fr.data(), 8 * nvol);
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    grad = open(os.path.join(CSRC, "grad.cu")).read()
    sten = open(os.path.join(CSRC, "stencil.cu")).read()
    common = open(os.path.join(CSRC, "common.cuh")).read()
    prob = re.search(r"struct ProbDesc \{.*?\n\};", common, re.S).group(0)
    g0 = grad.index("__device__ __forceinline__ int64_t nidx(")
    g1 = grad.index("void launch_gradients(")
    s0 = sten.index("// IMEX right-hand side of one backward-Euler step")
    s1 = sten.index("// y = a*x + y  (FP64)")
    d = tmp_path_factory.mktemp("grad_imex_host")
    code = ('#include "cuda_host_shim.h"\nnamespace ddst {\n' + prob + "\n" + grad[g0:g1] + "\n" +
            sten[s0:s1] + "\n}  // namespace ddst\n" + MAIN)
    (d / "grad_imex_host.cpp").write_text(code)
    exe = d / "grad_imex_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "grad_imex_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


def test_gradients_and_imex_rhs_on_the_host_match_the_oracle(harness):
    d, exe = harness
    probs = [I.make_problem("convdiff2d", n=20, w=5), I.make_problem("helmholtz2d", n=16, w=4),
             I.make_problem("vardiff3d", n=8, w=2)]
    rng = np.random.default_rng(4)
    dt = 6.94e-3
    hdr, A_, G_, U_, L_, V_ = b"", [], [], [], [], []
    vol_off = node_off = 0
    offs = []
    for p in probs:
        dim, n = p["dim"], p["n"]
        nint, nnode = (n - 1) ** dim, (n + 1) ** dim
        bb = list(p["b"]) + [0.0] * (3 - len(p["b"]))
        hdr += struct.pack("6q", dim, n, nint, nnode, vol_off, node_off) + struct.pack("4d", 1.0 / n, *bb)
        A_.append(np.asarray(p["a"]).ravel())
        G_.append(np.asarray(p["g"]).ravel())
        U_.append(rng.standard_normal(nint))
        L_.append(rng.standard_normal(nint))
        V_.append([rng.standard_normal(nnode) for _ in range(3)])
        offs.append((vol_off, nint, node_off, nnode))
        vol_off += nint
        node_off += nnode
    vel = np.zeros((3, node_off))
    for (o, nint, no, nnode), v in zip(offs, V_):
        for c in range(3):
            vel[c, no:no + nnode] = v[c]
    path = d / "case.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("3q", len(probs), vol_off, node_off) + struct.pack("d", 1.0 / dt) + hdr)
        for arrs in (A_, G_, U_, L_):
            f.write(np.concatenate(arrs).astype(np.float64).tobytes())
        f.write(vel.tobytes())
    out = d / "case.out"
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    raw = np.fromfile(out, dtype=np.float64)
    dg, da, fr = raw[:node_off], raw[node_off:2 * node_off], raw[2 * node_off:]
    for q, (p, (o, nint, no, nnode)) in enumerate(zip(probs, offs)):
        dLdf, dLdg, dLda = O.gradients(p, U_[q], L_[q])
        assert np.abs(dg[no:no + nnode] - np.ravel(dLdg)).max() <= 1e-11 * np.abs(dLdg).max()
        assert np.abs(da[no:no + nnode] - np.ravel(dLda)).max() <= 1e-11 * np.abs(dLda).max()
        dim, n = p["dim"], p["n"]
        want = O.imex_rhs(dim, n, U_[q], [V_[q][c].reshape((n + 1,) * dim) for c in range(dim)], dt)
        assert np.abs(fr[o:o + nint] - want).max() <= 1e-12 * np.abs(want).max()
