"""The dense interface operator (Sec. 1, Eq. (modelS)): `k_apply_dense` (y = (I - K) x, or K x)
and the tiled transposed `k_apply_dense_T` ((I - K)^T x, or K^T x), compiled for the host from
`csrc/krylov.cu` and run with one OS thread per CUDA thread under AddressSanitizer
(`tests/hostemu/cuda_host_shim.h`), against the oracle's dense I - K (O4) on a chain of double
slabs with ragged tiles, including a slab whose neighbour holds no explicit block."""
import os
import re
import shutil
import struct
import subprocess

import numpy as np
import pytest

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
  const int nds = (int)h[0]; const int64_t ng = h[1], nS = h[2]; const int mode = (int)h[3];
  std::vector<SlabDesc> slabs(nds);
  for (int q = 0; q < nds; ++q) {
    int64_t a[2]; f.read((char*)a, 16);
    SlabDesc s{};
    s.prob = 0; s.j = q + 1; s.ng = ng; s.sp_off = a[0]; s.sn_off = a[1]; s.if_off = q * ng;
    slabs[q] = s;
  }
  ProbDesc P{}; P.nds = nds; P.ng = ng;
  std::vector<double> S(nS), x(nds * ng), y(nds * ng, 0.0);
  f.read((char*)S.data(), 8 * nS); f.read((char*)x.data(), 8 * nds * ng);
  const int transpose = mode & 1, konly = mode >> 1;
  const unsigned gx = (unsigned)((ng + 127) / 128);
  std::vector<unsigned char> dyn((transpose ? 2 * ng + 128 * 33 : 2 * ng) * sizeof(double));
  host_dynamic_smem = dyn.data();
  if (!transpose)
    host_launch2(gx, nds, 256, [&] { k_apply_dense<double>(slabs.data(), &P, S.data(), x.data(), y.data(), nullptr, 0, konly); });
  else
    host_launch2(gx, nds, 256, [&] { k_apply_dense_T<double>(slabs.data(), &P, S.data(), x.data(), y.data(), nullptr, 0, konly, ng); });
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)y.data(), 8 * nds * ng);
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "krylov.cu")).read()
    common = open(os.path.join(CSRC, "common.cuh")).read()
    structs = [re.search(r"struct %s \{.*?\n\};" % n, common, re.S).group(0)
               for n in ("ProbDesc", "SlabDesc")]
    i = src.index("// y_j = x_j - S_{j,j-1} x_{j-1} - S_{j,j+1} x_{j+1}")
    j = src.index("// GMRES solution from the Krylov basis")
    body = src[i:j]
    dyn = "extern __shared__ __align__(16) unsigned char smem_raw[];"
    assert body.count(dyn) == 2
    body = body.replace(dyn, "unsigned char* smem_raw = host_dynamic_smem;")
    d = tmp_path_factory.mktemp("krylov_host")
    code = ('#include "cuda_host_shim.h"\nstatic unsigned char* host_dynamic_smem = nullptr;\n'
            "namespace ddst {\n" + "\n".join(structs) + "\n" + body + "\n}  // namespace ddst\n" + MAIN)
    (d / "krylov_host.cpp").write_text(code)
    exe = d / "krylov_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "krylov_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


@pytest.mark.parametrize("nds,ng,missing", [(4, 150, None), (3, 31, None), (5, 129, 2)])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_dense_interface_apply_on_the_host(harness, nds, ng, missing, mode):
    """mode bit 0: transposed; bit 1: K alone.  `missing`: slab whose S_{j,j+1} is absent (a
    neighbour applied matrix-free contributes nothing to the explicit apply)."""
    d, exe = harness
    rng = np.random.default_rng(nds * 1000 + ng + mode)
    Sp = [None] + [rng.standard_normal((ng, ng)) for _ in range(nds - 1)]
    Sn = [rng.standard_normal((ng, ng)) for _ in range(nds - 1)] + [None]
    if missing is not None:
        Sn[missing] = None
    blocks, offs = [], []
    off = 0
    for q in range(nds):
        o = []
        for B in (Sp[q], Sn[q]):
            if B is None:
                o.append(-1)
            else:
                o.append(off)
                blocks.append(np.ascontiguousarray(B.T).ravel())  # column-major
                off += ng * ng
        offs.append(o)
    x = rng.standard_normal(nds * ng)
    path = d / f"case_{nds}_{ng}_{missing}_{mode}.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("4q", nds, ng, off, mode))
        for o in offs:
            f.write(struct.pack("2q", *o))
        f.write(np.concatenate(blocks).tobytes())
        f.write(x.tobytes())
    out = d / (path.name + ".y")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    y = np.fromfile(out, dtype=np.float64)
    M = O.interface_matrix(Sp, Sn, ng)
    if mode & 1:
        M = M.T
    want = M @ x
    if mode & 2:
        want = x - want  # K x (or K^T x)
    assert np.abs(y - want).max() <= 1e-12 * np.abs(want).max()
