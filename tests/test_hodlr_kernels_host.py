"""The tiled transposed product of the HODLR compression's power iteration (`k_sblk_gemv_t`,
y_b = S_b^T x_b for every dense transfer block, Sec. 2.4's ||S||_2 estimate) compiled for the host
from `csrc/hodlr.cu` and run with one OS thread per CUDA thread under AddressSanitizer
(`tests/hostemu/cuda_host_shim.h`), against the plain product on blocks with ragged tiles."""
import os
import re
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_25991_gb300", "csrc")

MAIN = r'''
#include <fstream>
using namespace ddst;
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  int64_t h[2]; f.read((char*)h, 16);
  const int nb = (int)h[0]; const int64_t stride = h[1];
  std::vector<SBlk> sb(nb);
  int64_t tot = 0, maxng = 0;
  for (auto& b : sb) { int64_t a[2]; f.read((char*)a, 16); b.off = a[0]; b.ng = a[1]; tot = std::max(tot, a[0] + a[1] * a[1]); maxng = std::max(maxng, a[1]); }
  std::vector<double> S(tot), x(nb * stride), y(nb * stride, 0.0);
  f.read((char*)S.data(), 8 * tot); f.read((char*)x.data(), 8 * nb * stride);
  const unsigned gz = (unsigned)((maxng + 127) / 128);
  host_launch2(gz, nb, 256, [&] { k_sblk_gemv_t<double>(sb.data(), S.data(), x.data(), y.data(), stride); });
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)y.data(), 8 * nb * stride);
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "hodlr.cu")).read()
    sblk = re.search(r"struct SBlk \{.*?\n\};", src, re.S).group(0)
    i = src.index("// y = S^T x for every S block")
    j = src.index("// x_b <- y_b / ||y_b||")
    d = tmp_path_factory.mktemp("hodlr_host")
    code = ('#include "cuda_host_shim.h"\nnamespace ddst {\n' + sblk + "\n" + src[i:j] +
            "\n}  // namespace ddst\n" + MAIN)
    (d / "sblk_host.cpp").write_text(code)
    exe = d / "sblk_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", "-fsanitize=address",
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "sblk_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


@pytest.mark.parametrize("ngs", [(300, 129), (31,), (128, 257, 64)])
def test_transposed_block_products_on_the_host(harness, ngs):
    d, exe = harness
    rng = np.random.default_rng(sum(ngs))
    stride = max(ngs)
    blocks, offs, off = [], [], 0
    for ng in ngs:
        blocks.append(rng.standard_normal((ng, ng)))
        offs.append(off)
        off += ng * ng
    x = rng.standard_normal((len(ngs), stride))
    path = d / ("case_" + "_".join(map(str, ngs)) + ".bin")
    with open(path, "wb") as f:
        f.write(struct.pack("2q", len(ngs), stride))
        for o, ng in zip(offs, ngs):
            f.write(struct.pack("2q", o, ng))
        for B in blocks:
            f.write(np.ascontiguousarray(B.T).tobytes())  # column-major, as the library stores S
        f.write(x.tobytes())
    out = d / (path.name + ".y")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    y = np.fromfile(out, dtype=np.float64).reshape(len(ngs), stride)
    for q, (B, ng) in enumerate(zip(blocks, ngs)):
        want = B.T @ x[q, :ng]
        assert np.abs(y[q, :ng] - want).max() <= 1e-12 * np.abs(want).max()
