"""Kernels of the direct interface solver (block cyclic reduction of I - K, Sec. 4 "Direct
solvers"), compiled for the host from `csrc/bcr.cu` and run with one OS thread per CUDA thread
under AddressSanitizer (`tests/hostemu/cuda_host_shim.h`):
* `k_bcr_init`: a transfer block stored column by column becomes a padded row-major block scaled
  by a sign (identity for the diagonal blocks, padding included);
* `k_block_mv_n` / `k_block_mv_t`: y = x0 + coef (op(M_0) v_0 + op(M_1) v_1) over the first n
  rows of blocks with a larger leading dimension, with absent terms and absent x0, shared-memory
  staging on and off."""
import os
import re
import shutil
import struct
import subprocess

import numpy as np
import pytest

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
  int64_t h[6]; f.read((char*)h, 48);
  const int what = (int)h[0];
  if (what == 0) {  // k_bcr_init
    const int64_t n = h[1]; const int NG = (int)h[2], has_src = (int)h[3];
    const double sign = (double)h[4];
    std::vector<double> src(n * n), dst(NG * NG, -7.0);
    f.read((char*)src.data(), 8 * n * n);
    host_launch2d(NG / 32, NG / 32, 32, 8, [&] { k_bcr_init<double>(has_src ? src.data() : nullptr, n, dst.data(), NG, sign); });
    std::ofstream o(argv[2], std::ios::binary);
    o.write((const char*)dst.data(), 8 * NG * NG);
    return 0;
  }
  const int n = (int)h[1], ldm = (int)h[2], ntasks = (int)h[3], transpose = (int)h[4], staged = (int)h[5];
  std::vector<std::vector<double>> M(2 * ntasks, std::vector<double>(ldm * ldm)), v(2 * ntasks, std::vector<double>(n)),
      x0(ntasks, std::vector<double>(n)), y(ntasks, std::vector<double>(n, 0.0));
  std::vector<BlockMv<double>> tasks(ntasks);
  for (int q = 0; q < ntasks; ++q) {
    int64_t flags[3]; double coef; f.read((char*)flags, 24); f.read((char*)&coef, 8);
    for (int s2 = 0; s2 < 2; ++s2) { f.read((char*)M[2 * q + s2].data(), 8 * ldm * ldm); f.read((char*)v[2 * q + s2].data(), 8 * n); }
    f.read((char*)x0[q].data(), 8 * n);
    BlockMv<double> t{};
    t.y = y[q].data(); t.x0 = flags[2] ? x0[q].data() : nullptr; t.coef = coef;
    for (int s2 = 0; s2 < 2; ++s2) {
      t.M[s2] = flags[s2] ? M[2 * q + s2].data() : nullptr;
      t.v[s2] = flags[s2] ? v[2 * q + s2].data() : nullptr;
    }
    tasks[q] = t;
  }
  std::vector<double> dyn(staged ? 2 * n : 1);
  host_dynamic_vs = dyn.data();
  if (!transpose)
    host_launch2((n + 7) / 8, ntasks, 256, [&] { k_block_mv_n<double>(tasks.data(), n, ldm, staged); });
  else
    host_launch2((n + 31) / 32, ntasks, 256, [&] { k_block_mv_t<double>(tasks.data(), n, ldm); });
  std::ofstream o(argv[2], std::ios::binary);
  for (int q = 0; q < ntasks; ++q) o.write((const char*)y[q].data(), 8 * n);
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "bcr.cu")).read()
    kh = open(os.path.join(CSRC, "kernels.cuh")).read()
    bmv = re.search(r"template <typename T>\nstruct BlockMv \{.*?\n\};", kh, re.S).group(0)
    i = src.index("template <typename T>\n__global__ void __launch_bounds__(256) k_bcr_init(")
    j = src.index("template <typename T>\nvoid launch_block_mv(")
    body = src[i:j]
    dyn = "extern __shared__ double vs[];"
    assert body.count(dyn) == 1
    body = body.replace(dyn, "double* vs = host_dynamic_vs;")
    d = tmp_path_factory.mktemp("bcr_host")
    code = ('#include "cuda_host_shim.h"\nstatic double* host_dynamic_vs = nullptr;\nnamespace ddst {\n' +
            bmv + "\n" + body + "\n}  // namespace ddst\n" + MAIN)
    (d / "bcr_host.cpp").write_text(code)
    exe = d / "bcr_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "bcr_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


def _run(d, exe, name, payload):
    path = d / name
    path.write_bytes(payload)
    out = d / (name + ".out")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.fromfile(out, dtype=np.float64)


@pytest.mark.parametrize("n,NG,has_src,sign", [(50, 64, 1, -1), (64, 64, 1, 1), (31, 64, 0, 1),
                                               (97, 128, 1, -1)])
def test_bcr_init_on_the_host(harness, n, NG, has_src, sign):
    d, exe = harness
    S = np.random.default_rng(n).standard_normal((n, n))
    payload = struct.pack("6q", 0, n, NG, has_src, sign, 0) + np.ascontiguousarray(S.T).tobytes()
    out = _run(d, exe, f"init_{n}_{NG}_{has_src}.bin", payload).reshape(NG, NG)
    want = np.zeros((NG, NG))
    if has_src:
        want[:n, :n] = sign * S
    else:
        want = np.eye(NG)
    assert np.array_equal(out, want)


@pytest.mark.parametrize("n,ldm,transpose,staged", [(100, 128, 0, 1), (100, 128, 0, 0),
                                                    (37, 64, 1, 0), (128, 128, 1, 0),
                                                    (200, 256, 0, 1)])
def test_block_products_on_the_host(harness, n, ldm, transpose, staged):
    d, exe = harness
    rng = np.random.default_rng(n + ldm + transpose)
    flags_list = [(1, 1, 1), (1, 0, 0), (0, 1, 1), (0, 0, 1)]  # M_0, M_1, x0 present
    payload = struct.pack("6q", 1, n, ldm, len(flags_list), transpose, staged)
    want = []
    for fl in flags_list:
        coef = float(rng.standard_normal())
        Ms = [rng.standard_normal((ldm, ldm)) for _ in range(2)]
        vs = [rng.standard_normal(n) for _ in range(2)]
        x0 = rng.standard_normal(n)
        payload += struct.pack("3q", *fl) + struct.pack("d", coef)
        for M, v in zip(Ms, vs):
            payload += np.ascontiguousarray(M).tobytes() + v.tobytes()  # row-major, leading dim ldm
        payload += x0.tobytes()
        acc = np.zeros(n)
        for present, M, v in zip(fl[:2], Ms, vs):
            if present:
                acc += (M[:n, :n].T if transpose else M[:n, :n]) @ v
        want.append((x0 if fl[2] else 0.0) + coef * acc)
    out = _run(d, exe, f"mv_{n}_{ldm}_{transpose}_{staged}.bin", payload).reshape(len(flags_list), n)
    for q, w in enumerate(want):
        assert np.abs(out[q] - w).max() <= 1e-12 * max(1.0, np.abs(w).max())
