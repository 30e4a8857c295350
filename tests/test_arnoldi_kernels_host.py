"""The GMRES step kernels (Arnoldi on K with classical Gram-Schmidt and a second pass when the
first cancels more than half of ||w||, then the Givens update of the (I - K) Hessenberg column:
`k_arn_dots`, `k_arn_update`, `k_arn_finish` of `csrc/krylov.cu`), compiled for the host and run
with one OS thread per CUDA thread under AddressSanitizer (`tests/hostemu/cuda_host_shim.h`) in
the order the library launches them, over vectors of several 1024-entry chunks with a ragged
tail, from the normalised start vector (`k_normalize_start`) to the solution (`k_trisolve`,
`k_combine_basis`).  The residual estimates and the solution equal those of the oracle's unrestarted GMRES on
I - K (O4; Sec. 5.2: x0 = 0, CGS2, Givens rotations): the Krylov spaces of K and I - K coincide."""
import os
import re
import shutil
import struct
import subprocess

import numpy as np
import pytest
import scipy.linalg as sla

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
  const int64_t n = h[0]; const int kmax = (int)h[1], maxit = (int)h[2];
  std::vector<double> K(n * n), b(n);
  f.read((char*)K.data(), 8 * n * n); f.read((char*)b.data(), 8 * n);
  const int nchunk = (int)((n + ARN_CHUNK - 1) / ARN_CHUNK), ldh = kmax + 1;
  std::vector<double> V((kmax + 1) * n, 0.0), w(n), h1(kmax + 1), h2(kmax + 1),
      part(3 * (int64_t)(kmax + 1) * nchunk), H((int64_t)ldh * kmax, 0.0), cs(kmax + 1), sn(kmax + 1),
      gv(kmax + 1, 0.0), resid(kmax, 0.0), beta(1);
  int kdev[2] = {1, 0};
  unsigned ticket = 0;
  double bn2 = 0.0;
  for (double v : b) bn2 += v * v;
  beta[0] = std::sqrt(bn2); gv[0] = beta[0];
  std::vector<double> dynbuf(kmax + 1);
  host_dynamic_smem = dynbuf.data();
  host_launch(4, 256, [&] { k_normalize_start(b.data(), &bn2, V.data(), n); });  // V[0] = b / ||b||
  double* P1 = part.data();
  double* P2 = P1 + (int64_t)(kmax + 1) * nchunk;
  double* Pn = P2 + (int64_t)(kmax + 1) * nchunk;
  for (int it = 0; it < maxit; ++it) {
    const int k = kdev[0];
    const double* v = V.data() + (int64_t)(k - 1) * n;
    for (int64_t r = 0; r < n; ++r) {  // w = K V[k-1]
      double a = 0.0;
      for (int64_t c = 0; c < n; ++c) a += K[r * n + c] * v[c];
      w[r] = a;
    }
    host_launch(nchunk, ARN_T, [&] { k_arn_dots(V.data(), w.data(), n, kdev, P1, nchunk); });
    host_launch(nchunk, ARN_T, [&] { k_arn_update(V.data(), w.data(), n, kdev, P1, h1.data(), P2, Pn, nchunk, 1); });
    host_launch(nchunk, ARN_T, [&] { k_arn_update(V.data(), w.data(), n, kdev, P2, h2.data(), nullptr, Pn, nchunk, 0); });
    host_launch(nchunk, ARN_T, [&] { k_arn_finish(V.data(), w.data(), n, kdev, Pn, nchunk, h1.data(), h2.data(), H.data(), ldh, cs.data(), sn.data(), gv.data(), beta.data(), resid.data(), kmax, &ticket); });
  }
  // the solution: R y = g by back substitution, then x = V y
  std::vector<double> y(maxit), x(n);
  host_launch(1, 256, [&] { k_trisolve(H.data(), ldh, gv.data(), maxit, y.data()); });
  host_launch(4, 256, [&] { k_combine_basis(V.data(), x.data(), y.data(), maxit, n); });
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)x.data(), 8 * n);
  o.write((const char*)resid.data(), 8 * maxit);
  o.write((const char*)gv.data(), 8 * (maxit + 1));
  o.write((const char*)H.data(), 8 * (int64_t)ldh * kmax);
  o.write((const char*)V.data(), 8 * (int64_t)(kmax + 1) * n);
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "krylov.cu")).read()
    i = src.index("constexpr int ARN_T")
    j = src.index("int arnoldi_chunks(int64_t n)")
    s0 = src.index("// GMRES solution from the Krylov basis")
    s1 = src.index("// ---- Arnoldi step with device-resident state")
    sol = src[s0:s1]
    for dyn in ("extern __shared__ double sh[];", "extern __shared__ double rhs[];"):
        assert sol.count(dyn) == 1
        sol = sol.replace(dyn, "double* %s = host_dynamic_smem;" % dyn.split()[-1][:-3])
    d = tmp_path_factory.mktemp("arnoldi_host")
    code = ('#include "cuda_host_shim.h"\nusing std::sqrt; using std::fmax; using std::hypot; using std::fabs;\n'
            "static double* host_dynamic_smem = nullptr;\n"
            "namespace ddst {\n" + sol + "\n" + src[i:j] + "\n}  // namespace ddst\n" + MAIN)
    (d / "arnoldi_host.cpp").write_text(code)
    exe = d / "arnoldi_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "arnoldi_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


@pytest.mark.parametrize("n,rho,shift", [(2100, 0.8, 0.0), (1024, 0.95, 0.0), (2100, 0.6, 0.85)])
def test_gmres_step_kernels_on_the_host_match_the_oracle(harness, n, rho, shift):
    """shift: K = shift I + (1 - shift) K0 makes K V[k-1] lie mostly in span(V), so the first
    Gram-Schmidt pass cancels most of ||w|| and the second pass (`arn_chunk_dots`) runs."""
    d, exe = harness
    rng = np.random.default_rng(n)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    ev = rho * np.exp(2j * np.pi * rng.random(n // 2))  # eigenvalues of K inside a disc
    blocks = [np.array([[e.real, e.imag], [-e.imag, e.real]]) for e in ev]
    K = Q @ sla.block_diag(*blocks) @ Q.T
    if K.shape[0] < n:
        K = sla.block_diag(K, np.eye(n - K.shape[0]) * 0.5)
    K = shift * np.eye(n) + (1.0 - shift) * K
    b = rng.standard_normal(n)
    kmax, maxit = 40, 24
    path = d / f"case_{n}_{shift}.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("3q", n, kmax, maxit))
        f.write(np.ascontiguousarray(K).tobytes())
        f.write(b.tobytes())
    out = d / (path.name + ".out")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    raw = np.fromfile(out, dtype=np.float64)
    x_k, raw = raw[:n], raw[n:]
    resid = raw[:maxit]
    gv = raw[maxit:2 * maxit + 1]
    H = raw[2 * maxit + 1:2 * maxit + 1 + (kmax + 1) * kmax].reshape(kmax, kmax + 1).T
    V = raw[2 * maxit + 1 + (kmax + 1) * kmax:].reshape(kmax + 1, n)
    x_o, its, hist = O.gmres(lambda v: v - K @ v, b, tol=0.0, maxit=maxit)
    assert its == maxit
    hist = np.array(hist[1:])
    assert np.all(np.abs(resid - hist) <= 1e-8 * hist + 1e-14), np.abs(resid - hist).max()
    y = sla.solve_triangular(H[:maxit, :maxit], gv[:maxit])
    x = V[:maxit].T @ y
    assert np.linalg.norm(x - x_o) <= 1e-9 * np.linalg.norm(x_o)
    # the library's own solution kernels (back substitution, basis combination)
    assert np.linalg.norm(x_k - x_o) <= 1e-9 * np.linalg.norm(x_o)
