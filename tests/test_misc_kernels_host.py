"""Two more kernels compiled for the host and run with one OS thread per CUDA thread under
AddressSanitizer (`tests/hostemu/cuda_host_shim.h`):
* `k_residual_noalloc` + `k_norms_noalloc` (`csrc/noalloc.cu`): r = b(f, g) - A u with ||r||,
  ||b|| over 256-unknown partial sums, against the oracle's assembled system (O1), in 2D with
  convection and reaction and in 3D;
* `k_gemm_fma` (`csrc/gemm_tc.cu`, the FP64 block products of the direct interface solver):
  C = alpha A B (+ C) on 128-wide tiles, against the plain product;
* the FP64 reductions of `csrc/stencil.cu` (`k_dot_partial` + `k_sum_partials`: the inner
  products of the refinement; `k_prob_sqnorm_partial` + `k_sum_partials`: per-problem squared
  norms of a batch) and `k_axpy`, on ragged lengths, against numpy;
* `k_pack_split` (`csrc/gemm_tc.cu`): the TF32 hi/lo operand tiles of the tensor-core product;
* `k_hbs_cvt` (`csrc/hbs.cu`): caller-given test matrices into the working precision."""
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

NOALLOC_MAIN = r'''
#include <fstream>
using namespace ddst;
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  int64_t h[4]; double bc[3]; f.read((char*)h, 32); f.read((char*)bc, 24);
  const int dim = (int)h[0], n = (int)h[1], has_c = (int)h[2]; const int64_t nnode = h[3];
  int64_t ni = 1; for (int d = 0; d < dim; ++d) ni *= (n - 1);
  std::vector<double> a(nnode), c(nnode), g(nnode), fv(ni), u(ni), r(ni), part(2 * kNoallocMaxBlocks, 0.0), norms(2);
  f.read((char*)a.data(), 8 * nnode); f.read((char*)c.data(), 8 * nnode); f.read((char*)g.data(), 8 * nnode);
  f.read((char*)fv.data(), 8 * ni); f.read((char*)u.data(), 8 * ni);
  const unsigned nblk = (unsigned)((ni + kNoallocThreads - 1) / kNoallocThreads);
  host_launch(nblk, kNoallocThreads, [&] { k_residual_noalloc(dim, n, bc[0], bc[1], bc[2], a.data(), has_c ? c.data() : nullptr, fv.data(), g.data(), u.data(), r.data(), part.data(), ni); });
  host_launch(1, 256, [&] { k_norms_noalloc(part.data(), (int)nblk, norms.data()); });
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)r.data(), 8 * ni); o.write((const char*)norms.data(), 16);
  return 0;
}
'''

GEMM_MAIN = r'''
#include <fstream>
using namespace ddst;
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  int64_t h[2]; f.read((char*)h, 16);
  const int nT = (int)h[0], ntasks = (int)h[1]; const int64_t ld = (int64_t)nT * BT;
  std::vector<std::vector<double>> A(ntasks, std::vector<double>(ld * ld)), B = A, Cm = A;
  std::vector<GemmTaskT<double>> tasks(ntasks);
  for (int q = 0; q < ntasks; ++q) {
    double alpha; int64_t acc; f.read((char*)&alpha, 8); f.read((char*)&acc, 8);
    f.read((char*)A[q].data(), 8 * ld * ld); f.read((char*)B[q].data(), 8 * ld * ld); f.read((char*)Cm[q].data(), 8 * ld * ld);
    tasks[q] = GemmTaskT<double>{A[q].data(), B[q].data(), Cm[q].data(), alpha, (int)acc};
  }
  host_launch2(nT * nT, ntasks, 256, [&] { k_gemm_fma<double>(tasks.data(), nT); });
  std::ofstream o(argv[2], std::ios::binary);
  for (int q = 0; q < ntasks; ++q) o.write((const char*)Cm[q].data(), 8 * ld * ld);
  return 0;
}
'''


def _build(d, name, code):
    cxx = shutil.which("g++")
    (d / f"{name}.cpp").write_text(code)
    exe = d / name
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / f"{name}.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


@pytest.fixture(scope="module")
def workdir(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    return tmp_path_factory.mktemp("misc_host")


@pytest.mark.parametrize("name,n,over", [("convdiff2d", 24, {}), ("helmholtz2d", 20, {}),
                                         ("vardiff3d", 10, {"b": (1.0, -0.5, 2.0)})])
def test_noalloc_residual_on_the_host(workdir, name, n, over):
    src = open(os.path.join(CSRC, "noalloc.cu")).read()
    # The kernels and their constants: from the constants to the host-side helpers, without the
    # file-scope device array (the host test passes its own partial-sum buffer).
    body = src[src.index("constexpr int kNoallocThreads"):src.index("namespace {")]
    body = re.sub(r"static __device__ __align__\(256\) double g_noalloc_partials\[[^\]]*\];", "", body)
    assert "g_noalloc_partials" not in body and "k_norms_noalloc" in body
    code = '#include "cuda_host_shim.h"\nnamespace ddst {\n' + body + "\n}  // namespace ddst\n" + NOALLOC_MAIN
    exe = _build(workdir, "noalloc_host", code)
    prob = I.make_problem(name, n=n, w=n // 4, **over)
    dim = prob["dim"]
    nnode = (n + 1) ** dim
    has_c = prob.get("c") is not None
    bb = list(prob["b"]) + [0.0] * (3 - len(prob["b"]))
    A, b = O.assemble(prob)
    u = np.random.default_rng(n).standard_normal(b.size)
    path = workdir / f"noalloc_{name}.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("4q", dim, n, int(has_c), nnode) + struct.pack("3d", *bb))
        for arr in (prob["a"], prob["c"] if has_c else np.zeros(nnode), prob["g"], prob["f"]):
            f.write(np.asarray(arr, dtype=np.float64).ravel().tobytes())
        f.write(u.tobytes())
    out = workdir / (path.name + ".out")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    raw = np.fromfile(out, dtype=np.float64)
    want = b - A @ u
    assert np.abs(raw[:-2] - want).max() <= 1e-11 * np.abs(want).max()
    assert abs(raw[-2] - np.linalg.norm(want)) <= 1e-12 * np.linalg.norm(want)
    assert abs(raw[-1] - np.linalg.norm(b)) <= 1e-12 * np.linalg.norm(b)


def test_gemm_fma_on_the_host(workdir):
    src = open(os.path.join(CSRC, "gemm_tc.cu")).read()
    kh = open(os.path.join(CSRC, "kernels.cuh")).read()
    task = re.search(r"template <typename T>\nstruct GemmTaskT \{.*?\n\};", kh, re.S).group(0)
    i = src.index("template <typename T>\n__global__ void __launch_bounds__(256) k_gemm_fma(")
    j = src.index("\n}\n", i) + 3
    code = ('#include "cuda_host_shim.h"\nnamespace ddst {\nconstexpr int BT = 128;\n' + task + "\n" +
            src[i:j] + "\n}  // namespace ddst\n" + GEMM_MAIN)
    exe = _build(workdir, "gemm_host", code)
    nT, rng = 2, np.random.default_rng(3)
    ld = nT * 128
    cases = [(1.0, 0), (-0.5, 1), (2.0, 1)]
    mats = []
    path = workdir / "gemm.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("2q", nT, len(cases)))
        for alpha, acc in cases:
            A, B, C = (rng.standard_normal((ld, ld)) for _ in range(3))
            mats.append((alpha, acc, A, B, C))
            f.write(struct.pack("d", alpha) + struct.pack("q", acc))
            f.write(A.tobytes() + B.tobytes() + C.tobytes())
    out = workdir / "gemm.out"
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    got = np.fromfile(out, dtype=np.float64).reshape(len(cases), ld, ld)
    for q, (alpha, acc, A, B, C) in enumerate(mats):
        want = alpha * (A @ B) + (C if acc else 0.0)
        assert np.abs(got[q] - want).max() <= 1e-11 * np.abs(want).max()


REDUCE_MAIN = r"""
#include <fstream>
using namespace ddst;
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  int64_t h[4]; double a; f.read((char*)h, 32); f.read((char*)&a, 8);
  const int64_t n = h[0], off1 = h[1], n0 = h[2], n1 = h[3];
  std::vector<double> x(n), y(n), part(64, 0.0), out(4, 0.0);
  f.read((char*)x.data(), 8 * n); f.read((char*)y.data(), 8 * n);
  // <x, y> over n with 7 CTAs (grid-stride), then one CTA sums the partials
  host_launch(7, 256, [&] { k_dot_partial(x.data(), y.data(), n, part.data()); });
  host_launch(1, 256, [&] { k_sum_partials(part.data(), 7, out.data()); });
  // per-problem ||x||^2: problem 0 = x[0, n0), problem 1 = x[off1, off1 + n1); 5 CTAs each
  std::vector<ProbDesc> P(2);
  P[0].vol_off = 0; P[0].nint = n0; P[1].vol_off = off1; P[1].nint = n1;
  host_launch2(5, 2, 256, [&] { k_prob_sqnorm_partial(P.data(), x.data(), part.data()); });
  host_launch(2, 256, [&] { k_sum_partials(part.data(), 5, out.data() + 1); });
  host_launch(3, 128, [&] { k_axpy(n, a, x.data(), y.data()); });
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)out.data(), 24); o.write((const char*)y.data(), 8 * n);
  return 0;
}
"""


def test_reductions_and_axpy_on_the_host(workdir):
    src = open(os.path.join(CSRC, "stencil.cu")).read()
    common = open(os.path.join(CSRC, "common.cuh")).read()
    prob = re.search(r"struct ProbDesc \{.*?\n\};", common, re.S).group(0)
    red = src[src.index("// Partial sums of x.y over n elements"):src.index("// IMEX right-hand side")]
    axpy = src[src.index("// y = a*x + y  (FP64)"):src.index("// Host launchers")]
    code = ('#include "cuda_host_shim.h"\nnamespace ddst {\n' + prob + "\n" + red + "\n" + axpy +
            "\n}  // namespace ddst\n" + REDUCE_MAIN)
    exe = _build(workdir, "reduce_host", code)
    rng = np.random.default_rng(5)
    n, off1, n0, n1, a = 10007, 5000, 4999, 3001, -0.75
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    path = workdir / "reduce.bin"
    path.write_bytes(struct.pack("4q", n, off1, n0, n1) + struct.pack("d", a) + x.tobytes() +
                     y.tobytes())
    out = workdir / "reduce.out"
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    raw = np.fromfile(out, dtype=np.float64)
    # summation in another order: |error| <= n eps sum |x_i y_i| (Higham, Sec. 3.1)
    assert abs(raw[0] - x @ y) <= n * 2.2e-16 * np.abs(x * y).sum()
    assert abs(raw[1] - x[:n0] @ x[:n0]) <= 1e-13 * (x[:n0] @ x[:n0])
    assert abs(raw[2] - x[off1:off1 + n1] @ x[off1:off1 + n1]) <= 1e-13 * (x[off1:off1 + n1] @ x[off1:off1 + n1])
    # one rounding, or none where the compiler contracts to a fused multiply-add
    want = y + a * x
    assert (np.abs(raw[3:] - want) <= 2.3e-16 * (np.abs(want) + np.abs(a * x))).all()


PACK_MAIN = r"""
#include <fstream>
using namespace ddst;
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  const int nT = 2; const int64_t ld = nT * BT;
  std::vector<float> src(ld * ld), dA(nT * nT * SPLIT_TILE, -1.f), dB(dA.size(), -1.f);
  f.read((char*)src.data(), 4 * ld * ld);
  std::vector<PackTask> tasks = {PackTask{src.data(), dA.data(), 0}, PackTask{src.data(), dB.data(), 1}};
  std::vector<float> smem(PACK_SMEM / sizeof(float));
  host_dynamic_smem = smem.data();
  host_launch2(nT * nT, 2, 256, [&] { k_pack_split(tasks.data(), nT); });
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)dA.data(), 4 * dA.size()); o.write((const char*)dB.data(), 4 * dB.size());
  return 0;
}
"""


def test_split_packing_on_the_host(workdir):
    """`k_pack_split` (`csrc/gemm_tc.cu`): 128 x 128 tiles of an A operand (tile (I, kt) holds
    src(128 I + r, 128 kt + k)) and of a B operand packed as B^T (tile (J, kt) holds
    src(128 kt + k, 128 J + r)), as TF32 hi/lo parts in 16-wide K chunks of the K-major
    core-matrix layout; hi + lo equals the FP32 value to 2^-21."""
    src = open(os.path.join(CSRC, "gemm_tc.cu")).read()
    kern = open(os.path.join(CSRC, "kernels.cuh")).read()
    umma = open(os.path.join(CSRC, "umma.cuh")).read()
    split = open(os.path.join(CSRC, "splittile.cuh")).read()
    task = re.search(r"struct PackTask \{.*?\n\};", kern, re.S).group(0)
    off = re.search(r"__host__ __device__ __forceinline__ uint32_t umma_off\(.*?\n\}", umma, re.S).group(0)
    sp_ = split[split.index("constexpr int BT = 128;"):split.index("}  // namespace ddst")]
    body = src[src.index("constexpr int PK_LS = BT + 1;"):src.index("// -----", src.index("k_pack_split("))]
    body = body.replace("extern __shared__ float S[];", "float* S = host_dynamic_smem;")
    rna = ("inline float tf32_rna(float x) {  // 10-bit significand, nearest, ties away\n"
           "  uint32_t u; std::memcpy(&u, &x, 4); u = (u + 0x1000u) & ~0x1fffu;\n"
           "  float r; std::memcpy(&r, &u, 4); return r;\n}\n")
    code = ('#include "cuda_host_shim.h"\n#include <cstring>\nstatic float* host_dynamic_smem = nullptr;\n'
            "namespace ddst {\n" + task + "\n" + rna + off + "\n" + sp_ + "\n" + body +
            "\n}  // namespace ddst\n" + PACK_MAIN)
    exe = _build(workdir, "pack_host", code)
    rng = np.random.default_rng(9)
    A = rng.standard_normal((256, 256)).astype(np.float32)
    path = workdir / "pack.bin"
    path.write_bytes(A.tobytes())
    out = workdir / "pack.out"
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    raw = np.fromfile(out, dtype=np.float32)
    st = 2 * 128 * 128
    dA, dB = raw[:4 * st], raw[4 * st:]
    rr, kk = np.meshgrid(np.arange(128), np.arange(128), indexing="ij")
    c = kk % 16
    idx = (kk // 16) * 2048 + (rr >> 3) * 128 + (c >> 2) * 32 + (rr & 7) * 4 + (c & 3)
    A64 = A.astype(np.float64)
    for I_ in range(2):
        for kt in range(2):
            for dst, want in ((dA, A64[128 * I_:128 * I_ + 128, 128 * kt:128 * kt + 128]),
                              (dB, A64[128 * kt:128 * kt + 128, 128 * I_:128 * I_ + 128].T)):
                tile = dst[(I_ * 2 + kt) * st:(I_ * 2 + kt + 1) * st]
                hi, lo = tile[:128 * 128][idx], tile[128 * 128:][idx]
                assert np.all(hi.view(np.uint32) & 0x1FFF == 0) and np.all(lo.view(np.uint32) & 0x1FFF == 0)
                got = hi.astype(np.float64) + lo.astype(np.float64)
                assert np.all(np.abs(got - want) <= 2.0 ** -21 * np.abs(want))


CVT_MAIN = r"""
#include <fstream>
using namespace ddst;
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  const int64_t n = 1000;
  std::vector<double> x(n); f.read((char*)x.data(), 8 * n);
  std::vector<float> y(n + 3, -7.f);
  std::vector<double> z(n + 3, -7.0);
  host_launch(3, 64, [&] { k_hbs_cvt<float>(x.data(), y.data(), n); });
  host_launch(2, 96, [&] { k_hbs_cvt<double>(x.data(), z.data(), n); });
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)y.data(), 4 * y.size()); o.write((const char*)z.data(), 8 * z.size());
  return 0;
}
"""


def test_sample_conversion_on_the_host(workdir):
    """`k_hbs_cvt` (`csrc/hbs.cu`): caller-given FP64 test matrices into the working precision,
    every element once (grid-stride), round to nearest, nothing written past the end."""
    src = open(os.path.join(CSRC, "hbs.cu")).read()
    i = src.index("template <typename T>\n__global__ void k_hbs_cvt(")
    body = src[i:src.index("\n}\n", i) + 3]
    exe = _build(workdir, "cvt_host", '#include "cuda_host_shim.h"\nnamespace ddst {\n' + body +
                 "\n}  // namespace ddst\n" + CVT_MAIN)
    x = np.random.default_rng(4).standard_normal(1000) * 10.0 ** np.linspace(-30, 30, 1000)
    path = workdir / "cvt.bin"
    path.write_bytes(x.tobytes())
    out = workdir / "cvt.out"
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    raw = out.read_bytes()
    y = np.frombuffer(raw[:4 * 1003], dtype=np.float32)
    z = np.frombuffer(raw[4 * 1003:], dtype=np.float64)
    assert np.array_equal(y[:1000], x.astype(np.float32)) and np.all(y[1000:] == -7.0)
    assert np.array_equal(z[:1000], x) and np.all(z[1000:] == -7.0)
