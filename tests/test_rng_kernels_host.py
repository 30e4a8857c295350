"""The library's random-number generators, compiled for the host (`tests/hostemu/cuda_host_shim.h`)
and checked against what their published definitions and the randomized method fix:

* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11; the HODLR test matrices of Alg. 1 and
  the power-iteration start vectors) on the known-answer vectors published with the generator;
* the splitmix64 finalizer (Steele, Lea and Flood, OOPSLA'14; the HBS test matrices) on the
  first outputs of the generator from seed 0;
* the Gaussian test matrices that Alg. 1 draws (`k_hbs_gen` in FP64 and FP32, `k_gen_omega`,
  `k_sblk_init`): every slot of the layout written once and nothing outside it, standard normal
  by the Kolmogorov-Smirnov test and the first two moments, Omega and Psi, blocks and seeds
  uncorrelated, and the FP32 draw equal to the FP64 one up to FP32 rounding.
"""
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

# Known-answer vectors of Philox4x32-10: (counter, key) -> output, as published with the
# generator's reference implementation (Random123).
PHILOX_KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]
# splitmix64 from state 0: the first three outputs (the state advances by the golden-ratio
# increment before each finalization).
SPLITMIX_SEED0 = [0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f]

MAIN = r'''
#include <cstdio>
#include <fstream>
#include <limits>
using namespace ddst;
static const double NaN = std::numeric_limits<double>::quiet_NaN();
template <typename V> static void put(std::ofstream& o, const V& v) { o.write((const char*)v.data(), sizeof(v[0]) * v.size()); }
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  std::ofstream o(argv[2], std::ios::binary);
  int64_t h[2]; f.read((char*)h, 16);
  const uint64_t seed = (uint64_t)h[0];
  // 1. Philox known answers and splitmix64 finalizer
  for (int t = 0; t < 3; ++t) {
    uint32_t c[6]; f.read((char*)c, 24);
    const U4 r = philox4x32_10(U4{c[0], c[1], c[2], c[3]}, c[4], c[5]);
    const uint32_t out[4] = {r.x, r.y, r.z, r.w}; o.write((const char*)out, 16);
  }
  for (int t = 0; t < 3; ++t) { const uint64_t z = mix64(0x9e3779b97f4a7c15ull * (uint64_t)t); o.write((const char*)&z, 8); }
  // 2. HBS test matrices: two blocks, rows row0 .. row0 + ng - 1, s per row, guard rows around
  const int s = 23; const int64_t ng0 = 300, ng1 = 157, guard = 5;
  std::vector<SampBlk> sb = {SampBlk{nullptr, ng0, guard}, SampBlk{nullptr, ng1, guard + ng0 + guard}};
  const int64_t rows = guard + ng0 + guard + ng1 + guard;
  std::vector<double> Od(rows * s, NaN), Pd(rows * s, NaN);
  std::vector<float> Of(rows * s, (float)NaN), Pf(rows * s, (float)NaN);
  host_launch2(3, 2, 64, [&] { k_hbs_gen<double>(sb.data(), Od.data(), Pd.data(), s, seed); });
  host_launch2(3, 2, 64, [&] { k_hbs_gen<float>(sb.data(), Of.data(), Pf.data(), s, seed); });
  put(o, Od); put(o, Pd); put(o, Of); put(o, Pf);
  std::vector<double> Od2(rows * s, NaN), Pd2(rows * s, NaN);
  host_launch2(3, 2, 64, [&] { k_hbs_gen<double>(sb.data(), Od2.data(), Pd2.data(), s, seed + 1); });
  put(o, Od2);
  // 3. HODLR test matrices: q x s column-major at v_off of each block, s not a multiple of 4
  std::vector<HDev> hd(2);
  hd[0] = HDev{0, 0, 0, 200, 30, 0, 0, 7};
  hd[1] = HDev{0, 0, 0, 77, 13, 0, 0, 7 + 200 * 30 + 9};
  const int64_t uvn = 7 + 200 * 30 + 9 + 77 * 13 + 11;
  std::vector<float> UV(uvn, (float)NaN);
  host_launch2(4, 2, 64, [&] { k_gen_omega<float>(hd.data(), UV.data(), seed); });
  put(o, UV);
  // 4. power-iteration start vectors: three blocks, stride above the largest ng
  std::vector<SBlk> sbl = {SBlk{0, 1000}, SBlk{0, 333}, SBlk{0, 5}};
  const int64_t stride = 1010;
  std::vector<double> X(3 * stride, NaN);
  host_launch(3, 128, [&] { k_sblk_init(sbl.data(), X.data(), stride, seed); });
  put(o, X);
  return 0;
}
'''


def _extract(src, start, end_marker=None, *, func=False):
    i = src.index(start)
    if func:
        return src[i:src.index("\n}\n", i) + 3]
    return src[i:src.index(end_marker, i)]


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("rng_host")
    hod = open(os.path.join(CSRC, "hodlr.cu")).read()
    hbs = open(os.path.join(CSRC, "hbs.cu")).read()
    parts = [
        _extract(hod, "struct U4 {", "struct SBlk {"),                      # philox, u01, gauss4
        re.search(r"struct SBlk \{.*?\n\};", hod, re.S).group(0),
        re.search(r"struct HDev \{.*?\n\};", hod, re.S).group(0),
        _extract(hod, "__global__ void k_sblk_init(", func=True),
        _extract(hod, "template <typename T>\n__global__ void k_gen_omega(", func=True),
        _extract(hbs, "__device__ __forceinline__ uint64_t mix64(", "struct SampItem {"),
        _extract(hbs, "template <typename T>\n__global__ void k_hbs_gen(", func=True),
    ]
    code = ('#include "cuda_host_shim.h"\nnamespace ddst {\n' + "\n".join(parts) +
            "\n}  // namespace ddst\n" + MAIN)
    (d / "rng.cpp").write_text(code)
    exe = d / "rng"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "rng.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    inp = d / "in.bin"
    with open(inp, "wb") as f:
        f.write(struct.pack("2q", 20251030, 0))
        for ctr, key, _ in PHILOX_KAT:
            f.write(struct.pack("6I", *ctr, *key))
    out = d / "out.bin"
    r = subprocess.run([str(exe), str(inp), str(out)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    raw = out.read_bytes()
    res, pos = {}, 0

    def take(name, dtype, count):
        nonlocal pos
        nb = np.dtype(dtype).itemsize * count
        res[name] = np.frombuffer(raw[pos:pos + nb], dtype=dtype).copy()
        pos += nb

    s, rows = 23, 5 + 300 + 5 + 157 + 5
    take("philox", np.uint32, 12)
    take("splitmix", np.uint64, 3)
    for nm, dt in (("Od", np.float64), ("Pd", np.float64), ("Of", np.float32), ("Pf", np.float32),
                   ("Od2", np.float64)):
        take(nm, dt, rows * s)
    take("UV", np.float32, 7 + 200 * 30 + 9 + 77 * 13 + 11)
    take("X", np.float64, 3 * 1010)
    assert pos == len(raw)
    return res


def _blocks(a, s=23):
    """Rows of the two HBS blocks and the guard rows around them."""
    m = a.reshape(-1, s)
    return m[5:305], m[310:467], np.concatenate([m[:5], m[305:310], m[467:]])


def _assert_standard_normal(x, what):
    stats = pytest.importorskip("scipy.stats")
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    assert abs(x.mean()) < 4.5 / np.sqrt(n), what
    assert abs(x.var() - 1.0) < 4.5 * np.sqrt(2.0 / n), what
    assert stats.kstest(x, "norm").pvalue > 1e-4, what


def test_philox_known_answers(run):
    got = run["philox"].reshape(3, 4)
    for t, (_, _, want) in enumerate(PHILOX_KAT):
        assert tuple(int(v) for v in got[t]) == want


def test_splitmix_finalizer_first_outputs(run):
    assert [int(v) for v in run["splitmix"]] == SPLITMIX_SEED0


def test_hbs_test_matrices_fill_exactly_their_rows(run):
    for nm in ("Od", "Pd", "Of", "Pf", "Od2"):
        b0, b1, g = _blocks(run[nm])
        assert np.isfinite(b0).all() and np.isfinite(b1).all(), nm
        assert np.isnan(g).all(), nm


def test_hbs_test_matrices_are_standard_normal_and_independent(run):
    b0, b1, _ = _blocks(run["Od"])
    p0, p1, _ = _blocks(run["Pd"])
    o2, _, _ = _blocks(run["Od2"])
    for x, what in ((b0, "Omega block 0"), (b1, "Omega block 1"), (p0, "Psi block 0"),
                    (np.concatenate([b0.ravel(), b1.ravel(), p0.ravel(), p1.ravel()]), "all")):
        _assert_standard_normal(x.ravel(), what)
    n = b0.size
    for a, b, what in ((b0, p0, "Omega vs Psi"), (b0[:157], b1, "block 0 vs block 1"),
                       (b0, o2, "seed vs seed + 1")):
        rho = np.corrcoef(a.ravel(), b.ravel())[0, 1]
        assert abs(rho) < 4.5 / np.sqrt(min(a.size, b.size)), what
    flat = b0.ravel()
    assert abs(np.corrcoef(flat[:-1], flat[1:])[0, 1]) < 4.5 / np.sqrt(n)   # along a row
    col = b0[:, 0]
    assert abs(np.corrcoef(col[:-1], col[1:])[0, 1]) < 4.5 / np.sqrt(col.size)  # down a column


def test_hbs_fp32_draw_is_the_fp64_draw_rounded(run):
    for a, b in (("Of", "Od"), ("Pf", "Pd")):
        f32 = np.concatenate([x.ravel() for x in _blocks(run[a])[:2]]).astype(np.float64)
        f64 = np.concatenate([x.ravel() for x in _blocks(run[b])[:2]])
        d = np.abs(f32 - f64) / (1.0 + np.abs(f64))
        # The bulk: a few units of FP32 rounding (24-bit uniforms, FP32 logarithm and cosine).
        assert np.quantile(d, 0.999) < 4e-6
        # Every sample: the 24-bit radius uniform u1 >= 2^-24 moves log u1 by at most 2^-24 / u1,
        # so g = r cos(2 pi u2) with r^2 = -2 log u1 moves by at most |g| 2^-24 / (u1 r^2).  As
        # u1 r^2 = r^2 exp(-r^2 / 2) falls for r^2 > 2, that is at most |g| / (48 ln 2) < 0.031 |g|
        # up to the largest radius sqrt(48 ln 2); below r^2 = 2 it is at most 2^-24 / r, and r is 0
        # or at least sqrt(2^-23), so under 2e-4 (u1 = 1 in FP32 gives 0 for a sample below 3.5e-4).
        assert (np.abs(f32 - f64) <= 0.031 * np.abs(f64) + 4e-4).all()


def test_hodlr_test_matrix_layout_and_distribution(run):
    uv = run["UV"].astype(np.float64)
    o0 = 7
    blk0 = uv[o0:o0 + 200 * 30]
    o1 = o0 + 200 * 30 + 9
    blk1 = uv[o1:o1 + 77 * 13]
    guards = np.concatenate([uv[:o0], uv[o0 + 200 * 30:o1], uv[o1 + 77 * 13:]])
    assert np.isfinite(blk0).all() and np.isfinite(blk1).all()
    assert np.isnan(guards).all()
    _assert_standard_normal(np.concatenate([blk0, blk1]), "Omega of the HODLR sketch")
    m0 = blk0.reshape(30, 200)       # column-major q x s: sample j is a contiguous column
    rho = np.corrcoef(m0[0], m0[1])[0, 1]   # the first two of four Box-Muller outputs
    assert abs(rho) < 4.5 / np.sqrt(200)
    rho = np.corrcoef(m0[0], m0[4])[0, 1]   # next counter
    assert abs(rho) < 4.5 / np.sqrt(200)


def test_power_iteration_start_vectors(run):
    X = run["X"].reshape(3, 1010)
    for b, ng in enumerate((1000, 333, 5)):
        assert np.isfinite(X[b, :ng]).all() and np.isnan(X[b, ng:]).all()
    _assert_standard_normal(np.concatenate([X[0, :1000], X[1, :333]]), "start vectors")
    assert abs(np.corrcoef(X[0, :333], X[1, :333])[0, 1]) < 4.5 / np.sqrt(333)
