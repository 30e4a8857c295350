"""HODLR kernels of `csrc/hodlr.cu` compiled for the host and run with one OS thread per CUDA
thread under AddressSanitizer (`tests/hostemu/cuda_host_shim.h`):
* the tiled transposed product of the compression's power iteration (`k_sblk_gemv_t`,
  y_b = S_b^T x_b for every dense transfer block, Sec. 2.4's ||S||_2 estimate), against the
  plain product on blocks with ragged tiles;
* the whole power iteration (`k_sblk_gemv`, `k_sblk_gemv_t`, `k_sblk_normalize`, two steps in
  FP64 and FP32) against the same iteration in numpy, and its estimate of ||S||_2^2 bounded
  above by the largest squared singular value (an underestimate, as the compression assumes);
* the interface apply (`k_h_inner` + `k_h_owner`: (I - K) x, its transpose, K x, K^T x in FP64
  and FP32) on the oracle's HODLR factors (O6) in the library's layout, against O6's apply."""
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
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
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


# ---------------------------------------------------------------------------------------------
# The power iteration of the compression: ||S||_2^2 ~ ||S^T S x|| after two normalised steps
# ---------------------------------------------------------------------------------------------
POWER_MAIN = r"""
#include <cstring>
#include <fstream>
using namespace ddst;
template <typename T>
void run(std::ifstream& f, std::ofstream& o, const std::vector<SBlk>& sb, int64_t tot, int64_t stride) {
  const int nb = (int)sb.size();
  int64_t maxng = 0;
  for (auto& b : sb) maxng = std::max(maxng, b.ng);
  std::vector<double> S64(tot), x(nb * stride), y(nb * stride), nrm(nb, -1.0);
  f.read((char*)S64.data(), 8 * tot); f.read((char*)x.data(), 8 * nb * stride);
  std::vector<T> S(S64.begin(), S64.end());
  const unsigned gr = (unsigned)((maxng + 255) / 256), gz = (unsigned)((maxng + 127) / 128);
  for (int it = 0; it < 2; ++it) {
    std::fill(y.begin(), y.end(), 0.0);
    host_launch3(gr, nb, gz, 256, [&] { k_sblk_gemv<T>(sb.data(), S.data(), x.data(), y.data(), stride); });
    host_launch2(gz, nb, 256, [&] { k_sblk_gemv_t<T>(sb.data(), S.data(), y.data(), x.data(), stride); });
    host_launch(nb, 256, [&] { k_sblk_normalize(sb.data(), x.data(), x.data(), stride, nrm.data()); });
  }
  o.write((const char*)x.data(), 8 * nb * stride);
  o.write((const char*)nrm.data(), 8 * nb);
}
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  int64_t h[3]; f.read((char*)h, 24);
  const int nb = (int)h[0]; const int64_t stride = h[1], esz = h[2];
  std::vector<SBlk> sb(nb);
  int64_t tot = 0;
  for (auto& b : sb) { int64_t a[2]; f.read((char*)a, 16); b.off = a[0]; b.ng = a[1]; tot = std::max(tot, a[0] + a[1] * a[1]); }
  std::ofstream o(argv[2], std::ios::binary);
  if (esz == 8) run<double>(f, o, sb, tot, stride); else run<float>(f, o, sb, tot, stride);
  return 0;
}
"""


@pytest.fixture(scope="module")
def power_harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "hodlr.cu")).read()
    sblk = re.search(r"struct SBlk \{.*?\n\};", src, re.S).group(0)
    i = src.index("template <typename T>\n__global__ void k_sblk_gemv(")
    j = src.index("__global__ void k_sblk_init(")
    d = tmp_path_factory.mktemp("power_host")
    code = ('#include "cuda_host_shim.h"\nnamespace ddst {\n' + sblk + "\n" + src[i:j] +
            "\n}  // namespace ddst\n" + POWER_MAIN)
    (d / "power_host.cpp").write_text(code)
    exe = d / "power_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "power_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


@pytest.mark.parametrize("esz", [8, 4])
def test_power_iteration_on_the_host(power_harness, esz):
    d, exe = power_harness
    rng = np.random.default_rng(11)
    ngs = (300, 129, 1, 257)
    stride = 310
    blocks, offs, off = [], [], 0
    for q, ng in enumerate(ngs):
        if q == 0:   # geometric spectrum, like a transfer operator's
            U, _ = np.linalg.qr(rng.standard_normal((ng, ng)))
            V, _ = np.linalg.qr(rng.standard_normal((ng, ng)))
            B = (U * 0.6 ** np.arange(ng)) @ V.T
        else:
            B = rng.standard_normal((ng, ng)) / np.sqrt(ng)
        blocks.append(B)
        offs.append(off)
        off += ng * ng
    x0 = rng.standard_normal((len(ngs), stride))
    path = d / f"power_{esz}.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("3q", len(ngs), stride, esz))
        for o, ng in zip(offs, ngs):
            f.write(struct.pack("2q", o, ng))
        for B in blocks:
            f.write(np.ascontiguousarray(B.T).tobytes())
        f.write(x0.tobytes())
    out = d / (path.name + ".out")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    raw = np.fromfile(out, dtype=np.float64)
    x, nrm = raw[:len(ngs) * stride].reshape(len(ngs), stride), raw[len(ngs) * stride:]
    tol = 1e-12 if esz == 8 else 2e-5
    for q, (B, ng) in enumerate(zip(blocks, ngs)):
        Bw = B if esz == 8 else B.astype(np.float32).astype(np.float64)
        v = x0[q, :ng].copy()
        for _ in range(2):
            v = Bw.T @ (Bw @ v)
            nv = np.linalg.norm(v)
            v /= nv
        assert abs(nrm[q] - nv) <= tol * nv
        assert np.abs(x[q, :ng] - v).max() <= 10 * tol
        smax2 = np.linalg.norm(Bw, 2) ** 2
        assert nrm[q] <= smax2 * (1 + tol)            # a unit vector's ||S^T S x|| <= sigma_max^2


# ---------------------------------------------------------------------------------------------
# The HODLR interface apply (k_h_inner + k_h_owner), the operator of every GMRES iteration
# ---------------------------------------------------------------------------------------------
APPLY_MAIN = r'''
#include <fstream>
using namespace ddst;
template <typename T>
int run(std::ifstream& f, const char* outp, int64_t nblk, int64_t nleaf, int64_t nown,
        int64_t nuv, int64_t nd, int64_t tl, int64_t nx, int mode) {
  std::vector<HBlock> bl(nblk); std::vector<HLeaf> lv(nleaf); std::vector<HOwn> own(nown);
  for (auto& b : bl) {
    int64_t a[12]; f.read((char*)a, 96);
    b.sblk = (int)a[0]; b.level = (int)a[1]; b.row0 = a[2]; b.nrows = a[3]; b.col0 = a[4];
    b.ncols = a[5]; b.rank = (int)a[6]; b.u_off = a[7]; b.v_off = a[8]; b.t_off = a[9];
    b.in_if = a[10]; b.out_if = a[11];
  }
  for (auto& l : lv) {
    int64_t a[7]; f.read((char*)a, 56);
    l.sblk = (int)a[0]; l.lo = a[1]; l.len = a[2]; l.ld = a[3]; l.d_off = a[4]; l.in_if = a[5]; l.out_if = a[6];
  }
  for (auto& o : own) {
    int64_t a[6 + 2 * HOWN_MAXL]; f.read((char*)a, 8 * (6 + 2 * HOWN_MAXL));
    o.out = a[0]; o.lo = a[1]; o.len = (int)a[2]; o.nsrc = (int)a[3]; o.leaf[0] = (int)a[4]; o.leaf[1] = (int)a[5];
    for (int q = 0; q < 2; ++q)
      for (int l = 0; l < HOWN_MAXL; ++l) o.hb[q][l] = (int)a[6 + q * HOWN_MAXL + l];
  }
  std::vector<double> uv64(nuv), d64(nd), x(nx), y(nx, 0.0), t(std::max<int64_t>(tl, 1), 0.0);
  f.read((char*)uv64.data(), 8 * nuv); f.read((char*)d64.data(), 8 * nd); f.read((char*)x.data(), 8 * nx);
  std::vector<T> UV(uv64.begin(), uv64.end()), D(d64.begin(), d64.end());
  const int transpose = mode & 1, konly = mode >> 1;
  if (nblk > 0)
    host_launch((unsigned)((nblk + 7) / 8), 256, [&] { k_h_inner<T>(bl.data(), (int)nblk, UV.data(), x.data(), t.data(), transpose, nullptr, 0); });
  host_launch((unsigned)nown, OWN_T, [&] { k_h_owner<T>(own.data(), bl.data(), lv.data(), UV.data(), D.data(), t.data(), x.data(), y.data(), transpose, konly, nullptr, 0); });
  std::ofstream o(outp, std::ios::binary);
  o.write((const char*)y.data(), 8 * nx);
  return 0;
}
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  int64_t h[9]; f.read((char*)h, 72);
  return h[8] == 8 ? run<double>(f, argv[2], h[0], h[1], h[2], h[3], h[4], h[5], h[6], (int)h[7])
                   : run<float>(f, argv[2], h[0], h[1], h[2], h[3], h[4], h[5], h[6], (int)h[7]);
}
'''


@pytest.fixture(scope="module")
def apply_harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "hodlr.cu")).read()
    hdr = open(os.path.join(CSRC, "hodlr.cuh")).read()
    structs = [re.search(r"struct %s \{.*?\n\};" % n, hdr, re.S).group(0) for n in ("HBlock", "HLeaf")]
    consts = re.search(r"constexpr int HOWN_MAXL.*?struct HOwn \{.*?\n\};", hdr, re.S).group(0)
    i = src.rindex("// ----", 0, src.index("// Application: y = x - K x"))
    j = src.rindex("// ----", 0, src.index("void HodlrSet::clear()"))
    d = tmp_path_factory.mktemp("hodlr_apply_host")
    code = ('#include "cuda_host_shim.h"\nnamespace ddst {\ninline void pdl_wait() {}\ninline void pdl_release() {}\n' +
            "\n".join(structs) + "\n" + consts + "\n" + src[i:j] + "\n}  // namespace ddst\n" + APPLY_MAIN)
    (d / "hodlr_apply_host.cpp").write_text(code)
    exe = d / "hodlr_apply_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "hodlr_apply_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


def _levels(ng, leaf):
    L = 0
    while -(-ng // (1 << L)) > leaf:
        L += 1
    return L


@pytest.mark.parametrize("nds,ng,leaf,tol", [(4, 150, 32, 1e-3), (3, 100, 64, 0.0), (2, 40, 32, 1e-6)])
@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("esz", [8, 4])
def test_hodlr_interface_apply_on_the_host(apply_harness, nds, ng, leaf, tol, mode, esz):
    """(I - K) x, (I - K)^T x, K x and K^T x through the library's HODLR blocks, laid out as its
    build lays them out (per S block: low-rank blocks by level, then the dense leaves; output
    items per interface leaf range) from the oracle's truncated-SVD HODLR (O6), against O6's
    apply of the same factors.  Random blocks give full ranks above 16 (the owner kernel's tail
    path); tol = 0 keeps every rank."""
    from oracle import ddst_oracle as O
    d, exe = apply_harness
    rng = np.random.default_rng(nds * 100 + ng + mode)
    Sp = [None] + [rng.standard_normal((ng, ng)) for _ in range(nds - 1)]
    Sn = [rng.standard_normal((ng, ng)) for _ in range(nds - 1)] + [None]
    L = _levels(ng, leaf)
    blocks, leaves, uv, dd, sb_fb, sb_fl, sblist, tl = [], [], [], [], [], [], [], 0
    uvo = ddo = 0
    Hs = []
    for q in range(nds):
        for side, S in ((-1, Sp[q]), (1, Sn[q])):
            if S is None:
                continue
            b = len(sblist)
            sblist.append((q, side))
            H = O.hodlr_compress(S, tol=tol, leaf=leaf)
            assert H["L"] == L
            Hs.append(H)
            in_if, out_if = (q + side) * ng, q * ng
            sb_fb.append(len(blocks))
            sb_fl.append(len(leaves))
            for lev in range(1, L + 1):
                for t in range(1 << (lev - 1)):
                    lo1, hi1 = ((2 * t) * ng) >> lev, ((2 * t + 1) * ng) >> lev
                    lo2, hi2 = hi1, ((2 * t + 2) * ng) >> lev
                    for e, (r0, r1, c0, c1) in enumerate(((lo1, hi1, lo2, hi2), (lo2, hi2, lo1, hi1))):
                        U, V = H["levels"][lev - 1][2 * t + e]
                        rank = U.shape[1]
                        blocks.append([b, lev, r0, r1 - r0, c0, c1 - c0, rank, uvo, uvo + (r1 - r0) * rank,
                                       tl, in_if, out_if])
                        uv += [U.T.ravel(), V.T.ravel()]
                        uvo += (r1 - r0 + c1 - c0) * rank
                        tl += rank
            for t in range(1 << L):
                lo, hi = (t * ng) >> L, ((t + 1) * ng) >> L
                ln = hi - lo
                ld = (ln + 3) // 4 * 4
                Dm = np.zeros((ld, ln))
                Dm[:ln] = H["leaves"][t]
                leaves.append([b, lo, ln, ld, ddo, in_if, out_if])
                dd.append(Dm.T.ravel())
                ddo += ld * ln
    sb_fb.append(len(blocks))
    own = []
    tr = mode & 1
    for q in range(nds):
        iface = q * ng
        src = [b for b in range(len(sblist)) if leaves[sb_fl[b]][6 if tr == 0 else 5] == iface]
        assert len(src) <= 2
        for tt in range(1 << L):
            lo = (tt * ng) >> L
            rec = [iface, lo, (((tt + 1) * ng) >> L) - lo, len(src), 0, 0] + [-1] * 24
            for qq, b in enumerate(src):
                rec[4 + qq] = sb_fl[b] + tt
                for bi in range(sb_fb[b], sb_fb[b + 1]):
                    B = blocks[bi]
                    a0, an = (B[4], B[5]) if tr else (B[2], B[3])
                    if B[6] > 0 and a0 <= lo < a0 + an:
                        rec[6 + qq * 12 + B[1] - 1] = bi
            own.append(rec)
    x = rng.standard_normal(nds * ng)
    path = d / f"apply_{nds}_{ng}_{leaf}_{mode}_{esz}.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("9q", len(blocks), len(leaves), len(own), uvo, ddo, tl, nds * ng, mode, esz))
        for rec in blocks:
            f.write(struct.pack("12q", *rec))
        for rec in leaves:
            f.write(struct.pack("7q", *rec))
        for rec in own:
            f.write(struct.pack("30q", *rec))
        f.write(np.concatenate(uv).astype(np.float64).tobytes() if uv else b"")
        f.write(np.concatenate(dd).astype(np.float64).tobytes())
        f.write(x.tobytes())
    out = d / (path.name + ".y")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    y = np.fromfile(out, dtype=np.float64)
    X = x.reshape(nds, ng)
    Kx = np.zeros((nds, ng))
    for b, (q, side) in enumerate(sblist):
        Hd = O.hodlr_dense(Hs[b])
        if tr == 0:
            Kx[q] += O.hodlr_apply(Hs[b], X[q + side])
        else:
            Kx[q + side] += Hd.T @ X[q]
    want = (Kx if mode & 2 else X - Kx).ravel()
    tolr = 1e-12 if esz == 8 else 2e-5
    assert np.abs(y - want).max() <= tolr * np.abs(want).max()
