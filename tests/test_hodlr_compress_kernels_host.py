"""The HODLR compression kernels of `csrc/hodlr.cu` (Sec. 2.4; Alg. 1's randomized sampling),
compiled for the host and run with one OS thread per CUDA thread under AddressSanitizer
(`tests/hostemu/cuda_host_shim.h`), on a transfer operator S_{j,j+1} of the oracle (O3) split
into the off-diagonal blocks of the weak-admissibility cluster tree, in the library's layout:
* `k_gen_omega` + `k_sketch`: Y = B Omega for every block, against the plain product;
* `k_range_cgs2`: the kept columns Q are orthonormal, and B - Q Q^T B is within the
  randomized range finder's bound 10 sqrt(2/pi) thr of the adaptive stopping rule (Halko,
  Martinsson and Tropp 2011, Sec. 4.4; thr = tol ||S||_2), so the rank is at least the number
  of singular values above that bound; O6's truncated SVD at the same threshold meets it too;
* `k_project`: V = B^T Q, against the plain product;
* `k_copy_leaves`: the dense diagonal leaves with their zero padding rows.
In FP64 and FP32.
"""
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

MAIN = r'''
#include <fstream>
using namespace ddst;
template <typename V> static void put(std::ofstream& o, const V& v) {
  for (auto e : v) { const double d = (double)e; o.write((const char*)&d, 8); }
}
template <typename T, int SC>
void sketch(unsigned n, const HItem* it, const HDev* hd, const T* S, T* UV) {
  host_launch(n, 256, [&] { k_sketch<T, SC>(it, hd, S, UV); });
}
template <typename T, int SC>
void project(unsigned n, const HItem* it, const HDev* hd, const int* rk, const T* S, T* UV) {
  host_launch(n, 256, [&] { k_project<T, SC>(it, hd, rk, S, UV); });
}
template <typename T>
int run(std::ifstream& f, std::ofstream& o, const int64_t* h, const double* d) {
  const int64_t ng = h[0], nblk = h[1], nleaf = h[2], uvn = h[3], dln = h[4];
  const int kmax = (int)h[5], run_len = (int)h[6], SC = (int)h[7];
  const uint64_t seed = (uint64_t)h[8];
  std::vector<double> S64(ng * ng);
  f.read((char*)S64.data(), 8 * ng * ng);
  std::vector<T> S(S64.begin(), S64.end());
  std::vector<HDev> hd(nblk);
  int64_t maxp = 0;
  for (auto& b : hd) {
    int64_t a[8]; f.read((char*)a, 64);
    b.s_off = a[0]; b.ng = a[1]; b.p = a[2]; b.q = a[3]; b.s = (int)a[4]; b.sblk = (int)a[5];
    b.u_off = a[6]; b.v_off = a[7];
    maxp = std::max(maxp, b.p);
  }
  std::vector<HLeaf> lv(nleaf);
  for (auto& l : lv) {
    int64_t a[4]; f.read((char*)a, 32);
    l.sblk = 0; l.lo = a[0]; l.len = a[1]; l.ld = a[2]; l.d_off = a[3]; l.in_if = 0; l.out_if = 0;
  }
  std::vector<HItem> items, pitems;
  for (int b = 0; b < nblk; ++b) {
    for (int64_t lo = 0; lo < hd[b].p; lo += 64) items.push_back({b, lo});
    for (int64_t lo = 0; lo < hd[b].q; lo += 64) pitems.push_back({b, lo});
  }
  std::vector<T> UV(uvn, T(0)), D(dln, T(-1));
  host_launch2(32, nblk, 256, [&] { k_gen_omega<T>(hd.data(), UV.data(), seed); });
  switch (SC) {
    case 32: sketch<T, 32>(items.size(), items.data(), hd.data(), S.data(), UV.data()); break;
    case 64: sketch<T, 64>(items.size(), items.data(), hd.data(), S.data(), UV.data()); break;
    default: sketch<T, 96>(items.size(), items.data(), hd.data(), S.data(), UV.data()); break;
  }
  put(o, UV);
  const double snorm = d[1];
  std::vector<int> rank(nblk, -1);
  std::vector<unsigned char> dyn(sizeof(T) * maxp);
  host_dynamic_smem = dyn.data();
  host_launch(nblk, 512, [&] {
    k_range_cgs2<T>(hd.data(), UV.data(), &snorm, d[0], kmax, run_len, rank.data());
  });
  int maxr = 0;
  for (int v : rank) maxr = std::max(maxr, v);
  const int SCp = maxr <= 16 ? 16 : (maxr <= 32 ? 32 : (maxr <= 64 ? 64 : 96));
  if (maxr > 0) {
    switch (SCp) {
      case 16: project<T, 16>(pitems.size(), pitems.data(), hd.data(), rank.data(), S.data(), UV.data()); break;
      case 32: project<T, 32>(pitems.size(), pitems.data(), hd.data(), rank.data(), S.data(), UV.data()); break;
      case 64: project<T, 64>(pitems.size(), pitems.data(), hd.data(), rank.data(), S.data(), UV.data()); break;
      default: project<T, 96>(pitems.size(), pitems.data(), hd.data(), rank.data(), S.data(), UV.data()); break;
    }
  }
  const int64_t soff = 0;
  host_launch2(3, nleaf, 64, [&] { k_copy_leaves<T>(lv.data(), &soff, &ng, S.data(), D.data()); });
  put(o, UV); put(o, rank); put(o, D);
  return 0;
}
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  std::ofstream o(argv[2], std::ios::binary);
  int64_t h[10]; double d[2];
  f.read((char*)h, 80); f.read((char*)d, 16);
  return h[9] == 8 ? run<double>(f, o, h, d) : run<float>(f, o, h, d);
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "hodlr.cu")).read()
    hh = open(os.path.join(CSRC, "hodlr.cuh")).read()
    common = open(os.path.join(CSRC, "common.cuh")).read()
    eps = src_between(common, "template <typename T> struct Eps;", "// -----")
    parts = [
        eps,
        re.search(r"struct HLeaf \{.*?\n\};", hh, re.S).group(0),
        src_between(src, "struct U4 {", "struct SBlk {"),                 # philox, gauss4
        re.search(r"struct HItem \{.*?\n\};", src, re.S).group(0),
        re.search(r"struct HDev \{.*?\n\};", src, re.S).group(0),
        src_between(src, "template <typename T>\n__global__ void k_gen_omega(",
                    "// Dense leaves:"),
        src_between(src, "// Dense leaves:", "\n}\n") + "\n}\n",
    ]
    body = "\n".join(parts)
    dyn = "extern __shared__ __align__(16) unsigned char smem_raw[];"
    assert body.count(dyn) == 1
    body = body.replace(dyn, "unsigned char* smem_raw = host_dynamic_smem;")
    code = ('#include "cuda_host_shim.h"\nstatic unsigned char* host_dynamic_smem = nullptr;\n'
            "namespace ddst {\n" + body + "\n}  // namespace ddst\n" + MAIN)
    d = tmp_path_factory.mktemp("hodlr_compress_host")
    (d / "hc_host.cpp").write_text(code)
    exe = d / "hc_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "hc_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    return d, exe


def src_between(src, start, end):
    i = src.index(start)
    return src[i:src.index(end, i + len(start))]


def _transfer_operator():
    """S_{1,2} of a 3D variable-coefficient problem with convection (n = 16, w = 4: 225 points
    per interface), from the oracle's explicit transfer blocks."""
    prob = I.make_problem("vardiff3d", n=16, w=4, b=(1.0, -0.5, 0.75))
    A = sp.csr_matrix(O.assemble(prob)[0])
    geo = O.slab_geometry(3, 16, 4)
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo), slabs=[0])
    return Sn[0]


@pytest.fixture(scope="module")
def transfer_op():
    return _transfer_operator()


@pytest.mark.parametrize("esz,tol", [(8, 1e-8), (4, 1e-3)])
def test_hodlr_compression_on_the_host(harness, transfer_op, esz, tol):
    d, exe = harness
    S = transfer_op
    ng = S.shape[0]
    leaf, kmax, over, seed = 32, 64, 10, 12345
    s_req = min(128, kmax + over)
    SC = 32
    while SC < s_req:
        SC += 32
    L = O.hodlr_levels(ng, leaf)
    blocks, uv = [], 0
    for lev in range(1, L + 1):
        for t in range(1 << (lev - 1)):
            lo1, hi1 = O.hodlr_node(ng, lev, 2 * t)
            lo2, hi2 = O.hodlr_node(ng, lev, 2 * t + 1)
            for r0, r1, c0, c1 in ((lo1, hi1, lo2, hi2), (lo2, hi2, lo1, hi1)):
                p, q = r1 - r0, c1 - c0
                s = min(s_req, p, q)
                blocks.append(dict(r0=r0, c0=c0, p=p, q=q, s=s, u=uv, v=uv + p * s))
                uv += (p + q) * s
    leaves, dl = [], 0
    for t in range(1 << L):
        lo, hi = O.hodlr_node(ng, L, t)
        ld = (hi - lo + 3) // 4 * 4
        leaves.append((lo, hi - lo, ld, dl))
        dl += ld * (hi - lo)
    snorm = np.linalg.norm(S, 2)
    path = d / f"hc_{esz}.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("10q", ng, len(blocks), len(leaves), uv, dl, kmax, over, SC, seed, esz))
        f.write(struct.pack("2d", tol, snorm))
        f.write(np.ascontiguousarray(S.T).tobytes())          # column-major, as stored
        for b in blocks:
            f.write(struct.pack("8q", b["c0"] * ng + b["r0"], ng, b["p"], b["q"], b["s"], 0,
                                b["u"], b["v"]))
        for lf in leaves:
            f.write(struct.pack("4q", *lf))
    out = path.with_suffix(".out")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    raw = np.fromfile(out, dtype=np.float64)
    UVs, UV = raw[:uv], raw[uv:2 * uv]
    ranks = raw[2 * uv:2 * uv + len(blocks)].astype(int)
    D = raw[2 * uv + len(blocks):]
    assert D.size == dl
    assert ranks.min() > 0                 # every block of this operator has numerical rank
    Sw = S if esz == 8 else S.astype(np.float32).astype(np.float64)
    u = 2.0 ** -53 if esz == 8 else 2.0 ** -24
    thr = tol * snorm
    bound = 10.0 * np.sqrt(2.0 / np.pi) * thr
    H = O.hodlr_compress(S, tol, leaf)
    o6 = [blk for lev in H["levels"] for blk in lev]
    for i, b in enumerate(blocks):
        B = Sw[b["r0"]:b["r0"] + b["p"], b["c0"]:b["c0"] + b["q"]]
        p, q, s = b["p"], b["q"], b["s"]
        Om = UVs[b["v"]:b["v"] + q * s].reshape(s, q).T
        Y = UVs[b["u"]:b["u"] + p * s].reshape(s, p).T
        Yr = B @ Om
        assert np.abs(Y - Yr).max() <= 4 * q * u * np.abs(B).max() * np.abs(Om).max()
        r = ranks[i]
        assert 0 <= r <= min(s, kmax)
        Q = UV[b["u"]:b["u"] + p * r].reshape(r, p).T
        V = UV[b["v"]:b["v"] + q * r].reshape(r, q).T
        assert np.abs(Q.T @ Q - np.eye(r)).max() <= 64 * p * u
        assert np.abs(V - B.T @ Q).max() <= 4 * p * u * np.abs(B).max()
        err = np.linalg.norm(B - Q @ V.T, 2) if min(p, q) else 0.0
        assert err <= bound + 64 * p * u * snorm, (i, err, bound)
        sig = np.linalg.svd(B, compute_uv=False)
        assert r >= int(np.sum(sig > bound + 64 * p * u * snorm))
        # O6 (truncated SVD at thr) meets the same bound with rank at most the kernel's + over
        U6, V6 = o6[i]
        assert np.linalg.norm(S[b["r0"]:b["r0"] + p, b["c0"]:b["c0"] + q] - U6 @ V6.T, 2) <= thr * (1 + 1e-10)
        assert U6.shape[1] <= r + over
    for lo, ln, ld, off in leaves:
        blk = D[off:off + ld * ln].reshape(ln, ld).T          # column-major ld x len
        assert np.array_equal(blk[:ln], Sw[lo:lo + ln, lo:lo + ln])
        assert np.all(blk[ln:] == 0.0)
