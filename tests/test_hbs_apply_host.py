"""The HBS kernels compiled for the host from `csrc/hbs.cu` itself and run with one OS thread per
CUDA thread (`tests/hostemu/cuda_host_shim.h`).  CPU only: this checks the kernels' index
arithmetic and their barriers, including races between threads of a CTA, which a sequential
re-statement of the same arithmetic would hide.

* The apply kernels (upward pass, levels above the cut, downward pass with output) on HBS
  factors that the oracle's O9 computes, laid out in the library's device format (heap-ordered
  nodes, U, V and D column-major): the output equals the oracle's telescoping apply (Sec. 2.4)
  to rounding, in both directions, on trees of depth 0 to 6 with ragged leaves.
* The node compression kernel, level by level from the leaves, on the oracle's samples
  (Alg. 1's Y = S Omega, Z = S^T Psi): the operator its factors define equals the oracle's.
* The sampling kernel: Y = S Omega and Z = S^T Psi with ragged tiles equal the plain product.

Every build runs under AddressSanitizer with buffers at the sizes the library allocates."""
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
# AddressSanitizer turns every out-of-bounds access of the kernels (shared arrays are statics,
# device buffers are host vectors) into a failure
SANITIZE = [SANITIZE, "-fno-omit-frame-pointer"]

MAIN = r'''
#include <cstdio>
#include <fstream>
using namespace ddst;
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  auto rd = [&](int64_t* p, int n) { f.read((char*)p, 8 * n); };
  int64_t h[9]; rd(h, 9);
  const int ng = (int)h[0], k = (int)h[1], leaf = (int)h[2], tr = (int)h[3];
  const int nn = (int)h[5], nup = (int)h[6], nown = (int)h[7];
  const int64_t nf = h[8];
  int64_t so; rd(&so, 1);
  std::vector<HbsNode> nodes(nn);
  for (auto& nd : nodes) {
    int64_t a[10]; rd(a, 10);
    nd.blk = (int)a[0]; nd.level = (int)a[1]; nd.n = (int)a[2]; nd.t = (int)a[3]; nd.lo = a[4];
    nd.in_row = a[5]; nd.out_row = a[6]; nd.u_off = a[7]; nd.v_off = a[8]; nd.d_off = a[9];
  }
  int64_t bb[5]; rd(bb, 5);
  HbsBlock blk{};
  blk.ng = bb[0]; blk.L = (int)bb[1]; blk.node0 = (int)bb[2]; blk.xh_off = bb[3]; blk.yh_off = bb[4];
  blk.in_if = 0; blk.out_if = 0;
  std::vector<HbsLeafItem> up(nup);
  for (auto& u : up) { int64_t a[2]; rd(a, 2); u.blk = (int)a[0]; u.node = (int)a[1]; }
  std::vector<HbsOwn> own(nown);
  for (auto& o : own) {
    int64_t a[8]; rd(a, 8);
    o.out = a[0]; o.lo = a[1]; o.len = (int)a[2]; o.nsrc = (int)a[3];
    o.blk[0] = (int)a[4]; o.blk[1] = (int)a[5]; o.node[0] = (int)a[6]; o.node[1] = (int)a[7];
  }
  std::vector<double> F(nf), x(ng), y(ng, 0.0), scratch(so, 0.0);
  f.read((char*)F.data(), 8 * nf); f.read((char*)x.data(), 8 * ng);
  if (blk.L > 0) {
    host_launch(nup, 256, [&] { k_hbs_up<double>(up.data(), &blk, nodes.data(), F.data(), x.data(),
                                                scratch.data(), tr, k, nullptr, 0); });
    host_launch(1, 256, [&] { k_hbs_top<double>(&blk, nodes.data(), F.data(), scratch.data(), tr, k); });
  }
  host_launch(nown, 256, [&] { k_hbs_down<double>(own.data(), &blk, nodes.data(), F.data(),
                                                  scratch.data(), x.data(), y.data(), tr, 1, k,
                                                  leaf, nullptr, 0); });
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)y.data(), 8 * ng);
  return 0;
}
'''


def _cut_level():
    """The tree cut of the apply, read from the kernel source (L > c ? L - c : 1)."""
    src = open(os.path.join(CSRC, "hbs.cu")).read()
    m = re.search(r"int hbs_cut_level\(int L\) \{ return L > (\d+) \? L - (\d+) : 1; \}", src)
    assert m and m.group(1) == m.group(2), "hbs_cut_level not found"
    c = int(m.group(1))
    return lambda L: L - c if L > c else 1


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "hbs.cu")).read()
    hdr = open(os.path.join(CSRC, "hbs.cuh")).read()
    i = src.index("// Apply\n")
    i = src.rindex("// ----", 0, i)
    j = src.index("// Host side\n")
    j = src.rindex("// ----", 0, j)
    structs = [re.search(r"struct %s \{.*?\n\};" % n, hdr, re.S).group(0)
               for n in ("HbsNode", "HbsBlock", "HbsOwn", "HbsLeafItem")]
    d = tmp_path_factory.mktemp("hbs_host")
    code = ('#include "cuda_host_shim.h"\nnamespace ddst {\n' + "\n".join(structs) + "\n" +
            src[i:j] + "\n}  // namespace ddst\n" + MAIN)
    (d / "hbs_apply_host.cpp").write_text(code)
    exe = d / "hbs_apply_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", *SANITIZE, "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "hbs_apply_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


def _case(d, ng, k, leaf, tr, cut):
    """Oracle HBS factors of a random S in the device layout, the apply's work items, and x."""
    rng = np.random.default_rng(ng * 7 + k)
    s = 3 * k + 10
    S = rng.standard_normal((ng, ng))
    Om, Ps = rng.standard_normal((ng, s)), rng.standard_normal((ng, s))
    H = O.hbs_compress(S @ Om, S.T @ Ps, Om, Ps, k, leaf)
    L, lv = H["L"], H["levels"]
    F, nodes, fo = [], [], 0
    for lev in range(L + 1):
        for t in range(1 << lev):
            lo = (t * ng) >> lev
            n = (((t + 1) * ng) >> lev) - lo if lev == L else 2 * k
            u = v = -1
            if lev > 0:
                U, V, D = lv[lev][t]
                u = fo; F.append(U.T.ravel()); fo += n * k
                v = fo; F.append(V.T.ravel()); fo += n * k
            else:
                D = lv[0]
                n = D.shape[0]
            dd = fo; F.append(D.T.ravel()); fo += n * n
            nodes.append((0, lev, n, t, lo, 0, 0, u, v, dd))
    F = np.concatenate(F)
    so = ((2 << L) - 1) * k + max(1, (1 << L) - 1) * 2 * k
    ls = 0 if L == 0 else cut(L)
    up = [(0, (1 << ls) - 1 + t) for t in range(1 << ls)] if L > 0 else []
    own = []
    for t in range(1 << ls):
        nd = (1 << ls) - 1 + t
        lo = nodes[nd][4]
        own.append((0, lo, (((t + 1) * ng) >> ls) - lo, 1, 0, 0, nd, 0))
    x = rng.standard_normal(ng)
    path = d / f"case_{ng}_{k}_{leaf}_{tr}.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("9q", ng, k, leaf, tr, L, len(nodes), len(up), len(own), F.size))
        f.write(struct.pack("q", so))
        for nd in nodes:
            f.write(struct.pack("10q", *nd))
        f.write(struct.pack("5q", ng, L, 0, 0, ((2 << L) - 1) * k))
        for it in up:
            f.write(struct.pack("2q", *it))
        for o in own:
            f.write(struct.pack("8q", *o))
        f.write(F.astype(np.float64).tobytes())
        f.write(x.tobytes())
    return path, O.hbs_apply(H, x, transpose=bool(tr)), L


@pytest.mark.parametrize("ng,k,leaf", [(200, 6, 12), (137, 4, 8), (64, 8, 16), (9, 3, 12),
                                       (40, 10, 20), (1000, 8, 16)])
@pytest.mark.parametrize("tr", [0, 1])
def test_hbs_apply_kernels_on_the_host_match_the_oracle(harness, ng, k, leaf, tr):
    d, exe = harness
    path, want, L = _case(d, ng, k, leaf, tr, _cut_level())
    out = d / (path.name + ".y")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    y = np.fromfile(out, dtype=np.float64)
    assert np.abs(y - want).max() <= 1e-12 * np.abs(want).max(), (L, np.abs(y - want).max())


# ---------------------------------------------------------------------------------------------
# The compression kernel (one CTA per tree node, level by level) on the host
# ---------------------------------------------------------------------------------------------
NODE_MAIN = r'''
#include <cstdio>
#include <fstream>
using namespace ddst;
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  auto rd = [&](int64_t* p, int n) { f.read((char*)p, 8 * n); };
  int64_t h[8]; rd(h, 8);
  const int ng = (int)h[0], k = (int)h[1], s = (int)h[2], nn = (int)h[3], nsteps = (int)h[4];
  const int64_t nf = h[5], rows_max = h[7]; const int nmax = (int)h[6];
  std::vector<HbsNode> nodes(nn);
  for (auto& nd : nodes) {
    int64_t a[10]; rd(a, 10);
    nd.blk = (int)a[0]; nd.level = (int)a[1]; nd.n = (int)a[2]; nd.t = (int)a[3]; nd.lo = a[4];
    nd.in_row = a[5]; nd.out_row = a[6]; nd.u_off = a[7]; nd.v_off = a[8]; nd.d_off = a[9];
  }
  std::vector<std::vector<int>> steps(nsteps);
  for (auto& st : steps) {
    int64_t c; rd(&c, 1);
    st.resize(c);
    for (auto& id : st) { int64_t v; rd(&v, 1); id = (int)v; }
  }
  const int64_t rows = (int64_t)ng;
  std::vector<double> arr[8];  // the level arrays at the size the library allocates
  for (auto& a : arr) a.assign(rows_max * s, 0.0);
  for (int q = 0; q < 4; ++q) f.read((char*)arr[q].data(), 8 * rows * s);  // Y, Z, Omega, Psi
  std::vector<double> F(nf, 0.0);
  // the node workspace of the launch, exactly the size the library requests
  std::vector<unsigned char> dyn(hbs_node_smem(nmax, s, k, sizeof(double)));
  host_dynamic_smem = dyn.data();
  double *Yc = arr[0].data(), *Zc = arr[1].data(), *Oc = arr[2].data(), *Pc = arr[3].data();
  double *Yn = arr[4].data(), *Zn = arr[5].data(), *On = arr[6].data(), *Pn = arr[7].data();
  for (int d = 0; d < nsteps; ++d) {
    const std::vector<int>& lst = steps[d];
    host_launch((unsigned)lst.size(), 256, [&] {
      k_hbs_node<double>(nodes.data(), lst.data(), Yc, Zc, Oc, Pc, Yn, Zn, On, Pn, F.data(), k, s, nmax);
    });
    std::swap(Yc, Yn); std::swap(Zc, Zn); std::swap(Oc, On); std::swap(Pc, Pn);
  }
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)F.data(), 8 * nf);
  return 0;
}
'''


@pytest.fixture(scope="module")
def node_harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "hbs.cu")).read()
    hdr = open(os.path.join(CSRC, "hbs.cuh")).read()
    i = src.rindex("// ----", 0, src.index("// Node compression\n"))
    j = src.rindex("// ----", 0, src.index("// Apply\n"))
    body = src[i:j]
    dyn = "extern __shared__ __align__(16) unsigned char hbs_smem[];"
    assert body.count(dyn) == 1
    body = body.replace(dyn, "unsigned char* hbs_smem = host_dynamic_smem;")  # sized exactly below
    structs = [re.search(r"struct %s \{.*?\n\};" % n, hdr, re.S).group(0) for n in ("HbsNode",)]
    d = tmp_path_factory.mktemp("hbs_node_host")
    code = ('#include "cuda_host_shim.h"\nstatic unsigned char* host_dynamic_smem = nullptr;\n'
            "namespace ddst {\n" + "\n".join(structs) + "\n" + body + "\n}  // namespace ddst\n" + NODE_MAIN)
    (d / "hbs_node_host.cpp").write_text(code)
    exe = d / "hbs_node_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", *SANITIZE, "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "hbs_node_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


def _node_case(d, S, k, leaf, rng):
    """Samples of S and the node table of one operator in the library's layout: heap-ordered
    nodes with U, V, D offsets, and per step from the leaves the nodes with the rows of their
    samples (in_row) and of their k reduced rows in the next level's arrays (out_row)."""
    ng = S.shape[0]
    s = 3 * k + 10
    Om, Ps = rng.standard_normal((ng, s)), rng.standard_normal((ng, s))
    Y, Z = S @ Om, S.T @ Ps
    L = O.hodlr_levels(ng, leaf)
    nodes, fo = [], 0
    for lev in range(L + 1):
        for t in range(1 << lev):
            lo = (t * ng) >> lev
            n = (((t + 1) * ng) >> lev) - lo if lev == L else (2 * k if L > 0 else ng)
            nd = dict(level=lev, t=t, lo=lo, n=n, in_row=0, out_row=0, u=-1, v=-1)
            if lev > 0:
                nd["u"] = fo; fo += n * k
                nd["v"] = fo; fo += n * k
            nd["d"] = fo; fo += n * n
            nodes.append(nd)
    steps = [[(1 << lev) - 1 + t for t in range(1 << lev)] for lev in range(L, -1, -1)]
    for dd, ids in enumerate(steps):
        nxt = 0
        for i in ids:
            nd = nodes[i]
            if dd == 0:
                nd["in_row"] = nd["lo"]
            if nd["level"] > 0:
                nd["out_row"] = nxt
                nxt += k
                if nd["t"] % 2 == 0:
                    nodes[(1 << (nd["level"] - 1)) - 1 + nd["t"] // 2]["in_row"] = nd["out_row"]
    path = d / f"node_{ng}_{k}_{leaf}.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("8q", ng, k, s, len(nodes), len(steps), fo, max(nd["n"] for nd in nodes),
                            max(ng, (1 << L) * k)))
        for nd in nodes:
            f.write(struct.pack("10q", 0, nd["level"], nd["n"], nd["t"], nd["lo"], nd["in_row"],
                                nd["out_row"], nd["u"], nd["v"], nd["d"]))
        for ids in steps:
            f.write(struct.pack("q", len(ids)))
            f.write(struct.pack("%dq" % len(ids), *ids))
        for a in (Y, Z, Om, Ps):
            f.write(np.ascontiguousarray(a, dtype=np.float64).tobytes())
    return path, nodes, L, O.hbs_compress(Y, Z, Om, Ps, k, leaf)


def _expand(F, nodes, L, k):
    """Dense operator of the factors: A_0 = D_0, A_l = U_l A_{l-1} V_l^T + D_l."""
    import scipy.linalg as sla

    def mat(off, r, c):
        return F[off:off + r * c].reshape(c, r).T

    A = mat(nodes[0]["d"], nodes[0]["n"], nodes[0]["n"])
    for lev in range(1, L + 1):
        lv = nodes[(1 << lev) - 1:(2 << lev) - 1]
        A = (sla.block_diag(*[mat(nd["u"], nd["n"], k) for nd in lv]) @ A
             @ sla.block_diag(*[mat(nd["v"], nd["n"], k) for nd in lv]).T
             + sla.block_diag(*[mat(nd["d"], nd["n"], nd["n"]) for nd in lv]))
    return A


@pytest.mark.parametrize("kind,ng,k,leaf", [("exact", 200, 6, 12), ("exact", 137, 4, 8),
                                            ("exact", 9, 3, 12), ("exact", 40, 5, 10),
                                            ("transfer", 127, 8, 16)])
def test_hbs_node_kernel_on_the_host_matches_the_oracle(node_harness, kind, ng, k, leaf):
    """Same S, Omega, Psi: the factors the node kernel writes define the oracle's operator."""
    d, exe = node_harness
    rng = np.random.default_rng(ng + 3 * k)
    if kind == "exact":
        from test_oracle_pins import _random_hbs
        S = _random_hbs(ng, k, leaf, rng)
    else:
        import ddst_inputs as I
        prob = I.make_problem("convdiff2d", n=128, w=16)
        A, b = O.assemble(prob)
        geo = O.slab_geometry(2, 128, 16)
        S = np.asarray(O.transfer_blocks(A, geo, O.factor_local(A, geo), slabs=[2])[1][0])
    path, nodes, L, Ho = _node_case(d, S, k, leaf, rng)
    out = d / (path.name + ".F")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    F = np.fromfile(out, dtype=np.float64)
    Do = O.hbs_dense(Ho)
    err_o = np.linalg.norm(Do - S) / np.linalg.norm(S)
    assert np.linalg.norm(_expand(F, nodes, L, k) - Do) <= max(1e-10, 2 * err_o) * np.linalg.norm(S)


# ---------------------------------------------------------------------------------------------
# The sampling kernel (Y = S Omega, Z = S^T Psi) on the host
# ---------------------------------------------------------------------------------------------
SAMPLE_MAIN = r'''
#include <fstream>
using namespace ddst;
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  int64_t h[3]; f.read((char*)h, 24);
  const int64_t ng = h[0]; const int s = (int)h[1], trans = (int)h[2];
  std::vector<double> S(ng * ng), G(ng * s), Y(ng * s, 0.0);
  f.read((char*)S.data(), 8 * ng * ng); f.read((char*)G.data(), 8 * ng * s);
  SampBlk sb{S.data(), ng, 0};
  std::vector<SampItem> items;
  for (int64_t lo = 0; lo < ng; lo += 64) items.push_back(SampItem{0, lo});
  auto run = [&](auto kern) {
    host_launch((unsigned)items.size(), 256, [&] { kern(items.data(), &sb, G.data(), Y.data(), s, trans); });
  };
  if (s <= 32) run(k_hbs_sample<double, 2>);
  else if (s <= 64) run(k_hbs_sample<double, 4>);
  else run(k_hbs_sample<double, 6>);
  std::ofstream o(argv[2], std::ios::binary);
  o.write((const char*)Y.data(), 8 * ng * s);
  return 0;
}
'''


@pytest.fixture(scope="module")
def sample_harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "hbs.cu")).read()
    structs = [re.search(r"struct %s \{.*?\n\};" % n, src, re.S).group(0) for n in ("SampBlk", "SampItem")]
    i = src.index("// Y = S Omega (trans 0) or Z = S^T Psi (trans 1)")
    j = src.rindex("// ----", 0, src.index("// Node compression\n"))
    d = tmp_path_factory.mktemp("hbs_sample_host")
    code = ('#include "cuda_host_shim.h"\nnamespace ddst {\n' + "\n".join(structs) + "\n" + src[i:j] +
            "\n}  // namespace ddst\n" + SAMPLE_MAIN)
    (d / "hbs_sample_host.cpp").write_text(code)
    exe = d / "hbs_sample_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", *SANITIZE, "-I",
                        os.path.join(ROOT, "tests", "hostemu"), str(d / "hbs_sample_host.cpp"),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


@pytest.mark.parametrize("ng,s", [(200, 28), (77, 58), (130, 94), (31, 19)])
@pytest.mark.parametrize("trans", [0, 1])
def test_hbs_sample_kernel_on_the_host(sample_harness, ng, s, trans):
    """Y = S Omega (Z = S^T Psi) over 64-row tiles with ragged row, column and sample tails,
    S column-major as the library stores it, against the plain product."""
    d, exe = sample_harness
    rng = np.random.default_rng(ng + s + trans)
    S = rng.standard_normal((ng, ng))
    G = rng.standard_normal((ng, s))
    path = d / f"sample_{ng}_{s}_{trans}.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("3q", ng, s, trans))
        f.write(np.ascontiguousarray(S.T).tobytes())  # column-major S
        f.write(G.tobytes())
    out = d / (path.name + ".y")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    Y = np.fromfile(out, dtype=np.float64).reshape(ng, s)
    want = (S.T if trans else S) @ G
    assert np.abs(Y - want).max() <= 1e-12 * np.abs(want).max()
