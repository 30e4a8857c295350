"""The slab-geometry kernels of `csrc/stencil.cu`, compiled for the host and run with one OS
thread per CUDA thread under AddressSanitizer (`tests/hostemu/cuda_host_shim.h`), against the
oracle's index sets of the overlapping double slabs (Sec. 2, Fig. 2.1; Sec. 2.5: I_j, C_j,
J_{j,j'}) and its assembled matrix (O1):
* `k_gather`: every slab-local vector is the volume restricted to I_j (padding zero);
* `k_extract_center`: the local values at the central plane are those at Gamma_j (C_j);
* `k_add_iface_dirichlet`: the neighbouring interfaces enter the local right-hand side as
  -A(I_j, J_{j,j-1}) u_{j-1} - A(I_j, J_{j,j+1}) u_{j+1} (from the stencil pack);
* `k_scatter`: the owned planes of the slabs partition the interior unknowns;
* `k_gather_T`: adds each unknown once per double slab that contains it (1 or 2);
* `k_gather_owned`: the gather restricted to the planes each slab owns (adjoint of the scatter);
* `k_iface_dirichlet_T`, `k_inject_center`: the transposes of the two interface maps
  (dot-product identities), in 2D and 3D."""
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
int main(int argc, char** argv) {
  std::ifstream f(argv[1], std::ios::binary);
  int64_t h[6]; double d[4]; f.read((char*)h, 48); f.read((char*)d, 32);
  const int dim = (int)h[0], n = (int)h[1], w = (int)h[2], M = (int)h[3], has_c = (int)h[4];
  const int64_t nnode = h[5];
  ProbDesc P{}; P.dim = dim; P.n = n; P.w = w; P.nds = n / w - 1; P.has_c = has_c;
  P.h = d[0]; P.b[0] = d[1]; P.b[1] = d[2]; P.b[2] = d[3];
  const int p = dim == 2 ? 1 : n - 1, m = (2 * w - 1) * p, nb = n - 1, nds = P.nds;
  const int64_t ng = (int64_t)nb * p, nint = (int64_t)nb * nb * p, nloc = (int64_t)nds * nb * M;
  P.nint = nint; P.ng = ng;
  std::vector<SlabDesc> slabs(nds);
  for (int q = 0; q < nds; ++q) {
    SlabDesc s{};
    s.prob = 0; s.j = q + 1; s.M = M; s.m = m; s.nb = nb; s.p = p; s.w = w; s.n = n; s.ng = ng;
    s.pack_off = (int64_t)q * nb * PK_NFIELDS * M; s.loc_off = (int64_t)q * nb * M;
    s.vol_off = 0; s.node_off = 0; s.if_off = (int64_t)q * ng;
    slabs[q] = s;
  }
  std::vector<double> A(nnode), C(nnode), uG(nds * ng), z(nloc);
  f.read((char*)A.data(), 8 * nnode); f.read((char*)C.data(), 8 * nnode);
  f.read((char*)uG.data(), 8 * nds * ng); f.read((char*)z.data(), 8 * nloc);
  std::vector<double> pack((int64_t)nds * nb * PK_NFIELDS * M), vol(nint), gmap(nloc, -1.0),
      center(nds * ng, 0.0), dir(nloc, 0.0), ones(nloc, 1.0), scat(nint, 0.0), gT(nint, 0.0),
      idT(nds * ng, 0.0), inj(nloc, 0.0), owned(nloc, -1.0);
  for (int64_t e = 0; e < nint; ++e) vol[e] = (double)e;
  auto L = [&](std::function<void()> fn) { host_launch2(2, nds, 128, fn); };
  host_launch2(nb, nds, 128, [&] { k_stencil_pack<double>(slabs.data(), &P, A.data(), C.data(), pack.data()); });
  L([&] { k_gather<double>(slabs.data(), vol.data(), gmap.data()); });
  L([&] { k_extract_center<double>(slabs.data(), gmap.data(), center.data()); });
  L([&] { k_add_iface_dirichlet<double>(slabs.data(), &P, pack.data(), uG.data(), dir.data()); });
  L([&] { k_scatter<double>(slabs.data(), &P, ones.data(), scat.data(), 1); });
  L([&] { k_gather_T<double>(slabs.data(), ones.data(), gT.data()); });
  L([&] { k_iface_dirichlet_T<double>(slabs.data(), &P, pack.data(), z.data(), idT.data()); });
  L([&] { k_inject_center<double>(slabs.data(), uG.data(), inj.data()); });
  L([&] { k_gather_owned<double>(slabs.data(), &P, vol.data(), owned.data()); });
  std::ofstream o(argv[2], std::ios::binary);
  for (auto* v : {&gmap, &center, &dir, &scat, &gT, &idT, &inj, &owned}) o.write((const char*)v->data(), 8 * v->size());
  return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = open(os.path.join(CSRC, "stencil.cu")).read()
    common = open(os.path.join(CSRC, "common.cuh")).read()
    structs = [re.search(r"struct %s \{.*?\n\};" % nme, common, re.S).group(0)
               for nme in ("ProbDesc", "SlabDesc")]
    enum = re.search(r"enum PackField \{.*?\};", common, re.S).group(0)
    vidx = re.search(r"__device__ __forceinline__ int64_t vol_index\(.*?\n\}", common, re.S).group(0)
    i = src.index("__device__ __forceinline__ int64_t node_index(")
    j = src.index("// b = f + (Dirichlet neighbour terms)")
    k0 = src.index("// Slab-local gather:")
    k1 = src.index("// Partial sums of x.y over n elements")
    d = tmp_path_factory.mktemp("slab_host")
    code = ('#include "cuda_host_shim.h"\nnamespace ddst {\n' + enum + "\n" + "\n".join(structs) +
            "\n" + vidx + "\n" + src[i:j] + "\n" + src[k0:k1] + "\n}  // namespace ddst\n" + MAIN)
    (d / "slab_host.cpp").write_text(code)
    exe = d / "slab_host"
    r = subprocess.run([cxx, "-std=c++20", "-O1", "-pthread", SANITIZE,
                        "-fno-omit-frame-pointer", "-I", os.path.join(ROOT, "tests", "hostemu"),
                        str(d / "slab_host.cpp"), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return d, exe


@pytest.mark.parametrize("name,n,w", [("convdiff2d", 16, 4), ("vardiff3d", 8, 2)])
def test_slab_geometry_kernels_on_the_host(harness, name, n, w):
    d, exe = harness
    prob = I.make_problem(name, n=n, w=w)
    dim = prob["dim"]
    p = 1 if dim == 2 else n - 1
    m, nb = (2 * w - 1) * p, n - 1
    M = ((m + 31) // 32) * 32 + (32 if m % 32 == 0 else 0)
    geo = O.slab_geometry(dim, n, w)
    nds, ng = geo.nds, geo.ngamma
    nint, nloc = nb ** dim, nds * nb * M
    rng = np.random.default_rng(n)
    uG = rng.standard_normal(nds * ng)
    z = rng.standard_normal(nloc)
    has_c = prob.get("c") is not None
    bb = list(prob["b"]) + [0.0] * (3 - len(prob["b"]))
    nnode = (n + 1) ** dim
    path = d / f"slab_{name}.bin"
    with open(path, "wb") as f:
        f.write(struct.pack("6q", dim, n, w, M, int(has_c), nnode) + struct.pack("4d", 1.0 / n, *bb))
        f.write(np.asarray(prob["a"], dtype=np.float64).ravel().tobytes())
        f.write((np.asarray(prob["c"], dtype=np.float64).ravel() if has_c else np.zeros(nnode)).tobytes())
        f.write(uG.tobytes())
        f.write(z.tobytes())
    out = d / (path.name + ".out")
    r = subprocess.run([str(exe), str(path), str(out)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    raw = np.fromfile(out, dtype=np.float64)
    sizes = [nloc, nds * ng, nloc, nint, nint, nds * ng, nloc, nloc]
    gmap, center, dirv, scat, gT, idT, inj, owned = np.split(raw, np.cumsum(sizes)[:-1])
    gmap = gmap.reshape(nds, nb, M)
    A = sp.csr_matrix(O.assemble(prob)[0])
    count = np.zeros(nint)
    for j in range(nds):
        loc = gmap[j, :, :m].ravel()
        assert np.all(gmap[j, :, m:] == 0.0)                       # padding
        assert sorted(loc.astype(np.int64)) == sorted(geo.I[j])     # the unknowns of Psi_j
        assert np.array_equal(center[j * ng:(j + 1) * ng].astype(np.int64), geo.G[j])  # Gamma_j
        gm = loc.astype(np.int64)
        want = np.zeros(gm.size)
        if geo.Jprev[j] is not None:
            want -= A[gm][:, geo.Jprev[j]] @ uG[(j - 1) * ng:j * ng]
        if geo.Jnext[j] is not None:
            want -= A[gm][:, geo.Jnext[j]] @ uG[(j + 1) * ng:(j + 2) * ng]
        got = dirv.reshape(nds, nb, M)[j, :, :m].ravel()
        assert np.abs(got - want).max() <= 1e-12 * max(1.0, np.abs(want).max())
        count[geo.I[j]] += 1
    assert np.all(scat == 1.0)             # owned planes partition the interior
    # gather restricted to the owned planes (the adjoint of the scatter): slab j owns its first
    # w x-planes, the last slab all 2w - 1; the rest of the row and the padding are zero
    owned = owned.reshape(nds, nb, M)
    for j in range(nds):
        ncx = 2 * w - 1 if j == nds - 1 else w
        mask = np.zeros(M, dtype=bool)
        mask[:ncx * p] = True
        assert np.array_equal(owned[j][:, mask], gmap[j][:, mask])
        assert np.all(owned[j][:, ~mask] == 0.0)
    assert np.array_equal(gT, count)       # overlap multiplicity
    # transposes: <dirichlet(uG), z> = <uG, dirichlet_T(z)>, <inject(uG), z> = <uG, extract(z)>
    assert abs(dirv @ z - uG @ idT) <= 1e-11 * max(1.0, abs(dirv @ z))
    zc = z.reshape(nds, nb, M)[:, :, (w - 1) * p:w * p].reshape(nds, -1)  # extract of z
    assert abs(inj @ z - uG @ zc.ravel()) <= 1e-11 * max(1.0, abs(inj @ z))
