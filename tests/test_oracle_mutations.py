"""Planted mistakes in the oracle: every one must make at least one pin fail.

Each case replaces one line of ``oracle/ddst_oracle.py`` (in a copy, on the CPU) by a
plausible error -- a dropped term, a wrong sign, index or scale, a transposed or swapped
operand -- and runs ``tests/test_oracle_pins.py`` against the copy.  The run must fail.

One variant is left out on purpose: recording only the first Gram-Schmidt pass's
coefficients in the Hessenberg column while still orthogonalizing twice.  The second-pass
coefficients are of the order of rounding, so that variant gives the same iterates to
rounding and no pin can tell it apart; skipping the second pass altogether is included.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle", "ddst_oracle.py")

MUTATIONS = [
 ("O1 face mean dropped (a_p instead of (a_p+a_q)/2)", "af = 0.5 * (ap + aq)\n            coef", "af = ap\n            coef"),
 ("O1 convection sign", "coef = -af / h ** 2 + s * bconv[d]", "coef = -af / h ** 2 - s * bconv[d]"),
 ("O1 convection scale 1/h instead of 1/(2h)", "s * bconv[d] / (2.0 * h)", "s * bconv[d] / h"),
 ("O1 boundary data sign", "rhs[P[bnd]] -= coef[bnd]", "rhs[P[bnd]] += coef[bnd]"),
 ("O1 reaction dropped", "diag += c[_interior(dim, n)].ravel()", "diag += 0.0"),
 ("O1 diagonal from a_p instead of face mean", "diag += af / h ** 2", "diag += ap / h ** 2"),
 ("geometry: central plane off by one", "geo.C.append((j * w - lo) * rest", "geo.C.append((j * w - lo + 1) * rest"),
 ("geometry: previous interface plane off by one", "plane((j - 1) * w) if j >= 2", "plane((j - 1) * w + 1) if j >= 2"),
 ("geometry: double slab one plane short", "lo, hi = (j - 1) * w + 1, (j + 1) * w - 1", "lo, hi = (j - 1) * w + 1, (j + 1) * w - 2"),
 ("O3 sign of S", "out.append(-lu.solve(rhs)[C, :])", "out.append(lu.solve(rhs)[C, :])"),
 ("O3 S_{j,j-1} and S_{j,j+1} swapped", "Sp.append(out[0]); Sn.append(out[1])", "Sp.append(out[1]); Sn.append(out[0])"),
 ("O3 S transposed", "out.append(-lu.solve(rhs)[C, :])", "out.append(-lu.solve(rhs)[C, :].T)"),
 ("O3 fhat from the neighbouring slab's factor", "return [facs[j].solve(np.asarray(b)[geo.I[j]])[geo.C[j]]", "return [facs[max(j - 1, 0)].solve(np.asarray(b)[geo.I[j]])[geo.C[j]]"),
 ("O4 interface matrix sign", "M[j * m:(j + 1) * m, (j - 1) * m:j * m] = -Sp[j]", "M[j * m:(j + 1) * m, (j - 1) * m:j * m] = Sp[j]"),
 ("O4 interface matrix block transposed", "M[j * m:(j + 1) * m, (j + 1) * m:(j + 2) * m] = -Sn[j]", "M[j * m:(j + 1) * m, (j + 1) * m:(j + 2) * m] = -Sn[j].T"),
 ("O4 apply with transposed S", "Y[j] -= Sp[j] @ X[j - 1]", "Y[j] -= Sp[j].T @ X[j - 1]"),
 ("O4 block Thomas back-substitution sign", "u[j] = sla.solve(Dm[j], r[j] + Sn[j] @ u[j + 1])", "u[j] = sla.solve(Dm[j], r[j] - Sn[j] @ u[j + 1])"),
 ("O4 GMRES single classical Gram-Schmidt pass", "        h2 = V[:k] @ wv\n        wv = wv - V[:k].T @ h2\n        hcol = h1 + h2\n", "        hcol = h1\n"),
 ("O4 GMRES Givens sign", "gvec[k] = -sn[k - 1] * gvec[k - 1]", "gvec[k] = sn[k - 1] * gvec[k - 1]"),
 ("O4 GMRES rotation of new column sign", "H[i + 1, k - 1] = -sn[i] * H[i, k - 1] + cs[i] * H[i + 1, k - 1]", "H[i + 1, k - 1] = sn[i] * H[i, k - 1] + cs[i] * H[i + 1, k - 1]"),
 ("O5 Dirichlet data sign in reconstruction", "rhs -= A[I][:, geo.Jprev[j]] @ U[j - 1]", "rhs += A[I][:, geo.Jprev[j]] @ U[j - 1]"),
 ("O5 kept planes off by one", "keep = w * rest if j < nds - 1", "keep = (w - 1) * rest if j < nds - 1"),
 ("O6 rank one short", "r = int(np.sum(s > thr))", "r = max(int(np.sum(s > thr)) - 1, 0)"),
 ("O6 lower block taken from the upper one", "for (r0, r1, c0, c1) in ((lo1, hi1, lo2, hi2), (lo2, hi2, lo1, hi1)):", "for (r0, r1, c0, c1) in ((lo1, hi1, lo2, hi2), (lo1, hi1, lo2, hi2)):"),
 ("O6 tree node boundary off by one", "return (t * ng) >> level, ((t + 1) * ng) >> level", "return (t * ng + 1) >> level, ((t + 1) * ng + 1) >> level"),
 ("O6 apply reads the wrong half of x", "y[lo1:hi1] += U @ (V.T @ x[lo2:hi2])", "y[lo1:hi1] += U @ (V.T @ x[lo1:hi1])"),
 ("O6 threshold relative to max|S| instead of ||S||_2", "norm2 = np.linalg.norm(S, 2)", "norm2 = np.abs(S).max()"),
 ("O7 adjoint without transpose", "lu = spla.splu(sp.csc_matrix(sp.csr_matrix(A).T))", "lu = spla.splu(sp.csc_matrix(sp.csr_matrix(A)))"),
 ("O7 dL/da face sign", "dface = -(lam_full[lo] - lam_full[hi])", "dface = (lam_full[lo] - lam_full[hi])"),
 ("O7 dL/da face not split between nodes", "dLda[lo] += 0.5 * dface", "dLda[lo] += dface"),
 ("O7 dL/dg convection sign (upper boundary)", "lam_full[lo] * (af / h ** 2 - bconv[d] / (2 * h))", "lam_full[lo] * (af / h ** 2 + bconv[d] / (2 * h))"),
 ("O7 dL/dg convection sign (lower boundary)", "lam_full[hi] * (af / h ** 2 + bconv[d] / (2 * h))", "lam_full[hi] * (af / h ** 2 - bconv[d] / (2 * h))"),
 ("O2b sine-transform eigenvalue pi k / n instead of pi k / (2n)", "lam1 = 4.0 * n * n * np.sin(np.pi * k / (2.0 * n)) ** 2", "lam1 = 4.0 * n * n * np.sin(np.pi * k / n) ** 2"),
 ("O3b transverse eigenvalue pi k / n instead of pi k / (2n)", "mu1 = 4.0 * np.sin(np.pi * k / (2.0 * n)) ** 2", "mu1 = 4.0 * np.sin(np.pi * k / n) ** 2"),
 ("O2b DST of type 2 instead of 1", "bh = sfft.dstn(b.reshape((n - 1,) * dim), type=1)", "bh = sfft.dstn(b.reshape((n - 1,) * dim), type=2)"),
 ("O2c lambda_min without the dimension factor", "return dim * 4.0 * n * n * math.sin", "return 4.0 * n * n * math.sin"),
 ("O2c a_min dropped from the eigenvalue bound", "lam = float(np.min(prob[\"a\"])) * laplacian_lambda_min", "lam = 1.0 * laplacian_lambda_min"),
 ("O3b closed-form multiplier at the slab edge instead of the centre", "s = 1.0 / (2.0 * np.cosh(w * theta))", "s = 1.0 / (2.0 * np.cosh(2 * w * theta))"),
 ("O7 dL/da boundary u_q from 0 instead of g", "u_full = np.array(g, dtype=np.float64).copy()", "u_full = np.zeros_like(np.array(g, dtype=np.float64))"),
 ("O8 central difference without the 1/2", "U[_shifted(dim, n, d, -1)]) / (2.0 * h)", "U[_shifted(dim, n, d, -1)]) / h"),
 ("O8 convection term added", "f = f - np.asarray(vel[d])[_interior(dim, n)] * grad", "f = f + np.asarray(vel[d])[_interior(dim, n)] * grad"),
 ("O8 U_n / dt dropped", "f = U[_interior(dim, n)] / dt", "f = U[_interior(dim, n)] * 1.0"),
 ("O9 null basis from the row-space columns", "return Q[:, Om.shape[0]:]", "return Q[:, :Om.shape[0]]"),
 ("O9 D without the (I - U U^T) projection", "D = X1 - U @ (U.T @ X1) + U", "D = X1 + U"),
 ("O9 reduced column samples with D instead of D^T", "V.T @ (Zt - D.T @ Pt)", "V.T @ (Zt - D @ Pt)"),
 ("O9 reduced test matrices swapped", "V.T @ Ot, U.T @ Pt))", "U.T @ Ot, V.T @ Pt))"),
 ("O9 apply takes the sibling's slot of the parent", "slot = ys[t // 2][(t % 2) * k:(t % 2 + 1) * k]", "slot = ys[t // 2][(1 - t % 2) * k:(2 - t % 2) * k]"),
 ("O9 transposed apply keeps D untransposed", "nxt.append((D.T if transpose else D) @ xt", "nxt.append(D @ xt"),
 ("O8 one step fewer", "    for _ in range(nsteps):\n        u = lu.solve(imex_rhs(dim, n, u, vel, dt))", "    for _ in range(nsteps - 1):\n        u = lu.solve(imex_rhs(dim, n, u, vel, dt))"),
]


def _run_planted(d, old, new):
    """Runs the pins against a copy of the oracle with `old` replaced by `new`, in folder d."""
    src = open(ORACLE).read()
    shutil.copytree(os.path.join(ROOT, "tests"), d / "tests",
                    ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copytree(os.path.join(ROOT, "ddst_inputs"), d / "ddst_inputs",
                    ignore=shutil.ignore_patterns("__pycache__"))
    (d / "oracle").mkdir()
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), d / "oracle" / "__init__.py")
    (d / "oracle" / "ddst_oracle.py").write_text(src.replace(old, new))
    env = dict(os.environ, OMP_NUM_THREADS="2", OPENBLAS_NUM_THREADS="2", MKL_NUM_THREADS="2")
    return subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-x", "-q",
                           "-p", "no:cacheprovider"], cwd=d, capture_output=True, text=True,
                          timeout=600, env=env)


@pytest.fixture(scope="module")
def planted_runs(tmp_path_factory):
    """All planted variants, four pin runs at a time (each is its own Python process)."""
    dirs = [tmp_path_factory.mktemp("planted") for _ in MUTATIONS]
    with ThreadPoolExecutor(max_workers=4) as ex:
        runs = list(ex.map(lambda a: _run_planted(a[0], a[1][1], a[1][2]), zip(dirs, MUTATIONS)))
    return {m[0]: r for m, r in zip(MUTATIONS, runs)}


@pytest.mark.slow
@pytest.mark.timeout(1200)
@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_oracle_mistake_fails_a_pin(planted_runs, name, old, new):
    assert open(ORACLE).read().count(old) == 1, f"mutation site not found: {name}"
    r = planted_runs[name]
    assert r.returncode == 1, f"{name}: no pin failed\n{r.stdout[-2000:]}"
