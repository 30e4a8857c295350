"""Two more workloads at full size (mixed precision, the default launch configuration):

* Helmholtz, 4096^2 grid, kappa = 200, 127 double slabs of 64 cells (the ranks-vs-tolerance
  configuration): sampled transfer-operator rows against oracle transposed local solves, and
  HODLR compression at tol 1e-6 / 1e-8 against the dense operator (ranks non-decreasing, error
  within 10 tol or the FP32 floor of the mixed path).  The interface GMRES of this strongly indefinite global problem is not part
  of the check: with 127 slabs at 32 wavelengths it does not converge in the iteration cap
  (the reduced-size Helmholtz tests cover the solve).
* The uneven batch of 64 independent diffusion problems (256^2 .. 1024^2 grids, 8-32 slabs):
  one batched setup, solve and adjoint; loss and gradients of three sampled problems (smallest,
  median, largest) against the oracle.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import ddst_inputs as I
from oracle import ddst_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _norm2(M, iters=30, seed=0):
    """||M||_2 by power iteration on M^T M (host)."""
    x = np.random.default_rng(seed).standard_normal(M.shape[1])
    s = 0.0
    for _ in range(iters):
        y = M.T @ (M @ x)
        s = np.linalg.norm(y)
        x = y / s
    return np.sqrt(s)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25991_gb300 import build as B
    B.build()


def test_helmholtz_4096_transfer_rows_and_hodlr_tolerances():
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("helmholtz2d")
    n, w = prob["n"], prob["w"]
    assert (n, w) == (4096, 32)
    sol = D.Solver(dict(dim=2, n=n, w=w, a=_dev(prob["a"]), b=tuple(prob["b"]) + (0.0,), c=_dev(prob["c"])),
                   precision="mixed", k_max=64, oversample=10)
    sol.build_transfer()
    geo = O.slab_geometry(2, n, w)
    ng = geo.ngamma
    j = geo.nds // 2
    dense = {}
    for side in (-1, 1):
        out = np.empty((ng, ng))
        D.ddst_get_transfer(sol.ctx, 0, j + 1, side, out)
        dense[side] = out
    # sampled rows against oracle transposed local solves
    A, b = O.assemble(prob)
    Acsr = sp.csr_matrix(A)
    I_ = geo.I[j]
    lu = spla.splu(sp.csc_matrix(Acsr[I_][:, I_].T))
    rows = np.random.default_rng(7).choice(ng, 6, replace=False)
    E = np.zeros((len(I_), len(rows)))
    E[geo.C[j][rows], np.arange(len(rows))] = 1.0
    Y = lu.solve(E)
    for side, J in ((-1, geo.Jprev[j]), (1, geo.Jnext[j])):
        ref = -(Acsr[I_][:, J].T @ Y).T
        assert np.abs(dense[side][rows] - ref).max() <= 1e-3 * np.abs(ref).max()
    del A, Acsr, lu
    # HODLR at two tolerances against the dense (FP32) operator.  In FP32 the range finder rejects
    # samples below 1e3 eps_32 of their own norm as rounding noise, which floors the compression
    # error there (the FP64 refinement of the solve removes it); the FP64 compression at these
    # tolerances and at 1e-10 is checked at reduced size.
    floor = 1e3 * float(np.finfo(np.float32).eps)
    ranks = []
    for tol in (1e-6, 1e-8):
        sol.compress(tol)
        ranks.append(D.ddst_query(sol.ctx)[2])
        for side in (-1, 1):
            out = np.empty((ng, ng))
            D.ddst_get_transfer(sol.ctx, 0, j + 1, side, out)
            err = _norm2(out - dense[side]) / _norm2(dense[side])
            assert err <= max(10 * tol, floor), (tol, side, err)
    assert 0 < ranks[0] <= ranks[1] <= 64, ranks
    sol.close()


def test_adjoint_batch_of_64_uneven_problems():
    from paper_2510_25991_gb300 import ddst as D
    specs = I.batch_specs(64)
    probs = [I.batch_problem(s) for s in specs]
    sol = D.Solver([dict(dim=2, n=p["n"], w=p["w"], a=_dev(p["a"]), b=(0.0, 0.0, 0.0)) for p in probs],
                   precision="mixed")
    sol.build_transfer()
    us = [torch.empty((p["n"] - 1, p["n"] - 1), dtype=torch.float64, device="cuda") for p in probs]
    D.ddst_solve_batch(sol.ctx, [_dev(p["f"]) for p in probs], [_dev(p["g"]) for p in probs], us)
    rng = np.random.default_rng(11)
    obs = [rng.standard_normal((p["n"] - 1) ** 2) for p in probs]
    dLdu = [_dev((u.cpu().numpy().ravel() - o).reshape(u.shape)) for u, o in zip(us, obs)]
    dfs = [torch.empty_like(u) for u in us]
    dgs = [torch.empty((p["n"] + 1, p["n"] + 1), dtype=torch.float64, device="cuda") for p in probs]
    das = [torch.empty_like(x) for x in dgs]
    D.ddst_solve_adjoint_batch(sol.ctx, dLdu, dfs, dgs, das)
    sol.close()
    order = np.argsort([p["n"] for p in probs], kind="stable")
    for i in (order[0], order[len(order) // 2], order[-1]):
        p = probs[i]
        L, dLdf, dLdg, dLda, uref, lam = O.loss_and_gradients(p, obs[i])
        u = us[i].cpu().numpy().ravel()
        assert np.linalg.norm(u - uref) / np.linalg.norm(uref) <= 1e-8
        assert abs(0.5 * np.sum((u - obs[i]) ** 2) - L) <= 1e-7 * L
        dLdf, dLda = np.ravel(dLdf), np.ravel(dLda)
        assert np.linalg.norm(dfs[i].cpu().numpy().ravel() - dLdf) <= 1e-8 * np.linalg.norm(dLdf)
        assert np.linalg.norm(das[i].cpu().numpy().ravel() - dLda) <= 1e-7 * np.linalg.norm(dLda)
