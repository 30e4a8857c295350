"""HODLR compression of the transfer operators (Sec. 2.4) against the oracle's truncated-SVD
reference on the same cluster tree."""
import numpy as np
import pytest

import ddst_inputs as I
from oracle import ddst_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25991_gb300 import build as B
    B.build()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def solver(prob, precision, **opts):
    from paper_2510_25991_gb300 import ddst as D
    sol = D.Solver(dict(dim=prob["dim"], n=prob["n"], w=prob["w"], a=dev(prob["a"]),
                        b=tuple(prob["b"]) + (0.0,) * (3 - len(prob["b"])),
                        c=dev(prob["c"]) if prob.get("c") is not None else None),
                   precision=precision, **opts)
    sol.build_transfer()
    return sol


def oracle_blocks(prob):
    A, b = O.assemble(prob)
    geo = O.slab_geometry(prob["dim"], prob["n"], prob["w"])
    return geo, O.transfer_blocks(A, geo, O.factor_local(A, geo))


def test_hodlr_exact_when_tolerance_vanishes():
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("convdiff2d", n=64, w=16)
    geo, (Sp, Sn) = oracle_blocks(prob)
    sol = solver(prob, "fp64", leaf_size=8, k_max=64, oversample=10)
    sol.compress(1e-15)
    out = np.empty((geo.ngamma, geo.ngamma))
    for j in range(geo.nds):
        for side, ref in ((-1, Sp[j]), (1, Sn[j])):
            if ref is None:
                continue
            D.ddst_get_transfer(sol.ctx, 0, j + 1, side, out)
            assert np.abs(out - ref).max() <= 1e-10 * np.abs(ref).max()
    sol.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_compress_with_leaf_covering_the_whole_block(precision):
    """n_Gamma = 63 <= leaf size: the cluster tree has no low-rank level, every S block is one
    dense leaf; compression, both applies and the solve still work."""
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("convdiff2d", n=64, w=16)
    A, b = O.assemble(prob)
    uref = O.global_solve(A, b)
    geo, (Sp, Sn) = oracle_blocks(prob)
    sol = solver(prob, precision, gmres_tol=1e-12 if precision == "fp64" else 0.0)
    sol.compress(1e-8)
    _, _, rank = D.ddst_query(sol.ctx)
    assert rank == 0
    u = torch.empty((63, 63), dtype=torch.float64, device="cuda")
    st, info = sol.solve(dev(prob["f"]), dev(prob["g"]), u)
    assert np.linalg.norm(u.cpu().numpy().ravel() - uref) / np.linalg.norm(uref) <= 1e-8, info
    rng = np.random.default_rng(5)
    nif = geo.nds * geo.ngamma
    x = rng.standard_normal(nif)
    K = np.zeros((nif, nif))
    for j in range(geo.nds):
        rows = slice(j * geo.ngamma, (j + 1) * geo.ngamma)
        if Sp[j] is not None:
            K[rows, (j - 1) * geo.ngamma:j * geo.ngamma] = Sp[j]
        if Sn[j] is not None:
            K[rows, (j + 1) * geo.ngamma:(j + 2) * geo.ngamma] = Sn[j]
    tol = 1e-12 if precision == "fp64" else 1e-3  # FP32 transfer operators (as for S itself)
    for tr, Kop in ((0, K), (1, K.T)):
        y = np.empty(nif)
        D.ddst_apply_interface(sol.ctx, 0, x, y, tr)
        ref = x - Kop @ x
        assert np.abs(y - ref).max() <= tol * np.abs(ref).max()
    sol.close()


@pytest.mark.parametrize("tol", [1e-6, 1e-8])
def test_hodlr_error_within_ten_tol_and_ranks_near_optimal(tol):
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("convdiff2d", n=256, w=32)
    geo, (Sp, Sn) = oracle_blocks(prob)
    leaf, q = 32, 10
    sol = solver(prob, "fp64", leaf_size=leaf, k_max=64, oversample=q)
    sol.compress(tol)
    _, _, gpu_max_rank = D.ddst_query(sol.ctx)
    out = np.empty((geo.ngamma, geo.ngamma))
    worst, opt_max_rank = 0.0, 0
    for j in range(geo.nds):
        for side, ref in ((-1, Sp[j]), (1, Sn[j])):
            if ref is None:
                continue
            nrm = np.linalg.norm(ref, 2)
            H = O.hodlr_compress(ref, tol, leaf, norm2=nrm)
            opt_max_rank = max(opt_max_rank, max(U.shape[1] for lev in H["levels"] for U, _ in lev))
            if j in (1, geo.nds // 2, geo.nds - 2):
                D.ddst_get_transfer(sol.ctx, 0, j + 1, side, out)
                worst = max(worst, np.linalg.norm(out - ref, 2) / nrm)
    sol.close()
    assert worst <= 10 * tol, worst
    # randomized range finder: ranks at most the optimal (truncated SVD) rank + oversampling
    assert opt_max_rank <= gpu_max_rank <= opt_max_rank + q, (gpu_max_rank, opt_max_rank)


@pytest.fixture(scope="module")
def helmholtz_blocks():
    """Helmholtz at 512^2, kappa = 100, 2w = 16-cell slabs (positive definite local operators by
    ~1%, the margin of the 4096^2, kappa = 200, w = 32 workload): every transfer block."""
    prob = I.make_problem("helmholtz2d", n=512, w=8, kappa=100.0)
    return (prob,) + oracle_blocks(prob)


@pytest.mark.parametrize("tol", [1e-6, 1e-8, 1e-10])
def test_helmholtz_hodlr_ranks_vs_tol(helmholtz_blocks, tol):
    """Ranks against the tolerance for the Helmholtz transfer operators: the error stays within
    10 tol and the ranks between the truncated-SVD optimum and optimum + oversampling."""
    from paper_2510_25991_gb300 import ddst as D
    prob, geo, (Sp, Sn) = helmholtz_blocks
    leaf, q = 32, 10
    sol = solver(prob, "fp64", leaf_size=leaf, k_max=64, oversample=q)
    sol.compress(tol)
    _, _, gpu_max_rank = D.ddst_query(sol.ctx)
    out = np.empty((geo.ngamma, geo.ngamma))
    worst, opt_max_rank = 0.0, 0
    for j in range(geo.nds):
        for side, ref in ((-1, Sp[j]), (1, Sn[j])):
            if ref is None:
                continue
            nrm = np.linalg.norm(ref, 2)
            H = O.hodlr_compress(ref, tol, leaf, norm2=nrm)
            opt_max_rank = max(opt_max_rank, max(U.shape[1] for lev in H["levels"] for U, _ in lev))
            if j in (1, geo.nds // 2, geo.nds - 2):
                D.ddst_get_transfer(sol.ctx, 0, j + 1, side, out)
                worst = max(worst, np.linalg.norm(out - ref, 2) / nrm)
    sol.close()
    assert worst <= 10 * tol, worst
    assert opt_max_rank <= gpu_max_rank <= opt_max_rank + q, (gpu_max_rank, opt_max_rank)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("mixed", 1e-8), ("mixed", 1e-6)])
def test_solve_through_hodlr(precision, tol):
    prob = I.make_problem("convdiff2d", n=256, w=32)
    A, b = O.assemble(prob)
    uref = O.global_solve(A, b)
    opts = dict(gmres_tol=1e-12) if precision == "fp64" else {}
    sol = solver(prob, precision, leaf_size=32, **opts)
    sol.compress(tol)
    u = torch.empty((255, 255), dtype=torch.float64, device="cuda")
    st, info = sol.solve(dev(prob["f"]), dev(prob["g"]), u)
    sol.close()
    err = np.linalg.norm(u.cpu().numpy().ravel() - uref) / np.linalg.norm(uref)
    assert err <= 1e-8, (err, info)
    assert info["max_rank"] > 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hodlr_transpose_apply(precision):
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("convdiff2d", n=128, w=16)
    sol = solver(prob, precision, leaf_size=16)
    sol.compress(1e-8)
    nds, ng, _ = D.ddst_query(sol.ctx)
    rng = np.random.default_rng(4)
    x, y = rng.standard_normal(nds * ng), rng.standard_normal(nds * ng)
    ax, aty = np.empty_like(x), np.empty_like(y)
    D.ddst_apply_interface(sol.ctx, 0, x, ax, False)
    D.ddst_apply_interface(sol.ctx, 0, y, aty, True)
    sol.close()
    # FP32 factors: both sides round differently, ~sqrt(terms) u_32 relative
    assert abs(ax @ y - x @ aty) <= (1e-12 if precision == "fp64" else 2e-5) * abs(ax @ y)
