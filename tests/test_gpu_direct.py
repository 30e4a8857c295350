"""The direct interface solver (interface_solver = 1): block cyclic reduction of the
block-tridiagonal equilibrium system (I - K) u = fhat (Sec. 1, Eq. (modelS); the direct solvers of
Sec. 4), against the oracle's block elimination (O4 block_thomas) on the oracle's own transfer
blocks, element by element, and the full solve against the global sparse solve (O2) and the
adjoint against O7.

Interface counts N_ds = 2, 3, 4, 7 and 15 give reduction trees with every shape of level (an even
or odd number of blocks, a last block with and without a right neighbour).  Tolerances: FP64
1e-10 relative to the largest entry; FP32 (transfer blocks and reduction in FP32, 3xTF32 tensor
cores) 2e-5 of the largest entry times the system's condition estimate, bounded by 1e-3."""
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


def _spec(p):
    return dict(dim=p["dim"], n=p["n"], w=p["w"], a=dev(p["a"]),
                b=tuple(p["b"]) + (0.0,) * (3 - len(p["b"])),
                c=dev(p["c"]) if p.get("c") is not None else None)


def _relerr(x, ref):
    return np.linalg.norm(x - ref) / np.linalg.norm(ref)


# (n, w): N_ds = n / w - 1 interfaces of n - 1 points
SHAPES = [(48, 16), (64, 16), (80, 16), (64, 8), (128, 8)]


@pytest.mark.parametrize("n,w", SHAPES)
@pytest.mark.parametrize("precision,tc", [("fp64", 0), ("mixed", 1), ("mixed", 0)])
def test_direct_interface_solve_matches_block_elimination(n, w, precision, tc):
    from paper_2510_25991_gb300 import ddst as D
    p = I.make_problem("convdiff2d", n=n, w=w)
    A, b = O.assemble(p)
    geo = O.slab_geometry(2, n, w)
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo))
    Mi = O.interface_matrix(Sp, Sn, geo.ngamma)
    rng = np.random.default_rng(n + w)
    r = rng.standard_normal(geo.nds * geo.ngamma)
    ref = O.block_thomas(Sp, Sn, list(r.reshape(geo.nds, geo.ngamma)))
    refT = np.linalg.solve(Mi.T, r)
    sol = D.Solver(_spec(p), precision=precision, tensor_cores=tc)
    sol.build_transfer()
    x = torch.empty(r.size, dtype=torch.float64, device="cuda")
    xt = torch.empty_like(x)
    D.ddst_solve_interface(sol.ctx, 0, dev(r), x)
    D.ddst_solve_interface(sol.ctx, 0, dev(r), xt, transpose=True)
    sol.close()
    cond = np.linalg.cond(Mi)
    tol = 1e-10 if precision == "fp64" else min(1e-3, 2e-5 * cond)
    assert np.abs(x.cpu().numpy() - ref).max() <= tol * np.abs(ref).max(), cond
    assert np.abs(xt.cpu().numpy() - refT).max() <= tol * np.abs(refT).max(), cond


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_direct_solve_and_adjoint_match_oracle(precision):
    from paper_2510_25991_gb300 import ddst as D
    p = I.make_problem("convdiff2d", n=256, w=16)  # 15 interfaces of 255 points
    n = p["n"]
    A, b = O.assemble(p)
    uref = O.global_solve(A, b)
    sol = D.Solver(_spec(p), precision=precision, interface_solver=1)
    sol.build_transfer()
    u = torch.empty((n - 1, n - 1), dtype=torch.float64, device="cuda")
    st, info = sol.solve(dev(p["f"]), dev(p["g"]), u)
    assert info["gmres_iters"] == 0 and info["t_direct"] > 0.0
    uh = u.cpu().numpy().ravel()
    assert _relerr(uh, uref) <= (1e-10 if precision == "fp64" else 1e-8), info
    rng = np.random.default_rng(8)
    obs = rng.standard_normal(uh.size)
    df = torch.empty_like(u)
    D.ddst_solve_adjoint(sol.ctx, dev((uh - obs).reshape(n - 1, n - 1)), df, None, None)
    # a second solve reuses the factored system
    st, info2 = sol.solve(dev(p["f"]), dev(p["g"]), u)
    sol.close()
    assert _relerr(u.cpu().numpy().ravel(), uref) <= (1e-10 if precision == "fp64" else 1e-8)
    lam = O.adjoint_solve(A, uh - obs)
    assert _relerr(df.cpu().numpy().ravel(), lam) <= (1e-10 if precision == "fp64" else 1e-8)


def test_direct_solver_after_compression_and_in_a_batch():
    """Two problems of different sizes in one context, HODLR-compressed operators: the direct
    solver eliminates the dense S (kept after compression); both solutions against O2."""
    from paper_2510_25991_gb300 import ddst as D
    probs = [I.make_problem("convdiff2d", n=128, w=16), I.make_problem("poisson2d", n=96, w=32)]
    sol = D.Solver([_spec(p) for p in probs], precision="mixed", interface_solver=1, leaf_size=32)
    sol.build_transfer()
    sol.compress(1e-6)
    us = [torch.empty((p["n"] - 1,) * 2, dtype=torch.float64, device="cuda") for p in probs]
    D.ddst_solve_batch(sol.ctx, [dev(p["f"]) for p in probs], [dev(p["g"]) for p in probs], us)
    sol.close()
    for p, u in zip(probs, us):
        A, b = O.assemble(p)
        assert _relerr(u.cpu().numpy().ravel(), O.global_solve(A, b)) <= 1e-8, p["name"]


def test_direct_solver_needs_explicit_operators():
    from paper_2510_25991_gb300 import ddst as D
    p = I.make_problem("convdiff2d", n=64, w=8)
    sol = D.Solver(_spec(p), precision="mixed", explicit_S=0, interface_solver=1)
    sol.build_transfer()
    u = torch.empty((63, 63), dtype=torch.float64, device="cuda")
    with pytest.raises(D.DDSTError) as e:
        sol.solve(dev(p["f"]), dev(p["g"]), u)
    sol.close()
    assert e.value.name == "NOT_IMPLEMENTED"


def test_direct_fp64_solves_the_indefinite_case_where_gmres_stalls():
    """Helmholtz at 512^2, kappa = 100, 63 double slabs of 2w = 16 cells: unrestarted GMRES on
    (I - K) does not converge there even in the FP64 oracle (relative residual 1e-2 after 1500
    iterations), while the system itself is well posed.  The FP64 block cyclic reduction solves
    it to the global solve's accuracy.  In mixed precision the FP32 reduction of this indefinite
    system is not an approximate inverse (the refinement's corrections grow), which the solve
    reports as NOT_CONVERGED."""
    from paper_2510_25991_gb300 import ddst as D
    p = I.make_problem("helmholtz2d", n=512, w=8, kappa=100.0)
    A, b = O.assemble(p)
    uref = O.global_solve(A, b)
    sol = D.Solver(_spec(p), precision="fp64", interface_solver=1)
    sol.build_transfer()
    u = torch.empty((511, 511), dtype=torch.float64, device="cuda")
    st, info = sol.solve(dev(p["f"]), dev(p["g"]), u)
    sol.close()
    assert _relerr(u.cpu().numpy().ravel(), uref) <= 1e-10, info
    sol = D.Solver(_spec(p), precision="mixed", interface_solver=1, refine_max=6)
    sol.build_transfer()
    st, info = sol.solve(dev(p["f"]), dev(p["g"]), u, raise_on_error=False)
    sol.close()
    assert D.L.STATUS_NAMES[st] == "NOT_CONVERGED" and info["refine_rho"] > 1.0, info
