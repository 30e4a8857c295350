"""Options that change how the method is carried out, checked against the oracle.

* recompute_factors: the local factors are released once the transfer operators exist and
  recomputed for every solve, adjoint or matrix-free application; results must not change.
"""
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


def relerr(x, ref):
    return np.linalg.norm(x - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("name,n,w,compress", [("convdiff2d", 256, 32, 1e-8), ("vardiff3d", 24, 6, None)])
def test_recompute_factors_gives_the_same_solutions_and_gradients(name, n, w, compress):
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem(name, n=n, w=w)
    dim = prob["dim"]
    sol = D.Solver(dict(dim=dim, n=n, w=w, a=dev(prob["a"]), b=tuple(prob["b"]) + (0.0,) * (3 - dim)),
                   precision="mixed", recompute_factors=1)
    sol.build_transfer()
    if compress:
        sol.compress(compress)
    A, b = O.assemble(prob)
    uref = O.global_solve(A, b)
    u = torch.empty((n - 1,) * dim, dtype=torch.float64, device="cuda")
    for _ in range(2):  # factors recomputed for each call
        st, info = sol.solve(dev(prob["f"]), dev(prob["g"]), u)
        assert relerr(u.cpu().numpy().ravel(), uref) <= 1e-8, info
    uh = u.cpu().numpy().ravel()
    obs = np.random.default_rng(1).standard_normal(uh.size)
    df = torch.empty_like(u)
    D.ddst_solve_adjoint(sol.ctx, dev((uh - obs).reshape(u.shape)), df, None, None)
    assert relerr(df.cpu().numpy().ravel(), O.adjoint_solve(A, uh - obs)) <= 1e-8
    nds, ng, _ = D.ddst_query(sol.ctx)
    x = np.random.default_rng(2).standard_normal(nds * ng)
    y = torch.empty(x.size, dtype=torch.float64, device="cuda")
    D.ddst_apply_interface(sol.ctx, 0, dev(x), y)  # matrix-free: refactors first
    geo = O.slab_geometry(dim, n, w)
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo))
    ref = O.apply_interface(Sp, Sn, x)
    tol = 2e-5 if compress is None else 1e-3
    assert np.abs(y.cpu().numpy() - ref).max() <= tol * np.abs(ref).max()
    sol.close()


@pytest.mark.parametrize("name,n,w", [("convdiff2d", 256, 32), ("vardiff3d", 32, 8)])
def test_tf32_mode_reaches_the_target_after_refinement(name, n, w):
    """DDST_MIXED_TF32: one TF32 product per tensor-core step (2D: the transfer build; 3D: the
    large-block factorization) instead of 3xTF32.  The operators are TF32-accurate, and the FP64
    refinement still reaches 1e-8 against O2, with at least as many refinement steps."""
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem(name, n=n, w=w)
    dim = prob["dim"]
    A, b = O.assemble(prob)
    uref = O.global_solve(A, b)
    steps = {}
    for prec in ("mixed", "mixed_tf32"):
        sol = D.Solver(dict(dim=dim, n=n, w=w, a=dev(prob["a"]), b=tuple(prob["b"]) + (0.0,) * (3 - dim)),
                       precision=prec)
        assert sol.precision == prec
        sol.build_transfer()
        u = torch.empty((n - 1,) * dim, dtype=torch.float64, device="cuda")
        st, info = sol.solve(dev(prob["f"]), dev(prob["g"]), u)
        sol.close()
        assert relerr(u.cpu().numpy().ravel(), uref) <= 1e-8, (prec, info)
        steps[prec] = info["refine_iters"]
    assert steps["mixed_tf32"] >= steps["mixed"], steps
