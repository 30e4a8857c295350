"""Large dense blocks (m > 128, or > 64 in FP64) and the matrix-free interface operator, against
the FP64 CPU oracle, element by element on the same seeded inputs.

The large-block kernels factor every double slab by a one-sided block LU whose pivot inverses
are formed by 128-wide Gauss-Jordan panels (tensor cores in FP32, FMA in FP64); the interface
operator is applied through local solves (no explicit S).  Sizes span several 128-tiles and a
ragged last tile (m = 217, 465, 741 padded to 256, 512, 768).

Tolerances: FP64 solution 1e-10, mixed solution after FP64 refinement 1e-8 (as for the
single-CTA path).  The interface operator in FP32 is compared to 2e-5 relative to the largest
entry of the result: its error is that of one FP32 local solve per slab (kappa(A_j) u_32 with
kappa(A_j) ~ 1e2 for these slabs); in FP64 to 1e-11.
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


def make_solver(prob, precision, **opts):
    from paper_2510_25991_gb300 import ddst as D
    spec = dict(dim=prob["dim"], n=prob["n"], w=prob["w"], a=dev(prob["a"]),
                b=tuple(prob["b"]) + (0.0,) * (3 - len(prob["b"])),
                c=dev(prob["c"]) if prob.get("c") is not None else None)
    sol = D.Solver(spec, precision=precision, **opts)
    sol.build_transfer()
    return sol


def solve(sol, prob):
    n, dim = prob["n"], prob["dim"]
    u = torch.empty((n - 1,) * dim, dtype=torch.float64, device="cuda")
    st, info = sol.solve(dev(prob["f"]), dev(prob["g"]), u)
    return u.cpu().numpy().ravel(), info


def relerr(x, ref):
    return np.linalg.norm(x - ref) / np.linalg.norm(ref)


# (workload, n, w): block sizes 217 (3D, pad 256), 465 (3D, pad 512), 255 (2D, pad 256)
CASES = [("vardiff3d", 32, 4), ("vardiff3d", 32, 8), ("convdiff2d", 512, 128)]


@pytest.mark.parametrize("name,n,w", CASES)
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_large_block_solution_matches_global_solve(name, n, w, precision):
    prob = I.make_problem(name, n=n, w=w)
    A, b = O.assemble(prob)
    uref = O.global_solve(A, b)
    opts = dict(gmres_tol=1e-12) if precision == "fp64" else {}
    sol = make_solver(prob, precision, **opts)
    u, info = solve(sol, prob)
    sol.close()
    assert info["bytes_transfer"] == 0  # matrix-free: no S formed
    assert relerr(u, uref) <= (1e-10 if precision == "fp64" else 1e-8)


@pytest.mark.parametrize("name,n,w,explicit", [("vardiff3d", 24, 6, -1), ("convdiff2d", 64, 8, 0)])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_matrix_free_interface_operator_matches_oracle_transfer_blocks(name, n, w, explicit,
                                                                       precision):
    """(I - K) x and (I - K)^T x through local solves against the oracle's dense transfer
    blocks (O3): a 3D case on the large-block kernels (m = 253, pad 256) and a 2D case with
    explicit_S = 0 on the single-CTA two-sided factors."""
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem(name, n=n, w=w)
    A, b = O.assemble(prob)
    geo = O.slab_geometry(prob["dim"], n, w)
    facs = O.factor_local(A, geo)
    Sp, Sn = O.transfer_blocks(A, geo, facs)
    Mi = O.interface_matrix(Sp, Sn, geo.ngamma)
    sol = make_solver(prob, precision, explicit_S=explicit)
    rng = np.random.default_rng(11)
    tol = 1e-11 if precision == "fp64" else 2e-5
    for tr in (False, True):
        x = rng.standard_normal(geo.nds * geo.ngamma)
        y = torch.empty(x.size, dtype=torch.float64, device="cuda")
        D.ddst_apply_interface(sol.ctx, 0, dev(x), y, transpose=tr)
        ref = (Mi.T if tr else Mi) @ x
        assert np.abs(y.cpu().numpy() - ref).max() <= tol * np.abs(ref).max(), tr
    with pytest.raises(D.DDSTError) as e:
        sol.compress(1e-8)
    assert e.value.name == "NOT_IMPLEMENTED"
    sol.close()


def test_tensor_core_factor_matches_fma_factor():
    """The tcgen05 Gauss-Jordan panels (3xTF32) against the FP32 FMA panels on the same
    problem: the two factorizations differ by FP32 rounding only, so the interface operator
    applied through them agrees to a few FP32 units relative to its largest entry."""
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("vardiff3d", n=40, w=10)  # m = 741, pad 768: 6 panels, ragged tile
    rng = np.random.default_rng(5)
    x = rng.standard_normal(3 * 39 * 39)
    ys = []
    for tc in (1, 0):
        sol = make_solver(prob, "mixed", tensor_cores=tc)
        y = torch.empty(x.size, dtype=torch.float64, device="cuda")
        D.ddst_apply_interface(sol.ctx, 0, dev(x), y)
        ys.append(y.cpu().numpy())
        sol.close()
    assert np.abs(ys[0] - ys[1]).max() <= 2e-5 * np.abs(ys[1]).max()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_large_block_adjoint_matches_oracle(precision):
    """dL/df = A^{-T} dL/du, dL/dg and dL/da through the transposed large-block solves and the
    transposed matrix-free operator, against O7."""
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("vardiff3d", n=24, w=6)
    n = prob["n"]
    A, b = O.assemble(prob)
    uref = O.global_solve(A, b)
    rng = np.random.default_rng(9)
    uobs = uref + 1e-2 * rng.standard_normal(uref.size)
    opts = dict(gmres_tol=1e-12) if precision == "fp64" else {}
    sol = make_solver(prob, precision, **opts)
    u, _ = solve(sol, prob)
    dLdu = dev((u - uobs).reshape((n - 1,) * 3))
    df = torch.empty((n - 1,) * 3, dtype=torch.float64, device="cuda")
    dg = torch.empty((n + 1,) * 3, dtype=torch.float64, device="cuda")
    da = torch.empty((n + 1,) * 3, dtype=torch.float64, device="cuda")
    D.ddst_solve_adjoint(sol.ctx, dLdu, df, dg, da)
    sol.close()
    lam = O.adjoint_solve(A, u - uobs)
    _, gg, ga = O.gradients(prob, u, lam)
    tol = 1e-10 if precision == "fp64" else 1e-8
    assert relerr(df.cpu().numpy().ravel(), lam) <= tol
    assert relerr(dg.cpu().numpy().ravel(), np.asarray(gg).ravel()) <= tol
    assert relerr(da.cpu().numpy().ravel(), np.asarray(ga).ravel()) <= tol


def test_large_block_batch_with_uneven_slab_counts():
    """One matrix-free context holding problems of different y-extents (nb = 23, 511, 255) in
    one large-block class (m = 253 and 255, pad 256) and a problem in a single-CTA class (pad 32):
    every slab advances through the batched factor and solve launches only while it has rows
    left, and the interface operator dispatches each class to its own local solves."""
    from paper_2510_25991_gb300 import ddst as D
    probs = [I.make_problem("vardiff3d", n=24, w=6), I.make_problem("convdiff2d", n=512, w=128),
             I.make_problem("convdiff2d", n=256, w=128), I.make_problem("convdiff2d", n=64, w=16)]
    spec = [dict(dim=p["dim"], n=p["n"], w=p["w"], a=dev(p["a"]),
                 b=tuple(p["b"]) + (0.0,) * (3 - len(p["b"]))) for p in probs]
    sol = D.Solver(spec, precision="mixed")
    sol.build_transfer()
    us = [torch.empty((p["n"] - 1,) * p["dim"], dtype=torch.float64, device="cuda") for p in probs]
    D.ddst_solve_batch(sol.ctx, [dev(p["f"]) for p in probs], [dev(p["g"]) for p in probs], us)
    sol.close()
    for p, u in zip(probs, us):
        A, b = O.assemble(p)
        assert relerr(u.cpu().numpy().ravel(), O.global_solve(A, b)) <= 1e-8, p["name"]


def test_mixed_context_hodlr_plus_matrix_free_with_adjoint():
    """One context with explicit classes (HODLR-compressed) and a large-block class (matrix-free):
    the compressed apply covers the explicit problems, the matrix-free apply then writes the
    large-block problem's interfaces.  Forward solutions and dL/df of every problem against
    O2 / O7."""
    from paper_2510_25991_gb300 import ddst as D
    probs = [I.make_problem("convdiff2d", n=128, w=16), I.make_problem("convdiff2d", n=256, w=128),
             I.make_problem("poisson2d", n=128, w=32)]
    spec = [dict(dim=2, n=p["n"], w=p["w"], a=dev(p["a"]), b=tuple(p["b"]) + (0.0,) * (3 - len(p["b"])))
            for p in probs]
    sol = D.Solver(spec, precision="mixed", leaf_size=32)
    sol.build_transfer()
    sol.compress(1e-8)
    assert D.ddst_query(sol.ctx, 0)[2] > 0
    us = [torch.empty((p["n"] - 1,) * 2, dtype=torch.float64, device="cuda") for p in probs]
    D.ddst_solve_batch(sol.ctx, [dev(p["f"]) for p in probs], [dev(p["g"]) for p in probs], us)
    rng = np.random.default_rng(4)
    obs = [rng.standard_normal((p["n"] - 1) ** 2) for p in probs]
    dLdu = [dev((u.cpu().numpy().ravel() - o).reshape(u.shape)) for u, o in zip(us, obs)]
    dfs = [torch.empty_like(u) for u in us]
    D.ddst_solve_adjoint_batch(sol.ctx, dLdu, dfs, [None] * 3, [None] * 3)
    with pytest.raises(D.DDSTError) as e:
        D.ddst_get_transfer(sol.ctx, 1, 1, 1, np.empty((255, 255)))
    assert e.value.name == "NOT_IMPLEMENTED"
    sol.close()
    for p, u, df, o in zip(probs, us, dfs, obs):
        A, b = O.assemble(p)
        uh = u.cpu().numpy().ravel()
        assert relerr(uh, O.global_solve(A, b)) <= 1e-8, p["name"]
        assert relerr(df.cpu().numpy().ravel(), O.adjoint_solve(A, uh - o)) <= 1e-8, p["name"]
