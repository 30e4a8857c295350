"""CUDA path vs the FP64 CPU oracle (element by element on the same seeded inputs).

Tolerances (derived in the design notes):
* FP64 path, uncompressed: 1e-10 relative (transfer blocks and solutions).
* Mixed path (FP32 local operators) after FP64 refinement: 1e-8 relative solution error.
* FP32 transfer blocks: 1e-3 relative to max |S|: a backward-stable FP32 local solve has
  forward error up to kappa(A_j) u_32, and kappa(A_j) ~ 4e5 for the variable-coefficient
  double slabs tested (u_32 = 6e-8); measured 2.4e-4 on the 256^2 case.
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


def make_solver(prob, precision, compress_tol=None, **opts):
    from paper_2510_25991_gb300 import ddst as D
    spec = dict(dim=prob["dim"], n=prob["n"], w=prob["w"], a=dev(prob["a"]),
                b=tuple(prob["b"]) + (0.0,) * (3 - len(prob["b"])),
                c=dev(prob["c"]) if prob.get("c") is not None else None)
    sol = D.Solver(spec, precision=precision, **opts)
    sol.build_transfer()
    if compress_tol:
        sol.compress(compress_tol)
    return sol


def solve(sol, prob, **kw):
    n, dim = prob["n"], prob["dim"]
    u = torch.empty((n - 1,) * dim, dtype=torch.float64, device="cuda")
    st, info = sol.solve(dev(prob["f"]), dev(prob["g"]), u, **kw)
    return u.cpu().numpy().ravel(), info, st


def relerr(x, ref):
    return np.linalg.norm(x - ref) / np.linalg.norm(ref)


CASES = [("poisson2d", 32, 8, 2), ("convdiff2d", 64, 16, 2), ("convdiff2d", 256, 32, 2),
         ("vardiff3d", 8, 2, 3), ("vardiff3d", 16, 2, 3)]


def _prob(name, n, w, dim):
    p = I.make_problem(name, n=n, w=w)
    assert p["dim"] == dim
    return p


@pytest.mark.parametrize("name,n,w,dim", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_transfer_blocks_match_oracle(name, n, w, dim, precision):
    from paper_2510_25991_gb300 import ddst as D
    prob = _prob(name, n, w, dim)
    A, b = O.assemble(prob)
    geo = O.slab_geometry(dim, n, w)
    facs = O.factor_local(A, geo)
    Sp, Sn = O.transfer_blocks(A, geo, facs)
    sol = make_solver(prob, precision)
    tol = 1e-10 if precision == "fp64" else 1e-3
    ng = geo.ngamma
    out = np.empty((ng, ng))
    worst = 0.0
    for j in range(geo.nds):
        for side, ref in ((-1, Sp[j]), (1, Sn[j])):
            if ref is None:
                continue
            D.ddst_get_transfer(sol.ctx, 0, j + 1, side, out)
            worst = max(worst, np.abs(out - ref).max() / np.abs(ref).max())
    sol.close()
    assert worst <= tol, worst


@pytest.mark.parametrize("name,n,w,dim", CASES + [("poisson2d", 128, 16, 2)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solution_matches_global_solve(name, n, w, dim, precision):
    prob = _prob(name, n, w, dim)
    A, b = O.assemble(prob)
    uref = O.global_solve(A, b)
    opts = dict(gmres_tol=1e-12) if precision == "fp64" else {}
    sol = make_solver(prob, precision, **opts)
    u, info, st = solve(sol, prob)
    sol.close()
    err = relerr(u, uref)
    assert err <= (1e-10 if precision == "fp64" else 1e-8), (err, info)
    assert info["rel_residual"] <= 1e-9


def test_manufactured_harmonic_on_gpu():
    """P1 through the CUDA path: f = 0, g harmonic quadratic -> u = g at every node."""
    prob = I.make_problem("poisson2d", n=128, w=16)
    prob["f"] = np.zeros_like(prob["f"])
    sol = make_solver(prob, "fp64", gmres_tol=1e-13)
    u, info, st = solve(sol, prob)
    sol.close()
    assert np.abs(u - prob["g"][1:128, 1:128].ravel()).max() <= 1e-12


def test_gmres_iterations_match_oracle_and_paper_3d():
    """3D Poisson 16^3, 8 slabs: GMRES iterations to 1e-8 as printed (19) within +-10%."""
    prob = I.make_problem("vardiff3d", n=16, w=2, const_a=True)
    sol = make_solver(prob, "fp64", gmres_tol=1e-8, refine_max=0)
    u, info, st = solve(sol, prob)
    sol.close()
    assert abs(info["gmres_iters_first"] - 19) <= 3, info


def test_gmres_iterations_config1_vs_oracle():
    prob = I.make_problem("poisson2d")
    _, _, oinfo = O.dd_solve(prob, use_gmres=True, tol=1e-8)
    sol = make_solver(prob, "fp64", gmres_tol=1e-8, refine_max=0)
    u, info, st = solve(sol, prob)
    sol.close()
    assert abs(info["gmres_iters_first"] - oinfo["iters"]) <= 1, (info, oinfo["iters"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_interface_apply_transpose_consistency(precision):
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("convdiff2d", n=64, w=8)
    sol = make_solver(prob, precision)
    nds, ng, _ = D.ddst_query(sol.ctx)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(nds * ng)
    y = rng.standard_normal(nds * ng)
    ax = np.empty_like(x)
    aty = np.empty_like(y)
    D.ddst_apply_interface(sol.ctx, 0, x, ax, False)
    D.ddst_apply_interface(sol.ctx, 0, y, aty, True)
    sol.close()
    lhs, rhs = ax @ y, x @ aty
    assert abs(lhs - rhs) <= (1e-12 if precision == "fp64" else 1e-6) * abs(lhs)
    # and (I - K) x against the oracle's dense interface matrix
    A, b = O.assemble(prob)
    geo = O.slab_geometry(2, 64, 8)
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo))
    ref = O.apply_interface(Sp, Sn, x)
    assert relerr(ax, ref) <= (1e-12 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_gradients_match_oracle(precision):
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("convdiff2d", n=64, w=16)
    n = 64
    rng = np.random.default_rng(11)
    u_obs = rng.standard_normal((n - 1) ** 2)
    L, dLdf, dLdg, dLda, uref, lam = O.loss_and_gradients(prob, u_obs)
    opts = dict(gmres_tol=1e-12) if precision == "fp64" else {}
    sol = make_solver(prob, precision, **opts)
    u, info, st = solve(sol, prob)
    dLdu = dev((u - u_obs).reshape(n - 1, n - 1))
    df = torch.empty((n - 1, n - 1), dtype=torch.float64, device="cuda")
    dg = torch.empty((n + 1, n + 1), dtype=torch.float64, device="cuda")
    da = torch.empty((n + 1, n + 1), dtype=torch.float64, device="cuda")
    D.ddst_solve_adjoint(sol.ctx, dLdu, df, dg, da)
    sol.close()
    tol = 1e-10 if precision == "fp64" else 1e-8
    assert relerr(df.cpu().numpy(), dLdf) <= tol
    mask = np.ones((n + 1, n + 1), bool)
    mask[1:n, 1:n] = False
    assert relerr(dg.cpu().numpy()[mask], dLdg[mask]) <= tol
    assert relerr(da.cpu().numpy(), dLda) <= 10 * tol


def test_batch_of_uneven_problems():
    from paper_2510_25991_gb300 import ddst as D
    probs = [I.make_problem("convdiff2d", n=64, w=16), I.make_problem("poisson2d", n=128, w=16),
             I.make_problem("convdiff2d", n=96, w=32)]
    specs = [dict(dim=2, n=p["n"], w=p["w"], a=dev(p["a"]), b=tuple(p["b"]) + (0.0,)) for p in probs]
    sol = D.Solver(specs, precision="mixed")
    sol.build_transfer()
    us = [torch.empty((p["n"] - 1, p["n"] - 1), dtype=torch.float64, device="cuda") for p in probs]
    D.ddst_solve_batch(sol.ctx, [dev(p["f"]) for p in probs], [dev(p["g"]) for p in probs], us)
    sol.close()
    for p, u in zip(probs, us):
        A, b = O.assemble(p)
        assert relerr(u.cpu().numpy().ravel(), O.global_solve(A, b)) <= 1e-8


def test_host_buffers_are_staged():
    """The C ABI accepts host arrays: same answer as with device arrays."""
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("convdiff2d", n=64, w=16)
    sol = D.Solver(dict(dim=2, n=64, w=16, a=np.ascontiguousarray(prob["a"]), b=(20.0, 10.0, 0.0)),
                   precision="mixed")
    sol.build_transfer()
    u = np.empty((63, 63))
    sol.solve(np.ascontiguousarray(prob["f"]), np.ascontiguousarray(prob["g"]), u)
    sol.close()
    A, b = O.assemble(prob)
    assert relerr(u.ravel(), O.global_solve(A, b)) <= 1e-8


def test_errors_are_reported_not_raised_on_device():
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("poisson2d", n=32, w=8)
    # state error: solve before build_transfer
    sol = D.Solver(dict(dim=2, n=32, w=8, a=dev(prob["a"])), precision="mixed")
    u = torch.empty((31, 31), dtype=torch.float64, device="cuda")
    with pytest.raises(D.DDSTError) as e:
        sol.solve(dev(prob["f"]), dev(prob["g"]), u)
    assert e.value.name == "STATE"
    # not converged: 2 GMRES iterations, no refinement
    sol.close()
    sol = make_solver(prob, "mixed", gmres_max_iter=2, refine_max=0, check_every=1)
    st, info = sol.solve(dev(prob["f"]), dev(prob["g"]), u, raise_on_error=False)
    assert st == 5 and info["gmres_iters"] == 2
    sol.close()
    # invalid argument: slab width not dividing n
    with pytest.raises(D.DDSTError) as e:
        D.Solver(dict(dim=2, n=32, w=7, a=dev(prob["a"])))
    assert e.value.name == "INVALID_ARG"


def test_singular_local_operator_is_detected():
    """A reaction coefficient that cancels the stencil diagonal at one node makes the first
    pivot of slab 1 exactly zero: setup must report SINGULAR with slab and block."""
    from paper_2510_25991_gb300 import ddst as D
    n, w = 32, 8
    prob = I.make_problem("poisson2d", n=n, w=w)
    c = np.zeros((n + 1, n + 1))
    c[1, 1] = -4.0 * n * n          # diag = 4 a / h^2 + c = 0 at node (1, 1)
    for precision in ("fp64", "mixed"):
        with pytest.raises(D.DDSTError) as e:
            D.Solver(dict(dim=2, n=n, w=w, a=dev(prob["a"]), c=dev(c)), precision=precision)
        assert e.value.name == "SINGULAR"
        assert "slab 0" in str(e.value) and "block 1" in str(e.value)


@pytest.mark.parametrize("precision,warmup", [("mixed", 128), ("fp64", 240)])
def test_chunked_pivot_sweeps_match_oracle(precision, warmup):
    """Warm-started chunks (forced: 4 per slab sweep) reproduce the exact transfer operators
    and solution; the convergence check passes, so the chunks are kept."""
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("convdiff2d", n=512, w=16)
    A, b = O.assemble(prob)
    geo = O.slab_geometry(2, 512, 16)
    js = (1, geo.nds // 2)
    facs = O.factor_local(A, geo)
    Sp, Sn = O.transfer_blocks(A, geo, facs, slabs=js)
    opts = dict(factor_chunks=4, factor_warmup=warmup)
    if precision == "fp64":
        opts["gmres_tol"] = 1e-12
    sol = make_solver(prob, precision, **opts)
    out = np.empty((geo.ngamma, geo.ngamma))
    tol = 1e-10 if precision == "fp64" else 1e-3
    for i, j in enumerate(js):
        for side, ref in ((-1, Sp[i]), (1, Sn[i])):
            D.ddst_get_transfer(sol.ctx, 0, j + 1, side, out)
            assert np.abs(out - ref).max() <= tol * np.abs(ref).max()
    u, info, st = solve(sol, prob)
    sol.close()
    assert info["factor_chunks"] == 4, info
    assert relerr(u, O.global_solve(A, b)) <= (1e-10 if precision == "fp64" else 1e-8)


def test_chunked_pivot_sweeps_fall_back_when_warmup_is_too_short():
    """A 2-row warm-up cannot converge: the check fails and the exact sweeps are used."""
    prob = I.make_problem("convdiff2d", n=512, w=16)
    A, b = O.assemble(prob)
    sol = make_solver(prob, "mixed", factor_chunks=4, factor_warmup=2)
    u, info, st = solve(sol, prob)
    sol.close()
    assert info["factor_chunks"] == 1 and info["factor_check"] > 1e-5, info
    assert relerr(u, O.global_solve(A, b)) <= 1e-8


# (64, 16): one CTA holding a single partly filled tile; (256, 32): two tiles, the second ragged;
# (514, 2): M = 32, n_Gamma = 513 = 2 * 256 + 1, so the last CTA has one source and a one-block
# downward sweep.
@pytest.mark.parametrize("n,w", [(64, 16), (256, 32), (514, 2)])
def test_tensor_core_transfer_build_matches_fma_kernel(n, w):
    """tcgen05 (3xTF32) and FP32-FMA transfer builds agree to FP32 rounding, and both match the
    oracle within the FP32 tolerance."""
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("convdiff2d", n=n, w=w)
    geo = O.slab_geometry(2, n, w)
    A, b = O.assemble(prob)
    js = sorted({1, geo.nds // 2, geo.nds - 2})
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo), slabs=js)
    mats = {}
    for tc in (0, 1):
        sol = make_solver(prob, "mixed", tensor_cores=tc)
        for j in js:
            for side in (-1, 1):
                out = np.empty((geo.ngamma, geo.ngamma))
                D.ddst_get_transfer(sol.ctx, 0, j + 1, side, out)
                mats[(tc, j, side)] = out
        sol.close()
    for jj, j in enumerate(js):
        for side, ref in ((-1, Sp[jj]), (1, Sn[jj])):
            scale = np.abs(ref).max()
            assert np.abs(mats[(1, j, side)] - mats[(0, j, side)]).max() <= 2e-5 * scale
            assert np.abs(mats[(1, j, side)] - ref).max() <= 1e-3 * scale


def test_autograd_function_gradients_match_oracle():
    """DDSTSolve (torch.autograd.Function): backward is the hand-written adjoint."""
    from paper_2510_25991_gb300 import ddst as D
    n, w = 64, 16
    prob = I.make_problem("convdiff2d", n=n, w=w)
    rng = np.random.default_rng(3)
    u_obs = rng.standard_normal((n - 1) ** 2)
    L, dLdf, dLdg, dLda, uref, lam = O.loss_and_gradients(prob, u_obs)
    a = dev(prob["a"]).requires_grad_(True)
    f = dev(prob["f"]).requires_grad_(True)
    g = dev(prob["g"]).requires_grad_(True)
    spec = dict(dim=2, n=n, w=w, b=(20.0, 10.0, 0.0), precision="fp64",
                options=dict(gmres_tol=1e-12))
    u = D.DDSTSolve.apply(a, f, g, spec)
    loss = 0.5 * ((u.reshape(-1) - dev(u_obs)) ** 2).sum()
    loss.backward()
    assert abs(loss.item() - L) <= 1e-10 * L
    assert relerr(f.grad.cpu().numpy(), dLdf) <= 1e-10
    assert relerr(a.grad.cpu().numpy(), dLda) <= 1e-9
    mask = np.ones((n + 1, n + 1), bool)
    mask[1:n, 1:n] = False
    assert relerr(g.grad.cpu().numpy()[mask], dLdg[mask]) <= 1e-10


def test_batched_adjoint_matches_oracle():
    from paper_2510_25991_gb300 import ddst as D
    probs = [I.make_problem("convdiff2d", n=64, w=16), I.make_problem("poisson2d", n=96, w=32)]
    specs = [dict(dim=2, n=p["n"], w=p["w"], a=dev(p["a"]), b=tuple(p["b"]) + (0.0,)) for p in probs]
    sol = D.Solver(specs, precision="mixed")
    sol.build_transfer()
    us = [torch.empty((p["n"] - 1, p["n"] - 1), dtype=torch.float64, device="cuda") for p in probs]
    D.ddst_solve_batch(sol.ctx, [dev(p["f"]) for p in probs], [dev(p["g"]) for p in probs], us)
    rng = np.random.default_rng(9)
    obs = [rng.standard_normal((p["n"] - 1) ** 2) for p in probs]
    dLdu = [dev((u.cpu().numpy().ravel() - o).reshape(u.shape)) for u, o in zip(us, obs)]
    dfs = [torch.empty_like(u) for u in us]
    dgs = [torch.empty((p["n"] + 1, p["n"] + 1), dtype=torch.float64, device="cuda") for p in probs]
    das = [torch.empty_like(x) for x in dgs]
    D.ddst_solve_adjoint_batch(sol.ctx, dLdu, dfs, dgs, das)
    sol.close()
    for p, o, df, da in zip(probs, obs, dfs, das):
        L, dLdf, dLdg, dLda, uref, lam = O.loss_and_gradients(p, o)
        assert relerr(df.cpu().numpy(), dLdf) <= 1e-8
        assert relerr(da.cpu().numpy(), dLda) <= 1e-7


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_helmholtz_transfer_blocks_reduced_size(precision):
    """Helmholtz (Gaussian bump in the wavenumber) at 512^2, kappa = 100, slabs of 2w = 16 cells:
    the local operators are positive definite by ~1% (lowest slab eigenvalue ~ (32 pi)^2 >
    kappa^2), the same margin as the 4096^2, kappa = 200, w = 32 workload.  Transfer operators of
    the first, middle and last interior slabs against the oracle."""
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("helmholtz2d", n=512, w=8, kappa=100.0)
    A, b = O.assemble(prob)
    geo = O.slab_geometry(2, 512, 8)
    js = [1, geo.nds // 2, geo.nds - 2]
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo), slabs=js)
    sol = make_solver(prob, precision)
    tol = 1e-10 if precision == "fp64" else 1e-3
    out = np.empty((geo.ngamma, geo.ngamma))
    worst = 0.0
    for jj, j in enumerate(js):
        for side, ref in ((-1, Sp[jj]), (1, Sn[jj])):
            D.ddst_get_transfer(sol.ctx, 0, j + 1, side, out)
            worst = max(worst, np.abs(out - ref).max() / np.abs(ref).max())
    sol.close()
    assert worst <= tol, worst


def test_helmholtz_indefinite_local_operators():
    """Helmholtz at 512^2, kappa = 100, with 15 double slabs of 2w = 64 cells, where the interface
    GMRES converges (~350 iterations): each slab holds propagating modes, so the local operators
    are indefinite and the unpivoted block elimination meets leading minors near zero (down to
    1e-3 |diag| in exact arithmetic).  FP64 solves it; FP32 either solves it or reports the
    pivot (SINGULAR with its slab and block); DDST_AUTO falls back to FP64 and solves it."""
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("helmholtz2d", n=512, w=32, kappa=100.0)
    A, b = O.assemble(prob)
    uref = O.global_solve(A, b)
    sol = make_solver(prob, "fp64", gmres_tol=1e-12)
    u, info, st = solve(sol, prob)
    sol.close()
    assert relerr(u, uref) <= 1e-10, info
    try:
        sol = make_solver(prob, "mixed")
    except D.DDSTError as e:
        assert e.name == "SINGULAR" and "slab" in str(e) and "block" in str(e)
    else:
        u, info, st = solve(sol, prob)
        sol.close()
        assert relerr(u, uref) <= 1e-8, info
    sol = make_solver(prob, "auto")
    assert sol.precision in ("fp64", "mixed")
    u, info, st = solve(sol, prob)
    sol.close()
    assert relerr(u, uref) <= 1e-8, info
