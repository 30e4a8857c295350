"""The allocation-free residual entry point, for callers that cannot allocate device memory.

ddst_residual_noalloc keeps its scratch (partial sums) in a file-scope device array instead of
calling cudaMalloc.  This test calls it through the C ABI twice in a row, on two different
problems, and checks each result against the existing entry point: the relative residual
ddst_solve reports for the same solution, and the residual vector of the FP64 oracle.
It runs alone in a fresh process as well as after the other GPU tests.
"""
import numpy as np
import pytest

import ddst_inputs as I
from oracle import ddst_oracle as O

torch = pytest.importorskip("torch")


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


@pytest.mark.gpu
def test_residual_noalloc_matches_solver_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25991_gb300 import build as B
    from paper_2510_25991_gb300 import ddst as D
    B.build()
    probs = [I.make_problem("convdiff2d", n=128, w=16), I.make_problem("poisson2d", n=64, w=8)]
    for prob in probs:  # two calls in a row share the same scratch array
        n = prob["n"]
        b3 = tuple(prob["b"]) + (0.0,) * (3 - len(prob["b"]))
        a, f, g = _dev(prob["a"]), _dev(prob["f"]), _dev(prob["g"])
        sol = D.Solver(dict(dim=2, n=n, w=prob["w"], a=a, b=b3), precision="mixed")
        sol.build_transfer()
        u = torch.empty((n - 1, n - 1), dtype=torch.float64, device="cuda")
        st, info = sol.solve(f, g, u)
        sol.close()
        r = torch.full_like(u, float("nan"))
        norms = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        D.ddst_residual_noalloc(2, n, a, f, g, u, r, norms, b=b3)
        torch.cuda.synchronize()
        rel = float(norms[0] / norms[1])
        # same quantity as the solver's own FP64 residual check, to summation order
        assert abs(rel - info["rel_residual"]) <= 1e-6 * info["rel_residual"] + 1e-18
        A, bvec = O.assemble(prob)
        uh = u.cpu().numpy().ravel()
        rref = bvec - A @ uh
        assert np.abs(r.cpu().numpy().ravel() - rref).max() <= 1e-12 * np.abs(bvec).max()
        assert abs(float(norms[1]) - np.linalg.norm(bvec)) <= 1e-12 * np.linalg.norm(bvec)


@pytest.mark.gpu
def test_residual_noalloc_3d_and_reaction_term_match_oracle():
    """The 3D index decode and strides, and the nodal reaction term c, against the oracle's
    residual of the same (random) u: a 16^3 variable-coefficient problem, then a 2D problem with
    c != 0, called in a row on the shared scratch array."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25991_gb300 import build as B
    from paper_2510_25991_gb300 import ddst as D
    B.build()
    p3 = I.make_problem("vardiff3d", n=16, w=4)
    p2 = I.make_problem("convdiff2d", n=64, w=16)
    rng = np.random.default_rng(7)
    p2["c"] = 50.0 + 100.0 * rng.random((65, 65))
    for prob in (p3, p2):
        dim, n = prob["dim"], prob["n"]
        b3 = tuple(prob["b"]) + (0.0,) * (3 - len(prob["b"]))
        u = rng.standard_normal((n - 1,) * dim)
        r = torch.full(u.shape, float("nan"), dtype=torch.float64, device="cuda")
        norms = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        c = _dev(prob["c"]) if prob["c"] is not None else None
        D.ddst_residual_noalloc(dim, n, _dev(prob["a"]), _dev(prob["f"]), _dev(prob["g"]), _dev(u),
                                r, norms, b=b3, c=c)
        torch.cuda.synchronize()
        A, bvec = O.assemble(prob)
        rref = bvec - A @ u.ravel()
        scale = np.abs(bvec).max() + np.abs(A).max() * np.abs(u).max()
        assert np.abs(r.cpu().numpy().ravel() - rref).max() <= 1e-12 * scale
        assert abs(float(norms[0]) - np.linalg.norm(rref)) <= 1e-12 * np.linalg.norm(rref)
        assert abs(float(norms[1]) - np.linalg.norm(bvec)) <= 1e-12 * np.linalg.norm(bvec)


def test_residual_noalloc_binding_checks_sizes_before_any_launch():
    """The library gets plain pointers and cannot check array sizes; the binding must refuse a
    wrong-size array (ValueError) before the library is even called.  Host arrays suffice: the
    size check comes first, so this runs without a GPU."""
    from paper_2510_25991_gb300 import ddst as D
    n = 16
    a, g = np.ones((n + 1, n + 1)), np.zeros((n + 1, n + 1))
    f, r = np.zeros((n - 1, n - 1)), np.zeros((n - 1, n - 1))
    with pytest.raises(ValueError, match="u has"):
        D.ddst_residual_noalloc(2, n, a, f, g, np.zeros((n - 2, n - 1)), r, np.zeros(2))
    with pytest.raises(ValueError, match="c has"):
        D.ddst_residual_noalloc(2, n, a, f, g, np.zeros((n - 1, n - 1)), r, np.zeros(2),
                                c=np.zeros((n - 1, n - 1)))
    with pytest.raises(ValueError, match="norms"):
        D.ddst_residual_noalloc(2, n, a, f, g, np.zeros((n - 1, n - 1)), r, np.zeros(1))


@pytest.mark.gpu
def test_residual_noalloc_rejects_host_arrays_and_oversize_grids():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25991_gb300 import ddst as D
    n = 32
    a = _dev(np.ones((n + 1, n + 1)))
    f = _dev(np.zeros((n - 1, n - 1)))
    g = _dev(np.zeros((n + 1, n + 1)))
    u = _dev(np.zeros((n - 1, n - 1)))
    r = torch.empty_like(u)
    norms = torch.empty(2, dtype=torch.float64, device="cuda")
    with pytest.raises(D.DDSTError) as e:
        D.ddst_residual_noalloc(2, n, a, f, g, u.cpu().numpy(), r, norms)
    assert e.value.name == "INVALID_ARG" and "device arrays" in str(e.value)
    big = 4098  # 4097^2 interior unknowns: above the 16,777,216 limit
    ab = torch.ones((big + 1, big + 1), dtype=torch.float64, device="cuda")
    vb = torch.zeros((big - 1, big - 1), dtype=torch.float64, device="cuda")
    with pytest.raises(D.DDSTError) as e:
        D.ddst_residual_noalloc(2, big, ab, vb, ab, vb, vb, norms)
    assert e.value.name == "INVALID_ARG" and "at most" in str(e.value)
