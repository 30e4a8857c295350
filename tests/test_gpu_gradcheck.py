"""Adjoint gradients against central finite differences of the GPU solver's own loss.

L(a, f, g) = 1/2 ||u(a, f, g) - u_obs||^2 with u from the C ABI solve.  L is quadratic in f and
in g, so the central difference with a unit step is exact up to rounding there; in a it has an
O(eps^2) truncation error (eps = 1e-4 relative).  The directional derivative <dL/dx, d> from
ddst_solve_adjoint must match to 1e-5 relative, in FP64 and in mixed precision."""
import numpy as np
import pytest

import ddst_inputs as I

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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_gradients_match_central_differences(precision):
    from paper_2510_25991_gb300 import ddst as D
    n, w = 48, 12
    p = I.make_problem("convdiff2d", n=n, w=w)
    b = tuple(p["b"]) + (0.0,)
    opts = dict(gmres_tol=1e-12, refine_tol=1e-13) if precision == "fp64" else dict(refine_tol=1e-12)
    rng = np.random.default_rng(12)
    u_obs = rng.standard_normal((n - 1) ** 2)

    def solve(a, f, g):
        sol = D.Solver(dict(dim=2, n=n, w=w, a=dev(a), b=b), precision=precision, **opts)
        sol.build_transfer()
        u = torch.empty((n - 1, n - 1), dtype=torch.float64, device="cuda")
        sol.solve(dev(f), dev(g), u)
        return sol, u

    def loss(a, f, g):
        sol, u = solve(a, f, g)
        sol.close()
        return 0.5 * float(np.sum((u.cpu().numpy().ravel() - u_obs) ** 2))

    a, f, g = p["a"], p["f"], p["g"]
    sol, u = solve(a, f, g)
    dLdu = dev((u.cpu().numpy().ravel() - u_obs).reshape(n - 1, n - 1))
    df = torch.empty_like(u)
    dg = torch.empty((n + 1, n + 1), dtype=torch.float64, device="cuda")
    da = torch.empty_like(dg)
    D.ddst_solve_adjoint(sol.ctx, dLdu, df, dg, da)
    sol.close()
    df, dg, da = df.cpu().numpy(), dg.cpu().numpy(), da.cpu().numpy()
    # directions: f anywhere, g on the boundary nodes only, a smooth and relative to a
    d_f = rng.standard_normal(f.shape)
    d_g = rng.standard_normal(g.shape)
    d_g[1:n, 1:n] = 0.0
    x = np.linspace(0.0, 1.0, n + 1)
    d_a = a * np.outer(np.sin(2 * np.pi * x), np.cos(np.pi * x))
    for name, grad, d, eps, args in (
            ("f", df, d_f, 1.0, lambda s: (a, f + s * d_f, g)),
            ("g", dg, d_g, 1.0, lambda s: (a, f, g + s * d_g)),
            ("a", da, d_a, 1e-4, lambda s: (a + s * d_a, f, g))):
        fd = (loss(*args(eps)) - loss(*args(-eps))) / (2.0 * eps)
        ad = float(np.sum(grad * d))
        assert abs(fd - ad) <= 1e-5 * abs(ad), (name, fd, ad)
