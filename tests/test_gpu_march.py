"""IMEX backward-Euler time marching (Sec. 6, Example 1) through ddst_march against the oracle's
march (O8), element by element on the same seeded inputs: the screened operator is set up and
its transfer operators built once, then reused by every step (GMRES or the direct interface
solver), and each step's refinement starts from the previous state.  Tolerances as for a solve:
1e-8 relative (mixed), 1e-10 (FP64), after the last step."""
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
    return dict(dim=p["dim"], n=p["n"], w=p["w"], a=dev(p["a"]), b=(0.0, 0.0, 0.0), c=dev(p["c"]))


def _relerr(x, ref):
    return np.linalg.norm(x - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("precision,isol", [("mixed", 0), ("mixed", 1), ("fp64", 0), ("fp64", 1)])
def test_march_2d_matches_oracle(precision, isol):
    from paper_2510_25991_gb300 import ddst as D
    p = I.march_problem(2, 128, 16)
    nsteps = 12
    ref = O.imex_march(p, p["u0"], p["vel"], p["dt"], nsteps)
    sol = D.Solver(_spec(p), precision=precision, interface_solver=isol)
    sol.build_transfer()
    u = torch.empty((127, 127), dtype=torch.float64, device="cuda")
    st, info = D.ddst_march(sol.ctx, nsteps, p["dt"], [dev(np.stack(p["vel"]))], [dev(p["u0"])], [u])
    sol.close()
    assert info["refine_iters"] >= nsteps and (info["gmres_iters"] == 0) == (isol == 1)
    assert _relerr(u.cpu().numpy().ravel(), ref) <= (1e-10 if precision == "fp64" else 1e-8), info


def test_march_3d_large_blocks_and_a_batch():
    """A 3D problem on the large-block kernels (matrix-free operators) marched together with a
    2D problem in one batched context: both states against O8."""
    from paper_2510_25991_gb300 import ddst as D
    ps = [I.march_problem(3, 24, 6), I.march_problem(2, 64, 8)]
    nsteps = 5
    sol = D.Solver([_spec(p) for p in ps], precision="mixed")
    sol.build_transfer()
    us = [torch.empty((p["n"] - 1,) * p["dim"], dtype=torch.float64, device="cuda") for p in ps]
    D.ddst_march(sol.ctx, nsteps, ps[0]["dt"], [dev(np.stack(p["vel"])) for p in ps],
                 [dev(p["u0"]) for p in ps], us)
    sol.close()
    for p, u in zip(ps, us):
        ref = O.imex_march(p, p["u0"], p["vel"], p["dt"], nsteps)
        assert _relerr(u.cpu().numpy().ravel(), ref) <= 1e-8, p["name"]


def test_march_zero_steps_returns_the_initial_state():
    from paper_2510_25991_gb300 import ddst as D
    p = I.march_problem(2, 32, 8)
    sol = D.Solver(_spec(p), precision="mixed")
    sol.build_transfer()
    u = torch.empty((31, 31), dtype=torch.float64, device="cuda")
    D.ddst_march(sol.ctx, 0, p["dt"], [dev(np.stack(p["vel"]))], [dev(p["u0"])], [u])
    with pytest.raises(D.DDSTError) as e:
        D.ddst_march(sol.ctx, 1, 0.0, [dev(np.stack(p["vel"]))], [dev(p["u0"])], [u])
    sol.close()
    assert e.value.name == "INVALID_ARG"
    assert np.array_equal(u.cpu().numpy(), p["u0"])
