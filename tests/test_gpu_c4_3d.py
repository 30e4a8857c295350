"""The 3D variable-coefficient workload at full size, in the benchmark's configuration: 128^3
cells (127^3 = 2,048,383 unknowns), 8 slabs of 16 cells (7 double slabs with dense blocks of
31 * 127 = 3937 unknowns, padded to 3968), mixed precision (tensor-core block LU with FP64
refinement), transfer operators applied matrix-free.

The oracle's global sparse direct solve does not finish at this size (659 s at 64^3 on the
build host, growing like n^6), so parity at full size rests on facts that hold at any size:
* a = 1: the exact discrete solution by the sine transform (O2b), element by element; the
  transfer operators of the first, middle and last double slab probed against their closed form
  (O3b); and the plain DD GMRES iteration count against the paper's printed 19 (Sec. 5.2,
  Table fd_poisson_fixedH, 128^3 row).
* the workload's variable coefficient: the rigorous residual bound O2c on the solution.
Element-by-element parity of the same kernels against O2 is in test_gpu_bigblock.py.
"""
import numpy as np
import pytest

import ddst_inputs as I
from oracle import ddst_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, W = 128, 16


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25991_gb300 import build as B
    B.build()


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def run(prob, **opts):
    from paper_2510_25991_gb300 import ddst as D
    sol = D.Solver(dict(dim=3, n=N, w=W, a=dev(prob["a"])), precision="mixed", **opts)
    sol.build_transfer()
    u = torch.empty((N - 1,) * 3, dtype=torch.float64, device="cuda")
    st, info = sol.solve(dev(prob["f"]), dev(prob["g"]), u)
    return sol, u.cpu().numpy().ravel(), info


def test_c4_poisson_solution_matches_sine_transform():
    """a = 1 in the benchmark's configuration: relative error <= 1e-8 against O2b, in the 2-norm
    (the metric's error) and entry by entry."""
    prob = I.make_problem("vardiff3d", n=N, w=W, const_a=True)
    sol, u, info = run(prob)
    sol.close()
    ex = O.poisson_dst_solve(prob)
    assert np.linalg.norm(u - ex) / np.linalg.norm(ex) <= 1e-8, info
    assert np.abs(u - ex).max() <= 1e-8 * np.abs(ex).max()


def test_c4_poisson_transfer_operators_match_closed_form():
    """(I - K) x with x nonzero on one interface returns -S_{j,j'} x on both neighbours: slabs
    0, 1, 3, 4 (S_{j,j+1}) and 2, 3, 5, 6 (S_{j,j-1}) against O3b.  The FP32 local solve is
    accurate relative to the solution inside the double slab, whose size is set by the Dirichlet
    data x (S x on the central plane is two orders smaller), so the bound is 2e-5 of max |x|:
    kappa(A_j) u_32 with kappa(A_j) ~ 1.1e3 for these slabs."""
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("vardiff3d", n=N, w=W, const_a=True)
    sol = D.Solver(dict(dim=3, n=N, w=W, a=dev(prob["a"])), precision="mixed")
    sol.build_transfer()
    nds, ng = N // W - 1, (N - 1) ** 2
    rng = np.random.default_rng(3)
    for blk in (1, 2, 4, 5):
        x = np.zeros((nds, ng))
        x[blk] = rng.standard_normal(ng)
        y = torch.empty(nds * ng, dtype=torch.float64, device="cuda")
        D.ddst_apply_interface(sol.ctx, 0, dev(x.ravel()), y)
        y = y.cpu().numpy().reshape(nds, ng)
        ref = O.poisson_transfer_apply(3, N, W, x[blk])
        for j in (blk - 1, blk + 1):
            assert np.abs(-y[j] - ref).max() <= 2e-5 * np.abs(x[blk]).max(), (blk, j)
        assert np.abs(y[blk] - x[blk]).max() == 0.0
    sol.close()


def test_c4_poisson_gmres_iterations_match_paper():
    """Plain DD solve (no refinement) to 1e-8: the paper prints 19 iterations for the 3D
    finite-difference Poisson problem at 128^3 with H = 1/8 (Table fd_poisson_fixedH)."""
    prob = I.make_problem("vardiff3d", n=N, w=W, const_a=True)
    sol, u, info = run(prob, gmres_tol=1e-8, refine_max=0)
    sol.close()
    assert 17 <= info["gmres_iters"] <= 21, info["gmres_iters"]


def test_c4_variable_coefficient_solution_is_certified():
    """The workload itself (a = exp of 8 Fourier modes): with the refinement driven to a relative
    residual near FP64 rounding, the oracle's rigorous bound O2c certifies ||u - u*|| / ||u*||
    <= 1e-8.  At the benchmark's own stopping point (error estimate <= 1e-9) the same bound is
    looser (it divides by a_min lambda_min(L), well below lambda_min(A) for this coefficient) and
    is checked at 1e-6, next to the estimate."""
    prob = I.make_problem("vardiff3d", n=N, w=W)
    sol, u, info = run(prob, refine_tol=1e-12, refine_max=12)
    sol.close()
    bound = O.diffusion_error_bound(prob, u)
    assert bound <= 1e-8, (bound, info)
    sol, u2, info2 = run(prob)
    sol.close()
    assert info2["est_rel_error"] <= 1e-9
    assert O.diffusion_error_bound(prob, u2) <= 1e-6
