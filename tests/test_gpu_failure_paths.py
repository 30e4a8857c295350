"""Device-side error paths, exercised without faulting the GPU.

* A pipeline wait of the tensor-core transfer build that runs out (DDST_WAIT_CYCLES shortens the
  budget of the role waits; waits for copies and MMAs already issued keep the full budget): the
  call returns TIMEOUT, and the same context then builds the operators and solves correctly.
* A failed device allocation (DDST_FAIL_ALLOC fails the k-th allocation on the host, without
  calling cudaMalloc): setup and solve return OOM and leave the context usable.
* HODLR ranks above 16, the owner kernel's tail that reads the low-rank coefficients beyond its
  shared-memory stage from global memory, against the oracle's dense transfer operators.
"""
import numpy as np
import pytest

import ddst_inputs as I
from oracle import ddst_oracle as O

torch = pytest.importorskip("torch")


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25991_gb300 import build as B
    B.build()


def _spec(prob):
    return dict(dim=prob["dim"], n=prob["n"], w=prob["w"], a=dev(prob["a"]),
                b=tuple(prob["b"]) + (0.0,) * (3 - len(prob["b"])))


def _solve(sol, prob):
    u = torch.empty((prob["n"] - 1,) * prob["dim"], dtype=torch.float64, device="cuda")
    st, info = sol.solve(dev(prob["f"]), dev(prob["g"]), u)
    return u.cpu().numpy().ravel(), info


@pytest.mark.gpu
def test_transfer_build_wait_timeout_is_reported_and_the_context_recovers(monkeypatch):
    _gpu()
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("convdiff2d", n=128, w=16)  # 31-row blocks: tensor-core transfer build
    sol = D.Solver(_spec(prob), precision="mixed")
    monkeypatch.setenv("DDST_WAIT_CYCLES", "1")
    with pytest.raises(D.DDSTError) as e:
        sol.build_transfer()
    assert e.value.name == "TIMEOUT" and "bounded device wait expired" in str(e.value)
    monkeypatch.delenv("DDST_WAIT_CYCLES")
    sol.build_transfer()
    u, info = _solve(sol, prob)
    sol.close()
    A, b = O.assemble(prob)
    uref = O.global_solve(A, b)
    assert np.linalg.norm(u - uref) / np.linalg.norm(uref) <= 1e-8


@pytest.mark.gpu
def test_allocation_failure_is_reported_and_the_context_recovers(monkeypatch):
    _gpu()
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("convdiff2d", n=64, w=16)
    monkeypatch.setenv("DDST_FAIL_ALLOC", "6")  # during setup
    with pytest.raises(D.DDSTError) as e:
        D.Solver(_spec(prob), precision="mixed")
    assert e.value.name == "OOM" and "cudaMalloc" in str(e.value)
    monkeypatch.delenv("DDST_FAIL_ALLOC")
    sol = D.Solver(_spec(prob), precision="mixed")
    sol.build_transfer()
    monkeypatch.setenv("DDST_FAIL_ALLOC", "3")  # the solve's first buffer allocations
    with pytest.raises(D.DDSTError) as e:
        _solve(sol, prob)
    assert e.value.name == "OOM"
    monkeypatch.delenv("DDST_FAIL_ALLOC")
    u, info = _solve(sol, prob)
    sol.close()
    A, b = O.assemble(prob)
    uref = O.global_solve(A, b)
    assert np.linalg.norm(u - uref) / np.linalg.norm(uref) <= 1e-8


def test_allocation_failure_at_setup_needs_no_gpu(monkeypatch):
    """The injected failure comes before any CUDA call, so this runs on a host without a GPU."""
    from paper_2510_25991_gb300 import ddst as D
    monkeypatch.setenv("DDST_FAIL_ALLOC", "1")
    with pytest.raises(D.DDSTError) as e:
        D.ddst_setup_batch([dict(dim=2, n=16, w=4, a=np.ones((17, 17)))])
    assert e.value.name == "OOM"


@pytest.mark.gpu
def test_hodlr_ranks_above_16_apply_against_dense_operator():
    """3D, n = 16, w = 2: the transfer operators of the 15 x 15 interfaces have optimal ranks up
    to 45 at tol 1e-10 (O6), so the owner kernel reads most coefficients through its tail path.
    Both applications of the compressed operator agree with the oracle's dense I - K to 10 tol
    relative to ||I - K|| (FP64 path)."""
    _gpu()
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("vardiff3d", n=16, w=2)
    tol = 1e-10
    sol = D.Solver(_spec(prob), precision="fp64", leaf_size=16, k_max=64, oversample=10)
    sol.build_transfer()
    sol.compress(tol)
    _, _, max_rank = D.ddst_query(sol.ctx)
    A, b = O.assemble(prob)
    geo = O.slab_geometry(3, 16, 2)
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo))
    opt = max(max(U.shape[1] for U, V in lv)
              for S in Sp + Sn if S is not None
              for lv in O.hodlr_compress(S, tol, 16)["levels"])
    assert max_rank > 16 and opt <= max_rank <= opt + 10, (max_rank, opt)
    Mi = O.interface_matrix(Sp, Sn, geo.ngamma)
    nrm = np.linalg.norm(Mi, 2)
    rng = np.random.default_rng(2)
    for tr in (False, True):
        x = rng.standard_normal(geo.nds * geo.ngamma)
        y = torch.empty(x.size, dtype=torch.float64, device="cuda")
        D.ddst_apply_interface(sol.ctx, 0, dev(x), y, transpose=tr)
        ref = (Mi.T if tr else Mi) @ x
        assert np.linalg.norm(y.cpu().numpy() - ref) <= 10 * tol * nrm * np.linalg.norm(x), tr
    u, info = _solve(sol, prob)
    sol.close()
    uref = O.global_solve(A, b)
    assert np.linalg.norm(u - uref) / np.linalg.norm(uref) <= 1e-9
