"""The 2048^2 nonsymmetric workload in the benchmark's launch configuration (mixed precision,
HODLR tol 1e-8, sketch 64 + 10): sampled transfer-operator rows against oracle local solves,
and the solution against the oracle's global sparse direct solve (about two minutes of host
time)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import ddst_inputs as I
from oracle import ddst_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25991_gb300 import build as B
    from paper_2510_25991_gb300 import ddst as D
    B.build()
    prob = I.make_problem("convdiff2d")
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    sol = D.Solver(dict(dim=2, n=prob["n"], w=prob["w"], a=dev(prob["a"]), b=(20.0, 10.0, 0.0)),
                   precision="mixed", k_max=64, oversample=10)
    sol.build_transfer()
    n = prob["n"]
    u = torch.empty((n - 1, n - 1), dtype=torch.float64, device="cuda")
    yield prob, sol, u, dev
    sol.close()


def test_sampled_transfer_rows_match_oracle(full):
    """Rows of S_{j,j-1}, S_{j,j+1} from oracle transposed local solves (first/middle/last slab)."""
    from paper_2510_25991_gb300 import ddst as D
    prob, sol, u, dev = full
    n, w = prob["n"], prob["w"]
    A, b = O.assemble(prob)
    geo = O.slab_geometry(2, n, w)
    ng = geo.ngamma
    out = np.empty((ng, ng))
    rng = np.random.default_rng(5)
    Acsr = sp.csr_matrix(A)
    worst = 0.0
    for j in (0, geo.nds // 2, geo.nds - 1):
        I_ = geo.I[j]
        lu = spla.splu(sp.csc_matrix(Acsr[I_][:, I_].T))
        rows = rng.choice(ng, 6, replace=False)
        E = np.zeros((len(I_), len(rows)))
        E[geo.C[j][rows], np.arange(len(rows))] = 1.0
        Y = lu.solve(E)                      # columns of A_j^{-T} at central points
        for side, J in ((-1, geo.Jprev[j]), (1, geo.Jnext[j])):
            if J is None:
                continue
            ref = -(Acsr[I_][:, J].T @ Y).T   # rows of S_{j,j'} = -R_C A_j^{-1} A(I_j, J)
            D.ddst_get_transfer(sol.ctx, 0, j + 1, side, out)
            worst = max(worst, np.abs(out[rows] - ref).max() / np.abs(ref).max())
    assert worst <= 1e-3, worst


def test_full_solution_matches_global_sparse_solve(full):
    """Relative error <= 1e-8 against the oracle's global sparse direct solve (O2), plus the
    interface traces, on the full 2048^2 workload in the benchmark's configuration."""
    from paper_2510_25991_gb300 import ddst as D
    prob, sol, u, dev = full
    sol.compress(1e-8)
    st, info = sol.solve(dev(prob["f"]), dev(prob["g"]), u)
    n, w = prob["n"], prob["w"]
    A, b = O.assemble(prob)
    uref = O.global_solve(A, b)
    uh = u.cpu().numpy().ravel()
    err = np.linalg.norm(uh - uref) / np.linalg.norm(uref)
    assert err <= 1e-8, (err, info)
    geo = O.slab_geometry(2, n, w)
    uG = np.empty(geo.nds * geo.ngamma)
    D.ddst_interface_trace(sol.ctx, 0, uG)
    gref = uref[np.concatenate(geo.G)]
    assert np.linalg.norm(uG - gref) / np.linalg.norm(gref) <= 1e-8
