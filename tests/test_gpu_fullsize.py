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


def test_mixed_hodlr_against_dense_operator_and_optimal_ranks(full):
    """Mixed-precision compression of this workload's transfer operators on the first, middle and
    last double slab, at tol 1e-5.  That is the smallest tolerance the mixed path meets: its FP32
    sketch and range finder (samples below 1e3 eps_32 of their own norm are rejected as rounding
    noise) floor the error near 2e-5 of ||S|| (measured 2.3e-5, 1.0e-5 and 7.6e-6 on these three
    blocks for any request below 1e-5, the benchmark's 1e-8 included), and the FP64 refinement of
    the solve restores the 1e-8 solution.  Checked: error against the dense FP32 operator it
    compresses <= 10 tol (2-norm), and the largest rank between the truncated-SVD optimum of O6 on
    the oracle's operator (O3) and that optimum plus the oversampling."""
    from paper_2510_25991_gb300 import ddst as D
    prob, sol, u, dev = full
    n, w = prob["n"], prob["w"]
    tol, leaf, q = 1e-5, 128, 10
    geo = O.slab_geometry(2, n, w)
    ng = geo.ngamma
    picks = ((0, 1), (geo.nds // 2, 1), (geo.nds - 1, -1))
    dense = {}
    for j, side in picks:
        out = np.empty((ng, ng))
        D.ddst_get_transfer(sol.ctx, 0, j + 1, side, out)
        dense[j] = out
    sol.compress(tol)
    _, _, gpu_rank = D.ddst_query(sol.ctx)
    A, b = O.assemble(prob)
    Acsr = sp.csr_matrix(A)
    opt = 0
    for j, side in picks:
        out = np.empty((ng, ng))
        D.ddst_get_transfer(sol.ctx, 0, j + 1, side, out)
        nrm = np.linalg.norm(dense[j], 2)
        assert np.linalg.norm(out - dense[j], 2) <= 10 * tol * nrm, j
        facs = [None] * geo.nds
        I_ = geo.I[j]
        facs[j] = spla.splu(sp.csc_matrix(Acsr[I_][:, I_]))
        Sp, Sn = O.transfer_blocks(A, geo, facs, slabs=[j])
        ref = Sn[0] if side > 0 else Sp[0]
        H = O.hodlr_compress(ref, tol, leaf)
        opt = max(opt, max(U.shape[1] for lev in H["levels"] for U, _ in lev))
    # max over every block of the context against the max over the three blocks of the oracle
    assert opt <= gpu_rank <= opt + q, (gpu_rank, opt)


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
