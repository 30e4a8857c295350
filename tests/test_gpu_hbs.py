"""Nested-basis HBS compression (Sec. 2.4; Alg. 1's s = 3k + q Gaussian samples) on the GPU
against the oracle's O9 on the same test matrices, with device-drawn samples against the
Eckart-Young bounds of the tree, and the HBS operators inside the solver against the oracle's
global solve, transfer operators and adjoint."""
import numpy as np
import pytest
import scipy.linalg as sla

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


def random_hbs(ng, k, leaf, rng):
    """Exactly HBS of rank k on the bisection tree: A_l = U_l A_{l-1} V_l^T + D_l."""
    L = O.hodlr_levels(ng, leaf)
    if L == 0:
        return rng.standard_normal((ng, ng))
    A = rng.standard_normal((2 * k, 2 * k))
    for lev in range(1, L + 1):
        if lev == L:
            sizes = [hi - lo for lo, hi in (O.hodlr_node(ng, L, t) for t in range(1 << L))]
        else:
            sizes = [2 * k] * (1 << lev)
        orth = lambda n: np.linalg.qr(rng.standard_normal((n, k)))[0]
        A = (sla.block_diag(*[orth(n) for n in sizes]) @ A
             @ sla.block_diag(*[orth(n) for n in sizes]).T
             + sla.block_diag(*[rng.standard_normal((n, n)) for n in sizes]))
    return A


def transfer_block(n, w, j=2):
    prob = I.make_problem("convdiff2d", n=n, w=w)
    A, b = O.assemble(prob)
    geo = O.slab_geometry(2, n, w)
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo), slabs=[j])
    return np.asarray(Sn[0])


def sigma_ref(S, k, leaf):
    """sigma_{k+1} of the worst off-diagonal block row or column of the tree: no rank-k HBS on
    this tree is closer to S in the 2-norm."""
    ng = S.shape[0]
    L = O.hodlr_levels(ng, leaf)
    worst = 0.0
    for lev in range(1, L + 1):
        for t in range(1 << lev):
            lo, hi = O.hodlr_node(ng, lev, t)
            rest = np.r_[0:lo, hi:ng]
            for B in (S[lo:hi][:, rest], S[rest][:, lo:hi]):
                sv = np.linalg.svd(B, compute_uv=False)
                if len(sv) > k:
                    worst = max(worst, sv[k])
    return worst


CASES = [("exact", 200, 6, 12), ("exact", 137, 4, 8), ("exact", 9, 3, 12),
         ("exact", 1000, 8, 16), ("transfer", 128, 8, 16), ("transfer", 512, 12, 24)]


def _matrix(kind, size, k, leaf, rng):
    if kind == "exact":
        return random_hbs(size, k, leaf, rng)
    return transfer_block(size, size // 16 if size <= 128 else 32)


@pytest.mark.parametrize("kind,size,k,leaf", CASES, ids=[f"{c[0]}-{c[1]}-k{c[2]}" for c in CASES])
def test_hbs_fp64_matches_oracle_on_the_same_samples(kind, size, k, leaf):
    """Same S, Omega, Psi: the GPU factors define the oracle's operator (apply, transposed
    apply and dense expansion agree to rounding; where the pivoted QR of a node meets a near tie
    both are valid compressions, so the bound also admits twice the oracle's own error)."""
    from paper_2510_25991_gb300 import ddst as D
    rng = np.random.default_rng(size + k)
    S = _matrix(kind, size, k, leaf, rng)
    ng = S.shape[0]
    s = 3 * k + 10
    Om = rng.standard_normal((ng, s))
    Psi = rng.standard_normal((ng, s))
    Ho = O.hbs_compress(S @ Om, S.T @ Psi, Om, Psi, k, leaf)
    Do = O.hbs_dense(Ho)
    nS = np.linalg.norm(S)
    err_o = np.linalg.norm(Do - S) / nS
    if kind == "exact":
        assert err_o <= 1e-12
    H = D.HBS(S, k, s, leaf, Om, Psi, precision="fp64")
    try:
        assert H.stats() == (Ho["L"], O.hbs_entries(Ho))
        tol = max(1e-9, 2.0 * err_o)
        assert np.linalg.norm(H.dense() - Do) <= tol * nS
        for tr in (False, True):
            x = rng.standard_normal(ng)
            y = np.empty(ng)
            H.apply(x, y, transpose=tr)
            yo = O.hbs_apply(Ho, x, transpose=tr)
            assert np.abs(y - yo).max() <= tol * nS * np.abs(x).max(), tr
            # device vectors take the same path
            yd = torch.empty(ng, dtype=torch.float64, device="cuda")
            H.apply(dev(x), yd, transpose=tr)
            assert np.abs(yd.cpu().numpy() - y).max() <= 1e-14 * nS * np.abs(x).max()
    finally:
        H.close()


@pytest.mark.parametrize("kind,size,k,leaf", [CASES[0], CASES[4], CASES[5]],
                         ids=["exact-200", "transfer-128", "transfer-512"])
def test_hbs_fp32_within_its_precision_of_the_oracle(kind, size, k, leaf):
    """FP32 storage and FP32 node algebra: within 1e-4 ||S|| of the oracle's FP64 operator."""
    from paper_2510_25991_gb300 import ddst as D
    rng = np.random.default_rng(3 * size + k)
    S = _matrix(kind, size, k, leaf, rng)
    ng = S.shape[0]
    s = 3 * k + 10
    Om = rng.standard_normal((ng, s))
    Psi = rng.standard_normal((ng, s))
    Ho = O.hbs_compress(S @ Om, S.T @ Psi, Om, Psi, k, leaf)
    Do = O.hbs_dense(Ho)
    nS = np.linalg.norm(S)
    err_o = np.linalg.norm(Do - S) / nS
    H = D.HBS(S, k, s, leaf, Om, Psi, precision="mixed")
    try:
        assert np.linalg.norm(H.dense() - Do) <= (1e-4 + 2.0 * err_o) * nS
        x = rng.standard_normal(ng)
        y = np.empty(ng)
        H.apply(x, y, transpose=True)
        assert np.abs(y - O.hbs_apply(Ho, x, transpose=True)).max() <= \
            (1e-4 + 2.0 * err_o) * nS * np.abs(x).max()
    finally:
        H.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hbs_device_samples_between_eckart_young_bounds(precision):
    """Samples drawn on the device: the 2-norm error of the compressed transfer operator lies
    between sigma_ref (no rank-k HBS on the tree does better) and 30 sigma_ref (plus the FP32
    floor in mixed precision)."""
    from paper_2510_25991_gb300 import ddst as D
    S = transfer_block(256, 16)
    nS = np.linalg.norm(S, 2)
    for k in (6, 10):
        H = D.HBS(S, k, precision=precision)
        try:
            err = np.linalg.norm(H.dense() - S, 2)
        finally:
            H.close()
        ref = sigma_ref(S, k, 2 * k)
        floor = 0.0 if precision == "fp64" else 1e-5 * nS
        assert ref * (1 - 1e-6) <= err + floor and err <= 30 * ref + floor, (k, err / nS, ref / nS)


def _solver(probs, precision, **opts):
    from paper_2510_25991_gb300 import ddst as D
    sol = D.Solver([dict(dim=p["dim"], n=p["n"], w=p["w"], a=dev(p["a"]),
                         b=tuple(p["b"]) + (0.0,) * (3 - len(p["b"])),
                         c=dev(p["c"]) if p.get("c") is not None else None) for p in probs],
                   precision=precision, **opts)
    sol.build_transfer()
    return sol


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hbs_operators_in_the_solver(precision):
    """compress_hbs on a 128^2 convection-diffusion problem: every expanded transfer operator
    within the Eckart-Young bounds of the oracle's, the interface operator accordingly, and the
    refined solution and adjoint within 1e-8 of the oracle's global solves."""
    from paper_2510_25991_gb300 import ddst as D
    prob = I.make_problem("convdiff2d", n=128, w=16)
    A, b = O.assemble(prob)
    geo = O.slab_geometry(2, 128, 16)
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo))
    k = 8
    sol = _solver([prob], precision)
    try:
        sol.compress_hbs(k)
        ng = geo.ngamma
        out = np.empty((ng, ng))
        floor = 0.0 if precision == "fp64" else 1e-5
        worst = 0.0  # largest 2-norm error of a block
        for j in range(geo.nds):
            for side, ref in ((-1, Sp[j]), (1, Sn[j])):
                if ref is None:
                    continue
                D.ddst_get_transfer(sol.ctx, 0, j + 1, side, out)
                nS = np.linalg.norm(ref, 2)
                err = np.linalg.norm(out - ref, 2)
                worst = max(worst, err)
                assert err <= 30 * sigma_ref(ref, k, 2 * k) + floor * nS, (j, side, err / nS)
        x = np.random.default_rng(1).standard_normal(geo.nds * ng)
        M = O.interface_matrix(Sp, Sn, ng)
        for tr in (False, True):
            y = np.empty_like(x)
            D.ddst_apply_interface(sol.ctx, 0, x, y, transpose=tr)
            yo = (M.T if tr else M) @ x
            # two blocks per interface, |E x|_inf <= sqrt(ng) ||E||_2 |x|_inf
            assert np.abs(y - yo).max() <= 2 * np.sqrt(ng) * worst * np.abs(x).max() + 1e-12
        u = torch.empty((127, 127), dtype=torch.float64, device="cuda")
        st, info = sol.solve(dev(prob["f"]), dev(prob["g"]), u)
        assert info["max_rank"] == k
        ref = O.global_solve(A, b).reshape(127, 127)
        assert np.abs(u.cpu().numpy() - ref).max() <= 1e-8 * np.abs(ref).max(), info
        dLdu = np.random.default_rng(2).standard_normal((127, 127))
        df = torch.empty((127, 127), dtype=torch.float64, device="cuda")
        D.ddst_solve_adjoint(sol.ctx, dev(dLdu), df)
        lam = O.adjoint_solve(A, dLdu.ravel()).reshape(127, 127)
        assert np.abs(df.cpu().numpy() - lam).max() <= 1e-8 * np.abs(lam).max()
    finally:
        sol.close()


def test_hbs_batch_with_a_single_interface_problem():
    """A batch whose first problem has one interface (K = 0 there) and a second of 7 double
    slabs: both solves within 1e-8 of the oracle after HBS compression."""
    from paper_2510_25991_gb300 import ddst as D
    probs = [I.make_problem("convdiff2d", n=64, w=32), I.make_problem("convdiff2d", n=128, w=16)]
    sol = _solver(probs, "mixed")
    try:
        sol.compress_hbs(8)
        us, fs, gs = [], [], []
        for p in probs:
            n = p["n"]
            us.append(torch.empty((n - 1, n - 1), dtype=torch.float64, device="cuda"))
            fs.append(dev(p["f"]))
            gs.append(dev(p["g"]))
        D.ddst_solve_batch(sol.ctx, fs, gs, us)
        for p, u in zip(probs, us):
            A, b = O.assemble(p)
            ref = O.global_solve(A, b).reshape(u.shape)
            assert np.abs(u.cpu().numpy() - ref).max() <= 1e-8 * np.abs(ref).max()
    finally:
        sol.close()


def test_hbs_bad_arguments_are_errors():
    from paper_2510_25991_gb300 import ddst as D
    S = np.eye(40)
    with pytest.raises(D.DDSTError):
        D.HBS(S, 8, nsamples=20, leaf=16)       # leaf rows + rank above the sample count
    with pytest.raises(D.DDSTError):
        D.HBS(S, 40, nsamples=96, leaf=16)      # rank above 32
    prob = I.make_problem("convdiff2d", n=64, w=16)
    sol = _solver([prob], "mixed")
    try:
        with pytest.raises(D.DDSTError):
            sol.compress_hbs(0)
        with pytest.raises(D.DDSTError):
            sol.compress_hbs(30, oversample=10)   # 3 * 30 + 10 > 96
        sol.compress_hbs(6)                      # the context stays usable
        n = 64
        u = torch.empty((n - 1, n - 1), dtype=torch.float64, device="cuda")
        sol.solve(dev(prob["f"]), dev(prob["g"]), u)
        A, b = O.assemble(prob)
        ref = O.global_solve(A, b).reshape(n - 1, n - 1)
        assert np.abs(u.cpu().numpy() - ref).max() <= 1e-8 * np.abs(ref).max()
    finally:
        sol.close()
