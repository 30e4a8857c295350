"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each check uses a closed form, a structural
identity the paper proves, an independent dense computation, or a value the paper prints.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import ddst_inputs as I
from oracle import ddst_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _manufactured(dim, n, w, bconv, c0):
    """Linear ``a``, constant ``b``, variable ``c`` and quadratic ``u``: the stencil is exact."""
    X = I.node_coords(dim, n)
    alpha = [0.5, 0.25, -0.3][:dim]
    a = 1.0 + sum(alpha[d] * X[d] for d in range(dim))
    q = [1.0, -0.5, 0.7][:dim]
    u = sum(q[d] * X[d] ** 2 for d in range(dim)) + 0.3 * X[0] * X[1] + X[0]
    grad = []
    for d in range(dim):
        gd = 2 * q[d] * X[d]
        if d == 0:
            gd = gd + 0.3 * X[1] + 1.0
        if d == 1:
            gd = gd + 0.3 * X[0]
        grad.append(gd)
    # -div(a grad u) = -(grad a . grad u + a lap u)
    lap = sum(2 * q[d] for d in range(dim))
    f = -(sum(alpha[d] * grad[d] for d in range(dim)) + a * lap)
    # reaction varies along every axis, so a misplaced node index of c changes the answer
    beta = [0.5, -0.25, 0.4][:dim]
    c = c0 * (1.0 + sum(beta[d] * X[d] for d in range(dim)) + 0.3 * X[0] * X[1])
    f = f + sum(bconv[d] * grad[d] for d in range(dim)) + c * u
    inner = tuple(slice(1, n) for _ in range(dim))
    prob = dict(dim=dim, n=n, w=w, a=a, b=tuple(bconv), c=c, f=f[inner], g=u)
    return prob, u[inner].ravel()


@pytest.mark.parametrize("dim,n,w", [(2, 16, 4), (2, 24, 8), (3, 8, 2)])
def test_p1_manufactured_quadratic_exact(dim, n, w):
    """P1: five/seven-point stencil with face means is exact for linear a x quadratic u."""
    prob, uex = _manufactured(dim, n, w, bconv=[3.0, -2.0, 1.0][:dim], c0=1.5)
    A, b = O.assemble(prob)
    us = O.global_solve(A, b)
    assert np.abs(us - uex).max() <= 1e-12 * np.abs(uex).max()
    ud, uG, _ = O.dd_solve(prob)
    assert np.abs(ud - uex).max() <= 1e-12 * np.abs(uex).max()


def test_p1_harmonic_boundary_poisson():
    """P1: Poisson with f = 0 and g = x^2 - y^2 + xy reproduces g at every interior node."""
    prob = I.make_problem("poisson2d", n=32, w=8)
    prob["f"] = np.zeros_like(prob["f"])
    ud, _, _ = O.dd_solve(prob)
    gex = prob["g"][1:32, 1:32].ravel()
    assert np.abs(ud - gex).max() <= 1e-13


def _schur_route(A, geo):
    """Interface Schur complement T = A_JJ - A_JI A_II^{-1} A_IJ (Sec. 2.1), densely."""
    A = A.toarray()
    J = np.concatenate(geo.G)
    Ic = np.setdiff1d(np.arange(A.shape[0]), J)
    T = A[np.ix_(J, J)] - A[np.ix_(J, Ic)] @ np.linalg.solve(A[np.ix_(Ic, Ic)], A[np.ix_(Ic, J)])
    return T, J, Ic


@pytest.mark.parametrize("name,n,w", [("convdiff2d", 16, 4), ("poisson2d", 20, 4)])
def test_p2_two_route_identity(name, n, w):
    """P2: local-solve S equals -T_jj^{-1} T_jj' from the global Schur complement (Sec. 2.1)."""
    prob = I.make_problem(name, n=n, w=w)
    A, b = O.assemble(prob)
    geo = O.slab_geometry(2, n, w)
    facs = O.factor_local(A, geo)
    Sp, Sn = O.transfer_blocks(A, geo, facs)
    fh = O.equivalent_load(b, geo, facs)
    T, J, Ic = _schur_route(A, geo)
    m = geo.ngamma
    Ad = A.toarray()
    fprime = b[J] - Ad[np.ix_(J, Ic)] @ np.linalg.solve(Ad[np.ix_(Ic, Ic)], b[Ic])
    for j in range(geo.nds):
        Tjj = T[j * m:(j + 1) * m, j * m:(j + 1) * m]
        if Sp[j] is not None:
            ref = -np.linalg.solve(Tjj, T[j * m:(j + 1) * m, (j - 1) * m:j * m])
            assert np.abs(Sp[j] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
        if Sn[j] is not None:
            ref = -np.linalg.solve(Tjj, T[j * m:(j + 1) * m, (j + 1) * m:(j + 2) * m])
            assert np.abs(Sn[j] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
        fref = np.linalg.solve(Tjj, fprime[j * m:(j + 1) * m])
        assert np.abs(fh[j] - fref).max() <= 1e-11 * max(1.0, np.abs(fref).max())


def test_p3_brute_force_dense():
    """P3: every route equals a dense LAPACK solve of the global system on a tiny grid."""
    prob = I.make_problem("convdiff2d", n=16, w=4)
    A, b = O.assemble(prob)
    ud_dense = np.linalg.solve(A.toarray(), b)
    u1, uG1, _ = O.dd_solve(prob)
    u2, uG2, info = O.dd_solve(prob, use_gmres=True, tol=1e-13)
    scale = np.abs(ud_dense).max()
    assert np.abs(u1 - ud_dense).max() <= 1e-12 * scale
    assert np.abs(u2 - ud_dense).max() <= 1e-10 * scale
    geo = O.slab_geometry(2, 16, 4)
    assert np.abs(uG1 - ud_dense[np.concatenate(geo.G)]).max() <= 1e-12 * scale


def test_p3_block_thomas_vs_dense_and_reconstruct():
    prob = I.make_problem("convdiff2d", n=24, w=4)
    A, b = O.assemble(prob)
    geo = O.slab_geometry(2, 24, 4)
    facs = O.factor_local(A, geo)
    Sp, Sn = O.transfer_blocks(A, geo, facs)
    fh = O.equivalent_load(b, geo, facs)
    M = O.interface_matrix(Sp, Sn, geo.ngamma)
    ref = np.linalg.solve(M, np.concatenate(fh))
    uG = O.block_thomas(Sp, Sn, fh)
    assert np.abs(uG - ref).max() <= 1e-12 * np.abs(ref).max()
    x = np.random.default_rng(3).standard_normal(M.shape[0])
    assert np.abs(O.apply_interface(Sp, Sn, x) - M @ x).max() <= 1e-13 * np.abs(M @ x).max()
    # reconstruction from the exact traces gives the global solution
    us = O.global_solve(A, b)
    ur = O.reconstruct(A, b, geo, facs, us[np.concatenate(geo.G)])
    assert np.abs(ur - us).max() <= 1e-12 * np.abs(us).max()


def test_p4_constants_and_maximum_principle():
    """P4: g = 1, f = 0, c = 0 gives u = 1; S >= 0 entrywise; fhat + S 1 + S 1 = 1."""
    n, w = 32, 8
    # b scaled so the cell Peclet number is below 1: A is then an M-matrix
    prob = I.make_problem("convdiff2d", n=n, w=w, b=(2.0, 1.0))
    prob["f"] = np.zeros_like(prob["f"])
    prob["g"] = np.ones_like(prob["g"])
    A, b = O.assemble(prob)
    off = A - sp.diags(A.diagonal())
    assert off.max() <= 0.0
    ud, uG, _ = O.dd_solve(prob)
    assert np.abs(ud - 1.0).max() <= 1e-12
    geo = O.slab_geometry(2, n, w)
    facs = O.factor_local(A, geo)
    Sp, Sn = O.transfer_blocks(A, geo, facs)
    fh = O.equivalent_load(b, geo, facs)
    one = np.ones(geo.ngamma)
    for j in range(geo.nds):
        tot = fh[j].copy()
        for S in (Sp[j], Sn[j]):
            if S is not None:
                assert S.min() >= -1e-15
                tot += S @ one
        assert np.abs(tot - 1.0).max() <= 1e-12
    # rows of [S_{j,j-1} S_{j,j+1}] sum to < 1 for interior slabs (physical boundary leaks)
    j = geo.nds // 2
    assert (Sp[j] @ one + Sn[j] @ one).max() < 1.0


@pytest.mark.parametrize("name", ["convdiff2d", "poisson2d"])
def test_p5_spectrum_symmetric_about_one(name):
    """P5: eigenvalues of I - K pair up as 1 +- mu (two-coloured slab chain, Sec. 4.2)."""
    n, w = 24, 4
    prob = I.make_problem(name, n=n, w=w)
    A, b = O.assemble(prob)
    geo = O.slab_geometry(2, n, w)
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo))
    M = O.interface_matrix(Sp, Sn, geo.ngamma)
    ev = np.linalg.eigvals(M) - 1.0
    # every mu has a partner -mu (nearest-neighbour match of the spectrum with its negation)
    dist = np.abs(ev[:, None] + ev[None, :]).min(axis=1)
    assert dist.max() <= 1e-8
    if name == "poisson2d":
        # SPD: real spectrum in (0, 2] (red-black bound, Sec. 4.2; Thm. in Sec. 4.3)
        assert np.abs(ev.imag).max() <= 1e-10
        lam = ev.real + 1.0
        assert lam.min() > 0.0 and lam.max() <= 2.0 + 1e-12


def test_p6_energy_symmetry():
    """P6: with D = blkdiag(T_jj), D (I - K) = T is symmetric for an SPD problem (Sec. 4.2)."""
    n, w = 20, 4
    prob = I.make_problem("vardiff3d", n=n, w=w, dim=2, b=(0.0, 0.0))
    A, b = O.assemble(prob)
    assert abs(A - A.T).max() == 0.0
    geo = O.slab_geometry(2, n, w)
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo))
    M = O.interface_matrix(Sp, Sn, geo.ngamma)
    T, _, _ = _schur_route(A, geo)
    m = geo.ngamma
    D = np.zeros_like(T)
    for j in range(geo.nds):
        D[j * m:(j + 1) * m, j * m:(j + 1) * m] = T[j * m:(j + 1) * m, j * m:(j + 1) * m]
    DS = D @ M
    assert np.abs(DS - DS.T).max() <= 1e-9 * np.abs(DS).max()
    assert np.abs(DS - T).max() <= 1e-9 * np.abs(T).max()


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(t) for t in line.split()])
    return rows


def test_p7_printed_poisson_table_first_row():
    """P7: 3D Poisson, 16^3 grid, 8 slabs: kappa_2(S_H) and GMRES iterations as printed."""
    N, iters, kappa = _golden("fd_poisson_fixedH.txt")[0]
    n = round(N ** (1 / 3))
    prob = I.make_problem("vardiff3d", n=n, w=n // 8, const_a=True)
    A, b = O.assemble(prob)
    geo = O.slab_geometry(3, n, n // 8)
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo))
    M = O.interface_matrix(Sp, Sn, geo.ngamma)
    s = np.linalg.svd(M, compute_uv=False)
    assert abs(s[0] / s[-1] - kappa) <= 0.01
    rhs = np.random.default_rng(0).uniform(-1, 1, M.shape[0])
    _, its, _ = O.gmres(lambda v: M @ v, rhs, tol=1e-8)
    assert abs(its - iters) <= 0.1 * iters + 1


def _separable_poisson(dim, n, w):
    """Closed form of I - K for constant-coefficient Poisson, by separation of variables.

    The discrete sine modes of the interface directions diagonalize every S_{j,j+-1} at once.
    Mode k has the 1D Dirichlet eigenvalue mu_k = 4 sin^2(pi k / 2n) per direction, and the
    x-direction recurrence -u_{i-1} + (2 + mu) u_i - u_{i+1} = 0 on the 2w - 1 interior
    columns of a double slab.  Its solution, 1 on one outer column and 0 on the other, is
    sinh((2w - i) theta) / sinh(2 w theta) with cosh theta = 1 + mu / 2.  At the central
    column this is s = 1 / (2 cosh(w theta)).  Per mode, I - K is therefore tridiag(-s, 1, -s)
    over the N_ds interfaces, with eigenvalues 1 - 2 s cos(pi l / (N_ds + 1)).
    Returns (s per mode, N_ds).
    """
    k = np.arange(1, n)
    mu1 = 4.0 * np.sin(np.pi * k / (2 * n)) ** 2
    mu = mu1 if dim == 2 else (mu1[:, None] + mu1[None, :]).ravel()
    theta = np.arccosh(1.0 + mu / 2.0)
    return 1.0 / (2.0 * np.cosh(w * theta)), n // w - 1


def _separable_eigs(dim, n, w):
    s, nds = _separable_poisson(dim, n, w)
    c = np.cos(np.pi * np.arange(1, nds + 1) / (nds + 1))
    return np.sort((1.0 - 2.0 * s[:, None] * c[None, :]).ravel())


@pytest.mark.parametrize("dim,n,w", [(2, 24, 4), (2, 30, 5), (3, 8, 2), (3, 12, 3), (3, 12, 2)])
def test_p5_constant_coefficient_spectrum_closed_form(dim, n, w):
    """P5: the oracle's I - K for Poisson has exactly the separable closed-form spectrum."""
    name = "poisson2d" if dim == 2 else "vardiff3d"
    prob = I.make_problem(name, n=n, w=w, **({} if dim == 2 else dict(const_a=True)))
    prob["b"] = (0.0,) * dim
    A, _ = O.assemble(prob)
    geo = O.slab_geometry(dim, n, w)
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo))
    M = O.interface_matrix(Sp, Sn, geo.ngamma)
    assert M.shape[0] == (n // w - 1) * (n - 1) ** (dim - 1)
    ev = np.linalg.eigvals(M)
    assert np.abs(ev.imag).max() <= 1e-12
    assert np.abs(np.sort(ev.real) - _separable_eigs(dim, n, w)).max() <= 1e-12


def _separable_gmres_iterations(n, w, seed):
    """Oracle GMRES on the mode-diagonalized I - K (unitarily similar to the full operator).

    Applying the orthonormal sine transform on every interface is a unitary similarity, so
    GMRES from x0 = 0 takes the same steps on the transformed system; a Gaussian right-hand
    side stays Gaussian under it.
    """
    s, nds = _separable_poisson(3, n, w)

    def matvec(v):
        V = v.reshape(nds, s.size)
        Y = V.copy()
        Y[1:] -= s * V[:-1]
        Y[:-1] -= s * V[1:]
        return Y.ravel()

    rhs = np.random.default_rng(seed).standard_normal(nds * s.size)
    _, its, hist = O.gmres(matvec, rhs, tol=1e-8, maxit=100)
    assert hist[-1] <= 1e-8
    return its


@pytest.mark.parametrize("table,col_n", [("fd_poisson_fixedH.txt", "N"),
                                         ("fd_shrinkingH.txt", "invH")])
def test_p7_printed_poisson_tables_closed_form(table, col_n):
    """P7: both printed 3D Poisson tables of Sec. 5.2 at their own grid sizes.

    kappa_2(S_H) from the closed form (pinned to the oracle above) within 0.01 of each printed
    value, and oracle GMRES iterations within 10% + 1 of the printed S_H counts.
    """
    for row in _golden(table):
        if col_n == "N":
            n = round(row[0] ** (1 / 3))
            w = n // 8
        else:
            n = 64
            w = n // round(row[0])
        iters, kappa = row[1], row[2]
        ev = _separable_eigs(3, n, w)
        assert abs(ev.max() / ev.min() - kappa) <= 0.01, (n, w)
        its = _separable_gmres_iterations(n, w, seed=n + w)
        assert abs(its - iters) <= 0.1 * iters + 1, (n, w, its)


def test_gmres_finite_termination_and_residual():
    """GMRES on a diagonalizable matrix with k distinct eigenvalues stops after k steps."""
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    lam = np.repeat([0.5, 1.0, 1.7, 2.5, 3.0], 12)
    M = Q @ np.diag(lam) @ Q.T
    rhs = rng.standard_normal(60)
    x, its, hist = O.gmres(lambda v: M @ v, rhs, tol=1e-12)
    assert its == 5
    assert np.linalg.norm(M @ x - rhs) <= 1e-11 * np.linalg.norm(rhs)
    # nonsymmetric: residual estimate equals the true residual
    B = np.eye(40) + 0.3 * rng.standard_normal((40, 40)) / np.sqrt(40)
    rhs = rng.standard_normal(40)
    x, its, hist = O.gmres(lambda v: B @ v, rhs, tol=1e-10)
    true = np.linalg.norm(B @ x - rhs) / np.linalg.norm(rhs)
    assert true <= 2e-10 and abs(true - hist[-1]) <= 1e-12


def test_benchmark_convection_needs_no_upwinding():
    """Central convection keeps the nonsymmetric workload an M-matrix: every face coefficient
    a_face / h^2 exceeds |b_d| / (2h), i.e. the cell Peclet number |b_d| h / (2 a_face) < 1.
    Checked on the full 2048^2 coefficient field, and on the oracle's assembled operator at
    512^2 (off-diagonals <= 0, rows weakly diagonally dominant)."""
    prob = I.make_problem("convdiff2d")
    a, n = prob["a"], prob["n"]
    h = 1.0 / n
    fx, fy = 0.5 * (a[1:, :] + a[:-1, :]), 0.5 * (a[:, 1:] + a[:, :-1])
    bx, by = abs(prob["b"][0]), abs(prob["b"][1])
    assert max(bx * h / (2 * fx.min()), by * h / (2 * fy.min())) < 0.05
    small = I.make_problem("convdiff2d", n=512, w=32)
    A, _ = O.assemble(small)
    off = A - sp.diags(A.diagonal())
    assert off.max() <= 0.0
    assert (np.asarray(A.sum(axis=1)).ravel() >= -1e-9 * A.diagonal().max()).all()


def test_helmholtz_local_operators_definite_by_a_small_margin():
    """Helmholtz reading: c = -kappa^2 (1 - 0.5 exp(-25 |x - x_c|^2)) >= -kappa^2, so by Weyl
    lambda_min(-Lap_h) - kappa^2 <= lambda_min(A_j) <= lambda_min(-Lap_h) - kappa^2 (1 - bump/2),
    bump = the largest exp(-25 |x - x_c|^2) over the slab, with the closed form
    lambda_min(-Lap_h) = (4/h^2)(sin^2(pi/4w) + sin^2(pi/2n)) of the (2w-1) x (n-1) slab.
    At 4096^2, w = 32, kappa = 200 the margin is about 1%; the 512^2, kappa = 100, w = 8 case
    keeps it (0.8%), and every local operator the oracle assembles lies in its bracket."""
    import scipy.sparse.linalg as spla
    lap = lambda n, w: 4.0 * n * n * (np.sin(np.pi / (4 * w)) ** 2 + np.sin(np.pi / (2 * n)) ** 2)
    assert 0.01 <= lap(4096, 32) / 200.0 ** 2 - 1.0 <= 0.012
    n, w, kappa = 512, 8, 100.0
    assert 0.005 <= lap(n, w) / kappa ** 2 - 1.0 <= 0.01
    prob = I.make_problem("helmholtz2d", n=n, w=w, kappa=kappa)
    A, _ = O.assemble(prob)
    geo = O.slab_geometry(2, n, w)
    X = I.node_coords(2, n)
    bump = np.exp(-25.0 * ((X[0] - 0.5) ** 2 + (X[1] - 0.5) ** 2))
    for j in (0, 1, geo.nds // 2, geo.nds - 1):
        Aj = sp.csc_matrix(A[geo.I[j]][:, geo.I[j]])
        lam = spla.eigsh(Aj, k=1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
        xs = slice(j * w + 1, (j + 2) * w)            # interior x-nodes of double slab j
        top = bump[xs, 1:n].max()
        lo, hi = lap(n, w) - kappa ** 2, lap(n, w) - kappa ** 2 * (1.0 - 0.5 * top)
        assert lo * (1 - 1e-9) <= lam <= hi * (1 + 1e-9), (j, lam, lo, hi)
        assert lam > 0.0


def test_gmres_orthogonal_basis_keeps_finite_termination():
    """GMRES ends by step n on an n x n matrix when the Krylov basis stays orthogonal.

    A normal matrix with 200 eigenvalues graded from 1 to 1e-6: in exact arithmetic GMRES
    terminates by step 200.  Gram-Schmidt applied twice keeps the basis orthogonal to
    rounding, so the computed run reaches 1e-10 by then with the true residual at the
    estimate; a single classical pass loses orthogonality here and stalls near 1e-9.
    """
    rng = np.random.default_rng(0)
    n = 200
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = Q @ np.diag(np.logspace(0, -6, n)) @ Q.T
    rhs = rng.standard_normal(n)
    x, its, hist = O.gmres(lambda v: M @ v, rhs, tol=1e-10, maxit=n)
    assert its <= n and hist[-1] <= 1e-10
    assert np.linalg.norm(M @ x - rhs) <= 1e-9 * np.linalg.norm(rhs)


def test_p9_hodlr_ranks_exact_on_cs_decomposition():
    """P9: level-1 ranks equal #{sigma_i > tol ||S||_2} where the sigma_i are known exactly.

    Q = diag(U1, U2) [[C, -S], [S, C]] diag(V1, V2)^T with C = diag(cos theta), S = diag(sin
    theta) and U1, U2, V1, V2 orthogonal is orthogonal, so ||Q||_2 = 1, and its off-diagonal
    halves -U1 S V2^T and U2 S V1^T have singular values sin theta_i exactly (the CS
    decomposition).
    """
    rng = np.random.default_rng(7)
    h = 32
    orth = [np.linalg.qr(rng.standard_normal((h, h)))[0] for _ in range(4)]
    U1, U2, V1, V2 = orth
    sig = 10.0 ** (-0.4 * np.arange(h) - 0.1)   # never within a factor 10^0.1 of a power of 10
    cth = np.sqrt(1.0 - sig ** 2)
    Z = np.zeros((h, h))
    Q = (np.block([[U1, Z], [Z, U2]]) @ np.block([[np.diag(cth), -np.diag(sig)],
                                                  [np.diag(sig), np.diag(cth)]])
         @ np.block([[V1, Z], [Z, V2]]).T)
    assert np.abs(Q @ Q.T - np.eye(2 * h)).max() <= 1e-13
    for tol in (1e-2, 1e-5, 1e-8, 1e-11):
        want = int(np.sum(sig > tol))
        H = O.hodlr_compress(Q, tol=tol, leaf=8)
        assert [U.shape[1] for (U, V) in H["levels"][0]] == [want, want]
        H = O.hodlr_compress(Q, tol=tol, leaf=8, kmax=3)
        assert [U.shape[1] for (U, V) in H["levels"][0]] == [min(want, 3)] * 2


def test_p8_gradients_linear_directions_and_fd_in_a():
    """P8: adjoint gradients vs central differences (exact in f, g; 1e-5 relative in a)."""
    n, w = 16, 4
    prob = I.make_problem("convdiff2d", n=n, w=w)
    rng = np.random.default_rng(7)
    u_obs = rng.standard_normal((n - 1) ** 2)
    L, dLdf, dLdg, dLda, u, lam = O.loss_and_gradients(prob, u_obs)

    def loss(p):
        A, b = O.assemble(p)
        r = O.global_solve(A, b) - u_obs
        return 0.5 * float(r @ r)

    for key, grad in (("f", dLdf), ("g", dLdg), ("a", dLda)):
        d = rng.standard_normal(prob[key].shape)
        if key == "g":  # only boundary values of g matter
            mask = np.ones_like(d); mask[1:n, 1:n] = 0.0; d *= mask
        eps = 1e-3 if key != "a" else 1e-6
        pp = dict(prob); pm = dict(prob)
        pp[key] = prob[key] + eps * d
        pm[key] = prob[key] - eps * d
        fd = (loss(pp) - loss(pm)) / (2 * eps)
        an = float(np.sum(grad * d))
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-12), (key, fd, an)


def test_p8_adjoint_dot_product():
    prob = I.make_problem("convdiff2d", n=16, w=4)
    A, b = O.assemble(prob)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(A.shape[0]); y = rng.standard_normal(A.shape[0])
    lhs = O.global_solve(A, x) @ y
    rhs = x @ O.adjoint_solve(A, y)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_p9_hodlr_tree_and_exact_limits():
    """P9: tree partitions the index range; tol -> 0 reproduces S; known low rank found."""
    for ng in (31, 127, 2047, 1000):
        for leaf in (16, 64, 128):
            L = O.hodlr_levels(ng, leaf)
            spans = [O.hodlr_node(ng, L, t) for t in range(1 << L)]
            assert spans[0][0] == 0 and spans[-1][1] == ng
            assert all(spans[i][1] == spans[i + 1][0] for i in range(len(spans) - 1))
            assert max(hi - lo for lo, hi in spans) <= leaf
    prob = I.make_problem("convdiff2d", n=64, w=8)
    A, b = O.assemble(prob)
    geo = O.slab_geometry(2, 64, 8)
    facs = O.factor_local(A, geo)
    Sp, Sn = O.transfer_blocks(A, geo, facs, slabs=[3])
    S = Sp[0]
    H = O.hodlr_compress(S, tol=0.0, leaf=8)
    assert np.abs(O.hodlr_dense(H) - S).max() <= 1e-13 * np.abs(S).max()
    # truncation error per block is sigma_{r+1} <= tol ||S||_2 (Eckart-Young), total <= L * that
    tol = 1e-6
    H = O.hodlr_compress(S, tol=tol, leaf=8)
    err = np.linalg.norm(O.hodlr_dense(H) - S, 2) / np.linalg.norm(S, 2)
    assert err <= 2 * H["L"] * tol
    x = np.random.default_rng(0).standard_normal(S.shape[0])
    assert np.abs(O.hodlr_apply(H, x) - O.hodlr_dense(H) @ x).max() <= 1e-12 * np.abs(S @ x).max()
    # a matrix built from rank-2 off-diagonal pieces: exactly rank <= 2 everywhere
    ng = 64
    t = np.linspace(0, 1, ng)
    K = np.outer(np.cos(t), np.sin(t)) + np.outer(t, t ** 2)
    H = O.hodlr_compress(K + np.diag(t), tol=1e-12, leaf=8)
    assert max(U.shape[1] for lev in H["levels"] for (U, V) in lev) <= 2


@pytest.mark.parametrize("dim,n", [(2, 32), (3, 12), (3, 10)])
def test_o2b_sine_transform_poisson_matches_sparse_direct(dim, n):
    """O2b against O2 (SuperLU) on the same constant-coefficient Poisson system, and against the
    exact manufactured solution: with f = 0 and harmonic quadratic boundary data the discrete
    solution is the quadratic itself (the stencil is exact on quadratics)."""
    prob = I.make_problem("poisson2d" if dim == 2 else "vardiff3d", n=n, w=2, const_a=True)
    A, b = O.assemble(prob)
    u = O.global_solve(A, b)
    assert np.abs(O.poisson_dst_solve(prob) - u).max() <= 1e-12 * np.abs(u).max()
    harm = dict(prob, f=np.zeros_like(prob["f"]))
    inner = tuple(slice(1, n) for _ in range(dim))
    exact = prob["g"][inner].ravel()
    assert np.abs(O.poisson_dst_solve(harm) - exact).max() <= 1e-12 * np.abs(exact).max()
    with pytest.raises(ValueError):
        O.poisson_dst_solve(I.make_problem("vardiff3d", n=8, w=2))


@pytest.mark.parametrize("dim,n", [(2, 24), (3, 10)])
def test_o2c_error_bound_holds_and_is_tight_on_the_lowest_mode(dim, n):
    """O2c is an upper bound for a variable-coefficient operator and random perturbations of the
    exact solution, and it is attained (to 1%) when the error is the lowest Laplacian mode of a
    constant-coefficient operator: then A e = a lambda_min e exactly."""
    rng = np.random.default_rng(3)
    prob = I.make_problem("poisson2d" if dim == 2 else "vardiff3d", n=n, w=2)
    if dim == 2:
        prob["a"] = I.fourier_log_field(2, n, 77)
    for bconv in ((0.0,) * dim, (40.0, -25.0, 10.0)[:dim]):  # skew-symmetric convection too
        pb = dict(prob, b=bconv)
        A, b = O.assemble(pb)
        us = O.global_solve(A, b)
        for scale in (1e-3, 1e-8):
            u = us + scale * np.abs(us).max() * rng.standard_normal(us.size)
            true = np.linalg.norm(u - us) / np.linalg.norm(us)
            assert O.diffusion_error_bound(pb, u) >= true
    # the worst case: the error along the singular vector of the smallest singular value of A
    pb = dict(prob, b=(40.0, -25.0, 10.0)[:dim])
    A, b = O.assemble(pb)
    us = O.global_solve(A, b)
    _, sv, Vt = np.linalg.svd(A.toarray())
    e = 1e-6 * np.linalg.norm(us) * Vt[-1]
    true = np.linalg.norm(e) / np.linalg.norm(us)
    assert O.diffusion_error_bound(pb, us + e) >= true
    # a = 0.5 everywhere: lambda_min(A) = 0.5 lambda_min(L)
    pc = dict(prob, a=np.full_like(prob["a"], 0.5))
    A, b = O.assemble(pc)
    us = O.global_solve(A, b)
    grids = np.meshgrid(*([np.arange(1, n)] * dim), indexing="ij")
    mode = np.prod([np.sin(np.pi * gd / n) for gd in grids], axis=0).ravel()
    e = 1e-6 * np.linalg.norm(us) * mode / np.linalg.norm(mode)
    true = np.linalg.norm(e) / np.linalg.norm(us)
    bound = O.diffusion_error_bound(pc, us + e)
    assert true <= bound <= 1.01 * true
    assert abs(O.laplacian_lambda_min(dim, n) * 0.5 - (A @ mode)[0] / mode[0]) <= 1e-9 * n * n


@pytest.mark.parametrize("dim,n,w", [(2, 24, 4), (3, 12, 3), (3, 10, 5)])
def test_o3b_poisson_transfer_closed_form_matches_local_solves(dim, n, w):
    """O3b against O3: the closed-form transfer operator of constant-coefficient Poisson equals
    both S_{j,j-1} and S_{j,j+1} formed by sparse LU local solves, on every slab."""
    prob = I.make_problem("poisson2d" if dim == 2 else "vardiff3d", n=n, w=w, const_a=True)
    prob["b"] = (0.0,) * dim
    A, _ = O.assemble(prob)
    geo = O.slab_geometry(dim, n, w)
    Sp, Sn = O.transfer_blocks(A, geo, O.factor_local(A, geo))
    rng = np.random.default_rng(21)
    for j in range(geo.nds):
        x = rng.standard_normal(geo.ngamma)
        ref = O.poisson_transfer_apply(dim, n, w, x)
        for S in (Sp[j], Sn[j]):
            if S is not None:
                assert np.abs(S @ x - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dim,n,k", [(2, 16, (2, 3)), (3, 8, (1, 2, 1))])
def test_o8_eigenmode_decays_by_the_backward_euler_factor(dim, n, k):
    """O8 with D = 1, no convection and c = 1/dt: a product of sines is an eigenvector of the
    discrete Laplacian with eigenvalue lam = (4/h^2) sum_d sin^2(pi k_d h / 2), so each backward
    Euler step divides it by 1 + dt lam exactly (up to rounding)."""
    dt, nsteps = 2e-3, 5
    h = 1.0 / n
    x = np.arange(1, n) * h
    mode = np.ones((n - 1,) * dim)
    for d in range(dim):
        shape = [1] * dim
        shape[d] = n - 1
        mode = mode * np.sin(np.pi * k[d] * x).reshape(shape)
    lam = 4.0 / h ** 2 * sum(np.sin(np.pi * kd * h / 2.0) ** 2 for kd in k)
    prob = dict(dim=dim, n=n, w=n // 2, a=np.ones((n + 1,) * dim), b=(0.0,) * dim,
                c=np.full((n + 1,) * dim, 1.0 / dt))
    vel = [np.zeros((n + 1,) * dim)] * dim
    u = O.imex_march(prob, mode.ravel(), vel, dt, nsteps)
    ref = mode.ravel() / (1.0 + dt * lam) ** nsteps
    assert np.abs(u - ref).max() <= 1e-12 * np.abs(ref).max()


def test_o8_convection_term_exact_on_quadratics():
    """Central differences are exact on a function quadratic along each axis, so for
    U = x(1-x) y(1-y) (zero on the boundary) and arbitrary nodal velocities the right-hand side
    equals U/dt - v_x dU/dx - v_y dU/dy at every interior node (up to rounding)."""
    n, dt = 12, 0.05
    x = np.linspace(0.0, 1.0, n + 1)
    X, Y = np.meshgrid(x, x, indexing="ij")
    U = X * (1 - X) * Y * (1 - Y)
    rng = np.random.default_rng(4)
    vel = [rng.standard_normal((n + 1, n + 1)), rng.standard_normal((n + 1, n + 1))]
    f = O.imex_rhs(2, n, U[1:n, 1:n].ravel(), vel, dt)
    Ux = (1 - 2 * X) * Y * (1 - Y)
    Uy = X * (1 - X) * (1 - 2 * Y)
    ref = (U / dt - vel[0] * Ux - vel[1] * Uy)[1:n, 1:n].ravel()
    assert np.abs(f - ref).max() <= 1e-12 * np.abs(ref).max()


def test_o8_march_is_the_sequence_of_global_solves():
    """O8 against O1 + O2 step by step on the workload's inputs (a variable D and the shear
    velocity): every step is the global solve of the screened operator for O8's right-hand
    side, and the bump is damped and carried along -x."""
    p = I.march_problem(2, 24, 6)
    u = p["u0"].ravel()
    for _ in range(3):
        q = dict(p, f=O.imex_rhs(2, 24, u, p["vel"], p["dt"]).reshape(23, 23))
        A, b = O.assemble(q)
        u = O.global_solve(A, b)
    um = O.imex_march(p, p["u0"], p["vel"], p["dt"], 3)
    assert np.abs(um - u).max() <= 1e-12 * np.abs(u).max()
    assert np.linalg.norm(um) < np.linalg.norm(p["u0"])


def _random_hbs(ng, k, leaf, rng):
    """A matrix that is exactly HBS of rank k on the bisection tree, built by the telescoping
    recursion A_l = U_l A_{l-1} V_l^T + D_l from random orthonormal bases and random blocks."""
    import scipy.linalg as sla
    L = O.hodlr_levels(ng, leaf)
    if L == 0:
        return rng.standard_normal((ng, ng))

    def orth(n):
        return np.linalg.qr(rng.standard_normal((n, k)))[0]

    A = rng.standard_normal((2 * k, 2 * k))
    for lev in range(1, L + 1):
        if lev == L:
            sizes = [hi - lo for lo, hi in (O.hodlr_node(ng, L, t) for t in range(1 << L))]
        else:
            sizes = [2 * k] * (1 << lev)
        A = (sla.block_diag(*[orth(n) for n in sizes]) @ A
             @ sla.block_diag(*[orth(n) for n in sizes]).T
             + sla.block_diag(*[rng.standard_normal((n, n)) for n in sizes]))
    return A


def _hbs_sigma_ref(S, k, leaf):
    """max over tree nodes of sigma_{k+1} of the off-diagonal block row and column: no HBS of
    rank k on this tree can be closer to S (Eckart-Young on each block row / column)."""
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


@pytest.mark.parametrize("ng,k,leaf", [(200, 6, 12), (137, 4, 8), (64, 8, 16), (9, 3, 12)])
def test_p10_hbs_recovers_an_exact_hbs_matrix(ng, k, leaf):
    """P10: from s = 3k + q Gaussian samples of a matrix that is exactly HBS of rank k, the
    compression reproduces it to rounding (the defining property of sample-based HBS
    compression, Sec. 2.4); apply and transposed apply equal the dense expansion; storage is
    the O(kN) count of the format (leaves n^2 + 2nk, inner nodes 8k^2, root 4k^2)."""
    rng = np.random.default_rng(ng + k)
    S = _random_hbs(ng, k, leaf, rng)
    s = 3 * k + 10
    Om = rng.standard_normal((ng, s))
    Psi = rng.standard_normal((ng, s))
    H = O.hbs_compress(S @ Om, S.T @ Psi, Om, Psi, k, leaf)
    assert np.linalg.norm(O.hbs_dense(H) - S) <= 1e-12 * np.linalg.norm(S)
    x = rng.standard_normal(ng)
    assert np.abs(O.hbs_apply(H, x) - S @ x).max() <= 1e-12 * np.abs(S).sum(1).max() * np.abs(x).max()
    assert np.abs(O.hbs_apply(H, x, transpose=True) - S.T @ x).max() <= \
        1e-12 * np.abs(S).sum(0).max() * np.abs(x).max()
    L = H["L"]
    if L == 0:
        want = ng * ng
    else:
        leaves = [hi - lo for lo, hi in (O.hodlr_node(ng, L, t) for t in range(1 << L))]
        want = sum(n * n + 2 * n * k for n in leaves) + 8 * k * k * ((1 << L) - 2) + 4 * k * k
    assert O.hbs_entries(H) == want


def test_p10_hbs_error_between_eckart_young_bounds():
    """P10: on a transfer operator of a 2D double slab the HBS error lies between the best any
    rank-k HBS on the tree can do (sigma_{k+1} of the worst block row or column) and a small
    multiple of it, and falls as k grows."""
    prob = I.make_problem("convdiff2d", n=128, w=16)
    A, b = O.assemble(prob)
    geo = O.slab_geometry(2, 128, 16)
    facs = O.factor_local(A, geo)
    Sp, Sn = O.transfer_blocks(A, geo, facs, slabs=[2])
    S = Sn[0]
    ng = S.shape[0]
    nS = np.linalg.norm(S, 2)
    rng = np.random.default_rng(11)
    errs = []
    for k in (4, 6, 8, 12):
        s = 3 * k + 10
        Om = rng.standard_normal((ng, s))
        Psi = rng.standard_normal((ng, s))
        H = O.hbs_compress(S @ Om, S.T @ Psi, Om, Psi, k, 2 * k)
        err = np.linalg.norm(O.hbs_dense(H) - S, 2)
        ref = _hbs_sigma_ref(S, k, 2 * k)
        assert ref <= err * (1 + 1e-12) and err <= 30 * ref, (k, err / nS, ref / nS)
        errs.append(err / nS)
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))
    assert errs[-1] <= 1e-6
