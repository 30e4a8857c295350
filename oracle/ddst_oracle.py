"""FP64 CPU oracle for the overlapping solution-transfer domain decomposition.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously-correct reference that
the CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product library never does, and it shares no
code with the CUDA path (inputs come from the separate ``ddst_inputs`` generators).

Everything is FP64 NumPy/SciPy.  Each function cites the passage of arXiv 2510.25991 it
follows ("the paper" below):

* O1 ``assemble``: finite-difference discretization ``A u = b`` of the boundary value problem
  (Sec. 1, Eq. (basic)) with the five-point stencil of Sec. 2.1 (seven-point in 3D, Sec. 5.2); variable ``a`` enters through
  face values ``a_pq = (a_p + a_q)/2``; convection by central differences; Dirichlet
  neighbours moved to the right-hand side.
* O2 ``global_solve``: sparse direct solve of the global system (SuperLU).
* O2b ``poisson_dst_solve``: the same global solution for the constant-coefficient Poisson
  operator (``a = 1``, ``b = 0``, ``c = 0``; the Poisson experiments of Sec. 5.2, Table
  fd_poisson_fixedH) by the sine transform that diagonalizes it (separation of variables); exact
  to rounding and fast at any size.
* O2c ``diffusion_error_bound``: a rigorous a-posteriori bound on ``||u - u*|| / ||u*||`` (constant
  convection, ``c >= 0``) from the FP64 residual of O1 and the closed-form smallest eigenvalue of
  the constant-coefficient Laplacian, used where O2 is too large to run.
* O3 ``transfer_blocks`` / ``equivalent_load``: the local solution-transfer operators
  ``S_{j,j'} = -R_{C_j} A_j(I_j,I_j)^{-1} A_j(I_j,J_{j,j'})`` (Sec. 2.2, Eq. (defS); Sec. 2.5)
  and the equivalent loads ``fhat_j`` (Sec. 2.2, Eq. (equilib1), Fig. genBC: local solve with the global load and physical data,
  zero Dirichlet data on the neighbouring interfaces, restricted to ``Gamma_j``), computed by
  local sparse LU solves on each double slab ``Psi_j``.
* O3b ``poisson_transfer_apply``: ``S_{j,j'} x`` for the constant-coefficient Poisson operator
  in closed form: in the transverse sine basis every transfer operator is diagonal, with the
  separable solution of the double slab as multiplier (used to probe the transfer operators
  where forming O3 is too large).
* O4 ``interface_matrix`` / ``block_thomas`` / ``gmres``: the equilibrium system
  ``(I - K) u = fhat`` of Sec. 1, Eq. (modelS) / Sec. 2.2, Eq. (modelScond) solved exactly by block Gaussian elimination, and by
  unrestarted GMRES (Sec. 5 and Sec. 5.2, x0 = 0, classical Gram-Schmidt applied twice, Givens rotations).
* O5 ``reconstruct``: volume values from the interface traces by local Dirichlet solves (the
  local solutions patch together: Sec. 3.1, proof of the Fredholm-structure proposition).
* O6 ``hodlr_compress``: weak-admissibility hierarchical compression of each ``S_{j,j'}``
  (Sec. 2.4) on a balanced bisection tree shared by source and target interface, every
  off-diagonal block truncated by SVD at the smallest rank with
  ``sigma_{r+1} <= tol * ||S_{j,j'}||_2``; diagonal leaves kept dense.
* O9 ``hbs_compress`` / ``hbs_apply``: the nested-basis HBS form of a transfer block computed
  from random samples ``Y = S Om`` and ``Z = S^T Psi`` alone (Sec. 2.4; Alg. 1 draws
  ``s = 3k + q`` Gaussian samples): per tree node the bases from the samples projected onto the
  null space of the node's test rows, the uncaptured diagonal part from pseudo-inverses, and the
  samples of the reduced matrix passed to the parent; the telescoping apply over the tree.
* O7 ``adjoint_solve`` / ``gradients``: discrete adjoint of the FD system for a loss on ``u``
  (``lambda = A^{-T} dL/du``) and the gradients with respect to ``f``, ``g`` and nodal ``a``.
* O8 ``imex_rhs`` / ``imex_march``: backward-Euler IMEX time marching of the convection-diffusion
  example (Sec. 6, Example 1, Eq. (convdiff)): the screened operator ``-div(D grad U) + U/dt`` is
  solved every step for ``U_n/dt - v . grad U_n``, the convection term by central differences
  with ``U_n = 0`` on the boundary (the library's Dirichlet stand-in for the example's Neumann
  and periodic sides).

Conventions: grid and array layout as documented in ``ddst_inputs``; slabs are normal to the
x axis; interface ``Gamma_j`` (``j = 1..N_ds``, ``N_ds = n/w - 1``) is the node plane
``x = j w h``; double slab ``Psi_j`` holds the interior x-planes ``(j-1)w+1 .. (j+1)w-1``.
Interface values are ordered like the remaining axes in C order.

Every function above is pinned by ``tests/test_oracle_pins.py`` to facts the paper and the
mathematics fix (closed forms, exact identities, printed values, brute force), and
``tests/test_oracle_mutations.py`` checks that one-line mistakes planted in a copy of this
module make a pin fail.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "assemble", "global_solve", "poisson_dst_solve", "laplacian_lambda_min",
    "diffusion_error_bound", "SlabGeometry", "slab_geometry", "factor_local",
    "transfer_blocks", "poisson_transfer_apply", "equivalent_load", "interface_matrix", "apply_interface",
    "block_thomas", "gmres", "reconstruct", "dd_solve", "hodlr_levels", "hodlr_node",
    "hodlr_compress", "hodlr_dense", "hodlr_apply", "adjoint_solve", "gradients",
    "loss_and_gradients", "imex_rhs", "imex_march", "hbs_compress", "hbs_dense", "hbs_apply",
    "hbs_entries",
]


# ---------------------------------------------------------------------------------------
# O1  Discretization (Sec. 1 Eq. (basic); five-point stencil Sec. 2.1; seven-point Sec. 5.2)
# ---------------------------------------------------------------------------------------

def _interior(dim, n):
    return tuple(slice(1, n) for _ in range(dim))


def _shifted(dim, n, d, s):
    sl = [slice(1, n)] * dim
    sl[d] = slice(1 + s, n + s)
    return tuple(sl)


def assemble(prob: dict):
    """Sparse FP64 matrix ``A`` on the interior nodes and the right-hand side ``b``.

    ``(A u)_p = sum_faces a_pq (u_p - u_q)/h^2 + sum_d b_d (u_{p+e_d} - u_{p-e_d})/(2h)
    + c_p u_p`` with ``a_pq = (a_p + a_q)/2``.  Boundary neighbours ``q`` carry ``u_q = g_q``
    and move to the right-hand side: ``b_p = f_p - coef_pq g_q``.
    Returns ``(A, b)`` with ``A`` CSR of size ``(n-1)^dim`` and ``b`` flat (C order).
    """
    dim, n = prob["dim"], prob["n"]
    a, f, g = prob["a"], prob["f"], prob["g"]
    bconv = prob.get("b") or (0.0,) * dim
    c = prob.get("c")
    h = 1.0 / n
    N = (n - 1) ** dim
    idx = -np.ones((n + 1,) * dim, dtype=np.int64)
    idx[_interior(dim, n)] = np.arange(N).reshape((n - 1,) * dim)
    P = idx[_interior(dim, n)].ravel()
    ap = a[_interior(dim, n)].ravel()
    diag = np.zeros(N)
    rhs = np.array(f, dtype=np.float64).ravel().copy()
    rows, cols, vals = [], [], []
    for d in range(dim):
        for s in (+1, -1):
            sl = _shifted(dim, n, d, s)
            aq = a[sl].ravel()
            af = 0.5 * (ap + aq)
            coef = -af / h ** 2 + s * bconv[d] / (2.0 * h)
            diag += af / h ** 2
            Q = idx[sl].ravel()
            inner = Q >= 0
            rows.append(P[inner]); cols.append(Q[inner]); vals.append(coef[inner])
            bnd = ~inner
            rhs[P[bnd]] -= coef[bnd] * g[sl].ravel()[bnd]
    if c is not None:
        diag += c[_interior(dim, n)].ravel()
    rows.append(P); cols.append(P); vals.append(diag)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    A.sum_duplicates()
    return A, rhs


# ---------------------------------------------------------------------------------------
# O2  Global sparse direct solve
# ---------------------------------------------------------------------------------------

def global_solve(A, b):
    """``u* = A^{-1} b`` by SuperLU (FP64)."""
    lu = spla.splu(sp.csc_matrix(A))
    return lu.solve(np.asarray(b, dtype=np.float64))


def poisson_dst_solve(prob: dict):
    """O2b: ``u* = A^{-1} b`` for ``a = 1``, ``b = 0``, ``c = 0`` by the discrete sine transform.

    The five/seven-point Dirichlet Laplacian on the interior nodes is the Kronecker sum of the
    1D operators ``tridiag(-1, 2, -1)/h^2``, whose eigenvectors are ``sin(pi i k / n)``
    (``k = 1..n-1``) with eigenvalues ``(4/h^2) sin^2(pi k / (2n))``.  The type-1 DST applies
    that eigenbasis (up to a scale its inverse removes), so the solve is: transform ``b``,
    divide by the eigenvalue sums, transform back.  ``b`` is O1's right-hand side (load plus
    boundary data).
    """
    dim, n = prob["dim"], prob["n"]
    if not (np.all(np.asarray(prob["a"]) == 1.0) and prob.get("c") is None
            and not any(prob.get("b") or ())):
        raise ValueError("poisson_dst_solve needs a = 1, b = 0 and no reaction term")
    _, b = assemble(prob)
    k = np.arange(1, n)
    lam1 = 4.0 * n * n * np.sin(np.pi * k / (2.0 * n)) ** 2
    lam = np.zeros((n - 1,) * dim)
    for d in range(dim):
        shape = [1] * dim
        shape[d] = n - 1
        lam = lam + lam1.reshape(shape)
    bh = sfft.dstn(b.reshape((n - 1,) * dim), type=1)
    return sfft.idstn(bh / lam, type=1).ravel()


def laplacian_lambda_min(dim: int, n: int) -> float:
    """Smallest eigenvalue of the constant-coefficient Dirichlet Laplacian (O2b's basis):
    ``dim (4/h^2) sin^2(pi h / 2)``."""
    return dim * 4.0 * n * n * math.sin(math.pi / (2.0 * n)) ** 2


def diffusion_error_bound(prob: dict, u):
    """O2c: rigorous bound on ``||u - u*||_2 / ||u*||_2`` for ``-div(a grad u) + b . grad u + c u
    = f`` with constant ``b`` and ``c >= 0``.

    O1's diffusion part is ``sum_faces a_pq (e_p - e_q)(e_p - e_q)^T / h^2`` (boundary faces keep
    only ``e_p e_p^T``) plus ``diag(c)``; every term is positive semidefinite and ``a_pq`` is at
    least ``a_min`` (the smallest nodal value), so it is ``>= a_min L`` with ``L`` the
    constant-coefficient Laplacian.  The central-difference convection part with constant ``b``
    couples interior neighbours by ``+-b_d / (2h)``, a skew-symmetric matrix, so ``x^T A x`` sees
    only the diffusion part and ``||A x|| ||x|| >= x^T A x >= a_min lambda_min(L) ||x||^2``.
    Hence ``||u - u*|| = ||A^{-1} r|| <= ||r|| / (a_min lambda_min(L))``, with ``r = b - A u``
    evaluated in FP64 and enlarged by the rounding bound of that evaluation (at most 8 terms per
    row: ``gamma_8 (|b| + |A| |u|)``).
    """
    if prob.get("c") is not None and np.min(prob["c"]) < 0:
        raise ValueError("the bound needs c >= 0")
    A, b = assemble(prob)
    u = np.asarray(u, dtype=np.float64).ravel()
    r = b - A @ u
    eps = np.finfo(np.float64).eps
    gam = 8 * eps / (1 - 8 * eps)
    rnorm = np.linalg.norm(r) + gam * np.linalg.norm(np.abs(b) + abs(A) @ np.abs(u))
    lam = float(np.min(prob["a"])) * laplacian_lambda_min(prob["dim"], prob["n"])
    err = rnorm / lam
    un = np.linalg.norm(u)
    return err / (un - err) if un > err else math.inf


# ---------------------------------------------------------------------------------------
# Slab geometry (Sec. 2, Fig. 2.1; index sets I_j, C_j, J_{j,j'} of Sec. 2.5)
# ---------------------------------------------------------------------------------------

@dataclass
class SlabGeometry:
    dim: int
    n: int
    w: int
    nds: int
    ngamma: int
    I: list = field(default_factory=list)        # global interior indices of Psi_j
    C: list = field(default_factory=list)        # positions (within I_j) of Gamma_j
    Jprev: list = field(default_factory=list)    # global indices of Gamma_{j-1} (or None)
    Jnext: list = field(default_factory=list)    # global indices of Gamma_{j+1} (or None)
    G: list = field(default_factory=list)        # global indices of Gamma_j


def slab_geometry(dim: int, n: int, w: int) -> SlabGeometry:
    """Index sets of the ``N_ds = n/w - 1`` overlapping double slabs (slabs normal to x)."""
    if n % w != 0 or n // w < 2:
        raise ValueError("slab width must divide n and give at least two slabs")
    nds = n // w - 1
    rest = (n - 1) ** (dim - 1)
    geo = SlabGeometry(dim=dim, n=n, w=w, nds=nds, ngamma=rest)
    plane = lambda i: (i - 1) * rest + np.arange(rest)   # global indices of x-plane i
    for j in range(1, nds + 1):
        lo, hi = (j - 1) * w + 1, (j + 1) * w - 1
        I = np.concatenate([plane(i) for i in range(lo, hi + 1)])
        geo.I.append(I)
        geo.C.append((j * w - lo) * rest + np.arange(rest))
        geo.G.append(plane(j * w))
        geo.Jprev.append(plane((j - 1) * w) if j >= 2 else None)
        geo.Jnext.append(plane((j + 1) * w) if j <= nds - 1 else None)
    return geo


def factor_local(A, geo: SlabGeometry):
    """Sparse LU of every local operator ``A_j(I_j, I_j)`` (Alg. 2, factorization step).

    The FD discretization is compatible (Sec. 4), so ``A_j(I_j, I_j)`` is the restriction of
    the global matrix to the double-slab interior.
    """
    A = sp.csr_matrix(A)
    return [spla.splu(sp.csc_matrix(A[I][:, I])) for I in geo.I]


# ---------------------------------------------------------------------------------------
# O3  Local solution-transfer operators and equivalent loads (Sec. 2.2; Alg. 1)
# ---------------------------------------------------------------------------------------

def transfer_blocks(A, geo: SlabGeometry, facs, slabs=None):
    """Dense ``S_{j,j-1}`` and ``S_{j,j+1}`` for each double slab (``None`` at the ends).

    ``S_{j,j'} = -R_{C_j} A_j(I_j,I_j)^{-1} A(I_j, J_{j,j'})`` (Sec. 2.2, Eq. (defS)), evaluated
    with the identity as test matrix (every column of ``A(I_j, J_{j,j'})`` solved).
    """
    A = sp.csr_matrix(A)
    Sp, Sn = [], []
    for j in (range(geo.nds) if slabs is None else slabs):
        I, C, lu = geo.I[j], geo.C[j], facs[j]
        out = []
        for J in (geo.Jprev[j], geo.Jnext[j]):
            if J is None:
                out.append(None)
                continue
            rhs = A[I][:, J].toarray()
            out.append(-lu.solve(rhs)[C, :])
        Sp.append(out[0]); Sn.append(out[1])
    return Sp, Sn


def poisson_transfer_apply(dim: int, n: int, w: int, x):
    """O3b: ``S_{j,j+1} x`` (equal to ``S_{j,j-1} x``) for ``a = 1``, ``b = 0``, ``c = 0``.

    Expand the Dirichlet data on the neighbouring interface in the transverse sine modes
    (``dim - 1`` axes, O2b's basis) with eigenvalue sums ``mu`` (in units of ``1/h^2``).  Across
    the double slab (x = 0 .. 2w with zero data on the far interface) each mode solves the
    three-term recurrence ``u_{i-1} - (2 + mu) u_i + u_{i+1} = 0``, i.e. ``u_i = sinh(i theta) /
    sinh(2 w theta)`` with ``cosh theta = 1 + mu / 2``; its value at the central plane ``i = w`` is
    ``1 / (2 cosh(w theta))``.  ``x`` holds ``n_Gamma = (n-1)^(dim-1)`` values in interface order.
    """
    k = np.arange(1, n)
    mu1 = 4.0 * np.sin(np.pi * k / (2.0 * n)) ** 2
    mu = np.zeros((n - 1,) * (dim - 1))
    for d in range(dim - 1):
        shape = [1] * (dim - 1)
        shape[d] = n - 1
        mu = mu + mu1.reshape(shape)
    theta = np.arccosh(1.0 + mu / 2.0)
    s = 1.0 / (2.0 * np.cosh(w * theta))
    xh = sfft.dstn(np.asarray(x, dtype=np.float64).reshape((n - 1,) * (dim - 1)), type=1)
    return sfft.idstn(s * xh, type=1).ravel()


def equivalent_load(b, geo: SlabGeometry, facs):
    """``fhat_j = R_{C_j} A_j(I_j,I_j)^{-1} b(I_j)`` (Sec. 2.2, Eq. (equilib1), Fig. genBC).

    ``b`` already carries the physical Dirichlet data; the neighbouring interfaces get zero
    data because their columns are simply not included.
    """
    return [facs[j].solve(np.asarray(b)[geo.I[j]])[geo.C[j]] for j in range(geo.nds)]


# ---------------------------------------------------------------------------------------
# O4  Equilibrium system (Sec. 1 Eq. (modelS); Sec. 2.2 Eq. (equilib2)) and its solvers
# ---------------------------------------------------------------------------------------

def interface_matrix(Sp, Sn, m):
    """Dense ``I - K``: identity diagonal, ``-S_{j,j-1}`` and ``-S_{j,j+1}`` off it (Sec. 1, Eq. (modelS)).

    ``m`` is the number of points per interface.
    """
    nds = len(Sp)
    M = np.eye(nds * m)
    for j in range(nds):
        if Sp[j] is not None:
            M[j * m:(j + 1) * m, (j - 1) * m:j * m] = -Sp[j]
        if Sn[j] is not None:
            M[j * m:(j + 1) * m, (j + 1) * m:(j + 2) * m] = -Sn[j]
    return M


def apply_interface(Sp, Sn, x):
    """``y = (I - K) x`` block row by block row (Sec. 2.2, Eq. (equilib2))."""
    nds = len(Sp)
    m = x.size // nds
    X = x.reshape(nds, m)
    Y = X.copy()
    for j in range(nds):
        if Sp[j] is not None:
            Y[j] -= Sp[j] @ X[j - 1]
        if Sn[j] is not None:
            Y[j] -= Sn[j] @ X[j + 1]
    return Y.ravel()


def block_thomas(Sp, Sn, fhat):
    """Exact solve of the block-tridiagonal, identity-diagonal system by block elimination."""
    nds = len(fhat)
    m = fhat[0].size
    Dm = [None] * nds
    r = [None] * nds
    Dm[0] = np.eye(m)
    r[0] = np.array(fhat[0], dtype=np.float64)
    for j in range(1, nds):
        # row j: -Sp[j] u_{j-1} + u_j - Sn[j] u_{j+1} = fhat_j
        L = -Sp[j]
        Uprev = -Sn[j - 1]
        W = sla.solve(Dm[j - 1], np.column_stack([Uprev, r[j - 1]]))
        Dm[j] = np.eye(m) - L @ W[:, :m]
        r[j] = fhat[j] - L @ W[:, m]
    u = [None] * nds
    u[-1] = sla.solve(Dm[-1], r[-1])
    for j in range(nds - 2, -1, -1):
        u[j] = sla.solve(Dm[j], r[j] + Sn[j] @ u[j + 1])
    return np.concatenate(u)


def gmres(matvec, b, tol=1e-8, maxit=None):
    """Unrestarted GMRES, ``x0 = 0``, stop when ``||b - A x||_2 <= tol ||b||_2`` (Sec. 5.2).

    Arnoldi uses classical Gram-Schmidt applied twice; the least-squares problem is reduced
    by Givens rotations.  Returns ``(x, iterations, relative residual history)``.
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    maxit = n if maxit is None else maxit
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros(n), 0, [0.0]
    V = np.zeros((maxit + 1, n))
    H = np.zeros((maxit + 1, maxit))
    cs, sn = np.zeros(maxit), np.zeros(maxit)
    gvec = np.zeros(maxit + 1)
    gvec[0] = beta
    V[0] = b / beta
    hist = [1.0]
    k = 0
    for k in range(1, maxit + 1):
        wv = matvec(V[k - 1])
        h1 = V[:k] @ wv
        wv = wv - V[:k].T @ h1
        h2 = V[:k] @ wv
        wv = wv - V[:k].T @ h2
        hcol = h1 + h2
        hn = np.linalg.norm(wv)
        H[:k, k - 1] = hcol
        H[k, k - 1] = hn
        for i in range(k - 1):
            t = cs[i] * H[i, k - 1] + sn[i] * H[i + 1, k - 1]
            H[i + 1, k - 1] = -sn[i] * H[i, k - 1] + cs[i] * H[i + 1, k - 1]
            H[i, k - 1] = t
        den = math.hypot(H[k - 1, k - 1], H[k, k - 1])
        cs[k - 1] = H[k - 1, k - 1] / den
        sn[k - 1] = H[k, k - 1] / den
        H[k - 1, k - 1] = den
        H[k, k - 1] = 0.0
        gvec[k] = -sn[k - 1] * gvec[k - 1]
        gvec[k - 1] = cs[k - 1] * gvec[k - 1]
        hist.append(abs(gvec[k]) / beta)
        if hist[-1] <= tol or hn == 0.0:
            break
        V[k] = wv / hn
    y = sla.solve_triangular(H[:k, :k], gvec[:k])
    return V[:k].T @ y, k, hist


# ---------------------------------------------------------------------------------------
# O5  Volume reconstruction from interface traces (Sec. 3.1, proof of the Fredholm proposition)
# ---------------------------------------------------------------------------------------

def reconstruct(A, b, geo: SlabGeometry, facs, uG):
    """Volume solution from traces: each double slab solved with Dirichlet data on its sides.

    Slab ``j`` supplies the x-planes ``(j-1)w+1 .. j w`` (its left half and ``Gamma_j``); the
    last slab also supplies its right half.
    """
    A = sp.csr_matrix(A)
    nds, w, rest = geo.nds, geo.w, geo.ngamma
    U = uG.reshape(nds, rest)
    u = np.zeros(A.shape[0])
    for j in range(nds):
        I = geo.I[j]
        rhs = np.asarray(b)[I].copy()
        if geo.Jprev[j] is not None:
            rhs -= A[I][:, geo.Jprev[j]] @ U[j - 1]
        if geo.Jnext[j] is not None:
            rhs -= A[I][:, geo.Jnext[j]] @ U[j + 1]
        x = facs[j].solve(rhs)
        keep = w * rest if j < nds - 1 else len(I)
        u[I[:keep]] = x[:keep]
    return u


def dd_solve(prob: dict, use_gmres=False, tol=1e-12):
    """Full DD solve (O1, O3, O4, O5; Alg. 1 and Alg. 2 with the identity as test matrix).  Returns ``(u, uG, info)``."""
    A, b = assemble(prob)
    geo = slab_geometry(prob["dim"], prob["n"], prob["w"])
    facs = factor_local(A, geo)
    Sp, Sn = transfer_blocks(A, geo, facs)
    fh = equivalent_load(b, geo, facs)
    info = {}
    if use_gmres:
        uG, its, hist = gmres(lambda x: apply_interface(Sp, Sn, x), np.concatenate(fh), tol=tol)
        info.update(iters=its, hist=hist)
    else:
        uG = block_thomas(Sp, Sn, fh)
    u = reconstruct(A, b, geo, facs, uG)
    return u, uG, info


# ---------------------------------------------------------------------------------------
# O6  Weak-admissibility hierarchical (HODLR) compression (Sec. 2.4)
# ---------------------------------------------------------------------------------------

def hodlr_levels(ng: int, leaf: int) -> int:
    """Tree depth ``L``: the smallest ``L`` with ``ceil(ng / 2^L) <= leaf``."""
    L = 0
    while -(-ng // (1 << L)) > leaf:
        L += 1
    return L


def hodlr_node(ng: int, level: int, t: int):
    """Index range ``[lo, hi)`` of node ``t`` at ``level`` of the balanced bisection tree."""
    return (t * ng) >> level, ((t + 1) * ng) >> level


def hodlr_compress(S, tol: float, leaf: int, norm2=None, kmax=None):
    """HODLR of a dense block by truncated SVD of every off-diagonal block.

    Shared cluster tree for rows and columns (the interfaces are discretized isomorphically,
    Sec. 2.4).  Rank ``r = min{r : sigma_{r+1} <= tol * ||S||_2}`` per block.  Returns a dict
    with ``levels`` (per level a list of ``(U, V)`` pairs for the blocks
    ``S[tau_{2t}, tau_{2t+1}]`` and ``S[tau_{2t+1}, tau_{2t}]``, ``S_block ~ U @ V.T``) and
    ``leaves`` (dense diagonal blocks).
    """
    S = np.asarray(S, dtype=np.float64)
    ng = S.shape[0]
    L = hodlr_levels(ng, leaf)
    if norm2 is None:
        norm2 = np.linalg.norm(S, 2)
    thr = tol * norm2
    levels = []
    for lev in range(1, L + 1):
        blocks = []
        for t in range(1 << (lev - 1)):
            lo1, hi1 = hodlr_node(ng, lev, 2 * t)
            lo2, hi2 = hodlr_node(ng, lev, 2 * t + 1)
            for (r0, r1, c0, c1) in ((lo1, hi1, lo2, hi2), (lo2, hi2, lo1, hi1)):
                B = S[r0:r1, c0:c1]
                U, s, Vt = np.linalg.svd(B, full_matrices=False)
                r = int(np.sum(s > thr))
                if kmax is not None:
                    r = min(r, kmax)
                blocks.append((U[:, :r] * s[:r], Vt[:r].T.copy()))
        levels.append(blocks)
    leaves = [S[slice(*hodlr_node(ng, L, t)), slice(*hodlr_node(ng, L, t))].copy()
              for t in range(1 << L)]
    return dict(ng=ng, L=L, levels=levels, leaves=leaves, thr=thr)


def hodlr_dense(H):
    """Expand a HODLR representation back into a dense matrix."""
    ng, L = H["ng"], H["L"]
    S = np.zeros((ng, ng))
    for lev, blocks in enumerate(H["levels"], start=1):
        for t in range(1 << (lev - 1)):
            lo1, hi1 = hodlr_node(ng, lev, 2 * t)
            lo2, hi2 = hodlr_node(ng, lev, 2 * t + 1)
            U, V = blocks[2 * t]
            S[lo1:hi1, lo2:hi2] = U @ V.T
            U, V = blocks[2 * t + 1]
            S[lo2:hi2, lo1:hi1] = U @ V.T
    for t, D in enumerate(H["leaves"]):
        lo, hi = hodlr_node(ng, L, t)
        S[lo:hi, lo:hi] = D
    return S


def hodlr_apply(H, x):
    """``y = S_H x`` using the factors (never forms the dense matrix)."""
    ng, L = H["ng"], H["L"]
    y = np.zeros(ng)
    for lev, blocks in enumerate(H["levels"], start=1):
        for t in range(1 << (lev - 1)):
            lo1, hi1 = hodlr_node(ng, lev, 2 * t)
            lo2, hi2 = hodlr_node(ng, lev, 2 * t + 1)
            U, V = blocks[2 * t]
            y[lo1:hi1] += U @ (V.T @ x[lo2:hi2])
            U, V = blocks[2 * t + 1]
            y[lo2:hi2] += U @ (V.T @ x[lo1:hi1])
    for t, D in enumerate(H["leaves"]):
        lo, hi = hodlr_node(ng, L, t)
        y[lo:hi] += D @ x[lo:hi]
    return y


# ---------------------------------------------------------------------------------------
# O9  Nested-basis HBS compression from random samples (Sec. 2.4; Alg. 1)
# ---------------------------------------------------------------------------------------

def _null_basis(Om):
    """Orthonormal basis of the null space of ``Om`` (``n x s``, ``n < s``): the trailing
    ``s - n`` columns of the full orthogonal factor of the Householder QR of ``Om^T``."""
    Q, _ = sla.qr(Om.T, mode="full")
    return Q[:, Om.shape[0]:]


def _col(X, k: int):
    """``col(X, k)``: the leading ``k`` columns of the orthogonal factor of the column-pivoted
    Householder QR of ``X`` (an orthonormal basis of ``k`` columns spanning most of range(X))."""
    Q, _, _ = sla.qr(X, mode="economic", pivoting=True)
    return Q[:, :k]


def hbs_compress(Y, Z, Om, Psi, k: int, leaf: int):
    """HBS (nested bases, weak admissibility) of ``S`` from ``Y = S Om`` and ``Z = S^T Psi``.

    ``Om`` and ``Psi`` are ``ng x s`` Gaussian test matrices; the paper draws ``s = 3 k + q``
    samples (Alg. 1).  The cluster tree is the balanced bisection of ``hodlr_node`` (shared by
    rows and columns, Sec. 2.4).  Level by level from the leaves, every node ``tau`` with row set
    of size ``n`` and samples ``(Y_t, Z_t, Om_t, Psi_t)`` (``n x s``) gets

    * ``U = col(Y_t P, k)``, ``P`` an orthonormal basis of null(``Om_t``): ``Y_t P`` samples the
      off-diagonal block row ``S(tau, tau^c)`` alone, since ``S(tau, tau) Om_t P = 0``;
      ``V = col(Z_t P', k)`` likewise for the block column;
    * ``D = (I - U U^T) Y_t Om_t^+ + U U^T ((I - V V^T) Z_t Psi_t^+)^T``, the part of the
      diagonal block that the bases do not carry (``S_tt - U U^T S_tt V V^T`` when the
      off-diagonal blocks have rank ``<= k``);
    * the samples of the reduced matrix ``U^T (S - D) V`` for the next level up:
      ``V^T Om_t``, ``U^T Psi_t``, ``U^T (Y_t - D Om_t)`` and ``V^T (Z_t - D^T Psi_t)``, a
      parent's row set being its two children's ``k`` reduced rows, first child first.

    The root keeps the reduced matrix itself, ``D_0 = Y_0 Om_0^+`` (``2k x 2k``; the whole block
    when the tree has one level).  ``S = U_L (... U_1 D_0 V_1^T + D_1 ...) V_L^T + D_L`` with
    block-diagonal ``U_l, V_l, D_l``: storage and apply cost are ``O(k N)``.
    """
    Y, Z, Om, Psi = (np.asarray(a, dtype=np.float64) for a in (Y, Z, Om, Psi))
    ng, s = Y.shape
    L = hodlr_levels(ng, leaf)
    cur = []
    for t in range(1 << L):
        lo, hi = hodlr_node(ng, L, t)
        cur.append((Y[lo:hi], Z[lo:hi], Om[lo:hi], Psi[lo:hi]))
    levels = [None] * (L + 1)
    for lev in range(L, 0, -1):
        nodes, red = [], []
        for (Yt, Zt, Ot, Pt) in cur:
            if Yt.shape[0] + k > s:
                raise ValueError("HBS: a node's row set plus k exceeds the sample count")
            U = _col(Yt @ _null_basis(Ot), k)
            V = _col(Zt @ _null_basis(Pt), k)
            X1 = Yt @ np.linalg.pinv(Ot)
            X2 = Zt @ np.linalg.pinv(Pt)
            D = X1 - U @ (U.T @ X1) + U @ (U.T @ (X2.T - (X2.T @ V) @ V.T))
            nodes.append((U, V, D))
            red.append((U.T @ (Yt - D @ Ot), V.T @ (Zt - D.T @ Pt), V.T @ Ot, U.T @ Pt))
        levels[lev] = nodes
        cur = [tuple(np.vstack((a, b)) for a, b in zip(red[2 * t], red[2 * t + 1]))
               for t in range(len(red) // 2)]
    Y0, _, O0, _ = cur[0]
    if Y0.shape[0] > s:
        raise ValueError("HBS: the root's row set exceeds the sample count")
    levels[0] = Y0 @ np.linalg.pinv(O0)
    return dict(ng=ng, L=L, k=k, levels=levels)


def hbs_dense(H):
    """Expand an HBS representation: ``A_0 = D_0``, ``A_l = U_l A_{l-1} V_l^T + D_l``."""
    A = H["levels"][0]
    for lev in range(1, H["L"] + 1):
        nodes = H["levels"][lev]
        A = (sla.block_diag(*[U for U, _, _ in nodes]) @ A
             @ sla.block_diag(*[V for _, V, _ in nodes]).T
             + sla.block_diag(*[D for _, _, D in nodes]))
    return A


def hbs_apply(H, x, transpose: bool = False):
    """``y = S_H x`` (or ``S_H^T x``) by the upward and downward passes over the tree (never
    forms the dense matrix): ``x_t <- V^T x_t`` from the leaves up, ``y_0 = D_0 x_0`` at the
    root, then ``y_t = D x_t + U (parent's y, rows of t)`` back down.  The transpose swaps the
    roles of ``U`` and ``V`` and transposes every ``D``."""
    ng, L, k, lv = H["ng"], H["L"], H["k"], H["levels"]
    x = np.asarray(x, dtype=np.float64)
    xs = [None] * (L + 1)
    xs[L] = [x[slice(*hodlr_node(ng, L, t))] for t in range(1 << L)]
    for lev in range(L, 0, -1):
        red = [(U if transpose else V).T @ xt for (U, V, _), xt in zip(lv[lev], xs[lev])]
        xs[lev - 1] = [np.concatenate((red[2 * t], red[2 * t + 1])) for t in range(len(red) // 2)]
    ys = [(lv[0].T if transpose else lv[0]) @ xs[0][0]]
    for lev in range(1, L + 1):
        nxt = []
        for t, ((U, V, D), xt) in enumerate(zip(lv[lev], xs[lev])):
            slot = ys[t // 2][(t % 2) * k:(t % 2 + 1) * k]
            nxt.append((D.T if transpose else D) @ xt + (V if transpose else U) @ slot)
        ys = nxt
    return np.concatenate(ys)


def hbs_entries(H) -> int:
    """Stored numbers of an HBS representation (leaves: ``n^2 + 2 n k``; inner nodes:
    ``4 k^2 + 4 k^2``; root: ``4 k^2``)."""
    tot = H["levels"][0].size
    for lev in range(1, H["L"] + 1):
        tot += sum(U.size + V.size + D.size for U, V, D in H["levels"][lev])
    return int(tot)


# ---------------------------------------------------------------------------------------
# O7  Discrete adjoint and gradients
# ---------------------------------------------------------------------------------------

def adjoint_solve(A, dLdu):
    """``lambda = A^{-T} dL/du`` (sparse direct solve with the transpose)."""
    lu = spla.splu(sp.csc_matrix(sp.csr_matrix(A).T))
    return lu.solve(np.asarray(dLdu, dtype=np.float64))


def gradients(prob: dict, u, lam):
    """Gradients of ``L(u(f, g, a))`` given ``u`` and ``lambda = A^{-T} dL/du``.

    * ``dL/df_p = lambda_p`` (interior nodes).
    * ``dL/dg_q = sum_{p ~ q} lambda_p * (a_pq/h^2 - s b_d/(2h))`` over interior neighbours
      ``p`` of boundary node ``q`` (``q = p + s e_d``): the derivative of ``b_p``.
    * ``dL/da_pq = -(lambda_p - lambda_q)(u_p - u_q)/h^2`` per face, with ``u_q = g_q`` and
      ``lambda_q = 0`` on boundary nodes; nodal ``dL/da_node = 1/2 sum_{faces at node}``.
    Returns ``(dLdf, dLdg, dLda)`` shaped like ``f``, ``g`` and ``a``.
    """
    dim, n = prob["dim"], prob["n"]
    a, g = prob["a"], prob["g"]
    bconv = prob.get("b") or (0.0,) * dim
    h = 1.0 / n
    shape_int = (n - 1,) * dim
    lam_full = np.zeros((n + 1,) * dim)
    lam_full[_interior(dim, n)] = np.asarray(lam).reshape(shape_int)
    u_full = np.array(g, dtype=np.float64).copy()
    u_full[_interior(dim, n)] = np.asarray(u).reshape(shape_int)
    dLdf = lam_full[_interior(dim, n)].copy()
    dLdg = np.zeros((n + 1,) * dim)
    dLda = np.zeros((n + 1,) * dim)
    for d in range(dim):
        # faces between node (.., i, ..) and (.., i+1, ..) along axis d, all nodes
        lo = [slice(None)] * dim; hi = [slice(None)] * dim
        lo[d] = slice(0, n); hi[d] = slice(1, n + 1)
        lo, hi = tuple(lo), tuple(hi)
        # a face contributes only if at least one endpoint is interior and the face lies in
        # the interior of the other axes
        mask = np.zeros(lam_full[lo].shape, dtype=bool)
        sl_other = [slice(None)] * dim
        for e in range(dim):
            if e != d:
                sl_other[e] = slice(1, n)
        m_other = np.zeros_like(mask)
        m_other[tuple(sl_other)] = True
        idx_d = np.arange(n).reshape([-1 if e == d else 1 for e in range(dim)])
        endpoint_interior = (idx_d >= 1) | (idx_d + 1 <= n - 1)
        mask = m_other & endpoint_interior
        dface = -(lam_full[lo] - lam_full[hi]) * (u_full[lo] - u_full[hi]) / h ** 2
        dface = np.where(mask, dface, 0.0)
        dLda[lo] += 0.5 * dface
        dLda[hi] += 0.5 * dface
        # boundary data: q = p + s e_d with p interior, q boundary
        af = 0.5 * (a[lo] + a[hi])
        # q = hi endpoint (s = +1), p = lo endpoint interior
        idx_hi = idx_d + 1
        p_int = (idx_d >= 1) & (idx_d <= n - 1)
        q_bnd_hi = (idx_hi == n)
        contrib_hi = np.where(m_other & p_int & q_bnd_hi,
                              lam_full[lo] * (af / h ** 2 - bconv[d] / (2 * h)), 0.0)
        dLdg[hi] += contrib_hi
        # q = lo endpoint (s = -1), p = hi endpoint interior
        p_int2 = (idx_hi >= 1) & (idx_hi <= n - 1)
        q_bnd_lo = (idx_d == 0)
        contrib_lo = np.where(m_other & p_int2 & q_bnd_lo,
                              lam_full[hi] * (af / h ** 2 + bconv[d] / (2 * h)), 0.0)
        dLdg[lo] += contrib_lo
    return dLdf, dLdg, dLda


def loss_and_gradients(prob: dict, u_obs):
    """``L = 1/2 ||u - u_obs||^2`` and its gradients w.r.t. ``f``, ``g``, nodal ``a`` (O7)."""
    A, b = assemble(prob)
    u = global_solve(A, b)
    r = u - np.asarray(u_obs).ravel()
    lam = adjoint_solve(A, r)
    L = 0.5 * float(r @ r)
    return (L,) + gradients(prob, u, lam) + (u, lam)


# ---------------------------------------------------------------------------------------
# O8  IMEX backward-Euler marching (Sec. 6, Example 1, Eq. (convdiff))
# ---------------------------------------------------------------------------------------

def imex_rhs(dim: int, n: int, u, vel, dt: float):
    """Explicit right-hand side of one step: ``U_n/dt - v . grad_h U_n`` on the interior nodes.

    ``u``: interior values of ``U_n`` (``(n-1)^dim``, C order); ``vel``: ``dim`` nodal arrays
    (``(n+1)^dim``) of the velocity components.  ``grad_h`` is the central difference
    ``(U_{p+e_d} - U_{p-e_d}) / (2h)``; boundary nodes carry ``U = 0``.
    """
    h = 1.0 / n
    U = np.zeros((n + 1,) * dim)
    U[_interior(dim, n)] = np.asarray(u, dtype=np.float64).reshape((n - 1,) * dim)
    f = U[_interior(dim, n)] / dt
    for d in range(dim):
        grad = (U[_shifted(dim, n, d, +1)] - U[_shifted(dim, n, d, -1)]) / (2.0 * h)
        f = f - np.asarray(vel[d])[_interior(dim, n)] * grad
    return f.ravel()


def imex_march(prob: dict, u0, vel, dt: float, nsteps: int):
    """``nsteps`` backward-Euler steps ``A U_{n+1} = U_n/dt - v . grad_h U_n``.

    ``A`` is O1's operator of ``prob`` (its ``a``, ``b``, ``c``: the example's screened operator
    has ``a = D``, ``b = 0``, ``c = 1/dt``) with zero Dirichlet data, factored once by SuperLU and
    reused by every step.  Returns the interior values of ``U_nsteps``.
    """
    dim, n = prob["dim"], prob["n"]
    q = dict(prob)
    q["f"] = np.zeros((n - 1,) * dim)
    q["g"] = np.zeros((n + 1,) * dim)
    A, _ = assemble(q)
    lu = spla.splu(sp.csc_matrix(A))
    u = np.asarray(u0, dtype=np.float64).ravel()
    for _ in range(nsteps):
        u = lu.solve(imex_rhs(dim, n, u, vel, dt))
    return u
