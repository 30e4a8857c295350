"""Seeded synthetic problem inputs shared by the oracle, the tests and the benchmark.

This module only *generates data*: grids, coefficient fields, loads and boundary data.
It holds none of the solver's arithmetic (no discretization, no local solves, no interface
system), so the FP64 CPU oracle and the CUDA path can both draw their inputs from it
without sharing any method code.

Conventions (both sides rely on them):

* ``n`` cells per side, mesh width ``h = 1/n``, nodes ``x_i = i h`` for ``i = 0..n``.
* Nodal fields (``a``, ``c``, ``g``) have shape ``(n+1,)*dim``; interior fields (``f``,
  ``u``) have shape ``(n-1,)*dim``.  Axis 0 is ``x`` (the slab-normal axis) and is the
  slowest-varying index in C order.
* The PDE is ``-div(a grad u) + b . grad u + c u = f`` in the unit square/cube with
  ``u = g`` on the boundary (Eq. 1.1 of the paper: ``f`` is the load, ``g`` the Dirichlet
  data).
* Seeds follow ``1000 * workload_id + field_id`` with field ids 0 = load, 1 = coefficient
  modes, 2 = observation noise, 3 = second coefficient perturbation.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "node_coords", "fourier_log_field", "uniform_load", "quadratic_boundary",
    "helmholtz_reaction", "gaussian_source", "make_problem", "batch_specs",
    "WORKLOADS",
]


def node_coords(dim: int, n: int):
    """Coordinates of all ``(n+1)^dim`` grid nodes, one array per axis (``ij`` indexing)."""
    x = np.arange(n + 1, dtype=np.float64) / n
    return np.meshgrid(*([x] * dim), indexing="ij")


def _mode_table(dim: int, kmax: float):
    ks = []
    r = int(math.floor(kmax))
    for k in itertools.product(range(-r, r + 1), repeat=dim):
        nk = math.sqrt(sum(t * t for t in k))
        if 1.0 <= nk <= kmax:
            ks.append(k)
    return np.array(ks, dtype=np.float64)


def fourier_log_field(dim: int, n: int, seed: int, n_modes: int = 8, amp: float = 0.3,
                      kmax: float = 4.0) -> np.ndarray:
    """Nodal ``a = exp(sum_m amp * cos(2 pi k_m . x + theta_m))``.

    ``k_m`` are drawn uniformly (with replacement) from the integer vectors with
    ``1 <= |k|_2 <= kmax``; ``theta_m ~ U[0, 2 pi)``.  Each mode has amplitude ``amp``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    table = _mode_table(dim, kmax)
    pick = rng.integers(0, len(table), size=n_modes)
    theta = rng.uniform(0.0, 2.0 * math.pi, size=n_modes)
    X = node_coords(dim, n)
    phi = np.zeros_like(X[0])
    for m in range(n_modes):
        k = table[pick[m]]
        arg = sum(k[d] * X[d] for d in range(dim))
        phi += amp * np.cos(2.0 * math.pi * arg + theta[m])
    return np.exp(phi)


def uniform_load(dim: int, n: int, seed: int) -> np.ndarray:
    """Interior load ``f ~ U(-1, 1)`` i.i.d., shape ``(n-1,)*dim``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-1.0, 1.0, size=(n - 1,) * dim)


def quadratic_boundary(dim: int, n: int) -> np.ndarray:
    """Nodal harmonic quadratic: ``x^2 - y^2 + x y`` (2D) or ``x^2 + y^2 - 2 z^2 + x y`` (3D)."""
    X = node_coords(dim, n)
    if dim == 2:
        return X[0] ** 2 - X[1] ** 2 + X[0] * X[1]
    return X[0] ** 2 + X[1] ** 2 - 2.0 * X[2] ** 2 + X[0] * X[1]


def helmholtz_reaction(dim: int, n: int, kappa: float, center=None, width: float = 25.0):
    """Nodal reaction ``c = -kappa^2 (1 - 0.5 exp(-width |x - center|^2))``."""
    X = node_coords(dim, n)
    if center is None:
        center = (0.5,) * dim
    r2 = sum((X[d] - center[d]) ** 2 for d in range(dim))
    return -(kappa ** 2) * (1.0 - 0.5 * np.exp(-width * r2))


def gaussian_source(dim: int, n: int, x0=None, sigma: float = 0.01) -> np.ndarray:
    """Interior load ``exp(-|x - x0|^2 / (2 sigma^2))``."""
    if x0 is None:
        x0 = (0.25,) + (0.5,) * (dim - 1)
    X = node_coords(dim, n)
    r2 = sum((X[d] - x0[d]) ** 2 for d in range(dim))
    full = np.exp(-r2 / (2.0 * sigma ** 2))
    return full[tuple(slice(1, n) for _ in range(dim))].copy()


# Named workloads: the paper-shaped synthetic problems.  ``n`` and ``w`` may be overridden to
# produce smaller instances of the same family for parity tests.
WORKLOADS = {
    # 2D Poisson, 128 cells, 8 slabs of 16 cells, f ~ U(-1,1), g harmonic quadratic.
    "poisson2d": dict(id=1, dim=2, n=128, w=16, kind="poisson"),
    # 2D nonsymmetric -div(a grad u) + b.grad u = f, 2048 cells, 64 slabs of 32 cells.
    "convdiff2d": dict(id=2, dim=2, n=2048, w=32, kind="convdiff", b=(20.0, 10.0)),
    # 2D Helmholtz with a Gaussian bump in the wavenumber, 4096 cells, 128 slabs of 32.
    "helmholtz2d": dict(id=3, dim=2, n=4096, w=32, kind="helmholtz", kappa=200.0),
    # 3D variable-coefficient diffusion, 128 cells, 8 slabs of 16.
    "vardiff3d": dict(id=4, dim=3, n=128, w=16, kind="vardiff"),
}


def make_problem(name: str, n: int | None = None, w: int | None = None, **overrides) -> dict:
    """Build the inputs of a named workload (optionally at a reduced size).

    Returns a dict with keys ``dim, n, w, a, b, c, f, g`` (NumPy FP64 arrays; ``b`` a tuple
    of constants, ``c`` ``None`` when absent) plus ``name``.
    """
    spec = dict(WORKLOADS[name])
    spec.update(overrides)
    dim = spec["dim"]
    n = spec["n"] if n is None else n
    w = spec["w"] if w is None else w
    cid = spec["id"]
    kind = spec["kind"]
    b = tuple(spec.get("b", (0.0,) * dim))
    c = None
    if kind == "poisson":
        a = np.ones((n + 1,) * dim)
        f = uniform_load(dim, n, 1000 * cid + 0)
        g = quadratic_boundary(dim, n)
    elif kind in ("convdiff", "vardiff"):
        a = fourier_log_field(dim, n, 1000 * cid + 1)
        f = uniform_load(dim, n, 1000 * cid + 0)
        g = quadratic_boundary(dim, n)
    elif kind == "helmholtz":
        a = np.ones((n + 1,) * dim)
        c = helmholtz_reaction(dim, n, spec["kappa"])
        f = gaussian_source(dim, n)
        g = np.zeros((n + 1,) * dim)
    else:  # pragma: no cover - guarded by WORKLOADS
        raise ValueError(kind)
    if spec.get("const_a"):
        a = np.ones((n + 1,) * dim)
    return dict(name=name, dim=dim, n=n, w=w, a=a, b=b, c=c, f=f, g=g)


def batch_specs(count: int = 64, seed0: int = 5000, wmax: int | None = None):
    """Uneven batch of independent 2D diffusion problems.

    Problem ``i``: ``n_i = 64 * m_i`` with ``m_i ~ U{4..16}`` (256..1024 cells) and a slab
    count drawn from ``{8, 16, 32}`` (slab width ``n_i / slabs``, 8 to 128 cells); seed
    ``seed0 + i``.  ``wmax`` optionally restricts the draw to slab counts whose width is at most
    ``wmax`` cells.  Returns a list of dicts with ``n, w, seed``.
    """
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(seed0 + i))
        m = int(rng.integers(4, 17))
        n = 64 * m
        choices = [s for s in (8, 16, 32) if wmax is None or n // s <= wmax]
        slabs = int(choices[int(rng.integers(0, len(choices)))])
        out.append(dict(n=n, w=n // slabs, seed=seed0 + i))
    return out


def batch_problem(spec: dict) -> dict:
    """Inputs of one problem of the uneven batch (2D ``-div(a grad u) = f``)."""
    n, w, seed = spec["n"], spec["w"], spec["seed"]
    a = fourier_log_field(2, n, seed * 10 + 1)
    f = uniform_load(2, n, seed * 10 + 0)
    g = quadratic_boundary(2, n)
    return dict(name=f"batch{seed}", dim=2, n=n, w=w, a=a, b=(0.0, 0.0), c=None, f=f, g=g)


def march_problem(dim: int = 2, n: int = 128, w: int = 16, dt: float = 6.94e-3) -> dict:
    """Inputs of the time-marching workload (the convection-diffusion example of Sec. 6,
    Example 1, on the unit square or cube with Dirichlet sides): diffusion
    ``D = D0 (1 + eps (s_y (2y - 1) + s_x cos(2 pi x)))`` with ``D0 = 0.1, eps = 0.3, s_y = 1,
    s_x = 0.5``, velocity ``v = (-2 y (1 - y), 0[, 0])``, time step ``dt`` (the example's
    6.94e-3) and a smooth bump as initial state (Gaussian of width 0.1 at the centre, scaled to
    vanish on the boundary).  Returns the problem dict (``a = D``, ``b = 0``, ``c = 1/dt``, ``f``
    and ``g`` zero) plus ``vel`` (``dim`` nodal arrays), ``u0`` (interior) and ``dt``."""
    x = np.linspace(0.0, 1.0, n + 1)
    grids = np.meshgrid(*([x] * dim), indexing="ij")
    X, Y = grids[0], grids[1]
    D = 0.1 * (1.0 + 0.3 * ((2.0 * Y - 1.0) + 0.5 * np.cos(2.0 * np.pi * X)))
    vel = [-2.0 * Y * (1.0 - Y)] + [np.zeros_like(X) for _ in range(dim - 1)]
    r2 = sum((G - 0.5) ** 2 for G in grids)
    cut = np.ones_like(X)
    for G in grids:
        cut = cut * (4.0 * G * (1.0 - G))
    bump = np.exp(-r2 / (2.0 * 0.1 ** 2)) * cut
    inner = tuple(slice(1, n) for _ in range(dim))
    return dict(name=f"march{dim}d", dim=dim, n=n, w=w, a=D, b=(0.0,) * dim,
                c=np.full((n + 1,) * dim, 1.0 / dt), f=np.zeros((n - 1,) * dim),
                g=np.zeros((n + 1,) * dim), vel=vel, u0=bump[inner].copy(), dt=dt)
