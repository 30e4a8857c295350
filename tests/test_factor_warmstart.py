"""The premise of the chunked factorization: the pivot recurrence forgets its start.

Along y the double-slab operator is block tridiagonal, and the forward pivots obey
Sigma_k = D_k - L_k Sigma_{k-1}^{-1} U_{k-1}.  The factorization splits each sweep into chunks
that start W rows early from Sigma = D and are accepted only when the warm-up's last inverse
matches the previous chunk's stored inverse of that row (relative 1e-5 in FP32, 1e-11 in FP64,
with W = 4 w and 10 w).  For the five-point Laplacian (h^2-scaled: D = tridiag(-1, 4, -1) of
size 2w - 1, L = U = -I) the slowest x-mode has eigenvalue mu = 4 sin^2(pi / 4w), and a scalar
pivot sigma = (2 + mu) - 1/sigma contracts towards its fixed point by exp(-2 theta) per row,
cosh(theta) = 1 + mu/2, theta ~ pi / (2 w): a warm start is off by about exp(-pi d / w) after
d rows.  These tests check that rate, that the chosen warm-ups sit inside the verification
tolerances, and that a Helmholtz-type negative reaction close to the slab's lowest eigenvalue
slows the decay enough for the check to reject the chunks, which is why the check and its
sequential fallback exist.
"""
import numpy as np
import pytest


def _slab_block(w, shift=0.0):
    m = 2 * w - 1
    return (np.diag(np.full(m, 4.0 - shift)) - np.diag(np.ones(m - 1), 1)
            - np.diag(np.ones(m - 1), -1))


def _warm_start_errors(w, rows, shift=0.0, k0=None):
    """Relative max-norm distance of warm-started pivot inverses from the exact ones.

    Exact: Sigma_1 = D, Sigma_k = D - Sigma_{k-1}^{-1}.  Warm start at row k0 from Sigma = D.
    Returns err[d-1] for d = 1..rows rows after the start.
    """
    D = _slab_block(w, shift)
    k0 = 3 * w if k0 is None else k0
    S = D.copy()
    exact = [S]
    for _ in range(k0 + rows):
        S = D - np.linalg.inv(S)
        exact.append(S)
    Sw = D.copy()
    errs = []
    for d in range(1, rows + 1):
        Sw = D - np.linalg.inv(Sw)
        Fi, Fw = np.linalg.inv(exact[k0 + d]), np.linalg.inv(Sw)
        errs.append(np.abs(Fw - Fi).max() / np.abs(Fi).max())
    return np.array(errs)


@pytest.mark.parametrize("w", [4, 8, 16, 32])
def test_warm_start_error_decays_like_exp_minus_pi_d_over_w(w):
    err = _warm_start_errors(w, 10 * w)
    d = np.arange(1, 10 * w + 1)
    assert (err <= 0.25 * np.exp(-np.pi * d / w)).all()
    # the warm-ups the factorization uses sit inside its verification tolerances
    assert err[4 * w - 1] <= 1e-5 / 10        # FP32: W = 4 w, check at 1e-5
    assert err[10 * w - 1] <= 1e-11 / 100     # FP64: W = 10 w, check at 1e-11


@pytest.mark.parametrize("w", [8, 16])
def test_helmholtz_shift_slows_the_decay_past_the_check(w):
    """A negative reaction at 95% of the slab's lowest eigenvalue (still definite): the FP32
    warm-up no longer converges within 4 w rows."""
    mu = 4.0 * np.sin(np.pi / (4 * w)) ** 2
    err = _warm_start_errors(w, 10 * w, shift=0.95 * mu)
    assert err[4 * w - 1] > 1e-5              # the check rejects the chunk -> sequential sweeps
    # the decay is still geometric, at the rate of the shifted mode
    theta = np.arccosh(1.0 + 0.05 * mu / 2.0)
    d = np.arange(1, 10 * w + 1)
    assert (err <= 2.0 * np.exp(-2.0 * theta * d)).all()
