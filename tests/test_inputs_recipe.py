"""The seeded input generators follow their stated recipe.

Both the oracle and the CUDA path take their inputs from ``ddst_inputs``; these checks tie
each generator to a property its definition fixes (spectrum, extreme values, harmonicity,
ranges, determinism), independently of how it is coded.
"""
import numpy as np
import pytest

import ddst_inputs as I


@pytest.mark.parametrize("dim,n,seed", [(2, 64, 2001), (2, 64, 2003), (3, 16, 2001), (3, 16, 4001)])
def test_log_coefficient_is_a_sum_of_few_low_cosines(dim, n, seed):
    """log a = sum of 8 cosines of amplitude 0.3 with integer wavevectors, 1 <= |k| <= 4."""
    a = I.fourier_log_field(dim, n, seed=seed)
    assert a.shape == (n + 1,) * dim and (a > 0).all()
    phi = np.log(a)
    assert np.abs(phi).max() <= 8 * 0.3 + 1e-12
    # integer wavevectors make phi periodic on the unit cell: drop the repeated last node
    per = phi[tuple(slice(0, n) for _ in range(dim))]
    assert np.allclose(phi[(n,) + (slice(0, n),) * (dim - 1)], per[0])
    F = np.abs(np.fft.fftn(per)) / per.size
    k = np.meshgrid(*([np.fft.fftfreq(n, 1.0 / n)] * dim), indexing="ij")
    kn = np.sqrt(sum(t ** 2 for t in k))
    assert F[kn < 1.0 - 1e-9].max() <= 1e-12           # no mean, no other sub-unit mode
    assert F[kn > 4.0 + 1e-9].max() <= 1e-12           # nothing above |k| = 4
    live = F > 1e-9
    assert 2 <= live.sum() <= 2 * 8                     # each cosine is a +-k pair
    # a cosine of amplitude 0.3 puts 0.15 on each of +-k (triangle inequality when modes repeat)
    assert F.sum() <= 8 * 0.3 + 1e-9
    if seed in (2003, 4001):  # these seeds draw eight distinct, non-opposite wavevectors
        assert live.sum() == 16
    if live.sum() == 16:  # eight distinct modes: every coefficient is exactly half the amplitude
        assert np.abs(F[live] - 0.15).max() <= 1e-12


def test_generators_are_deterministic_and_seed_dependent():
    a1 = I.fourier_log_field(2, 32, seed=11)
    assert np.array_equal(a1, I.fourier_log_field(2, 32, seed=11))
    assert not np.array_equal(a1, I.fourier_log_field(2, 32, seed=12))
    f1 = I.uniform_load(2, 32, seed=11)
    assert np.array_equal(f1, I.uniform_load(2, 32, seed=11))
    assert f1.shape == (31, 31) and f1.min() >= -1.0 and f1.max() < 1.0
    assert abs(f1.mean()) < 0.1 and 0.25 < f1.var() < 0.42   # U(-1, 1): variance 1/3


@pytest.mark.parametrize("dim", [2, 3])
def test_boundary_data_is_harmonic(dim):
    """g is a harmonic quadratic, so the 5/7-point Laplacian of it vanishes exactly."""
    n = 12
    g = I.quadratic_boundary(dim, n)
    h = 1.0 / n
    inner = tuple(slice(1, n) for _ in range(dim))
    lap = -2.0 * dim * g[inner]
    for d in range(dim):
        for s in (-1, 1):
            sl = [slice(1, n)] * dim
            sl[d] = slice(1 + s, n + s)
            lap = lap + g[tuple(sl)]
    assert np.abs(lap / h ** 2).max() <= 1e-10


def test_helmholtz_reaction_and_source():
    """c = -kappa^2 (1 - 0.5 exp(-25 |x - c0|^2)) with c0 the centre; unit Gaussian source."""
    n, kappa = 64, 200.0
    c = I.helmholtz_reaction(2, n, kappa)
    assert np.isclose(c[n // 2, n // 2], -0.5 * kappa ** 2)
    assert np.isclose(c[0, 0], -kappa ** 2 * (1.0 - 0.5 * np.exp(-25.0 * 0.5)))
    assert c.max() <= -0.5 * kappa ** 2 + 1e-9 and c.min() >= -kappa ** 2
    src = I.gaussian_source(2, n)
    assert src.shape == (n - 1, n - 1)
    i, j = np.unravel_index(np.argmax(src), src.shape)
    assert (i + 1, j + 1) == (n // 4, n // 2) and np.isclose(src[i, j], 1.0)
    # width 0.01: one mesh width (1/64) away the source has fallen to exp(-1.22)
    assert np.isclose(src[i + 1, j], np.exp(-(1.0 / n) ** 2 / (2 * 0.01 ** 2)))


def test_uneven_batch_specification():
    """64 problems: n = 64 m with m in 4..16, 8/16/32 slabs, slab width <= 64, seeds 5000+i."""
    specs = I.batch_specs(64)
    assert len(specs) == 64
    assert [s["seed"] for s in specs] == list(range(5000, 5064))
    for s in specs:
        n, w = s["n"], s["w"]
        assert n % 64 == 0 and 256 <= n <= 1024
        assert n % w == 0 and n // w in (8, 16, 32)
    assert len({s["n"] for s in specs}) > 5          # genuinely uneven
    assert max(s["w"] for s in specs) > 64           # wide slabs (blocks above 128) included
    assert all(s["w"] <= 64 for s in I.batch_specs(64, wmax=64))
    assert specs == I.batch_specs(64)
