"""Pins for the oracle's rate approximant and inverse-CDF tables.

The rate approximant is checked against direct quadrature (itself pinned to
scipy), the table nodes against an independent scipy CDF, and the sampler
against the exact CDF (Kolmogorov-Smirnov bound).
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import kv

import oracle


def test_rate_approximant_vs_quadrature(otables):
    for chi in np.logspace(-3, 3, 181)[::3]:
        assert otables.rate_F(0, chi) == pytest.approx(oracle.F_gamma_quad(chi), rel=1e-8), chi
    for chi in np.logspace(-2, 3, 151)[::3]:
        assert otables.rate_F(1, chi) == pytest.approx(oracle.F_pair_quad(chi), rel=1e-8), chi


def test_rate_approximant_outside_range(otables):
    f3 = otables.rate_F(0, 1e-3)
    assert otables.rate_F(0, 1e-4) == pytest.approx(0.1 * f3, rel=1e-12)
    f6 = otables.rate_F(0, 1e3)
    assert otables.rate_F(0, 8e3) == pytest.approx(4.0 * f6, rel=1e-12)
    assert otables.rate_F(1, 0.0099) == 0.0
    assert otables.rate_F(1, 8e3) == pytest.approx(4.0 * otables.rate_F(1, 1e3), rel=1e-9)
    assert otables.rate_F(0, 0.0) == 0.0


def _scipy_em_cdf(chi, delta):
    def i13(y):
        return quad(lambda s: kv(1 / 3, s), y, y + 60, epsabs=0, epsrel=1e-13, limit=200)[0]

    def f(d):
        y = 2 * d / (3 * chi * (1 - d))
        return ((1 - d) + 1 / (1 - d)) * kv(2 / 3, y) - i13(y)
    # the substitution d = v^3 removes the d^{-2/3} endpoint singularity
    g = lambda v: f(v ** 3) * 3 * v * v
    tot = quad(g, 0, 1, epsabs=0, epsrel=1e-12, limit=400, points=[0.1, 0.5, 0.9, 0.99])[0]
    part = quad(g, 0, delta ** (1 / 3), epsabs=0, epsrel=1e-12, limit=400)[0]
    return part / tot


def test_emission_table_nodes_are_cdf_roots(otables):
    tab = otables.icdf_em.reshape(oracle.EM_NCHI, oracle.EM_NS)
    for i, j in [(0, 100), (40, 128), (60, 20), (60, 200), (100, 150), (120, 128)]:
        chi = 10 ** (-3 + i / 20)
        s = -16 + 32 * j / 256
        u = 1 / (1 + math.exp(-s))
        y = math.exp(tab[i, j])
        delta = 3 * chi * y / (2 + 3 * chi * y)
        assert _scipy_em_cdf(chi, delta) == pytest.approx(u, rel=1e-8, abs=1e-12), (i, j)


def _scipy_pair_cdf(chi, delta):
    def i13(y):
        return quad(lambda s: kv(1 / 3, s), y, y + 60, epsabs=0, epsrel=1e-13, limit=200)[0]

    def f(d):
        y = 2 / (3 * chi * d * (1 - d))
        return (d / (1 - d) + (1 - d) / d) * kv(2 / 3, y) + i13(y)
    half = quad(f, 1e-6, 0.5, epsabs=0, epsrel=1e-12, limit=400, points=[0.05, 0.2, 0.35, 0.45])[0]
    part = quad(f, 1e-6, delta, epsabs=0, epsrel=1e-12, limit=400)[0]
    return part / (2 * half)


def test_pair_table_nodes_are_cdf_roots(otables):
    tab = otables.icdf_pair.reshape(oracle.PAIR_NCHI, oracle.PAIR_NS)
    for i, j in [(0, 64), (20, 100), (40, 30), (100, 120)]:
        chi = 10 ** (-2 + i / 20)
        s = -16 + 16 * j / 128
        u = 1 / (1 + math.exp(-s))
        delta = math.exp(tab[i, j])
        assert _scipy_pair_cdf(chi, delta) == pytest.approx(u, rel=1e-8, abs=1e-12), (i, j)
    assert np.allclose(tab[:, -1], -math.log(2.0), atol=1e-12, rtol=0)


def test_tables_monotone(otables):
    te = otables.icdf_em.reshape(oracle.EM_NCHI, oracle.EM_NS)
    tp = otables.icdf_pair.reshape(oracle.PAIR_NCHI, oracle.PAIR_NS)
    assert np.all(np.diff(te, axis=1) > 0)
    assert np.all(np.diff(tp, axis=1) > 0)
    assert np.all(np.isfinite(te)) and np.all(np.isfinite(tp))


@pytest.mark.parametrize("chi", [0.01, 1.0, 100.0])
def test_emission_sampler_ks(otables, chi):
    n = 40000
    rng = np.random.default_rng(7)
    u = rng.random(n)
    d = np.array([otables.sample_emission(chi, x)[0] for x in u])
    assert np.all((d > 0) & (d < 1))
    grid = np.quantile(d, np.linspace(0.005, 0.995, 60))
    F = np.array([oracle.em_cdf(chi, g) for g in grid])
    emp = np.searchsorted(np.sort(d), grid, side="right") / n
    D = np.max(np.abs(emp - F))
    assert D < 1.63 / math.sqrt(n), D          # KS critical value at p = 0.01


@pytest.mark.parametrize("chi", [0.05, 1.0, 100.0])
def test_pair_sampler_ks_and_symmetry(otables, chi):
    n = 40000
    rng = np.random.default_rng(11)
    u = rng.random(n)
    d = np.array([otables.sample_pair(chi, x)[0] for x in u])
    assert np.all((d > 0) & (d < 1))
    grid = np.quantile(d, np.linspace(0.005, 0.995, 40))
    F = np.array([oracle.pair_cdf(chi, g) for g in grid])
    emp = np.searchsorted(np.sort(d), grid, side="right") / n
    assert np.max(np.abs(emp - F)) < 1.63 / math.sqrt(n)
    for x in [2.0 ** -30, 0.125, 0.3125, 0.4921875]:    # 1 - x is exact
        a, am = otables.sample_pair(chi, x)
        b, bm = otables.sample_pair(chi, 1 - x)
        assert a == pytest.approx(bm, rel=1e-14) and b == pytest.approx(am, rel=1e-14)


def test_cdf_helpers_against_scipy():
    for chi, d in [(1.0, 0.3), (0.01, 0.005)]:
        assert oracle.em_cdf(chi, d) == pytest.approx(_scipy_em_cdf(chi, d), rel=1e-8)
    assert oracle.pair_cdf(1.0, 0.2) == pytest.approx(_scipy_pair_cdf(1.0, 0.2), rel=1e-8)
    assert oracle.pair_cdf(1.0, 0.8) == pytest.approx(1 - _scipy_pair_cdf(1.0, 0.2), rel=1e-8)
