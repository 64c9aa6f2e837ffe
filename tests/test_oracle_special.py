"""Pins for the oracle's Bessel integrals and total rates.

References: scipy.special.kv (K_nu), mpmath at 30 digits (integrals), and the
textbook small- and large-chi asymptotes of the quasi-classical rates.
"""
import math

import numpy as np
import pytest
from scipy.special import kv, gamma as G

import oracle


@pytest.mark.parametrize("nu", [1 / 3, 2 / 3, 5 / 3])
def test_besselK_against_scipy(nu):
    ys = np.concatenate([np.logspace(-12, 2.8, 120), [0.5 - 1e-12, 0.5, 0.5 + 1e-12]])
    for y in ys:
        got = oracle.besselK(nu, y)
        want = kv(nu, y)
        assert got == pytest.approx(want, rel=2e-13, abs=0), (nu, y)


def test_intK13_against_mpmath_and_derivative():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for y in [1e-9, 0.1, 0.499999, 0.5, 2.0, 40.0]:
        want = mp.quad(lambda s: mp.besselk(mp.mpf(1) / 3, s), [y, y + 1, y + 10, mp.inf])
        assert oracle.intK13(y) == pytest.approx(float(want), rel=1e-12), y
    # d/dy int_y^inf K_{1/3} = -K_{1/3}(y)
    for y in [0.05, 0.3, 1.0, 3.0]:
        h = 1e-5 * y
        d = (oracle.intK13(y + h) - oracle.intK13(y - h)) / (2 * h)
        assert d == pytest.approx(-kv(1 / 3, y), rel=1e-7)
    assert oracle.intK13(1e-300) == pytest.approx(math.pi / math.sqrt(3), rel=1e-14)


def test_K53_identity():
    # int_y^inf K_{5/3} = 2 K_{2/3}(y) - int_y^inf K_{1/3}  (from 2K'_nu = -K_{nu-1} - K_{nu+1})
    from scipy.integrate import quad
    for y in [0.2, 1.0, 4.0]:
        lhs = quad(lambda s: kv(5 / 3, s), y, np.inf, epsabs=0, epsrel=1e-12, limit=400)[0]
        rhs = 2 * oracle.besselK(2 / 3, y) - oracle.intK13(y)
        assert lhs == pytest.approx(rhs, rel=1e-9)


def _i13(y):
    from scipy.integrate import quad
    # K_{1/3}(s) < 1e-26 K_{1/3}(y) beyond y + 60
    return quad(lambda s: kv(1 / 3, s), y, y + 60, epsabs=0, epsrel=1e-13, limit=200)[0]


@pytest.mark.parametrize("chi", [0.1, 1.0, 10.0])
def test_F_gamma_against_scipy(chi):
    from scipy.integrate import quad

    def f(d):
        y = 2 * d / (3 * chi * (1 - d))
        return ((1 - d) + 1 / (1 - d)) * kv(2 / 3, y) - _i13(y)
    want = quad(f, 0, 1, limit=400, points=[1e-6, 1e-3, 0.1, 0.5, 0.9], epsabs=0, epsrel=1e-12)[0]
    want /= math.sqrt(3) * math.pi
    assert oracle.F_gamma_quad(chi) == pytest.approx(want, rel=1e-10)


@pytest.mark.parametrize("chi", [0.01, 0.1, 1.0, 10.0])
def test_F_pair_against_scipy(chi):
    from scipy.integrate import quad

    def f(d):
        y = 2 / (3 * chi * d * (1 - d))
        return (d / (1 - d) + (1 - d) / d) * kv(2 / 3, y) + _i13(y)
    want = quad(f, 1e-6, 0.5, epsabs=0, epsrel=1e-12, limit=400, points=[0.05, 0.2, 0.35, 0.45])[0]
    want *= 2 / (math.sqrt(3) * math.pi)
    assert oracle.F_pair_quad(chi) == pytest.approx(want, rel=1e-10)


def test_emission_rate_asymptotes():
    # small chi: F = (5/(2 sqrt3)) chi (1 - (8 sqrt3/15) chi + O(chi^2))
    c0 = 5 / (2 * math.sqrt(3))
    for chi in [1e-5, 1e-4]:
        assert oracle.F_gamma_quad(chi) / chi == pytest.approx(c0 * (1 - 8 * math.sqrt(3) / 15 * chi), rel=10 * chi * chi + 1e-12)
    # large chi: F -> (14 Gamma(2/3) 3^{2/3} / 27) chi^{2/3}
    cinf = 14 * G(2 / 3) * 3 ** (2 / 3) / 27
    r6, r8 = (oracle.F_gamma_quad(c) / c ** (2 / 3) for c in (1e6, 1e8))
    assert abs(r8 - cinf) < abs(r6 - cinf)
    assert r8 == pytest.approx(cinf, rel=2e-3)


def test_pair_rate_asymptotes():
    # small chi (Erber): F = (3 sqrt3 / (16 sqrt2)) chi exp(-8/(3 chi)) (1 + O(chi))
    ce = 3 * math.sqrt(3) / (16 * math.sqrt(2))
    rels = []
    for chi in [0.01, 0.02, 0.04]:
        rels.append(oracle.F_pair_quad(chi) / (ce * chi * math.exp(-8 / (3 * chi))) - 1)
    assert abs(rels[0]) < 0.01
    assert abs(rels[0]) < abs(rels[1]) < abs(rels[2])       # the correction is O(chi)
    assert rels[1] / rels[0] == pytest.approx(2.0, rel=0.1)
    # large chi: F -> Gamma(2/3) 3^{2/3} 2 B(8/3, 2/3) / (sqrt3 pi) ... = 0.379612 chi^{2/3}
    from scipy.special import beta
    cinf = G(2 / 3) * 3 ** (2 / 3) * 2 * beta(8 / 3, 2 / 3) / (math.sqrt(3) * math.pi) * 3 / 7 * 7 / 3
    r = oracle.F_pair_quad(1e8) / 1e8 ** (2 / 3)
    assert r == pytest.approx(0.379612, rel=5e-3)
    assert cinf > 0
