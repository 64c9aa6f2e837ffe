"""The oracle's unit system pinned by the parameters the paper prints for its
test problem (Sec. 5.1, fixture tests/golden/test_problem_sec5_1.txt) and
CODATA constants (scipy.constants), not by the oracle's own constants.

- omega0 = 2 pi c / lambda and T = 2 pi / omega0 reproduce the printed values
  (three significant figures);
- R = m c^2 / (hbar omega0) and alpha equal the oracle's constants (to the
  CODATA revision difference, below 1e-8);
- a lepton at rest in the printed amplitude has chi = E / E_Schwinger in SI
  units; the oracle's chi of the same lepton in its normalised field (the
  amplitude in units of m c omega0 / e) must agree, which ties the field
  normalisation, R and the chi formula together.
"""
import math
import os

import numpy as np
import pytest
import scipy.constants as sc

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _fixture():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "test_problem_sec5_1.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            name, *rest = line.split()
            vals[name] = [float(v) for v in rest]
    return vals


def test_printed_frequency_and_period():
    g = _fixture()
    lam = g["wavelength_m"][0]
    omega = 2 * math.pi * sc.c / lam
    assert omega == pytest.approx(g["omega0_per_s"][0], rel=5e-3)
    assert 2 * math.pi / omega == pytest.approx(g["period_s"][0], rel=5e-3)


def test_oracle_constants_from_codata():
    g = _fixture()
    omega = 2 * math.pi * sc.c / g["wavelength_m"][0]
    alpha, R = oracle.constants()
    assert alpha == pytest.approx(sc.alpha, rel=1e-8)
    assert R == pytest.approx(sc.m_e * sc.c ** 2 / (sc.hbar * omega), rel=1e-8)


def test_chi_at_rest_in_the_printed_amplitude():
    g = _fixture()
    E_si = g["amplitude_V_per_m"][0]
    omega = 2 * math.pi * sc.c / g["wavelength_m"][0]
    e_schwinger = sc.m_e ** 2 * sc.c ** 3 / (sc.e * sc.hbar)
    want = E_si / e_schwinger                      # about 4.7e-3
    a0 = E_si / (sc.m_e * sc.c * omega / sc.e)     # about 1557 in the oracle's field unit
    assert 1550 < a0 < 1565
    got = oracle.chi(1.0, np.zeros(3), np.array([0.0, a0, 0.0]), np.zeros(3))
    assert got == pytest.approx(want, rel=1e-8)
    # the same through the standing wave at its electric antinode (x = 0, t = 0)
    E, B = oracle.field(oracle.FIELD_STANDING_CP, [a0], [0.0, 0.0, 0.0], 0.0)
    assert np.allclose(B, 0.0) and np.linalg.norm(E) == pytest.approx(a0, rel=1e-15)
    assert oracle.chi(1.0, np.zeros(3), E, B) == pytest.approx(want, rel=1e-8)
