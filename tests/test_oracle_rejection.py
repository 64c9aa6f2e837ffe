"""Algorithm 1 against an independent generator of the same physics: the
subcycled rejection method (candidate energy fraction delta = r^3 accepted
with probability 3 r^2 (dW/d delta) h from the Bessel functions directly,
its own random stream).  In the uniform-B emission workload (chi0 = 1,
gamma0 = 1000) both give the same emission count, photon spectrum and
electron energy distribution within statistics; the mean count matches
the closed-form expectation (15.63 emissions per period at chi = 1)."""
import math

import numpy as np
import pytest

import oracle
from paper_2409_17299_gb300 import workloads as W

N, STEPS, NSUB = 2048, 30, 16


@pytest.fixture(scope="module")
def runs(otables):
    w = W.uniform_b_emission(n=N, seed=0)
    cfg = oracle.make_cfg(seed=21, push_photons=0, field_kind=w.field_kind, field_prm=w.field_prm)
    a = oracle.Ensemble.from_arrays(w.species, [N, 1, 8 * N])
    st = oracle.push_and_generate(a, otables, cfg, w.dt, STEPS, 0)
    ph = a.view(2)
    k_alg1 = np.sqrt(ph["px"] ** 2 + ph["py"] ** 2 + ph["pz"] ** 2)
    b = oracle.Ensemble.from_arrays(w.species, [N, 1, 1])
    k_rej, n_rej, amax = oracle.rejection_run(b, cfg, w.dt, STEPS, NSUB, seed=99)
    ga = np.sqrt(1 + a.view(0)["px"] ** 2 + a.view(0)["py"] ** 2 + a.view(0)["pz"] ** 2)
    gb = np.sqrt(1 + b.view(0)["px"] ** 2 + b.view(0)["py"] ** 2 + b.view(0)["pz"] ** 2)
    return st["emit_events"], k_alg1, n_rej, k_rej, amax, ga, gb, w


def test_acceptance_stays_small(runs):
    *_, amax, _, _, _ = runs
    assert 0 < amax < 0.05


def test_emission_counts_agree(runs):
    n1, _, n2, *_ , w = runs
    expect = N * STEPS * w.dt / (2 * math.pi) * 15.63      # at chi = 1; chi falls slowly as electrons recoil
    assert abs(n1 - n2) < 5 * math.sqrt(n1 + n2), (n1, n2)
    assert 0.9 * expect < n1 < expect + 5 * math.sqrt(expect), (n1, expect)


def test_photon_spectra_agree(runs):
    from scipy.stats import ks_2samp
    _, k1, _, k2, *_ = runs
    assert ks_2samp(k1, k2).pvalue > 0.001


def test_electron_energies_agree(runs):
    """Electrons that never emitted keep gamma0 (up to the rounding of 1 or
    16 Boris rotations per step): compare that fraction binomially and the
    energies of the others by KS."""
    from scipy.stats import ks_2samp
    *_, ga, gb, w = runs
    g0 = math.sqrt(1 + 1000.0 ** 2)
    qa, qb = np.abs(ga - g0) < 1e-6, np.abs(gb - g0) < 1e-6
    f = 0.5 * (qa.mean() + qb.mean())
    assert abs(qa.mean() - qb.mean()) < 5 * math.sqrt(2 * f * (1 - f) / N)
    assert ks_2samp(ga[~qa], gb[~qb]).pvalue > 0.001
