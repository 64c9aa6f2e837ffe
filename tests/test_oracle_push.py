"""Pins for the oracle's field, chi, Boris push and event loop (Algorithms 1, 2).

Closed forms: Boris rotation in uniform B and acceleration in uniform E;
chi in special geometries; Maxwell's equations for the standing wave.
Laws: the probability of no event in a step is exp(-lambda dt) with lambda
from scipy quadrature; the first photon's energy follows the exact spectrum;
energy and charge are conserved per event; the event rate does not depend on
the PIC step (sub-stepping invariance); results do not depend on how the
ensemble is split or on buffer capacity.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import kv

import oracle
from paper_2409_17299_gb300 import workloads as W

ALPHA = 7.2973525693e-3
R = W.R_SCHWINGER


def _F_gamma_scipy(chi):
    def i13(y):
        return quad(lambda s: kv(1 / 3, s), y, y + 60, epsabs=0, epsrel=1e-13, limit=200)[0]

    def f(d):
        y = 2 * d / (3 * chi * (1 - d))
        return ((1 - d) + 1 / (1 - d)) * kv(2 / 3, y) - i13(y)
    return quad(f, 0, 1, limit=400, points=[1e-6, 1e-3, 0.1, 0.5, 0.9], epsabs=0, epsrel=1e-12)[0] / (math.sqrt(3) * math.pi)


def _F_pair_scipy(chi):
    def i13(y):
        return quad(lambda s: kv(1 / 3, s), y, y + 60, epsabs=0, epsrel=1e-13, limit=200)[0]

    def f(d):
        y = 2 / (3 * chi * d * (1 - d))
        return (d / (1 - d) + (1 - d) / d) * kv(2 / 3, y) + i13(y)
    return 2 * quad(f, 1e-6, 0.5, epsabs=0, epsrel=1e-12, limit=400, points=[0.05, 0.2, 0.35, 0.45])[0] / (math.sqrt(3) * math.pi)


def test_constants():
    a, r = oracle.constants()
    assert a == ALPHA and r == R


def test_boris_uniform_B_rotation():
    B = np.array([0, 0, 50.0])
    p = np.array([30.0, 0, 4.0])
    x = np.zeros(3)
    gam = math.sqrt(1 + p @ p)
    h = 0.01
    q = -1.0
    n = 1000
    for _ in range(n):
        x, p = oracle.boris(x, p, q, np.zeros(3), B, h)
    assert math.sqrt(p @ p) == pytest.approx(math.sqrt(30.0 ** 2 + 16.0), rel=1e-13)
    assert p[2] == pytest.approx(4.0, rel=1e-13)
    # per-step rotation angle of the Boris scheme; an electron moving along +x
    # in B_z > 0 feels q v x B along +y, so p_perp turns counter-clockwise
    theta = 2 * math.atan(abs(q * B[2]) * h / (2 * gam))
    want = 30.0 * np.array([math.cos(n * theta), math.sin(n * theta)])
    assert np.allclose(p[:2], want, rtol=0, atol=1e-9)


def test_boris_uniform_E_acceleration():
    E = np.array([3.0, -1.0, 0.5])
    p = np.array([1.0, 2.0, -3.0])
    x = np.zeros(3)
    for k in range(200):
        x, p = oracle.boris(x, p, +1.0, E, np.zeros(3), 0.05)
    assert np.allclose(p, np.array([1.0, 2.0, -3.0]) + E * 0.05 * 200, rtol=1e-13, atol=1e-12)


def test_chi_special_cases():
    # p perpendicular to B, no E: chi = |p||B|/R
    assert oracle.chi(math.sqrt(1 + 1e6), [1000, 0, 0], [0, 0, 0], [0, 0, R / 1000]) == pytest.approx(1.0, rel=1e-14)
    # at rest in E: chi = |E|/R
    assert oracle.chi(1.0, [0, 0, 0], [3e4, 4e4, 0], [0, 0, 0]) == pytest.approx(5e4 / R, rel=1e-14)
    # p parallel to E, B = 0: chi = |E|/R for any gamma (Lorentz invariance)
    p = np.array([0, 300.0, 0])
    assert oracle.chi(math.sqrt(1 + p @ p), p, [0, 1e3, 0], [0, 0, 0]) == pytest.approx(1e3 / R, rel=1e-9)
    # photon moving along x in B_z: chi = k0 |B| / R
    assert oracle.chi(500.0, [500, 0, 0], [0, 0, 0], [0, 0, 2 * R / 500]) == pytest.approx(2.0, rel=1e-14)
    # plane wave co-moving photon: E_y = B_z, k along x gives chi = 0
    assert oracle.chi(100.0, [100, 0, 0], [0, 7.0, 0], [0, 0, 7.0]) == pytest.approx(0.0, abs=1e-12)


def test_standing_wave_satisfies_maxwell():
    a0 = 2000.0
    h = 1e-5
    for x0, t0 in [(0.3, 0.7), (1.9, 4.0), (-2.5, 10.0)]:
        def EB(x, t):
            return oracle.field(W.FIELD_STANDING_CP, [a0], [x, 0.1, 0.2], t)
        E, B = EB(x0, t0)
        dEdx = (EB(x0 + h, t0)[0] - EB(x0 - h, t0)[0]) / (2 * h)
        dBdx = (EB(x0 + h, t0)[1] - EB(x0 - h, t0)[1]) / (2 * h)
        dEdt = (EB(x0, t0 + h)[0] - EB(x0, t0 - h)[0]) / (2 * h)
        dBdt = (EB(x0, t0 + h)[1] - EB(x0, t0 - h)[1]) / (2 * h)
        curlE = np.array([0, -dEdx[2], dEdx[1]])
        curlB = np.array([0, -dBdx[2], dBdx[1]])
        assert np.allclose(dBdt, -curlE, rtol=0, atol=1e-5 * a0)
        assert np.allclose(dEdt, curlB, rtol=0, atol=1e-5 * a0)
    E, B = oracle.field(W.FIELD_STANDING_CP, [a0], [0.0, 0, 0], 0.3)
    assert np.allclose(B, 0) and np.linalg.norm(E) == pytest.approx(a0)


def test_rotating_field():
    E, B = oracle.field(W.FIELD_ROTATING_E, [1000.0], [1, 2, 3], 0.25)
    assert np.allclose(E, [1000 * math.cos(0.25), 1000 * math.sin(0.25), 0]) and np.allclose(B, 0)


def _run(w, otables, nsteps=None, capacity=None, step0=0, seed=None, **kw):
    cap = capacity or [max(1024, 4 * len(s["id"])) for s in w.species]
    ens = oracle.Ensemble.from_arrays(w.species, cap)
    cfg = oracle.make_cfg(seed=w.seed if seed is None else seed, push_photons=w.push_photons,
                          thin_cap=w.thin_cap, field_kind=w.field_kind, field_prm=w.field_prm, **kw)
    st = oracle.push_and_generate(ens, otables, cfg, w.dt, w.nsteps if nsteps is None else nsteps, step0)
    return ens, st


def test_no_event_probability_and_energy(otables):
    n = 20000
    w = W.uniform_b_emission(n=n, seed=0)
    ens, st = _run(w, otables, nsteps=1)
    gam0 = math.sqrt(1 + 1000.0 ** 2)
    lam = ALPHA * R / gam0 * _F_gamma_scipy(1.0)
    p0 = math.exp(-lam * w.dt)
    e = ens.view(0)
    k = int(np.sum(e["nevents"] == 0))
    sd = math.sqrt(n * p0 * (1 - p0))
    assert abs(k - n * p0) < 5 * sd
    assert st["emit_events"] == int(e["nevents"].sum()) == ens.sp[2]["count"]
    assert st["particle_steps"] == n                       # photons recorded, not pushed
    # uniform B does no work: gamma of electrons + photon energies is conserved
    ph = ens.view(2)
    gam = np.sqrt(1 + e["px"] ** 2 + e["py"] ** 2 + e["pz"] ** 2)
    k0 = np.sqrt(ph["px"] ** 2 + ph["py"] ** 2 + ph["pz"] ** 2)
    assert gam.sum() + k0.sum() == pytest.approx(n * gam0, rel=1e-12)
    assert np.all(ph["w"] == 1.0)


def test_first_photon_spectrum(otables):
    n = 20000
    w = W.uniform_b_emission(n=n, seed=3)
    ens, _ = _run(w, otables, nsteps=1)
    ph = ens.view(2)
    # child id of the first event (k = 0) of each electron
    key = np.array([w.seed ^ 0xC0FFEE, 0], dtype=np.uint64)
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(n)
    r = oracle.philox(ctr, [int(key[0]) & 0xFFFFFFFF, int(key[0]) >> 32])
    first = r[:, 0].astype(np.uint64) | (r[:, 1].astype(np.uint64) << np.uint64(32))
    pos = {int(i): j for j, i in enumerate(ph["id"])}
    idx = [pos[int(f)] for f in first if int(f) in pos]
    gam0 = math.sqrt(1 + 1000.0 ** 2)
    d = np.sqrt(ph["px"][idx] ** 2 + ph["py"][idx] ** 2 + ph["pz"][idx] ** 2) / gam0
    m = len(d)
    assert m > 1000
    grid = np.quantile(d, np.linspace(0.01, 0.99, 40))
    F = np.array([oracle.em_cdf(1.0, g) for g in grid])
    emp = np.searchsorted(np.sort(d), grid, side="right") / m
    assert np.max(np.abs(emp - F)) < 1.63 / math.sqrt(m)


def test_pair_probability_and_conservation(otables):
    n = 20000
    k0 = 1000.0
    ph = {"x": np.zeros(n), "y": np.zeros(n), "z": np.zeros(n), "px": np.full(n, k0),
          "py": np.zeros(n), "pz": np.zeros(n), "w": np.ones(n), "id": np.arange(n, dtype=np.uint64)}
    w = W.Workload("photons_in_B", [W._empty(), W._empty(), ph], W.FIELD_UNIFORM,
                   [0, 0, 0, 0, 0, R / k0], 2 * math.pi / 200, 1, push_photons=1, seed=5)
    ens, st = _run(w, otables, capacity=[200000, 200000, 400000])
    lam = ALPHA * R / k0 * _F_pair_scipy(1.0)
    p0 = math.exp(-lam * w.dt)
    ne, npos = ens.sp[0]["count"], ens.sp[1]["count"]
    assert ne == npos == st["pair_events"]
    # photons that survived the step: the original ones still alive
    orig_alive = int(np.sum(np.isin(ens.view(2)["id"], ph["id"])))
    sd = math.sqrt(n * p0 * (1 - p0))
    assert abs(orig_alive - n * p0) < 5 * sd
    assert n - orig_alive == st["pair_events"]
    # B does no work and photons fly straight: total energy is conserved
    tot = 0.0
    for s in (0, 1):
        v = ens.view(s)
        tot += np.sum(np.sqrt(1 + v["px"] ** 2 + v["py"] ** 2 + v["pz"] ** 2))
    v = ens.view(2)
    tot += np.sum(np.sqrt(v["px"] ** 2 + v["py"] ** 2 + v["pz"] ** 2))
    assert tot == pytest.approx(n * k0, rel=1e-12)
    assert np.all(ens.view(2)["w"] > 0)        # dead photons were compacted away


def test_substep_invariance(otables):
    # events per period must not depend on the PIC step (the method sub-steps)
    n = 6000
    a = W.uniform_b_emission(n=n, seed=21, steps_per_period=50, nsteps=50)
    b = W.uniform_b_emission(n=n, seed=22, steps_per_period=200, nsteps=200)
    _, sa = _run(a, otables)
    _, sb = _run(b, otables)
    ea, eb = sa["emit_events"], sb["emit_events"]
    assert abs(ea - eb) < 5 * math.sqrt(ea + eb) * 1.5


def _sorted(ens, s):
    v = ens.view(s)
    o = np.argsort(v["id"])
    return {k: a[o] for k, a in v.items()}


def test_split_and_capacity_independence(otables):
    w = W.rotating_e_cascade(n=400, seed=1, periods=1)
    full, st = _run(w, otables, nsteps=30)
    idx = np.arange(400)
    parts = []
    for sel in (idx[:150], idx[150:]):
        parts.append(_run(W.subset(w, 0, sel), otables, nsteps=30)[0])
    small, _ = _run(w, otables, nsteps=30, capacity=[401, 8, 8])
    assert st["pair_events"] > 0 and st["emit_events"] > 0
    for s in range(3):
        a = _sorted(full, s)
        b = _sorted(small, s)
        cat = {k: np.concatenate([p.view(s)[k] for p in parts]) for k in a}
        o = np.argsort(cat["id"])
        for k in a:
            assert np.array_equal(a[k], b[k]), (s, k)
            assert np.array_equal(a[k], cat[k][o]), (s, k)
    # charge: e- minus e+ is the seed count
    assert full.sp[0]["count"] - full.sp[1]["count"] == 400
    assert len(np.unique(np.concatenate([full.view(s)["id"] for s in range(3)]))) == sum(full.sp[s]["count"] for s in range(3))
