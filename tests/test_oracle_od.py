"""Pins for the oracle's accumulated optical-depth scheme (Sec. 3: the
inverse-sampling method of other PIC codes, rate once per step, at most one
event per particle and step).

Laws: with the optical depth d ~ Exp(1) falling by lambda dt per step, the
probability of an event in the first step is 1 - exp(-lambda dt) and a photon
in a constant field survives n steps with probability exp(-n lambda dt)
(lambda from scipy quadrature); the first photon's energy follows the exact
spectrum; energy and charge are conserved per event; for lambda dt -> 0 the
number of emissions over a fixed time matches Algorithm 1.  Readings pinned
per particle: d drawn from counter word 0xFFFFFFFE when not positive, kept
between steps and calls, redrawn from the event's words 0-1; newborns start
at the next step with d = 0 at the parent's end point.
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
OD = oracle.METHOD_OPTICAL_DEPTH


def _i13(y):
    return quad(lambda s: kv(1 / 3, s), y, y + 60, epsabs=0, epsrel=1e-13, limit=200)[0]


def _F_gamma_scipy(chi):
    def f(d):
        y = 2 * d / (3 * chi * (1 - d))
        return ((1 - d) + 1 / (1 - d)) * kv(2 / 3, y) - _i13(y)
    return quad(f, 0, 1, limit=400, points=[1e-6, 1e-3, 0.1, 0.5, 0.9], epsabs=0,
                epsrel=1e-12)[0] / (math.sqrt(3) * math.pi)


def _F_pair_scipy(chi):
    def f(d):
        y = 2 / (3 * chi * d * (1 - d))
        return (d / (1 - d) + (1 - d) / d) * kv(2 / 3, y) + _i13(y)
    return 2 * quad(f, 1e-6, 0.5, epsabs=0, epsrel=1e-12, limit=400,
                    points=[0.05, 0.2, 0.35, 0.45])[0] / (math.sqrt(3) * math.pi)


def _run(w, otables, nsteps=None, step0=0, ens=None, method=OD, capacity=None):
    if ens is None:
        cap = capacity or [max(1024, 4 * len(s["id"])) for s in w.species]
        ens = oracle.Ensemble.from_arrays(w.species, cap)
    cfg = oracle.make_cfg(seed=w.seed, push_photons=w.push_photons, thin_cap=w.thin_cap,
                          field_kind=w.field_kind, field_prm=w.field_prm, event_method=method)
    st = oracle.push_and_generate(ens, otables, cfg, w.dt, w.nsteps if nsteps is None else nsteps, step0)
    return ens, st


def _draws(seed, ids, step, word):
    """Philox(ids, step, word) under the run's seed: (n, 4) uint32."""
    ids = np.asarray(ids, dtype=np.uint64)
    ctr = np.zeros((len(ids), 4), dtype=np.uint32)
    ctr[:, 0] = (ids & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    ctr[:, 1] = (ids >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = step
    ctr[:, 3] = word
    return oracle.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])


def _neglog_u(r):
    return np.array([-math.log(oracle.u52(int(a), int(b))) for a, b in zip(r[:, 0], r[:, 1])])


def _photons_in_B(n, k0, steps_per_period, seed):
    ph = {"x": np.zeros(n), "y": np.zeros(n), "z": np.zeros(n), "px": np.full(n, k0),
          "py": np.zeros(n), "pz": np.zeros(n), "w": np.ones(n), "id": np.arange(n, dtype=np.uint64)}
    return W.Workload("photons_in_B", [W._empty(), W._empty(), ph], W.FIELD_UNIFORM,
                      [0, 0, 0, 0, 0, R / k0], 2 * math.pi / steps_per_period, 1, push_photons=1, seed=seed)


def test_first_step_probability_and_energy(otables):
    n = 20000
    w = W.uniform_b_emission(n=n, seed=7, steps_per_period=40, nsteps=1)
    ens, st = _run(w, otables, nsteps=1)
    gam0 = math.sqrt(1 + 1000.0 ** 2)
    lam = ALPHA * R / gam0 * _F_gamma_scipy(1.0)
    p1 = 1 - math.exp(-lam * w.dt)
    e = ens.view(0)
    k = int(np.sum(e["nevents"] == 1))
    assert abs(k - n * p1) < 5 * math.sqrt(n * p1 * (1 - p1))
    assert np.all(e["nevents"] <= 1) and st["max_subevents"] == 1
    assert st["emit_events"] == k == ens.sp[2]["count"] and st["particle_steps"] == n
    ph = ens.view(2)
    gam = np.sqrt(1 + e["px"] ** 2 + e["py"] ** 2 + e["pz"] ** 2)
    kk = np.sqrt(ph["px"] ** 2 + ph["py"] ** 2 + ph["pz"] ** 2)
    assert gam.sum() + kk.sum() == pytest.approx(n * gam0, rel=1e-12)
    assert np.all(e["od"] > 0) and np.all(ph["od"] == 0.0)


def test_persistence_counter_words_and_newborns(otables):
    """Per particle: d0 from word 0xFFFFFFFE; no event leaves d0 - lambda dt;
    an event leaves -ln u of the event's words 0-1; the photon sits at the
    parent's end point (not pushed in its birth step)."""
    n = 3000
    w = W.uniform_b_emission(n=n, seed=11, steps_per_period=40, nsteps=1)
    ens, _ = _run(w, otables, nsteps=1)
    e = ens.view(0)
    o = np.argsort(e["id"])
    e = {k: v[o] for k, v in e.items()}
    d0 = _neglog_u(_draws(w.seed, e["id"], 0, 0xFFFFFFFE))
    lam = otables.rate_lambda(False, [1000.0, 0, 0], [0, 0, 0], w.field_prm[3:6])
    ev = e["nevents"] == 1
    assert ev.sum() > 100 and (~ev).sum() > 100
    assert np.array_equal(ev, d0 - lam * w.dt <= 0)
    assert np.array_equal(e["od"][~ev], d0[~ev] - lam * w.dt)
    assert np.array_equal(e["od"][ev], _neglog_u(_draws(w.seed, e["id"][ev], 0, 0)))
    # child id: Philox(id, step, 0) under seed ^ 0xC0FFEE, words 0-1
    r = _draws(w.seed ^ 0xC0FFEE, e["id"][ev], 0, 0)
    cid = r[:, 0].astype(np.uint64) | (r[:, 1].astype(np.uint64) << np.uint64(32))
    ph = ens.view(2)
    pos = {int(i): j for j, i in enumerate(ph["id"])}
    j = np.array([pos[int(c)] for c in cid])
    for a in ("x", "y", "z"):
        assert np.array_equal(ph[a][j], e[a][ev])
    # the parent moved the full step: |x| is the chord of the Boris arc
    assert np.all(np.abs(e["x"]) > 0.9 * 1000.0 / math.sqrt(1 + 1e6) * w.dt)


def test_photon_survival_and_conversion_step(otables):
    """Constant chi: survival after n steps is exp(-n lambda dt); each photon
    converts in the first step where its d0 minus the accumulated decrements
    reaches 0 (d kept from step to step)."""
    n, k0, nst = 20000, 1000.0, 12
    w = _photons_in_B(n, k0, 100, seed=5)
    ens = oracle.Ensemble.from_arrays(w.species, [400000, 400000, 2 * n])
    alive = []
    for s in range(nst):
        ens, _ = _run(w, otables, nsteps=1, step0=s, ens=ens)
        ids = ens.view(2)["id"]
        alive.append(ids[ids < n])         # the original photons (children have Philox ids)
    lam = ALPHA * R / k0 * _F_pair_scipy(1.0)
    for s in (0, 3, 7, nst - 1):
        p = math.exp(-(s + 1) * lam * w.dt)
        m = len(alive[s])
        assert abs(m - n * p) < 5 * math.sqrt(n * p * (1 - p)), (s, m, n * p)
    # per photon: the step of conversion from d0 and the oracle's own rate
    lam_o = otables.rate_lambda(True, [k0, 0, 0], [0, 0, 0], w.field_prm[3:6])
    d = _neglog_u(_draws(w.seed, np.arange(n), 0, 0xFFFFFFFE))
    conv = np.full(n, -1)
    for s in range(nst):
        d = d - lam_o * w.dt
        conv[(conv < 0) & (d <= 0)] = s
    for s in range(nst):
        want = np.sort(np.nonzero((conv < 0) | (conv > s))[0]).astype(np.uint64)
        assert np.array_equal(np.sort(alive[s]), want), s
    # charge and energy: as many e- as e+, B does no work
    assert ens.sp[0]["count"] == ens.sp[1]["count"] >= int(np.sum(conv >= 0))
    tot = 0.0
    for sp in (0, 1):
        v = ens.view(sp)
        tot += np.sum(np.sqrt(1 + v["px"] ** 2 + v["py"] ** 2 + v["pz"] ** 2))
    v = ens.view(2)
    tot += np.sum(np.sqrt(v["px"] ** 2 + v["py"] ** 2 + v["pz"] ** 2))
    assert tot == pytest.approx(n * k0, rel=1e-11)


def test_calls_split_equal_one_call(otables):
    """d lives in the ensemble: two calls of 3 steps equal one call of 6."""
    w = W.rotating_e_cascade(n=300, seed=3, periods=1)
    a, sa = _run(w, otables, nsteps=6)
    b, _ = _run(w, otables, nsteps=3)
    b, _ = _run(w, otables, nsteps=3, step0=3, ens=b)
    assert sa["emit_events"] > 0
    for s in range(3):
        va, vb = a.view(s), b.view(s)
        oa, ob = np.argsort(va["id"]), np.argsort(vb["id"])
        for k in va:
            assert np.array_equal(va[k][oa], vb[k][ob]), (s, k)


def test_first_photon_spectrum(otables):
    n = 20000
    w = W.uniform_b_emission(n=n, seed=13, steps_per_period=20, nsteps=1)
    ens, _ = _run(w, otables, nsteps=1)
    ph = ens.view(2)
    gam0 = math.sqrt(1 + 1000.0 ** 2)
    d = np.sqrt(ph["px"] ** 2 + ph["py"] ** 2 + ph["pz"] ** 2) / gam0
    m = len(d)
    assert m > 2000
    grid = np.quantile(d, np.linspace(0.01, 0.99, 40))
    F = np.array([oracle.em_cdf(1.0, g) for g in grid])
    emp = np.searchsorted(np.sort(d), grid, side="right") / m
    assert np.max(np.abs(emp - F)) < 1.63 / math.sqrt(m)


def test_small_step_limit_matches_algorithm_1(otables):
    """Over one period with lambda dt ~ 0.01 the emission count and the mean
    final energy agree with Algorithm 1 within the statistics plus the
    scheme's O(lambda dt) bias (events at step ends)."""
    n = 3000
    w = W.uniform_b_emission(n=n, seed=17, steps_per_period=400, nsteps=400)
    a, sa = _run(w, otables, method=oracle.METHOD_SUBSTEP)
    b, sb = _run(w, otables)
    ea, eb = sa["emit_events"], sb["emit_events"]
    assert ea > 5 * n
    assert abs(ea - eb) < 5 * math.sqrt(ea + eb) + 0.02 * ea, (ea, eb)
    ga = np.sqrt(1 + np.sum(np.stack([a.view(0)[k] for k in ("px", "py", "pz")]) ** 2, axis=0))
    gb = np.sqrt(1 + np.sum(np.stack([b.view(0)[k] for k in ("px", "py", "pz")]) ** 2, axis=0))
    se = math.sqrt(ga.var() / n + gb.var() / n)
    assert abs(ga.mean() - gb.mean()) < 5 * se + 0.02 * (1000.0 - ga.mean())
