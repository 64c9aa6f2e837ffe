"""Pins for the oracle's global leveling (threshold equation, unbiasedness)."""
import math

import numpy as np
import pytest

import oracle


def test_threshold_equal_weights():
    w = np.full(10000, 2.5)
    assert oracle.level_threshold(w, 4000) == pytest.approx(2.5 * 10000 / 4000, rel=1e-13)
    assert oracle.level_threshold(w, 10000) == 0.0


def test_threshold_defining_equation():
    rng = np.random.default_rng(3)
    w = np.exp(rng.normal(size=50000))
    w[::7] = 0.0                      # dead entries are ignored
    cap = 20000
    ws = oracle.level_threshold(w, cap)
    alive = w[w > 0]
    assert np.sum(np.minimum(1.0, alive / ws)) == pytest.approx(cap, rel=1e-12)


def test_leveling_unbiased():
    rng = np.random.default_rng(4)
    n, cap = 100000, 30000
    w = np.exp(rng.normal(size=n))
    arr = {"x": np.zeros(n), "y": np.zeros(n), "z": np.zeros(n), "px": np.zeros(n), "py": np.zeros(n),
           "pz": np.zeros(n), "w": w.copy(), "id": np.arange(n, dtype=np.uint64)}
    ens = oracle.Ensemble.from_arrays([arr, None, None], [n, 1, 1])
    ws = oracle.level(ens, 0, cap, seed=9, step=17)
    out = ens.view(0)
    keep_p = np.minimum(1.0, w / ws)
    var_n = np.sum(keep_p * (1 - keep_p))
    assert abs(len(out["w"]) - cap) < 5 * math.sqrt(var_n)
    # heavy particles kept untouched, light survivors raised to w*
    heavy = w >= ws
    assert np.all(np.isin(np.arange(n)[heavy], out["id"]))
    ow = dict(zip(out["id"].tolist(), out["w"].tolist()))
    assert all(ow[i] == w[i] for i in np.nonzero(heavy)[0][:1000])
    light_kept = [i for i in out["id"].tolist() if not heavy[i]]
    assert all(ow[i] == ws for i in light_kept[:1000])
    # total weight conserved in expectation
    var_w = np.sum(np.where(heavy, 0.0, ws * ws * keep_p * (1 - keep_p)))
    assert abs(out["w"].sum() - w.sum()) < 5 * math.sqrt(var_w)
    # stable compaction keeps id order
    assert np.all(np.diff(out["id"].astype(np.int64)) > 0)
