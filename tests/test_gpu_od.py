"""GPU parity of the accumulated optical-depth scheme (Sec. 3, the
inverse-sampling method of other PIC codes) against the FP64 oracle.

Bars: FP64 per-particle event counts bit-exact, momenta and positions within
1e-5 relative, remaining optical depth within 1e-9 (absolute, the depths are
O(1)); FP32 (FP64 optical depth) event counts equal for at least 99% of the
particles, momenta within 1e-3 on those, totals within the statistics.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2409_17299_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_17299_gb300 as q  # noqa: E402
from test_gpu_parity import assert_same_fp64, by_id  # noqa: E402

OD = q.QED_METHOD_OPTICAL_DEPTH


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_17299_gb300 import build
    build.build()


def run_gpu(w, prec, nsteps, capacity, thin_cap=0, step0=0, ens=None):
    g = q.Generator(q.make_config(precision=prec, seed=w.seed, push_photons=w.push_photons,
                                  thin_cap=thin_cap, event_method=OD))
    if ens is None:
        ens = q.DeviceEnsemble.from_host(w.species, capacity, prec, optical_depth=True)
    st = g.push(ens, q.make_field(w.field_kind, w.field_prm), w.dt, nsteps, step0)
    torch.cuda.synchronize()
    g.close()
    return ens, st


def run_oracle(w, otables, nsteps, capacity, thin_cap=0):
    ens = oracle.Ensemble.from_arrays(w.species, capacity)
    cfg = oracle.make_cfg(seed=w.seed, push_photons=w.push_photons, thin_cap=thin_cap,
                          field_kind=w.field_kind, field_prm=w.field_prm,
                          event_method=oracle.METHOD_OPTICAL_DEPTH)
    st = oracle.push_and_generate(ens, otables, cfg, w.dt, nsteps)
    return [ens.view(s) for s in range(3)], st


def _same_od(g, o, what):
    g, o = by_id(g), by_id(o)
    assert np.array_equal(g["id"], o["id"]), what
    assert np.all((g["od"] == 0) == (o["od"] == 0)), what
    assert np.max(np.abs(g["od"] - o["od"]), initial=0.0) < 1e-9, what


@pytest.mark.parametrize("n,nsteps", [(1, 3), (33, 20), (1025, 10)])
def test_emission_fp64_ragged(n, nsteps, otables):
    w = W.uniform_b_emission(n=n, seed=3, steps_per_period=40, nsteps=nsteps)
    cap = [n, 8, 4 * n * nsteps + 8]
    ens, gs = run_gpu(w, q.QED_FP64, nsteps, cap)
    o, os_ = run_oracle(w, otables, nsteps, cap)
    for k in ("emit_events", "particle_steps", "max_subevents"):
        assert gs[k] == os_[k], k
    for s in (0, 2):
        g = ens.to_host(s)
        assert_same_fp64(g, o[s], what="species %d" % s)
        _same_od(g, o[s], "species %d" % s)


@pytest.mark.parametrize("make,nsteps,thin", [
    (lambda: W.rotating_e_cascade(n=600, seed=1, periods=1), 60, 0),
    (lambda: W.standing_wave_cascade(n=400, seed=4, periods=1), 50, 0),
    (lambda: W.rotating_e_cascade(n=500, seed=2, periods=1), 60, 900),
])
def test_cascade_fp64(make, nsteps, thin, otables):
    w = make()
    cap = [40000, 40000, 120000]
    ens, gs = run_gpu(w, q.QED_FP64, nsteps, cap, thin_cap=thin)
    o, os_ = run_oracle(w, otables, nsteps, cap, thin_cap=thin)
    assert os_["pair_events"] > 0 and os_["emit_events"] > 0
    for k in ("emit_events", "pair_events", "particle_steps", "max_subevents"):
        assert gs[k] == os_[k], k
    for s in range(3):
        g = ens.to_host(s)
        assert_same_fp64(g, o[s], what="species %d" % s)
        _same_od(g, o[s], "species %d" % s)


def test_two_calls_equal_one(otables):
    """The optical depth persists in the caller's arrays between calls."""
    w = W.rotating_e_cascade(n=300, seed=3, periods=1)
    cap = [20000, 20000, 60000]
    a, _ = run_gpu(w, q.QED_FP64, 40, cap)
    b, _ = run_gpu(w, q.QED_FP64, 20, cap)
    b, _ = run_gpu(w, q.QED_FP64, 20, cap, step0=20, ens=b)
    for s in range(3):
        x, y = by_id(a.to_host(s)), by_id(b.to_host(s))
        for k in x:
            assert np.array_equal(x[k], y[k]), (s, k)


def test_fp32_against_fp64_oracle(otables):
    w = W.uniform_b_emission(n=16384, seed=0, steps_per_period=100, nsteps=30)
    cap = [16384, 8, 300000]
    ens, gs = run_gpu(w, q.QED_FP32, 30, cap)
    o, os_ = run_oracle(w, otables, 30, cap)
    a, b = by_id(ens.to_host(0)), by_id(o[0])
    assert np.array_equal(a["id"], b["id"])
    same = a["nevents"] == b["nevents"]
    assert same.mean() > 0.99, same.mean()
    pa = np.stack([a[k][same] for k in ("px", "py", "pz")], 1)
    pb = np.stack([b[k][same] for k in ("px", "py", "pz")], 1)
    rel = np.linalg.norm(pa - pb, axis=1) / np.linalg.norm(pb, axis=1)
    assert rel.max() < 1e-3, rel.max()
    assert abs(gs["emit_events"] - os_["emit_events"]) < 5 * math.sqrt(os_["emit_events"])


def test_fp32_cascade_statistics(otables):
    w = W.rotating_e_cascade(n=3000, seed=1, periods=1)
    cap = [200000, 200000, 600000]
    ens, gs = run_gpu(w, q.QED_FP32, 60, cap)
    o, os_ = run_oracle(w, otables, 60, cap)
    for key in ("emit_events", "pair_events"):
        assert abs(gs[key] - os_[key]) < 6 * math.sqrt(os_[key]) + 5, key
    from scipy.stats import ks_2samp
    for s in range(3):
        g = ens.to_host(s)
        ea = np.sqrt(g["px"] ** 2 + g["py"] ** 2 + g["pz"] ** 2)
        eb = np.sqrt(o[s]["px"] ** 2 + o[s]["py"] ** 2 + o[s]["pz"] ** 2)
        assert ks_2samp(ea, eb).pvalue > 0.01, s


def test_rejected_configurations():
    w = W.uniform_b_emission(n=64, seed=1, nsteps=1)
    f = q.make_field(w.field_kind, w.field_prm)
    # no optical-depth arrays bound
    g = q.Generator(q.make_config(precision=q.QED_FP64, seed=1, push_photons=0, event_method=OD))
    ens = q.DeviceEnsemble.from_host(w.species, [64, 8, 64], q.QED_FP64)
    with pytest.raises(q.QedError):
        q.qed_push_and_generate(g.ctx, ens.struct(), f, w.dt, 1, 0)
    g.close()
    # unknown method
    g = q.Generator(q.make_config(precision=q.QED_FP64, seed=1, push_photons=0, event_method=7))
    with pytest.raises(q.QedError):
        q.qed_push_and_generate(g.ctx, ens.struct(), f, w.dt, 1, 0)
    g.close()
    # misaligned optical-depth pointer
    g = q.Generator(q.make_config(precision=q.QED_FP64, seed=1, push_photons=0, event_method=OD))
    buf = torch.zeros(80, dtype=torch.float64, device="cuda")
    with pytest.raises(q.QedError):
        q.qed_set_optical_depth(g.ctx, [buf.data_ptr() + 4, 0, 0])
    g.close()


def test_grid_field_fp64_matches_oracle(otables):
    """The optical-depth kernels are compiled for the gridded field too: the
    standing-wave cascade in a field held on the 128 x 4 x 4 node grid,
    FP64, against the oracle's optical-depth run in the same grid."""
    from test_gpu_grid import PRM, _grid_workload, standing_wave_grid
    w = _grid_workload(300, seed=8)
    grid = standing_wave_grid(1500.0, 0.0)       # one PIC step's fields, held for the call
    nsteps, cap = 40, [40000, 40000, 120000]
    g = q.Generator(q.make_config(precision=q.QED_FP64, seed=w.seed, push_photons=1, event_method=OD))
    dev = torch.tensor(grid, dtype=torch.float64, device="cuda")
    q.qed_set_field_grid(g.ctx, dev.data_ptr())
    ens = q.DeviceEnsemble.from_host(w.species, cap, q.QED_FP64, optical_depth=True)
    gs = g.push(ens, q.make_field(w.field_kind, w.field_prm), w.dt, nsteps, 0)
    torch.cuda.synchronize()
    g.close()
    oracle.set_field_grid(grid)
    oe = oracle.Ensemble.from_arrays(w.species, cap)
    cfg = oracle.make_cfg(seed=w.seed, push_photons=1, field_kind=oracle.FIELD_GRID, field_prm=PRM,
                          event_method=oracle.METHOD_OPTICAL_DEPTH)
    os_ = oracle.push_and_generate(oe, otables, cfg, w.dt, nsteps, 0)
    assert os_["emit_events"] > 0
    for k in ("emit_events", "pair_events", "particle_steps"):
        assert gs[k] == os_[k], k
    for s in range(3):
        got = ens.to_host(s)
        assert_same_fp64(got, oe.view(s), what="species %d" % s)
        _same_od(got, oe.view(s), "species %d" % s)


def test_network_sampler_rejected():
    """The optical-depth kernels sample energies from the tables only."""
    w = W.uniform_b_emission(n=64, seed=1, nsteps=1)
    g = q.Generator(q.make_config(precision=q.QED_FP32, seed=1, push_photons=0, event_method=OD,
                                  sampler=q.QED_SAMPLER_MLP))
    q.qed_mlp_set_params(g.ctx, np.zeros(oracle.mlp_nparams()))     # a network is loaded
    ens = q.DeviceEnsemble.from_host(w.species, [64, 8, 64], q.QED_FP32, optical_depth=True)
    with pytest.raises(q.QedError):
        g.push(ens, q.make_field(w.field_kind, w.field_prm), w.dt, 1, 0, auto_grow=False)
    g.close()
