"""Gridded field (a PIC step's node fields, trilinear interpolation) on the
GPU against the oracle: the same cascade in a grid sampled from the
standing circularly polarised wave, FP64 bit-exact in ids and event counts
and within 1e-5 in momenta, FP32 within its tolerance; the grid can be
rewritten between calls (a new PIC step), and calls without a grid fail."""
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

NX, NY, NZ = 128, 4, 4           # the paper's 1-wavelength box, 128 x 4 x 4 cells
LBOX = (2 * math.pi, 2 * math.pi, 2 * math.pi)
PRM = (NX, NY, NZ, *LBOX)


def standing_wave_grid(a0, t):
    """Node values of E = a0 cos x (0, cos t, sin t), B = a0 sin x (0, cos t,
    sin t) on the grid, layout (6, nz, ny, nx)."""
    x = np.arange(NX) * LBOX[0] / NX
    g = np.zeros((6, NZ, NY, NX))
    g[1] = a0 * np.cos(x) * math.cos(t)
    g[2] = a0 * np.cos(x) * math.sin(t)
    g[4] = a0 * np.sin(x) * math.cos(t)
    g[5] = a0 * np.sin(x) * math.sin(t)
    return g


def _grid_workload(n, seed):
    w = W.standing_wave_cascade(n=n, seed=seed, a0=1500.0, periods=1)
    w.field_kind = q.QED_FIELD_GRID
    w.field_prm = list(PRM)
    return w


def _run(w, prec, grid, nsteps, cap):
    g = q.Generator(q.make_config(precision=prec, seed=w.seed, push_photons=1))
    dev = torch.tensor(grid, dtype=torch.float64 if prec == q.QED_FP64 else torch.float32, device="cuda")
    q.qed_set_field_grid(g.ctx, dev.data_ptr())
    ens = q.DeviceEnsemble.from_host(w.species, cap, prec)
    st = g.push(ens, q.make_field(w.field_kind, w.field_prm), w.dt, nsteps, 0)
    torch.cuda.synchronize()
    out = [ens.to_host(s) for s in range(3)]
    g.close()
    return out, st


def _oracle(w, otables, grid, nsteps, cap):
    oracle.set_field_grid(grid)
    ens = oracle.Ensemble.from_arrays(w.species, cap)
    cfg = oracle.make_cfg(seed=w.seed, push_photons=1, field_kind=oracle.FIELD_GRID, field_prm=PRM)
    st = oracle.push_and_generate(ens, otables, cfg, w.dt, nsteps, 0)
    return [ens.view(s) for s in range(3)], st


def test_grid_cascade_fp64_matches_oracle(otables):
    w = _grid_workload(1500, seed=4)
    grid = standing_wave_grid(1500.0, 0.4)
    cap = [40000, 40000, 120000]
    g, gs = _run(w, q.QED_FP64, grid, 100, cap)
    o, os_ = _oracle(w, otables, grid, 100, cap)
    assert os_["emit_events"] > 40
    assert (gs["emit_events"], gs["pair_events"], gs["particle_steps"]) == \
        (os_["emit_events"], os_["pair_events"], os_["particle_steps"])
    for s in range(3):
        assert_same_fp64(g[s], o[s], what="species %d" % s)


def test_grid_cascade_fp32_within_tolerance(otables):
    w = _grid_workload(500, seed=5)
    grid = standing_wave_grid(1500.0, 1.1)
    cap = [40000, 40000, 120000]
    g, gs = _run(w, q.QED_FP32, grid, 25, cap)
    o, os_ = _oracle(w, otables, grid, 25, cap)
    # event counts: FP32 decisions may flip rarely
    for key in ("emit_events", "pair_events"):
        assert abs(gs[key] - os_[key]) <= 0.01 * os_[key] + 5, key
    a, b = by_id(g[0]), by_id(o[0])
    common, ia, ib = np.intersect1d(a["id"], b["id"], return_indices=True)
    assert len(common) >= 0.98 * len(b["id"])
    same = a["nevents"][ia] == b["nevents"][ib]
    assert same.mean() > 0.98
    pa = np.stack([a["px"][ia], a["py"][ia], a["pz"][ia]], 1)[same]
    pb = np.stack([b["px"][ib], b["py"][ib], b["pz"][ib]], 1)[same]
    rel = np.linalg.norm(pa - pb, axis=1) / np.maximum(np.linalg.norm(pb, axis=1), 1.0)
    assert np.quantile(rel, 0.99) < 1e-3


def test_grid_rewritten_between_calls(otables):
    """Two PIC steps: the grid is refilled with the fields at the new time
    between the calls; the result equals the oracle's run with the same two
    grids."""
    w = _grid_workload(300, seed=6)
    cap = [30000, 30000, 90000]
    g = q.Generator(q.make_config(precision=q.QED_FP64, seed=w.seed, push_photons=1))
    dev = torch.empty((6, NZ, NY, NX), dtype=torch.float64, device="cuda")
    q.qed_set_field_grid(g.ctx, dev.data_ptr())
    ens = q.DeviceEnsemble.from_host(w.species, cap, q.QED_FP64)
    oens = oracle.Ensemble.from_arrays(w.species, cap)
    cfg = oracle.make_cfg(seed=w.seed, push_photons=1, field_kind=oracle.FIELD_GRID, field_prm=PRM)
    for step in range(12):
        grid = standing_wave_grid(1500.0, step * w.dt)
        dev.copy_(torch.from_numpy(grid))
        g.push(ens, q.make_field(q.QED_FIELD_GRID, PRM), w.dt, 1, step)
        oracle.set_field_grid(grid)
        oracle.push_and_generate(oens, otables, cfg, w.dt, 1, step)
    torch.cuda.synchronize()
    for s in range(3):
        assert_same_fp64(ens.to_host(s), oens.view(s), what="species %d" % s)
    g.close()


def test_grid_required_and_validated():
    g = q.Generator(q.make_config(precision=q.QED_FP64, push_photons=1))
    w = _grid_workload(10, seed=7)
    ens = q.DeviceEnsemble.from_host(w.species, [64, 64, 64], q.QED_FP64)
    P = ens.struct()
    with pytest.raises(q.QedError) as e:               # no grid attached
        q.qed_push_and_generate(g.ctx, P, q.make_field(q.QED_FIELD_GRID, PRM), w.dt, 1, 0)
    assert e.value.status == q.QED_ERR_STATE
    dev = torch.zeros((6, NZ, NY, NX), dtype=torch.float64, device="cuda")
    q.qed_set_field_grid(g.ctx, dev.data_ptr())
    with pytest.raises(q.QedError) as e:               # zero nodes on an axis
        q.qed_push_and_generate(g.ctx, P, q.make_field(q.QED_FIELD_GRID, (NX, 0, NZ, *LBOX)), w.dt, 1, 0)
    assert e.value.status == q.QED_ERR_INVALID
    rc, _ = q.qed_push_and_generate(g.ctx, P, q.make_field(q.QED_FIELD_GRID, PRM), w.dt, 1, 0)
    assert rc == q.QED_OK
    g.close()
