"""Cascade growth in the shape of the paper's test problem (Sec. 5.1): the
standing circularly polarised wave at a0 = 1557, dt = T/200, electrons at
rest near the electric antinode.  The growth rate Gamma of the lepton count
(N ~ exp(Gamma t)), fitted over the second half of the first period, from
the FP32 mode and from the network sampler must agree with the FP64 table
run's: the paper's criterion for its optimized code is eta_Gamma < 0.5%."""
import math

import numpy as np
import pytest

from paper_2409_17299_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_17299_gb300 as q  # noqa: E402

N_SEED, NSTEPS, FIT_FROM = 2000, 200, 100


def _counts(prec, seed, sampler=q.QED_SAMPLER_TABLE, params=None):
    w = W.standing_wave_cascade(n=N_SEED, seed=seed, a0=1557.0, steps_per_period=200, periods=1, thin_cap=0)
    g = q.Generator(q.make_config(precision=prec, seed=w.seed, push_photons=1, sampler=sampler))
    if params is not None:
        q.qed_mlp_set_params(g.ctx, params)
    ens = q.DeviceEnsemble.from_host(w.species, [64 * N_SEED, 64 * N_SEED, 320 * N_SEED], prec)
    field = q.make_field(w.field_kind, w.field_prm)
    n = []
    for s in range(NSTEPS):
        g.push(ens, field, w.dt, 1, s)
        n.append(ens.count[0] + ens.count[1])
    g.close()
    return np.array(n, dtype=np.float64), w.dt


def _gamma(n, dt):
    """Least-squares slope of ln N against t over steps FIT_FROM..NSTEPS, in
    units of the inverse wave period."""
    t = (np.arange(len(n)) + 1) * dt
    sel = slice(FIT_FROM, len(n))
    slope = np.polyfit(t[sel], np.log(n[sel]), 1)[0]
    return slope * 2 * math.pi


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_growth_rate_fp32_matches_fp64(seed):
    n64, dt = _counts(q.QED_FP64, seed)
    n32, _ = _counts(q.QED_FP32, seed)
    assert n64[-1] > 20 * N_SEED                  # a real cascade: > 20x growth in one period
    g64, g32 = _gamma(n64, dt), _gamma(n32, dt)
    assert g64 > 1.0
    assert abs(g32 / g64 - 1) < 0.005, (g64, g32)


@pytest.fixture(scope="module")
def network():
    g = q.Generator(q.make_config(precision=q.QED_FP32))
    q.qed_train_surrogate(g.ctx, n_samples=10 ** 8, batch=8192, lr=4e-3, seed=7)
    P = q.qed_mlp_get_params(g.ctx)
    g.close()
    return P


def test_growth_rate_network_sampler(network):
    """Over three seeds the network sampler's mean growth rate agrees with the
    FP64 table run's within the paper's 0.5%, and each seed within 2%."""
    rel = []
    for seed in (4, 5, 6):
        n64, dt = _counts(q.QED_FP64, seed)
        nm, _ = _counts(q.QED_FP32, seed, sampler=q.QED_SAMPLER_MLP, params=network)
        rel.append(_gamma(nm, dt) / _gamma(n64, dt) - 1)
    assert max(abs(r) for r in rel) < 0.02, rel
    assert abs(np.mean(rel)) < 0.005, rel
