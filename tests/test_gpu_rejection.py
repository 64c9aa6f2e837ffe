"""The GPU's Algorithm 1 (table sampler, FP64 and FP32) against the oracle's
independent subcycled rejection generator (Bessel functions directly, its
own random stream), in uniform B at chi0 = 0.1, 1 and 10 (gamma0 = 1000):
emission counts, photon spectra and electron energies agree within
statistics."""
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

N, STEPS = 2048, 30
NSUB = {0.1: 16, 1.0: 16, 10.0: 64}      # sub-steps per step: acceptance kept below 0.1


def _workload(chi0):
    w = W.uniform_b_emission(n=N, seed=0)
    w.field_prm = list(w.field_prm)
    w.field_prm[5] *= chi0                     # B_z = chi0 R / gamma0
    return w


@pytest.mark.parametrize("chi0", [0.1, 1.0, 10.0])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_algorithm1_matches_rejection_generator(chi0, prec):
    from scipy.stats import ks_2samp
    w = _workload(chi0)
    P = q.QED_FP64 if prec == "fp64" else q.QED_FP32
    g = q.Generator(q.make_config(precision=P, seed=21, push_photons=0))
    ens = q.DeviceEnsemble.from_host(w.species, [N, 1, 16 * N], P)
    st = g.push(ens, q.make_field(w.field_kind, w.field_prm), w.dt, STEPS, 0)
    ph = ens.to_host(2)
    k1 = np.sqrt(ph["px"] ** 2 + ph["py"] ** 2 + ph["pz"] ** 2)
    e = ens.to_host(0)
    ga = np.sqrt(1 + e["px"] ** 2 + e["py"] ** 2 + e["pz"] ** 2)
    g.close()

    b = oracle.Ensemble.from_arrays(w.species, [N, 1, 1])
    cfg = oracle.make_cfg(seed=21, push_photons=0, field_kind=w.field_kind, field_prm=w.field_prm)
    k2, n2, amax = oracle.rejection_run(b, cfg, w.dt, STEPS, NSUB[chi0], seed=99)
    eb = b.view(0)
    gb = np.sqrt(1 + eb["px"] ** 2 + eb["py"] ** 2 + eb["pz"] ** 2)

    n1 = st["emit_events"]
    assert amax < 0.1
    assert abs(n1 - n2) < 5 * math.sqrt(n1 + n2) + 5, (n1, n2)
    assert ks_2samp(k1, k2).pvalue > 0.001
    g0 = math.sqrt(1 + 1000.0 ** 2)
    qa, qb = np.abs(ga - g0) < 1e-3, np.abs(gb - g0) < 1e-3
    f = 0.5 * (qa.mean() + qb.mean())
    assert abs(qa.mean() - qb.mean()) < 5 * math.sqrt(2 * f * (1 - f) / N) + 1e-3
    if (~qa).sum() > 50 and (~qb).sum() > 50:
        assert ks_2samp(ga[~qa], gb[~qb]).pvalue > 0.001
