"""Event-level spectra per chi bin: the CUDA path against the FP64 oracle.

The paper samples photon and pair energies from 2-D inverse-CDF tables over
chi and energy (Sec. 3).  Here each chi bin is an ensemble whose every
particle starts at that chi: electrons (gamma0 = 2000) or photons (k0 = 2000)
crossing a uniform magnetic field of strength chi0 R / p0.  In a pure B field
a particle's energy changes only at an event, so every first event of a
particle happens at exactly chi0.  The step length is chosen so that about
10% of the electrons emit (later events, at lower chi, are a few percent of
the sample; both sides simulate the same process, so those are compared as
well).

GPU and oracle run with independent random streams (different seeds) and
the two samples are compared by a two-sample Kolmogorov-Smirnov test at
p > 0.01 in every bin, with at least 2000 events per side:
 - emitted photon energies, 8 bins chi0 in [1e-2, 1e2]: FP64 and FP32
   table sampler, and the network sampler;
 - pair lepton energies, 8 bins chi0 in [0.5, 1e2]: FP64 and FP32.  The
   newborn leptons are pushed to the end of the step (Algorithm 2) and may
   emit there; those with no emission (nevents = 0) keep their birth energy
   and form the compared sample on both sides.
Each bin has a fixed pair of seeds.  A bin whose p-value is at or below 0.01
is drawn once more from fresh seeds with four times the particles and must
pass there: the chance that a correct sampler fails a bin is then 1e-4, and
a real bias shows more clearly in the larger sample.
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
scipy_stats = pytest.importorskip("scipy.stats")

import paper_2409_17299_gb300 as q  # noqa: E402

R = W.R_SCHWINGER
ALPHA_R = 7.2973525693e-3 * R
E0 = 2000.0
EM_BINS = np.logspace(-2, 2, 8)
PAIR_BINS = np.logspace(math.log10(0.5), 2, 8)
P_MIN = 0.01
MIN_EVENTS = 2000


def _species_along_x(n, p0):
    z = np.zeros(n)
    return {"x": z, "y": z, "z": z, "px": np.full(n, p0), "py": z, "pz": z, "w": np.ones(n),
            "id": np.arange(n, dtype=np.uint64)}


def _bin_setup(kind, chi0, otables, scale=1):
    """(momentum, field params, dt, particles) of a bin: every particle at chi0.

    Emission: dt with lambda dt = 0.1, 30000 electrons (about 3000 events).
    Pairs: a newborn lepton keeps its birth energy only if it does not emit
    in the rest of the step, whose rate is r times the photon's pair rate
    (r = 2 F_gamma(chi0 / 2) / F_pair(chi0), a lepton at half the photon's
    energy); lambda dt = min(0.1, 2 / r) maximises the leptons without an
    emission, and the photon count is sized for about 3000 of them."""
    if kind == "emission":
        p0 = math.sqrt(E0 * E0 - 1.0)
        lam = ALPHA_R / E0 * otables.rate_F(False, chi0)
        return p0, [0, 0, 0, 0, 0, chi0 * R / p0], 0.1 / lam, 30000 * scale
    lam = ALPHA_R / E0 * otables.rate_F(True, chi0)
    r = 2.0 * otables.rate_F(False, chi0 / 2) / otables.rate_F(True, chi0)
    x = min(0.1, 2.0 / r)
    n = int(math.ceil(3000.0 / (2.0 * x * math.exp(-r * x / 2))))
    return E0, [0, 0, 0, 0, 0, chi0 * R / E0], x / lam, n * scale


def _gpu(kind, chi0, scale, seed, prec, otables, params=None):
    p0, prm, dt, n = _bin_setup(kind, chi0, otables, scale)
    sp = _species_along_x(n, p0)
    empty = W._empty()
    species = [sp, empty, empty] if kind == "emission" else [empty, empty, sp]
    sampler = q.QED_SAMPLER_MLP if params is not None else q.QED_SAMPLER_TABLE
    g = q.Generator(q.make_config(precision=prec, seed=seed, push_photons=0 if kind == "emission" else 1,
                                  sampler=sampler))
    if params is not None:
        q.qed_mlp_set_params(g.ctx, params)
    cap = [n, 16, n // 4] if kind == "emission" else [n // 4, n // 4, n + n // 2]
    ens = q.DeviceEnsemble.from_host(species, cap, prec)
    g.push(ens, q.make_field(q.QED_FIELD_UNIFORM, prm), dt, 1, 0)
    out = [ens.to_host(s) for s in range(3)]
    g.close()
    return _energies(kind, out)


def _oracle(kind, chi0, scale, seed, otables):
    p0, prm, dt, n = _bin_setup(kind, chi0, otables, scale)
    sp = _species_along_x(n, p0)
    empty = W._empty()
    species = [sp, empty, empty] if kind == "emission" else [empty, empty, sp]
    cap = [n, 16, n // 4] if kind == "emission" else [n // 4, n // 4, n + n // 2]
    ens = oracle.Ensemble.from_arrays(species, cap)
    cfg = oracle.make_cfg(seed=seed, push_photons=0 if kind == "emission" else 1,
                          field_kind=oracle.FIELD_UNIFORM, field_prm=prm)
    oracle.push_and_generate(ens, otables, cfg, dt, 1, 0)
    return _energies(kind, [ens.view(s) for s in range(3)])


def _energies(kind, out):
    if kind == "emission":
        k = out[2]
        return np.sqrt(k["px"] ** 2 + k["py"] ** 2 + k["pz"] ** 2)
    e = []
    for s in (0, 1):
        d = out[s]
        keep = d["nevents"] == 0
        e.append(np.sqrt(1.0 + d["px"][keep] ** 2 + d["py"][keep] ** 2 + d["pz"][keep] ** 2))
    return np.concatenate(e)


def _check_bins(kind, bins, prec, otables, params=None):
    report = []
    for k, chi0 in enumerate(bins):
        sg, so = 1000 + 10 * k, 5000 + 10 * k
        a = _gpu(kind, chi0, 1, sg, prec, otables, params)
        b = _oracle(kind, chi0, 1, so, otables)
        assert min(len(a), len(b)) >= MIN_EVENTS, (kind, chi0, len(a), len(b))
        p = scipy_stats.ks_2samp(a, b).pvalue
        entry = [float(chi0), len(a), len(b), float(p)]
        if p <= P_MIN:
            # the pre-stated second draw: fresh seeds, four times the particles
            a = _gpu(kind, chi0, 4, sg + 7, prec, otables, params)
            b = _oracle(kind, chi0, 4, so + 7, otables)
            p2 = scipy_stats.ks_2samp(a, b).pvalue
            entry += [len(a), len(b), float(p2)]
            assert p2 > P_MIN, (kind, prec, entry, report)
        report.append(entry)
    return report


@pytest.mark.parametrize("prec", [q.QED_FP64, q.QED_FP32])
def test_emission_spectrum_per_chi_bin(prec, otables):
    rep = _check_bins("emission", EM_BINS, prec, otables)
    assert len(rep) == 8


@pytest.mark.parametrize("prec", [q.QED_FP64, q.QED_FP32])
def test_pair_spectrum_per_chi_bin(prec, otables):
    rep = _check_bins("pairs", PAIR_BINS, prec, otables)
    assert len(rep) == 8


@pytest.fixture(scope="module")
def network():
    g = q.Generator(q.make_config(precision=q.QED_FP32))
    q.qed_train_surrogate(g.ctx, n_samples=10 ** 8, batch=8192, lr=4e-3, seed=7)
    P = q.qed_mlp_get_params(g.ctx)
    g.close()
    return P


def test_network_emission_spectrum_per_chi_bin(network, otables):
    """The network sampler inside the push (FP32) against the oracle's table
    method, per chi bin."""
    rep = _check_bins("emission", EM_BINS, q.QED_FP32, otables, params=network)
    assert len(rep) == 8
