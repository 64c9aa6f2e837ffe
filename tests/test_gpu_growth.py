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


# ---------------------------------------------------------------------------
# The test problem at the paper's own scale (Sec. 5.1): 2.5e5 seed electrons
# and positrons at rest filling the box, a0 = 1557, dt = T/200, 5 T with
# global leveling, five seeds per mode.  Sec. 5.2's bound eta_Gamma < 0.5%
# applies to the mean growth rate of the FP32 mode and of the network sampler
# against the FP64 table mode; the lepton density profiles along x agree.
# The FP64 runs are tied to the oracle: at a step inside the fitted window,
# particles sampled from the FP64 state are pushed one by one by the oracle.
# ---------------------------------------------------------------------------
import bench  # noqa: E402
import oracle  # noqa: E402

TIE_STEP = 800


def _tie_to_oracle(otables, store):
    """hook for growth_run: before TIE_STEP, push a copy of the whole state one
    step without leveling and keep it with a sample of the state."""
    def hook(s, gen, ens, w, field):
        if s != TIE_STEP:
            return
        rng = np.random.default_rng(3)
        caps = list(ens.capacity)
        work = q.DeviceEnsemble(caps, q.QED_FP64)
        for k in range(3):
            for f, a in ens.arr[k].items():
                work.arr[k][f].copy_(a)
        work.count = list(ens.count)
        size = [1000, 1000, 10000]
        picks = [np.sort(rng.choice(ens.count[k], size=min(size[k], ens.count[k]), replace=False)) for k in range(3)]
        start = []
        for k in range(3):
            d = ens.arr[k]
            ii = torch.as_tensor(picks[k], dtype=torch.int64, device="cuda")
            o = {f: d[f].index_select(0, ii).double().cpu().numpy() for f in ("x", "y", "z", "px", "py", "pz", "w")}
            o["id"] = d["id"].index_select(0, ii).cpu().numpy().view(np.uint64)
            o["nevents"] = d["nevents"].index_select(0, ii).cpu().numpy().view(np.uint32)
            start.append(o)
        g0 = q.Generator(q.make_config(precision=q.QED_FP64, seed=w.seed, push_photons=1, thin_cap=0))
        g0.push(work, field, w.dt, 1, s)
        g0.close()
        oe = oracle.Ensemble.from_arrays(start, [100000, 100000, 400000])
        cfg = oracle.make_cfg(seed=w.seed, push_photons=1, thin_cap=0, field_kind=w.field_kind,
                              field_prm=w.field_prm)
        oracle.push_and_generate(oe, otables, cfg, w.dt, 1, s)
        store["work"], store["oracle"] = [work.to_host(k) for k in range(3)], [oe.view(k) for k in range(3)]
    return hook


@pytest.fixture(scope="module")
def paper_runs(network, otables):
    store = {}
    runs = {"fp64": [bench.growth_run("fp64", sd, hook=_tie_to_oracle(otables, store) if sd == 11 else None)
                     for sd in bench.GROWTH_SEEDS],
            "fp32": [bench.growth_run("fp32", sd) for sd in bench.GROWTH_SEEDS],
            "net": [bench.growth_run("fp32", sd, mlp_params=network) for sd in bench.GROWTH_SEEDS]}
    return runs, store


def test_paper_test_problem_growth_rate(paper_runs):
    runs, _ = paper_runs
    s64 = bench.growth_summary(runs["fp64"])
    assert s64["gamma_mean"] > 1.0                       # an exponential cascade (per period)
    for mode in ("fp32", "net"):
        s = bench.growth_summary(runs[mode])
        eta = s["gamma_mean"] / s64["gamma_mean"] - 1
        assert abs(eta) < 0.005, (mode, eta, s["gamma_per_period"], s64["gamma_per_period"])
        per_seed = np.array(s["gamma_per_period"]) / np.array(s64["gamma_per_period"]) - 1
        assert np.max(np.abs(per_seed)) < 0.02, (mode, per_seed)


def test_paper_test_problem_density_profile(paper_runs):
    runs, _ = paper_runs
    p64 = np.array(bench.growth_summary(runs["fp64"])["profile_mean"])
    assert p64.max() > 2.0 / bench.GROWTH_BINS            # the cascade concentrates leptons
    for mode in ("fp32", "net"):
        p = np.array(bench.growth_summary(runs[mode])["profile_mean"])
        assert np.abs(p - p64).sum() < 0.02, (mode, np.abs(p - p64).sum())


def test_paper_test_problem_fp64_step_matches_oracle(paper_runs):
    """At step 800 of the FP64 run (inside the fitted window, at the cap):
    every particle the oracle produces from the sampled ones is found by id
    in the GPU's state after the same step, with equal event counts and
    momenta and positions within 1e-9."""
    _, store = paper_runs
    total = found = 0
    for k in range(3):
        o, g = store["oracle"][k], store["work"][k]
        order = np.argsort(g["id"])
        gid = g["id"][order]
        at = np.searchsorted(gid, o["id"])
        hit = (at < len(gid)) & (gid[np.minimum(at, len(gid) - 1)] == o["id"])
        total += len(o["id"])
        found += int(hit.sum())
        m = order[at[hit]]
        assert np.array_equal(g["nevents"][m], o["nevents"][hit]), k
        for keys in (("px", "py", "pz"), ("x", "y", "z")):
            a = np.stack([g[f][m] for f in keys], 1)
            b = np.stack([o[f][hit] for f in keys], 1)
            err = np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-3)
            assert err.max() <= 1e-9, (k, keys, err.max())
    assert total > 10000 and found == total, (found, total)


def test_paper_test_problem_20_periods(network):
    """The paper's long runs (20 T; Sec. 5.1), four seeds per mode: the mean
    growth rates, fitted from 3.5 T to 20 T, of the FP32 mode and of the
    network sampler within Sec. 5.2's 0.5% of the FP64 mode's.  (Runs of one
    seed in two modes follow each other for about 1000 steps, then become
    independent realizations whose single-seed rates scatter by ~0.3%; the
    bound is on the means.)"""
    seeds = bench.GROWTH_SEEDS[:4]
    g64 = np.array([bench.growth_run("fp64", s, periods=20, fit=bench.GROWTH_FIT_20T)["gamma"] for s in seeds])
    assert g64.min() > 1.0
    for kw in ({}, {"mlp_params": network}):
        g = np.array([bench.growth_run("fp32", s, periods=20, fit=bench.GROWTH_FIT_20T, **kw)["gamma"]
                      for s in seeds])
        eta = g.mean() / g64.mean() - 1
        assert abs(eta) < 0.005, (list(kw), eta, g.tolist(), g64.tolist())
