"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Bars (written in each test): Philox and per-particle event counts bit-exact;
FP64 momenta within 1e-5 relative (observed ~1e-12); FP32 (FP64 sub-step clock)
within 1e-3 relative on particles whose event sequence matches, with the
fraction of mismatching particles bounded; spectra by two-sample KS.
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


@pytest.fixture(scope="module")
def gen64():
    from paper_2409_17299_gb300 import build
    build.build()
    g = q.Generator(q.make_config(precision=q.QED_FP64, seed=0))
    yield g
    g.close()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda").contiguous()


# ---------------------------------------------------------------------------
# components
# ---------------------------------------------------------------------------
def test_philox_bit_exact():
    rng = np.random.default_rng(0)
    n = 1 << 20
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [1, 2, 3, 4], [0, 0, 0xFFFFFFFF, 0xFFFFFFFF]]
    for key in (0, 0xC0FFEE, 0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF):
        dctr = torch.from_numpy(ctr.view(np.int32)).cuda()
        dout = torch.empty_like(dctr)
        q.qed_philox(dctr.data_ptr(), n, key, dout.data_ptr(), torch.cuda.current_stream().cuda_stream)
        got = dout.cpu().numpy().view(np.uint32).reshape(n, 4)
        want = oracle.philox(ctr, [key & 0xFFFFFFFF, key >> 32])
        assert np.array_equal(got, want)


def test_philox_empty_and_misaligned():
    q.qed_philox(0, 0, 0, 0)
    buf = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(q.QedError):
        q.qed_philox(buf.data_ptr() + 4, 1, 0, buf.data_ptr())


def test_tables_match_oracle(gen64, otables):
    ce, cp = np.zeros(66), np.zeros(55)
    ie, ip = np.zeros(121 * 257), np.zeros(101 * 129)
    q.qed_get_tables(gen64.ctx, ce.ctypes.data, cp.ctypes.data, ie.ctypes.data, ip.ctypes.data)
    # both sides build the same mathematical objects with independent quadrature
    assert np.allclose(ce, otables.cheb_em, rtol=0, atol=1e-11 * np.abs(otables.cheb_em).max())
    assert np.allclose(cp, otables.cheb_pair, rtol=0, atol=1e-10 * np.abs(otables.cheb_pair).max())
    assert np.max(np.abs(ie - otables.icdf_em)) < 1e-9
    assert np.max(np.abs(ip - otables.icdf_pair)) < 1e-9


@pytest.mark.parametrize("prec,tol", [(q.QED_FP64, 1e-11), (q.QED_FP32, 3e-5)])
def test_rate_approximant(prec, tol, otables):
    g = q.Generator(q.make_config(precision=prec))
    chi = np.concatenate([np.logspace(-5, 5, 4001), [0.0, 1e-3, 1e3, 0.01, 0.0099]])
    dchi = _dev(chi)
    F = torch.empty_like(dchi)
    for is_ph in (0, 1):
        q.qed_eval_rate(g.ctx, is_ph, dchi.data_ptr(), len(chi), F.data_ptr())
        got = F.cpu().numpy()
        want = np.array([otables.rate_F(is_ph, c) for c in chi])
        nz = want > 1e-30               # FP32 flushes rates below ~1e-38 to zero
        chk = nz | (want == 0)
        assert np.all((got[chk] == 0) == (want[chk] == 0)), "zero pattern"
        assert np.max(np.abs(got[nz] / want[nz] - 1)) < tol
    g.close()


@pytest.mark.parametrize("prec,tol", [(q.QED_FP64, 1e-10), (q.QED_FP32, 1e-4)])
def test_inverse_cdf_sampler(prec, tol, otables):
    g = q.Generator(q.make_config(precision=prec))
    rng = np.random.default_rng(5)
    n = 20000
    chi = 10 ** rng.uniform(-4, 4, n)
    u = rng.random(n)
    u[:4] = [2.0 ** -30, 0.5, 1 - 2.0 ** -20, 0.25]
    dchi, du = _dev(chi), _dev(u)
    d, om = torch.empty_like(dchi), torch.empty_like(dchi)
    for is_ph in (0, 1):
        q.qed_sample(g.ctx, is_ph, dchi.data_ptr(), du.data_ptr(), n, d.data_ptr(), om.data_ptr())
        gd, gom = d.cpu().numpy(), om.cpu().numpy()
        ref = [otables.sample_pair(c, x) if is_ph else otables.sample_emission(c, x) for c, x in zip(chi, u)]
        wd = np.array([r[0] for r in ref])
        wom = np.array([r[1] for r in ref])
        assert np.all((gd > 0) & (gd < 1))
        assert np.max(np.abs(gd / wd - 1)) < tol * 10
        assert np.max(np.abs(gom / wom - 1)) < tol * 10
        assert np.median(np.abs(gd / wd - 1)) < tol
    g.close()


# ---------------------------------------------------------------------------
# full steps
# ---------------------------------------------------------------------------
def run_gpu(w, prec, nsteps=None, capacity=None, thin_cap=None, gen=None, step0=0):
    cap = capacity or [max(64, 4 * len(s["id"])) for s in w.species]
    g = gen or q.Generator(q.make_config(precision=prec, seed=w.seed, push_photons=w.push_photons,
                                         thin_cap=w.thin_cap if thin_cap is None else thin_cap))
    ens = q.DeviceEnsemble.from_host(w.species, cap, prec)
    st = g.push(ens, q.make_field(w.field_kind, w.field_prm), w.dt, w.nsteps if nsteps is None else nsteps, step0)
    torch.cuda.synchronize()
    out = [ens.to_host(s) for s in range(3)]
    if gen is None:
        g.close()
    return out, st


def run_oracle(w, otables, nsteps=None, capacity=None, thin_cap=None, step0=0):
    cap = capacity or [max(64, 4 * len(s["id"])) for s in w.species]
    ens = oracle.Ensemble.from_arrays(w.species, cap)
    cfg = oracle.make_cfg(seed=w.seed, push_photons=w.push_photons,
                          thin_cap=w.thin_cap if thin_cap is None else thin_cap,
                          field_kind=w.field_kind, field_prm=w.field_prm)
    st = oracle.push_and_generate(ens, otables, cfg, w.dt, w.nsteps if nsteps is None else nsteps, step0)
    return [ens.view(s) for s in range(3)], st


def by_id(d):
    o = np.argsort(d["id"])
    return {k: v[o] for k, v in d.items()}


def assert_same_fp64(g, o, rtol=1e-5, what=""):
    assert len(g["id"]) == len(o["id"]), (what, len(g["id"]), len(o["id"]))
    if len(o["id"]) == 0:
        return
    g, o = by_id(g), by_id(o)
    assert np.array_equal(g["id"], o["id"]), what
    assert np.array_equal(g["nevents"], o["nevents"]), what
    # relative error of the momentum and position vectors (component-wise
    # relative errors blow up for components that pass through zero)
    for keys, floor in ((("px", "py", "pz"), 1e-3), (("x", "y", "z"), 1e-3)):
        gv = np.stack([g[k] for k in keys], 1)
        ov = np.stack([o[k] for k in keys], 1)
        err = np.linalg.norm(gv - ov, axis=1) / np.maximum(np.linalg.norm(ov, axis=1), floor)
        assert err.max() < rtol, (what, keys, err.max())
    assert np.allclose(g["w"], o["w"], rtol=1e-12, atol=0), what


@pytest.mark.parametrize("n,nsteps", [(1, 3), (33, 20), (1025, 10)])
def test_emission_fp64_ragged_sizes(n, nsteps, otables):
    w = W.uniform_b_emission(n=n, seed=3, nsteps=nsteps)
    g, gs = run_gpu(w, q.QED_FP64)
    o, os_ = run_oracle(w, otables)
    assert gs["emit_events"] == os_["emit_events"]
    assert gs["particle_steps"] == os_["particle_steps"] == n * nsteps
    for s in range(3):
        assert_same_fp64(g[s], o[s], what="species %d" % s)


def test_empty_ensemble(otables):
    w = W.uniform_b_emission(n=1, seed=0, nsteps=2)
    w.species[0] = W._empty()
    g, gs = run_gpu(w, q.QED_FP64, capacity=[8, 8, 8])
    assert gs["particle_steps"] == 0 and gs["emit_events"] == 0
    assert all(len(x["id"]) == 0 for x in g)


def test_emission_full_size_fp64(otables):
    """The uniform-B emission workload at full size: 16384 electrons, 200 steps,
    chi0 = 1, photons recorded (bit-exact event counts, momenta 1e-5)."""
    w = W.uniform_b_emission(n=16384, seed=0)
    g, gs = run_gpu(w, q.QED_FP64, capacity=[16384, 8, 400000])
    o, os_ = run_oracle(w, otables, capacity=[16384, 8, 400000])
    assert gs["emit_events"] == os_["emit_events"]
    assert gs["particle_steps"] == os_["particle_steps"]
    assert_same_fp64(g[0], o[0], what="electrons")
    assert_same_fp64(g[2], o[2], what="photons")


def test_cascade_fp64_rotating_field(otables):
    w = W.rotating_e_cascade(n=600, seed=1, periods=1)
    g, gs = run_gpu(w, q.QED_FP64, nsteps=60, capacity=[20000, 20000, 60000])
    o, os_ = run_oracle(w, otables, nsteps=60, capacity=[20000, 20000, 60000])
    assert os_["pair_events"] > 0
    assert (gs["emit_events"], gs["pair_events"], gs["particle_steps"]) == \
        (os_["emit_events"], os_["pair_events"], os_["particle_steps"])
    for s in range(3):
        assert_same_fp64(g[s], o[s], what="species %d" % s)


def test_cascade_fp64_standing_wave(otables):
    w = W.standing_wave_cascade(n=400, seed=4, periods=1)
    g, gs = run_gpu(w, q.QED_FP64, nsteps=40, capacity=[20000, 20000, 60000])
    o, os_ = run_oracle(w, otables, nsteps=40, capacity=[20000, 20000, 60000])
    assert (gs["emit_events"], gs["pair_events"]) == (os_["emit_events"], os_["pair_events"])
    for s in range(3):
        assert_same_fp64(g[s], o[s], what="species %d" % s)


def test_overflow_restores_and_replays(otables):
    w = W.rotating_e_cascade(n=300, seed=1, periods=1)
    big, _ = run_gpu(w, q.QED_FP64, nsteps=30, capacity=[20000, 20000, 60000])
    # raw ABI: too small a photon buffer -> QED_ERR_CAPACITY with the state put back
    gen = q.Generator(q.make_config(precision=q.QED_FP64, seed=w.seed, push_photons=1))
    ens = q.DeviceEnsemble.from_host(w.species, [20000, 20000, 16], q.QED_FP64)
    before = ens.to_host(0)
    P = ens.struct()
    rc, st = q.qed_push_and_generate(gen.ctx, P, q.make_field(w.field_kind, w.field_prm), w.dt, 30, 0)
    assert rc == q.QED_ERR_CAPACITY and st["overflow"] == 1 and st["needed_capacity"][2] > 16
    ens.pull_counts(P)
    after = ens.to_host(0)
    assert ens.count == [300, 0, 0]
    for f in before:
        assert np.array_equal(before[f], after[f])
    # grow and replay: identical to the large-capacity run
    gen.push(ens, q.make_field(w.field_kind, w.field_prm), w.dt, 30, 0)
    for s in range(3):
        a, b = by_id(big[s]), by_id(ens.to_host(s))
        for f in a:
            assert np.array_equal(a[f], b[f]), (s, f)
    gen.close()


def test_thinning_fp64_matches_oracle(otables):
    w = W.rotating_e_cascade(n=500, seed=1, periods=1)
    cap = 700
    g, gs = run_gpu(w, q.QED_FP64, nsteps=50, capacity=[20000, 20000, 60000], thin_cap=cap)
    o, os_ = run_oracle(w, otables, nsteps=50, capacity=[20000, 20000, 60000], thin_cap=cap)
    assert any(len(x["id"]) > 0.8 * cap for x in o)
    for s in range(3):
        assert len(g[s]["id"]) <= cap * 1.2 + 100
        assert_same_fp64(g[s], o[s], what="species %d" % s)


def test_fp32_against_fp64_oracle(otables):
    """FP32 storage/push/rates/sampling (FP64 sub-step clock): momenta within
    1e-3 of the FP64 oracle for particles whose event count matches; at most
    1% of particles may take a different event sequence after 20 steps."""
    w = W.uniform_b_emission(n=16384, seed=0, nsteps=20)
    g, gs = run_gpu(w, q.QED_FP32, capacity=[16384, 8, 100000])
    o, os_ = run_oracle(w, otables, capacity=[16384, 8, 100000])
    a, b = by_id(g[0]), by_id(o[0])
    assert np.array_equal(a["id"], b["id"])
    same = a["nevents"] == b["nevents"]
    assert same.mean() > 0.99, same.mean()
    pa = np.stack([a[k][same] for k in ("px", "py", "pz")], 1)
    pb = np.stack([b[k][same] for k in ("px", "py", "pz")], 1)
    rel = np.linalg.norm(pa - pb, axis=1) / np.linalg.norm(pb, axis=1)
    assert rel.max() < 1e-3, rel.max()
    assert abs(gs["emit_events"] - os_["emit_events"]) < 5 * math.sqrt(os_["emit_events"])
    # photon spectrum: two-sample KS between GPU FP32 and the oracle
    from scipy.stats import ks_2samp
    ka = np.sqrt(g[2]["px"] ** 2 + g[2]["py"] ** 2 + g[2]["pz"] ** 2)
    kb = np.sqrt(o[2]["px"] ** 2 + o[2]["py"] ** 2 + o[2]["pz"] ** 2)
    assert ks_2samp(ka, kb).pvalue > 0.01


def test_fp32_cascade_statistics(otables):
    w = W.rotating_e_cascade(n=3000, seed=1, periods=1)
    g, gs = run_gpu(w, q.QED_FP32, nsteps=60, capacity=[100000, 100000, 300000])
    o, os_ = run_oracle(w, otables, nsteps=60, capacity=[100000, 100000, 300000])
    for key in ("emit_events", "pair_events"):
        assert abs(gs[key] - os_[key]) < 6 * math.sqrt(os_[key]) + 5, key
    from scipy.stats import ks_2samp
    for s in range(3):
        ea = np.sqrt(g[s]["px"] ** 2 + g[s]["py"] ** 2 + g[s]["pz"] ** 2)
        eb = np.sqrt(o[s]["px"] ** 2 + o[s]["py"] ** 2 + o[s]["pz"] ** 2)
        assert ks_2samp(ea, eb).pvalue > 0.01, s


def _chi_cases(rng, n):
    """Random momenta and fields, plus cancelling geometries: a lepton or
    photon co-moving with a plane wave (E = a y, B = a z, p along x), and E
    parallel to B (standing circularly polarised wave)."""
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p = d * 10 ** rng.uniform(-2, 4, (n, 1))
    E = rng.normal(size=(n, 3)) * 10 ** rng.uniform(0, 3.5, (n, 1))
    B = rng.normal(size=(n, 3)) * 10 ** rng.uniform(0, 3.5, (n, 1))
    m = n // 8
    a = 10 ** rng.uniform(1, 3.5, m)
    P = 10 ** rng.uniform(0, 3.5, m)
    p[:m] = np.stack([P, 1e-3 * rng.normal(size=m), np.zeros(m)], 1)
    E[:m] = np.stack([np.zeros(m), a, np.zeros(m)], 1)
    B[:m] = np.stack([np.zeros(m), np.zeros(m), a], 1)
    u = rng.normal(size=(m, 3))
    E[m:2 * m] = u * a[:, None]
    B[m:2 * m] = u * (0.7 * a)[:, None]
    return p, E, B


def _chi_exact(p, E, B, photon):
    """50-digit decimal evaluation of the direct form on the given doubles."""
    from decimal import Decimal as D, getcontext
    getcontext().prec = 50
    R = D(W.R_SCHWINGER)
    out, cf = [], []
    for pi, Ei, Bi in zip(p, E, B):
        pv = [D(float(v)) for v in pi]
        Ev = [D(float(v)) for v in Ei]
        Bv = [D(float(v)) for v in Bi]
        p2 = sum(v * v for v in pv)
        e0 = p2.sqrt() if photon else (1 + p2).sqrt()
        cx = [pv[1] * Bv[2] - pv[2] * Bv[1], pv[2] * Bv[0] - pv[0] * Bv[2], pv[0] * Bv[1] - pv[1] * Bv[0]]
        u = [e0 * Ev[i] + cx[i] for i in range(3)]
        s = sum(pv[i] * Ev[i] for i in range(3))
        uu = sum(v * v for v in u)
        qq = uu - s * s
        out.append(float(max(qq, D(0)).sqrt() / R))
        # condition number of the direct form: magnitudes of all terms over the result
        mag = [abs(e0 * Ev[0]) + abs(pv[1] * Bv[2]) + abs(pv[2] * Bv[1]),
               abs(e0 * Ev[1]) + abs(pv[2] * Bv[0]) + abs(pv[0] * Bv[2]),
               abs(e0 * Ev[2]) + abs(pv[0] * Bv[1]) + abs(pv[1] * Bv[0])]
        sm = sum(abs(pv[i] * Ev[i]) for i in range(3))
        cf.append(float((sum(m * m for m in mag) + sm * sm) / qq) if qq > 0 else float("inf"))
    return np.array(out), np.array(cf)


@pytest.mark.parametrize("prec", [q.QED_FP64, q.QED_FP32])
@pytest.mark.parametrize("photon", [False, True])
def test_chi_against_exact(prec, photon):
    """chi in FP64 mode and in FP32 mode (FP32 split S + T with FP64 fallback)
    against a 50-digit evaluation on the same (rounded) inputs.  Bound: the
    mode's rounding plus the FP64 cancellation loss ~2^-52 c of the direct form,
    c = (sum_i (sum of |terms of u_i|)^2 + (sum |p_i E_i|)^2) / chi^2 R^2."""
    rng = np.random.default_rng(17 + photon)
    n = 4000
    p, E, B = _chi_cases(rng, n)
    if prec == q.QED_FP32:
        p, E, B = (a.astype(np.float32).astype(np.float64) for a in (p, E, B))
    g = q.Generator(q.make_config(precision=prec))
    dp, dE, dB = _dev(p.ravel()), _dev(E.ravel()), _dev(B.ravel())
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    n64 = q.qed_eval_chi(g.ctx, photon, dp.data_ptr(), dE.data_ptr(), dB.data_ptr(), n, out.data_ptr())
    got = out.cpu().numpy()
    want, cf = _chi_exact(p, E, B, photon)
    base = 1e-13 if prec == q.QED_FP64 else 6e-6
    ok = want > 0
    rel = np.abs(got[ok] - want[ok]) / want[ok]
    bound = base + 4e-16 * cf[ok]
    assert np.all(rel <= bound), (rel / bound).max()
    assert np.all(np.abs(got[~ok]) <= 1e-7 * np.linalg.norm(E[~ok], axis=1))
    if prec == q.QED_FP32:
        assert n64 >= (n // 8) * 0.9          # the co-moving cases fell back to FP64
        assert n64 <= n // 4                  # the rest stayed in FP32
    g.close()


@pytest.mark.parametrize("weights", ["classes", "lognormal"])
def test_leveling_matches_oracle(weights):
    """qed_compact with a cap: the survivor set and the new weights equal the
    oracle's.  "classes" has 5 distinct weights (class path); "lognormal"
    has ~1e5 distinct weights (histogram path)."""
    rng = np.random.default_rng(9)
    n, cap = 100000, 30000
    if weights == "classes":
        w = rng.choice([0.5, 1.0, 1.25, 2.0, 7.0], size=n)
    else:
        w = np.exp(rng.normal(size=n))
    w[::11] = 0.0                                    # a few dead entries as well
    sp = {"x": rng.normal(size=n), "y": rng.normal(size=n), "z": rng.normal(size=n),
          "px": rng.normal(size=n), "py": rng.normal(size=n), "pz": rng.normal(size=n), "w": w,
          "id": rng.permutation(10 * n)[:n].astype(np.uint64)}
    g = q.Generator(q.make_config(precision=q.QED_FP64, seed=9, thin_cap=cap))
    e = q.DeviceEnsemble.from_host([sp, W._empty(), W._empty()], [n, 1, 1], q.QED_FP64)
    g.compact(e, 17)
    got = by_id(e.to_host(0))
    oe = oracle.Ensemble.from_arrays([sp, None, None], [n, 1, 1])
    oracle.compact(oe, 0)
    oracle.level(oe, 0, cap, seed=9, step=17)
    want = by_id(oe.view(0))
    assert np.array_equal(got["id"], want["id"])
    assert np.allclose(got["w"], want["w"], rtol=1e-14, atol=0)
    for f in ("x", "px", "nevents"):
        assert np.array_equal(got[f], want[f])
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sharded_leveling_matches_oracle(prec):
    """One species split in three device shards (as on three GPUs): shard
    sums from qed_level_eval, added on the host, the library's iteration
    step, then qed_level_apply per shard.  The union of the survivors and
    their weights equal the oracle's leveling of the whole species."""
    rng = np.random.default_rng(21)
    n, cap = 90000, 25000
    w = np.exp(rng.normal(size=n))
    w[::13] = 0.0
    P = q.QED_FP64 if prec == "fp64" else q.QED_FP32
    if P == q.QED_FP32:
        w = w.astype(np.float32).astype(np.float64)
    sp = {"x": rng.normal(size=n), "y": rng.normal(size=n), "z": rng.normal(size=n),
          "px": rng.normal(size=n), "py": rng.normal(size=n), "pz": rng.normal(size=n), "w": w,
          "id": rng.permutation(10 * n)[:n].astype(np.uint64)}
    g = q.Generator(q.make_config(precision=P, seed=9))
    cuts = [0, 20000, 61000, n]
    shards = []
    for a, b in zip(cuts[:-1], cuts[1:]):
        part = {k: v[a:b] for k, v in sp.items()}
        shards.append(q.DeviceEnsemble.from_host([part, W._empty(), W._empty()], [b - a, 1, 1], P))

    def evaluate(at):
        vals = [q.qed_level_eval(g.ctx, e.struct().s[0], 0, at) for e in shards]
        return (sum(v[0] for v in vals), sum(v[1] for v in vals), sum(v[2] for v in vals),
                max(v[3] for v in vals))
    st = q.level_threshold_sharded(evaluate, lambda v: v, cap)
    want_ws = oracle.level_threshold(w, cap)
    assert st.wstar == pytest.approx(want_ws, rel=1e-14)
    for e in shards:
        arr = e.struct()
        q.qed_level_apply(g.ctx, arr, 0, st.wstar, 17)
        e.pull_counts(arr)
    got = [e.to_host(0) for e in shards]
    got = by_id({k: np.concatenate([d[k] for d in got]) for k in got[0]})
    oe = oracle.Ensemble.from_arrays([sp, None, None], [n, 1, 1])
    oracle.compact(oe, 0)
    oracle.level(oe, 0, cap, seed=9, step=17)
    want = by_id(oe.view(0))
    assert np.array_equal(got["id"], want["id"])
    rtol = 1e-14 if P == q.QED_FP64 else 2 ** -23
    assert np.allclose(got["w"], want["w"], rtol=rtol, atol=0)
    assert np.array_equal(got["x"] if P == q.QED_FP64 else got["x"].astype(np.float32),
                          want["x"] if P == q.QED_FP64 else want["x"].astype(np.float32))
    g.close()
