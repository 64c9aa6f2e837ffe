"""Batched, step-fused push (many independent ensembles in one launch):
parity with the oracle run ensemble by ensemble, autotuner safety, and
equality with the per-step path."""
import ctypes as C

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


def _batch(sizes, seed=2, nsteps=20):
    ws = W.batched_uniform_b(n_ens=len(sizes), seed=seed, nsteps=nsteps)
    out = []
    id0 = 0
    for w, n in zip(ws, sizes):
        n = min(n, len(w.species[0]["id"]))
        sub = W.subset(w, 0, slice(0, n))
        sub.species[0]["id"] = np.arange(id0, id0 + n, dtype=np.uint64)
        id0 += n
        out.append(sub)
    return out


def _device(ws, prec, ph_factor=10.0):
    ens = []
    for w in ws:
        n = len(w.species[0]["id"])
        ens.append(q.DeviceEnsemble.from_host(w.species, [n, 1, int(n * w.nsteps * 0.3 * ph_factor) + 64], prec))
    arr = (q.QedParticles * len(ens))()
    fields = (q.QedFieldDesc * len(ens))()
    for k, (e, w) in enumerate(zip(ens, ws)):
        arr[k] = e.struct()
        fields[k] = q.make_field(w.field_kind, w.field_prm)
    return ens, arr, fields


def _pull(ens, arr):
    for k, e in enumerate(ens):
        e.pull_counts(arr[k])


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_batch_fp64_matches_oracle(threads, otables):
    ws = _batch([1, 33, 300, 1025, 2000], nsteps=20)
    g = q.Generator(q.make_config(precision=q.QED_FP64, seed=2, push_photons=0, block_threads=threads))
    ens, arr, fields = _device(ws, q.QED_FP64)
    rc, st = q.qed_batch_push(g.ctx, arr, fields, ws[0].dt, 20, 0)
    assert rc == q.QED_OK
    _pull(ens, arr)
    torch.cuda.synchronize()
    tot_ev = 0
    for e, w in zip(ens, ws):
        n = len(w.species[0]["id"])
        oe = oracle.Ensemble.from_arrays(w.species, [n, 1, int(n * 20 * 3) + 64])
        cfg = oracle.make_cfg(seed=2, push_photons=0, field_kind=w.field_kind, field_prm=w.field_prm)
        ost = oracle.push_and_generate(oe, otables, cfg, w.dt, 20, 0)
        tot_ev += ost["emit_events"]
        assert_same_fp64(e.to_host(0), oe.view(0), what="leptons")
        assert_same_fp64(e.to_host(2), oe.view(2), what="photons")
    assert st["emit_events"] == tot_ev
    assert st["particle_steps"] == 20 * sum(len(w.species[0]["id"]) for w in ws)
    g.close()


def test_autotuner_leaves_buffers_and_picks_a_shape():
    ws = _batch([500, 4000, 20000, 100000], nsteps=10)
    g = q.Generator(q.make_config(precision=q.QED_FP32, seed=2, push_photons=0))
    ens, arr, fields = _device(ws, q.QED_FP32)
    before = [e.to_host(0) for e in ens]
    chosen, ms = q.qed_autotune_batch(g.ctx, arr, fields, ws[0].dt, 4)
    assert chosen in (128, 256, 512) and all(m > 0 for m in ms)
    threads, budget = q.qed_batch_shape(g.ctx)
    assert threads == chosen and budget in (1, 2, 4)
    for e, b in zip(ens, before):
        a = e.to_host(0)
        for f in b:
            assert np.array_equal(a[f], b[f])
        assert e.count[2] == 0
    # tuned shape and the default shape give the same ensembles
    rc, _ = q.qed_batch_push(g.ctx, arr, fields, ws[0].dt, 10, 0)
    _pull(ens, arr)
    g2 = q.Generator(q.make_config(precision=q.QED_FP32, seed=2, push_photons=0, block_threads=256))
    ens2, arr2, fields2 = _device(ws, q.QED_FP32)
    q.qed_batch_push(g2.ctx, arr2, fields2, ws[0].dt, 10, 0)
    _pull(ens2, arr2)
    _assert_shapes_agree(ens, ens2, "fp32")
    g.close()
    g2.close()


def _assert_shapes_agree(ens_a, ens_b, prec):
    """Two runs of the same ensembles with different block shapes.  The
    shapes are separate instantiations of the fused kernel and the compiler
    may contract multiply-adds differently in each, so results can differ in
    the last bits, and a last-bit change can move a waiting-time decision.
    Required: the same leptons, the same event count for nearly all of them,
    and momenta agreeing to the precision's rounding where the counts agree."""
    rtol = 1e-11 if prec == "fp64" else 1e-4
    tot = agree = 0
    for e1, e2 in zip(ens_a, ens_b):
        a, b = by_id(e1.to_host(0)), by_id(e2.to_host(0))
        assert np.array_equal(a["id"], b["id"])
        same_n = a["nevents"] == b["nevents"]
        pa = np.stack([a["px"], a["py"], a["pz"]], 1)
        pb = np.stack([b["px"], b["py"], b["pz"]], 1)
        close = np.linalg.norm(pa - pb, axis=1) <= rtol * np.linalg.norm(pb, axis=1) + 1e-9
        assert np.all(close[same_n]), (prec, np.count_nonzero(~close[same_n]))
        tot += len(same_n)
        agree += int(same_n.sum())
    assert agree >= (0.999 if prec == "fp64" else 0.995) * tot, (prec, agree, tot)


def _assert_shapes_identical(ens_a, ens_b):
    """FP64: every field of every lepton and photon bit for bit."""
    for e1, e2 in zip(ens_a, ens_b):
        for s in (0, 2):
            a, b = by_id(e1.to_host(s)), by_id(e2.to_host(s))
            assert len(a["id"]) == len(b["id"]), s
            for f in a:
                assert np.array_equal(a[f], b[f]), (s, f)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_block_shapes_agree(prec):
    """The three block shapes of the fused kernel on the same ensembles: in
    FP64 bit for bit (the step arithmetic has one inlined copy per
    instantiation, computed in the same order); in FP32 to rounding (see
    _assert_shapes_agree)."""
    ws = _batch([700, 5000, 20000], nsteps=10)
    P = q.QED_FP64 if prec == "fp64" else q.QED_FP32
    res = {}
    for nt in (128, 256, 512):
        g = q.Generator(q.make_config(precision=P, seed=5, push_photons=0, block_threads=nt))
        ens, arr, fields = _device(ws, P)
        rc, _ = q.qed_batch_push(g.ctx, arr, fields, ws[0].dt, 10, 0)
        assert rc == q.QED_OK
        _pull(ens, arr)
        res[nt] = ens
        g.close()
    for nt in (128, 512):
        if prec == "fp64":
            _assert_shapes_identical(res[nt], res[256])
        else:
            _assert_shapes_agree(res[nt], res[256], prec)
        # photons: the same number recorded, to within the rare split events
        for ea, eb in zip(res[nt], res[256]):
            assert abs(ea.count[2] - eb.count[2]) <= 2 + 0.005 * eb.count[2]


def test_batch_fp32_equals_per_step_calls():
    ws = _batch([3000, 7000], nsteps=15)
    g = q.Generator(q.make_config(precision=q.QED_FP32, seed=2, push_photons=0, block_threads=256))
    ens, arr, fields = _device(ws, q.QED_FP32)
    q.qed_batch_push(g.ctx, arr, fields, ws[0].dt, 15, 0)
    _pull(ens, arr)
    for k, w in enumerate(ws):
        n = len(w.species[0]["id"])
        one = q.DeviceEnsemble.from_host(w.species, [n, 1, int(n * 15 * 3) + 64], q.QED_FP32)
        for s in range(15):
            g.push(one, fields[k], w.dt, 1, s)
        # the two kernels round differently in FP32 (FMA contraction around
        # the hardware reciprocal square root, logarithm and exponential, each
        # within 2 ulp), so the states agree to a few ulps per step, not bit
        # for bit
        for sp in (0, 2):
            a, b = by_id(ens[k].to_host(sp)), by_id(one.to_host(sp))
            assert np.array_equal(a["id"], b["id"])
            assert np.mean(a["nevents"] == b["nevents"]) > 0.999
            pa = np.stack([a[f] for f in ("px", "py", "pz")], 1)
            pb = np.stack([b[f] for f in ("px", "py", "pz")], 1)
            rel = np.linalg.norm(pa - pb, axis=1) / np.maximum(np.linalg.norm(pb, axis=1), 1e-3)
            assert np.median(rel) < 4e-6 and np.mean(rel < 1e-4) > 0.999, (sp, np.median(rel), rel.max())
    g.close()


def test_batch_rejects_cascade_config():
    ws = _batch([10], nsteps=2)
    g = q.Generator(q.make_config(precision=q.QED_FP32, seed=2, push_photons=1))
    ens, arr, fields = _device(ws, q.QED_FP32)
    with pytest.raises(q.QedError):
        q.qed_batch_push(g.ctx, arr, fields, ws[0].dt, 2, 0)
    g.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_budget_changes_nothing(prec):
    """The step budget only decides when a lepton rejoins its block's queue:
    the same kernel instantiation computes every particle, so any budget
    gives bit-identical ensembles."""
    ws = _batch([900, 6000], nsteps=12)
    P = q.QED_FP64 if prec == "fp64" else q.QED_FP32
    res = []
    for budget in (1, 3, 64):
        g = q.Generator(q.make_config(precision=P, seed=6, push_photons=0, block_threads=256,
                                      batch_step_budget=budget))
        assert q.qed_batch_shape(g.ctx) == (256, budget)
        ens, arr, fields = _device(ws, P)
        rc, _ = q.qed_batch_push(g.ctx, arr, fields, ws[0].dt, 12, 0)
        assert rc == q.QED_OK
        _pull(ens, arr)
        res.append([(by_id(e.to_host(0)), by_id(e.to_host(2))) for e in ens])
        g.close()
    for other in res[1:]:
        for (a0, a2), (b0, b2) in zip(res[0], other):
            for f in a0:
                assert np.array_equal(a0[f], b0[f]), f
            for f in a2:
                assert np.array_equal(a2[f], b2[f]), ("photon", f)
