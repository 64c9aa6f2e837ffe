"""Bounded device-side waits that run out report it, and the context stays
usable.

Two loops on the device have an iteration limit: the newborn-pass loop of a
step (Algorithm 2's repeated sweeps, a while node of the step graph) and the
grid barrier of the training kernel.  Here each limit is set low enough to
run out on purpose: the call returns QED_ERR_TIMEOUT (the device wrote the
status; nothing faulted or hung), and the same context then computes a
correct result."""
import numpy as np
import pytest

from paper_2409_17299_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_17299_gb300 as q  # noqa: E402

PREC = q.QED_FP32


def _copy(ens):
    out = q.DeviceEnsemble(list(ens.capacity), PREC)
    for k in range(3):
        for f, a in ens.arr[k].items():
            out.arr[k][f].copy_(a)
    out.count = list(ens.count)
    return out


@pytest.fixture(scope="module")
def cascade():
    """The rotating-E cascade (4000 seeds, no leveling) after 200 steps:
    photons and pairs, so a step runs several newborn passes."""
    w = W.rotating_e_cascade(n=4000, seed=1, thin_cap=0)
    g = q.Generator(q.make_config(precision=PREC, seed=w.seed, push_photons=1))
    ens = q.DeviceEnsemble.from_host(w.species, [2_000_000, 2_000_000, 8_000_000], PREC)
    field = q.make_field(w.field_kind, w.field_prm)
    g.push(ens, field, w.dt, 200, 0)
    g.close()
    return w, ens, field


def _one_step(ctx_gen, ens, field, dt, step):
    ctx_gen._bind(ens)
    P = ens.struct()
    try:
        rc, st = q.qed_push_and_generate(ctx_gen.ctx, P, field, dt, 1, step)
    except q.QedError as e:
        rc, st = e.status, None
    ens.pull_counts(P)
    return rc, st


def test_newborn_pass_limit_runs_out(cascade):
    w, ens, field = cascade
    # the same step with the default limit needs two or more newborn passes
    ref = _copy(ens)
    g0 = q.Generator(q.make_config(precision=PREC, seed=w.seed, push_photons=1))
    rc, st = _one_step(g0, ref, field, w.dt, 200)
    g0.close()
    assert rc == q.QED_OK and st["passes"] >= 2, st
    # limit 1: the step stops after its first newborn pass and reports it
    g1 = q.Generator(q.make_config(precision=PREC, seed=w.seed, push_photons=1, pass_limit=1))
    work = _copy(ens)
    rc, _ = _one_step(g1, work, field, w.dt, 200)
    assert rc == q.QED_ERR_TIMEOUT
    # the context still works: a step needing one newborn pass (photons from
    # electrons at chi0 = 0.1, too soft to create pairs) completes, with the
    # same ensemble as on a fresh context
    e = W.uniform_b_emission(n=4000, seed=3, chi0=0.1, nsteps=1)
    outs = []
    for gen in (g1, q.Generator(q.make_config(precision=PREC, seed=w.seed, push_photons=1))):
        one = q.DeviceEnsemble.from_host(e.species, [4000, 16, 4000], PREC)
        rc, st = _one_step(gen, one, q.make_field(e.field_kind, e.field_prm), e.dt, 0)
        assert rc == q.QED_OK and st["passes"] <= 1, st
        outs.append([one.to_host(s) for s in (0, 2)])
    g1.close()
    for a, b in zip(*outs):
        assert len(a["id"]) == len(b["id"])
        order_a, order_b = np.argsort(a["id"]), np.argsort(b["id"])
        for f in ("px", "py", "pz"):
            assert np.array_equal(a[f][order_a], b[f][order_b]), f


def test_training_grid_barrier_runs_out():
    g = q.Generator(q.make_config(precision=PREC, wait_polls=1))
    with pytest.raises(q.QedError) as ei:
        q.qed_train_surrogate(g.ctx, n_samples=8192 * 50, batch=8192, lr=4e-3, seed=7)
    assert ei.value.status == q.QED_ERR_TIMEOUT
    # the context still works: the network it holds (the initialisation; the
    # failed launch wrote nothing back) gives the same outputs as a fresh
    # context loaded with the same parameters
    P = q.qed_mlp_get_params(g.ctx)
    assert np.all(np.isfinite(P))
    g2 = q.Generator(q.make_config(precision=PREC))
    q.qed_mlp_set_params(g2.ctx, P)
    rng = np.random.default_rng(5)
    feat = torch.from_numpy(rng.uniform(-1, 1, size=(4096, 2)).astype(np.float32)).cuda()
    ys = []
    for gen in (g, g2):
        y = torch.empty(4096, dtype=torch.float32, device="cuda")
        q.qed_mlp_forward(gen.ctx, feat.data_ptr(), 4096, y.data_ptr())
        ys.append(y.cpu().numpy())
    assert np.array_equal(ys[0], ys[1])
    # and a training with the default limit succeeds on a new context
    g3 = q.Generator(q.make_config(precision=PREC))
    loss = q.qed_train_surrogate(g3.ctx, n_samples=8192 * 50, batch=8192, lr=4e-3, seed=7)
    assert np.isfinite(loss)
    for gen in (g, g2, g3):
        gen.close()
