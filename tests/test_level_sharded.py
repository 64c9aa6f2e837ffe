"""Global leveling of a species split over ranks (multi-GPU path, host side):
world_size-2 gloo ranks on the CPU each hold a shard of the weights, add
their sums with an all-reduce every iteration and advance with the
library's own iteration step (host code, no GPU).  The threshold must be
the one the oracle finds on the union of the shards."""
import math
import os
import socket

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

import paper_2409_17299_gb300 as q  # noqa: E402


def _shard_sums(w, at):
    """(A, C, N, max) of one shard at point `at`, exactly as defined: A the
    sum of alive weights below `at`, C the alive count at or above it."""
    alive = w[w > 0]
    below = alive[alive < at]
    return (math.fsum(below.tolist()), int(len(alive) - len(below)), int(len(alive)),
            float(alive.max()) if len(alive) else 0.0)


def _weights(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "lognormal":
        w = np.exp(rng.normal(size=n))
    elif kind == "classes":           # a few distinct values, as after earlier leveling
        w = rng.choice([0.5, 1.0, 3.0, 7.25], size=n)
    else:                             # all equal
        w = np.full(n, 2.0)
    w[rng.random(n) < 0.1] = 0.0      # dead entries are ignored
    return w


CASES = [("lognormal", 40000, 15000), ("classes", 30000, 9000), ("equal", 20000, 5000),
         ("lognormal", 5000, 10000)]  # the last one fits: no leveling


def _worker(rank, world, port, out_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = []
    for k, (kind, n, cap) in enumerate(CASES):
        w = _weights(kind, n, seed=11 + k)
        shard = np.array_split(w, world)[rank]
        st = q.level_threshold_sharded(lambda at: _shard_sums(shard, at), q.torch_allreduce(), cap)
        res.append((st.wstar, st.iters, st.alive))
    if rank == 0:
        np.save(out_path, np.array(res, dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_sharded_threshold_two_ranks(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "res.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    res = np.load(out)
    for (kind, n, cap), (ws, iters, alive) in zip(CASES, res):
        w = _weights(kind, n, seed=11 + CASES.index((kind, n, cap)))
        want = oracle.level_threshold(w, cap)
        assert alive == np.count_nonzero(w > 0)
        if want == 0.0:
            assert ws == 0.0                  # fits under the cap: nothing to thin
            continue
        assert ws == pytest.approx(want, rel=1e-13), (kind, ws, want)
        a = w[w > 0]
        assert math.fsum(np.minimum(1.0, a / ws).tolist()) == pytest.approx(cap, rel=1e-12)
        assert iters <= 12


def test_single_rank_matches_split_sums():
    """One rank with the identity all-reduce, and four shards added by hand:
    the same threshold (the split changes only the rounding of A)."""
    w = _weights("lognormal", 30000, seed=5)
    cap = 12000
    one = q.level_threshold_sharded(lambda at: _shard_sums(w, at), lambda v: v, cap)
    shards = np.array_split(w, 4)

    def four(at):
        parts = [_shard_sums(s, at) for s in shards]
        return (math.fsum(p[0] for p in parts), sum(p[1] for p in parts), sum(p[2] for p in parts),
                max(p[3] for p in parts))
    split = q.level_threshold_sharded(four, lambda v: v, cap)
    assert split.wstar == pytest.approx(one.wstar, rel=1e-14)
    assert one.wstar == pytest.approx(oracle.level_threshold(w, cap), rel=1e-13)


def test_advance_rejects_bad_input():
    st = q.qed_level_begin()
    assert st.w == math.inf and st.done == 0
    with pytest.raises(q.QedError):
        q.qed_level_advance(st, -1.0, 0, 10, 1.0, 5)
    with pytest.raises(q.QedError):
        q.qed_level_advance(st, 1.0, 0, 10, 1.0, 0)


@pytest.mark.parametrize("case", CASES[:3])
def test_warm_start_reaches_the_same_threshold(case):
    """The device starts a species' iteration at its previous threshold.  The
    first pass then evaluates at a finite w: from below, at or above the
    root the iteration (the library's own step, compiled for the host) must
    end at the threshold the oracle finds, in few passes."""
    kind, n, cap = case
    w = _weights(kind, n, seed=31)
    want = oracle.level_threshold(w, cap)
    for f in (0.3, 0.9, 0.999999, 1.0, 1.000001, 1.1, 3.0):
        st = q.qed_level_begin()
        st.w = want * f
        while not st.done:
            q.qed_level_advance(st, *_shard_sums(w, st.w), cap)
        assert st.wstar == pytest.approx(want, rel=1e-13), (kind, f)
        assert st.iters <= 12, (kind, f, st.iters)
