"""The multi-rank path of bench.py on the CPU (gloo, world size 2): each
rank runs its own replica, the line reports work summed over the ranks and
the slowest rank's time, replicas draw independent inputs, and the
reference arm prints on rank 0 only."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
torch = pytest.importorskip("torch")

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ps, ev, secs = bench.reduce_over_ranks(1000.0 * (rank + 1), 10.0 * (rank + 1), 0.5 + rank, world)
    if rank == 0:
        np.save(out, np.array([ps, ev, secs]))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_ranks(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "r.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    ps, ev, secs = np.load(out)
    assert ps == 3000.0 and ev == 30.0 and secs == 1.5      # sum, sum, max


def test_single_rank_is_identity():
    assert bench.reduce_over_ranks(5.0, 2.0, 0.25, 1) == (5.0, 2.0, 0.25)


@pytest.mark.parametrize("name", ["rotating_e_cascade", "standing_wave_cascade"])
def test_replicas_draw_independent_inputs(name):
    a = bench.make_workload(name, 0.01, rank=0)
    b = bench.make_workload(name, 0.01, rank=1)
    assert a.seed != b.seed                                   # independent Philox streams
    assert not np.array_equal(a.species[0]["x"], b.species[0]["x"])
    assert len(a.species[0]["id"]) == len(b.species[0]["id"])  # weak scaling: same work per rank


def test_reference_arm_other_ranks_print_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
