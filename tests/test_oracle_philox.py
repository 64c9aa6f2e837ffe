"""Pins for the oracle's Philox4x32-10 and its uniform mapping.

Philox4x32-10 (Salmon et al., SC'11) is checked bit for bit against an
independent implementation: Triton's own Philox, run by Triton's CPU
interpreter in a child process.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

_TRITON_SCRIPT = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(c0p, c1p, c2p, c3p, out, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    a, b, c, d = tl.philox(seed, tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i), tl.load(c3p + i))
    tl.store(out + 4 * i, a); tl.store(out + 4 * i + 1, b)
    tl.store(out + 4 * i + 2, c); tl.store(out + 4 * i + 3, d)

req = json.loads(sys.stdin.read())
res = []
for seed, ctr in req:
    ctr = np.array(ctr, dtype=np.uint32).reshape(-1, 4)
    n = ctr.shape[0]
    cols = [torch.tensor(ctr[:, j].view(np.int32).copy()) for j in range(4)]
    out = torch.zeros(4 * n, dtype=torch.int32)
    k[(1,)](cols[0], cols[1], cols[2], cols[3], out, seed, N=n)
    res.append(out.numpy().view(np.uint32).reshape(-1, 4).tolist())
print(json.dumps(res))
"""


def test_philox_matches_independent_library():
    pytest.importorskip("triton")
    rng = np.random.default_rng(123)
    req = []
    seeds = [0, 1, 0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF, int(rng.integers(0, 2**63))]
    for seed in seeds:
        ctr = rng.integers(0, 2**32, size=(16, 4), dtype=np.uint64).astype(np.uint32)
        ctr[0] = 0
        ctr[1] = 0xFFFFFFFF
        req.append([seed, ctr.tolist()])
    p = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(req),
                       capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, TRITON_INTERPRET="1"))
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr[-300:])
    ref = json.loads(p.stdout.strip().splitlines()[-1])
    for (seed, ctr), want in zip(req, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        got = oracle.philox(np.array(ctr, dtype=np.uint32), key)
        assert got.tolist() == want


def test_philox_is_a_bijection_of_the_counter():
    # distinct counters under one key give distinct outputs (a sample)
    ctr = np.zeros((4096, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(4096)
    out = oracle.philox(ctr, [7, 9])
    assert len({tuple(r) for r in out.tolist()}) == 4096


def test_u52_range_and_bits():
    two52 = 2.0 ** 52
    assert oracle.u52(0, 0) == 0.5 / two52
    assert oracle.u52(0xFFFFFFFF, 0xFFFFFFFF) == (two52 - 0.5) / two52
    assert oracle.u52(0xFFFFFFFF, 0xFFFFFFFF) < 1.0
    # low 12 bits of the second word are discarded
    assert oracle.u52(5, 0xABC) == oracle.u52(5, 0)
    assert oracle.u52(0, 1 << 12) == 1.5 / two52
    assert oracle.u52(1, 0) == (2.0 ** 20 + 0.5) / two52
