"""Compaction that allocates nothing, for callers that cannot call cudaMalloc
(their device memory belongs to another allocator's pool, or their time loop
cannot accept the synchronisation an allocation may cause).

Its result must equal that of the ordinary, context-based compaction
(qed_compact) on the same input, on two calls in a row; both implement the
same deterministic hole filling, so the comparison is exact.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2409_17299_gb300 as q  # noqa: E402
from paper_2409_17299_gb300 import build  # noqa: E402

FIELDS = ("x", "y", "z", "px", "py", "pz", "w", "id", "nevents")


def _species(n, seed, dead_frac):
    rng = np.random.default_rng(seed)
    sp = {f: rng.normal(size=n) for f in ("x", "y", "z", "px", "py", "pz")}
    w = rng.random(n) + 0.5
    w[rng.random(n) < dead_frac] = 0.0
    sp["w"] = w
    sp["id"] = rng.permutation(n).astype(np.uint64)
    sp["nevents"] = rng.integers(0, 5, n).astype(np.uint32)
    return sp


def _ensemble(sp, prec):
    n = len(sp["id"])
    empty = {f: np.zeros(0) for f in ("x", "y", "z", "px", "py", "pz", "w")}
    empty["id"] = np.zeros(0, dtype=np.uint64)
    return q.DeviceEnsemble.from_host([sp, empty, empty], [n, 1, 1], prec)


@pytest.mark.parametrize("prec", [q.QED_FP64, q.QED_FP32])
def test_noalloc_compaction_matches_context_compaction(prec):
    build.build()
    stream = torch.cuda.current_stream()
    gen = q.Generator(q.make_config(precision=prec, thin_cap=0))
    cases = [(70001, 0.3, 1), (q.QED_NOALLOC_MAX_ENTRIES, 0.6, 2)]   # two calls in a row
    for n, frac, seed in cases:
        sp = _species(n, seed, frac)
        ref = _ensemble(sp, prec)
        gen.compact(ref, 0)                      # existing entry point (context scratch)
        new = _ensemble(sp, prec)
        P = new.struct()
        q.qed_compact_species_noalloc(P.s[0], prec, stream.cuda_stream)
        new.pull_counts(P)
        torch.cuda.synchronize()
        alive = int(np.sum(sp["w"] > 0))
        assert new.count[0] == ref.count[0] == alive
        a, b = ref.to_host(0), new.to_host(0)
        for f in FIELDS:
            assert np.array_equal(a[f], b[f]), f
        assert np.all(b["w"] > 0)
        assert sorted(b["id"].tolist()) == sorted(sp["id"][sp["w"] > 0].tolist())
    gen.close()


def test_noalloc_rejects_oversized_species():
    build.build()
    e = _ensemble(_species(16, 3, 0.5), q.QED_FP64)
    P = e.struct()
    P.s[0].count = q.QED_NOALLOC_MAX_ENTRIES + 1
    P.s[0].capacity = q.QED_NOALLOC_MAX_ENTRIES + 1
    with pytest.raises(q.QedError) as ei:
        q.qed_compact_species_noalloc(P.s[0], q.QED_FP64, torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == q.QED_ERR_INVALID
