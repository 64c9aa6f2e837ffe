"""Compaction that allocates nothing, for callers that cannot call cudaMalloc
(their device memory belongs to another allocator's pool, or their time loop
cannot accept the synchronisation an allocation may cause).

Its result must equal that of the ordinary, context-based compaction
(qed_compact) on the same input, on two calls in a row; both implement the
same deterministic hole filling, so the comparison is exact.  With an
optical-depth array the array must move with its particles, as it does in
qed_compact when the array is bound with qed_set_optical_depth.  A call must
leave the device's free memory unchanged, and misaligned arrays are rejected
before any work is issued.
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


def _species(n, seed, dead_frac, od=False):
    rng = np.random.default_rng(seed)
    sp = {f: rng.normal(size=n) for f in ("x", "y", "z", "px", "py", "pz")}
    w = rng.random(n) + 0.5
    w[rng.random(n) < dead_frac] = 0.0
    sp["w"] = w
    sp["id"] = rng.permutation(n).astype(np.uint64)
    sp["nevents"] = rng.integers(0, 5, n).astype(np.uint32)
    if od:
        sp["od"] = rng.exponential(size=n)
    return sp


def _ensemble(sp, prec, od=False):
    n = len(sp["id"])
    empty = {f: np.zeros(0) for f in ("x", "y", "z", "px", "py", "pz", "w")}
    empty["id"] = np.zeros(0, dtype=np.uint64)
    return q.DeviceEnsemble.from_host([sp, empty, empty], [n, 1, 1], prec, optical_depth=od)


def _check(ref, new, sp, fields):
    alive = int(np.sum(sp["w"] > 0))
    assert new.count[0] == ref.count[0] == alive
    a, b = ref.to_host(0), new.to_host(0)
    for f in fields:
        assert np.array_equal(a[f], b[f]), f
    assert np.all(b["w"] > 0)
    assert sorted(b["id"].tolist()) == sorted(sp["id"][sp["w"] > 0].tolist())


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
        _check(ref, new, sp, FIELDS)
    gen.close()


@pytest.mark.parametrize("prec", [q.QED_FP64, q.QED_FP32])
def test_noalloc_moves_optical_depth(prec):
    """The optical-depth array follows its particles (two calls in a row)."""
    build.build()
    stream = torch.cuda.current_stream()
    gen = q.Generator(q.make_config(precision=prec, thin_cap=0, event_method=q.QED_METHOD_OPTICAL_DEPTH))
    for n, frac, seed in [(50003, 0.4, 5), (300001, 0.2, 6)]:
        sp = _species(n, seed, frac, od=True)
        ref = _ensemble(sp, prec, od=True)
        gen.compact(ref, 0)                      # binds the od arrays, then qed_compact
        new = _ensemble(sp, prec, od=True)
        P = new.struct()
        q.qed_compact_species_noalloc(P.s[0], prec, stream.cuda_stream, od_dev_ptr=new.od_ptrs()[0])
        new.pull_counts(P)
        torch.cuda.synchronize()
        _check(ref, new, sp, FIELDS + ("od",))
        # each surviving particle keeps its own optical depth
        b = new.to_host(0)
        by_id = dict(zip(sp["id"].tolist(), sp["od"].tolist()))
        want = np.array([by_id[i] for i in b["id"].tolist()])
        dt = np.float32 if prec == q.QED_FP32 else np.float64
        assert np.array_equal(b["od"], want.astype(dt).astype(np.float64))
    gen.close()


def test_noalloc_allocates_nothing():
    """After a first call (which looks up the scratch array's address), a
    further call leaves the device's free memory exactly as it was."""
    build.build()
    stream = torch.cuda.current_stream()
    sp = _species(200003, 7, 0.5)
    first, second = _ensemble(sp, q.QED_FP32), _ensemble(sp, q.QED_FP32)
    P1 = first.struct()
    q.qed_compact_species_noalloc(P1.s[0], q.QED_FP32, stream.cuda_stream)
    torch.cuda.synchronize()
    P2 = second.struct()
    free0, _ = torch.cuda.mem_get_info()
    q.qed_compact_species_noalloc(P2.s[0], q.QED_FP32, stream.cuda_stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    second.pull_counts(P2)
    assert second.count[0] == int(np.sum(sp["w"] > 0))


def test_noalloc_rejects_oversized_species():
    build.build()
    e = _ensemble(_species(16, 3, 0.5), q.QED_FP64)
    P = e.struct()
    P.s[0].count = q.QED_NOALLOC_MAX_ENTRIES + 1
    P.s[0].capacity = q.QED_NOALLOC_MAX_ENTRIES + 1
    with pytest.raises(q.QedError) as ei:
        q.qed_compact_species_noalloc(P.s[0], q.QED_FP64, torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == q.QED_ERR_INVALID


def test_noalloc_rejects_misaligned_arrays():
    """Misaligned or missing arrays are refused on the host before any kernel
    is launched (the species is left as it was)."""
    build.build()
    stream = torch.cuda.current_stream().cuda_stream
    sp = _species(64, 4, 0.5, od=True)
    e = _ensemble(sp, q.QED_FP64, od=True)
    for field, shift in (("x", 4), ("id", 8), ("nevents", 4)):
        P = e.struct()
        S = P.s[0]
        saved = getattr(S, field)
        setattr(S, field, saved + shift)
        with pytest.raises(q.QedError) as ei:
            q.qed_compact_species_noalloc(S, q.QED_FP64, stream)
        assert ei.value.status == q.QED_ERR_INVALID
        setattr(S, field, saved)
    P = e.struct()
    saved = P.s[0].w
    P.s[0].w = None
    with pytest.raises(q.QedError) as ei:
        q.qed_compact_species_noalloc(P.s[0], q.QED_FP64, stream)
    assert ei.value.status == q.QED_ERR_INVALID
    P.s[0].w = saved
    with pytest.raises(q.QedError) as ei:
        q.qed_compact_species_noalloc(P.s[0], q.QED_FP64, stream, od_dev_ptr=e.od_ptrs()[0] + 4)
    assert ei.value.status == q.QED_ERR_INVALID
    assert P.s[0].count == 64
    assert np.array_equal(e.to_host(0)["id"], sp["id"])
