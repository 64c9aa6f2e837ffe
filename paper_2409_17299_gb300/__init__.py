"""GB300 strong-field QED event generator (arXiv:2409.17299 method).

Thin Python binding of the C ABI declared in ``include/sfqed.h``.  Every
function with a ``qed_`` name marshals its arguments and calls the function
of the same name in ``libsfqed.so``; all computation runs in the library's
CUDA kernels.  PyTorch only provides device memory and streams
(``DeviceEnsemble``).  There is no CPU fallback: importing the binding
without the compiled library raises.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB, up_to_date  # noqa: F401

QED_OK, QED_ERR_INVALID, QED_ERR_CAPACITY, QED_ERR_CUDA, QED_ERR_TIMEOUT, QED_ERR_NOMEM, QED_ERR_STATE = range(7)
QED_FP64, QED_FP32 = 0, 1
QED_SAMPLER_TABLE, QED_SAMPLER_MLP = 0, 1
QED_METHOD_SUBSTEP, QED_METHOD_OPTICAL_DEPTH = 0, 1
QED_ELECTRON, QED_POSITRON, QED_PHOTON = 0, 1, 2
QED_FIELD_UNIFORM, QED_FIELD_ROTATING_E, QED_FIELD_STANDING_CP, QED_FIELD_GRID = 0, 1, 2, 3

EXPORTED = ("qed_init_tables", "qed_push_and_generate", "qed_push_async", "qed_push_wait", "qed_batch_push", "qed_autotune_batch", "qed_compact", "qed_get_stats", "qed_strerror",
            "qed_destroy", "qed_philox", "qed_get_tables", "qed_eval_rate", "qed_sample", "qed_eval_chi",
            "qed_compact_species_noalloc", "qed_train_surrogate", "qed_mlp_set_params", "qed_mlp_get_params",
            "qed_mlp_forward", "qed_mlp_grad", "qed_level_begin", "qed_level_advance", "qed_level_eval",
            "qed_level_apply", "qed_batch_shape", "qed_set_field_grid", "qed_set_optical_depth",
            "qed_measure_fp64_peak")
QED_NOALLOC_MAX_ENTRIES = 1 << 20


class QedConfig(C.Structure):
    _fields_ = [("precision", C.c_int), ("sampler", C.c_int), ("seed", C.c_uint64),
                ("push_photons", C.c_int), ("soft_photon_filter", C.c_int), ("thin_cap", C.c_int64),
                ("restore_on_overflow", C.c_int), ("block_threads", C.c_int), ("blocks_per_sm", C.c_int),
                ("profile", C.c_int), ("batch_step_budget", C.c_int), ("event_method", C.c_int),
                ("pass_limit", C.c_int), ("wait_polls", C.c_int), ("reserved", C.c_int * 1)]


class QedLevelState(C.Structure):
    _fields_ = [("lo", C.c_double), ("hi", C.c_double), ("w", C.c_double), ("wstar", C.c_double),
                ("iters", C.c_int64), ("done", C.c_int64), ("alive", C.c_int64)]


class QedSpecies(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("px", C.c_void_p),
                ("py", C.c_void_p), ("pz", C.c_void_p), ("w", C.c_void_p), ("id", C.c_void_p),
                ("nevents", C.c_void_p), ("count", C.c_int64), ("capacity", C.c_int64)]


class QedParticles(C.Structure):
    _fields_ = [("s", QedSpecies * 3)]


class QedFieldDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("params", C.c_double * 16)]


class QedStats(C.Structure):
    _fields_ = [("particle_steps", C.c_int64), ("emit_events", C.c_int64), ("pair_events", C.c_int64),
                ("needed_capacity", C.c_int64 * 3), ("max_subevents", C.c_int64), ("overflow", C.c_int64),
                ("passes", C.c_int64), ("thinned", C.c_int64), ("lepton_steps", C.c_int64),
                ("photon_steps", C.c_int64), ("launches", C.c_int64), ("chi_fp64", C.c_int64),
                ("kernel_ms", C.c_double * 4), ("sync_ms", C.c_double), ("call_ms", C.c_double),
                ("moved", C.c_int64)]

    def as_dict(self):
        return {"particle_steps": self.particle_steps, "emit_events": self.emit_events,
                "pair_events": self.pair_events, "needed_capacity": list(self.needed_capacity),
                "max_subevents": self.max_subevents, "overflow": self.overflow,
                "passes": self.passes, "thinned": self.thinned, "lepton_steps": self.lepton_steps,
                "photon_steps": self.photon_steps, "launches": self.launches, "chi_fp64": self.chi_fp64,
                "kernel_ms": list(self.kernel_ms), "sync_ms": self.sync_ms, "call_ms": self.call_ms,
                "moved": self.moved}


class QedError(RuntimeError):
    def __init__(self, status, where, stats=None):
        super().__init__("%s: %s (status %d)" % (where, qed_strerror(status), status))
        self.status = status
        self.stats = stats


_lib = None


def lib():
    """Load libsfqed.so from the package tree; raise if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise ImportError("libsfqed.so is not built; run paper_2409_17299_gb300.build.build() "
                          "(the CUDA library is required: there is no CPU path)")
    L = C.CDLL(LIB)
    p, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    sig = {
        "qed_init_tables": (i32, [C.POINTER(p), C.POINTER(QedConfig), p]),
        "qed_push_and_generate": (i32, [p, C.POINTER(QedParticles), C.POINTER(QedFieldDesc), C.c_double, i32, i64,
                                        C.POINTER(QedStats)]),
        "qed_push_async": (i32, [p, C.POINTER(QedParticles), C.POINTER(QedFieldDesc), C.c_double, i32, i64]),
        "qed_push_wait": (i32, [p, C.POINTER(QedParticles), C.POINTER(QedStats)]),
        "qed_compact": (i32, [p, C.POINTER(QedParticles), i64]),
        "qed_batch_push": (i32, [p, C.POINTER(QedParticles), C.POINTER(QedFieldDesc), i32, C.c_double, i32, i64,
                                 C.POINTER(QedStats)]),
        "qed_autotune_batch": (i32, [p, C.POINTER(QedParticles), C.POINTER(QedFieldDesc), i32, C.c_double, i32,
                                     C.POINTER(i32), C.POINTER(C.c_double)]),
        "qed_get_stats": (i32, [p, C.POINTER(QedStats), i32]),
        "qed_strerror": (C.c_char_p, [i32]),
        "qed_destroy": (None, [p]),
        "qed_philox": (i32, [p, i64, C.c_uint64, p, p]),
        "qed_get_tables": (i32, [p, p, p, p, p]),
        "qed_eval_rate": (i32, [p, i32, p, i64, p]),
        "qed_sample": (i32, [p, i32, p, p, i64, p, p]),
        "qed_compact_species_noalloc": (i32, [C.POINTER(QedSpecies), p, i32, p]),
        "qed_eval_chi": (i32, [p, i32, p, p, p, i64, p, C.POINTER(i64)]),
        "qed_train_surrogate": (i32, [p, i64, i32, C.c_double, C.c_uint64, C.POINTER(C.c_double)]),
        "qed_mlp_set_params": (i32, [p, p]),
        "qed_mlp_get_params": (i32, [p, p]),
        "qed_mlp_forward": (i32, [p, p, i64, p]),
        "qed_mlp_grad": (i32, [p, p, p, i64, p, C.POINTER(C.c_double)]),
        "qed_level_begin": (None, [C.POINTER(QedLevelState)]),
        "qed_level_advance": (i32, [C.POINTER(QedLevelState), C.c_double, i64, i64, C.c_double, i64]),
        "qed_level_eval": (i32, [p, C.POINTER(QedSpecies), i32, C.c_double, C.POINTER(C.c_double),
                                 C.POINTER(i64), C.POINTER(i64), C.POINTER(C.c_double)]),
        "qed_level_apply": (i32, [p, p, i32, C.c_double, i64]),
        "qed_batch_shape": (i32, [p, C.POINTER(i32), C.POINTER(i32)]),
        "qed_set_field_grid": (i32, [p, p]),
        "qed_set_optical_depth": (i32, [p, C.POINTER(C.c_void_p)]),
        "qed_measure_fp64_peak": (i32, [i32, C.POINTER(C.c_double), C.POINTER(C.c_double), p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


# --------------------------------------------------------------------------
# one Python function per C entry point (argument marshalling only)
# --------------------------------------------------------------------------
def qed_strerror(status: int) -> str:
    return lib().qed_strerror(int(status)).decode()


def qed_init_tables(cfg: QedConfig, cuda_stream: int | None = None) -> C.c_void_p:
    ctx = C.c_void_p()
    st = lib().qed_init_tables(C.byref(ctx), C.byref(cfg), C.c_void_p(cuda_stream or 0))
    if st != QED_OK:
        raise QedError(st, "qed_init_tables")
    return ctx


def qed_push_and_generate(ctx, particles: QedParticles, field: QedFieldDesc, dt: float, nsteps: int,
                          step0: int = 0):
    """Returns (status, stats dict); QED_ERR_CAPACITY is returned, not raised."""
    st = QedStats()
    rc = lib().qed_push_and_generate(ctx, C.byref(particles), C.byref(field), float(dt), int(nsteps),
                                     int(step0), C.byref(st))
    if rc not in (QED_OK, QED_ERR_CAPACITY):
        raise QedError(rc, "qed_push_and_generate")
    return rc, st.as_dict()


def qed_push_async(ctx, particles: QedParticles, field: QedFieldDesc, dt: float, nsteps: int,
                   step0: int = 0) -> None:
    """Enqueue nsteps steps without waiting for the GPU (the counts stay on
    the device until qed_push_wait)."""
    rc = lib().qed_push_async(ctx, C.byref(particles), C.byref(field), float(dt), int(nsteps), int(step0))
    if rc != QED_OK:
        raise QedError(rc, "qed_push_async")


def qed_push_wait(ctx, particles: QedParticles):
    """Wait for the enqueued steps; returns (status, stats dict) and updates
    the counts in particles.  QED_ERR_CAPACITY is returned, not raised."""
    st = QedStats()
    rc = lib().qed_push_wait(ctx, C.byref(particles), C.byref(st))
    if rc not in (QED_OK, QED_ERR_CAPACITY):
        raise QedError(rc, "qed_push_wait", st.as_dict())
    return rc, st.as_dict()


def qed_batch_push(ctx, ensembles, fields, dt: float, nsteps: int, step0: int = 0):
    """ensembles: ctypes array of QedParticles; fields: ctypes array of
    QedFieldDesc (same length).  Returns (status, stats dict)."""
    st = QedStats()
    rc = lib().qed_batch_push(ctx, ensembles, fields, len(ensembles), float(dt), int(nsteps), int(step0),
                              C.byref(st))
    if rc not in (QED_OK, QED_ERR_CAPACITY):
        raise QedError(rc, "qed_batch_push")
    return rc, st.as_dict()


def qed_autotune_batch(ctx, ensembles, fields, dt: float, nsteps: int):
    """Returns (chosen threads per block, [ms for 128, 256, 512])."""
    chosen = C.c_int(0)
    ms = (C.c_double * 3)()
    rc = lib().qed_autotune_batch(ctx, ensembles, fields, len(ensembles), float(dt), int(nsteps),
                                  C.byref(chosen), ms)
    if rc != QED_OK:
        raise QedError(rc, "qed_autotune_batch")
    return chosen.value, list(ms)


def qed_compact(ctx, particles: QedParticles, step: int) -> int:
    rc = lib().qed_compact(ctx, C.byref(particles), int(step))
    if rc != QED_OK:
        raise QedError(rc, "qed_compact")
    return rc


def qed_set_optical_depth(ctx, ptrs) -> None:
    """Bind the three per-species optical-depth arrays (device pointers of
    arrays of the context's precision, or 0) for QED_METHOD_OPTICAL_DEPTH."""
    arr = (C.c_void_p * 3)(*[C.c_void_p(int(v or 0)) for v in ptrs])
    rc = lib().qed_set_optical_depth(ctx, arr)
    if rc != QED_OK:
        raise QedError(rc, "qed_set_optical_depth")


def qed_set_field_grid(ctx, grid_dev_ptr) -> None:
    """Attach the gridded field's node values (device pointer, 6 x nz x ny x nx
    values of the context's precision); 0/None detaches."""
    rc = lib().qed_set_field_grid(ctx, C.c_void_p(grid_dev_ptr or 0))
    if rc != QED_OK:
        raise QedError(rc, "qed_set_field_grid")


def qed_batch_shape(ctx):
    """(threads, step budget) of qed_batch_push in this context."""
    t, b = C.c_int(), C.c_int()
    rc = lib().qed_batch_shape(ctx, C.byref(t), C.byref(b))
    if rc != QED_OK:
        raise QedError(rc, "qed_batch_shape")
    return t.value, b.value


def qed_level_begin() -> QedLevelState:
    st = QedLevelState()
    lib().qed_level_begin(C.byref(st))
    return st


def qed_level_advance(st: QedLevelState, A: float, C_: int, N: int, max_w: float, cap: int) -> None:
    rc = lib().qed_level_advance(C.byref(st), float(A), int(C_), int(N), float(max_w), int(cap))
    if rc != QED_OK:
        raise QedError(rc, "qed_level_advance")


def qed_level_eval(ctx, species: QedSpecies, s: int, w: float):
    """This shard's (A, C, N, max_w) at point w."""
    A, Cc, N, M = C.c_double(), C.c_int64(), C.c_int64(), C.c_double()
    rc = lib().qed_level_eval(ctx, C.byref(species), int(s), float(w), C.byref(A), C.byref(Cc), C.byref(N),
                              C.byref(M))
    if rc != QED_OK:
        raise QedError(rc, "qed_level_eval")
    return A.value, Cc.value, N.value, M.value


def qed_level_apply(ctx, particles: QedParticles, s: int, wstar: float, step: int) -> None:
    rc = lib().qed_level_apply(ctx, C.byref(particles), int(s), float(wstar), int(step))
    if rc != QED_OK:
        raise QedError(rc, "qed_level_apply")


def level_threshold_sharded(evaluate, allreduce, cap: int) -> QedLevelState:
    """Global leveling threshold of a species split over ranks.  evaluate(w)
    returns this rank's (A, C, N, max_w) at w; allreduce(values) returns
    them combined over all ranks (A, C, N summed, max_w maximum).  The
    iteration itself is the library's (qed_level_advance)."""
    st = qed_level_begin()
    while not st.done:
        qed_level_advance(st, *allreduce(evaluate(st.w)), cap)
    return st


def torch_allreduce(group=None):
    """An allreduce for level_threshold_sharded over a torch.distributed group."""
    import torch
    import torch.distributed as dist

    def reduce(v):
        A, Cc, N, M = v
        s = torch.tensor([A], dtype=torch.float64)
        c = torch.tensor([Cc, N], dtype=torch.int64)
        m = torch.tensor([M], dtype=torch.float64)
        dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(c, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(m, op=dist.ReduceOp.MAX, group=group)
        return float(s[0]), int(c[0]), int(c[1]), float(m[0])
    return reduce


def qed_get_stats(ctx, reset: bool = False) -> dict:
    st = QedStats()
    rc = lib().qed_get_stats(ctx, C.byref(st), int(reset))
    if rc != QED_OK:
        raise QedError(rc, "qed_get_stats")
    return st.as_dict()


def qed_destroy(ctx) -> None:
    lib().qed_destroy(ctx)


def qed_philox(ctr_dev_ptr: int, n: int, key: int, out_dev_ptr: int, cuda_stream: int | None = None) -> None:
    rc = lib().qed_philox(C.c_void_p(ctr_dev_ptr), int(n), C.c_uint64(key), C.c_void_p(out_dev_ptr),
                          C.c_void_p(cuda_stream or 0))
    if rc != QED_OK:
        raise QedError(rc, "qed_philox")


def qed_get_tables(ctx, cheb_em_ptr=None, cheb_pair_ptr=None, icdf_em_ptr=None, icdf_pair_ptr=None) -> None:
    rc = lib().qed_get_tables(ctx, C.c_void_p(cheb_em_ptr or 0), C.c_void_p(cheb_pair_ptr or 0),
                              C.c_void_p(icdf_em_ptr or 0), C.c_void_p(icdf_pair_ptr or 0))
    if rc != QED_OK:
        raise QedError(rc, "qed_get_tables")


def qed_eval_rate(ctx, is_photon: bool, chi_dev_ptr: int, n: int, F_dev_ptr: int) -> None:
    rc = lib().qed_eval_rate(ctx, int(is_photon), C.c_void_p(chi_dev_ptr), int(n), C.c_void_p(F_dev_ptr))
    if rc != QED_OK:
        raise QedError(rc, "qed_eval_rate")


def qed_eval_chi(ctx, is_photon: bool, p_dev_ptr: int, E_dev_ptr: int, B_dev_ptr: int, n: int,
                 chi_dev_ptr: int) -> int:
    """Returns how many evaluations took the FP64 form."""
    n64 = C.c_int64(0)
    rc = lib().qed_eval_chi(ctx, int(is_photon), C.c_void_p(p_dev_ptr), C.c_void_p(E_dev_ptr),
                            C.c_void_p(B_dev_ptr), int(n), C.c_void_p(chi_dev_ptr), C.byref(n64))
    if rc != QED_OK:
        raise QedError(rc, "qed_eval_chi")
    return n64.value


def qed_sample(ctx, is_photon: bool, chi_dev_ptr: int, u_dev_ptr: int, n: int, delta_dev_ptr: int,
               one_minus_dev_ptr: int | None = None) -> None:
    rc = lib().qed_sample(ctx, int(is_photon), C.c_void_p(chi_dev_ptr), C.c_void_p(u_dev_ptr), int(n),
                          C.c_void_p(delta_dev_ptr), C.c_void_p(one_minus_dev_ptr or 0))
    if rc != QED_OK:
        raise QedError(rc, "qed_sample")


MLP_NPARAMS = 8577


def qed_train_surrogate(ctx, n_samples: int, batch: int = 8192, lr: float = 4e-3, seed: int = 12345) -> float:
    loss = C.c_double(0.0)
    rc = lib().qed_train_surrogate(ctx, int(n_samples), int(batch), float(lr), C.c_uint64(seed), C.byref(loss))
    if rc != QED_OK:
        raise QedError(rc, "qed_train_surrogate")
    return loss.value


def qed_mlp_set_params(ctx, params_host) -> None:
    import numpy as np
    P = np.ascontiguousarray(params_host, dtype=np.float32)
    rc = lib().qed_mlp_set_params(ctx, P.ctypes.data)
    if rc != QED_OK:
        raise QedError(rc, "qed_mlp_set_params")


def qed_mlp_get_params(ctx):
    import numpy as np
    P = np.zeros(MLP_NPARAMS, dtype=np.float32)
    rc = lib().qed_mlp_get_params(ctx, P.ctypes.data)
    if rc != QED_OK:
        raise QedError(rc, "qed_mlp_get_params")
    return P


def qed_mlp_forward(ctx, feat_dev_ptr: int, n: int, y_dev_ptr: int) -> None:
    rc = lib().qed_mlp_forward(ctx, C.c_void_p(feat_dev_ptr), int(n), C.c_void_p(y_dev_ptr))
    if rc != QED_OK:
        raise QedError(rc, "qed_mlp_forward")


def qed_mlp_grad(ctx, feat_dev_ptr: int, target_dev_ptr: int, n: int):
    import numpy as np
    g = np.zeros(MLP_NPARAMS, dtype=np.float32)
    loss = C.c_double(0.0)
    rc = lib().qed_mlp_grad(ctx, C.c_void_p(feat_dev_ptr), C.c_void_p(target_dev_ptr), int(n), g.ctypes.data,
                            C.byref(loss))
    if rc != QED_OK:
        raise QedError(rc, "qed_mlp_grad")
    return g, loss.value


def qed_measure_fp64_peak(iters: int = 1 << 16, cuda_stream: int | None = None):
    """(FP64 FLOP/s, ms of the timed launch) of the current device."""
    f, ms = C.c_double(), C.c_double()
    rc = lib().qed_measure_fp64_peak(int(iters), C.byref(f), C.byref(ms), C.c_void_p(cuda_stream or 0))
    if rc != QED_OK:
        raise QedError(rc, "qed_measure_fp64_peak")
    return f.value, ms.value


def qed_compact_species_noalloc(species: QedSpecies, precision: int, cuda_stream: int | None = None,
                                od_dev_ptr: int | None = None) -> int:
    """Compaction of one species that allocates no device memory (for callers
    whose device memory is owned by another allocator); species.count is
    updated in place and the optical-depth array, if given, moves with the
    particles.  Overlapping calls on the GPU race (shared scratch)."""
    rc = lib().qed_compact_species_noalloc(C.byref(species), C.c_void_p(od_dev_ptr or 0), int(precision),
                                           C.c_void_p(cuda_stream or 0))
    if rc != QED_OK:
        raise QedError(rc, "qed_compact_species_noalloc")
    return rc


# --------------------------------------------------------------------------
# small helpers around the ABI structs (no computation)
# --------------------------------------------------------------------------
def make_config(precision=QED_FP64, seed=0, push_photons=1, soft_photon_filter=0, thin_cap=0,
                restore_on_overflow=1, block_threads=0, blocks_per_sm=0, profile=0,
                sampler=QED_SAMPLER_TABLE, batch_step_budget=0, event_method=QED_METHOD_SUBSTEP,
                pass_limit=0, wait_polls=0) -> QedConfig:
    c = QedConfig()
    c.precision = int(precision)
    c.sampler = int(sampler)
    c.seed = int(seed)
    c.push_photons = int(push_photons)
    c.soft_photon_filter = int(soft_photon_filter)
    c.thin_cap = int(thin_cap)
    c.restore_on_overflow = int(restore_on_overflow)
    c.block_threads = int(block_threads)
    c.blocks_per_sm = int(blocks_per_sm)
    c.profile = int(profile)
    c.batch_step_budget = int(batch_step_budget)
    c.event_method = int(event_method)
    c.pass_limit = int(pass_limit)
    c.wait_polls = int(wait_polls)
    return c


def make_field(kind: int, params) -> QedFieldDesc:
    f = QedFieldDesc()
    f.kind = int(kind)
    for i, v in enumerate(params):
        f.params[i] = float(v)
    return f


_FIELDS = ("x", "y", "z", "px", "py", "pz", "w")


class DeviceEnsemble:
    """Three species of structure-of-arrays particle buffers in torch device
    memory (caller-owned memory in the sense of the ABI)."""

    def __init__(self, capacity, precision=QED_FP64, device="cuda", optical_depth=False):
        import torch
        self.torch = torch
        self.precision = precision
        self.device = device
        self.fdtype = torch.float32 if precision == QED_FP32 else torch.float64
        self.capacity = [int(c) for c in capacity]
        self.count = [0, 0, 0]
        self.arr = []
        for cap in self.capacity:
            c = max(cap, 1)
            d = {f: torch.zeros(c, dtype=self.fdtype, device=device) for f in _FIELDS}
            d["id"] = torch.zeros(c, dtype=torch.int64, device=device)
            d["nevents"] = torch.zeros(c, dtype=torch.int32, device=device)
            if optical_depth:               # QED_METHOD_OPTICAL_DEPTH: remaining optical depth (0: not drawn)
                d["od"] = torch.zeros(c, dtype=self.fdtype, device=device)
            self.arr.append(d)

    @classmethod
    def from_host(cls, species, capacity, precision=QED_FP64, device="cuda", optical_depth=False):
        """species: 3 dicts of numpy arrays (x..w float64, id uint64[, nevents][, od])."""
        import numpy as np
        e = cls(capacity, precision, device, optical_depth)
        for s, sp in enumerate(species):
            n = len(sp["id"])
            if n > e.capacity[s]:
                raise ValueError("capacity %d < count %d for species %d" % (e.capacity[s], n, s))
            if n == 0:
                continue
            for f in _FIELDS:
                e.arr[s][f][:n].copy_(e.torch.from_numpy(np.asarray(sp[f], dtype=np.float64)).to(e.fdtype))
            e.arr[s]["id"][:n].copy_(e.torch.from_numpy(np.asarray(sp["id"], dtype=np.uint64).view(np.int64)))
            if "nevents" in sp:
                e.arr[s]["nevents"][:n].copy_(e.torch.from_numpy(np.asarray(sp["nevents"], dtype=np.uint32).view(np.int32)))
            if optical_depth and "od" in sp:
                e.arr[s]["od"][:n].copy_(e.torch.from_numpy(np.asarray(sp["od"], dtype=np.float64)).to(e.fdtype))
            e.count[s] = n
        return e

    def struct(self) -> QedParticles:
        """The ABI view of the ensemble.  The pointers are cached while the
        arrays stay the same tensors (a per-step call then only refreshes the
        counts); the returned object is shared between calls."""
        key = tuple(id(t) for d in self.arr for t in d.values())
        P = getattr(self, "_P", None)
        if P is None or self._P_key != key:
            P = QedParticles()
            for s in range(3):
                d = self.arr[s]
                S = P.s[s]
                for f in _FIELDS:
                    setattr(S, f, d[f].data_ptr())
                S.id = d["id"].data_ptr()
                S.nevents = d["nevents"].data_ptr()
            # the cache holds the tensors, so no other object can take one of
            # their ids while the cached pointers are in use
            self._P, self._P_key = P, key
            self._P_refs = [t for d in self.arr for t in d.values()]
        for s in range(3):
            S = P.s[s]
            S.count = self.count[s]
            S.capacity = self.capacity[s]
        return P

    def pull_counts(self, P: QedParticles):
        for s in range(3):
            self.count[s] = int(P.s[s].count)

    def to_host(self, s):
        import numpy as np
        n = self.count[s]
        d = self.arr[s]
        out = {f: d[f][:n].double().cpu().numpy() for f in _FIELDS}
        out["id"] = d["id"][:n].cpu().numpy().view(np.uint64)
        out["nevents"] = d["nevents"][:n].cpu().numpy().view(np.uint32)
        if "od" in d:
            out["od"] = d["od"][:n].double().cpu().numpy()
        return out

    def od_ptrs(self):
        return [d["od"].data_ptr() if "od" in d else 0 for d in self.arr]

    def grow(self, capacity):
        torch = self.torch
        for s in range(3):
            cap = max(int(capacity[s]), self.capacity[s])
            if cap == self.capacity[s]:
                continue
            d = self.arr[s]
            for f in list(d.keys()):
                a = torch.zeros(cap, dtype=d[f].dtype, device=self.device)
                a[: self.count[s]].copy_(d[f][: self.count[s]])
                d[f] = a
            self.capacity[s] = cap


class Generator:
    """Context + ensemble convenience wrapper used by the tests and benchmark."""

    def __init__(self, cfg: QedConfig, stream=None):
        import torch
        self.cfg = cfg
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.ctx = qed_init_tables(cfg, self.stream.cuda_stream)

    def push(self, ens: DeviceEnsemble, field: QedFieldDesc, dt: float, nsteps: int, step0: int = 0,
             auto_grow: bool = True):
        while True:
            self._bind(ens)
            P = ens.struct()
            rc, st = qed_push_and_generate(self.ctx, P, field, dt, nsteps, step0)
            ens.pull_counts(P)
            if rc == QED_OK:
                return st
            if not auto_grow:
                raise QedError(rc, "qed_push_and_generate", st)
            need = [max(2 * ens.capacity[s], 2 * st["needed_capacity"][s]) for s in range(3)]
            ens.grow(need)

    def push_async(self, ens: DeviceEnsemble, field: QedFieldDesc, dt: float, nsteps: int, step0: int = 0):
        """Enqueue steps and return at once; ens.count is stale until wait()."""
        if not getattr(self, "_open", False):
            self._bind(ens)
            self._open = True
        qed_push_async(self.ctx, ens.struct(), field, dt, nsteps, step0)

    def wait(self, ens: DeviceEnsemble):
        """Finish the enqueued steps: counts of ens updated; stats returned.
        A capacity overflow raises (grow the ensemble and replay the batch)."""
        P = ens.struct()
        self._open = False
        rc, st = qed_push_wait(self.ctx, P)
        ens.pull_counts(P)
        if rc != QED_OK:
            raise QedError(rc, "qed_push_wait", st)
        return st

    def _bind(self, ens):
        """The ensemble's optical-depth arrays (bound on every call: buffers
        move when an ensemble grows)."""
        if self.cfg.event_method == QED_METHOD_OPTICAL_DEPTH or any(ens.od_ptrs()):
            qed_set_optical_depth(self.ctx, ens.od_ptrs())

    def compact(self, ens: DeviceEnsemble, step: int):
        self._bind(ens)
        P = ens.struct()
        qed_compact(self.ctx, P, step)
        ens.pull_counts(P)

    def level_sharded(self, ens: DeviceEnsemble, s: int, step: int, cap: int, allreduce) -> float:
        """Global leveling of species s when it is split over ranks (each rank
        calls this with its own shard; allreduce combines the shard sums)."""
        st = level_threshold_sharded(lambda w: qed_level_eval(self.ctx, ens.struct().s[s], s, w), allreduce, cap)
        arr = ens.struct()
        qed_level_apply(self.ctx, arr, s, st.wstar, step)
        ens.pull_counts(arr)
        return st.wstar

    def close(self):
        if self.ctx:
            qed_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
