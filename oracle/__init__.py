"""Plain FP64 CPU oracle for the strong-field QED event generator.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never uses it and shares no code with it.

The arithmetic lives in ``sfqed_oracle.c`` (plain C, FP64, IEEE, no FMA
contraction); this module only compiles it with gcc and marshals numpy
arrays through ctypes.  Every function of the C file cites the passage of
arXiv:2409.17299 it restates.

Parity status: every C function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py``; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfqed_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

EM_NCHI, EM_NS = 121, 257
PAIR_NCHI, PAIR_NS = 101, 129
CHEB_N = 11

FIELD_UNIFORM, FIELD_ROTATING_E, FIELD_STANDING_CP, FIELD_GRID = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library with gcc (no CUDA)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-std=gnu11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class Species(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("px", C.c_void_p), ("py", C.c_void_p), ("pz", C.c_void_p),
                ("w", C.c_void_p), ("id", C.c_void_p), ("nevents", C.c_void_p),
                ("od", C.c_void_p), ("count", C.c_int64), ("capacity", C.c_int64)]


class RunCfg(C.Structure):
    _fields_ = [("push_photons", C.c_int), ("soft_photon_filter", C.c_int),
                ("thin_cap", C.c_int64), ("seed", C.c_uint64),
                ("field_kind", C.c_int), ("field_prm", C.c_double * 16),
                ("event_method", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("particle_steps", C.c_int64), ("emit_events", C.c_int64),
                ("pair_events", C.c_int64), ("needed_capacity", C.c_int64 * 3),
                ("max_subevents", C.c_int64), ("overflow", C.c_int64)]

    def as_dict(self):
        return {"particle_steps": self.particle_steps, "emit_events": self.emit_events,
                "pair_events": self.pair_events, "needed_capacity": list(self.needed_capacity),
                "max_subevents": self.max_subevents, "overflow": self.overflow}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, p, i64, u32, i32 = C.c_double, C.c_void_p, C.c_int64, C.c_uint32, C.c_int
            sig = {
                "or_philox_batch": (None, [i64, p, p, p]),
                "or_u52": (d, [u32, u32]),
                "or_besselK": (d, [d, d]),
                "or_intK13": (d, [d]),
                "or_em_bracket": (d, [d, d]),
                "or_pair_bracket": (d, [d, d]),
                "or_F_gamma_quad": (d, [d]),
                "or_F_pair_quad": (d, [d]),
                "or_build_rate_coefs": (None, [p, p]),
                "or_rate_F": (d, [p, p, i32, d]),
                "or_build_icdf_tables": (None, [p, p]),
                "or_em_cdf": (d, [d, d]),
                "or_pair_cdf": (d, [d, d]),
                "or_sample_emission": (d, [p, d, d, p]),
                "or_sample_pair": (d, [p, d, d, p]),
                "or_field": (None, [i32, p, p, d, p, p]),
                "or_set_field_grid": (None, [p]),
                "or_rejection_run": (C.c_int64, [p, p, d, i32, i32, C.c_uint64, p, C.c_int64, p]),
                "or_chi": (d, [d, p, p, p]),
                "or_boris": (None, [p, p, d, p, p, d]),
                "or_compact": (None, [p]),
                "or_level_threshold": (d, [p, i64, i64]),
                "or_level": (d, [p, i64, C.c_uint64, u32]),
                "or_push_and_generate": (i32, [p, p, p, p, p, p, d, i32, i64, p]),
                "or_rate_lambda": (d, [p, p, i32, p, p, p]),
                "or_const": (d, [i32]),
                "or_mlp_nparams": (i32, []),
                "or_mlp_forward": (None, [p, i64, p, p]),
                "or_mlp_loss_grad": (d, [p, i64, p, p, p]),
                "or_mlp_forward_q": (None, [p, i64, p, p]),
                "or_mlp_loss_grad_q": (d, [p, i64, p, p, p]),
                "or_mlp_features": (None, [d, d, p]),
                "or_mlp_delta": (d, [d, d, p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


ALPHA = None
R = None


def constants():
    L = lib()
    return L.or_const(0), L.or_const(1)


# --------------------------------------------------------------------------
# Philox4x32-10
# --------------------------------------------------------------------------
def philox(ctr: np.ndarray, key) -> np.ndarray:
    """ctr: (n,4) uint32 counters, key: 2 uint32 words -> (n,4) uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(ctr)
    lib().or_philox_batch(ctr.shape[0], _ptr(ctr), _ptr(k), _ptr(out))
    return out


def u52(a: int, b: int) -> float:
    return lib().or_u52(int(a), int(b))


# --------------------------------------------------------------------------
# special functions, spectra, rates
# --------------------------------------------------------------------------
def besselK(nu: float, y: float) -> float:
    return lib().or_besselK(float(nu), float(y))


def intK13(y: float) -> float:
    return lib().or_intK13(float(y))


def em_bracket(chi, delta):
    return lib().or_em_bracket(float(chi), float(delta))


def pair_bracket(chi, delta):
    return lib().or_pair_bracket(float(chi), float(delta))


def F_gamma_quad(chi: float) -> float:
    return lib().or_F_gamma_quad(float(chi))


def F_pair_quad(chi: float) -> float:
    return lib().or_F_pair_quad(float(chi))


def em_cdf(chi, delta):
    return lib().or_em_cdf(float(chi), float(delta))


def pair_cdf(chi, delta):
    return lib().or_pair_cdf(float(chi), float(delta))


class Tables:
    """Rate coefficients and inverse-CDF tables, built by the oracle itself."""

    def __init__(self, cheb_em, cheb_pair, icdf_em, icdf_pair):
        self.cheb_em = np.ascontiguousarray(cheb_em, dtype=np.float64)
        self.cheb_pair = np.ascontiguousarray(cheb_pair, dtype=np.float64)
        self.icdf_em = np.ascontiguousarray(icdf_em, dtype=np.float64)
        self.icdf_pair = np.ascontiguousarray(icdf_pair, dtype=np.float64)

    def rate_F(self, is_photon: bool, chi: float) -> float:
        return lib().or_rate_F(_ptr(self.cheb_em), _ptr(self.cheb_pair), int(is_photon), float(chi))

    def sample_emission(self, chi: float, u: float):
        om = np.zeros(1)
        d = lib().or_sample_emission(_ptr(self.icdf_em), float(chi), float(u), _ptr(om))
        return d, float(om[0])

    def sample_pair(self, chi: float, u: float):
        om = np.zeros(1)
        d = lib().or_sample_pair(_ptr(self.icdf_pair), float(chi), float(u), _ptr(om))
        return d, float(om[0])

    def rate_lambda(self, is_photon, p, E, B):
        p = np.ascontiguousarray(p, dtype=np.float64)
        E = np.ascontiguousarray(E, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
        return lib().or_rate_lambda(_ptr(self.cheb_em), _ptr(self.cheb_pair), int(is_photon),
                                    _ptr(p), _ptr(E), _ptr(B))


_tables_cache = None


def build_tables() -> Tables:
    """Build (once per process) the oracle's own rate coefficients and tables."""
    global _tables_cache
    with _lock:
        if _tables_cache is not None:
            return _tables_cache
    cache = os.path.join(_BUILD, "tables_v1.npz")
    if os.path.exists(cache) and os.path.getmtime(cache) > os.path.getmtime(_SRC):
        z = np.load(cache)
        t = Tables(z["cheb_em"], z["cheb_pair"], z["icdf_em"], z["icdf_pair"])
    else:
        L = lib()
        ce = np.zeros(6 * CHEB_N)
        cp = np.zeros(5 * CHEB_N)
        ie = np.zeros(EM_NCHI * EM_NS)
        ip = np.zeros(PAIR_NCHI * PAIR_NS)
        L.or_build_rate_coefs(_ptr(ce), _ptr(cp))
        L.or_build_icdf_tables(_ptr(ie), _ptr(ip))
        t = Tables(ce, cp, ie, ip)
        os.makedirs(_BUILD, exist_ok=True)
        tmp = cache + ".%d.tmp.npz" % os.getpid()
        np.savez(tmp, cheb_em=ce, cheb_pair=cp, icdf_em=ie, icdf_pair=ip)
        os.replace(tmp, cache)
    with _lock:
        _tables_cache = t
    return t


# --------------------------------------------------------------------------
# fields, chi, Boris
# --------------------------------------------------------------------------
def field(kind: int, prm, x, t):
    prm16 = np.zeros(16)
    prm16[: len(prm)] = prm
    x = np.ascontiguousarray(x, dtype=np.float64)
    E = np.zeros(3)
    B = np.zeros(3)
    lib().or_field(int(kind), _ptr(prm16), _ptr(x), float(t), _ptr(E), _ptr(B))
    return E, B


_grid_keep = None


def set_field_grid(g):
    """Node values of the gridded field (FIELD_GRID), shape (6, nz, ny, nx):
    E_x, E_y, E_z, B_x, B_y, B_z.  The oracle keeps a reference until the
    next call; field_prm of the run is (nx, ny, nz, Lx, Ly, Lz)."""
    global _grid_keep
    _grid_keep = np.ascontiguousarray(g, dtype=np.float64)
    lib().or_set_field_grid(_ptr(_grid_keep))


def rejection_run(ens: "Ensemble", cfg: "RunCfg", dt: float, nsteps: int, nsub: int, seed: int,
                  delta_cap: int = 1 << 22):
    """The subcycled rejection generator on the electrons of ens (species 0,
    updated in place): returns (photon energies, emission count, largest
    acceptance probability)."""
    arr = ens.structs()
    out = np.zeros(delta_cap)
    amax = np.zeros(1)
    n = lib().or_rejection_run(C.cast(C.byref(arr[0]), C.c_void_p), C.byref(cfg), float(dt), int(nsteps),
                               int(nsub), C.c_uint64(seed), _ptr(out), int(delta_cap), _ptr(amax))
    ens.pull(arr)
    return out[: min(n, delta_cap)].copy(), int(n), float(amax[0])


def chi(e0, p, E, B) -> float:
    p = np.ascontiguousarray(p, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    return lib().or_chi(float(e0), _ptr(p), _ptr(E), _ptr(B))


def boris(x, p, q, E, B, h):
    x = np.array(x, dtype=np.float64)
    p = np.array(p, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    lib().or_boris(_ptr(x), _ptr(p), float(q), _ptr(E), _ptr(B), float(h))
    return x, p


# --------------------------------------------------------------------------
# ensembles and the step
# --------------------------------------------------------------------------
_FIELDS = ("x", "y", "z", "px", "py", "pz", "w")
_ALL = _FIELDS + ("id", "nevents", "od")
METHOD_SUBSTEP, METHOD_OPTICAL_DEPTH = 0, 1


class Ensemble:
    """Three species (0 e-, 1 e+, 2 photon) of FP64 SoA arrays with capacity."""

    def __init__(self, capacity=(1024, 1024, 1024)):
        self.sp = []
        for cap in capacity:
            d = {f: np.zeros(cap) for f in _FIELDS}
            d["id"] = np.zeros(cap, dtype=np.uint64)
            d["nevents"] = np.zeros(cap, dtype=np.uint32)
            d["od"] = np.zeros(cap)       # remaining optical depth, 0 = not drawn yet
            d["count"] = 0
            self.sp.append(d)

    @classmethod
    def from_arrays(cls, species_arrays, capacity):
        """species_arrays: list of 3 dicts with x,y,z,px,py,pz,w,id[,nevents][,od]."""
        e = cls(capacity)
        for s, arr in enumerate(species_arrays):
            n = len(arr["id"]) if arr is not None else 0
            if n > capacity[s]:
                raise ValueError("capacity too small")
            for f in _FIELDS:
                if n:
                    e.sp[s][f][:n] = arr[f]
            if n:
                e.sp[s]["id"][:n] = arr["id"]
                for f in ("nevents", "od"):
                    if f in arr:
                        e.sp[s][f][:n] = arr[f]
            e.sp[s]["count"] = n
        return e

    def structs(self):
        arr = (Species * 3)()
        for s in range(3):
            d = self.sp[s]
            for f in _ALL:
                setattr(arr[s], f, d[f].ctypes.data)
            arr[s].count = d["count"]
            arr[s].capacity = len(d["id"])
        return arr

    def pull(self, arr):
        for s in range(3):
            self.sp[s]["count"] = int(arr[s].count)

    def grow(self, capacity):
        for s in range(3):
            d = self.sp[s]
            cap = max(capacity[s], len(d["id"]))
            if cap == len(d["id"]):
                continue
            for f in _ALL:
                a = np.zeros(cap, dtype=d[f].dtype)
                a[: len(d[f])] = d[f]
                d[f] = a

    def copy(self):
        e = Ensemble([len(d["id"]) for d in self.sp])
        for s in range(3):
            for f in _ALL:
                e.sp[s][f][:] = self.sp[s][f]
            e.sp[s]["count"] = self.sp[s]["count"]
        return e

    def view(self, s):
        d = self.sp[s]
        n = d["count"]
        return {f: d[f][:n].copy() for f in _ALL}


def make_cfg(seed=0, push_photons=1, soft_photon_filter=0, thin_cap=0,
             field_kind=FIELD_UNIFORM, field_prm=(), event_method=METHOD_SUBSTEP):
    c = RunCfg()
    c.event_method = int(event_method)
    c.push_photons = int(push_photons)
    c.soft_photon_filter = int(soft_photon_filter)
    c.thin_cap = int(thin_cap)
    c.seed = int(seed)
    c.field_kind = int(field_kind)
    for i, v in enumerate(field_prm):
        c.field_prm[i] = float(v)
    return c


def push_and_generate(ens: Ensemble, tables: Tables, cfg: RunCfg, dt: float, nsteps: int,
                      step0: int = 0, auto_grow: bool = True) -> dict:
    """Run nsteps steps of Algorithm 2 over the ensemble, in place.

    On capacity overflow the ensemble is restored from a copy, grown, and the
    whole call repeated: the counter-based random streams make the repeat
    identical."""
    backup = ens.copy() if auto_grow else None
    while True:
        st = Stats()
        arr = ens.structs()
        rc = lib().or_push_and_generate(C.cast(arr, C.c_void_p), _ptr(tables.cheb_em), _ptr(tables.cheb_pair),
                                        _ptr(tables.icdf_em), _ptr(tables.icdf_pair), C.byref(cfg),
                                        float(dt), int(nsteps), int(step0), C.byref(st))
        ens.pull(arr)
        if rc == 0:
            return st.as_dict()
        if not auto_grow:
            raise RuntimeError("oracle: capacity overflow %s" % (st.as_dict(),))
        need = [max(2 * len(backup.sp[s]["id"]), 2 * int(st.needed_capacity[s])) for s in range(3)]
        ens.__dict__.update(backup.copy().__dict__)
        ens.grow(need)
        backup.grow(need)


def level(ens: Ensemble, species: int, cap: int, seed: int, step: int) -> float:
    arr = ens.structs()
    ws = lib().or_level(C.cast(C.byref(arr[species]), C.c_void_p), int(cap), int(seed), int(step))
    ens.pull(arr)
    return ws


def level_threshold(w: np.ndarray, cap: int) -> float:
    w = np.ascontiguousarray(w, dtype=np.float64)
    return lib().or_level_threshold(_ptr(w), len(w), int(cap))


def compact(ens: Ensemble, species: int):
    arr = ens.structs()
    lib().or_compact(C.cast(C.byref(arr[species]), C.c_void_p))
    ens.pull(arr)


# --------------------------------------------------------------------------
# surrogate network (FP64 reference of the forward and backward passes)
# --------------------------------------------------------------------------
def mlp_nparams() -> int:
    return lib().or_mlp_nparams()


def mlp_forward(params, feat, bf16_storage=False) -> np.ndarray:
    """Network output; bf16_storage: hidden activations stored as bfloat16."""
    P = np.ascontiguousarray(params, dtype=np.float64)
    F = np.ascontiguousarray(feat, dtype=np.float64).reshape(-1, 2)
    y = np.zeros(F.shape[0])
    f = lib().or_mlp_forward_q if bf16_storage else lib().or_mlp_forward
    f(_ptr(P), F.shape[0], _ptr(F), _ptr(y))
    return y


def mlp_loss_grad(params, feat, target, bf16_storage=False):
    """Mean squared error and its gradient; bf16_storage: activations and
    back-propagated deltas stored as bfloat16."""
    P = np.ascontiguousarray(params, dtype=np.float64)
    F = np.ascontiguousarray(feat, dtype=np.float64).reshape(-1, 2)
    T = np.ascontiguousarray(target, dtype=np.float64)
    g = np.zeros_like(P)
    f = lib().or_mlp_loss_grad_q if bf16_storage else lib().or_mlp_loss_grad
    loss = f(_ptr(P), F.shape[0], _ptr(F), _ptr(T), _ptr(g))
    return loss, g


def mlp_features(chi, u):
    f = np.zeros(2)
    lib().or_mlp_features(float(chi), float(u), _ptr(f))
    return f


def mlp_delta(chi, y):
    om = np.zeros(1)
    d = lib().or_mlp_delta(float(chi), float(y), _ptr(om))
    return d, float(om[0])
