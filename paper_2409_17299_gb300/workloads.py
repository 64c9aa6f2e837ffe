"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds none of the method's arithmetic: it only draws initial
ensembles and field parameters.  It is the one module that both the CUDA
path's callers and the CPU oracle's callers use.

Normalised units (wavelength 0.8 um): time 1/omega, length c/omega,
momentum m c, fields m c omega / e.  One laser period is 2 pi.

Shapes follow arXiv:2409.17299 Sec. 5.1 (seed e-/e+ at rest in a strong
rotating or standing field, cascade growth) and the benchmark's five
configurations (photon emission in a uniform B at chi0 = 1; a rotating-E
cascade; 64 uneven ensembles; a surrogate sampler; a standing-wave cascade).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi
# m c^2 / (hbar omega) for a 0.8 um wavelength (CODATA 2018): the field, in
# these units, at which chi = 1 for a particle at rest.
R_SCHWINGER = 329718.75885517005

FIELD_UNIFORM, FIELD_ROTATING_E, FIELD_STANDING_CP, FIELD_GRID = 0, 1, 2, 3
SPECIES = ("electron", "positron", "photon")


@dataclass
class Workload:
    name: str
    species: list            # 3 dicts (x,y,z,px,py,pz,w,id) of float64 / uint64 arrays
    field_kind: int
    field_prm: list
    dt: float
    nsteps: int
    push_photons: int = 1
    thin_cap: int = 0
    seed: int = 0
    notes: dict = field(default_factory=dict)

    def counts(self):
        return [len(s["id"]) for s in self.species]


def _empty():
    z = np.zeros(0)
    return {"x": z, "y": z, "z": z, "px": z, "py": z, "pz": z, "w": z,
            "id": np.zeros(0, dtype=np.uint64)}


def _ensemble(x, y, z, px, py, pz, id0=0):
    n = len(x)
    return {"x": np.asarray(x, float), "y": np.asarray(y, float), "z": np.asarray(z, float),
            "px": np.asarray(px, float), "py": np.asarray(py, float), "pz": np.asarray(pz, float),
            "w": np.ones(n), "id": np.arange(id0, id0 + n, dtype=np.uint64)}


def uniform_b_emission(n=16384, seed=0, p0=1000.0, chi0=1.0, steps_per_period=200, nsteps=200):
    """Electrons with momentum p0 along x in a static uniform B along z with
    |B| = chi0 R / p0, so chi = chi0 at the start; photons recorded, not pushed."""
    rng = np.random.default_rng(seed)
    del rng  # every electron starts identical; the seed keys the event streams
    e = _ensemble(np.zeros(n), np.zeros(n), np.zeros(n), np.full(n, p0), np.zeros(n), np.zeros(n))
    bz = chi0 * R_SCHWINGER / p0
    return Workload("uniform_b_emission", [e, _empty(), _empty()], FIELD_UNIFORM,
                    [0, 0, 0, 0, 0, bz], TWO_PI / steps_per_period, nsteps, push_photons=0,
                    seed=seed, notes={"n": n, "p0": p0, "chi0": chi0})


def rotating_e_cascade(n=100000, seed=1, a0=1000.0, radius_wavelengths=0.1, steps_per_period=100,
                       periods=3, thin_cap=50_000_000):
    """Electrons at rest, uniform in a ball of radius 0.1 wavelength, in
    E = a0 (cos t, sin t, 0); Compton + Breit-Wheeler cascade."""
    rng = np.random.default_rng(seed)
    r = radius_wavelengths * TWO_PI * rng.random(n) ** (1.0 / 3.0)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pos = v * r[:, None]
    e = _ensemble(pos[:, 0], pos[:, 1], pos[:, 2], np.zeros(n), np.zeros(n), np.zeros(n))
    return Workload("rotating_e_cascade", [e, _empty(), _empty()], FIELD_ROTATING_E, [a0],
                    TWO_PI / steps_per_period, steps_per_period * periods, push_photons=1,
                    thin_cap=thin_cap, seed=seed, notes={"n": n, "a0": a0})


def standing_wave_cascade(n=1_000_000, seed=4, a0=2000.0, steps_per_period=100, periods=10,
                          thin_cap=200_000_000, sigma_wavelengths=0.05):
    """Electrons at rest near the electric antinode (x = 0) of a standing
    circularly polarised wave; x ~ N(0, (0.05 wavelength)^2) wrapped to the
    periodic wavelength, y and z uniform over one wavelength."""
    rng = np.random.default_rng(seed)
    x = rng.normal(0.0, sigma_wavelengths * TWO_PI, n)
    x = (x + math.pi) % TWO_PI - math.pi
    y = rng.random(n) * TWO_PI
    z = rng.random(n) * TWO_PI
    e = _ensemble(x, y, z, np.zeros(n), np.zeros(n), np.zeros(n))
    return Workload("standing_wave_cascade", [e, _empty(), _empty()], FIELD_STANDING_CP, [a0],
                    TWO_PI / steps_per_period, steps_per_period * periods, push_photons=1,
                    thin_cap=thin_cap, seed=seed, notes={"n": n, "a0": a0})


def paper_test_problem(n=250_000, seed=11, a0=1557.0, steps_per_period=200, periods=5, thin_cap=2_000_000):
    """The paper's test problem (Sec. 5.1): seed electrons and positrons
    (n / 2 each) at rest, uniformly filling the one-wavelength periodic box,
    in the standing circularly polarised wave at the printed amplitude
    6.25e15 V/m (a0 = 1557 in these units), dt = T/200, 5 periods, global
    leveling at thin_cap per species (the paper does not print its cap)."""
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * TWO_PI
    pos[:, 0] -= math.pi                       # x in [-pi, pi): the electric antinode at the box centre
    half = n // 2
    z = np.zeros(n - half)
    e = _ensemble(pos[:half, 0], pos[:half, 1], pos[:half, 2], np.zeros(half), np.zeros(half), np.zeros(half))
    p = _ensemble(pos[half:, 0], pos[half:, 1], pos[half:, 2], z, z, z, id0=half)
    return Workload("paper_test_problem", [e, p, _empty()], FIELD_STANDING_CP, [a0],
                    TWO_PI / steps_per_period, steps_per_period * periods, push_photons=1,
                    thin_cap=thin_cap, seed=seed, notes={"n": n, "a0": a0})


GRID_SHAPE = (128, 4, 4)          # the paper's box: one wavelength, 128 x 4 x 4 cells (Sec. 5.1)


def standing_wave_grid(n=1_000_000, seed=4, a0=2000.0, steps_per_period=100, periods=10,
                       thin_cap=200_000_000):
    """The standing-wave cascade with its field given on a periodic node grid
    (one wavelength cubed, 128 x 4 x 4 nodes) that the caller refills each
    step with grid_values(a0, t): the input a PIC code would pass."""
    w = standing_wave_cascade(n=n, seed=seed, a0=a0, steps_per_period=steps_per_period, periods=periods,
                              thin_cap=thin_cap)
    nx, ny, nz = GRID_SHAPE
    w.name = "standing_wave_grid"
    w.field_kind = FIELD_GRID
    w.field_prm = [nx, ny, nz, TWO_PI, TWO_PI, TWO_PI]
    w.notes["a0"] = a0
    return w


def grid_values(a0, t, shape=GRID_SHAPE):
    """Node values (6, nz, ny, nx) of the standing circularly polarised wave
    E = a0 cos x (0, cos t, sin t), B = a0 sin x (0, cos t, sin t) at time t
    on the one-wavelength grid."""
    nx, ny, nz = shape
    x = np.arange(nx) * TWO_PI / nx
    g = np.zeros((6, nz, ny, nx))
    g[1] = a0 * np.cos(x) * math.cos(t)
    g[2] = a0 * np.cos(x) * math.sin(t)
    g[4] = a0 * np.sin(x) * math.cos(t)
    g[5] = a0 * np.sin(x) * math.sin(t)
    return g


def batched_uniform_b(n_ens=64, seed=2, size_lo=1e3, size_hi=1e6, chi_lo=1e-2, chi_hi=1e2,
                      gamma0=2000.0, steps_per_period=100, nsteps=100, size_scale=1.0):
    """64 independent ensembles, sizes log-uniform in [1e3, 1e6], each in a
    uniform B perpendicular to p with chi0 log-uniform in [1e-2, 1e2]."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(np.exp(rng.uniform(math.log(size_lo), math.log(size_hi), n_ens)) * size_scale).astype(np.int64)
    sizes = np.maximum(sizes, 1)
    chi0 = np.exp(rng.uniform(math.log(chi_lo), math.log(chi_hi), n_ens))
    p0 = math.sqrt(gamma0 * gamma0 - 1.0)
    out = []
    id0 = 0
    for k in range(n_ens):
        n = int(sizes[k])
        e = _ensemble(np.zeros(n), np.zeros(n), np.zeros(n), np.full(n, p0), np.zeros(n), np.zeros(n), id0=id0)
        id0 += n
        bz = chi0[k] * R_SCHWINGER / p0
        out.append(Workload("batched_uniform_b[%d]" % k, [e, _empty(), _empty()], FIELD_UNIFORM,
                            [0, 0, 0, 0, 0, bz], TWO_PI / steps_per_period, nsteps, push_photons=1,
                            seed=seed, notes={"chi0": float(chi0[k]), "n": n}))
    return out


def subset(w: Workload, species: int, idx):
    """A copy of the workload holding only particles idx of one species
    (particles are independent under analytic fields)."""
    sp = []
    for s in range(3):
        src = w.species[s]
        if s == species:
            sp.append({k: np.asarray(v)[idx].copy() for k, v in src.items()})
        else:
            sp.append(_empty())
    return Workload(w.name + "[subset]", sp, w.field_kind, list(w.field_prm), w.dt, w.nsteps,
                    w.push_photons, w.thin_cap, w.seed, dict(w.notes))
