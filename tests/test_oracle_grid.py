"""Pins for the oracle's gridded field (trilinear interpolation on a periodic
node grid, the field a PIC step holds constant during the step): node values
are returned exactly, multilinear functions are reproduced exactly inside the
box, the interpolant is periodic and continuous across cell faces, and a
smooth field is approximated to second order in the cell size."""
import math

import numpy as np
import pytest

import oracle

NX, NY, NZ = 8, 4, 4
L = (2 * math.pi, 1.0, 1.5)
PRM = (NX, NY, NZ, *L)


def _nodes():
    i, j, k = np.meshgrid(np.arange(NX), np.arange(NY), np.arange(NZ), indexing="ij")
    return i * L[0] / NX, j * L[1] / NY, k * L[2] / NZ      # arrays indexed [i, j, k]


def _grid_from(fun):
    """Node values of fun(x, y, z) -> six components, layout (6, nz, ny, nx)."""
    x, y, z = _nodes()
    comps = fun(x, y, z)
    return np.stack([np.transpose(c, (2, 1, 0)) for c in comps])


def _eval(x):
    return oracle.field(oracle.FIELD_GRID, PRM, np.asarray(x, dtype=np.float64), 0.0)


def test_node_values_exact():
    rng = np.random.default_rng(1)
    g = rng.normal(size=(6, NZ, NY, NX))
    oracle.set_field_grid(g)
    for i, j, k in [(0, 0, 0), (3, 1, 2), (NX - 1, NY - 1, NZ - 1)]:
        E, B = _eval([i * L[0] / NX, j * L[1] / NY, k * L[2] / NZ])
        assert np.array_equal(np.concatenate([E, B]), g[:, k, j, i])


def test_multilinear_reproduced_inside_box():
    # f = a + b x + c y + d z + e x y + f y z + g x z + h x y z is trilinear
    coef = np.arange(1, 9) * 0.37

    def f(x, y, z):
        v = (coef[0] + coef[1] * x + coef[2] * y + coef[3] * z + coef[4] * x * y + coef[5] * y * z
             + coef[6] * x * z + coef[7] * x * y * z)
        return [v * (c + 1) for c in range(6)]
    oracle.set_field_grid(_grid_from(f))
    rng = np.random.default_rng(2)
    for _ in range(200):
        # stay inside the last cell in every direction (no periodic wrap)
        p = rng.random(3) * np.array([L[0] * (NX - 1) / NX, L[1] * (NY - 1) / NY, L[2] * (NZ - 1) / NZ])
        E, B = _eval(p)
        want = f(*[np.array(t) for t in p])
        assert np.allclose(np.concatenate([E, B]), np.array(want, dtype=float), rtol=1e-13, atol=1e-13)


def test_periodic_and_continuous():
    rng = np.random.default_rng(3)
    oracle.set_field_grid(rng.normal(size=(6, NZ, NY, NX)))
    for _ in range(100):
        p = rng.random(3) * np.array(L)
        a = np.concatenate(_eval(p))
        shifted = p + np.array(L) * rng.integers(-3, 4, size=3)
        b = np.concatenate(_eval(shifted))
        assert np.allclose(a, b, rtol=0, atol=1e-12)
    # across the wrap face x = Lx: values just inside and just outside agree
    p = np.array([L[0] - 1e-12, 0.3, 0.7])
    a = np.concatenate(_eval(p))
    b = np.concatenate(_eval(p + np.array([2e-12, 0, 0])))
    assert np.allclose(a, b, atol=1e-9)


@pytest.mark.parametrize("n", [8, 16, 32])
def test_second_order_in_cell_size(n):
    """Interpolating the standing wave's E_y = a0 cos x (t = 0) on grids of n
    cells per wavelength: the error falls as (h)^2 (ratio ~4 per halving)."""
    errs = []
    for nx in (n, 2 * n):
        prm = (nx, 1, 1, 2 * math.pi, 1.0, 1.0)
        xs = np.arange(nx) * 2 * math.pi / nx
        g = np.zeros((6, 1, 1, nx))
        g[1, 0, 0, :] = np.cos(xs)
        oracle.set_field_grid(g)
        pts = np.linspace(0, 2 * math.pi, 997)
        err = max(abs(oracle.field(oracle.FIELD_GRID, prm, np.array([x, 0.2, 0.4]), 0.0)[0][1] - math.cos(x))
                  for x in pts)
        errs.append(err)
    ratio = errs[0] / errs[1]
    assert 3.5 < ratio < 4.5, (n, errs)
    assert errs[0] <= (2 * math.pi / n) ** 2 / 8 * 1.001      # max |f''| h^2 / 8
