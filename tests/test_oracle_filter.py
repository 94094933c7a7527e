"""Pins of the oracle's current filter along z (oracle/pic_oracle.c: or_filter_z).

The paper runs with a "5 pass filter" (Sec. 2.2, 2.3, Table 2) without defining it.  The reading:
four binomial passes (1/4, 1/2, 1/4) and one compensating pass (-5/4, 7/2, -5/4) along z.  Its
symbol is pinned by Table 2's three filtered self-forces (tests/test_oracle_kspace.py); the tests
here pin the real-space filter to that symbol and to independent formulations (discrete
convolution, products of tridiagonal matrices), and the whole step's Gauss law with the filter.
"""
import math

import numpy as np
import pytest

from oracle import core as oc
from oracle import fit, kspace

RNG = np.random.default_rng(23)
TABLE1 = np.loadtxt(__file__.replace("test_oracle_filter.py", "golden/table1_coefficients.txt"))


def row_grid(nz, nx=3, periodic_z=False):
    return oc.Grid(2, nz, nx, 1, periodic_z=periodic_z)


@pytest.mark.parametrize("nz", [16, 30])
def test_fourier_modes_scale_by_the_symbol(nz):
    """Periodic z: every discrete mode is an eigenvector with eigenvalue the k-space symbol at
    khat = k dz / 2 = pi m / nz."""
    g = row_grid(nz, nx=2, periodic_z=True)
    i = np.arange(nz)
    for m in range(nz):
        phi = RNG.uniform(0, 2 * math.pi)
        x = np.zeros(g.fshape[1:])
        x[0, 0] = np.cos(2 * math.pi * m * i / nz + phi)
        x[0, 1] = 0.3 * np.sin(2 * math.pi * m * i / nz)
        y = x.copy()
        oc.filter_z(g, y)
        lam = kspace.filter_symbol(math.pi * m / nz)
        assert np.max(np.abs(y - lam * x)) < 1e-13, m


def test_impulse_response_is_the_convolution_of_the_passes():
    """Away from the ends a unit impulse gives the convolution of the five three-point passes:
    binomial(8)/256 convolved with (-5/4, 7/2, -5/4), eleven taps summing to one."""
    nz = 41
    g = row_grid(nz, nx=1)
    x = np.zeros(g.fshape[1:])
    x[0, 0, 20] = 1.0
    oc.filter_z(g, x)
    taps = np.array([1.0])
    for _ in range(4):
        taps = np.convolve(taps, [0.25, 0.5, 0.25])
    assert np.allclose(taps * 256, [math.comb(8, k) for k in range(9)])
    taps = np.convolve(taps, [-1.25, 3.5, -1.25])
    want = np.zeros(nz)
    want[15:26] = taps
    assert np.max(np.abs(x[0, 0] - want)) < 1e-15
    assert taps.sum() == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("nz", [4, 7, 12])
def test_open_ends_are_products_of_truncated_tridiagonal_matrices(nz):
    """Open z (zero outside 0 <= i < nz): each pass is the truncated tridiagonal matrix
    w0 I + w1 (S + S^T), applied in order; the filter is their product."""
    g = row_grid(nz, nx=4)
    x = RNG.normal(size=g.fshape[1:])
    y = x.copy()
    oc.filter_z(g, y)
    T = np.eye(nz, k=1) + np.eye(nz, k=-1)
    Bm = 0.5 * np.eye(nz) + 0.25 * T
    Km = 3.5 * np.eye(nz) - 1.25 * T
    Fm = Km @ np.linalg.matrix_power(Bm, 4)
    want = np.einsum("ab,...b->...a", Fm, x)
    assert np.max(np.abs(y - want)) < 1e-14
    # the passes commute, so the filter is symmetric
    assert np.max(np.abs(Fm - Fm.T)) < 1e-15


def test_nyquist_removed_and_constants_kept():
    g = row_grid(24, nx=2, periodic_z=True)
    alt = np.zeros(g.fshape[1:])
    alt[0, :] = (-1.0) ** np.arange(24)
    oc.filter_z(g, alt)
    assert np.max(np.abs(alt)) < 1e-15
    c = np.full(g.fshape[1:], 2.5)
    oc.filter_z(g, c)
    assert np.max(np.abs(c - 2.5)) < 1e-14


def test_filter_acts_on_every_component_of_a_field_array():
    g = oc.Grid(3, 12, 4, 3)
    J = RNG.normal(size=g.fshape)
    Jf = J.copy()
    oc.filter_z(g, Jf)
    for c in range(3):
        one = J[c].copy()
        oc.filter_z(g, one)
        assert np.array_equal(one, Jf[c])


SIMS = [("yee-quad-2d", 2, 2, None), ("custom-quad-2d", 2, 2, "table1"), ("custom-lin-3d", 3, 1, "fit")]


@pytest.mark.parametrize("name,ndim,shape,solver", SIMS)
def test_whole_step_keeps_gauss_law_for_the_filtered_charge(name, ndim, shape, solver):
    """The filter commutes with the difference operators, so with every current component filtered
    d-.E - F rho is unchanged by a step (away from the open z ends); d-.E - rho is not."""
    nz, nx, ny = (96, 12, 1) if ndim == 2 else (80, 8, 6)
    dz, dx, dy = 0.5, 0.5, 0.5
    if solver is None:
        C, h = (1.0,), None
        dt = 0.9 * fit.cfl_dt(dz, [dx] + ([dy] if ndim == 3 else []))
    else:
        kappa = 3.0
        C = TABLE1 if solver == "table1" else fit.fit_coefficients(kappa, M=8)
        dt = dz / 4.0 if solver == "table1" else dz / kappa
        h = fit.correction_kernel(C, hlen=40)
    g = oc.Grid(ndim, nz, nx, ny, dz, dx, dy, dt, C=C, shape=shape)
    n = 40
    xi = np.zeros((n, 3))
    xi[:, 0] = RNG.uniform(40, 56, n)
    xi[:, 1] = RNG.uniform(0, nx, n)
    if ndim == 3:
        xi[:, 2] = RNG.uniform(0, ny, n)
    u = RNG.normal(size=(n, 3)) * 0.8
    u[:, 0] += 3.0
    sim = oc.Sim(g, [oc.Species(xi, u, -1.0, 1.0, 0.05)], h=h, filt=True)
    G0 = sim.gauss()
    r0 = sim.rho()
    scale = np.max(np.abs(r0))
    for _ in range(12):
        sim.step()
    G = sim.gauss()
    inner = (slice(None),) * (G.ndim - 1) + (slice(45, 70),)
    assert np.max(np.abs(G - G0)[inner]) < 1e-11 * scale
    # against the unfiltered charge the residual moves by O(rho)
    raw = oc.gauss(g, sim.E, sim.rho()) - oc.gauss(g, np.zeros_like(sim.E), r0)
    assert np.max(np.abs(raw)[inner]) > 1e-3 * scale
