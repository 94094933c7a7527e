"""Pins of the oracle's split axial operators: Sec. 3 notes that solvers with [k]_E1 != [k]_B1
(the E-side d+ of Faraday's law and the B-side d- of Ampere's and Gauss's laws built from
different coefficients) and [k]_E1 [k]_B1 = [k1]_t^2 are possible.  What the mathematics fixes:
the dispersion relation of Eq. wave with the product [k]_E . [k]_B, the transpose relation of
each coefficient set's d+ / d- pair, div curl = 0 for the B-side d-, and Gauss's law kept by
whole steps when the Sec. 3 correction is built from the B-side coefficients."""
import math

import numpy as np
import pytest

from oracle import core as oc
from oracle import fit

RNG = np.random.default_rng(19)
TABLE1 = np.loadtxt(__file__.replace("test_oracle_split.py", "golden/table1_coefficients.txt"))

# (E-side, B-side) pairs: Yee against a fitted stencil, and two unrelated consistent stencils
PAIRS = [
    ("yee-E-fit-B", (1.0,), tuple(fit.fit_coefficients(3.0, M=8))),
    ("fit-E-yee-B", tuple(fit.fit_coefficients(3.0, M=8)), (1.0,)),
    ("two-stencils", (1.1, -0.04, 0.006), (0.95, 0.02, -0.003, 0.001)),
]


def axial(C, kz, dz):
    return 2.0 / dz * sum(c * math.sin((2 * l + 1) * kz * dz / 2) for l, c in enumerate(C))


@pytest.mark.parametrize("name,CE,CB", PAIRS)
@pytest.mark.parametrize("ndim", [2, 3])
def test_dispersion_uses_the_product_of_the_axial_symbols(name, CE, CB, ndim):
    """Eq. wave with [k]_E . [k]_B: a mode started in the range of d+ x rotates by theta per step,
    sin(theta/2) = (dt/2) sqrt([k]_E1 [k]_B1 + [k]_2^2 (+ [k]_3^2))."""
    nz, nx, ny = 40, 12, (6 if ndim == 3 else 1)
    g = oc.Grid(ndim, nz, nx, ny, dz=1.0, dx=1.3, dy=0.9, dt=0.25, C=CE, Cb=CB, periodic_z=True)
    assert g.dt < fit.cfl_dt(g.dz, [g.dx] + ([g.dy] if ndim == 3 else []), CE, Cb=CB)
    kz, kx = 2 * np.pi * 3 / (nz * g.dz), 2 * np.pi * 2 / (nx * g.dx)
    ky = 2 * np.pi / (ny * g.dy) if ndim == 3 else 0.0
    k_, j_, i_ = np.meshgrid(np.arange(g.ny), np.arange(g.nx), np.arange(g.nz), indexing="ij")
    E = g.zeros()
    for c in range(3):
        E[c] = np.cos(kz * i_ * g.dz + kx * j_ * g.dx + ky * k_ * g.dy + RNG.uniform(0, 2 * np.pi))
    B = g.zeros()
    oc.faraday_half(g, E, B)
    E[:] = 0.0
    B0 = B.copy()
    J = g.zeros()
    n = 60
    for _ in range(n):
        oc.field_advance(g, E, B, J)
    kk = axial(CE, kz, g.dz) * axial(CB, kz, g.dz) + (2 / g.dx * math.sin(kx * g.dx / 2)) ** 2
    if ndim == 3:
        kk += (2 / g.dy * math.sin(ky * g.dy / 2)) ** 2
    theta = 2 * math.asin(g.dt / 2 * math.sqrt(kk))
    assert np.max(np.abs(B - math.cos(n * theta) * B0)) < 1e-12 * np.max(np.abs(B0))
    # the symmetric solver of either set rotates at another rate: the product is what counts
    for C in (CE, CB):
        k1 = axial(C, kz, g.dz) ** 2 + kk - axial(CE, kz, g.dz) * axial(CB, kz, g.dz)
        th = 2 * math.asin(g.dt / 2 * math.sqrt(k1))
        assert abs(math.cos(n * th) - math.cos(n * theta)) > 1e-6


def curl_matrices(g):
    N = g.nz * g.nx * g.ny
    T = np.zeros((3 * N, 3 * N))
    S = np.zeros((3 * N, 3 * N))
    J = g.zeros()
    for c in range(3 * N):
        E = g.zeros()
        E.reshape(-1)[c] = 1.0
        B = g.zeros()
        oc.faraday_half(g, E, B)
        T[:, c] = -B.reshape(-1) / (0.5 * g.dt)
        E2 = g.zeros()
        Bu = g.zeros()
        Bu.reshape(-1)[c] = 1.0
        oc.ampere(g, E2, Bu, J)
        S[:, c] = E2.reshape(-1) / g.dt
    return T, S


@pytest.mark.parametrize("name,CE,CB", PAIRS)
def test_each_side_uses_its_own_coefficients(name, CE, CB):
    """Faraday's d+ x is that of the E-side set, Ampere's d- x the transpose of the B-side set's d+ x."""
    kw = dict(dz=0.7, dx=1.1, dy=0.8, dt=0.3)
    split = oc.Grid(3, 7, 5, 4, C=CE, Cb=CB, **kw)
    Te, _ = curl_matrices(oc.Grid(3, 7, 5, 4, C=CE, **kw))
    Tb, _ = curl_matrices(oc.Grid(3, 7, 5, 4, C=CB, **kw))
    T, S = curl_matrices(split)
    assert np.max(np.abs(T - Te)) < 1e-13 * np.max(np.abs(Te))
    assert np.max(np.abs(S - Tb.T)) < 1e-13 * np.max(np.abs(Tb))
    assert np.max(np.abs(S - Te.T)) > 1e-3


@pytest.mark.parametrize("name,CE,CB", PAIRS)
def test_ampere_keeps_the_b_side_divergence(name, CE, CB):
    g = oc.Grid(2, 40, 6, 1, dz=0.7, dx=1.1, dt=0.3, C=CE, Cb=CB)
    E = RNG.normal(size=g.fshape)
    B = RNG.normal(size=g.fshape)
    rho0 = np.zeros(g.fshape[1:])
    G0 = oc.gauss(g, E, rho0)
    oc.ampere(g, E, B, g.zeros())
    G1 = oc.gauss(g, E, rho0)
    assert np.max(np.abs(G1 - G0)) < 1e-12 * np.max(np.abs(G0))


@pytest.mark.parametrize("ndim,shape", [(2, 2), (3, 1)])
@pytest.mark.parametrize("name,CE,CB", PAIRS)
def test_whole_step_keeps_gauss_law_with_the_b_side_correction(name, CE, CB, ndim, shape):
    """Esirkepov's current satisfies the Yee continuity equation; with J1 <- P_B^-1 J1, P_B the
    B-side symbol over the Yee symbol, d-.E - rho (B-side d-) is unchanged by every step."""
    nz, nx, ny = (96, 12, 1) if ndim == 2 else (80, 8, 6)
    dz, dx, dy = 0.5, 0.5, 0.5
    dt = 0.8 * fit.cfl_dt(dz, [dx] + ([dy] if ndim == 3 else []), CE, Cb=CB)
    h = None if len(CB) == 1 else fit.correction_kernel(CB, hlen=40)
    g = oc.Grid(ndim, nz, nx, ny, dz, dx, dy, dt, C=CE, Cb=CB, shape=shape)
    n = 40
    xi = np.zeros((n, 3))
    xi[:, 0] = RNG.uniform(40, 56, n)
    xi[:, 1] = RNG.uniform(0, nx, n)
    if ndim == 3:
        xi[:, 2] = RNG.uniform(0, ny, n)
    u = RNG.normal(size=(n, 3)) * 0.8
    u[:, 0] += 3.0
    sim = oc.Sim(g, [oc.Species(xi, u, -1.0, 1.0, 0.05)], h=h)
    G0 = sim.gauss()
    scale = np.max(np.abs(sim.rho()))
    for _ in range(12):
        sim.step()
    G = sim.gauss()
    inner = (slice(None),) * (G.ndim - 1) + (slice(45, 70),)
    assert np.max(np.abs(G - G0)[inner]) < 1e-11 * scale
    assert np.max(np.abs(sim.E)) > 1e-3 * scale * dz


def test_cfl_of_a_split_pair_is_that_of_the_product():
    CE, CB = (1.0,), tuple(fit.fit_coefficients(3.0, M=8))
    kh = np.linspace(0, math.pi / 2, 20001)
    prod = fit.axial_symbol(CE, kh) * fit.axial_symbol(CB, kh)
    want = 2.0 / math.sqrt(prod.max() * 4.0 + 4.0)
    assert fit.cfl_dt(1.0, [1.0], CE, Cb=CB) == pytest.approx(want, rel=1e-12)
    with pytest.raises(ValueError):
        fit.cfl_dt(1.0, [1.0], (1.0,), Cb=(-1.0,))
