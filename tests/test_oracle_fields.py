"""Pins of the oracle field advance (oracle/pic_oracle.c) to what Sec. 2.1, Sec. 2.2 and
Appendix C fix: the numerical dispersion relation of Eq. wave, the adjoint pair d+/d-, and
div d- x = 0 (Gauss's law is kept by the field advance)."""
import math

import numpy as np
import pytest

from oracle import core as oc
from oracle import fit

RNG = np.random.default_rng(7)
TABLE1 = np.loadtxt(__file__.replace("test_oracle_fields.py", "golden/table1_coefficients.txt"))


def symbol_sq(g, kz, kx, ky=0.0):
    """[k]_1^2 + [k]_2^2 (+ [k]_3^2): Appendix C axial symbol, Yee transverse symbols (Sec. 2.2)."""
    k1 = 2.0 / g.dz * sum(c * math.sin((2 * l + 1) * kz * g.dz / 2) for l, c in enumerate(g.C))
    k2 = 2.0 / g.dx * math.sin(kx * g.dx / 2)
    k3 = 2.0 / g.dy * math.sin(ky * g.dy / 2) if g.ndim == 3 else 0.0
    return k1 * k1 + k2 * k2 + k3 * k3


def mode_field(g, kz, kx, ky, seed):
    rng = np.random.default_rng(seed)
    k_, j_, i_ = np.meshgrid(np.arange(g.ny), np.arange(g.nx), np.arange(g.nz), indexing="ij")
    E = g.zeros()
    for c in range(3):
        ph = rng.uniform(0, 2 * np.pi)
        E[c] = np.cos(kz * i_ * g.dz + kx * j_ * g.dx + ky * k_ * g.dy + ph)
    return E


CASES = [
    ("yee-2d", 2, (1.0,)),
    ("custom-2d", 2, tuple(TABLE1)),
    ("yee-3d", 3, (1.0,)),
    ("custom-3d", 3, (1.1, -0.04, 0.006)),   # any consistent stencil: sum (2l-1) C_l = 1.008
]


@pytest.mark.parametrize("name,ndim,C", CASES)
def test_plane_wave_dispersion(name, ndim, C):
    """Eq. wave: a transverse Fourier mode rotates by theta per step, sin(theta/2) = (dt/2)|[k]|."""
    nz, nx, ny = 40, 12, (6 if ndim == 3 else 1)
    g = oc.Grid(ndim, nz, nx, ny, dz=1.0, dx=1.3, dy=0.9, dt=0.25, C=C, periodic_z=True)
    kz, kx, ky = 2 * np.pi * 3 / (nz * g.dz), 2 * np.pi * 2 / (nx * g.dx), (2 * np.pi / (ny * g.dy) if ndim == 3 else 0.0)
    E = mode_field(g, kz, kx, ky, 1)
    B = g.zeros()
    oc.faraday_half(g, E, B)            # B in the range of d+ x
    E[:] = 0.0
    B0 = B.copy()
    J = g.zeros()
    n = 60
    for _ in range(n):
        oc.field_advance(g, E, B, J)
    theta = 2 * math.asin(g.dt / 2 * math.sqrt(symbol_sq(g, kz, kx, ky)))
    assert np.max(np.abs(B - math.cos(n * theta) * B0)) < 1e-12 * np.max(np.abs(B0))


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


@pytest.mark.parametrize("ndim,C,pz", [(2, (1.0,), False), (2, (1.2, -0.07, 0.01, 0.003), False),
                                       (3, (1.0,), False), (3, (1.1, -0.05, 0.01), True)])
def test_curl_pair_is_adjoint(ndim, C, pz):
    """d- x is the transpose of d+ x (Appendix C: the d+ / d- pair; zero outside z or periodic)."""
    g = oc.Grid(ndim, 7, 5, 4, dz=0.7, dx=1.1, dy=0.8, dt=0.3, C=C, periodic_z=pz)
    T, S = curl_matrices(g)
    assert np.max(np.abs(S - T.T)) < 1e-13 * np.max(np.abs(T))
    assert np.max(np.abs(T)) > 0


@pytest.mark.parametrize("ndim,C", [(2, tuple(TABLE1)), (3, (1.1, -0.05, 0.01))])
def test_ampere_keeps_divergence(ndim, C):
    """With J = 0 the Ampere step leaves d-.E unchanged at every node (div curl = 0)."""
    g = oc.Grid(ndim, 40, 6, 5, dz=0.7, dx=1.1, dy=0.8, dt=0.3, C=C)
    E = RNG.normal(size=g.fshape)
    B = RNG.normal(size=g.fshape)
    rho0 = np.zeros(g.fshape[1:])
    G0 = oc.gauss(g, E, rho0)
    oc.ampere(g, E, B, g.zeros())
    G1 = oc.gauss(g, E, rho0)
    assert np.max(np.abs(G1 - G0)) < 1e-12 * np.max(np.abs(G0))


def test_single_step_from_rest_closed_form():
    """From E = B = 0 one step gives E = -dt J and B = -(dt/2) d+ x (-dt J)."""
    g = oc.Grid(2, 16, 8, dz=0.5, dx=0.5, dt=0.2, C=(1.0,))
    J = RNG.normal(size=g.fshape)
    E, B = g.zeros(), g.zeros()
    oc.field_advance(g, E, B, J)
    assert np.allclose(E, -g.dt * J, rtol=0, atol=1e-15)
    B2 = g.zeros()
    oc.faraday_half(g, -g.dt * J, B2)
    assert np.allclose(B, B2, rtol=0, atol=1e-15)


def test_energy_bounded_under_cfl():
    """Leapfrog with an adjoint pair below the CFL limit keeps the field energy bounded."""
    C = TABLE1
    dt = 0.95 * fit.cfl_dt(1.0, [1.0], C)
    g = oc.Grid(2, 64, 16, dz=1.0, dx=1.0, dt=dt, C=C)
    E = RNG.normal(size=g.fshape)
    B = g.zeros()
    W0 = np.sum(E ** 2)
    for _ in range(200):
        oc.field_advance(g, E, B, g.zeros())
    W = np.sum(E ** 2) + np.sum(B ** 2)
    assert W < 3 * W0
