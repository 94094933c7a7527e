"""Pins of the oracle particle routines: gather, Boris push, Esirkepov deposition, and the whole
step's conservation of Gauss's law (Sec. 2.1: Gauss's law is kept by charge conservation)."""
import math

import numpy as np
import pytest

from oracle import core as oc
from oracle import fit

RNG = np.random.default_rng(11)
TABLE1 = np.loadtxt(__file__.replace("test_oracle_particles.py", "golden/table1_coefficients.txt"))
STAG = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]


def rand_xi(g, n, margin=4):
    xi = np.zeros((n, 3))
    xi[:, 0] = RNG.uniform(margin, g.nz - margin, n)
    xi[:, 1] = RNG.uniform(0, g.nx, n)
    if g.ndim == 3:
        xi[:, 2] = RNG.uniform(0, g.ny, n)
    return xi


@pytest.mark.parametrize("ndim,shape", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_gather_reproduces_linear_fields(ndim, shape):
    """B-spline interpolation is exact for fields linear in z and constant across x, y (any
    staggering): this fixes the half-cell offsets of all six components."""
    g = oc.Grid(ndim, 24, 8, 6, dz=0.4, dx=0.3, dy=0.2, dt=0.1, shape=shape)
    E, B = g.zeros(), g.zeros()
    i_ = np.arange(g.nz)[None, None, :]
    coef = RNG.normal(size=(6, 2))
    for c in range(6):
        f = coef[c, 0] + coef[c, 1] * (i_ + STAG[c][0]) + 0 * np.zeros(g.fshape[1:])
        (E if c < 3 else B)[c % 3] = f
    xi = rand_xi(g, 50)
    out = oc.gather(g, E, B, xi)
    for c in range(6):
        assert np.allclose(out[:, c], coef[c, 0] + coef[c, 1] * xi[:, 0], rtol=0, atol=1e-12)


@pytest.mark.parametrize("ndim,shape", [(2, 1), (2, 2), (3, 2)])
def test_gather_transverse_linear_on_periodic_axis(ndim, shape):
    """Along x the interpolation of a field linear in x (away from the periodic seam) is exact."""
    g = oc.Grid(ndim, 12, 32, 6, dz=0.4, dx=0.3, dy=0.2, dt=0.1, shape=shape)
    E, B = g.zeros(), g.zeros()
    j_ = np.arange(g.nx)[None, :, None]
    for c in range(6):
        (E if c < 3 else B)[c % 3] = 0.3 + 0.7 * (j_ + STAG[c][1]) + np.zeros(g.fshape[1:])
    xi = rand_xi(g, 40)
    xi[:, 1] = RNG.uniform(4, g.nx - 4, 40)
    out = oc.gather(g, E, B, xi)
    assert np.allclose(out, (0.3 + 0.7 * xi[:, 1])[:, None], atol=1e-12)


def test_boris_uniform_magnetic_field():
    """Uniform B: |u| is kept and u turns by 2 atan(|eps B|/gamma) per step about B."""
    n = 5
    u = RNG.normal(size=(n, 3)) * 3
    Bv = np.array([0.2, -0.5, 0.9])
    eb = np.zeros((n, 6))
    eb[:, 3:] = Bv
    eps = -0.3
    u0 = u.copy()
    steps = 37
    for _ in range(steps):
        oc.boris(eb, u, eps)
    gam = np.sqrt(1 + np.sum(u0 ** 2, axis=1))
    bhat = Bv / np.linalg.norm(Bv)
    for p in range(n):
        ang = steps * 2 * math.atan(abs(eps) * np.linalg.norm(Bv) / gam[p])
        ang = ang * (-1 if eps > 0 else 1)   # rotation sense of the charge
        par = np.dot(u0[p], bhat) * bhat
        perp = u0[p] - par
        rot = par + perp * math.cos(ang) + np.cross(bhat, perp) * math.sin(ang)
        assert np.allclose(u[p], rot, atol=1e-11)
        assert np.linalg.norm(u[p]) == pytest.approx(np.linalg.norm(u0[p]), rel=1e-13)


def test_boris_uniform_electric_field():
    """B = 0: u^{n+1/2} = u^{n-1/2} + 2 eps E exactly (eps = q dt / 2m)."""
    u = RNG.normal(size=(4, 3))
    eb = np.zeros((4, 6))
    eb[:, :3] = [0.3, -1.0, 2.0]
    u0 = u.copy()
    for _ in range(10):
        oc.boris(eb, u, 0.05)
    assert np.allclose(u, u0 + 10 * 2 * 0.05 * eb[:, :3], atol=1e-13)


def _continuity(g, xi0, xi1, u, Q):
    J = g.zeros()
    oc.deposit(g, xi0, xi1, u, Q, J)
    r0 = oc.rho(g, xi0, Q)
    xi1w = xi1.copy()
    xi1w[:, 1] %= g.nx
    if g.ndim == 3:
        xi1w[:, 2] %= g.ny
    r1 = oc.rho(g, xi1w, Q)
    # (rho1 - rho0)/dt + d-.J (Yee d-) = 0
    gy = oc.Grid(g.ndim, g.nz, g.nx, g.ny, g.dz, g.dx, g.dy, g.dt, C=(1.0,), shape=g.shape)
    divJ = oc.gauss(gy, J, np.zeros(g.fshape[1:]))
    return (r1 - r0) / g.dt + divJ, J, r0


@pytest.mark.parametrize("ndim,shape", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_esirkepov_continuity(ndim, shape):
    g = oc.Grid(ndim, 20, 10, 8, dz=0.5, dx=0.4, dy=0.3, dt=0.2, shape=shape)
    n = 30
    xi0 = rand_xi(g, n)
    xi0[:3, 1] = [0.1, g.nx - 0.2, 0.0]      # across the periodic seam
    d = RNG.uniform(-0.95, 0.95, (n, 3))
    if ndim == 2:
        d[:, 2] = 0
    xi1 = xi0 + d
    u = RNG.normal(size=(n, 3))
    res, J, r0 = _continuity(g, xi0, xi1, u, -0.7)
    assert np.max(np.abs(res)) < 1e-12 * np.max(np.abs(r0)) / g.dt


@pytest.mark.parametrize("ndim,shape", [(2, 1), (2, 2), (3, 2)])
def test_esirkepov_total_current(ndim, shape):
    """sum_nodes J_a V = Q (displacement along a)/dt; in 2D sum J3 V = Q v3."""
    g = oc.Grid(ndim, 20, 10, 8, dz=0.5, dx=0.4, dy=0.3, dt=0.2, shape=shape)
    xi0 = rand_xi(g, 1)
    d = np.array([[0.37, -0.61, 0.44 if ndim == 3 else 0.0]])
    u = np.array([[0.5, -0.2, 1.7]])
    J = g.zeros()
    Q = 1.3
    oc.deposit(g, xi0, xi0 + d, u, Q, J)
    V = g.cell_volume()
    h = [g.dz, g.dx, g.dy]
    for a in range(ndim):
        assert np.sum(J[a]) * V == pytest.approx(Q * d[0, a] * h[a] / g.dt, rel=1e-12)
    if ndim == 2:
        v3 = u[0, 2] / math.sqrt(1 + np.sum(u ** 2))
        assert np.sum(J[2]) * V == pytest.approx(Q * v3, rel=1e-12)


def test_esirkepov_special_cases():
    g = oc.Grid(2, 20, 10, dz=0.5, dx=0.4, dt=0.2, shape=2)
    xi0 = rand_xi(g, 5)
    # at rest: no current
    J = g.zeros()
    oc.deposit(g, xi0, xi0.copy(), np.zeros((5, 3)), 1.0, J)
    assert np.max(np.abs(J)) == 0.0
    # axial motion with v3 = 0: only J1
    J = g.zeros()
    xi1 = xi0.copy()
    xi1[:, 0] += 0.45
    oc.deposit(g, xi0, xi1, np.zeros((5, 3)), 1.0, J)
    assert np.max(np.abs(J[1])) == 0.0 and np.max(np.abs(J[2])) == 0.0 and np.max(np.abs(J[0])) > 0


@pytest.mark.parametrize("shape", [1, 2])
def test_2d_j3_is_3d_current_integrated_over_y(shape):
    """The 2D out-of-plane current equals the 3D Esirkepov J3 summed over y for a move with
    dy = v3 dt: this fixes the 1/3 term of the 2D W3."""
    g2 = oc.Grid(2, 16, 10, dz=0.5, dx=0.4, dt=0.2, shape=shape)
    g3 = oc.Grid(3, 16, 10, 12, dz=0.5, dx=0.4, dy=0.3, dt=0.2, shape=shape)
    xi0 = np.array([[7.3, 4.6, 5.2]])
    d = np.array([[0.41, -0.73, 0.0]])
    u = np.array([[0.8, -1.1, 0.9]])
    v3 = u[0, 2] / math.sqrt(1 + np.sum(u ** 2))
    J2 = g2.zeros()
    oc.deposit(g2, xi0, xi0 + d, u, 1.0, J2)
    d3 = d.copy()
    d3[0, 2] = v3 * g3.dt / g3.dy
    J3 = g3.zeros()
    oc.deposit(g3, xi0, xi0 + d3, u, 1.0, J3)
    lhs = J2[2, 0]
    rhs = J3[2].sum(axis=0) * g3.dy
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(lhs))


@pytest.mark.parametrize("ndim,shape", [(2, 1), (3, 2)])
def test_rho_partition_of_unity(ndim, shape):
    g = oc.Grid(ndim, 20, 10, 8, dz=0.5, dx=0.4, dy=0.3, dt=0.2, shape=shape)
    xi = rand_xi(g, 7)
    r = oc.rho(g, xi, 0.9)
    assert np.sum(r) * g.cell_volume() == pytest.approx(7 * 0.9, rel=1e-13)


SIMS = [
    ("yee-lin-2d", 2, 1, None),
    ("yee-quad-2d", 2, 2, None),
    ("custom-quad-2d", 2, 2, "table1"),
    ("yee-quad-3d", 3, 2, None),
    ("custom-lin-3d", 3, 1, "fit"),
]


@pytest.mark.parametrize("name,ndim,shape,solver", SIMS)
def test_whole_step_keeps_gauss_law(name, ndim, shape, solver):
    """Sec. 2.1: with charge-conserving deposition (and the Sec. 3 correction for the customised
    stencil) d-.E - rho does not change from step to step, away from the open z ends."""
    nz, nx, ny = (96, 12, 1) if ndim == 2 else (80, 8, 6)
    dz, dx, dy = 0.5, 0.5, 0.5
    if solver is None:
        C, h = (1.0,), None
        dt = 0.9 * fit.cfl_dt(dz, [dx] + ([dy] if ndim == 3 else []))
    else:
        kappa = 3.0
        C = TABLE1 if solver == "table1" else fit.fit_coefficients(kappa, M=8)
        dt = dz / 4.0 if solver == "table1" else dz / kappa
        assert dt < fit.cfl_dt(dz, [dx] + ([dy] if ndim == 3 else []), C)
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
    sim = oc.Sim(g, [oc.Species(xi, u, -1.0, 1.0, 0.05)], h=h)
    G0 = sim.gauss()
    scale = np.max(np.abs(sim.rho()))
    for _ in range(12):
        sim.step()
    G = sim.gauss()
    inner = (slice(None),) * (G.ndim - 1) + (slice(45, 70),)
    assert np.max(np.abs(G - G0)[inner]) < 1e-11 * scale
    assert np.max(np.abs(sim.E)) > 1e-3 * scale * dz


def test_moving_window_shift_and_injection():
    g = oc.Grid(2, 10, 4, dz=0.5, dx=0.5, dt=0.3, shape=1)
    sp = oc.Species(np.array([[0.2, 1.5, 0], [5.5, 2.5, 0]]), np.zeros((2, 3)), -1, 1, 1)
    sim = oc.Sim(g, [sp], moving_window=True, inject=dict(species=0, ppc=(2, 2), next_id=100))
    sim.E[:] = np.arange(10)[None, None, None, :] + 1.0
    sim.shift()
    assert np.all(sim.E[..., :9] == (np.arange(1, 10) + 1.0)[None, None, None, :])
    assert np.all(sim.E[..., 9] == 0)
    sp = sim.species[0]
    assert list(sp.ids[:1]) == [1] and len(sp.ids) == 1 + 16
    assert sp.xi[0, 0] == 4.5
    assert np.allclose(sp.xi[1:5, 0], [9.25, 9.25, 9.75, 9.75]) and np.allclose(sp.xi[1:5, 1], [0.25, 0.75] * 2)
    assert oc.window_due(2, 0.3, 0.5, 0) and not oc.window_due(1, 0.3, 0.5, 0)
