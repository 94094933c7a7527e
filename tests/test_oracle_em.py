"""Pin of the finite-difference step against the paper's per-mode fields of a drifting charge
(Sec. 2.1, Eq. EM): for a charge mode rho~ at k = (k1, k2) moving along x1 at beta (w = beta k1),
with D = [w]_t^2 - [k]_E1 [k]_B1 - [k]_E2 [k]_B2,

    E1 = -(i/[k]_B1) ([w]_t^2 - [k]_E1 [k]_B1)/D rho~,   E2 = i [k]_E2/D rho~,
    B3 = i ([k]_E2/[k]_B1) [w]_t/D rho~,                 J1 = ([w]_t/[k]_B1) rho~ (continuity),

E at integer and B at half-integer times.  The step here keeps B at integer times (two half
steps), whose amplitude is then B3 cos(w dt/2).  One step of the oracle must carry these fields to
e^{-i w dt} times themselves, for the Yee solver, the Appendix C stencil (Table 1, where the E1
numerator nearly vanishes at beta = 1: the point of Sec. 3) and the split pair with a Yee E side
and the B side fitted to [k1]_t^2 / [k]_Yee ([k]_E1 != [k]_B1)."""
import numpy as np
import pytest

from oracle import core as oc
from oracle import fit
from oracle import spectral as ks

TABLE1 = np.loadtxt(__file__.replace("test_oracle_em.py", "golden/table1_coefficients.txt"))


def em_mode(g, CE, CB, m1, m2, beta):
    """Real staggered arrays of the Eq. EM mode at step 0 (J at step 1/2) and at step 1."""
    k1, k2 = 2 * np.pi * m1 / (g.nz * g.dz), 2 * np.pi * m2 / (g.nx * g.dx)
    kE1 = float(ks.axis_symbol("custom", 0, np.array([k1]), g, C=CE)[0])
    kB1 = float(ks.axis_symbol("custom", 0, np.array([k1]), g, C=CB)[0])
    kE2 = kB2 = 2 / g.dx * np.sin(k2 * g.dx / 2)
    w = beta * k1
    wt = 2 / g.dt * np.sin(w * g.dt / 2)
    D = wt ** 2 - kE1 * kB1 - kE2 * kB2
    E1 = -1j / kB1 * (wt ** 2 - kE1 * kB1) / D
    E2 = 1j * kE2 / D
    B3 = 1j * kE2 / kB1 * wt / D * np.cos(w * g.dt / 2)
    J1 = wt / kB1 * np.exp(-0.5j * w * g.dt)
    Z, X = np.meshgrid(np.arange(g.nz) * g.dz, np.arange(g.nx) * g.dx)

    def f(amp, sz, sx):
        return np.real(amp * np.exp(1j * (k1 * (Z + sz * g.dz) + k2 * (X + sx * g.dx))))

    def fields(t):
        E, B = g.zeros(), g.zeros()
        E[0, 0], E[1, 0], B[2, 0] = f(E1 * t, 0.5, 0), f(E2 * t, 0, 0.5), f(B3 * t, 0.5, 0.5)
        return E, B

    J = g.zeros()
    J[0, 0] = f(J1, 0.5, 0)
    E0, B0 = fields(1.0)
    En, Bn = fields(np.exp(-1j * w * g.dt))
    return E0, B0, J, En, Bn, abs(E1)


SOLVERS = {"yee": ((1.0,), None), "appendix_c": (TABLE1, None), "pair": ((1.0,), "fit")}


def _sets(name, dz, dt):
    CE, CB = SOLVERS[name]
    if CB == "fit":
        CB = fit.fit_coefficients(dz / dt, M=16, CE=[1.0])
    return np.asarray(CE, dtype=np.float64), (None if CB is None else np.asarray(CB, dtype=np.float64))


@pytest.mark.parametrize("name", list(SOLVERS))
@pytest.mark.parametrize("beta", [1.0, 0.9])
def test_one_step_carries_the_eq_em_fields(name, beta):
    dz = dx = 1.0
    dt = 0.25
    CE, CB = _sets(name, dz, dt)
    g = oc.Grid(2, 64, 16, 1, dz, dx, dx, dt, C=CE, Cb=CB, periodic_z=True)
    E, B, J, En, Bn, e1 = em_mode(g, CE, CE if CB is None else CB, 5, 2, beta)
    oc.field_advance(g, E, B, J)
    scale = np.abs(En).max()
    assert np.abs(E - En).max() < 1e-12 * scale
    assert np.abs(B - Bn).max() < 1e-12 * scale
    if name == "appendix_c" and beta == 1.0:
        assert e1 < 1e-6 * scale            # [w]_t^2 - [k]_E1 [k]_B1 ~ 0: E1 of the drifting charge vanishes
    if name == "yee" and beta == 1.0:
        assert e1 > 1e-2 * scale


def test_open_z_interior_matches():
    """With open z ends (the PIC runs) the same holds more than 3 M + 2 cells from both ends."""
    dz = dx = 1.0
    dt = 0.25
    g = oc.Grid(2, 256, 16, 1, dz, dx, dx, dt, C=TABLE1)
    E, B, J, En, Bn, _ = em_mode(g, TABLE1, TABLE1, 20, 2, 1.0)
    oc.field_advance(g, E, B, J)
    inner = (Ellipsis, slice(50, g.nz - 50))
    scale = np.abs(En).max()
    assert np.abs(E[inner] - En[inner]).max() < 1e-12 * scale
    assert np.abs(B[inner] - Bn[inner]).max() < 1e-12 * scale


@pytest.mark.parametrize("kind", ["spectral", "kt"])
@pytest.mark.parametrize("beta", [1.0, 0.9])
def test_kspace_leapfrog_carries_the_eq_em_fields(kind, beta):
    """The k-space leapfrog (oracle/spectral.py) with [k]_1 = k1 (Sec. 2.3) or [k1]_t (Sec. 3) and
    [k]_2 = k2 or the Yee symbol: the same Eq. EM mode, its current given to the advance divided by
    the scaling [k]_Yee / [k] that the advance applies.  For "kt" at beta = 1 the E1 numerator
    [w]_t^2 - [k]_1^2 vanishes identically."""
    g = oc.Grid(2, 64, 16, 1, 1.0, 1.0, 1.0, 0.25, periodic_z=True)
    k1, k2 = 2 * np.pi * 5 / g.nz, 2 * np.pi * 2 / g.nx
    kap1 = float(ks.axis_symbol(kind, 0, np.array([k1]), g)[0])
    kap2 = float(ks.axis_symbol(kind, 1, np.array([k2]), g)[0])
    w = beta * k1
    wt = 2 / g.dt * np.sin(w * g.dt / 2)
    D = wt ** 2 - kap1 ** 2 - kap2 ** 2
    E1 = -1j / kap1 * (wt ** 2 - kap1 ** 2) / D
    E2 = 1j * kap2 / D
    B3 = 1j * kap2 / kap1 * wt / D * np.cos(w * g.dt / 2)
    ratio1 = (2 * np.sin(k1 / 2)) / kap1
    J1 = wt / kap1 * np.exp(-0.5j * w * g.dt) / ratio1
    Z, X = np.meshgrid(np.arange(g.nz) * 1.0, np.arange(g.nx) * 1.0)

    def f(amp, sz, sx):
        return np.real(amp * np.exp(1j * (k1 * (Z + sz) + k2 * (X + sx))))

    E, B, J = g.zeros(), g.zeros(), g.zeros()
    E[0, 0], E[1, 0], B[2, 0], J[0, 0] = f(E1, .5, 0), f(E2, 0, .5), f(B3, .5, .5), f(J1, .5, 0)
    ks.advance(g, E, B, J, kind)
    ph = np.exp(-1j * w * g.dt)
    scale = max(abs(E2), abs(B3))
    assert np.abs(E[0, 0] - f(E1 * ph, .5, 0)).max() < 1e-12 * scale
    assert np.abs(E[1, 0] - f(E2 * ph, 0, .5)).max() < 1e-12 * scale
    assert np.abs(B[2, 0] - f(B3 * ph, .5, .5)).max() < 1e-12 * scale
    if kind == "kt" and beta == 1.0:
        assert abs(E1) < 1e-12 * scale


@pytest.mark.parametrize("name", ["yee", "appendix_c"])
def test_one_step_carries_the_eq_em_fields_in_3d(name):
    """3D: the mode at k = (k1, k2, k3) adds E3 = i [k]_E3/D rho~ (at (i, j, k+1/2)) and
    B2 = -i ([k]_E3/[k]_B1) [w]_t/D rho~ (at (i+1/2, j, k+1/2)); B1 = 0."""
    dz, dx, dy, dt, beta = 1.0, 1.0, 1.2, 0.25, 0.95
    C = (1.0,) if name == "yee" else TABLE1
    g = oc.Grid(3, 64, 12, 10, dz, dx, dy, dt, C=C, periodic_z=True)
    k1, k2, k3 = 2 * np.pi * 5 / (g.nz * dz), 2 * np.pi * 2 / (g.nx * dx), 2 * np.pi * 3 / (g.ny * dy)
    kE1 = float(ks.axis_symbol("custom", 0, np.array([k1]), g, C=np.asarray(C, dtype=np.float64))[0])
    kE2 = 2 / dx * np.sin(k2 * dx / 2)
    kE3 = 2 / dy * np.sin(k3 * dy / 2)
    w = beta * k1
    wt = 2 / dt * np.sin(w * dt / 2)
    D = wt ** 2 - kE1 ** 2 - kE2 ** 2 - kE3 ** 2
    cw = np.cos(w * dt / 2)
    amp = {"E1": -1j / kE1 * (wt ** 2 - kE1 ** 2) / D, "E2": 1j * kE2 / D, "E3": 1j * kE3 / D,
           "B2": -1j * kE3 / kE1 * wt / D * cw, "B3": 1j * kE2 / kE1 * wt / D * cw,
           "J1": wt / kE1 * np.exp(-0.5j * w * dt)}
    stag = {"E1": (.5, 0, 0), "E2": (0, .5, 0), "E3": (0, 0, .5), "B2": (.5, 0, .5), "B3": (.5, .5, 0),
            "J1": (.5, 0, 0)}
    Y, X, Z = np.meshgrid(np.arange(g.ny) * dy, np.arange(g.nx) * dx, np.arange(g.nz) * dz, indexing="ij")

    def f(key, t=1.0):
        sz, sx, sy = stag[key]
        return np.real(amp[key] * t * np.exp(1j * (k1 * (Z + sz * dz) + k2 * (X + sx * dx) + k3 * (Y + sy * dy))))

    E, B, J = g.zeros(), g.zeros(), g.zeros()
    E[0], E[1], E[2], B[1], B[2], J[0] = f("E1"), f("E2"), f("E3"), f("B2"), f("B3"), f("J1")
    oc.field_advance(g, E, B, J)
    ph = np.exp(-1j * w * dt)
    want_E = np.stack([f("E1", ph), f("E2", ph), f("E3", ph)])
    want_B = np.stack([np.zeros_like(Z), f("B2", ph), f("B3", ph)])
    scale = max(np.abs(want_E).max(), np.abs(want_B).max())
    assert np.abs(E - want_E).max() < 1e-12 * scale
    assert np.abs(B - want_B).max() < 1e-12 * scale
