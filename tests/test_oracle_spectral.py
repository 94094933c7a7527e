"""Pins of the k-space field advance (oracle/spectral.py): the spectral solver of Sec. 2.3 and the
Sec. 3 operator [k]_1 = [k1]_t applied exactly in k space.

* With the Yee symbol on every axis, and with the Appendix C symbol along z, the k-space step is
  the finite-difference step of Eq. 1 (the C oracle, periodic along z) to round-off: this fixes
  the staggering phases, the curl signs and the order of the half steps.
* A single Fourier mode follows the leapfrog's closed form E_n = E_0 cos(n w dt) with
  cos(w dt) = 1 - (dt kappa)^2 / 2 (kappa = k for the spectral solver); with [k1]_t along z the
  phase velocity along z is exactly c (w = k1), the property Sec. 3 builds the operator for.
* With particles (Esirkepov current) Gauss's law d-.E = rho is kept to round-off, and it drifts
  when the k-space correction of the current is left out.
* The stability limit of each solver: the mode at the limit neither grows nor decays."""
import numpy as np
import pytest

from oracle import core as oc
from oracle import spectral as ks

TABLE1 = np.loadtxt(__file__.replace("test_oracle_spectral.py", "golden/table1_coefficients.txt"))


def _grid(nd, C=(1.0,), periodic=True, shape=2):
    if nd == 2:
        return oc.Grid(2, 48, 12, 1, 0.5, 0.4, 0.45, 0.15, C=C, shape=shape, periodic_z=periodic)
    return oc.Grid(3, 40, 10, 6, 0.5, 0.4, 0.45, 0.12, C=C, shape=shape, periodic_z=periodic)


@pytest.mark.parametrize("nd", [2, 3])
def test_yee_symbols_equal_finite_differences(nd):
    g = _grid(nd)
    rng = np.random.default_rng(3)
    E, B, J = (rng.normal(size=g.fshape) for _ in range(3))
    E1, B1 = E.copy(), B.copy()
    oc.field_advance(g, E1, B1, J)
    E2, B2 = E.copy(), B.copy()
    ks.advance(g, E2, B2, J, "yee")
    scale = max(np.abs(E1).max(), np.abs(B1).max())
    assert np.abs(E2 - E1).max() < 1e-12 * scale
    assert np.abs(B2 - B1).max() < 1e-12 * scale


@pytest.mark.parametrize("nd", [2, 3])
def test_appendix_c_symbol_equals_finite_differences(nd):
    """M = 16 Appendix C stencil along z (Table 1), J = 0 (the k-space step also scales the current,
    which the FD oracle does by a separate truncated correction)."""
    g = _grid(nd, C=TABLE1)
    rng = np.random.default_rng(4)
    E, B = rng.normal(size=g.fshape), rng.normal(size=g.fshape)
    J = g.zeros()
    E1, B1 = E.copy(), B.copy()
    oc.field_advance(g, E1, B1, J)
    E2, B2 = E.copy(), B.copy()
    ks.advance(g, E2, B2, J, "custom", C=TABLE1)
    scale = max(np.abs(E1).max(), np.abs(B1).max())
    assert np.abs(E2 - E1).max() < 1e-12 * scale
    assert np.abs(B2 - B1).max() < 1e-12 * scale


def _mode_run(g, kind, axis, m, nsteps):
    """E polarised across `axis` (E2 for a z mode, E1 for an x or y mode), varying as cos along
    `axis` at the component's own staggered positions, B = 0; returns E_n / E_0 on that component
    and the symbol kappa of the mode."""
    E, B, J = g.zeros(), g.zeros(), g.zeros()
    n = (g.nz, g.nx, g.ny)[axis]
    h = (g.dz, g.dx, g.dy)[axis]
    k = 2 * np.pi * m / (n * h)
    comp = 1 if axis == 0 else 0
    # positions of that component along the axis: E2 sits on z nodes; E1 sits on x and y nodes
    pos = np.arange(n) * h
    prof = np.cos(k * pos)
    shape = [1, 1, 1]
    shape[2 - axis] = n
    E[comp] = np.broadcast_to(prof.reshape(shape), g.fshape[1:])
    E0 = E[comp].copy()
    for _ in range(nsteps):
        ks.advance(g, E, B, J, kind)
    kap = float(ks.axis_symbol(kind, axis, np.array([k]), g)[0])
    return E[comp], E0, kap


@pytest.mark.parametrize("kind,axis", [("spectral", 0), ("spectral", 1), ("kt", 1), ("yee", 0)])
def test_single_mode_follows_leapfrog_closed_form(kind, axis):
    g = _grid(2)
    En, E0, kap = _mode_run(g, kind, axis, 5, 37)
    w_dt = np.arccos(1.0 - 0.5 * (g.dt * kap) ** 2)
    assert np.abs(En - np.cos(37 * w_dt) * E0).max() < 1e-11


def test_spectral_mode_along_y_in_3d():
    g = _grid(3)
    En, E0, kap = _mode_run(g, "spectral", 2, 2, 25)
    w_dt = np.arccos(1.0 - 0.5 * (g.dt * kap) ** 2)
    assert abs(kap - 2 * np.pi * 2 / (g.ny * g.dy)) < 1e-12
    assert np.abs(En - np.cos(25 * w_dt) * E0).max() < 1e-11


@pytest.mark.parametrize("m", [1, 7, 20])
def test_kt_operator_gives_phase_velocity_c_along_z(m):
    """[k]_1 = [k1]_t: cos(w dt) = 1 - 2 sin^2(k1 dt/2) = cos(k1 dt), so w = k1 for every mode
    (the numerical Cerenkov condition of Sec. 3 removed along z)."""
    g = _grid(2)
    En, E0, kap = _mode_run(g, "kt", 0, m, 40)
    k1 = 2 * np.pi * m / (g.nz * g.dz)
    assert np.abs(En - np.cos(40 * k1 * g.dt) * E0).max() < 1e-11
    # the spectral and Yee operators do not have it
    for other in ("spectral", "yee"):
        Eo, _, _ = _mode_run(g, other, 0, m, 40)
        assert np.abs(Eo - np.cos(40 * k1 * g.dt) * E0).max() > 1e-4


def _particles(g, n, seed):
    rng = np.random.default_rng(seed)
    xi = np.zeros((n, 3))
    xi[:, 0] = rng.uniform(0.35 * g.nz, 0.65 * g.nz, n)
    xi[:, 1] = rng.uniform(0, g.nx, n)
    if g.ndim == 3:
        xi[:, 2] = rng.uniform(0, g.ny, n)
    u = rng.normal(size=(n, 3)) * 1.5
    return oc.Species(xi, u, -1.0, 1.0, 0.3)


def _gauss_k(sim, kind):
    r = sim.rho()
    return ks.div_minus(sim.g, sim.E, kind) - r


@pytest.mark.parametrize("nd,kind,shape", [(2, "spectral", 2), (2, "kt", 1), (3, "spectral", 1), (3, "kt", 2)])
def test_gauss_law_kept_with_particles(nd, kind, shape):
    g = _grid(nd, periodic=False, shape=shape)
    sim = oc.Sim(g, [_particles(g, 40, 11 + nd)], kspace=kind)
    G0 = _gauss_k(sim, kind)
    rmax = np.abs(sim.rho()).max()
    for _ in range(12):
        sim.step()
    assert len(sim.species[0].xi) == 40                      # nobody reached the z ends
    G = _gauss_k(sim, kind)
    assert np.abs(G - G0).max() < 1e-11 * rmax
    assert np.abs(ks.div_plus(g, sim.B, kind)).max() < 1e-11 * max(np.abs(sim.B).max(), 1e-300)
    assert np.abs(sim.E).max() > 1e-3 * rmax                 # the particles did radiate


def test_gauss_law_drifts_without_the_current_scaling():
    """The same run with the current passed in pre-divided by the ratio kappa_Yee / kappa (so that
    the advance effectively uses the raw Esirkepov current): Gauss's law is no longer kept."""
    g = _grid(2, periodic=False)
    sp = _particles(g, 40, 13)
    sim = oc.Sim(g, [sp], kspace="spectral")
    G0 = _gauss_k(sim, "spectral")
    rmax = np.abs(sim.rho()).max()
    _, _, ratio = ks.operators(g, "spectral")
    for _ in range(12):
        g_ = sim.g
        sim.J[:] = 0.0
        for s in sim.species:
            eb = oc.gather(g_, sim.E, sim.B, s.xi)
            oc.boris(eb, s.u, s.q * g_.dt / (2.0 * s.m))
            xi1 = oc.move(g_, s.xi, s.u)
            oc.deposit(g_, s.xi, xi1, s.u, s.Q, sim.J)
            s.xi = xi1
        Jk = np.fft.rfftn(sim.J, axes=(1, 2, 3))
        Jk = np.stack([Jk[c] / ratio[c] for c in range(3)])
        J_raw_in = np.fft.irfftn(Jk, s=(g.ny, g.nx, g.nz), axes=(1, 2, 3))
        ks.advance(g_, sim.E, sim.B, J_raw_in, "spectral")
        for s in sim.species:
            s.xi[:, 1] %= g_.nx
    G = _gauss_k(sim, "spectral")
    assert np.abs(G - G0).max() > 1e-4 * rmax


@pytest.mark.parametrize("kind,nd", [("spectral", 2), ("spectral", 3), ("kt", 2), ("kt", 3)])
def test_stability_limit(kind, nd):
    """At dt slightly below the limit the fastest mode stays bounded; slightly above it grows."""
    dz, dx, dy = 0.5, 0.4, 0.45
    dtmax = ks.cfl_dt(nd, kind, dz, dx, dy)
    if kind == "spectral":
        perp = [dx] + ([dy] if nd == 3 else [])
        assert abs(dtmax - 2.0 / np.sqrt(sum((np.pi / h) ** 2 for h in [dz] + perp))) < 1e-15
    for f, grows in ((0.999, False), (1.01, True)):
        ny = 8 if nd == 3 else 1
        g = oc.Grid(nd, 16, 8, ny, dz, dx, dy, f * dtmax)
        E, B, J = g.zeros(), g.zeros(), g.zeros()
        # the checkerboard: Nyquist along every axis
        iz, ix, iy = np.meshgrid(np.arange(g.nz), np.arange(g.nx), np.arange(g.ny), indexing="ij")
        chk = ((-1.0) ** (iz + ix + iy)).transpose(2, 1, 0)
        E[0], E[1], E[2] = chk, -chk, 0.5 * chk
        for _ in range(400):
            ks.advance(g, E, B, J, kind)
        amp = np.abs(E).max()
        assert (amp > 1e3) == grows, (f, amp)


# ---------------------------------------------------------------- PSATD (Appendix B) ---

def _odd_grid(nd, dt=0.3, shape=None):
    if nd == 2:
        return oc.Grid(2, 47, 13, 1, 0.5, 0.4, 0.45, dt, shape=2 if shape is None else shape)
    return oc.Grid(3, 39, 11, 7, 0.5, 0.4, 0.45, dt, shape=1 if shape is None else shape)


@pytest.mark.parametrize("axis", [0, 1])
def test_psatd_vacuum_modes_are_exact(axis):
    """E_n = E_0 cos(n k dt) for a transverse mode (w = |k| in every direction), also at a dt
    above the leapfrog limit of the spectral solver."""
    g = oc.Grid(2, 48, 12, 1, 0.5, 0.4, 0.45, 0.9 * 0.4, shape=2, periodic_z=True)
    assert g.dt > ks.cfl_dt(2, "spectral", g.dz, g.dx)
    En, E0, kap = _mode_run(g, "psatd", axis, 5, 37)
    k = 2 * np.pi * 5 / ((g.nz, g.nx)[axis] * (g.dz, g.dx)[axis])
    assert np.abs(En - np.cos(37 * k * g.dt) * E0).max() < 1e-11


@pytest.mark.parametrize("nd", [2, 3])
def test_psatd_keeps_a_static_longitudinal_field(nd):
    """E = -d+ phi (spectral forward difference of a random potential), B = 0, J = 0: unchanged."""
    g = _odd_grid(nd)
    rng = np.random.default_rng(8)
    phi_k = np.fft.rfftn(rng.normal(size=(g.ny, g.nx, g.nz)))
    dp, _, _ = ks.operators(g, "spectral")
    E = np.stack([np.fft.irfftn(-dp[a] * phi_k, s=(g.ny, g.nx, g.nz), axes=(0, 1, 2)) for a in range(3)])
    B, J = g.zeros(), g.zeros()
    E0 = E.copy()
    for _ in range(5):
        ks.advance(g, E, B, J, "psatd")
    assert np.abs(E - E0).max() < 1e-12 * np.abs(E0).max()
    assert np.abs(B).max() < 1e-12 * np.abs(E0).max()


@pytest.mark.parametrize("nd", [2, 3])
def test_psatd_conserves_vacuum_energy_beyond_the_leapfrog_limit(nd):
    g = _odd_grid(nd, dt=2.0 * ks.cfl_dt(nd, "spectral", 0.5, 0.4, 0.45))
    rng = np.random.default_rng(9)
    E, B, J = rng.normal(size=g.fshape), g.zeros(), g.zeros()
    # remove the longitudinal part so that the whole field propagates
    Ek = np.fft.rfftn(E, axes=(1, 2, 3))
    dp, dm, _ = ks.operators(g, "spectral")
    kz, kx, ky = ks._axes_k(g)
    k2 = kz ** 2 + kx ** 2 + ky ** 2
    div = sum(dm[a] * Ek[a] for a in range(3))
    phi = np.where(k2 == 0, 0.0, div / np.where(k2 == 0, 1.0, -k2))
    E = E - np.stack([np.fft.irfftn(dp[a] * phi, s=(g.ny, g.nx, g.nz), axes=(0, 1, 2)) for a in range(3)])
    W0 = np.sum(E ** 2) + np.sum(B ** 2)
    for _ in range(100):
        ks.advance(g, E, B, J, "psatd")
    assert abs(np.sum(E ** 2) + np.sum(B ** 2) - W0) < 1e-10 * W0
    assert np.sum(B ** 2) > 0.1 * W0                            # the field did oscillate


def test_psatd_approaches_the_spectral_leapfrog_as_dt_shrinks():
    """With J = 0 PSATD is exact in time and the leapfrog's local error is O(dt^3): halving dt
    divides the one-step difference by about 8 (smooth fields, low modes)."""
    g = _odd_grid(2, dt=0.08)
    kz, kx, _ = ks._axes_k(g)
    rng = np.random.default_rng(10)
    Ek = np.zeros((3,) + (g.ny, g.nx, g.nz // 2 + 1), dtype=complex)
    low = (np.abs(kz) < 2.5) & (np.abs(kx) < 2.5)
    for c in range(3):
        Ek[c] = np.where(low, rng.normal(size=low.shape) + 1j * rng.normal(size=low.shape), 0.0)
    E0 = np.fft.irfftn(Ek, s=(g.ny, g.nx, g.nz), axes=(1, 2, 3))
    diffs = []
    for dt in (0.08, 0.04):
        g = _odd_grid(2, dt=dt)
        Ea, Ba = E0.copy(), g.zeros()
        Eb, Bb = E0.copy(), g.zeros()
        ks.advance(g, Ea, Ba, g.zeros(), "psatd")
        ks.advance(g, Eb, Bb, g.zeros(), "spectral")
        diffs.append(max(np.abs(Ea - Eb).max(), np.abs(Ba - Bb).max()))
    assert 6.0 < diffs[0] / diffs[1] < 10.0


@pytest.mark.parametrize("nd,shape", [(2, 2), (3, 1)])
def test_psatd_gauss_law_kept_with_particles(nd, shape):
    g = _odd_grid(nd, shape=shape)
    sim = oc.Sim(g, [_particles(g, 40, 21 + nd)], kspace="psatd")
    G0 = _gauss_k(sim, "spectral")
    rmax = np.abs(sim.rho()).max()
    for _ in range(12):
        sim.step()
    assert len(sim.species[0].xi) == 40
    G = _gauss_k(sim, "spectral")
    assert np.abs(G - G0).max() < 1e-11 * rmax
    assert np.abs(sim.E).max() > 1e-3 * rmax


@pytest.mark.parametrize("nd", [2, 3])
def test_correction_taps_match_the_exact_kspace_ratio(nd):
    """Two independent routes to the Sec. 3 correction: the finite-difference step after
    J1 <- h * J1 with the truncated taps of 1/P (fit.correction_kernel, 40 per side) equals the
    k-space step with the Appendix C symbol, whose current is scaled by [k]_Yee / [k]_1 = 1/P
    exactly, up to the taps' truncation.  The oracle's correction treats the z ends as open (zero
    outside), so the comparison is on the cells more than 40 + 3 M from both ends."""
    from oracle import fit
    if nd == 2:
        g = oc.Grid(2, 256, 12, 1, 0.5, 0.4, 0.45, 0.15, C=TABLE1, shape=2, periodic_z=True)
    else:
        g = oc.Grid(3, 224, 10, 6, 0.5, 0.4, 0.45, 0.12, C=TABLE1, shape=1, periodic_z=True)
    rng = np.random.default_rng(12)
    E, B, J = (rng.normal(size=g.fshape) for _ in range(3))
    E1, B1, J1 = E.copy(), B.copy(), J.copy()
    oc.correct_j1(g, fit.correction_kernel(TABLE1, hlen=40), J1)
    oc.field_advance(g, E1, B1, J1)
    E2, B2 = E.copy(), B.copy()
    ks.advance(g, E2, B2, J, "custom", C=TABLE1)
    m = 40 + 3 * 16 + 2
    inner = (Ellipsis, slice(m, g.nz - m))
    scale = max(np.abs(E1).max(), np.abs(B1).max())
    assert np.abs(E2[inner] - E1[inner]).max() < 1e-12 * scale
    assert np.abs(B2[inner] - B1[inner]).max() < 1e-12 * scale
    # without the correction the two differ at the level of the current itself
    E3, B3 = E.copy(), B.copy()
    oc.field_advance(g, E3, B3, J)
    assert np.abs(E3[inner] - E2[inner]).max() > 1e-3 * scale


def psatd_b4_mode(g, m1, m2, beta):
    """Appendix B, Eq. B4: the fields of a charge mode rho~ = 1 at k = (k1, k2) (2D) drifting along
    x1 at beta (w = beta k1), with F = sin(k dt)/(k dt) (1 - cos w dt)/(cos w dt - cos k dt):
        E1 = -i k1/k^2 + i k2^2/(k1 k^2) F,   E2 = -i (1 + F) k2/k^2,
        B3 = -i k2/(k1 k^2) sin(w dt)/dt (1 - cos k dt)/(cos w dt - cos k dt);
    the current that carries it, from the discrete continuity equation
    (rho^{n+1} - rho^n)/dt + i k1 J1^{n+1/2} = 0 with J1^{n+1/2} = J1~ e^{-i w dt n}:
    J1 = i (e^{-i w dt} - 1)/(k1 dt).  Returns the real staggered arrays of the mode at step 0
    (J1 pre-divided by the current scaling [k]_Yee / k the advance applies) and at step 1."""
    k1, k2 = 2 * np.pi * m1 / (g.nz * g.dz), 2 * np.pi * m2 / (g.nx * g.dx)
    k = np.hypot(k1, k2)
    w = beta * k1
    ph = np.exp(-1j * w * g.dt)
    den = np.cos(w * g.dt) - np.cos(k * g.dt)
    F = np.sin(k * g.dt) / (k * g.dt) * (1 - np.cos(w * g.dt)) / den
    E1 = -1j * k1 / k ** 2 + 1j * k2 ** 2 / (k1 * k ** 2) * F
    E2 = -1j * (1 + F) * k2 / k ** 2
    B3 = -1j * k2 / (k1 * k ** 2) * np.sin(w * g.dt) / g.dt * (1 - np.cos(k * g.dt)) / den
    J1 = 1j * (ph - 1) / (k1 * g.dt) / ((2 / g.dz * np.sin(k1 * g.dz / 2)) / k1)
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
    E1_, B1_ = fields(ph)
    return E0, B0, J, E1_, B1_


@pytest.mark.parametrize("beta", [1.0, 0.9])
def test_psatd_reproduces_the_drifting_charge_fields_of_appendix_b(beta):
    """One PSATD step carries the Eq. B4 fields of a drifting charge mode to e^{-i w dt} times
    themselves (kappa = dx1/dt = 4, r = 1, as in the paper's Fig. 6)."""
    g = oc.Grid(2, 32, 16, 1, 1.0, 1.0, 1.0, 0.25, periodic_z=True)
    E, B, J, E1, B1 = psatd_b4_mode(g, 3, 2, beta)
    ks.advance(g, E, B, J, "psatd")
    assert np.abs(E - E1).max() < 1e-12 * np.abs(E1).max()
    assert np.abs(B - B1).max() < 1e-12 * np.abs(E1).max()
