"""GPU parity of the k-space field advance (PIC_SOLVER_SPECTRAL: Sec. 2.3, [k]_a = k_a;
PIC_SOLVER_KT: Sec. 3, [k]_1 = [k1]_t along z in k space; PIC_SOLVER_PSATD: Appendix B) against
the FP64 oracle (oracle/spectral.py), through the C ABI.

Tolerance as for the finite-difference solvers: 1e-5 of the largest |field| (positions 1e-5 cell,
momenta 1e-5 of max |u|).  Grids with even and odd sizes (the r2c axis z and the full axes x, y),
random fields with a random current, whole steps with two species, and Gauss's law with the
solver's own divergence."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import core as oc  # noqa: E402
from oracle import spectral as ks  # noqa: E402
from paper_1910_13529_gb300 import workloads as wl  # noqa: E402

from parity_util import field_error, field_rel_l2, gpu_particles, gpu_sim, oracle_sim, particle_errors  # noqa: E402

TOL = 1e-5


@pytest.fixture(autouse=True)
def _needs_cufft():
    """A library built without cuFFT refuses the k-space solvers; say so instead of failing."""
    import paper_1910_13529_gb300 as P
    try:
        sim = gpu_sim(dict(ndim=2, nz=16, nx=8, ny=1, dz=0.5, dx=0.4, dy=0.45, dt=0.05, solver="spectral"), [])
        sim.close()
    except P.PicError as e:
        if "cuFFT" in str(e) or "cuFFT" in P.pic_last_error():
            pytest.skip("libpic built without cuFFT")
        raise


def kgrid(nd, nz, nx, ny, solver, shape=2, frac=0.9, d=(0.5, 0.4, 0.45)):
    dt = frac * ks.cfl_dt(nd, solver, *d)
    return dict(ndim=nd, nz=nz, nx=nx, ny=ny, dz=d[0], dx=d[1], dy=d[2], dt=dt, solver=solver, shape=shape)


CASES = [
    ("2d-spectral-even", 2, 96, 20, 1, "spectral"),
    ("2d-kt-odd", 2, 95, 21, 1, "kt"),
    ("3d-spectral-odd", 3, 49, 12, 9, "spectral"),
    ("3d-kt-even", 3, 48, 10, 8, "kt"),
    ("2d-psatd-odd", 2, 95, 21, 1, "psatd"),
    ("3d-psatd-even", 3, 48, 10, 8, "psatd"),
]


def _without_nyquist(g, G):
    """G with the Nyquist planes of even axes removed (PSATD removes those modes of E and B)."""
    Gk = np.fft.rfftn(G, axes=(0, 1, 2))
    if g.nz % 2 == 0:
        Gk[:, :, g.nz // 2] = 0
    if g.nx % 2 == 0:
        Gk[:, g.nx // 2, :] = 0
    if g.ndim == 3 and g.ny % 2 == 0:
        Gk[g.ny // 2, :, :] = 0
    return np.fft.irfftn(Gk, s=G.shape, axes=(0, 1, 2))


@pytest.mark.parametrize("name,nd,nz,nx,ny,solver", CASES)
def test_kspace_field_advance(name, nd, nz, nx, ny, solver):
    grid = kgrid(nd, nz, nx, ny, solver)
    sim = gpu_sim(grid, [])
    osim = oracle_sim(grid, [])
    rng = np.random.default_rng(5)
    for a, oa in ((sim.E, osim.E), (sim.B, osim.B), (sim.J, osim.J)):
        v = rng.normal(size=oa.shape).astype(np.float32)
        a.copy_(torch.from_numpy(v))
        oa[:] = v
    J0 = sim.J.clone()
    for n in range(12):
        sim.field_advance()
        ks.advance(osim.g, osim.E, osim.B, osim.J, solver)
        if n == 0:
            assert field_error(sim, osim) < TOL
            assert torch.equal(sim.J, J0)                 # the forward transforms keep their input
    assert field_error(sim, osim) < TOL
    assert field_rel_l2(sim, osim) < TOL
    sim.close()


@pytest.mark.parametrize("name,nd,nz,nx,ny,solver", CASES)
def test_kspace_steps_with_particles(name, nd, nz, nx, ny, solver):
    """Two species away from the z ends (the fields are periodic along z, the particles are not),
    15 whole steps (fused gather + push + deposit, then the k-space advance)."""
    grid = kgrid(nd, nz, nx, ny, solver, shape=2 if nd == 2 else 1)
    m = int(0.35 * nz)
    sps = [wl.random_particles(nd, nz, nx, ny, 1500, seed=11, u_scale=1.0, u_drift=(1.0, 0, 0), margin=m),
           wl.random_particles(nd, nz, nx, ny, 400, seed=12, u_scale=0.2, margin=m, q=1.0, m=5.0, w=0.02)]
    sim = gpu_sim(grid, sps)
    osim = oracle_sim(grid, sps)
    nsteps = 15
    sim.step(nsteps)
    for _ in range(nsteps):
        osim.step()
    assert field_error(sim, osim) < TOL
    for s in range(2):
        dx, du = particle_errors(sim, osim, s, nd)
        assert dx < TOL and du < TOL, (s, dx, du)
    # Gauss's law with the solver's own d-, from the GPU's fields and particles: the change of
    # d-.E - rho over the run stays at FP32 round-off (E started at zero)
    g = osim.g
    rho, rho0 = np.zeros(g.fshape[1:]), np.zeros(g.fshape[1:])
    for s, sp in enumerate(sps):
        _, xi, _ = gpu_particles(sim, s, nd)
        oc.rho(g, xi, sp["q"] * sp["w"], rho)
        oc.rho(g, wl.xi_of(sp, nd), sp["q"] * sp["w"], rho0)
    div_kind = "spectral" if solver == "psatd" else solver
    G = ks.div_minus(g, sim.E.double().cpu().numpy(), div_kind) - rho + rho0
    if solver == "psatd":
        G = _without_nyquist(g, G)
    assert np.abs(G).max() < 1e-4 * np.abs(rho0).max()
    sim.close()


def test_kt_vacuum_wave_moves_at_c():
    """A z-directed vacuum wave on the GPU: with [k1]_t along z, E2 after n steps equals
    cos(n k dt) E2(0) (phase velocity exactly c), against cos(n w dt) with w < k for the spectral
    solver."""
    grid = kgrid(2, 128, 8, 1, "kt", frac=0.7)
    for solver, exact in (("kt", True), ("spectral", False)):
        grid["solver"] = solver
        sim = gpu_sim(grid, [])
        k = 2 * np.pi * 9 / (grid["nz"] * grid["dz"])
        prof = np.cos(k * np.arange(grid["nz"]) * grid["dz"]).astype(np.float32)
        E = torch.zeros_like(sim.E)
        E[1] = torch.from_numpy(np.broadcast_to(prof, (1, grid["nx"], grid["nz"])).copy())
        sim.E.copy_(E)
        sim.B.zero_()
        sim.J.zero_()
        sim.step(50)
        got = sim.E[1].double().cpu().numpy()
        want = np.cos(50 * k * grid["dt"]) * prof
        err = np.abs(got - want).max()
        assert (err < 1e-4) == exact, (solver, err)
        sim.close()


def test_psatd_vacuum_waves_move_at_c_beyond_the_leapfrog_limit():
    """PSATD on the GPU: a transverse mode along x and one along z follow E_n = E_0 cos(n k dt)
    (w = |k| in every direction) at dt = 0.9 min(h), above the spectral leapfrog's limit."""
    grid = kgrid(2, 127, 33, 1, "psatd", frac=0.9)
    assert grid["dt"] > ks.cfl_dt(2, "spectral", grid["dz"], grid["dx"])
    for axis, comp, m in ((0, 1, 9), (1, 0, 4)):
        sim = gpu_sim(grid, [])
        n, h = ((grid["nz"], grid["dz"]), (grid["nx"], grid["dx"]))[axis]
        k = 2 * np.pi * m / (n * h)
        prof = np.cos(k * np.arange(n) * h)
        E = torch.zeros_like(sim.E)
        shape = (1, 1, n) if axis == 0 else (1, n, 1)
        E[comp] = torch.from_numpy(np.broadcast_to(prof.reshape(shape), E.shape[1:]).astype(np.float32).copy())
        sim.E.copy_(E)
        sim.step(40)
        got = sim.E[comp].double().cpu().numpy()
        want = np.cos(40 * k * grid["dt"]) * np.broadcast_to(prof.reshape(shape), got.shape)
        assert np.abs(got - want).max() < 1e-4, axis
        sim.close()


@pytest.mark.parametrize("beta", [1.0, 0.9])
def test_psatd_drifting_charge_fields_of_appendix_b(beta):
    """The GPU's PSATD step carries the Eq. B4 fields of a drifting charge mode (Appendix B) to
    e^{-i w dt} times themselves, as the oracle does (test_oracle_spectral.psatd_b4_mode)."""
    from test_oracle_spectral import psatd_b4_mode
    g = oc.Grid(2, 32, 16, 1, 1.0, 1.0, 1.0, 0.25, periodic_z=True)
    E, B, J, E1, B1 = psatd_b4_mode(g, 3, 2, beta)
    sim = gpu_sim(dict(ndim=2, nz=32, nx=16, ny=1, dz=1.0, dx=1.0, dy=1.0, dt=0.25, solver="psatd", shape=1), [])
    for t, a in ((sim.E, E), (sim.B, B), (sim.J, J)):
        t.copy_(torch.from_numpy(a.astype(np.float32)))
    sim.field_advance()
    scale = np.abs(E1).max()
    assert np.abs(sim.E.double().cpu().numpy() - E1).max() < TOL * scale
    assert np.abs(sim.B.double().cpu().numpy() - B1).max() < TOL * scale
    sim.close()
