"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on identical seeded inputs.

Tolerance (FP32 kernels vs FP64 oracle): fields within 1e-5 of the largest |field| of the
oracle run; particle positions within 1e-5 cell; momenta within 1e-5 of the largest |u|.
Sizes span several CTA tiles with ragged tails (e.g. nz = 300 over 128-cell tiles, nx = 21
over 8-row tiles)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import core as oc  # noqa: E402
from oracle import fit  # noqa: E402
from paper_1910_13529_gb300 import decode_cells  # noqa: E402
from paper_1910_13529_gb300 import workloads as wl  # noqa: E402

from parity_util import (TABLE1, field_error, field_rel_l2, gpu_particles, gpu_sim,  # noqa: E402
                         oracle_sim, particle_errors)

TOL = 1e-5
FIT8 = fit.fit_coefficients(3.0, M=8)


def grid_of(ndim, nz, nx, ny, solver, shape, dt_frac=0.9, d=(0.5, 0.4, 0.45), C=None):
    dperp = [d[1]] + ([d[2]] if ndim == 3 else [])
    dt = dt_frac * fit.cfl_dt(d[0], dperp, None if solver == "yee" else C)
    return dict(ndim=ndim, nz=nz, nx=nx, ny=ny, dz=d[0], dx=d[1], dy=d[2], dt=dt, solver=solver, shape=shape)


FIELD_CASES = [
    ("2d-yee", 2, 300, 21, 1, "yee", None),
    ("2d-custom16", 2, 300, 21, 1, "custom", TABLE1),
    ("3d-yee", 3, 150, 10, 7, "yee", None),
    ("3d-custom8", 3, 150, 10, 7, "custom", FIT8),
]


@pytest.mark.parametrize("name,nd,nz,nx,ny,solver,C", FIELD_CASES)
def test_field_advance(name, nd, nz, nx, ny, solver, C):
    grid = grid_of(nd, nz, nx, ny, solver, 1, C=C)
    sim = gpu_sim(grid, [], coef=C)
    osim = oracle_sim(grid, [], coef=C)
    rng = np.random.default_rng(21)
    for a, oa in ((sim.E, osim.E), (sim.B, osim.B), (sim.J, osim.J)):
        v = rng.normal(size=oa.shape).astype(np.float32)
        a.copy_(torch.from_numpy(v))
        oa[:] = v
    for n in range(12):
        sim.field_advance()
        oc.field_advance(osim.g, osim.E, osim.B, osim.J)
        if n == 0:
            assert field_error(sim, osim) < TOL
    assert field_error(sim, osim) < TOL
    assert field_rel_l2(sim, osim) < TOL
    sim.close()


def test_field_advance_window_shift():
    grid = grid_of(2, 200, 16, 1, "custom", 1, C=TABLE1)
    grid["dt"] = 0.6 * grid["dz"]
    grid["dt"] = min(grid["dt"], 0.95 * fit.cfl_dt(grid["dz"], [grid["dx"]], TABLE1))
    grid["moving_window"] = True
    sim = gpu_sim(grid, [], coef=TABLE1)
    osim = oracle_sim(grid, [], coef=TABLE1)
    rng = np.random.default_rng(3)
    for a, oa in ((sim.E, osim.E), (sim.B, osim.B)):
        v = rng.normal(size=oa.shape).astype(np.float32)
        a.copy_(torch.from_numpy(v))
        oa[:] = v
    shifts = 0
    for _ in range(5):
        sim.field_advance()
        oc.field_advance(osim.g, osim.E, osim.B, osim.J)
        osim.n += 1
        if oc.window_due(osim.n, osim.g.dt, osim.g.dz, osim.shifts):
            osim.shift()
    step, sh, pend = sim.state()
    assert step == 5 and sh == osim.shifts and sh >= 2
    assert field_error(sim, osim) < TOL
    sim.close()


PUSH_CASES = [
    ("2d-yee-lin", 2, "yee", 1, None),
    ("2d-yee-quad", 2, "yee", 2, None),
    ("2d-custom-quad", 2, "custom", 2, TABLE1),
    ("3d-yee-lin", 3, "yee", 1, None),
    ("3d-custom-quad", 3, "custom", 2, FIT8),
]


@pytest.mark.parametrize("name,nd,solver,shape,C", PUSH_CASES)
def test_gather_push_deposit(name, nd, solver, shape, C):
    nz, nx, ny = (200, 24, 1) if nd == 2 else (120, 12, 10)
    grid = grid_of(nd, nz, nx, ny, solver, shape, C=C)
    sp = wl.random_particles(nd, nz, nx, ny, 3000, seed=7, u_scale=1.5, u_drift=(2.0, 0.3, -0.2), margin=6)
    sim = gpu_sim(grid, [sp], coef=C)
    osim = oracle_sim(grid, [sp], coef=C)
    rng = np.random.default_rng(5)
    for a, oa in ((sim.E, osim.E), (sim.B, osim.B)):
        v = (0.3 * rng.normal(size=oa.shape)).astype(np.float32)
        a.copy_(torch.from_numpy(v))
        oa[:] = v
    sim.gather_push()
    sim.deposit()
    # oracle: the same sub-steps
    g = osim.g
    s = osim.species[0]
    eb = oc.gather(g, osim.E, osim.B, s.xi)
    oc.boris(eb, s.u, s.q * g.dt / (2 * s.m))
    xi1 = oc.move(g, s.xi, s.u)
    J = g.zeros()
    oc.deposit(g, s.xi, xi1, s.u, s.Q, J)
    if osim.h is not None:
        oc.correct_j1(g, osim.h, J)
    s.xi = xi1
    s.xi[:, 1] %= g.nx
    if nd == 3:
        s.xi[:, 2] %= g.ny
    s.keep((s.xi[:, 0] >= 0) & (s.xi[:, 0] < g.nz))
    Jg = sim.J.double().cpu().numpy()
    assert np.abs(Jg - J).max() < TOL * np.abs(J).max()
    dx, du = particle_errors(sim, osim, 0, nd)
    assert dx < TOL and du < TOL
    sim.close()


STEP_CASES = [
    ("2d-yee-lin", 2, "yee", 1, None),
    ("2d-custom-quad", 2, "custom", 2, TABLE1),
    ("3d-yee-quad", 3, "yee", 2, None),
    ("3d-custom-lin", 3, "custom", 1, FIT8),
]


@pytest.mark.parametrize("name,nd,solver,shape,C", STEP_CASES)
def test_steps(name, nd, solver, shape, C):
    nz, nx, ny = (260, 20, 1) if nd == 2 else (100, 10, 9)
    grid = grid_of(nd, nz, nx, ny, solver, shape, C=C)
    sps = [wl.random_particles(nd, nz, nx, ny, 2000, seed=11, u_scale=1.0, u_drift=(3.0, 0, 0), margin=30),
           wl.random_particles(nd, nz, nx, ny, 500, seed=12, u_scale=0.2, margin=30, q=1.0, m=5.0, w=0.02)]
    sim = gpu_sim(grid, sps, coef=C)
    osim = oracle_sim(grid, sps, coef=C)
    nsteps = 15
    sim.step(nsteps)
    for _ in range(nsteps):
        osim.step()
    assert field_error(sim, osim) < TOL
    for s in range(2):
        dx, du = particle_errors(sim, osim, s, nd)
        assert dx < TOL and du < TOL, (s, dx, du)
    sim.close()


def test_unfused_calls_equal_pic_step():
    grid = grid_of(2, 200, 16, 1, "custom", 2, C=TABLE1)
    sp = wl.random_particles(2, 200, 16, 1, 3000, seed=2, u_scale=1.0, u_drift=(2.0, 0, 0), margin=20)
    a = gpu_sim(grid, [sp], coef=TABLE1)
    b = gpu_sim(grid, [sp], coef=TABLE1)
    for _ in range(5):
        a.gather_push()
        a.deposit()
        a.field_advance()
    b.step(5)
    scale = max(b.E.abs().max().item(), b.B.abs().max().item())
    assert (a.E - b.E).abs().max().item() < 1e-5 * scale
    assert (a.B - b.B).abs().max().item() < 1e-5 * scale
    ia, xa, ua = gpu_particles(a, 0, 2)
    ib, xb, ub = gpu_particles(b, 0, 2)
    assert np.array_equal(ia, ib) and np.abs(xa - xb).max() < 1e-5 and np.abs(ua - ub).max() < 1e-4
    a.close()
    b.close()


@pytest.mark.parametrize("solver,shape,C", [("yee", 1, None), ("custom", 2, TABLE1)])
def test_single_particle_200_steps(solver, shape, C):
    """The 256 x 128 single-particle vacuum run (gamma = 1000, dt = 0.45 dz), 200 steps."""
    grid, sps = wl.single_particle(shape=shape, solver=solver)
    if solver == "custom":
        assert grid["dt"] < fit.cfl_dt(grid["dz"], [grid["dx"]], C)
    sim = gpu_sim(grid, sps, coef=C)
    osim = oracle_sim(grid, sps, coef=C)
    sim.step(200)
    for _ in range(200):
        osim.step()
    assert field_rel_l2(sim, osim) < TOL
    assert field_error(sim, osim) < TOL
    dx, du = particle_errors(sim, osim, 0, 2)
    assert dx < TOL and du < TOL
    sim.close()


@pytest.mark.parametrize("nd,solver,shape,C", [(2, "yee", 2, None), (2, "custom", 2, TABLE1),
                                               (3, "custom", 2, FIT8)])
def test_gauss_law_kept_on_gpu(nd, solver, shape, C):
    nz, nx, ny = (256, 32, 1) if nd == 2 else (128, 12, 12)
    grid = grid_of(nd, nz, nx, ny, solver, shape, C=C)
    sps = [wl.random_particles(nd, nz, nx, ny, 20000, seed=13, u_scale=1.0, u_drift=(2.0, 0, 0), margin=50)]
    sim = gpu_sim(grid, sps, coef=C)
    G0 = sim.gauss()
    rmax = sim.rho().abs().max().item()
    sim.step(40)
    G = sim.gauss()
    m = 48 if solver == "custom" else 3
    inner = (G - G0)[..., m:-m]
    assert inner.abs().max().item() < 1e-5 * rmax
    d = sim.diag()
    assert d["count"] == 20000 and d["step"] == 40
    sim.close()


def test_moving_window_beam_plasma():
    """Small beam-in-plasma run with the moving window and plasma injection, 24 steps."""
    grid, sps = wl.beam_plasma(ndim=2, nz=160, nx=24, n_beam=3000, sigma_z=0.25, sigma_r=0.08,
                               behind_front=1.5, gamma=2e4, solver="custom")
    grid["shape"] = 2
    C = fit.fit_coefficients(grid["dz"] / grid["dt"])
    sim = gpu_sim(grid, sps, coef=C, cap_extra=20000)
    osim = oracle_sim(grid, sps, coef=C)
    n = 24
    sim.step(n)
    for _ in range(n):
        osim.step()
    step, shifts, pend = sim.state()
    assert shifts == osim.shifts and shifts >= 10
    assert field_error(sim, osim) < TOL
    assert field_rel_l2(sim, osim) < TOL
    for s in range(2):
        dx, du = particle_errors(sim, osim, s, 2, pending_shift=pend)
        assert dx < TOL and du < TOL, (s, dx, du)
    sim.close()


def test_sort_keeps_particles_and_orders_cells():
    grid = grid_of(2, 64, 16, 1, "yee", 1)
    sp = wl.random_particles(2, 64, 16, 1, 5000, seed=4, u_scale=1.0, margin=2)
    sim = gpu_sim(grid, [sp])
    sim.step(3)                      # some particles leave through the z ends
    before = gpu_particles(sim, 0, 2)
    n_live = len(before[0])
    sim.sort()
    p = sim.particles(0)
    assert len(p["cell"]) == n_live and np.all(p["cell"] >= 0)
    iz, ix, _ = decode_cells(p["cell"], sim.nz, sim.nx)
    ntz = (sim.nz + 2 + 7) // 8
    col = ix // 8
    tz = np.where(col % 2 == 1, ntz - 1 - (iz + 1) // 8, (iz + 1) // 8)  # 8 x 8 tiles, snaking along z
    tile = col * ntz + tz
    assert np.all(np.diff(tile) >= 0)
    inner = ((ix % 8) * 8 + (iz + 1) % 8)
    same = np.diff(tile) == 0
    assert np.all(np.diff(inner)[same] >= 0)
    after = gpu_particles(sim, 0, 2)
    assert np.array_equal(before[0], after[0])
    assert np.array_equal(before[1], after[1]) and np.array_equal(before[2], after[2])
    sim.close()


def test_sort_orders_3d_cells_in_cubic_tiles():
    grid = grid_of(3, 40, 12, 10, "yee", 2)
    sp = wl.random_particles(3, 40, 12, 10, 6000, seed=14, u_scale=1.0, margin=2)
    sim = gpu_sim(grid, [sp])
    sim.step(3)
    before = gpu_particles(sim, 0, 3)
    sim.sort()
    p = sim.particles(0)
    assert len(p["cell"]) == len(before[0]) and np.all(p["cell"] >= 0)
    iz, ix, iy = decode_cells(p["cell"], sim.nz, sim.nx)
    izg = iz + 1
    ntz, ntx = (sim.nz + 2 + 3) // 4, (sim.nx + 3) // 4
    ty = iy // 4
    col = ty * ntx + np.where(ty % 2 == 1, ntx - 1 - ix // 4, ix // 4)   # 4 x 4 x 4 tiles, snaking
    tile = col * ntz + np.where(col % 2 == 1, ntz - 1 - izg // 4, izg // 4)
    assert np.all(np.diff(tile) >= 0)
    inner = ((iy % 4) * 4 + ix % 4) * 4 + izg % 4
    same = np.diff(tile) == 0
    assert np.all(np.diff(inner)[same] >= 0)
    after = gpu_particles(sim, 0, 3)
    assert np.array_equal(before[0], after[0])
    assert np.array_equal(before[1], after[1]) and np.array_equal(before[2], after[2])
    sim.close()


@pytest.mark.parametrize("shape,solver,C", [(1, "yee", None), (2, "custom", TABLE1)])
def test_switch_point_offsets_and_seam(shape, solver, C):
    """Particles at the offsets where the shape supports switch nodes (0, 1/4, 1/2, 3/4 and the
    largest FP32 below 1), in the first and last x columns so that their stencils and moves cross
    the periodic seam, with momenta along and against z and x; 12 steps against the oracle."""
    nz, nx = 96, 12
    grid = grid_of(2, nz, nx, 1, solver, shape, C=C)
    offs = np.array([0.0, 0.25, 0.5, 0.75, np.nextafter(np.float32(1), np.float32(0))], np.float32)
    oz, ox = np.meshgrid(offs, offs, indexing="ij")
    oz, ox = oz.ravel(), ox.ravel()
    k = len(oz)
    iz = np.repeat(np.arange(30, 30 + 4 * 6, 6), k)[: 4 * k]
    ix = np.tile(np.concatenate([np.zeros(k, np.int64), np.full(k, nx - 1, np.int64)]), 2)
    off = np.stack([np.tile(oz, 4), np.tile(ox, 4)])
    rng = np.random.default_rng(17)
    u = rng.normal(size=(3, 4 * k)).astype(np.float32) * 0.8
    u[1, : 2 * k] = np.abs(u[1, : 2 * k]) * np.where(ix[: 2 * k] == 0, -1.0, 1.0)   # towards the seam
    sp = wl.species(iz, ix, np.zeros_like(iz), off, u, -1.0, 1.0, 0.05)
    sim = gpu_sim(grid, [sp], coef=C)
    osim = oracle_sim(grid, [sp], coef=C)
    for _ in range(12):
        sim.step(1)
        osim.step()
    assert field_error(sim, osim) < TOL
    dx, du = particle_errors(sim, osim, 0, 2)
    assert dx < TOL and du < TOL
    sim.close()


def test_sorted_run_matches_oracle():
    grid = grid_of(2, 200, 16, 1, "yee", 2)
    sp = wl.random_particles(2, 200, 16, 1, 4000, seed=9, u_scale=1.0, u_drift=(2.0, 0, 0), margin=20)
    sim = gpu_sim(grid, [sp], sort_every=3)
    osim = oracle_sim(grid, [sp])
    sim.step(10)
    for _ in range(10):
        osim.step()
    assert field_error(sim, osim) < TOL
    dx, du = particle_errors(sim, osim, 0, 2)
    assert dx < TOL and du < TOL
    sim.close()


DENSE_CASES = [("2d-lin", 2, 1), ("2d-quad", 2, 2), ("3d-lin", 3, 1), ("3d-quad", 3, 2)]


@pytest.mark.parametrize("name,nd,shape", DENSE_CASES)
def test_dense_cluster_fused_steps(name, nd, shape):
    """4000 particles in three cells (70% in one), sorted every step: most lanes of a warp share
    their deposition window, so the fused kernels sum each deposit over the lanes of a window
    before the shared-memory add (the dense-beam path).  Fields and particles after 4 steps
    against the oracle."""
    nz, nx, ny = (96, 16, 1) if nd == 2 else (64, 12, 10)
    grid = grid_of(nd, nz, nx, ny, "yee", shape)
    rng = np.random.default_rng(31)
    n = 4000
    which = rng.choice(3, size=n, p=[0.7, 0.2, 0.1])
    cz = 40 + np.array([0, 0, 1])[which]
    cx = 6 + np.array([0, 1, 0])[which]
    cy = np.full(n, 4 if nd == 3 else 0)
    off = rng.uniform(0.2, 0.8, size=(nd, n))
    u = rng.normal(size=(3, n)) * 0.05 + np.array([[0.5], [0.1], [-0.05]])
    sp = wl.species(cz, cx, cy, off, u, -1.0, 1.0, 0.01)
    sim = gpu_sim(grid, [sp], sort_every=1)
    osim = oracle_sim(grid, [sp])
    sim.step(4)
    for _ in range(4):
        osim.step()
    assert field_error(sim, osim) < TOL
    dx, du = particle_errors(sim, osim, 0, nd)
    assert dx < TOL and du < TOL
    sim.close()


def test_empty_species_and_diag_energies():
    grid = grid_of(2, 64, 16, 1, "yee", 1)
    empty = wl.random_particles(2, 64, 16, 1, 0, seed=1)
    sp = wl.random_particles(2, 64, 16, 1, 100, seed=1, u_scale=2.0, margin=10)
    sim = gpu_sim(grid, [empty, sp])
    sim.step(4)
    d = sim.diag()
    E = sim.E.double()
    B = sim.B.double()
    W = 0.5 * float((E ** 2).sum() + (B ** 2).sum()) * grid["dz"] * grid["dx"]
    assert d["field_energy"] == pytest.approx(W, rel=1e-9)
    ids, xi, u = gpu_particles(sim, 1, 2)
    K = sp["w"] * np.sum(np.sqrt(1 + np.sum(u ** 2, axis=1)) - 1)
    assert d["kinetic"] == pytest.approx(K, rel=1e-9)
    assert d["count"] == len(ids)
    sim.close()


def test_moving_window_long_grid_with_dead_slots():
    """Window run on a longer grid: particles leave through the back, so sorted chunks far from the
    origin hold dead slots next to live ones (the shared-memory current box must ignore them)."""
    grid, sps = wl.beam_plasma(ndim=2, nz=1024, nx=64, n_beam=4000, sigma_z=0.4, sigma_r=0.1,
                               behind_front=2.0, gamma=2e4, ppc=(1, 1, 1), solver="custom")
    C = fit.fit_coefficients(grid["dz"] / grid["dt"])
    sim = gpu_sim(grid, sps, coef=C, cap_extra=20000, sort_every=8)
    osim = oracle_sim(grid, sps, coef=C)
    n = 30
    sim.step(n)
    for _ in range(n):
        osim.step()
    step, shifts, pend = sim.state()
    assert shifts == osim.shifts and shifts >= 12
    assert field_error(sim, osim) < TOL
    for s in range(2):
        dx, du = particle_errors(sim, osim, s, 2, pending_shift=pend)
        assert dx < TOL and du < TOL, (s, dx, du)
    sim.close()
