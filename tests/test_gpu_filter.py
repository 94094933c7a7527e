"""GPU parity of the 5-pass current filter along z (the "5 pass filter" of Sec. 2.2, 2.3 and
Table 2; its definition is pinned in tests/test_oracle_filter.py) against the FP64 oracle.

Covered: the filter alone on seeded currents (rows of 4 and 7 cells, ragged rows that are not a
multiple of four, rows longer than one CTA segment, the full 2048 x 512 and 512 x 256 x 256 grids on
sampled rows), the deposit with the filter, whole steps, the moving window, Gauss's law for the
filtered charge (pic_gauss, pic_gauss_static, pic_diag) and batched instances.  Tolerance as in
test_gpu_parity.py: 1e-5 of the largest |oracle value|."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1910_13529_gb300 as P  # noqa: E402
from oracle import core as oc  # noqa: E402
from oracle import fit  # noqa: E402
from paper_1910_13529_gb300 import workloads as wl  # noqa: E402
from paper_1910_13529_gb300.runtime import Batch  # noqa: E402

from parity_util import TABLE1, field_error, field_rel_l2, gpu_sim, oracle_sim, particle_errors  # noqa: E402

TOL = 1e-5
FIT8 = fit.fit_coefficients(3.0, M=8)


def grid_of(ndim, nz, nx, ny, solver, shape, C=None, filt=True, d=(0.5, 0.4, 0.45)):
    dperp = [d[1]] + ([d[2]] if ndim == 3 else [])
    dt = 0.9 * fit.cfl_dt(d[0], dperp, None if solver == "yee" else C)
    return dict(ndim=ndim, nz=nz, nx=nx, ny=ny, dz=d[0], dx=d[1], dy=d[2], dt=dt, solver=solver, shape=shape,
                current_filter=filt)


ROWS = [(2, 4, 4, 1), (2, 7, 5, 1), (2, 200, 24, 1), (2, 301, 9, 1), (2, 1024, 6, 1), (2, 2100, 5, 1),
        (2, 5003, 4, 1), (3, 37, 6, 5), (3, 120, 12, 10)]


@pytest.mark.parametrize("nd,nz,nx,ny", ROWS)
def test_filter_alone(nd, nz, nx, ny):
    sim = gpu_sim(grid_of(nd, nz, nx, ny, "yee", 1), [])
    rng = np.random.default_rng(1000 + nz)
    J = rng.normal(size=(3, ny, nx, nz)).astype(np.float32)
    sim.J.copy_(torch.from_numpy(J))
    sim.filter_current()
    ref = J.astype(np.float64)
    oc.filter_z(oc.Grid(nd, nz, nx, ny), ref)
    got = sim.J.double().cpu().numpy()
    assert np.abs(got - ref).max() < TOL * np.abs(ref).max()
    sim.close()


@pytest.mark.parametrize("nd,nz,nx,ny", [(2, 2048, 512, 1), (3, 512, 256, 256)])
def test_filter_full_size_sampled_rows(nd, nz, nx, ny):
    """The bench grids: every row filtered on the GPU, up to 2000 sampled rows recomputed by the oracle."""
    sim = gpu_sim(grid_of(nd, nz, nx, ny, "yee", 1), [])
    gen = torch.Generator().manual_seed(77)
    J = torch.randn((3, ny, nx, nz), generator=gen, dtype=torch.float32)
    sim.J.copy_(J)
    sim.filter_current()
    rows = J.reshape(-1, nz)
    ns = min(2000, rows.shape[0])
    idx = np.random.default_rng(5).choice(rows.shape[0], size=ns, replace=False)
    sample = rows[torch.from_numpy(idx)].double().numpy().reshape(1, 1, ns, nz).copy()
    oc.filter_z(oc.Grid(2, nz, ns), sample)
    got = sim.J.reshape(-1, nz)[torch.from_numpy(idx).to(sim.device)].double().cpu().numpy()
    ref = sample.reshape(ns, nz)
    assert np.abs(got - ref).max() < TOL * np.abs(ref).max()
    sim.close()


DEPOSIT_CASES = [
    ("2d-yee-lin", 2, "yee", 1, None),
    ("2d-custom-quad", 2, "custom", 2, TABLE1),
    ("3d-yee-quad", 3, "yee", 2, None),
    ("3d-custom-lin", 3, "custom", 1, FIT8),
]


@pytest.mark.parametrize("name,nd,solver,shape,C", DEPOSIT_CASES)
def test_deposit_with_filter(name, nd, solver, shape, C):
    nz, nx, ny = (203, 24, 1) if nd == 2 else (120, 12, 10)
    grid = grid_of(nd, nz, nx, ny, solver, shape, C=C)
    sp = wl.random_particles(nd, nz, nx, ny, 3000, seed=17, u_scale=1.5, u_drift=(2.0, 0.3, -0.2), margin=6)
    sim = gpu_sim(grid, [sp], coef=C)
    osim = oracle_sim(grid, [sp], coef=C)
    sim.gather_push()
    sim.deposit()
    g = osim.g
    s = osim.species[0]
    eb = oc.gather(g, osim.E, osim.B, s.xi)
    oc.boris(eb, s.u, s.q * g.dt / (2 * s.m))
    xi1 = oc.move(g, s.xi, s.u)
    J = g.zeros()
    oc.deposit(g, s.xi, xi1, s.u, s.Q, J)
    oc.filter_z(g, J)
    if osim.h is not None:
        oc.correct_j1(g, osim.h, J)
    Jg = sim.J.double().cpu().numpy()
    assert np.abs(Jg - J).max() < TOL * np.abs(J).max()
    sim.close()


@pytest.mark.parametrize("nz", [1000, 2048, 3001, 4100, 10180])
def test_fused_filter_and_correction_on_long_rows(nz):
    """The fused kernel at every CTA size it takes (128 threads up to nz = 1024, 256 beyond) and over
    several segments per row (nz > 2048), with and without 16-byte rows (nz % 4); at nz = 10180 the
    static and dynamic shared memory together just pass the 48 KB default limit."""
    grid = grid_of(2, nz, 4, 1, "custom", 2, C=TABLE1)
    sp = wl.random_particles(2, nz, 4, 1, 4000, seed=nz, u_scale=1.5, u_drift=(2.0, 0.3, -0.2), margin=6)
    sim = gpu_sim(grid, [sp], coef=TABLE1)
    osim = oracle_sim(grid, [sp], coef=TABLE1)
    P.pic_timing(sim.h, 1)
    sim.gather_push()
    sim.deposit()
    _, launches = P.pic_timing_read(sim.h, sim.stream)
    P.pic_timing(sim.h, 0)
    assert launches["filter"] == 1 and launches["correction"] == 0
    g = osim.g
    s = osim.species[0]
    eb = oc.gather(g, osim.E, osim.B, s.xi)
    oc.boris(eb, s.u, s.q * g.dt / (2 * s.m))
    xi1 = oc.move(g, s.xi, s.u)
    J = g.zeros()
    oc.deposit(g, s.xi, xi1, s.u, s.Q, J)
    oc.filter_z(g, J)
    oc.correct_j1(g, osim.h, J)
    Jg = sim.J.double().cpu().numpy()
    assert np.abs(Jg - J).max() < TOL * np.abs(J).max()
    sim.close()


@pytest.mark.parametrize("name,nd,solver,shape,C", DEPOSIT_CASES)
def test_steps_with_filter(name, nd, solver, shape, C):
    nz, nx, ny = (261, 20, 1) if nd == 2 else (100, 10, 9)
    grid = grid_of(nd, nz, nx, ny, solver, shape, C=C)
    sps = [wl.random_particles(nd, nz, nx, ny, 2000, seed=31, u_scale=1.0, u_drift=(3.0, 0, 0), margin=30),
           wl.random_particles(nd, nz, nx, ny, 500, seed=32, u_scale=0.2, margin=30, q=1.0, m=5.0, w=0.02)]
    sim = gpu_sim(grid, sps, coef=C)
    osim = oracle_sim(grid, sps, coef=C)
    P.pic_timing(sim.h, 1)
    nsteps = 15
    sim.step(nsteps)
    _, launches = P.pic_timing_read(sim.h, sim.stream)
    P.pic_timing(sim.h, 0)
    assert launches["filter"] == nsteps
    for _ in range(nsteps):
        osim.step()
    assert field_error(sim, osim) < TOL
    assert field_rel_l2(sim, osim) < TOL
    for s in range(2):
        dx, du = particle_errors(sim, osim, s, nd)
        assert dx < TOL and du < TOL, (s, dx, du)
    sim.close()


def test_filter_changes_the_run():
    """The same run without the filter differs from the filtered one by far more than the tolerance."""
    grid = grid_of(2, 200, 16, 1, "yee", 2)
    sp = wl.random_particles(2, 200, 16, 1, 2000, seed=8, u_scale=1.0, u_drift=(2.0, 0, 0), margin=30)
    a = gpu_sim(grid, [sp])
    b = gpu_sim(dict(grid, current_filter=False), [sp])
    a.step(10)
    b.step(10)
    scale = b.E.abs().max().item()
    assert (a.E - b.E).abs().max().item() > 100 * TOL * scale
    a.close()
    b.close()


def test_moving_window_beam_plasma_with_filter():
    grid, sps = wl.beam_plasma(ndim=2, nz=160, nx=24, n_beam=3000, sigma_z=0.25, sigma_r=0.08,
                               behind_front=1.5, gamma=2e4, solver="custom")
    grid["shape"] = 2
    grid["current_filter"] = True
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


@pytest.mark.parametrize("nd,solver,shape,C", [(2, "yee", 2, None), (2, "custom", 2, TABLE1),
                                               (3, "custom", 2, FIT8)])
def test_gauss_law_for_the_filtered_charge(nd, solver, shape, C):
    nz, nx, ny = (256, 32, 1) if nd == 2 else (128, 12, 12)
    grid = grid_of(nd, nz, nx, ny, solver, shape, C=C)
    grid["rho_bg"] = 0.0
    sps = [wl.random_particles(nd, nz, nx, ny, 20000, seed=13, u_scale=1.0, u_drift=(2.0, 0, 0), margin=50)]
    sim = gpu_sim(grid, sps, coef=C)
    osim = oracle_sim(grid, sps, coef=C)
    # the residual itself (fields zero: -F rho) against the oracle, every node
    G0 = sim.gauss()
    Go = osim.gauss()
    assert np.abs(G0.cpu().numpy() - Go).max() < 1e-9 * np.abs(Go).max()
    rmax = sim.rho().abs().max().item()
    sim.step(40)
    G = sim.gauss()
    m = (48 if solver == "custom" else 3) + 5
    inner = (G - G0)[..., m:-m]
    assert inner.abs().max().item() < 1e-5 * rmax
    # the fixed-scratch variant and pic_diag use the same filtered charge
    Gs = torch.full_like(G, float("nan"))
    P.pic_gauss_static(sim.h, Gs.data_ptr(), sim.stream)
    torch.cuda.synchronize()
    # (FP64 atomics in the charge deposit: equal up to the order of the additions)
    assert (Gs - G).abs().max().item() <= 1e-12 * G.abs().max().item()
    d = sim.diag()
    margin = (len(C) + 24 + 2 if solver == "custom" else 2) + 5
    assert d["gauss_max"] == pytest.approx(G[..., margin:-margin].abs().max().item(), rel=1e-9, abs=1e-300)
    sim.close()


def test_batch_with_filter_matches_oracle():
    rng = np.random.default_rng(4100)
    inst = []
    for i, (nz, nx) in enumerate(((150, 20), (203, 17), (96, 33), (260, 12))):
        solver = "custom" if i % 2 else "yee"
        d = 0.05
        if solver == "custom":
            kappa = 1.0 / (0.5 * rng.uniform(0.3, 0.9))
            C = fit.fit_coefficients(kappa, M=8)
            dt = d / kappa
        else:
            C = None
            dt = rng.uniform(0.3, 0.99) * fit.cfl_dt(d, [d])
        grid = dict(ndim=2, nz=nz, nx=nx, ny=1, dz=d, dx=d, dy=d, dt=dt, solver=solver, shape=1 + i % 2,
                    current_filter=i in (0, 1, 3))
        sp = wl.random_particles(2, nz, nx, 1, 300, seed=4100 + i, u_scale=1.0, u_drift=(2.0, 0, 0), margin=nz // 4)
        inst.append((grid, [sp], C))
    cfgs = []
    for grid, sps, C in inst:
        c = {k: grid[k] for k in ("ndim", "nz", "nx", "dz", "dx", "dt", "shape", "solver", "current_filter")}
        if C is not None:
            c["coef"] = C
        cfgs.append(c)
    batch = Batch(cfgs)
    for sim, (grid, sps, C) in zip(batch.instances, inst):
        sp = sps[0]
        sim.add_species(0, sp["iz"], sp["ix"], sp["iy"], sp["off"], sp["u"], sp["q"], sp["m"], sp["w"],
                        ids=sp["ids"])
    nsteps = 13
    batch.step(nsteps)
    torch.cuda.synchronize()
    for sim, (grid, sps, C) in zip(batch.instances, inst):
        osim = oracle_sim(grid, sps, coef=C)
        for _ in range(nsteps):
            osim.step()
        assert field_error(sim, osim) < TOL, grid
        dx, du = particle_errors(sim, osim, 0, 2)
        assert dx < TOL and du < TOL
    batch.close()
