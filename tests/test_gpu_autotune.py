"""The tile autotuner times every field-advance tile variant without changing the state, and
every variant computes the same step (compared with the FP64 oracle)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import core as oc  # noqa: E402

from parity_util import TABLE1, field_error, gpu_sim, oracle_sim  # noqa: E402


@pytest.mark.parametrize("nd,solver,C", [(2, "custom", TABLE1), (3, "yee", None)])
def test_autotune_keeps_state_and_result(nd, solver, C):
    nz, nx, ny = (520, 40, 1) if nd == 2 else (200, 12, 10)
    grid = dict(ndim=nd, nz=nz, nx=nx, ny=ny, dz=0.5, dx=0.4, dy=0.45, dt=0.08, solver=solver, shape=1)
    sim = gpu_sim(grid, [], coef=C)
    osim = oracle_sim(grid, [], coef=C)
    rng = np.random.default_rng(9)
    for a, oa in ((sim.E, osim.E), (sim.B, osim.B), (sim.J, osim.J)):
        v = rng.normal(size=oa.shape).astype(np.float32)
        a.copy_(torch.from_numpy(v))
        oa[:] = v
    E0, B0, J0 = sim.E.clone(), sim.B.clone(), sim.J.clone()
    variant, ms = sim.autotune()
    assert torch.equal(sim.E, E0) and torch.equal(sim.B, B0)
    assert len(ms) >= 3 and np.all(ms > 0) and 0 <= variant < len(ms)
    oc.field_advance(osim.g, osim.E, osim.B, osim.J)
    from paper_1910_13529_gb300 import pic_set_tuning
    for v in range(len(ms)):
        sim.E.copy_(E0)
        sim.B.copy_(B0)
        sim.J.copy_(J0)
        pic_set_tuning(sim.h, v)
        sim.field_advance()
        assert field_error(sim, osim) < 1e-5, v
    sim.close()


VARIANT_CASES = [
    # (ndim, nz, nx, ny, solver, coefficients): nz % 4 != 0 takes the scalar edge path of the
    # register-blocked tiles; nx, ny smaller than a tile make the x/y halos wrap around.
    (2, 203, 11, 1, "custom", TABLE1),
    (2, 130, 4, 1, "yee", None),
    (3, 101, 6, 5, "custom", "fit8"),
    (3, 64, 9, 4, "custom", TABLE1),
]


@pytest.mark.parametrize("nd,nz,nx,ny,solver,C", VARIANT_CASES)
@pytest.mark.parametrize("moving", [False, True])
def test_every_tile_variant_matches_oracle(nd, nz, nx, ny, solver, C, moving):
    from oracle import fit
    from paper_1910_13529_gb300 import pic_get_tuning, pic_set_tuning

    if isinstance(C, str):
        C = fit.fit_coefficients(2.0, M=8)
    d = (0.5, 0.4, 0.45)
    dt = 0.9 * fit.cfl_dt(d[0], [d[1]] + ([d[2]] if nd == 3 else []), C)
    if moving:
        dt = min(dt, 0.6 * d[0])
    grid = dict(ndim=nd, nz=nz, nx=nx, ny=ny, dz=d[0], dx=d[1], dy=d[2], dt=dt, solver=solver, shape=1,
                moving_window=moving)
    osim = oracle_sim(grid, [], coef=C)
    rng = np.random.default_rng(nz + 7 * nx)
    init = [rng.normal(size=a.shape).astype(np.float32) for a in (osim.E, osim.B, osim.J)]
    osim.E[:], osim.B[:], osim.J[:] = init
    nsteps = 4
    for _ in range(nsteps):
        oc.field_advance(osim.g, osim.E, osim.B, osim.J)
        osim.n += 1
        if moving and oc.window_due(osim.n, osim.g.dt, osim.g.dz, osim.shifts):
            osim.shift()
    if moving:
        assert osim.shifts >= 1
    sim = gpu_sim(grid, [], coef=C)
    nv = len(pic_get_tuning(sim.h)[1])
    assert nv == (12 if nd == 2 else 12)
    sim.close()
    for v in range(nv):
        sim = gpu_sim(grid, [], coef=C)
        pic_set_tuning(sim.h, v)
        for a, x in zip((sim.E, sim.B, sim.J), init):
            a.copy_(torch.from_numpy(x))
        for _ in range(nsteps):
            sim.field_advance()
        assert sim.state()[1] == osim.shifts
        assert field_error(sim, osim) < 1e-5, v
        sim.close()


CHUNK_CASES = [
    # 2D x-march (variants 8..11: z segments of 448, 384, 960, 192 cells marching along x in
    # chunks of at least 16 rows): nz = 1502 spans 2 to 8 segments with a ragged last one
    # (nz % 4 = 2), nx = 80 gives 5 x chunks
    (2, 1502, 80, 1, "custom", TABLE1, (8, 9, 10, 11)),
    (2, 1502, 80, 1, "yee", None, (8, 9, 10, 11)),
    # 3D y-march (6..9) and its prefetch ring (10, 11): ny = 20 gives 3 y chunks of >= 8 planes
    (3, 261, 12, 20, "custom", TABLE1, (6, 7, 8, 9, 10, 11)),
]


@pytest.mark.parametrize("nd,nz,nx,ny,solver,C,variants", CHUNK_CASES)
def test_marching_variants_across_chunks(nd, nz, nx, ny, solver, C, variants):
    """The marching field-advance variants on grids large enough for several z segments and
    several x (2D) or y (3D) chunks per launch, with and without the moving-window shift,
    against the FP64 oracle after four steps."""
    from oracle import fit
    from paper_1910_13529_gb300 import pic_set_tuning

    d = (0.5, 0.4, 0.45)
    for moving in (False, True):
        dt = 0.9 * fit.cfl_dt(d[0], [d[1]] + ([d[2]] if nd == 3 else []), C)
        if moving:
            dt = min(dt, 0.6 * d[0])
        grid = dict(ndim=nd, nz=nz, nx=nx, ny=ny, dz=d[0], dx=d[1], dy=d[2], dt=dt, solver=solver, shape=1,
                    moving_window=moving)
        osim = oracle_sim(grid, [], coef=C)
        rng = np.random.default_rng(nz + nx + ny)
        init = [rng.normal(size=a.shape).astype(np.float32) for a in (osim.E, osim.B, osim.J)]
        osim.E[:], osim.B[:], osim.J[:] = init
        nsteps = 4
        for _ in range(nsteps):
            oc.field_advance(osim.g, osim.E, osim.B, osim.J)
            osim.n += 1
            if moving and oc.window_due(osim.n, osim.g.dt, osim.g.dz, osim.shifts):
                osim.shift()
        for v in variants:
            sim = gpu_sim(grid, [], coef=C)
            pic_set_tuning(sim.h, v)
            for a, x in zip((sim.E, sim.B, sim.J), init):
                a.copy_(torch.from_numpy(x))
            for _ in range(nsteps):
                sim.field_advance()
            assert sim.state()[1] == osim.shifts
            assert field_error(sim, osim) < 1e-5, (v, moving)
            sim.close()
