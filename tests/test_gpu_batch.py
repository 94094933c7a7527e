"""Batched runs (pic_batch_*): heterogeneous independent instances advanced by one launch per
kernel class and step (CUDA graph), each compared with its own FP64 oracle run and with the
same instance advanced alone by pic_step.  Tolerance 1e-5 as in test_gpu_parity.py."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import fit  # noqa: E402
from paper_1910_13529_gb300 import workloads as wl  # noqa: E402
from paper_1910_13529_gb300.runtime import Batch  # noqa: E402

from parity_util import field_error, gpu_sim, oracle_sim, particle_errors  # noqa: E402

TOL = 1e-5


def instances(seed=4000, sizes=((150, 20), (200, 17), (96, 33), (260, 12), (128, 64), (300, 25))):
    rng = np.random.default_rng(seed)
    out = []
    for i, (nz, nx) in enumerate(sizes):
        solver = "custom" if i % 2 else "yee"
        shape = 1 + (i // 2) % 2
        d = 0.05
        if solver == "custom":
            kappa = 1.0 / (0.5 * rng.uniform(0.3, 0.9))
            C = fit.fit_coefficients(kappa, M=16 if i % 4 == 1 else 8)
            dt = d / kappa
            assert dt < fit.cfl_dt(d, [d], C)
        else:
            C = None
            dt = rng.uniform(0.3, 0.99) * fit.cfl_dt(d, [d])
        grid = dict(ndim=2, nz=nz, nx=nx, ny=1, dz=d, dx=d, dy=d, dt=dt, solver=solver, shape=shape)
        gamma = 10 ** rng.uniform(1, 5)
        _, sp1 = wl.single_particle(nz=nz, nx=nx, d=d, dt_over_dz=dt / d, gamma=gamma, z_cell=nz / 5,
                                    x_cell=nx / 2 + 0.3)
        extra = wl.random_particles(2, nz, nx, 1, 60, seed=seed + i, u_scale=1.0, u_drift=(2.0, 0, 0),
                                    margin=nz // 4)
        sp = {k: (np.concatenate([sp1[0][k], extra[k]], axis=-1) if isinstance(sp1[0][k], np.ndarray)
                  else sp1[0][k]) for k in sp1[0]}
        sp["ids"] = np.arange(len(sp["iz"]))
        out.append((grid, [sp], C))
    return out


def test_batch_matches_oracle_and_single_runs():
    inst = instances()
    cfgs = []
    for grid, sps, C in inst:
        c = {k: grid[k] for k in ("ndim", "nz", "nx", "dz", "dx", "dt", "shape", "solver")}
        if C is not None:
            c["coef"] = C
        cfgs.append(c)
    batch = Batch(cfgs)
    for sim, (grid, sps, C) in zip(batch.instances, inst):
        sp = sps[0]
        sim.add_species(0, sp["iz"], sp["ix"], sp["iy"], sp["off"], sp["u"], sp["q"], sp["m"], sp["w"],
                        ids=sp["ids"])
    nsteps = 21                                   # odd: the last step ends in the second buffer
    batch.step(nsteps)
    torch.cuda.synchronize()
    for sim, (grid, sps, C) in zip(batch.instances, inst):
        osim = oracle_sim(grid, sps, coef=C)
        for _ in range(nsteps):
            osim.step()
        assert field_error(sim, osim) < TOL
        dx, du = particle_errors(sim, osim, 0, 2)
        assert dx < TOL and du < TOL
        single = gpu_sim(grid, sps, coef=C)
        single.step(nsteps)
        # the batch may use another field-advance tile variant than the single run: agreement to
        # FP32 rounding order, within the parity tolerance
        scale = max(single.E.abs().max().item(), single.B.abs().max().item())
        assert (single.E - sim.E).abs().max().item() <= TOL * scale
        assert (single.B - sim.B).abs().max().item() <= TOL * scale
        single.close()
    batch.close()


def test_batch_graph_replays_consistently():
    """Two runs of 10 steps equal one run of 20 (graph replay across calls keeps the parity)."""
    inst = instances(seed=4100, sizes=((128, 16), (160, 24)))
    cfgs = []
    for grid, sps, C in inst:
        c = {k: grid[k] for k in ("ndim", "nz", "nx", "dz", "dx", "dt", "shape", "solver")}
        if C is not None:
            c["coef"] = C
        cfgs.append(c)
    a, b = Batch(cfgs), Batch(cfgs)
    for bt in (a, b):
        for sim, (grid, sps, C) in zip(bt.instances, inst):
            sp = sps[0]
            sim.add_species(0, sp["iz"], sp["ix"], sp["iy"], sp["off"], sp["u"], sp["q"], sp["m"], sp["w"])
    a.step(10)
    a.step(10)
    b.step(20)
    torch.cuda.synchronize()
    for sa, sb in zip(a.instances, b.instances):
        assert torch.equal(sa.E, sb.E) or (sa.E - sb.E).abs().max().item() < 1e-6 * sb.E.abs().max().item()
    a.close()
    b.close()


def test_batched_vacuum_scan_256_instances():
    """The batched scan as benchmarked: 256 instances of uneven grids (128..1024 x 64..256), gamma,
    dt and stencil drawn per instance, 400 steps in one pic_batch_step call; a seeded sample of
    instances (both stencils) against their FP64 oracle runs."""
    from oracle import core as oc
    cfgs, runs = [], []
    for grid, gamma in wl.batched_vacuum_scan(256, 4000):
        C = fit.fit_coefficients(grid["dz"] / grid["dt"], M=16) if grid["solver"] == "custom" else None
        _, sps = wl.single_particle(nz=grid["nz"], nx=grid["nx"], d=grid["dz"], dt_over_dz=grid["dt"] / grid["dz"],
                                    gamma=gamma, z_cell=grid["nz"] / 8, x_cell=grid["nx"] / 2)
        c = {k: grid[k] for k in ("ndim", "nz", "nx", "dz", "dx", "dt", "shape", "solver")}
        if C is not None:
            c["coef"] = C
        cfgs.append(c)
        runs.append((grid, sps, C))
    batch = Batch(cfgs)
    for sim, (grid, sps, C) in zip(batch.instances, runs):
        sp = sps[0]
        sim.add_species(0, sp["iz"], sp["ix"], sp["iy"], sp["off"], sp["u"], sp["q"], sp["m"], sp["w"],
                        ids=sp["ids"])
    nsteps = 400
    batch.step(nsteps)
    torch.cuda.synchronize()
    from paper_1910_13529_gb300 import pic_batch_get_tuning
    variants, ms = pic_batch_get_tuning(batch.b)
    assert variants[0] in (0, 1, 2) and variants[3] in (0, 1, 2) and ms[0, variants[0]] > 0
    rng = np.random.default_rng(7)
    yee = [i for i, r in enumerate(runs) if r[2] is None]
    cus = [i for i, r in enumerate(runs) if r[2] is not None]
    sample = list(rng.choice(yee, 3, replace=False)) + list(rng.choice(cus, 3, replace=False))
    prev = oc.set_threads(4)
    try:
        for i in sample:
            grid, sps, C = runs[i]
            osim = oracle_sim(grid, sps, coef=C)
            for _ in range(nsteps):
                osim.step()
            sim = batch.instances[i]
            assert field_error(sim, osim) < TOL, i
            dx, du = particle_errors(sim, osim, 0, 2)
            assert dx < TOL and du < TOL, i
    finally:
        oc.set_threads(1)
    batch.close()
