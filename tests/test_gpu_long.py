"""Long GPU runs against the FP64 oracle: the <= 1e-5 relative tolerance held over 1000 steps.

* Vacuum runs, linear or nearly so (a single particle, a rigid line of particles): E, B and the
  particle momenta are compared end to end after 1000 steps (and the stencil-tuning run at its
  own full size and length, 1024 x 256 for 500 steps).
* Beam in plasma with the moving window: trajectories of an FP32 and an FP64 plasma separate
  slowly, so the binding checks are one step of parity taken from the oracle's state every 100
  steps (E, B, positions and momenta at 1e-5) and the field relative L2 error of the two whole
  1000-step runs, next to Gauss's law kept on the GPU.

Each test reports max-abs and relative-L2 errors of E, B and u; with the environment variable
PIC_ACCURACY_REPORT set to a file name, they are appended there as JSON lines."""
import json
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import core as oc  # noqa: E402
from oracle import fit  # noqa: E402
import paper_1910_13529_gb300 as P  # noqa: E402
from paper_1910_13529_gb300 import workloads as wl  # noqa: E402

from parity_util import TABLE1, gpu_particles, gpu_sim, oracle_sim  # noqa: E402

TOL = 1e-5


def errors(sim, osim, species=(0,), pending_shift=0):
    """max-abs (relative to the largest oracle value) and relative-L2 errors of E, B and u."""
    out = {}
    for name, g, o in (("E", sim.E, osim.E), ("B", sim.B, osim.B)):
        a = g.double().cpu().numpy()
        scale = max(np.abs(o).max(), 1e-300)
        out[name] = dict(max_abs=float(np.abs(a - o).max()), max_rel=float(np.abs(a - o).max() / scale),
                         rel_l2=float(np.sqrt(np.sum((a - o) ** 2) / max(np.sum(o ** 2), 1e-300))))
    us, uo, dx = [], [], 0.0
    for s in species:
        ids, xi, u = gpu_particles(sim, s, sim.ndim, pending_shift)
        sp = osim.species[s]
        o = np.argsort(sp.ids, kind="stable")
        assert np.array_equal(ids, sp.ids[o]), "particle sets differ"
        d = xi - sp.xi[o]
        d[:, 1] = (d[:, 1] + sim.nx / 2) % sim.nx - sim.nx / 2
        dx = max(dx, float(np.abs(d).max()) if len(d) else 0.0)
        us.append(u)
        uo.append(sp.u[o])
    u, uo = np.concatenate(us), np.concatenate(uo)
    if len(u):
        scale = max(np.abs(uo).max(), 1e-300)
        out["u"] = dict(max_abs=float(np.abs(u - uo).max()), max_rel=float(np.abs(u - uo).max() / scale),
                        rel_l2=float(np.sqrt(np.sum((u - uo) ** 2) / max(np.sum(uo ** 2), 1e-300))))
    out["x_cells_max_abs"] = dx
    return out


def report(name, steps, errs):
    line = dict(case=name, steps=steps, **errs)
    print(json.dumps(line))
    path = os.environ.get("PIC_ACCURACY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(line) + "\n")


@pytest.mark.parametrize("solver,shape,C", [("yee", 1, None), ("custom", 2, TABLE1)])
def test_single_particle_1000_steps(solver, shape, C):
    """The 256 x 128 single-particle vacuum run (gamma = 1000, dt = 0.45 dz) with the window
    following the particle at c, 1000 steps (the particle crosses 450 cells)."""
    grid, sps = wl.single_particle(shape=shape, solver=solver)
    grid["moving_window"] = True
    sim = gpu_sim(grid, sps, coef=C)
    osim = oracle_sim(grid, sps, coef=C)
    n = 1000
    sim.step(n)
    for _ in range(n):
        osim.step()
    step, shifts, pend = sim.state()
    assert shifts == osim.shifts == 450
    e = errors(sim, osim, pending_shift=pend)
    report(f"single_particle_256x128_{solver}", n, e)
    assert e["E"]["max_rel"] < TOL and e["B"]["max_rel"] < TOL
    assert e["u"]["max_rel"] < TOL and e["x_cells_max_abs"] < TOL
    sim.close()


def _rigid(nz, nx, n):
    grid, sps = wl.rigid_line(nz=nz, nx=nx, d=0.05, dt_over_dz=0.25, gamma=1e4, n=n)
    sps[0]["m"] = 1e30                    # rigid: momenta never change
    grid.update(solver="custom", shape=1)
    return grid, sps


@pytest.mark.parametrize("nz,nx,n,steps", [(512, 128, 32, 1000), (1024, 256, 64, 500)])
def test_rigid_line(nz, nx, n, steps):
    """The stencil-tuning workload (a transverse line of electrons at gamma = 1e4, kappa = 4, M = 4
    fitted coefficients): a reduced grid for 1000 steps and the full 1024 x 256 run for its 500."""
    C4 = fit.fit_coefficients(4.0, M=4)
    grid, sps = _rigid(nz, nx, n)
    sim = gpu_sim(grid, sps, coef=C4)
    osim = oracle_sim(grid, sps, coef=C4)
    sim.step(steps)
    for _ in range(steps):
        osim.step()
    e = errors(sim, osim)
    report(f"rigid_line_{nz}x{nx}_M4", steps, e)
    assert e["E"]["max_rel"] < TOL and e["B"]["max_rel"] < TOL
    # rigid: momenta stay at their initial values up to the denormal noise of eps ~ 1e-32
    assert e["u"]["max_rel"] < 1e-12 and e["x_cells_max_abs"] < TOL
    sim.close()


def _plasma_grid():
    grid, sps = wl.beam_plasma(ndim=2, nz=192, nx=16, n_beam=2000, sigma_z=0.3, sigma_r=0.06,
                               behind_front=1.2, gamma=2e4, solver="custom")
    return grid, sps


def _species_from_oracle(osim, template):
    """FP32 (cell, offset) species dicts of the oracle's particles; the oracle side is rebuilt
    from the same rounded values, so both runs of the next step start from identical states."""
    out = []
    for sp, t in zip(osim.species, template):
        xi = sp.xi
        cell = np.floor(xi).astype(np.int64)
        off = (xi - cell).astype(np.float32)
        bad = off >= np.float32(1.0)
        off[bad] = np.nextafter(np.float32(1.0), np.float32(0.0))
        out.append(wl.species(cell[:, 0], cell[:, 1], np.zeros(len(xi), np.int64), off.T[:2],
                              sp.u.T.astype(np.float32), t["q"], t["m"], t["w"], ids=sp.ids))
    return out


def test_beam_plasma_1000_steps():
    grid, sps = _plasma_grid()
    C = fit.fit_coefficients(grid["dz"] / grid["dt"])
    sim = gpu_sim(grid, sps, coef=C, cap_extra=60000)
    osim = oracle_sim(grid, sps, coef=C)
    n_total, every = 1000, 100
    worst = {}
    for k in range(n_total // every):
        # one step from the oracle's state (rounded to FP32 on both sides)
        rs = _species_from_oracle(osim, sps)
        a = gpu_sim(grid, rs, coef=C, cap_extra=60000)
        b = oracle_sim(grid, rs, coef=C)
        E32, B32 = osim.E.astype(np.float32), osim.B.astype(np.float32)
        a.E.copy_(torch.from_numpy(E32))
        a.B.copy_(torch.from_numpy(B32))
        b.E[:], b.B[:] = E32, B32
        b.n, b.shifts = osim.n, osim.shifts
        b.inject["next_id"] = osim.inject["next_id"]
        P.pic_set_state(a.h, osim.n, osim.shifts, 0, osim.inject["next_id"])
        a.step(1)
        b.step()
        e1 = errors(a, b, species=(0, 1), pending_shift=a.state()[2])
        for q in ("E", "B", "u"):
            worst[q] = max(worst.get(q, 0.0), e1[q]["max_rel"])
        worst["x"] = max(worst.get("x", 0.0), e1["x_cells_max_abs"])
        assert e1["E"]["max_rel"] < TOL and e1["B"]["max_rel"] < TOL, (k, e1)
        assert e1["u"]["max_rel"] < TOL and e1["x_cells_max_abs"] < TOL, (k, e1)
        a.close()
        # both whole runs advance 100 steps
        sim.step(every)
        for _ in range(every):
            osim.step()
    step, shifts, pend = sim.state()
    assert step == n_total and shifts == osim.shifts
    E = sim.E.double().cpu().numpy()
    B = sim.B.double().cpu().numpy()
    rel_l2 = math.sqrt((np.sum((E - osim.E) ** 2) + np.sum((B - osim.B) ** 2)) /
                       (np.sum(osim.E ** 2) + np.sum(osim.B ** 2)))
    line = dict(one_step_worst_max_rel=worst, whole_run_field_rel_l2=rel_l2,
                whole_run_E=dict(max_rel=float(np.abs(E - osim.E).max() / np.abs(osim.E).max())),
                whole_run_B=dict(max_rel=float(np.abs(B - osim.B).max() / np.abs(osim.B).max())))
    report("beam_plasma_2d_192x16_window", n_total, line)
    # the separation of FP32 and FP64 plasma trajectories stays small over the run
    assert rel_l2 < 1e-3
    sim.close()
