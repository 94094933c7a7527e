"""Shared helpers of the GPU parity tests: build the CUDA run and the FP64 oracle run from the
same seeded workload and compare them.  Coefficients are given explicitly to both sides; the
oracle computes its own correction taps."""
import os

import numpy as np

from oracle import core as oc
from oracle import fit
from paper_1910_13529_gb300 import decode_cells
from paper_1910_13529_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLE1 = np.loadtxt(os.path.join(ROOT, "tests", "golden", "table1_coefficients.txt"))


def gpu_sim(grid, sps, coef=None, cap_extra=0, sort_every=0, ids=True):
    from paper_1910_13529_gb300.runtime import Simulation
    kw = dict(ndim=grid["ndim"], nz=grid["nz"], nx=grid["nx"], ny=grid.get("ny", 1), dz=grid["dz"],
              dx=grid["dx"], dy=grid.get("dy", grid["dx"]), dt=grid["dt"], shape=grid.get("shape", 1),
              solver=grid.get("solver", "yee"), moving_window=grid.get("moving_window", False),
              inject_species=grid.get("inject_species", -1), inject_ppc=grid.get("inject_ppc", (1, 1, 1)),
              rho_bg=grid.get("rho_bg", 0.0), sort_every=sort_every,
              current_filter=grid.get("current_filter", False))
    if kw["solver"] == "custom":
        kw["coef"] = coef
        if grid.get("coef_b") is not None:
            kw["coef_b"] = grid["coef_b"]
    sim = Simulation(device="cuda:0", **kw)
    for s, sp in enumerate(sps):
        n = len(sp["iz"])
        sim.add_species(s, sp["iz"], sp["ix"], sp["iy"], sp["off"], sp["u"], sp["q"], sp["m"], sp["w"],
                        cap=n + cap_extra, ids=sp["ids"] if ids else None)
    return sim


def oracle_sim(grid, sps, coef=None):
    nd = grid["ndim"]
    solver = grid.get("solver", "yee")
    kspace = solver if solver in ("spectral", "kt", "psatd") else None
    C = (1.0,) if solver in ("yee", "spectral", "kt", "psatd") else coef
    Cb = grid.get("coef_b") if grid.get("solver", "yee") == "custom" else None
    g = oc.Grid(nd, grid["nz"], grid["nx"], grid.get("ny", 1), grid["dz"], grid["dx"],
                grid.get("dy", grid["dx"]), grid["dt"], C=C, shape=grid.get("shape", 1), Cb=Cb)
    # Sec. 3 correction from the B-side coefficients (none when the B side is the Yee difference)
    CBeff = C if Cb is None else Cb
    yee_b = Cb is not None and np.allclose(np.asarray(Cb, dtype=np.float64), np.eye(1, len(Cb))[0], rtol=0, atol=0)
    h = None if solver != "custom" or yee_b else fit.correction_kernel(CBeff, hlen=40)
    species = [oc.Species(wl.xi_of(sp, nd), sp["u"].T.astype(np.float64), sp["q"], sp["m"], sp["w"],
                          ids=sp["ids"]) for sp in sps]
    inject = None
    if grid.get("inject_species", -1) >= 0:
        total = sum(len(sp["iz"]) for sp in sps[: grid["inject_species"] + 1])
        inject = dict(species=grid["inject_species"], ppc=grid["inject_ppc"],
                      next_id=max(len(sp["iz"]) for sp in sps))
    return oc.Sim(g, species, h=h, moving_window=grid.get("moving_window", False), inject=inject,
                  filt=grid.get("current_filter", False), kspace=kspace)


def field_error(sim, osim):
    """max |GPU - oracle| over E and B, relative to the largest |oracle field|."""
    E = sim.E.double().cpu().numpy()
    B = sim.B.double().cpu().numpy()
    scale = max(np.abs(osim.E).max(), np.abs(osim.B).max(), 1e-300)
    return max(np.abs(E - osim.E).max(), np.abs(B - osim.B).max()) / scale


def field_rel_l2(sim, osim):
    E = sim.E.double().cpu().numpy()
    B = sim.B.double().cpu().numpy()
    num = np.sqrt(np.sum((E - osim.E) ** 2) + np.sum((B - osim.B) ** 2))
    den = np.sqrt(np.sum(osim.E ** 2) + np.sum(osim.B ** 2))
    return num / max(den, 1e-300)


def gpu_particles(sim, s, ndim, pending_shift=0):
    """Live particles of species s as (ids, xi (n,3), u (n,3)) sorted by id, in the frame of the
    last completed step (a window shift still pending on the particles is applied here)."""
    p = sim.particles(s)
    alive = p["cell"] >= 0
    iz, ix, iy = decode_cells(p["cell"], sim.nz, sim.nx)
    alive &= (iz - pending_shift) >= 0
    iz, ix, iy = iz[alive] - pending_shift, ix[alive], iy[alive]
    xi = np.zeros((alive.sum(), 3))
    xi[:, 0] = iz + p["off"][0][alive].astype(np.float64)
    xi[:, 1] = ix + p["off"][1][alive].astype(np.float64)
    if ndim == 3:
        xi[:, 2] = iy + p["off"][2][alive].astype(np.float64)
    u = p["u"][:, alive].T.astype(np.float64)
    ids = p["id"][alive].astype(np.int64) if p["id"] is not None else np.arange(alive.sum())
    o = np.argsort(ids, kind="stable")
    return ids[o], xi[o], u[o]


def particle_errors(sim, osim, s, ndim, pending_shift=0):
    ids, xi, u = gpu_particles(sim, s, ndim, pending_shift)
    sp = osim.species[s]
    o = np.argsort(sp.ids, kind="stable")
    oids, oxi, ou = sp.ids[o], sp.xi[o], sp.u[o]
    assert np.array_equal(ids, oids), f"particle sets differ: {len(ids)} vs {len(oids)}"
    d = xi - oxi
    d[:, 1] = (d[:, 1] + sim.nx / 2) % sim.nx - sim.nx / 2
    if ndim == 3:
        d[:, 2] = (d[:, 2] + sim.ny / 2) % sim.ny - sim.ny / 2
    uscale = max(np.abs(ou).max() if len(ou) else 0.0, 1e-6)
    return (np.abs(d).max() if len(d) else 0.0), (np.abs(u - ou).max() / uscale if len(u) else 0.0)
