"""Parity at full size, in the launch configuration bench.py times (particles sorted by cell at step 0,
fused pic_step).

Cases: the 2D beam-in-plasma run (2048 x 512, 5.19M particles, customised M = 16, quadratic)
and the 3D run (512 x 256 x 256, 71M particles).  One step from seeded random fields; the
oracle recomputes sampled outputs one by one:
  * particles: gather + Boris + move of sampled particles on the full FP64 fields;
  * current and fields: for sampled cells, the oracle deposits the particles of a local box
    (wide enough for the Sec. 3 correction and the field stencil), corrects J1, and advances
    the fields of the sub-box around the cell; the dependency cone of the centre lies inside
    the box, so the centre values are exact;
  * Gauss's law: the change of d-.E - rho over the step, at every interior node (any size).
Tolerance 1e-5 as in test_gpu_parity.py."""
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

from parity_util import gpu_sim  # noqa: E402

TOL = 1e-5
CASES = {
    "beam2d_2048x512": lambda: wl.beam_plasma(),
    "beam3d_512x256x256": lambda: wl.beam_plasma_3d(),
}


def _random_fields(sim, rng, amp):
    host = []
    for t in (sim.E, sim.B):
        v = (amp * rng.standard_normal(size=tuple(t.shape), dtype=np.float32))
        t.copy_(torch.from_numpy(v))
        host.append(v)
    return host


def _box(center, half, n, periodic):
    """Indices of a window of +-half around center (wrapped if periodic, clipped otherwise)."""
    if periodic:
        return np.arange(center - half, center + half + 1) % n
    lo, hi = max(0, center - half), min(n, center + half + 1)
    return np.arange(lo, hi)


@pytest.mark.parametrize("case", list(CASES))
def test_fullsize_step_sampled(case):
    grid, sps = CASES[case]()
    nd, nz, nx, ny = grid["ndim"], grid["nz"], grid["nx"], grid.get("ny", 1)
    C = fit.fit_coefficients(grid["dz"] / grid["dt"])
    # sorted by cell before the step, as bench.py runs it (sort_every = 20 sorts at step 0)
    sim = gpu_sim(grid, sps, coef=C, cap_extra=100_000, sort_every=20)
    rng = np.random.default_rng(77)
    E0, B0 = _random_fields(sim, rng, 0.5)
    G0 = sim.gauss()
    rmax = float(sim.rho().abs().max())
    sim.step(1)
    torch.cuda.synchronize()
    st = sim.state()
    assert st[0] == 1 and st[1] == 0                  # no window shift at the first step

    # Gauss's law at every interior node
    dG = (sim.gauss() - G0)[..., 48:-48]
    assert float(dG.abs().max()) < TOL * rmax

    g = oc.Grid(nd, nz, nx, ny, grid["dz"], grid["dx"], grid["dy"], grid["dt"], C=C, shape=grid["shape"])
    E64, B64 = E0.astype(np.float64), B0.astype(np.float64)
    h = fit.correction_kernel(C, hlen=40)

    # sampled particles, found by id (the sort moved them; no deaths in one step at the centre)
    for s, sp in enumerate(sps):
        n = len(sp["iz"])
        idx = np.sort(rng.choice(n, size=min(400, n), replace=False))
        ngpu = sim.count(s)
        gid = sim.species[s]["id"][:ngpu].cpu().numpy().astype(np.int64)
        slot_of = np.full(n, -1, np.int64)
        ok_id = (gid >= 0) & (gid < n)
        slot_of[gid[ok_id]] = np.arange(ngpu)[ok_id]
        slots = slot_of[idx]
        assert np.all(slots >= 0)
        xi0 = wl.xi_of({k: (v[..., idx] if isinstance(v, np.ndarray) and v.shape[-1] == n else v)
                        for k, v in sp.items()}, nd)
        u = sp["u"][:, idx].T.astype(np.float64).copy()
        eb = oc.gather(g, E64, B64, xi0)
        oc.boris(eb, u, sp["q"] * g.dt / (2 * sp["m"]))
        xi1 = oc.move(g, xi0, u)
        d = sim.species[s]
        ts = torch.from_numpy(slots).to(d["cell"].device)
        cell = d["cell"][ts].cpu().numpy()
        off = d["off"][:, ts].cpu().numpy().astype(np.float64)
        ug = d["u"][:, ts].cpu().numpy().T.astype(np.float64)
        live = cell >= 0
        assert live.mean() > 0.99
        iz, ix, iy = decode_cells(cell[live], nz, nx)
        xg = np.stack([iz + off[0][live], ix + off[1][live],
                       (iy + off[2][live]) if nd == 3 else np.zeros(live.sum())], axis=1)
        dx = xg - xi1[live]
        dx[:, 1] = (dx[:, 1] + nx / 2) % nx - nx / 2
        if nd == 3:
            dx[:, 2] = (dx[:, 2] + ny / 2) % ny - ny / 2
        assert np.abs(dx).max() < TOL
        assert np.abs(ug[live] - u[live]).max() < TOL * max(np.abs(u).max(), 1.0)

    # sampled cells: local deposit + correction + field advance in the oracle
    allxi = [wl.xi_of(sp, nd) for sp in sps]
    Jg = sim.J.cpu().numpy()
    Eg, Bg = sim.E.cpu().numpy(), sim.B.cpu().numpy()
    M = len(C)
    Lf = 3 * M + 2                   # field-advance dependency (z)
    Lj = Lf + 40 + 3                 # + correction taps + shape support
    T = 2                            # transverse: stencil +-2, shape +-2
    beam = sps[1]
    picks = [(int(beam["iz"][k]), int(beam["ix"][k]), int(beam["iy"][k]))
             for k in rng.choice(len(beam["iz"]), size=6, replace=False)]
    picks += [(int(rng.integers(0, nz)), int(rng.integers(0, nx)), int(rng.integers(0, ny))) for _ in range(6)]
    picks += [(0, 0, 0), (nz - 1, nx - 1, ny - 1)]
    errJ, errF, scaleJ, scaleF = 0.0, 0.0, 0.0, 0.0
    for (ci, cj, ck) in picks:
        zi = _box(ci, Lj, nz, False)
        xj = _box(cj, T + 6, nx, True)
        yk = _box(ck, T + 6, ny, True) if nd == 3 else np.array([0])
        hx = len(xj) // 2
        hy = len(yk) // 2 if nd == 3 else 0

        def sub(F):
            return np.ascontiguousarray(F[:, yk][:, :, xj][:, :, :, zi])
        gb = oc.Grid(nd, len(zi), len(xj), len(yk), grid["dz"], grid["dx"], grid["dy"], grid["dt"], C=C,
                     shape=grid["shape"])
        J = gb.zeros()
        for s, sp in enumerate(sps):
            xi = allxi[s]
            rel_x = (xi[:, 1] - cj + nx / 2) % nx - nx / 2
            sel = (xi[:, 0] >= zi[0] - 3) & (xi[:, 0] < zi[-1] + 4) & (np.abs(rel_x) < hx - 1)
            if nd == 3:
                rel_y = (xi[:, 2] - ck + ny / 2) % ny - ny / 2
                sel &= np.abs(rel_y) < hy - 1
            if not sel.any():
                continue
            loc = xi[sel].copy()
            loc[:, 0] -= zi[0]
            loc[:, 1] = rel_x[sel] + hx
            if nd == 3:
                loc[:, 2] = rel_y[sel] + hy
            uu = sp["u"][:, sel].T.astype(np.float64).copy()
            eb = oc.gather(gb, sub(E64), sub(B64), loc)
            oc.boris(eb, uu, sp["q"] * g.dt / (2 * sp["m"]))
            loc1 = oc.move(gb, loc, uu)
            # the domain's z ends are the box's only where the box reaches them
            oc.deposit(gb, loc, loc1, uu, sp["q"] * sp["w"], J)
        oc.correct_j1(gb, h, J)
        zc = ci - zi[0]
        # the current at the centre node
        Jc = J[:, hy, hx, zc]
        Jgc = Jg[:, ck, cj, ci]
        errJ = max(errJ, np.abs(Jc - Jgc).max())
        scaleJ = max(scaleJ, np.abs(J[:, hy, hx, max(0, zc - 2):zc + 3]).max())
        # fields: advance the sub-box with that current
        Eb = sub(E64)
        Bb = sub(B64)
        oc.field_advance(gb, Eb, Bb, J)
        Ec, Bc = Eb[:, hy, hx, zc], Bb[:, hy, hx, zc]
        errF = max(errF, np.abs(Ec - Eg[:, ck, cj, ci]).max(), np.abs(Bc - Bg[:, ck, cj, ci]).max())
        scaleF = max(scaleF, np.abs(Eb).max(), np.abs(Bb).max())
    assert errJ <= TOL * max(scaleJ, 1e-30) or errJ < 1e-6
    assert errF <= TOL * scaleF
    sim.close()
