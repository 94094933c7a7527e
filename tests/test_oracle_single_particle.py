"""The oracle's field of one free-streaming relativistic particle against the paper's k-space
integral for E1 (Sec. 2.2, Eq. E12D with the Appendix D k2 integral), evaluated by quadrature.

Yee solver, dx1 = dx2 = 1 (r = 1), kappa = dx1/dt = 4, linear shape, beta -> 1 (gamma = 1e7),
moving window at c so the particle stays in the box; compared after 2000 steps (the particle
has crossed 500 cells), at a step where it sits on a node (N integer).  The integral keeps the
nu1 = 0 and nu1 = +-1 zones; Sec. 2.2 notes that the neglected higher zones matter next to the
particle, so |i'| <= 1 is excluded and the band is 10% of the largest |E1|."""
import math
import warnings

import numpy as np

from oracle import core as oc
from oracle import kspace

warnings.filterwarnings("ignore")


def test_yee_on_axis_e1_matches_kspace_integral():
    nz, nx = 256, 128
    g = oc.Grid(2, nz, nx, 1, 1.0, 1.0, 1.0, 0.25, C=(1.0,), shape=1)
    gam = 1e7
    xi = np.array([[nz - 40.0, nx // 2, 0.0]])
    u = np.array([[math.sqrt(gam * gam - 1.0), 0.0, 0.0]])
    sim = oc.Sim(g, [oc.Species(xi, u, 1.0, 1.0, 1.0)], moving_window=True)
    for _ in range(2000):
        sim.step()
    p = sim.species[0].xi[0]
    N, j0 = int(round(p[0])), int(round(p[1]))
    assert abs(p[0] - N) < 1e-6            # on a node: N = n dt / dx1 is an integer
    E1 = sim.E[0, 0, j0, :]
    ips = [i for i in range(-12, 13) if abs(i) >= 2]
    ref = np.array([kspace.e1_axis_yee(i, 4.0, 1.0, 1) for i in ips])
    sim_v = np.array([E1[N + i] for i in ips])
    band = 0.1 * np.max(np.abs(ref))
    assert np.max(np.abs(sim_v - ref)) < band
    # the Cerenkov wake lies behind the particle (Sec. 2.2)
    assert np.max(np.abs(E1[N - 40:N - 10])) > 20 * np.max(np.abs(E1[N + 10:N + 30]))


def test_customised_solver_removes_the_cerenkov_wake():
    """Sec. 3: with [k]_1 ~ [k1]_t there is no Cerenkov-like field from the fundamental zone, so
    the oscillating field behind a beta -> 1 particle is several times weaker than with Yee.
    The uniform part behind the particle (the same for both solvers: the periodic transverse
    box) is removed by comparing the spread about the mean over i' in [-150, -20]."""
    from oracle import fit
    C = np.loadtxt(__file__.replace("test_oracle_single_particle.py", "golden/table1_coefficients.txt"))
    nz, nx = 240, 64
    spread, mean = {}, {}
    for solver in ("yee", "custom"):
        g = oc.Grid(2, nz, nx, 1, 1.0, 1.0, 1.0, 0.25, C=(C if solver == "custom" else (1.0,)), shape=1)
        sim = oc.Sim(g, [oc.Species(np.array([[nz - 30.0, nx // 2, 0.0]]), np.array([[1e7, 0.0, 0.0]]), 1.0, 1.0,
                                    1.0)], h=(fit.correction_kernel(C, 40) if solver == "custom" else None),
                     moving_window=True)
        for _ in range(1000):
            sim.step()
        N = int(round(sim.species[0].xi[0, 0]))
        seg = sim.E[0, 0, nx // 2, N - 150:N - 20]
        spread[solver], mean[solver] = seg.std(), seg.mean()
    assert spread["custom"] < 0.35 * spread["yee"]
    assert abs(mean["custom"] - mean["yee"]) < 0.1 * abs(mean["yee"])
