"""Writes stencil_gradient_1024x256.txt: FP64 central finite differences, computed with the
oracle only, of the stencil-tuning loss (field energy left behind a rigid line of 64 electrons
at gamma = 1e4 after 500 steps on a 1024 x 256 grid, dz = dx = 0.05, dt = dz/4) with respect to
the 4 axial coefficients of the Appendix C fit at kappa = 4 (M = 4).

    python tests/golden/make_stencil_gradient.py
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

NSTEPS = 500
BEHIND = 2
RIGID_MASS = 1e30


def loss(C):
    from oracle import core as oc
    from oracle import fit
    from paper_1910_13529_gb300 import workloads as wl
    grid, sps = wl.rigid_line()
    C = np.asarray(C, dtype=np.float64)
    g = oc.Grid(2, grid["nz"], grid["nx"], 1, grid["dz"], grid["dx"], grid["dy"], grid["dt"], C=C, shape=1)
    species = [oc.Species(wl.xi_of(sp, 2), sp["u"].T.astype(np.float64), sp["q"], RIGID_MASS, sp["w"]) for sp in sps]
    sim = oc.Sim(g, species, h=fit.correction_kernel(C, hlen=40))
    for _ in range(NSTEPS):
        sim.step()
    zc = max(int(np.floor(min(s.xi[:, 0].min() for s in sim.species))) - BEHIND, 0)
    return 0.5 * (np.sum(sim.E[..., :zc] ** 2) + np.sum(sim.B[..., :zc] ** 2)) * grid["dz"] * grid["dx"]


def main():
    from oracle import fit
    C = fit.fit_coefficients(4.0, M=4)
    pts = [C.copy()]
    eps = []
    for l in range(4):
        e = 1e-5 * max(abs(C[l]), 1e-3)
        eps.append(e)
        for sgn in (1, -1):
            Cq = C.copy()
            Cq[l] += sgn * e
            pts.append(Cq)
    with mp.get_context("spawn").Pool(min(9, os.cpu_count() or 1)) as pool:
        vals = pool.map(loss, pts)
    grad = [(vals[1 + 2 * l] - vals[2 + 2 * l]) / (2 * eps[l]) for l in range(4)]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "stencil_gradient_1024x256.txt")
    with open(out, "w") as f:
        f.write("# FP64 oracle, central differences: 1024x256, 64 rigid electrons, gamma 1e4, 500 steps,\n")
        f.write("# dz = dx = 0.05, dt = dz/4, M = 4 coefficients of the Appendix C fit at kappa = 4.\n")
        f.write("# written by tests/golden/make_stencil_gradient.py (oracle only)\n")
        f.write(f"loss {float(vals[0])!r}\n")
        for l in range(4):
            f.write(f"C{l + 1} {float(C[l])!r} dL/dC{l + 1} {float(grad[l])!r}\n")
    print(open(out).read())


if __name__ == "__main__":
    main()
