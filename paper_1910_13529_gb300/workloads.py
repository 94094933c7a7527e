"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests and bench.py.

This module draws particle positions and momenta and states grid parameters; it holds none
of the PIC arithmetic.  Positions come out in the library's storage form -- integer cell
(iz, ix, iy) plus FP32 in-cell offsets in [0, 1) -- so both sides see identical inputs:
the oracle uses xi = cell + float64(offset).

Workloads (the paper's runs are OSIRIS simulations of one free-streaming particle at
dx1 = 1, r = 1, kappa = 4 and of a drifting 3D beam; no public dataset is involved):
  single_particle   one relativistic macro-electron along +z in 2D vacuum (Sec. 2-3 runs)
  beam_plasma       relativistic bi-Gaussian electron beam in uniform cold plasma with a
                    moving window (2D and 3D; Sec. 3 drifting-beam run)
  rigid_line        a transverse line of electrons at fixed gamma (stencil-tuning workload)
"""
import math

import numpy as np

# dt = 0.9 x the stricter of the Yee and customised stability limits at dz = dx = 0.02 (2D)
# and dz = 0.02, dx = dy = 0.05 (3D); the customised limit is the fixed point of the
# Appendix C fit at its own kappa (kappa_CFL = 1.6325 in 2D r = 1, 1.3214 in 3D).
DT_BEAM_2D = 0.011026
DT_BEAM_3D = 0.013623


def _split(xi):
    """Cell index and FP32 offset of cell-unit positions, offset strictly below 1."""
    cell = np.floor(xi).astype(np.int64)
    off = (xi - cell).astype(np.float32)
    bad = off >= np.float32(1.0)
    off[bad] = np.nextafter(np.float32(1.0), np.float32(0.0))
    return cell, off


def species(iz, ix, iy, off, u, q, m, w, ids=None):
    n = len(iz)
    return dict(iz=np.asarray(iz, np.int64), ix=np.asarray(ix, np.int64), iy=np.asarray(iy, np.int64),
                off=np.ascontiguousarray(off, dtype=np.float32), u=np.ascontiguousarray(u, dtype=np.float32),
                q=float(q), m=float(m), w=float(w),
                ids=np.arange(n, dtype=np.int64) if ids is None else np.asarray(ids, np.int64))


def xi_of(sp, ndim):
    """Cell-unit positions (n, 3) in FP64 of a species dict (exact widening of the FP32 offsets)."""
    n = len(sp["iz"])
    xi = np.zeros((n, 3))
    xi[:, 0] = sp["iz"] + sp["off"][0].astype(np.float64)
    xi[:, 1] = sp["ix"] + sp["off"][1].astype(np.float64)
    if ndim == 3:
        xi[:, 2] = sp["iy"] + sp["off"][2].astype(np.float64)
    return xi


def single_particle(nz=256, nx=128, d=0.05, dt_over_dz=0.45, gamma=1000.0, z_cell=64.0, x_cell=64.0,
                    shape=1, solver="yee"):
    """One macro-electron (q = -1, weight 1) at rest frame gamma along +z; 2D vacuum grid."""
    u = np.zeros((3, 1), np.float32)
    u[0, 0] = math.sqrt(gamma * gamma - 1.0)
    cz, oz = _split(np.array([z_cell]))
    cx, ox = _split(np.array([x_cell]))
    sp = species(cz, cx, [0], np.stack([oz, ox]), u, -1.0, 1.0, 1.0)
    grid = dict(ndim=2, nz=nz, nx=nx, ny=1, dz=d, dx=d, dy=d, dt=dt_over_dz * d, shape=shape, solver=solver)
    return grid, [sp]


def quiet_plasma(ndim, nz, nx, ny, ppc, d, z_range=None, density=1.0):
    """Cold uniform plasma, ppc = (pz, px[, py]) particles per cell at sub-cell centres."""
    pz, px = ppc[0], ppc[1]
    py = ppc[2] if ndim == 3 else 1
    z0, z1 = (0, nz) if z_range is None else z_range
    ks = np.arange(ny if ndim == 3 else 1)
    js = np.arange(nx)
    is_ = np.arange(z0, z1)
    K, Jx, I, A, Bb, Cc = np.meshgrid(ks, js, is_, np.arange(pz), np.arange(px), np.arange(py), indexing="ij")
    iz, ix, iy = I.ravel(), Jx.ravel(), K.ravel()
    oz = ((A.ravel() + 0.5) / pz).astype(np.float32)
    ox = ((Bb.ravel() + 0.5) / px).astype(np.float32)
    offs = [oz, ox]
    if ndim == 3:
        offs.append(((Cc.ravel() + 0.5) / py).astype(np.float32))
    n = len(iz)
    V = d[0] * d[1] * (d[2] if ndim == 3 else 1.0)
    w = density * V / (pz * px * py)
    return species(iz, ix, iy, np.stack(offs), np.zeros((3, n), np.float32), -1.0, 1.0, w)


def gaussian_beam(ndim, nz, nx, ny, d, n, sigma_z, sigma_r, gamma, spread, peak_density, z_centre,
                  seed, trunc=4.0):
    """Bi- (2D) or tri- (3D) Gaussian electron beam truncated at trunc sigma, centred on axis.

    gamma is uniform on gamma (1 +- spread/2); momenta along +z.  The weight gives a peak
    density of peak_density for the untruncated Gaussian."""
    rng = np.random.default_rng(seed)
    dims = 2 if ndim == 2 else 3

    def tnorm(size, sig):
        out = np.empty(0)
        while len(out) < size:
            x = rng.normal(0.0, sig, 2 * size)
            out = np.concatenate([out, x[np.abs(x) < trunc * sig]])
        return out[:size]

    z = z_centre + tnorm(n, sigma_z)
    x = nx * d[1] / 2 + tnorm(n, sigma_r)
    cz, oz = _split(z / d[0])
    cx, ox = _split(x / d[1])
    cx = np.mod(cx, nx)                      # periodic transverse axes
    offs = [oz, ox]
    cy = np.zeros(n, np.int64)
    if dims == 3:
        y = ny * d[2] / 2 + tnorm(n, sigma_r)
        cy, oy = _split(y / d[2])
        cy = np.mod(cy, ny)
        offs.append(oy)
    g = gamma * (1.0 + spread * (rng.uniform(size=n) - 0.5))
    u = np.zeros((3, n), np.float32)
    u[0] = np.sqrt(g * g - 1.0)
    if dims == 2:
        total = peak_density * 2 * math.pi * sigma_z * sigma_r * math.erf(trunc / math.sqrt(2)) ** 2
    else:
        total = peak_density * (2 * math.pi) ** 1.5 * sigma_z * sigma_r ** 2 * math.erf(trunc / math.sqrt(2)) ** 3
    return species(cz, cx, cy, np.stack(offs), u, -1.0, 1.0, total / n)


def beam_plasma(ndim=2, nz=2048, nx=512, ny=1, d=(0.02, 0.02, 0.02), dt=DT_BEAM_2D, n_beam=1_000_000,
                sigma_z=0.5, sigma_r=0.2, gamma=2e4, spread=0.02, ppc=(2, 2, 1), behind_front=3.0,
                peak_density=100.0, solver="custom", shape=2, seed=1002):
    """Relativistic beam in a uniform cold plasma (n_p = 1) with a moving window at c.

    Defaults: the 2D 2048 x 512 run (dz = dx = 0.02, 4 ppc, 1e6 beam particles, sigma_z = 0.5,
    sigma_x = 0.2, gamma = 2e4 with 2% spread, peak beam density 100 n_p)."""
    plasma = quiet_plasma(ndim, nz, nx, ny, ppc, d)
    beam = gaussian_beam(ndim, nz, nx, ny, d, n_beam, sigma_z, sigma_r, gamma, spread, peak_density,
                         nz * d[0] - behind_front, seed)
    grid = dict(ndim=ndim, nz=nz, nx=nx, ny=ny if ndim == 3 else 1, dz=d[0], dx=d[1], dy=d[2], dt=dt,
                shape=shape, solver=solver, moving_window=True, inject_species=0, inject_ppc=tuple(ppc),
                rho_bg=1.0)
    return grid, [plasma, beam]


def beam_plasma_3d(nz=512, nx=256, ny=256, n_beam=4_000_000, seed=1003, **kw):
    """The 3D 512 x 256 x 256 run: dz = 0.02, dx = dy = 0.05, 2 ppc, sigma_r = 0.1, gamma = 2e4."""
    args = dict(ndim=3, nz=nz, nx=nx, ny=ny, d=(0.02, 0.05, 0.05), dt=DT_BEAM_3D, n_beam=n_beam,
                sigma_z=0.5, sigma_r=0.1, gamma=2e4, spread=0.0, ppc=(2, 1, 1), seed=seed)
    args.update(kw)
    return beam_plasma(**args)


def random_particles(ndim, nz, nx, ny, n, seed, u_scale=1.0, u_drift=(0.0, 0.0, 0.0), margin=3, q=-1.0, m=1.0,
                     w=0.05):
    """Uniformly scattered particles with Gaussian momenta (unit tests of the kernels)."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(margin, nz - margin, n)
    x = rng.uniform(0, nx, n)
    cz, oz = _split(z)
    cx, ox = _split(x)
    cx = np.mod(cx, nx)
    offs = [oz, ox]
    cy = np.zeros(n, np.int64)
    if ndim == 3:
        cy, oy = _split(rng.uniform(0, ny, n))
        cy = np.mod(cy, ny)
        offs.append(oy)
    u = (rng.normal(size=(3, n)) * u_scale + np.asarray(u_drift)[:, None]).astype(np.float32)
    return species(cz, cx, cy, np.stack(offs), u, q, m, w)


def rigid_line(nz=1024, nx=256, d=0.05, dt_over_dz=0.25, gamma=1e4, n=64, z_cell=None):
    """A transverse line of n macro-electrons, one per x cell in the central n cells, at one z."""
    zc = nz // 4 if z_cell is None else z_cell
    cz = np.full(n, zc, np.int64)
    cx = np.arange(nx // 2 - n // 2, nx // 2 - n // 2 + n, dtype=np.int64)
    oz = np.full(n, 0.5, np.float32)
    ox = np.full(n, 0.5, np.float32)
    u = np.zeros((3, n), np.float32)
    u[0] = math.sqrt(gamma * gamma - 1.0)
    grid = dict(ndim=2, nz=nz, nx=nx, ny=1, dz=d, dx=d, dy=d, dt=dt_over_dz * d, shape=1)
    return grid, [species(cz, cx, np.zeros(n, np.int64), np.stack([oz, ox]), u, -1.0, 1.0, 1.0 / n)]


def quiet_plasma_sample(ndim, nz, nx, ny, ppc, d, frac, seed, density=1.0):
    """A random fraction of the quiet-start plasma of quiet_plasma() (same lattice, same weight),
    drawn without building the whole lattice: lattice indices in the order (k, j, i, a, b, c)."""
    pz, px = ppc[0], ppc[1]
    py = ppc[2] if ndim == 3 else 1
    nyy = ny if ndim == 3 else 1
    total = nyy * nx * nz * pz * px * py
    rng = np.random.default_rng(seed)
    idx = np.unique(rng.integers(0, total, max(int(frac * total), 1)))
    r = idx
    c, r = r % py, r // py
    b, r = r % px, r // px
    a, r = r % pz, r // pz
    i, r = r % nz, r // nz
    j, k = r % nx, r // nx
    offs = [((a + 0.5) / pz).astype(np.float32), ((b + 0.5) / px).astype(np.float32)]
    if ndim == 3:
        offs.append(((c + 0.5) / py).astype(np.float32))
    n = len(idx)
    V = d[0] * d[1] * (d[2] if ndim == 3 else 1.0)
    w = density * V / (pz * px * py)
    return species(i, j, k, np.stack(offs), np.zeros((3, n), np.float32), -1.0, 1.0, w), total


def beam_plasma_3d_sample(frac, seed=7):
    """A random fraction of the particles of beam_plasma_3d() (plasma and beam alike), with the
    full run's grid: for timing the FP64 oracle on a bounded piece of the 3D workload."""
    grid, _ = beam_plasma_3d(nz=8, nx=8, ny=8, n_beam=8)         # grid parameters only
    nz, nx, ny = 512, 256, 256
    grid.update(nz=nz, nx=nx, ny=ny)
    d = (grid["dz"], grid["dx"], grid["dy"])
    plasma, n_plasma = quiet_plasma_sample(3, nz, nx, ny, grid["inject_ppc"], d, frac, seed)
    beam = gaussian_beam(3, nz, nx, ny, d, 4_000_000, 0.5, 0.1, 2e4, 0.0, 100.0, nz * d[0] - 3.0, 1003)
    keep = np.random.default_rng(seed + 1).random(len(beam["iz"])) < frac
    beam = species(beam["iz"][keep], beam["ix"][keep], beam["iy"][keep], beam["off"][:, keep], beam["u"][:, keep],
                   beam["q"], beam["m"], beam["w"])
    return grid, [plasma, beam], n_plasma + 4_000_000


# customised-stencil stability fixed point at r = 1: kappa = dz/dt at which dt equals the limit
# of the stencil fitted at that same kappa (Appendix C fit)
KAPPA_CFL_CUSTOM_2D = 1.632488686516034


def batched_vacuum_scan(n=256, seed=4000):
    """Instance parameters of the batched vacuum scan: n independent 2D single-particle runs with
    nz ~ U{128..1024}, nx ~ U{64..256}, log10 gamma ~ U[1, 5], dt = U[0.3, 0.99] x the instance's
    own stability limit, Yee or customised (M = 16) by a fair coin, dz = dx = 0.05, linear shape.
    Returns [(grid dict, gamma)]."""
    rng = np.random.default_rng(seed)
    d = 0.05
    out = []
    for _ in range(n):
        nz = int(rng.integers(128, 1025))
        nx = int(rng.integers(64, 257))
        gamma = 10 ** rng.uniform(1, 5)
        frac = rng.uniform(0.3, 0.99)
        custom = bool(rng.integers(0, 2))
        dt = frac * (d / KAPPA_CFL_CUSTOM_2D if custom else d / math.sqrt(2))
        grid = dict(ndim=2, nz=nz, nx=nx, ny=1, dz=d, dx=d, dy=d, dt=dt, shape=1,
                    solver="custom" if custom else "yee", M=16)
        out.append((grid, gamma))
    return out
