"""GPU parity of the split axial operators ([k]_E1 != [k]_B1, which Sec. 3 allows; pinned in
tests/test_oracle_split.py) against the FP64 oracle: every field-advance tile variant in 2D and
3D, whole steps with particles and the Sec. 3 correction from the B-side set, Gauss's law with the
B-side d-, a batch with split and symmetric instances, and the refusals (adjoint, no explicit
E-side set, a sign-changing symbol product).  Tolerance 1e-5 as in test_gpu_parity.py."""
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
from paper_1910_13529_gb300.runtime import Batch, Simulation  # noqa: E402

from parity_util import TABLE1, field_error, field_rel_l2, gpu_sim, oracle_sim, particle_errors  # noqa: E402

TOL = 1e-5
FIT8 = fit.fit_coefficients(3.0, M=8)
# (E-side, B-side): Yee E side with a fitted B side, the reverse, two unrelated stencils (M = 16)
PAIRS = {
    "yeeE-fitB": ([1.0], list(FIT8)),
    "fitE-yeeB": (list(FIT8), [1.0]),
    "table1E-fitB": (list(TABLE1), list(FIT8)),
}


def grid_of(ndim, nz, nx, ny, pair, shape=1, frac=0.9, d=(0.5, 0.4, 0.45), **kw):
    CE, CB = PAIRS[pair]
    dt = frac * fit.cfl_dt(d[0], [d[1]] + ([d[2]] if ndim == 3 else []), CE, Cb=CB)
    g = dict(ndim=ndim, nz=nz, nx=nx, ny=ny, dz=d[0], dx=d[1], dy=d[2], dt=dt, solver="custom", shape=shape,
             coef_b=CB)
    g.update(kw)
    return g, CE


@pytest.mark.parametrize("nd,nz,nx,ny", [(2, 203, 11, 1), (3, 101, 6, 5)])
@pytest.mark.parametrize("pair", sorted(PAIRS))
def test_every_tile_variant_matches_oracle(nd, nz, nx, ny, pair):
    grid, CE = grid_of(nd, nz, nx, ny, pair)
    osim = oracle_sim(grid, [], coef=CE)
    rng = np.random.default_rng(nz + len(pair))
    init = [rng.normal(size=a.shape).astype(np.float32) for a in (osim.E, osim.B, osim.J)]
    osim.E[:], osim.B[:], osim.J[:] = init
    for _ in range(4):
        oc.field_advance(osim.g, osim.E, osim.B, osim.J)
    sim = gpu_sim(grid, [], coef=CE)
    Cb, split = P.pic_get_coefficients_b(sim.h)
    assert split and np.allclose(Cb[: len(PAIRS[pair][1])], PAIRS[pair][1])
    nv = len(P.pic_get_tuning(sim.h)[1])
    sim.close()
    for v in range(nv):
        sim = gpu_sim(grid, [], coef=CE)
        P.pic_set_tuning(sim.h, v)
        for a, x in zip((sim.E, sim.B, sim.J), init):
            a.copy_(torch.from_numpy(x))
        for _ in range(4):
            sim.field_advance()
        assert field_error(sim, osim) < TOL, v
        sim.close()


@pytest.mark.parametrize("nd,shape", [(2, 2), (3, 1)])
@pytest.mark.parametrize("pair", sorted(PAIRS))
def test_steps_match_oracle_and_keep_gauss(nd, shape, pair):
    nz, nx, ny = (200, 16, 1) if nd == 2 else (96, 10, 8)
    grid, CE = grid_of(nd, nz, nx, ny, pair, shape=shape, rho_bg=0.0)
    sps = [wl.random_particles(nd, nz, nx, ny, 3000, seed=41, u_scale=1.0, u_drift=(3.0, 0, 0), margin=35)]
    sim = gpu_sim(grid, sps, coef=CE)
    osim = oracle_sim(grid, sps, coef=CE)
    G0 = sim.gauss()
    rmax = sim.rho().abs().max().item()
    n = 15
    sim.step(n)
    for _ in range(n):
        osim.step()
    assert field_error(sim, osim) < TOL
    assert field_rel_l2(sim, osim) < TOL
    dx, du = particle_errors(sim, osim, 0, nd)
    assert dx < TOL and du < TOL
    G = sim.gauss()
    m = 16 + 24 + 2
    assert (G - G0)[..., m:-m].abs().max().item() < 1e-5 * rmax
    sim.close()


def test_batch_with_split_and_symmetric_instances():
    inst = []
    for i, (nz, nx) in enumerate(((150, 20), (203, 17), (96, 33))):
        d = 0.05
        if i == 1:
            grid = dict(ndim=2, nz=nz, nx=nx, ny=1, dz=d, dx=d, dy=d, dt=0.4 * d, solver="custom", shape=2)
            C = FIT8
        else:
            grid, C = grid_of(2, nz, nx, 1, "yeeE-fitB" if i == 0 else "table1E-fitB", shape=1 + i % 2,
                              d=(d, d, d))
        sp = wl.random_particles(2, nz, nx, 1, 300, seed=4200 + i, u_scale=1.0, u_drift=(2.0, 0, 0), margin=nz // 4)
        inst.append((grid, [sp], C))
    cfgs = []
    for grid, sps, C in inst:
        c = {k: grid[k] for k in ("ndim", "nz", "nx", "dz", "dx", "dt", "shape", "solver")}
        c["coef"] = C
        if grid.get("coef_b") is not None:
            c["coef_b"] = grid["coef_b"]
        cfgs.append(c)
    batch = Batch(cfgs)
    for sim, (grid, sps, C) in zip(batch.instances, inst):
        sp = sps[0]
        sim.add_species(0, sp["iz"], sp["ix"], sp["iy"], sp["off"], sp["u"], sp["q"], sp["m"], sp["w"],
                        ids=sp["ids"])
    nsteps = 11
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


def test_symmetric_handles_report_one_set():
    sim = gpu_sim(dict(ndim=2, nz=64, nx=8, ny=1, dz=0.5, dx=0.4, dy=0.4, dt=0.05, solver="custom", shape=1),
                  [], coef=FIT8)
    Cb, split = P.pic_get_coefficients_b(sim.h)
    C, _ = P.pic_get_coefficients(sim.h)
    assert not split and np.array_equal(Cb[: len(C)], C)
    sim.close()


def test_refusals():
    grid, CE = grid_of(2, 64, 8, 1, "yeeE-fitB")
    sim = gpu_sim(grid, [], coef=CE)
    z = torch.zeros_like(sim.E)
    grad = torch.zeros(16, dtype=torch.float64, device=sim.device)
    with pytest.raises(P.PicError) as ei:
        P.pic_adjoint_step(sim.h, z.data_ptr(), z.data_ptr(), z.data_ptr(), z.clone().data_ptr(),
                           z.clone().data_ptr(), grad.data_ptr(), sim.stream)
    assert ei.value.status == P.PIC_ERR_ARG
    sim.close()
    # coef_b without an explicit E-side set, and a product of symbols that changes sign
    for kw in (dict(coef=None), dict(coef_b=[-1.0])):
        g = dict(grid, **{k: v for k, v in kw.items() if k == "coef_b"})
        with pytest.raises(P.PicError):
            Simulation(device="cuda:0", ndim=2, nz=64, nx=8, dz=0.5, dx=0.4, dt=0.05, solver="custom",
                       coef=kw.get("coef", CE), coef_b=g["coef_b"])


def test_product_matched_pair_transverse_force():
    """The product-matched pair of Sec. 3 (Yee E side, B side fitted by the library to
    [k1]_t^2 / [k]_Yee, pic_fit_coefficients_b) on a beta -> 1 particle (gamma = 1e7, kappa = 4,
    r = 1, quadratic shape, moving window), 1600 steps against the FP64 oracle; the B3~/E2~ ratio
    measured on the GPU fields follows Eq. EM ([w]_t / [k]_B1, about -3.6% from 1 at k1 dz >= 0.7)."""
    from tforce_util import band_means, measured_ratio, predicted_ratio

    kappa, nz, nx, steps = 4.0, 384, 48, 1600
    CB = P.pic_fit_coefficients_b(kappa, [1.0], M=16)
    assert np.abs(CB - fit.fit_coefficients(kappa, M=16, CE=[1.0])).max() < 1e-6
    CE = np.zeros(16)
    CE[0] = 1.0
    sp = wl.species([nz - 130], [nx // 2], [0], np.array([[0.0], [0.5]], np.float32),
                    np.array([[1e7], [0.0], [0.0]], np.float32), 1.0, 1.0, 1.0)
    grid = dict(ndim=2, nz=nz, nx=nx, ny=1, dz=1.0, dx=1.0, dy=1.0, dt=1.0 / kappa, solver="custom", shape=2,
                coef_b=list(CB), moving_window=True)
    sim = gpu_sim(grid, [sp], coef=CE)
    osim = oracle_sim(grid, [sp], coef=CE)
    sim.step(steps)
    prev = oc.set_threads(4)
    try:
        for _ in range(steps):
            osim.step()
    finally:
        oc.set_threads(1)
    assert field_error(sim, osim) < TOL
    g = osim.g
    E = sim.E.double().cpu().numpy()
    B = sim.B.double().cpu().numpy()
    oc.faraday_half(g, E, B)
    step, shifts, pend = sim.state()
    zp = osim.species[0].xi[0, 0]
    j0 = nx // 2
    ks, r = measured_ratio(E[1, 0, j0 + 3, :], B[2, 0, j0 + 3, :], zp, kappa)
    m, p = band_means(ks, r, predicted_ratio(ks, kappa, CB))
    assert abs(m - p) < 5e-3 and m < -0.03, (m, p)
    sim.close()
