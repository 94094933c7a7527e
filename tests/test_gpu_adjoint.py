"""Adjoint of the field step (pic_adjoint_step) and the coefficient gradient of a rigid-beam
field-energy loss.

* Transpose test at the 1024 x 256 stencil-tuning size: <l, A x> = <A^T l, x> for random x, l.
* Gradient dL/dC_l (FP32 forward and adjoint, checkpoints) against FP64 central finite
  differences of the oracle on a reduced rigid-line problem; 1e-4 relative."""
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
from paper_1910_13529_gb300.runtime import Simulation, StencilLoss, StencilLossFn  # noqa: E402

C4 = fit.fit_coefficients(4.0, M=4)


def test_adjoint_is_the_transpose_at_full_size():
    nz, nx, d = 1024, 256, 0.05
    sim = Simulation(device="cuda:0", ndim=2, nz=nz, nx=nx, dz=d, dx=d, dt=d / 4, solver="custom", coef=C4)
    gen = torch.Generator(device="cuda:0").manual_seed(5)
    xE = torch.randn(sim.E.shape, device="cuda:0", generator=gen)
    xB = torch.randn(sim.B.shape, device="cuda:0", generator=gen)
    lE = torch.randn(sim.E.shape, device="cuda:0", generator=gen)
    lB = torch.randn(sim.B.shape, device="cuda:0", generator=gen)
    sim.E.copy_(xE)
    sim.B.copy_(xB)
    sim.J.zero_()
    sim.field_advance()                                   # y = A x
    lhs = float((lE.double() * sim.E.double()).sum() + (lB.double() * sim.B.double()).sum())
    aE, aB = lE.clone(), lB.clone()
    grad = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    J0 = torch.zeros_like(sim.J)
    P.pic_adjoint_step(sim.h, xE.data_ptr(), xB.data_ptr(), J0.data_ptr(), aE.data_ptr(), aB.data_ptr(),
                       grad.data_ptr(), sim.stream)
    torch.cuda.synchronize()
    rhs = float((aE.double() * xE.double()).sum() + (aB.double() * xB.double()).sum())
    scale = float(lE.double().norm() * xE.double().norm())
    assert abs(lhs - rhs) < 1e-5 * scale
    sim.close()


def _problem(nsteps=60):
    grid, sps = wl.rigid_line(nz=160, nx=48, d=0.05, dt_over_dz=0.25, gamma=1e4, n=16, z_cell=40)
    return grid, sps, nsteps


def _oracle_loss(C, grid, sps, nsteps, behind=2, filt=False):
    C = np.asarray(C, dtype=np.float64)
    g = oc.Grid(2, grid["nz"], grid["nx"], 1, grid["dz"], grid["dx"], grid["dy"], grid["dt"], C=C, shape=1)
    species = [oc.Species(wl.xi_of(sp, 2), sp["u"].T.astype(np.float64), sp["q"], StencilLoss.RIGID_MASS, sp["w"])
               for sp in sps]
    sim = oc.Sim(g, species, h=fit.correction_kernel(C, hlen=40), filt=filt)
    for _ in range(nsteps):
        sim.step()
    zc = max(int(np.floor(min(s.xi[:, 0].min() for s in sim.species))) - behind, 0)
    dV = grid["dz"] * grid["dx"]
    return 0.5 * (np.sum(sim.E[..., :zc] ** 2) + np.sum(sim.B[..., :zc] ** 2)) * dV


def test_coefficient_gradient_matches_fp64_finite_differences():
    grid, sps, nsteps = _problem()
    problem = StencilLoss(grid, sps, nsteps=nsteps, every=10)
    L, g = problem.loss_and_grad(C4)
    L64 = _oracle_loss(C4, grid, sps, nsteps)
    assert L == pytest.approx(L64, rel=1e-5)
    fd = np.zeros(4)
    for l in range(4):
        eps = 1e-5 * max(abs(C4[l]), 1e-3)
        Cp, Cm = C4.copy(), C4.copy()
        Cp[l] += eps
        Cm[l] -= eps
        fd[l] = (_oracle_loss(Cp, grid, sps, nsteps) - _oracle_loss(Cm, grid, sps, nsteps)) / (2 * eps)
    assert np.max(np.abs(g - fd)) < 1e-4 * np.max(np.abs(fd))


def test_coefficient_gradient_with_the_current_filter():
    """The filter precedes the correction and does not depend on C: the same adjoint, checked
    against FP64 central differences of the oracle run with the filter."""
    grid, sps, nsteps = _problem(nsteps=40)
    grid = dict(grid, current_filter=True)
    problem = StencilLoss(grid, sps, nsteps=nsteps, every=10)
    L, g = problem.loss_and_grad(C4)
    assert L == pytest.approx(_oracle_loss(C4, grid, sps, nsteps, filt=True), rel=1e-5)
    assert L != pytest.approx(_oracle_loss(C4, grid, sps, nsteps), rel=1e-3)
    fd = np.zeros(4)
    for l in range(4):
        eps = 1e-5 * max(abs(C4[l]), 1e-3)
        Cp, Cm = C4.copy(), C4.copy()
        Cp[l] += eps
        Cm[l] -= eps
        fd[l] = (_oracle_loss(Cp, grid, sps, nsteps, filt=True) - _oracle_loss(Cm, grid, sps, nsteps, filt=True)) / (2 * eps)
    assert np.max(np.abs(g - fd)) < 1e-4 * np.max(np.abs(fd))


def test_autograd_wrapper_and_descent_step():
    grid, sps, nsteps = _problem(40)
    problem = StencilLoss(grid, sps, nsteps=nsteps, every=10)
    C = torch.tensor(C4, dtype=torch.float64, requires_grad=True)
    L = StencilLossFn.apply(C, problem)
    L.backward()
    g = C.grad.numpy()
    assert np.all(np.isfinite(g)) and np.max(np.abs(g)) > 0
    # one projected descent step (keeping sum (2l-1) C_l = 1) lowers the loss
    w = 2 * np.arange(1, 5) - 1.0
    gp = g - w * (w @ g) / (w @ w)
    step = 0.02 * np.max(np.abs(C4)) / np.max(np.abs(gp))
    C1 = C4 - step * gp
    assert abs(w @ C1 - 1.0) < 1e-12
    assert fit.cfl_dt(grid["dz"], [grid["dx"]], C1) > grid["dt"]
    assert problem.loss(C1) < float(L.detach())


def _golden():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "stencil_gradient_1024x256.txt")
    C, g, L = [], [], None
    for line in open(path):
        if line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] == "loss":
            L = float(parts[1])
        else:
            C.append(float(parts[1]))
            g.append(float(parts[3]))
    return np.array(C), np.array(g), L


def test_full_size_gradient_matches_stored_fp64_finite_differences():
    """1024 x 256, 64 rigid electrons at gamma = 1e4, 500 steps, checkpoints every 50 steps."""
    C, g_ref, L_ref = _golden()
    grid, sps = wl.rigid_line()
    problem = StencilLoss(grid, sps, nsteps=500, every=50)
    L, g = problem.loss_and_grad(C)
    assert L == pytest.approx(L_ref, rel=1e-5)
    assert np.max(np.abs(g - g_ref)) < 1e-4 * np.max(np.abs(g_ref))


def test_stencil_tuning_lowers_the_wake_energy():
    """Projected descent with the adjoint gradient (tuning.tune_coefficients) from the Appendix C
    fit: the loss falls at every accepted step, the consistency constraint stays exact, and the
    FP64 oracle's loss at the tuned coefficients is lower than at the start."""
    from paper_1910_13529_gb300.tuning import tune_coefficients
    grid, sps, nsteps = _problem(60)
    problem = StencilLoss(grid, sps, nsteps=nsteps, every=10)
    hist = tune_coefficients(problem, C4, iters=6)
    losses = hist["loss"]
    assert len(losses) >= 3 and all(b < a for a, b in zip(losses, losses[1:]))
    w = 2 * np.arange(1, 5) - 1.0
    assert abs(w @ hist["C_final"] - 1.0) < 1e-12
    assert fit.cfl_dt(grid["dz"], [grid["dx"]], hist["C_final"]) > grid["dt"]
    # the tuned coefficients lower the FP64 oracle's loss too; the FP32 loss of a smaller residual
    # energy agrees with it to 1e-4 (the fields themselves to 1e-5 of their maximum)
    L_or0 = _oracle_loss(C4, grid, sps, nsteps)
    L_or1 = _oracle_loss(hist["C_final"], grid, sps, nsteps)
    assert L_or1 < L_or0
    assert hist["loss_final"] == pytest.approx(L_or1, rel=1e-4)
