"""Tuning of the axial stencil coefficients with the hand-written adjoint (Sec. 3, Appendix C).

The loss is the field energy left behind a rigidly moving beam (runtime.StencilLoss: the spurious
space-charge and Cerenkov fields of the finite-difference solver); its gradient with respect to
C_1..C_M comes from pic_adjoint_step.  The descent keeps the Appendix C consistency constraint
sum_l (2l - 1) C_l = 1 (a first-order accurate operator) by projecting each gradient onto that
plane, and accepts a step only if the loss decreases and dt stays below the leapfrog stability
limit of the new coefficients (pic_cfl_dt); otherwise the step is halved.  Host-side optimizer
bookkeeping only: every loss and gradient evaluation runs in the CUDA kernels."""
import numpy as np

from . import pic_cfl_dt


def project(g, M):
    """Component of g in the plane sum (2l - 1) x_l = 0."""
    w = 2.0 * np.arange(1, M + 1) - 1.0
    return g - w * (w @ g) / (w @ w)


def tune_coefficients(problem, C0, iters=20, rel_step=0.05, min_rel_step=1e-6):
    """Projected gradient descent with step halving.  problem: runtime.StencilLoss.  The first
    trial step moves C by rel_step of max |C| along the projected gradient; an accepted step
    grows the next trial by 1.5.  Returns a dict with the coefficient and loss history."""
    grid = problem.grid
    C = np.asarray(C0, dtype=np.float64).copy()
    M = len(C)
    w = 2.0 * np.arange(1, M + 1) - 1.0
    if abs(w @ C - 1.0) > 1e-9:
        raise ValueError("C0 must satisfy sum (2l - 1) C_l = 1")
    dperp = (grid["dx"],) if grid["ndim"] == 2 else (grid["dx"], grid["dy"])
    L, g = problem.loss_and_grad(C)
    hist = {"loss": [L], "C": [C.copy()], "grad_norm": [float(np.linalg.norm(project(g, M)))], "evals": 1}
    step = rel_step * np.max(np.abs(C))
    for _ in range(iters):
        gp = project(g, M)
        nrm = np.linalg.norm(gp)
        if nrm == 0.0:
            break
        accepted = False
        while step > min_rel_step * np.max(np.abs(C)):
            trial = C - step * gp / nrm
            trial += w * (1.0 - w @ trial) / (w @ w)          # stay on the plane to round-off
            dt_max = pic_cfl_dt(grid["ndim"], grid["dz"], grid["dx"], grid.get("dy", grid["dx"]), trial)
            if grid["dt"] < dt_max:
                Lt, gt = problem.loss_and_grad(trial)
                hist["evals"] += 1
                if Lt < L:
                    C, L, g = trial, Lt, gt
                    accepted = True
                    step *= 1.5
                    break
            step *= 0.5
        if not accepted:
            break
        hist["loss"].append(L)
        hist["C"].append(C.copy())
        hist["grad_norm"].append(float(np.linalg.norm(project(g, M))))
    hist["C_final"] = C
    hist["loss_final"] = L
    return hist
