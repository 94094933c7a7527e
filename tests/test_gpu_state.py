"""Run state on the GPU: checkpoint/resume reproduces an uninterrupted run, and a particle
capacity overflow during injection is reported as PIC_ERR_CAPACITY (a device status word read
on the host, no fault)."""
import os
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1910_13529_gb300 as P  # noqa: E402
from oracle import fit  # noqa: E402
from paper_1910_13529_gb300 import workloads as wl  # noqa: E402

from parity_util import gpu_particles, gpu_sim  # noqa: E402


def _case():
    grid, sps = wl.beam_plasma(ndim=2, nz=160, nx=24, n_beam=2000, sigma_z=0.25, sigma_r=0.06,
                               behind_front=1.5, solver="custom")
    return grid, sps, fit.fit_coefficients(grid["dz"] / grid["dt"])


def test_checkpoint_resume_matches_uninterrupted_run():
    grid, sps, C = _case()
    a = gpu_sim(grid, sps, coef=C, cap_extra=20000)
    a.step(30)
    b = gpu_sim(grid, sps, coef=C, cap_extra=20000)
    b.step(15)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ckpt.pt")
        b.save(path)
        b.close()
        c = gpu_sim(grid, [], coef=C)
        c.species = {}
        c.load(path)
    c.step(15)
    assert a.state() == c.state()
    scale = max(a.E.abs().max().item(), a.B.abs().max().item())
    assert (a.E - c.E).abs().max().item() < 1e-5 * scale
    assert (a.B - c.B).abs().max().item() < 1e-5 * scale
    for s in range(2):
        ia, xa, ua = gpu_particles(a, s, 2, a.state()[2])
        ic, xc, uc = gpu_particles(c, s, 2, c.state()[2])
        assert np.array_equal(ia, ic) and np.abs(xa - xc).max() < 1e-5
    a.close()
    c.close()


def test_capacity_overflow_is_reported():
    grid, sps, C = _case()
    sim = gpu_sim(grid, sps, coef=C, cap_extra=10)      # the first injected column does not fit
    sim.step(4)
    with pytest.raises(P.PicError) as ei:
        sim.diag()
    assert ei.value.status == P.PIC_ERR_CAPACITY
    with pytest.raises(P.PicError):
        sim.sync()
    sim.close()
