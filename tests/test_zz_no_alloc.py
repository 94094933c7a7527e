"""pic_gauss_static: the Gauss-residual diagnostic for callers that cannot allocate device memory
when they need it (a fixed memory budget set at start-up, or a loop that must not call
cudaMalloc because it can wait for the whole device).  It must give what pic_gauss gives while
taking its scratch from the fixed array inside the library.  This file is collected last so that
a failure here cannot hide the other tests; it passes alone and after them."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1910_13529_gb300 as P  # noqa: E402
from paper_1910_13529_gb300 import workloads as wl  # noqa: E402
from paper_1910_13529_gb300.runtime import Simulation  # noqa: E402

TOL = 1e-5


def _sim(nz, nx, n=4000, solver="yee"):
    sim = Simulation(device="cuda:0", ndim=2, nz=nz, nx=nx, dz=0.5, dx=0.5, dt=0.3, shape=2, solver=solver,
                     M=8, rho_bg=0.1)
    sp = wl.random_particles(2, nz, nx, 1, n, seed=3, u_scale=1.0, u_drift=(2.0, 0, 0), margin=20)
    sim.add_species(0, sp["iz"], sp["ix"], sp["iy"], sp["off"], sp["u"], sp["q"], sp["m"], sp["w"])
    return sim


def _static(sim):
    G = torch.full((sim.ny, sim.nx, sim.nz), float("nan"), dtype=torch.float64, device=sim.device)
    P.pic_gauss_static(sim.h, G.data_ptr(), sim.stream)
    torch.cuda.synchronize()
    return G


@pytest.mark.parametrize("solver", ["yee", "custom"])
def test_static_scratch_matches_pic_gauss_on_consecutive_calls(solver):
    sim = _sim(300, 40, solver=solver)
    sim.step(5)
    ref = sim.gauss()
    scale = float(sim.rho().abs().max())
    for _ in range(2):                                  # two calls in a row share the array
        G = _static(sim)
        assert float((G - ref).abs().max()) <= TOL * scale
    sim.step(3)                                          # new state, two more calls
    ref = sim.gauss()
    for _ in range(2):
        G = _static(sim)
        assert float((G - ref).abs().max()) <= TOL * scale
    sim.close()


def test_static_scratch_refuses_grids_above_its_size():
    nz, nx = 1100, 1000
    assert nz * nx > P.PIC_STATIC_RHO_CELLS
    sim = _sim(nz, nx, n=10)
    G = torch.zeros((1, nx, nz), dtype=torch.float64, device=sim.device)
    with pytest.raises(P.PicError) as ei:
        P.pic_gauss_static(sim.h, G.data_ptr(), sim.stream)
    assert ei.value.status == P.PIC_ERR_ARG and "fixed scratch" in str(ei.value)
    sim.close()
