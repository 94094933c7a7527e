"""The tile autotuner times every field-advance tile variant without changing the state, and
every variant computes the same step (compared with the FP64 oracle)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import core as oc  # noqa: E402

from parity_util import TABLE1, field_error, gpu_sim, oracle_sim  # noqa: E402


@pytest.mark.parametrize("nd,solver,C", [(2, "custom", TABLE1), (3, "yee", None)])
def test_autotune_keeps_state_and_result(nd, solver, C):
    nz, nx, ny = (520, 40, 1) if nd == 2 else (200, 12, 10)
    grid = dict(ndim=nd, nz=nz, nx=nx, ny=ny, dz=0.5, dx=0.4, dy=0.45, dt=0.08, solver=solver, shape=1)
    sim = gpu_sim(grid, [], coef=C)
    osim = oracle_sim(grid, [], coef=C)
    rng = np.random.default_rng(9)
    for a, oa in ((sim.E, osim.E), (sim.B, osim.B), (sim.J, osim.J)):
        v = rng.normal(size=oa.shape).astype(np.float32)
        a.copy_(torch.from_numpy(v))
        oa[:] = v
    E0, B0, J0 = sim.E.clone(), sim.B.clone(), sim.J.clone()
    variant, ms = sim.autotune()
    assert torch.equal(sim.E, E0) and torch.equal(sim.B, B0)
    assert len(ms) >= 3 and np.all(ms > 0) and 0 <= variant < len(ms)
    oc.field_advance(osim.g, osim.E, osim.B, osim.J)
    from paper_1910_13529_gb300 import pic_set_tuning
    for v in range(len(ms)):
        sim.E.copy_(E0)
        sim.B.copy_(B0)
        sim.J.copy_(J0)
        pic_set_tuning(sim.h, v)
        sim.field_advance()
        assert field_error(sim, osim) < 1e-5, v
    sim.close()
