"""The GPU's finite-difference step against the paper's per-mode fields of a drifting charge
(Sec. 2.1, Eq. EM; the same construction as tests/test_oracle_em.py): one step carries them to
e^{-i w dt} times themselves, on the cells more than 3 M + 2 from the open z ends, for the Yee
solver, the Appendix C stencil and the split pair."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import core as oc  # noqa: E402

from parity_util import gpu_sim  # noqa: E402
from test_oracle_em import _sets, em_mode  # noqa: E402


@pytest.mark.parametrize("name", ["yee", "appendix_c", "pair"])
@pytest.mark.parametrize("beta", [1.0, 0.9])
def test_gpu_step_carries_the_eq_em_fields(name, beta):
    dz = dx = 1.0
    dt = 0.25
    CE, CB = _sets(name, dz, dt)
    g = oc.Grid(2, 256, 16, 1, dz, dx, dx, dt, C=CE, Cb=CB)
    E, B, J, En, Bn, _ = em_mode(g, CE, CE if CB is None else CB, 20, 2, beta)
    grid = dict(ndim=2, nz=256, nx=16, ny=1, dz=dz, dx=dx, dy=dx, dt=dt,
                solver="yee" if name == "yee" else "custom", shape=1)
    if CB is not None:
        grid["coef_b"] = CB
    sim = gpu_sim(grid, [], coef=None if name == "yee" else CE)
    for t, a in ((sim.E, E), (sim.B, B), (sim.J, J)):
        t.copy_(torch.from_numpy(a.astype(np.float32)))
    sim.field_advance()
    inner = (Ellipsis, slice(50, g.nz - 50))
    scale = np.abs(En).max()
    assert np.abs(sim.E.double().cpu().numpy()[inner] - En[inner]).max() < 1e-5 * scale
    assert np.abs(sim.B.double().cpu().numpy()[inner] - Bn[inner]).max() < 1e-5 * scale
    sim.close()
