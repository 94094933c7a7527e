"""C ABI checks that need no GPU: the library loads, exports every symbol include/pic.h
declares, its host-side setup math matches the oracle, and bad configurations are refused
before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_1910_13529_gb300 import build
    build.build()
    import paper_1910_13529_gb300 as P
    return P


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    return sorted(set(re.findall(r"^\s*(?:pic_status|const char\*)\s+(pic_\w+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(P):
    names = declared_symbols()
    assert len(names) >= 20
    lib = ctypes.CDLL(P.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(P.EXPORTS) == names


def test_fit_matches_oracle(P):
    """The Appendix C system is ill-conditioned: coefficients agree to ~1e-7 while the fitted
    operator [k]_1 (the quantity the method uses) agrees to round-off inside the weighted band
    (khat <= 0.9, i.e. k <= 0.29 k_g where w = 1); near Nyquist the fit is unweighted."""
    from oracle import fit
    kh = np.linspace(0.0, 0.9, 2001)
    for kappa, M in [(4.0, 16), (1.8137, 16), (3.0, 8), (4.0, 4)]:
        a = P.pic_fit_coefficients(kappa, M)
        b = fit.fit_coefficients(kappa, M=M)
        assert np.max(np.abs(a - b)) < 5e-7
        assert np.max(np.abs(fit.axial_symbol(a, kh) - fit.axial_symbol(b, kh))) < 1e-9


def test_fit_reproduces_table1(P):
    C = P.pic_fit_coefficients(4.0, 16)
    ref = np.loadtxt(os.path.join(ROOT, "tests", "golden", "table1_coefficients.txt"))
    assert np.max(np.abs(C - ref)) < 5e-7


def test_taps_and_cfl_match_oracle(P):
    from oracle import fit
    C = np.loadtxt(os.path.join(ROOT, "tests", "golden", "table1_coefficients.txt"))
    assert np.max(np.abs(P.pic_correction_taps(C, 24) - fit.correction_kernel(C, hlen=24))) < 1e-14
    for nd, d in [(2, (0.02, 0.02, 0.02)), (3, (0.02, 0.05, 0.05))]:
        a = P.pic_cfl_dt(nd, *d, C)
        b = fit.cfl_dt(d[0], list(d[1:nd]), C)
        assert a == pytest.approx(b, rel=1e-9)
    assert P.pic_cfl_dt(2, 0.05, 0.05, 0.05, [1.0]) == pytest.approx(0.05 / np.sqrt(2), rel=1e-14)


def test_split_cfl_matches_oracle(P):
    """[k]_E1 != [k]_B1 (Sec. 3): the limit of the product of the two axial symbols."""
    from oracle import fit
    CE, CB = [1.0], fit.fit_coefficients(3.0, M=8)
    for nd, d in [(2, (0.02, 0.02, 0.02)), (3, (0.02, 0.05, 0.05))]:
        a = P.pic_cfl_dt_split(nd, *d, CE, CB)
        b = fit.cfl_dt(d[0], list(d[1:nd]), CE, Cb=CB)
        assert a == pytest.approx(b, rel=1e-9)
    # identical sets give the symmetric limit; a sign-changing product has none
    assert P.pic_cfl_dt_split(2, 0.05, 0.05, 0.05, CB, CB) == pytest.approx(P.pic_cfl_dt(2, 0.05, 0.05, 0.05, CB),
                                                                           rel=1e-14)
    with pytest.raises(P.PicError):
        P.pic_cfl_dt_split(2, 0.05, 0.05, 0.05, [1.0], [-1.0])


def _cfg(P, **kw):
    from paper_1910_13529_gb300.runtime import make_config
    base = dict(ndim=2, nz=64, nx=32, dz=0.05, dx=0.05, dt=0.02, shape=1)
    base.update(kw)
    return make_config(**base)


@pytest.mark.parametrize("kw,status", [
    (dict(ndim=4), 1), (dict(nz=2), 1), (dict(dt=-1.0), 1), (dict(shape=3), 1),
    (dict(solver="custom", M=40), 1), (dict(dt=0.05), 2),
    (dict(solver="custom", M=16, dt=0.05 / 1.2), 2), (dict(inject_species=9), 1),
])
def test_bad_configs_are_refused_on_host(P, kw, status):
    c, keep = _cfg(P, **kw)
    with pytest.raises(P.PicError) as ei:
        P.pic_create(c)
    assert ei.value.status == status
    assert len(P.pic_last_error()) > 0


def test_new_options_are_validated_on_host(P):
    from oracle import fit
    F8 = fit.fit_coefficients(3.0, M=8)
    c, keep = _cfg(P)
    c.current_filter = 7
    with pytest.raises(P.PicError) as ei:
        P.pic_create(c)
    assert ei.value.status == P.PIC_ERR_ARG and "current_filter" in P.pic_last_error()
    c, keep = _cfg(P)
    c.precision = 64                  # only the FP32 kernels are built
    with pytest.raises(P.PicError) as ei:
        P.pic_create(c)
    assert ei.value.status == P.PIC_ERR_ARG and "precision" in P.pic_last_error()
    bad = [
        (dict(solver="custom", coef_b=F8), P.PIC_ERR_ARG),                  # no explicit E-side set
        (dict(solver="yee", coef_b=F8), P.PIC_ERR_ARG),                     # split needs the customised solver
        (dict(solver="custom", coef=[1.0], coef_b=[-1.0]), P.PIC_ERR_ARG),  # product changes sign
        (dict(solver="custom", coef=[1.0], coef_b=F8, dt=0.05), P.PIC_ERR_CFL),
    ]
    for kw, status in bad:
        c, keep = _cfg(P, **kw)
        with pytest.raises(P.PicError) as ei:
            P.pic_create(c)
        assert ei.value.status == status, kw


def test_make_config_pads_the_two_coefficient_sets(P):
    c, keep = _cfg(P, solver="custom", coef=[1.0], coef_b=[0.9, 0.05, -0.01])
    assert c.M == 3
    ce, cb = keep
    assert list(ce) == [1.0, 0.0, 0.0] and list(cb) == [0.9, 0.05, -0.01]
    assert [c.coef[i] for i in range(3)] == [1.0, 0.0, 0.0]
    assert [c.coef_b[i] for i in range(3)] == [0.9, 0.05, -0.01]
    c, keep = _cfg(P, solver="custom", coef=[1.1, -0.05, 0.01, 0.002], coef_b=[1.0])
    assert c.M == 4 and [c.coef_b[i] for i in range(4)] == [1.0, 0.0, 0.0, 0.0]
    c, keep = _cfg(P)
    assert not c.coef_b and c.current_filter == P.PIC_FILTER_NONE


def test_null_handle_calls_return_arg_error(P):
    assert P.lib.pic_step(None, 1, None) == P.PIC_ERR_ARG
    assert P.lib.pic_diag(None, None, None) == P.PIC_ERR_ARG
    assert P.lib.pic_destroy(None) == P.PIC_OK


def test_kspace_limits_match_oracle_and_are_enforced(P):
    """The k-space solvers (Sec. 2.3 spectral, Sec. 3 [k1]_t): the library's stability limits equal
    the oracle's, dt above them and a moving window are refused before any device work."""
    from oracle import spectral as ks
    for nd, d in [(2, (0.05, 0.04, 0.04)), (3, (0.02, 0.05, 0.05))]:
        for name, solver in (("spectral", P.PIC_SOLVER_SPECTRAL), ("kt", P.PIC_SOLVER_KT)):
            a = P.pic_cfl_dt_kspace(nd, solver, *d)
            assert a == pytest.approx(ks.cfl_dt(nd, name, *d), rel=1e-12)
    with pytest.raises(P.PicError):
        P.pic_cfl_dt_kspace(2, P.PIC_SOLVER_CUSTOM, 0.05, 0.05)
    # PSATD: the field update is unconditionally stable, the particle move allows one cell
    assert P.pic_cfl_dt_kspace(3, P.PIC_SOLVER_PSATD, 0.05, 0.04, 0.045) == 0.04
    assert ks.cfl_dt(3, "psatd", 0.05, 0.04, 0.045) == 0.04
    lim = P.pic_cfl_dt_kspace(2, P.PIC_SOLVER_SPECTRAL, 0.05, 0.05)
    for kw, status in [(dict(solver="spectral", dt=1.01 * lim), P.PIC_ERR_CFL),
                       (dict(solver="kt", dt=0.051), P.PIC_ERR_CFL),
                       (dict(solver="spectral", dt=0.5 * lim, moving_window=True), P.PIC_ERR_ARG),
                       (dict(solver="psatd", dt=0.051), P.PIC_ERR_CFL)]:
        c, keep = _cfg(P, **kw)
        with pytest.raises(P.PicError) as ei:
            P.pic_create(c)
        assert ei.value.status == status, kw
