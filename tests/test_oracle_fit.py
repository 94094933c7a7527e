"""Pins of the Appendix C fit, the Sec. 3 current-correction kernel and the CFL limit (oracle/fit.py)."""
import math
import os

import numpy as np
import pytest

from oracle import fit

HERE = os.path.dirname(os.path.abspath(__file__))


def table1():
    return np.loadtxt(os.path.join(HERE, "golden", "table1_coefficients.txt"))


def test_table1_consistency_constraint():
    # Appendix C: M C = e1 with p = 2 is sum (2l-1) C_l = 1
    C = table1()
    assert np.sum((2 * np.arange(1, 17) - 1) * C) == pytest.approx(1.0, abs=1e-14)


def test_refit_reproduces_table1():
    # Appendix C with the reading p = 2, w_k1 = 0.6, n = 10 (kappa = 4, M = 16)
    C = fit.fit_coefficients(4.0, M=16, p=2, w_k1=0.6, n=10)
    assert np.max(np.abs(C - table1())) < 5e-7


def test_fit_constraint_holds_for_other_orders():
    for p in (2, 4, 6):
        C = fit.fit_coefficients(3.0, M=12, p=p)
        Mc = fit.constraint_matrix(12, p)
        e = np.zeros(p // 2)
        e[0] = 1.0
        assert np.allclose(Mc @ C, e, atol=1e-11)


def test_yee_is_the_m1_fit():
    # M = 1, p = 2: the only consistent coefficient is C_1 = 1 (the Yee operator)
    assert fit.fit_coefficients(4.0, M=1)[0] == pytest.approx(1.0, abs=1e-14)


def test_symbol_matches_time_operator_at_low_k():
    # Sec. 3: [k]_1 close to [k1]_t except at the highest k1
    C = table1()
    kh = np.linspace(1e-3, 1.0, 200)
    target = 4.0 * np.sin(kh / 4.0)
    rel = np.abs(fit.axial_symbol(C, kh) / target - 1.0)
    assert rel.max() < 1e-6
    kn = fit.axial_symbol(C, math.pi / 2) / (4.0 * math.sin(math.pi / 8)) - 1.0
    assert -0.1 < kn < -0.01


def test_symmetric_stencil_identity():
    # sum_l C_l sin((2l-1)t)/sin t == P_0 + 2 sum_m P_m cos(2 m t)
    C = table1()
    Pm = fit.symmetric_stencil(C)
    t = np.linspace(0.01, 1.5, 50)
    lhs = fit.axial_symbol(C, t) / np.sin(t)
    rhs = Pm[0] + 2 * sum(Pm[m] * np.cos(2 * m * t) for m in range(1, 16))
    assert np.allclose(lhs, rhs, rtol=1e-13)


def test_correction_kernel_inverts_p():
    C = table1()
    Pm = fit.symmetric_stencil(C)
    h = fit.correction_kernel(C, hlen=40)
    P = np.concatenate([Pm[::-1], Pm[1:]])  # m = -15..15
    conv = np.convolve(P, h)                # centre at index 15 + 40
    delta = np.zeros_like(conv)
    delta[15 + 40] = 1.0
    inner = slice(15 + 40 - 20, 15 + 40 + 21)
    assert np.max(np.abs(conv[inner] - delta[inner])) < 1e-13
    assert abs(h[40 + 24]) < 1e-9 and abs(h[40 + 40]) < 1e-14
    assert np.max(np.abs(h - h[::-1])) < 1e-16


def test_cfl_yee_closed_form():
    # (dt/2)^2 (4/dz^2 + 4/dx^2) = 1  ->  dt = 1/sqrt(1/dz^2 + 1/dx^2)
    assert fit.cfl_dt(0.05, [0.05]) == pytest.approx(0.05 / math.sqrt(2), rel=1e-14)
    assert fit.cfl_dt(0.02, [0.05, 0.05]) == pytest.approx(1 / math.sqrt(1 / 0.02**2 + 2 / 0.05**2), rel=1e-14)


def test_cfl_custom_2d_fixed_point():
    # the customised limit with C fitted at its own dt: kappa_CFL ~ 1.632 (2D, r = 1)
    dz = 1.0
    def resid(kappa):
        C = fit.fit_coefficients(kappa)
        return dz / fit.cfl_dt(dz, [dz], C) - kappa
    from scipy.optimize import brentq
    k = brentq(resid, 1.3, 3.0)
    assert k == pytest.approx(1.632, abs=2e-3)
