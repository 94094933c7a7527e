"""Pins of the k-space analysis module (oracle/kspace.py) to the numbers the paper prints.

Sec. 2.2 (Yee), Sec. 2.3 (spectral), Sec. 3 (proposed solver) and Appendix D.
"""
import math
import os
import warnings

import pytest

from oracle import kspace

warnings.filterwarnings("ignore")
HERE = os.path.dirname(os.path.abspath(__file__))


def printed():
    out = {}
    with open(os.path.join(HERE, "golden", "printed_constants.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, val, digits = line.split()[:3]
            out[name] = (float(val), int(digits))
    return out


def sig(x, n):
    return float(f"{x:.{n}g}") if x != 0 else 0.0


P = printed()


def check(name, value):
    ref, digits = P[name]
    assert sig(value, digits) == pytest.approx(ref, abs=1e-12), (name, value, ref)


def test_thresholds():
    check("r_star", kspace.r_star())
    check("spectral_kappa_r", kspace.kappa_r_spectral())
    check("custom_kappa_r", kspace.kappa_r_custom())
    # Sec. 2.2: kappa_r^2 sin^2(pi/(2 kappa_r)) = 1 + r^-2 has kappa_r = 2 exactly at r = 1
    assert kspace.kappa_r_yee(1.0) == pytest.approx(2.0, abs=1e-12)


@pytest.mark.parametrize("order,name", [(1, "yee_F1_linear"), (2, "yee_F1_quadratic")])
def test_self_force_yee(order, name):
    check(name, kspace.self_force_yee(4.0, 1.0, order))


@pytest.mark.parametrize("order,name", [(1, "spectral_F1_linear"), (2, "spectral_F1_quadratic")])
def test_self_force_spectral(order, name):
    check(name, kspace.self_force_spectral(4.0, 1.0, order))


@pytest.mark.parametrize("order,name", [(1, "custom_F1_linear"), (2, "custom_F1_quadratic")])
def test_self_force_custom(order, name):
    # the printed closed form reproduces the printed numbers ...
    check(name, kspace.self_force_custom(4.0, 1.0, order, printed=True))
    # ... and differs from Eq. E12D with [k]_B1 = [k1]_t by exactly kappa (reading recorded in DESIGN)
    a = kspace.self_force_custom(4.0, 1.0, order, printed=True)
    b = kspace.self_force_custom(4.0, 1.0, order, printed=False)
    assert a / b == pytest.approx(4.0, rel=1e-6)


def test_filtered_self_forces_table2():
    """Table 2 (and Sec. 2.2, 2.3): quadratic shape with the 5-pass current filter.  The filter is
    not defined in the paper; the reading (four (1,2,1)/4 passes and a (-5/4, 7/2, -5/4)
    compensator along x1) reproduces all three printed values, one per solver."""
    check("yee_F1_quadratic_5pass", kspace.self_force_yee(4.0, 1.0, 2, filt=True))
    check("spectral_F1_quadratic_5pass", kspace.self_force_spectral(4.0, 1.0, 2, filt=True))
    check("custom_F1_quadratic_5pass", kspace.self_force_custom(4.0, 1.0, 2, printed=True, filt=True))


MUTATED_FILTERS = {
    "flat compensator (-1, 3, -1)": ((0.25, 0.5),) * 4 + ((-1.0, 3.0),),
    "no compensator": ((0.25, 0.5),) * 4,
    "three binomial passes + compensator": ((0.25, 0.5),) * 3 + ((-1.25, 3.5),),
    "five binomial passes + compensator": ((0.25, 0.5),) * 5 + ((-1.25, 3.5),),
    "compensator first, then four passes (same product)": None,
}


@pytest.mark.parametrize("name", sorted(MUTATED_FILTERS))
def test_table2_pins_reject_other_filters(name, monkeypatch):
    """The Table 2 pins discriminate: every other plausible filter misses at least one printed
    value (the pass order alone cannot matter, the symbol being a product)."""
    passes = MUTATED_FILTERS[name]
    if passes is None:
        passes = ((-1.25, 3.5),) + ((0.25, 0.5),) * 4
    monkeypatch.setattr(kspace, "FILTER_PASSES", passes)
    got = [sig(kspace.self_force_yee(4.0, 1.0, 2, filt=True), 2),
           sig(kspace.self_force_spectral(4.0, 1.0, 2, filt=True), 2),
           sig(kspace.self_force_custom(4.0, 1.0, 2, printed=True, filt=True), 2)]
    want = [P[n][0] for n in ("yee_F1_quadratic_5pass", "spectral_F1_quadratic_5pass", "custom_F1_quadratic_5pass")]
    same = all(g == pytest.approx(w, abs=1e-12) for g, w in zip(got, want))
    assert same == ("same product" in name), (name, got)


def test_filter_symbol_limits():
    # DC passes unchanged, the grid Nyquist mode (khat = pi/2) is removed, the symbol stays in [0, 1.1]
    assert kspace.filter_symbol(0.0) == pytest.approx(1.0, abs=1e-15)
    assert abs(kspace.filter_symbol(math.pi / 2)) < 1e-15
    import numpy as np
    k = np.linspace(0, math.pi / 2, 2001)
    s = kspace.filter_symbol(k)
    assert s.min() >= -1e-15 and s.max() < 1.1


def test_sign_of_self_forces():
    # Sec. 2.2: Yee decelerates; Sec. 2.3 and Sec. 3: accelerate
    assert kspace.self_force_yee() < 0
    assert kspace.self_force_spectral() > 0
    assert kspace.self_force_custom() > 0


def test_quadratic_shape_reduces_self_force():
    for f in (kspace.self_force_yee, kspace.self_force_spectral, kspace.self_force_custom):
        assert abs(f(4.0, 1.0, 2)) < abs(f(4.0, 1.0, 1))


@pytest.mark.parametrize("A", [0.05, 0.3, 0.7, 0.95])
def test_appendix_d_sine_integral(A):
    pv, mag = kspace.int_sin_direct(A)
    closed = kspace.int_sin_closed(A, k1_positive=True)
    assert pv == pytest.approx(closed.real, abs=1e-9)
    assert mag == pytest.approx(abs(closed.imag), rel=1e-7)
    assert kspace.int_sin_closed(A, k1_positive=False) == -closed


@pytest.mark.parametrize("A", [0.1, 0.8, 2.0, 4.0, 9.0])
def test_appendix_d_quadratic_integral(A):
    pv, mag = kspace.int_quad_direct(A)
    closed = kspace.int_quad_closed(A)
    assert pv == pytest.approx(closed.real, rel=1e-9)
    assert mag == pytest.approx(abs(closed.imag), rel=1e-7, abs=1e-12)


def test_yee_aliased_zones_antisymmetric():
    # Sec. 2.2: for r = 1, kappa >= 2 the nu1 = +-1 field is pure space charge, antisymmetric
    # about the particle: E1(i') = -E1(-1-i') (staggered by half a cell)
    for ip in range(0, 6):
        a = kspace.e1_axis_yee(ip, zones=(-1, 1))
        b = kspace.e1_axis_yee(-1 - ip, zones=(-1, 1))
        assert a == pytest.approx(-b, abs=1e-10)


def test_yee_fundamental_zone_has_wake():
    # Sec. 2.2: the Cerenkov part extends behind the particle, not in front
    behind = max(abs(kspace.e1_axis_yee(-i, zones=(0,))) for i in range(20, 40))
    ahead = max(abs(kspace.e1_axis_yee(i, zones=(0,))) for i in range(20, 40))
    assert behind > 10 * ahead
