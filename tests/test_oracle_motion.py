"""Pins of the oracle's position update (or_move) together with its Boris push (or_boris):
the leapfrog of Sec. 2.1 moves a particle by x^{n+1} = x^n + dt u^{n+1/2} / gamma^{n+1/2} along
each axis, measured in cells of that axis.  Two closed forms of relativistic motion fix it:

* uniform E (B = 0): hyperbolic motion.  Started at rest at t = 0 (u^{-1/2} = -a dt/2), the
  Boris push gives u^{n+1/2} = a t_{n+1/2} exactly (a = qE/m), so x^N is the midpoint rule of
  X(T) = (sqrt(1 + (aT)^2) - 1)/a.  By the Euler-Maclaurin formula for the midpoint rule,
  x^N = X(T) - dt^2/24 (v'(T) - v'(0)) + O(dt^4), v'(t) = a/(1 + a^2 t^2)^{3/2}.
* crossed uniform E and B (|E| < |B|): the guiding centre drifts at E x B / B^2.

The cell sizes differ on every axis (dz != dx != dy), so an exchanged cell size, a gamma taken
from the wrong half step, or a wrong sign of the cross product fails one of these tests."""
import math

import numpy as np
import pytest

from oracle import core as oc

H = (0.4, 0.3, 0.2)        # dz, dx, dy


def _grid(ndim, dt):
    return oc.Grid(ndim, 64, 64, 64, dz=H[0], dx=H[1], dy=H[2], dt=dt)


@pytest.mark.parametrize("ndim,axis", [(3, 0), (3, 1), (3, 2), (2, 0), (2, 1)])
def test_hyperbolic_motion_along_each_axis(ndim, axis):
    dt, a, nsteps = 0.01, 1.3, 400
    g = _grid(ndim, dt)
    q, m = -1.0, 1.0
    eps = q * dt / (2 * m)
    eb = np.zeros((1, 6))
    eb[0, axis] = a * m / q                     # qE/m = a along the axis
    u = np.zeros((1, 3))
    u[0, axis] = -0.5 * a * dt                  # at rest at t = 0
    xi = np.array([[20.0, 20.0, 20.0]])
    xi0 = xi.copy()
    for _ in range(nsteps):
        oc.boris(eb, u, eps)
        xi = oc.move(g, xi, u)
    T = nsteps * dt
    X = (math.sqrt(1 + (a * T) ** 2) - 1) / a
    vp = lambda t: a / (1 + (a * t) ** 2) ** 1.5
    expect = X - dt * dt / 24 * (vp(T) - vp(0.0))
    disp = (xi - xi0)[0]
    assert disp[axis] * H[axis] == pytest.approx(expect, abs=1e-9)
    # no motion across the field, and none at all along y in 2D
    for d in range(3):
        if d != axis:
            assert disp[d] == 0.0
    assert u[0, axis] == pytest.approx(a * (T - 0.5 * dt), rel=1e-13)


def test_2d_move_ignores_the_out_of_plane_axis():
    """In 2D the out-of-plane momentum acts through gamma but the y coordinate is not advanced."""
    g = _grid(2, 0.05)
    u = np.array([[0.6, -0.8, 2.0]])
    xi0 = np.array([[10.0, 10.0, 0.25]])
    xi1 = oc.move(g, xi0, u)
    gam = math.sqrt(1 + 0.36 + 0.64 + 4.0)
    assert xi1[0, 0] - 10.0 == pytest.approx(0.05 * 0.6 / gam / H[0], rel=1e-14)
    assert xi1[0, 1] - 10.0 == pytest.approx(-0.05 * 0.8 / gam / H[1], rel=1e-14)
    assert xi1[0, 2] == 0.25


ORIENT = [(0, 1), (1, 2), (2, 0), (1, 0), (2, 1), (0, 2)]   # (axis of E, axis of B)


def test_e_cross_b_drift_in_every_orientation():
    """Crossed uniform fields, E/B = 0.3: a particle started at rest drifts at E x B / B^2
    (relativistic, |E| < |B|).  The drift velocity is the least-squares slope of the position
    over 400 gyrations; the gyration itself averages out to about 1e-4 of the drift."""
    dt, nsteps = 0.02, 0
    g = _grid(3, dt)
    q, m = -1.0, 1.0
    E0, B0 = 0.3, 1.0
    n = len(ORIENT)
    eb = np.zeros((n, 6))
    for p, (ea, ba) in enumerate(ORIENT):
        eb[p, ea] = E0
        eb[p, 3 + ba] = B0
    u = np.zeros((n, 3))
    xi = np.full((n, 3), 32.0)
    # the drift-frame gyro-frequency is |q| B / (m gamma_d^2) ~ 0.91: 400 turns ~ 2760 / dt steps
    nsteps = 140000
    every = 50
    ts, xs = [], []
    for s in range(nsteps):
        oc.boris(eb, u, q * dt / (2 * m))
        xi = oc.move(g, xi, u)
        if s % every == 0:
            ts.append((s + 1) * dt)
            xs.append(xi * np.asarray(H))
    ts = np.asarray(ts)
    xs = np.asarray(xs)                        # (samples, particle, axis), physical units
    A = np.stack([ts, np.ones_like(ts)], axis=1)
    for p, (ea, ba) in enumerate(ORIENT):
        Ev = np.zeros(3)
        Bv = np.zeros(3)
        Ev[ea], Bv[ba] = E0, B0
        vd = np.cross(Ev, Bv) / (B0 * B0)
        slope = np.linalg.lstsq(A, xs[:, p, :], rcond=None)[0][0]
        assert np.max(np.abs(slope - vd)) < 3e-4 * np.linalg.norm(vd), (ORIENT[p], slope, vd)
