"""Brute-force pins of the oracle's whole PIC step on tiny grids (8 x 8 in 2D, 8 x 8 x 4 in 3D).

Every operator is written here again from its definition, in a different form from the C
loops of the oracle, and the step is composed from those pieces:

* the field step of Eq. 1 as one dense matrix: the Appendix C axial operators
  d+ f_i = sum_l C_l (f_{i+l} - f_{i-l+1})/dz and d- f_i = sum_l C_l (f_{i+l-1} - f_{i-l})/dz
  and the two-point transverse differences (Sec. 2.2) are dense shift matrices (zero outside
  0 <= i < nz, periodic in x and y), the curls are 3 x 3 block matrices, and the leapfrog
  B half / E full / B half of Sec. 2.1 is the product of the three block updates;
* the gather as a dense weighted sum over every node of the grid (B-spline weights of the
  periodic distance to each staggered node, Sec. 1 "interpolate");
* the Esirkepov current in its symmetric form W_z = (S1_z - S0_z)(S0_x + S1_x)/2 (2D) and
  W_z = (S1_z - S0_z)(S0_x S0_y/3 + S0_x S1_y/6 + S1_x S0_y/6 + S1_x S1_y/3) (3D), cumulated
  along the axis on an unwrapped three-period range and folded into the periodic grid;
* the Boris rotation with numpy cross products;
* the Sec. 3 current correction as a dense Toeplitz matrix along z.

The oracle's Sim.step must agree with this composition to round-off."""
import math

import numpy as np
import pytest

from oracle import core as oc
from oracle import fit

STAG = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]
STAG2 = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0), (0, 0.5, 0), (0.5, 0, 0), (0.5, 0.5, 0)]   # 2D: E3, B1, B2


def spline(order, d):
    d = np.abs(np.asarray(d, dtype=np.float64))
    if order == 1:
        return np.where(d < 1, 1 - d, 0.0)
    return np.where(d <= 0.5, 0.75 - d * d, np.where(d < 1.5, 0.5 * (1.5 - d) ** 2, 0.0))


class Dense:
    def __init__(self, ndim, nz, nx, ny, dz, dx, dy, dt, C, Cb=None):
        self.ndim, self.nz, self.nx, self.ny = ndim, nz, nx, (ny if ndim == 3 else 1)
        self.dz, self.dx, self.dy, self.dt = dz, dx, dy, dt
        self.N = self.nz * self.nx * self.ny
        Cb = C if Cb is None else Cb
        I = np.eye(self.N)
        Dzp = sum(c * (self.sz(l) - self.sz(1 - l)) for l, c in enumerate(C, start=1)) / dz
        Dzm = sum(c * (self.sz(l - 1) - self.sz(-l)) for l, c in enumerate(Cb, start=1)) / dz
        Dxp, Dxm = (self.sx(1) - I) / dx, (I - self.sx(-1)) / dx
        if ndim == 3:
            Dyp, Dym = (self.sy(1) - I) / dy, (I - self.sy(-1)) / dy
        else:
            Dyp = Dym = np.zeros_like(I)
        Z = np.zeros_like(I)
        self.CP = np.block([[Z, -Dyp, Dxp], [Dyp, Z, -Dzp], [-Dxp, Dzp, Z]])
        self.CM = np.block([[Z, -Dym, Dxm], [Dym, Z, -Dzm], [-Dxm, Dzm, Z]])
        self.div_m = np.block([[Dzm, Dxm, Dym]])

    def lin(self, i, j, k):
        return (k * self.nx + j) * self.nz + i

    def _shift(self, di, dj, dk):
        S = np.zeros((self.N, self.N))
        for k in range(self.ny):
            for j in range(self.nx):
                for i in range(self.nz):
                    ii = i + di
                    if 0 <= ii < self.nz:
                        S[self.lin(i, j, k), self.lin(ii, (j + dj) % self.nx, (k + dk) % self.ny)] = 1.0
        return S

    def sz(self, s):
        return self._shift(s, 0, 0)

    def sx(self, s):
        return self._shift(0, s, 0)

    def sy(self, s):
        return self._shift(0, 0, s)

    def field_step(self, E, B, J):
        """(E, B) flattened component-major; Eq. 1 leapfrog: B half, E full, B half."""
        h = 0.5 * self.dt
        B1 = B - h * self.CP @ E
        E1 = E + self.dt * (self.CM @ B1 - J)
        return E1, B1 - h * self.CP @ E1

    # ---- particles ----
    def weights_on_grid(self, order, xi, stag):
        """Per-axis B-spline weights of every node (z: 0..nz-1; x, y: periodic distance)."""
        wz = spline(order, np.arange(self.nz) + stag[0] - xi[0])
        dxv = (np.arange(self.nx) + stag[1] - xi[1] + self.nx / 2) % self.nx - self.nx / 2
        wx = spline(order, dxv)
        if self.ndim == 3:
            dyv = (np.arange(self.ny) + stag[2] - xi[2] + self.ny / 2) % self.ny - self.ny / 2
            wy = spline(order, dyv)
        else:
            wy = np.ones(1)
        return wz, wx, wy

    def gather(self, order, E, B, xi):
        F = np.concatenate([E, B]).reshape(6, self.ny, self.nx, self.nz)
        st = STAG if self.ndim == 3 else STAG2
        out = np.zeros(6)
        for c in range(6):
            wz, wx, wy = self.weights_on_grid(order, xi, st[c])
            out[c] = np.einsum("kji,k,j,i->", F[c], wy, wx, wz)
        return out

    def current(self, order, xi0, xi1, u, Q):
        """Esirkepov current of one move, symmetric form, unwrapped ranges folded into the grid."""
        nd = self.ndim
        V = self.dz * self.dx * (self.dy if nd == 3 else 1.0)
        hh = (self.dz, self.dx, self.dy)
        # unwrapped node ranges: z extended by 4 on each side, x and y three periods
        rz = np.arange(-4, self.nz + 4)
        rx = np.arange(-self.nx, 2 * self.nx)
        ry = np.arange(-self.ny, 2 * self.ny) if nd == 3 else np.zeros(1, int)
        ranges = (rz, rx, ry)
        S0 = [spline(order, r - xi0[a]) if a < nd else np.ones(1) for a, r in enumerate(ranges)]
        S1 = [spline(order, r - xi1[a]) if a < nd else np.ones(1) for a, r in enumerate(ranges)]
        J = np.zeros((3, len(ry), len(rx), len(rz)))
        if nd == 2:
            Wz = np.outer(0.5 * (S0[1] + S1[1]), S1[0] - S0[0])[None]
            Wx = np.outer(S1[1] - S0[1], 0.5 * (S0[0] + S1[0]))[None]
            J[0] = -Q / V * self.dz / self.dt * np.cumsum(Wz, axis=2)
            J[1] = -Q / V * self.dx / self.dt * np.cumsum(Wx, axis=1)
            v3 = u[2] / math.sqrt(1.0 + u @ u)
            W3 = (np.outer(S0[1], S0[0]) / 3 + np.outer(S1[1], S0[0]) / 6 + np.outer(S0[1], S1[0]) / 6
                  + np.outer(S1[1], S1[0]) / 3)
            J[2] = Q / V * v3 * W3[None]
        else:
            def tw(a0, a1, b0, b1):        # T(b, a) weights of the two transverse axes
                return np.outer(b0, a0) / 3 + np.outer(b0, a1) / 6 + np.outer(b1, a0) / 6 + np.outer(b1, a1) / 3
            dS = [S1[a] - S0[a] for a in range(3)]
            # W along z: dSz(i) T(x, y)
            Tz = tw(S0[1], S1[1], S0[2], S1[2])                  # (y, x)
            Wz = Tz[:, :, None] * dS[0][None, None, :]
            Tx = tw(S0[0], S1[0], S0[2], S1[2])                  # (y, z)
            Wx = Tx[:, None, :] * dS[1][None, :, None]
            Ty = tw(S0[0], S1[0], S0[1], S1[1])                  # (x, z)
            Wy = Ty[None, :, :] * dS[2][:, None, None]
            J[0] = -Q / V * hh[0] / self.dt * np.cumsum(Wz, axis=2)
            J[1] = -Q / V * hh[1] / self.dt * np.cumsum(Wx, axis=1)
            J[2] = -Q / V * hh[2] / self.dt * np.cumsum(Wy, axis=0)
        # fold into the grid: drop z outside 0..nz-1, x and y modulo the period
        out = np.zeros((3, self.ny, self.nx, self.nz))
        inside = (rz >= 0) & (rz < self.nz)
        for ky, yv in enumerate(ry):
            for jx, xv in enumerate(rx):
                out[:, yv % self.ny, xv % self.nx, :] += J[:, ky, jx, inside]
        return out.reshape(3 * self.N)


def boris(u, eb, eps):
    um = u + eps * eb[:3]
    t = eps * eb[3:] / math.sqrt(1 + um @ um)
    s = 2 * t / (1 + t @ t)
    up = um + np.cross(um, t)
    return um + np.cross(up, s) + eps * eb[:3]


def toeplitz_z(d, h):
    """J1 <- sum_m h_m J1_{i-m} along z with zero outside, as a dense matrix."""
    hl = (len(h) - 1) // 2
    T = np.zeros((d.N, d.N))
    for m in range(-hl, hl + 1):
        if abs(m) < d.nz:
            T += h[m + hl] * d.sz(-m)
    return T


FIELD_CASES = [
    ("2d-yee", 2, (1.0,), None),
    ("2d-custom3", 2, (1.12, -0.05, 0.0066), None),
    ("2d-split", 2, (1.12, -0.05, 0.0066), (1.05, -0.02, 0.003)),
    ("3d-yee", 3, (1.0,), None),
    ("3d-custom3", 3, (1.12, -0.05, 0.0066), None),
]


@pytest.mark.parametrize("name,ndim,C,Cb", FIELD_CASES)
def test_field_step_is_the_dense_leapfrog(name, ndim, C, Cb):
    nz, nx, ny = 8, 8, 4
    d = Dense(ndim, nz, nx, ny, 0.5, 0.4, 0.45, 0.11, C, Cb)
    g = oc.Grid(ndim, nz, nx, ny, 0.5, 0.4, 0.45, 0.11, C=C, Cb=Cb)
    rng = np.random.default_rng(3)
    E, B, J = (rng.normal(size=g.fshape) for _ in range(3))
    Ed, Bd = d.field_step(E.ravel(), B.ravel(), J.ravel())
    oc.field_advance(g, E, B, J)
    assert np.max(np.abs(E.ravel() - Ed)) < 1e-12 * np.max(np.abs(Ed))
    assert np.max(np.abs(B.ravel() - Bd)) < 1e-12 * np.max(np.abs(Bd))
    # the dense operators themselves: d- = -(d+)^T (same coefficients) and div- curl- = 0
    if Cb is None:
        assert np.max(np.abs(d.CM - d.CP.T)) < 1e-12
    assert np.max(np.abs(d.div_m @ d.CM)) < 1e-10


STEP_CASES = [
    ("2d-yee-lin", 2, 1, (1.0,)),
    ("2d-yee-quad", 2, 2, (1.0,)),
    ("2d-custom3-quad", 2, 2, (1.12, -0.05, 0.0066)),
    ("3d-yee-quad", 3, 2, (1.0,)),
    ("3d-custom3-lin", 3, 1, (1.12, -0.05, 0.0066)),
]


@pytest.mark.parametrize("name,ndim,shape,C", STEP_CASES)
def test_whole_step_brute_force(name, ndim, shape, C):
    """Three PIC steps with three particles (one crossing the periodic x seam) on an 8 x 8
    (x 4) grid: the oracle's Sim against the dense composition above, to round-off."""
    nz, nx, ny = 8, 8, 4
    dz, dx, dy = 0.5, 0.4, 0.45
    dt = 0.8 * fit.cfl_dt(dz, [dx] + ([dy] if ndim == 3 else []), None if len(C) == 1 else C)
    d = Dense(ndim, nz, nx, ny, dz, dx, dy, dt, C)
    g = oc.Grid(ndim, nz, nx, ny, dz, dx, dy, dt, C=C, shape=shape)
    h = None if len(C) == 1 else fit.correction_kernel(C, hlen=40)
    T = None if h is None else toeplitz_z(d, h)
    rng = np.random.default_rng(8)
    xi = np.array([[3.3, 7.8, 1.2], [4.6, 0.3, 3.9], [3.9, 4.1, 0.6]])
    if ndim == 2:
        xi[:, 2] = 0.0
    u = rng.normal(size=(3, 3)) * 0.7
    u[0, 1] = 0.9                                # towards the seam at x = nx
    q, m, w = -1.0, 1.0, 0.3
    sim = oc.Sim(g, [oc.Species(xi, u, q, m, w)], h=h)
    E0 = rng.normal(size=g.fshape) * 0.2
    B0 = rng.normal(size=g.fshape) * 0.2
    sim.E[:] = E0
    sim.B[:] = B0
    E, B = E0.ravel().copy(), B0.ravel().copy()
    X, U = xi.copy(), u.copy()
    hh = np.array([dz, dx, dy])
    for _ in range(3):
        J = np.zeros(3 * d.N)
        for p in range(3):
            eb = d.gather(shape, E, B, X[p])
            U[p] = boris(U[p], eb, q * dt / (2 * m))
            x1 = X[p].copy()
            gam = math.sqrt(1 + U[p] @ U[p])
            x1[:ndim] += dt * U[p, :ndim] / gam / hh[:ndim]
            J += d.current(shape, X[p], x1, U[p], q * w)
            X[p] = x1
        if T is not None:
            J[: d.N] = T @ J[: d.N]
        E, B = d.field_step(E, B, J)
        X[:, 1] %= nx
        if ndim == 3:
            X[:, 2] %= ny
        sim.step()
    scale = max(np.abs(E).max(), np.abs(B).max())
    assert np.max(np.abs(sim.E.ravel() - E)) < 1e-12 * scale
    assert np.max(np.abs(sim.B.ravel() - B)) < 1e-12 * scale
    sp = sim.species[0]
    assert len(sp.xi) == 3
    assert np.max(np.abs(sp.xi - X)) < 1e-12
    assert np.max(np.abs(sp.u - U)) < 1e-12
