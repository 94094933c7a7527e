"""k-space field advance: the spectral solver of Sec. 2.3 ([k]_i = k_i) and the Sec. 3 operator
[k]_1 = [k1]_t applied exactly in k space ("easily implemented if the fields are advanced in k
space", Sec. 3).  Plain numpy FFTs in FP64.

TEST INFRASTRUCTURE ONLY (part of the oracle): only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may use it; the CUDA library never does.

The fields sit on the staggered grid of the finite-difference solver (E1 at (i+1/2, j, k), E2 at
(i, j+1/2, k), E3 at (i, j, k+1/2), B1 at (i, j+1/2, k+1/2), B2 at (i+1/2, j, k+1/2), B3 at
(i+1/2, j+1/2, k); arrays [c][y][x][z]) and are periodic along every axis.  Axis a carries a real,
odd symbol kappa_a(k) in place of the Yee (2/h_a) sin(k h_a/2) (Sec. 2.1-2.3):

    "spectral":  kappa_a = k_a on every axis                       (Sec. 2.3)
    "kt":        kappa_1 = [k1]_t = (2/dt) sin(k1 dt/2) along z,  Yee across   (Sec. 3)
    "yee":       the Yee symbol on every axis
    "custom":    kappa_1 = (2/dz) sum_l C_l sin((2l-1) k1 dz/2) along z (Appendix C), Yee across

The difference from a node to the half-cell point above it, d+, has the symbol
e^{i k h/2} i kappa(k), the one from a half-cell point to the node above it, d-,
e^{-i k h/2} i kappa(k); with the Yee symbol they are (e^{ikh} - 1)/h and (1 - e^{-ikh})/h, i.e.
the finite differences themselves.  One step is Eq. 1:

    B <- B - dt/2 curl+ E;    E <- E + dt (curl- B - J');    B <- B - dt/2 curl+ E,
    (curl F)_1 = d_x F3 - d_y F2,  (curl F)_2 = d_y F1 - d_z F3,  (curl F)_3 = d_z F2 - d_x F1.

J' scales each component by kappa_Yee,a / kappa_a: the Esirkepov current obeys the continuity
equation with the Yee d-, the scaled one the continuity equation with this solver's d-, so
Gauss's law d-.E = rho is kept (the k-space form of the Sec. 3 correction P^-1, here on every
axis whose operator is not Yee).

"psatd" is the analytic-time update of Appendix B (advance_psatd), on the same staggered fields.
"""
import numpy as np

KINDS = ("spectral", "kt", "yee", "custom", "psatd")


def yee_symbol(k, h):
    """(2/h) sin(k h/2)."""
    return 2.0 / h * np.sin(0.5 * k * h)


def wavenumbers(n, h, half):
    """Wavenumbers of the FFT indices along an axis of n cells of size h (half: the r2c axis,
    indices 0..n/2; else 0..n-1 with the upper half negative)."""
    if half:
        return 2.0 * np.pi * np.arange(n // 2 + 1) / (n * h)
    return 2.0 * np.pi * np.fft.fftfreq(n, d=h)


def axis_symbol(kind, axis, k, g, C=None):
    """kappa_a(k) of the solver `kind` on axis 0 (z), 1 (x) or 2 (y)."""
    h = (g.dz, g.dx, g.dy)[axis]
    if kind == "spectral":
        return np.array(k, dtype=np.float64)
    if axis == 0 and kind == "kt":
        return 2.0 / g.dt * np.sin(0.5 * k * g.dt)
    if axis == 0 and kind == "custom":
        C = np.asarray(C, dtype=np.float64)
        l = np.arange(1, len(C) + 1)
        return 2.0 / h * np.sum(C[:, None] * np.sin(np.outer(2 * l - 1, 0.5 * k * h)), axis=0)
    return yee_symbol(k, h)


def operators(g, kind, C=None):
    """Broadcastable d+, d- symbols and current ratios per axis, shaped for arrays [y][x][z]."""
    ks = [wavenumbers(g.nz, g.dz, True), wavenumbers(g.nx, g.dx, False),
          wavenumbers(g.ny, g.dy, False) if g.ndim == 3 else np.zeros(1)]
    shapes = [(1, 1, -1), (1, -1, 1), (-1, 1, 1)]
    dp, dm, ratio = [], [], []
    for a in range(3):
        k = ks[a]
        h = (g.dz, g.dx, g.dy)[a]
        kap = axis_symbol(kind, a, k, g, C)
        if a == 2 and g.ndim == 2:
            kap = np.zeros(1)
        yee = yee_symbol(k, h) if not (a == 2 and g.ndim == 2) else np.zeros(1)
        with np.errstate(divide="ignore", invalid="ignore"):
            r = np.where(kap == 0.0, 1.0, yee / np.where(kap == 0.0, 1.0, kap))
        ph = np.exp(0.5j * k * h)
        dp.append((ph * 1j * kap).reshape(shapes[a]))
        dm.append((np.conj(ph) * 1j * kap).reshape(shapes[a]))
        ratio.append(r.reshape(shapes[a]))
    return dp, dm, ratio


def _fwd(F):
    return np.fft.rfftn(F, axes=(1, 2, 3))


def _inv(Fk, g):
    return np.fft.irfftn(Fk, s=(g.ny, g.nx, g.nz), axes=(1, 2, 3))


def curl(d, F):
    """(curl F) with the per-axis symbols d = (d_z, d_x, d_y), F in k space [c][y][x][z]."""
    dz, dx, dy = d
    return np.stack([dx * F[2] - dy * F[1], dy * F[0] - dz * F[2], dz * F[1] - dx * F[0]])


def advance(g, E, B, J, kind, C=None):
    """One step of Eq. 1 in k space, in place on the real arrays E, B (J is not modified); "psatd"
    dispatches to advance_psatd."""
    if kind == "psatd":
        return advance_psatd(g, E, B, J)
    dp, dm, ratio = operators(g, kind, C)
    Ek, Bk, Jk = _fwd(E), _fwd(B), _fwd(J)
    Jk = np.stack([Jk[0] * ratio[0], Jk[1] * ratio[1], Jk[2] * ratio[2]])
    Bk = Bk - 0.5 * g.dt * curl(dp, Ek)
    Ek = Ek + g.dt * (curl(dm, Bk) - Jk)
    Bk = Bk - 0.5 * g.dt * curl(dp, Ek)
    E[:] = _inv(Ek, g)
    B[:] = _inv(Bk, g)


def div_minus(g, F, kind, C=None):
    """d-.F with this solver's symbols (real space, at the nodes)."""
    _, dm, _ = operators(g, kind, C)
    Fk = _fwd(F)
    return np.fft.irfftn(dm[0] * Fk[0] + dm[1] * Fk[1] + dm[2] * Fk[2], s=(g.ny, g.nx, g.nz), axes=(0, 1, 2))


def div_plus(g, F, kind, C=None):
    """d+.F (at the cell centres: zero for a magnetic field that started divergence-free)."""
    dp, _, _ = operators(g, kind, C)
    Fk = _fwd(F)
    return np.fft.irfftn(dp[0] * Fk[0] + dp[1] * Fk[1] + dp[2] * Fk[2], s=(g.ny, g.nx, g.nz), axes=(0, 1, 2))


# half-cell offsets of each component along (z, x, y): E1 z, E2 x, E3 y; B1 x y, B2 z y, B3 z x
STAGGER_E = ((1, 0, 0), (0, 1, 0), (0, 0, 1))
STAGGER_B = ((0, 1, 1), (1, 0, 1), (1, 1, 0))


def _axes_k(g):
    ks = [wavenumbers(g.nz, g.dz, True), wavenumbers(g.nx, g.dx, False),
          wavenumbers(g.ny, g.dy, False) if g.ndim == 3 else np.zeros(1)]
    shapes = [(1, 1, -1), (1, -1, 1), (-1, 1, 1)]
    return [k.reshape(sh) for k, sh in zip(ks, shapes)]


def _nyquist_mask(g):
    """Modes on the Nyquist plane of an even axis (their half-cell phases are not real)."""
    m = np.zeros((g.ny, g.nx, g.nz // 2 + 1), dtype=bool)
    if g.nz % 2 == 0:
        m[:, :, g.nz // 2] = True
    if g.nx % 2 == 0:
        m[:, g.nx // 2, :] = True
    if g.ndim == 3 and g.ny % 2 == 0:
        m[g.ny // 2, :, :] = True
    return m


def advance_psatd(g, E, B, J):
    """One PSATD step (Appendix B, Eqs. B1-B2, with c = cos(k dt), s = sin(k dt), k = |k|):
        E <- c E + i s khat x B - (s/k) J + (1 - c) khat (khat.E) + (s/k - dt) khat (khat.J)
        B <- c B - i s khat x E + i (1 - c)/k khat x J           (both from the old E, B)
    The formulas are for collocated fields: each staggered component is moved to the nodes by its
    half-cell phase e^{-i k h/2} per staggered axis, updated, and moved back.  The current is scaled
    per axis by [k]_Yee / k as for the spectral solver (so that the Esirkepov current obeys the
    spectral continuity equation and Gauss's law i k.E = rho holds).  Modes on the Nyquist plane of
    an even axis are removed (set to zero).  At k = 0: E <- E - dt J, B <- B."""
    kz, kx, ky = _axes_k(g)
    hs = (g.dz, g.dx, g.dy)
    kv = (kz, kx, ky)
    ph = [np.exp(-0.5j * kv[a] * hs[a]) for a in range(3)]
    if g.ndim == 2:
        ph[2] = np.ones(1).reshape(-1, 1, 1)

    def colloc(Fk, stag, inv=False):
        out = []
        for c in range(3):
            f = Fk[c]
            for a in range(3):
                if stag[c][a]:
                    f = f * (np.conj(ph[a]) if inv else ph[a])
            out.append(f)
        return out

    _, _, ratio = operators(g, "spectral")
    Ek = colloc(_fwd(E), STAGGER_E)
    Bk = colloc(_fwd(B), STAGGER_B)
    Jraw = _fwd(J)
    Jk = colloc(np.stack([Jraw[c] * ratio[c] for c in range(3)]), STAGGER_E)
    kn = np.sqrt(kz ** 2 + kx ** 2 + ky ** 2)
    zero = kn == 0.0
    kn_safe = np.where(zero, 1.0, kn)
    kh = [np.broadcast_to(k / kn_safe * (~zero), kn.shape) for k in (kz, kx, ky)]
    C, S = np.cos(kn * g.dt), np.sin(kn * g.dt)
    S_over_k = np.where(zero, g.dt, S / kn_safe)
    omc_over_k = np.where(zero, 0.0, (1.0 - C) / kn_safe)

    def cross(a, b):
        return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]

    def dot(a, b):
        return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]

    kxB, kxE, kxJ = cross(kh, Bk), cross(kh, Ek), cross(kh, Jk)
    kE, kJ = dot(kh, Ek), dot(kh, Jk)
    En = [C * Ek[c] + 1j * S * kxB[c] - S_over_k * Jk[c] + (1.0 - C) * kh[c] * kE + (S_over_k - g.dt) * kh[c] * kJ
          for c in range(3)]
    Bn = [C * Bk[c] - 1j * S * kxE[c] + 1j * omc_over_k * kxJ[c] for c in range(3)]
    nyq = _nyquist_mask(g)
    En = [np.where(nyq, 0.0, f) for f in En]
    Bn = [np.where(nyq, 0.0, f) for f in Bn]
    E[:] = _inv(np.stack(colloc(En, STAGGER_E, inv=True)), g)
    B[:] = _inv(np.stack(colloc(Bn, STAGGER_B, inv=True)), g)


def div_spectral(g, F):
    """i k.F of the collocated field (the divergence PSATD keeps), at the nodes; F staggered like E."""
    return div_minus(g, F, "spectral")


def cfl_dt(ndim, kind, dz, dx, dy=1.0):
    """Largest stable dt: the leapfrog needs (dt/2)^2 max_k sum_a kappa_a^2 <= 1.  For "kt" the z
    symbol depends on dt itself: sin^2(pi dt / (2 dz)) + sum_perp (dt/h)^2 ... <= 1 (dt < dz),
    solved by bisection."""
    perp = [dx] + ([dy] if ndim == 3 else [])
    if kind == "psatd":
        # unconditionally stable field update; the particle move is limited to one cell per step
        return min([dz] + perp)
    if kind == "spectral":
        return 2.0 / np.sqrt(sum((np.pi / h) ** 2 for h in [dz] + perp))
    if kind == "kt":
        f = lambda dt: np.sin(0.5 * np.pi * dt / dz) ** 2 + sum((dt / h) ** 2 for h in perp) - 1.0
        lo, hi = 0.0, dz
        if f(hi) <= 0.0:
            return hi
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if f(mid) <= 0.0 else (lo, mid)
        return lo
    raise ValueError(kind)
