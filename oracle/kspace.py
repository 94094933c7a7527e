"""k-space analysis of Sec. 2-3 and Appendix D, by direct quadrature (FP64, scipy).

TEST INFRASTRUCTURE ONLY (part of the oracle).  These integrals fix the numbers the
paper prints (self-forces, kappa_r, r*), and give the on-axis E1 the single-particle
runs are compared with.

Normalisation (Sec. 2.2): khat = k1 dx1/2, kappa = dx1/dt, r = dx2/dx1, beta = 1.
In these units [k1]_t dx1/2 = kappa sin(khat/kappa) and the Yee [k]_1 dx1/2 = sin(khat).
Shapes in k space (Sec. 2.1): linear S = (sin khat/khat)^2; quadratic S = (sin khat/khat)^3
(the B-spline of one order higher; the paper names only the linear form).
All forces are in units of q^2/dx1, fields in units of q/dx1.

Current filter (Sec. 2.2, 2.3, Table 2: "5 pass filter", not defined in the paper).  Reading:
four passes of the binomial smoother (1/4, 1/2, 1/4) and one compensating pass (-5/4, 7/2, -5/4)
along x1.  A symmetric three-point pass (w1, w0, w1) multiplies the grid mode khat by
w0 + 2 w1 cos(2 khat).  The filter acts on the grid current, i.e. at the fundamental-zone
wavenumber khat of each integrand; with it the three filtered self-forces of Table 2 follow.
"""
import math

import numpy as np
from scipy import integrate, optimize


def shape_k(khat, order):
    """B-spline shape factor in k space: (sin khat / khat)^(order+1)."""
    khat = np.asarray(khat, dtype=np.float64)
    s = np.where(np.abs(khat) < 1e-12, 1.0, np.sin(khat) / np.where(khat == 0, 1.0, khat))
    return s ** (order + 1)


def kt(x, kappa):
    """[x]_t in khat units: kappa sin(x / kappa) (leapfrog time operator, Sec. 2.1)."""
    return kappa * np.sin(np.asarray(x, dtype=np.float64) / kappa)


# ---------------------------------------------------------------- thresholds ---

def r_star():
    """Sec. 2.2: r threshold 2/sqrt(pi^2-4) separating the Yee Cerenkov scenarios."""
    return 2.0 / math.sqrt(math.pi ** 2 - 4.0)


def kappa_r_yee(r):
    """Sec. 2.2: kappa_r^2 sin^2(pi/(2 kappa_r)) = 1 + r^-2."""
    f = lambda k: k * k * math.sin(math.pi / (2 * k)) ** 2 - (1.0 + r ** -2)
    return optimize.brentq(f, 1.0 + 1e-9, 50.0)


def kappa_r_spectral():
    """Sec. 2.3: kappa_r^2 sin^2(3 pi/(2 kappa_r)) = pi^2/2 (r = 1)."""
    f = lambda k: k * k * math.sin(1.5 * math.pi / k) ** 2 - math.pi ** 2 / 2
    return optimize.brentq(f, 1.6, 10.0)


def kappa_r_custom():
    """Sec. 3: sin^2(3 pi/(2 kappa_r)) - sin^2(pi/(2 kappa_r)) = 1/kappa_r^2 (r = 1)."""
    f = lambda k: math.sin(1.5 * math.pi / k) ** 2 - math.sin(0.5 * math.pi / k) ** 2 - 1.0 / k ** 2
    return optimize.brentq(f, 2.0 + 1e-9, 10.0)


# ------------------------------------------------------------------- filter ---

FILTER_PASSES = ((0.25, 0.5),) * 4 + ((-1.25, 3.5),)   # (w1, w0) of each pass, in order


def filter_symbol(khat):
    """Product over the passes of w0 + 2 w1 cos(2 khat) (khat = k1 dx1/2)."""
    out = 1.0
    for w1, w0 in FILTER_PASSES:
        out = out * (w0 + 2.0 * w1 * np.cos(2.0 * np.asarray(khat, dtype=np.float64)))
    return out


def _filt(flag):
    return (lambda k: float(filter_symbol(k))) if flag else (lambda k: 1.0)


# ---------------------------------------------------------------- self-forces ---

def _root(f, a, b):
    return optimize.brentq(f, a, b, xtol=1e-15, rtol=1e-15, maxiter=500)


def self_force_yee(kappa=4.0, r=1.0, order=1, filt=False):
    """Sec. 2.2 (fundamental zone, Cerenkov part):
    F1 = -(1/pi) int_0^{khat_r} S^2/sin(khat) sqrt(D/(1 - r^2 D)) dkhat,
    D = kappa^2 sin^2(khat/kappa) - sin^2(khat), khat_r: D = r^-2.
    filt: the integrand carries the current filter's symbol at khat."""
    Fk = _filt(filt)
    D = lambda k: kt(k, kappa) ** 2 - math.sin(k) ** 2
    g = lambda k: D(k) - r ** -2
    kr = _root(g, 1e-6, math.pi / 2) if g(math.pi / 2) > 0 else math.pi / 2
    f = lambda k: Fk(k) * shape_k(k, order) ** 2 / math.sin(k) * math.sqrt(max(D(k), 0.0) / (1.0 - r * r * D(k)))
    val, _ = integrate.quad(f, 0.0, kr, limit=400, epsabs=1e-13, epsrel=1e-12)
    return -val / math.pi


def self_force_spectral(kappa=4.0, r=1.0, order=1, filt=False):
    """Sec. 2.3 (first aliasing zones, Cerenkov part):
    F1 = -(1/pi) int_{-khat_r1}^{-khat_r2} S(khat) S(khat+pi)/khat sqrt([khat+pi]_t^2 - khat^2) dkhat,
    [-khat_r1+pi]_t^2 = khat_r1^2,  [-khat_r2+pi]_t^2 - khat_r2^2 = (pi/(2r))^2.
    filt: the integrand carries the current filter's symbol at khat."""
    Fk = _filt(filt)
    X = lambda k: kt(k + math.pi, kappa) ** 2 - k * k
    r1 = -_root(lambda k: X(k), -math.pi / 2, -1e-9) if X(-math.pi / 2) < 0 else math.pi / 2
    r2 = -_root(lambda k: X(k) - (math.pi / (2 * r)) ** 2, -r1, -1e-9)
    f = lambda k: Fk(k) * shape_k(k, order) * shape_k(k + math.pi, order) / k * math.sqrt(max(X(k), 0.0))
    val, _ = integrate.quad(f, -r1, -r2, limit=400, epsabs=0.0, epsrel=1e-10)
    return -val / math.pi


def self_force_custom(kappa=4.0, r=1.0, order=1, printed=False, filt=False):
    """Sec. 3, solver with [k]_1 = [k1]_t (first aliasing zones, Cerenkov part):
    F1 = -(1/pi) int_{-pi/2}^{-khat_r} S(khat) S(khat+pi) / K(khat) sqrt(X/(1 - r^2 X)) dkhat,
    X = [khat+pi]_t^2 - [khat]_t^2, khat_r: X = r^-2.

    Eq. E12D divides by [k]_B1 = [k1]_t, i.e. K = kappa sin(khat/kappa) in khat units
    (printed=False).  The Sec. 3 closed form prints K = sin(khat/kappa) (printed=True); that
    form is kappa times larger and is the one that reproduces the printed 0.040 / 0.016.
    filt: the integrand carries the current filter's symbol at khat."""
    Fk = _filt(filt)
    X = lambda k: kt(k + math.pi, kappa) ** 2 - kt(k, kappa) ** 2
    kr = -_root(lambda k: X(k) - r ** -2, -math.pi / 2 + 1e-12, math.pi / 2)
    K = (lambda k: math.sin(k / kappa)) if printed else (lambda k: kt(k, kappa))
    f = lambda k: (Fk(k) * shape_k(k, order) * shape_k(k + math.pi, order) / K(k)
                   * math.sqrt(max(X(k), 0.0) / (1.0 - r * r * X(k))))
    val, _ = integrate.quad(f, -math.pi / 2, -kr, limit=400, epsabs=0.0, epsrel=1e-10)
    return -val / math.pi


# ---------------------------------------------------------- Appendix D forms ---

def int_sin_closed(A, k1_positive=True):
    """Appendix D: int_{-pi/2}^{pi/2} A/(A - sin^2 k2) dk2 = -/+ i pi sqrt(A/(1-A)), 0 < A < 1.

    The printed sqrt(A/(1-A^2)) is read as sqrt(A/(1-A)): the residue at asin(sqrt A) is
    A/(-2 sqrt(A) sqrt(1-A)).  The sign follows the causal pole placement (k1 > 0: -)."""
    v = math.pi * math.sqrt(A / (1.0 - A))
    return complex(0.0, -v if k1_positive else v)


def int_quad_closed(A):
    """Appendix D: int_{-pi/2}^{pi/2} A/(A - k2^2) dk2.

    sqrt(A) < pi/2 (pole inside the strip): -i pi sqrt(A) + 2 sqrt(A) atanh(pi/(2 sqrt A)), the
    atanh of an argument above 1 taken on the real axis (its real part, 1/2 ln((x+1)/(x-1))).
    sqrt(A) >= pi/2 (no pole): 2 sqrt(A) atanh(pi/(2 sqrt A)), real."""
    s = math.sqrt(A)
    x = math.pi / (2 * s)
    if x > 1.0:
        return complex(2 * s * 0.5 * math.log((x + 1) / (x - 1)), -math.pi * s)
    return complex(2 * s * math.atanh(x), 0.0)


def _pv_and_residues(den, A, roots):
    """Principal value of int A/den(k) over [-pi/2, pi/2] (scipy's Cauchy-weight rule around each
    simple root) and the Sokhotski-Plemelj magnitude pi A sum 1/|den'(root)|."""
    edges = [-math.pi / 2] + sorted(roots) + [math.pi / 2]
    mids = [0.5 * (edges[i] + edges[i + 1]) for i in range(len(edges) - 1)]
    cuts = sorted([-math.pi / 2, math.pi / 2] + mids)
    pv = 0.0
    for a, b in zip(cuts[:-1], cuts[1:]):
        inside = [r0 for r0 in roots if a < r0 < b]
        if inside:
            r0 = inside[0]
            def f(k, r0=r0):
                d = den(k)
                if abs(k - r0) < 1e-13:
                    return A / ((den(r0 + 1e-7) - den(r0 - 1e-7)) / 2e-7)
                return A * (k - r0) / d
            pv += integrate.quad(f, a, b, weight="cauchy", wvar=r0, limit=400)[0]
        else:
            pv += integrate.quad(lambda k: A / den(k), a, b, limit=400)[0]
    h = 1e-6
    res = sum(math.pi * A / abs((den(r0 + h) - den(r0 - h)) / (2 * h)) for r0 in roots)
    return pv, res


def int_sin_direct(A):
    """Direct evaluation of the Appendix D sine integral: (principal value, pole magnitude)."""
    k0 = math.asin(math.sqrt(A))
    return _pv_and_residues(lambda k: A - math.sin(k) ** 2, A, [-k0, k0])


def int_quad_direct(A):
    """Direct evaluation of the Appendix D quadratic integral: (principal value, pole magnitude)."""
    s = math.sqrt(A)
    roots = [-s, s] if s < math.pi / 2 else []
    return _pv_and_residues(lambda k: A - k * k, A, roots)


# --------------------------------------------------------- on-axis E1 (Yee) ---

def e1_axis_yee(ip_rel, kappa=4.0, r=1.0, order=1, zones=(0, -1, 1)):
    """On-axis E1 dx1/q at i1' = ip_rel (cells from the particle, staggered by 1/2), beta = 1,
    from Eq. E12D with the k2 integral done in closed form (Sec. 2.2, Appendix D):

      nu1 = 0:   E1 = -(1/pi) [ int_0^{kr} S/sin k sqrt(D/(1-r^2 D)) cos(k(2i'+1)) dk
                                - int_{kr}^{pi/2} S/sin k sqrt(-D/(1-r^2 D)) sin(k(2i'+1)) dk ],
      nu1 = +-1 (r = 1, kappa >= 2, pure space charge):
                 E1 = (1/pi) int_0^{pi/2} [S(k-pi) sqrt(-Dm/(1-r^2 Dm)) + S(k+pi) sqrt(-Dp/(1-r^2 Dp))]
                      / sin k  sin(k(2i'+1)) dk,
      D = kappa^2 sin^2(k/kappa) - sin^2 k, Dm/Dp the same with k -/+ pi in the time operator.
    """
    ip_rel = float(ip_rel)
    out = 0.0
    D = lambda k: kt(k, kappa) ** 2 - math.sin(k) ** 2
    if 0 in zones:
        g = lambda k: D(k) - r ** -2
        kr = _root(g, 1e-6, math.pi / 2) if g(math.pi / 2) > 0 else math.pi / 2
        f1 = lambda k: (shape_k(k, order) / math.sin(k) * math.sqrt(max(D(k), 0.0) / (1 - r * r * D(k)))
                        * math.cos(k * (2 * ip_rel + 1)))
        f2 = lambda k: (shape_k(k, order) / math.sin(k) * math.sqrt(max(-D(k), 0.0) / abs(1 - r * r * D(k)))
                        * math.sin(k * (2 * ip_rel + 1)))
        a = integrate.quad(f1, 0.0, kr, limit=1000, epsabs=1e-12)[0]
        # D > r^-2 beyond kr: -D/(1 - r^2 D) = D/(r^2 D - 1) > 0
        f2 = lambda k: (shape_k(k, order) / math.sin(k) * math.sqrt(D(k) / (r * r * D(k) - 1.0))
                        * math.sin(k * (2 * ip_rel + 1)))
        b = integrate.quad(f2, kr, math.pi / 2, limit=1000, epsabs=1e-12)[0] if kr < math.pi / 2 else 0.0
        out += -(a - b) / math.pi
    if -1 in zones or 1 in zones:
        Dm = lambda k: kt(k - math.pi, kappa) ** 2 - math.sin(k) ** 2
        Dp = lambda k: kt(k + math.pi, kappa) ** 2 - math.sin(k) ** 2
        def f(k):
            v = 0.0
            for DD, sh in ((Dm, k - math.pi), (Dp, k + math.pi)):
                d = DD(k)
                v += shape_k(sh, order) * math.sqrt(max(d, 0.0) / max(r * r * d - 1.0, 1e-300))
            return v / math.sin(k) * math.sin(k * (2 * ip_rel + 1))
        out += integrate.quad(f, 0.0, math.pi / 2, limit=1000, epsabs=1e-12)[0] / math.pi
    return out
