"""Appendix C stencil-coefficient fit and the Sec. 3 current-correction kernel, in numpy (FP64).

TEST INFRASTRUCTURE ONLY (part of the oracle).  Only tests/, __graft_entry__.smoke()
and bench.py's cpu_baseline leg import this module.

Appendix C: the axial operator [k1]_p = sum_l C_l sin((2l-1) k dz/2)/(dz/2) is fitted to
a target operator by weighted least squares under the consistency constraint
M C = e1 (M_ij = (2j-1)^(2i-1)/(2i-1)!, i = 1..p/2), solved through the Lagrange system
    ( A  M^T ) (C)   (b )
    ( M  0   ) (l) = (e1),
    A_ij = 2/pi^2 int_0^1/2 w sin((2i-1) pi k) sin((2j-1) pi k) dk,
    b_i  = 2/pi   int_0^1/2 w sin((2i-1) pi k) [k1]_target dk,
with k normalised to k_g = 2 pi/dz and the super-Gaussian weight
    w(k) = exp(-ln 2 (2k/w_k1)^n).
Sec. 3 fixes the target: [k1]_target = [k1]_t = sin(k dt/2)/(dt/2), i.e. (kappa/pi) sin(pi k/kappa)
after normalisation, kappa = dz/dt.  The paper does not print p, w_k1 or n for Table 1;
the reading p = 2, w_k1 = 0.6, n = 10 (1000-point Gauss-Legendre) reproduces Table 1.

Current correction (Sec. 3, method only cited): the customised d- differs from the
two-point d- used by Esirkepov's continuity equation by the symbol ratio
    P(phi) = sum_l C_l sin((2l-1) phi/2) / sin(phi/2) = sum_{|m|<M} P_m e^{i m phi},
    P_m = sum_{l > |m|} C_l,   phi = k dz,
so J1 <- P^{-1} J1 restores Gauss's law.  h is the impulse response of 1/P.
"""
import math

import numpy as np
from numpy.polynomial.legendre import leggauss


def constraint_matrix(M: int, p: int) -> np.ndarray:
    """M_ij = (2j-1)^(2i-1) / (2i-1)!, i = 1..p/2, j = 1..M (Appendix C)."""
    rows = []
    for i in range(1, p // 2 + 1):
        rows.append([(2 * j - 1) ** (2 * i - 1) / math.factorial(2 * i - 1) for j in range(1, M + 1)])
    return np.array(rows, dtype=np.float64)


def fit_coefficients(kappa: float, M: int = 16, p: int = 2, w_k1: float = 0.6, n: float = 10.0,
                     nq: int = 1000, CE=None) -> np.ndarray:
    """Solve the Appendix C Lagrange system for C_1..C_M with target [k1]_t (Sec. 3).

    With CE (coefficients of an E-side operator [k]_E1) the target is [k1]_t^2 / [k]_E1: the B side
    of a pair with [k]_E1 [k]_B1 = [k1]_t^2, the [k]_E1 != [k]_B1 option of Sec. 3."""
    x, wq = leggauss(nq)
    k = 0.25 * (x + 1.0)          # map [-1, 1] -> [0, 1/2]
    wq = 0.25 * wq
    w = np.exp(-math.log(2.0) * (2.0 * k / w_k1) ** n)
    s = np.array([np.sin((2 * l - 1) * math.pi * k) for l in range(1, M + 1)])
    target = kappa / math.pi * np.sin(math.pi * k / kappa)
    if CE is not None:
        ke = sum(c * np.sin((2 * l - 1) * math.pi * k) for l, c in enumerate(CE, start=1)) / math.pi
        target = target * target / ke
    A = 2.0 / math.pi ** 2 * (s * (w * wq)) @ s.T
    b = 2.0 / math.pi * (s * (w * wq)) @ target
    Mc = constraint_matrix(M, p)
    q = Mc.shape[0]
    K = np.zeros((M + q, M + q))
    K[:M, :M] = A
    K[:M, M:] = Mc.T
    K[M:, :M] = Mc
    rhs = np.zeros(M + q)
    rhs[:M] = b
    rhs[M] = 1.0
    return np.linalg.solve(K, rhs)[:M]


def axial_symbol(C, khat):
    """[k]_1 dz/2 = sum_l C_l sin((2l-1) khat), khat = k dz/2 (Appendix C)."""
    C = np.asarray(C, dtype=np.float64)
    khat = np.asarray(khat, dtype=np.float64)
    return sum(C[l - 1] * np.sin((2 * l - 1) * khat) for l in range(1, len(C) + 1))


def symmetric_stencil(C) -> np.ndarray:
    """P_m = sum_{l > |m|} C_l for m = 0..M-1 (one side of the symmetric stencil)."""
    C = np.asarray(C, dtype=np.float64)
    return np.array([C[m:].sum() for m in range(len(C))])


def correction_kernel(C, hlen: int = 40, nfft: int = 8192) -> np.ndarray:
    """Taps h_{-hlen..hlen} of the impulse response of 1/P(phi), by inverse DFT (FP64)."""
    Pm = symmetric_stencil(C)
    phi = 2.0 * math.pi * np.arange(nfft) / nfft
    P = Pm[0] + 2.0 * sum(Pm[m] * np.cos(m * phi) for m in range(1, len(Pm)))
    h = np.fft.ifft(1.0 / P).real
    return np.array([h[m % nfft] for m in range(-hlen, hlen + 1)])


def cfl_dt(dz: float, dx_perp, C=None, nscan: int = 20001, Cb=None) -> float:
    """Largest stable dt of the leapfrog: (dt/2)^2 (max [k]_E1 [k]_B1 + sum (2/dx_perp)^2) <= 1.

    Yee: C = None ([k]_1 max = 2/dz).  Customised: max over khat of the Appendix C symbol
    (squared), or of the product of the E-side (C) and B-side (Cb) symbols when they differ;
    a product that changes sign has no stable dt (ValueError).
    """
    if C is None:
        kmax2 = (2.0 / dz) ** 2
    else:
        kh = np.linspace(0.0, math.pi / 2, nscan)
        se = axial_symbol(C, kh)
        prod = se * (se if Cb is None else axial_symbol(Cb, kh))
        if prod.min() < -1e-12 * max(prod.max(), 1e-300):
            raise ValueError("[k]_E1 [k]_B1 < 0 somewhere: unstable for every dt")
        kmax2 = prod.max() * (2.0 / dz) ** 2
    s = kmax2 + sum((2.0 / d) ** 2 for d in dx_perp)
    return 2.0 / math.sqrt(s)
