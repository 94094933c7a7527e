"""The transverse-force measurement shared by the oracle pin and the GPU parity test.

Eq. EM gives, for a charge moving along x1 with velocity beta, B3 = ([w]_t / [k]_B1) E2 in Fourier
space (w = beta k1), so the transverse force on a co-moving charge is E2 - beta B3 = E2 (1 - beta
[beta k1]_t / [k]_B1); with [k]_B1 = [k1]_t (the Sec. 3 solver) it is E2 (1 - beta), free of
numerical error.  The ratio is measured on x lineouts of E2 (at integer z, time n) and of the
leapfrog B3 (at half-integer z, time n + 1/2) around the particle: Hann-windowed Fourier sums at
the same physical positions, the half time step undone for a pattern moving at c."""
import numpy as np

from oracle import fit


def measured_ratio(E2row, B3row, zp, kappa, L=100, ks=None):
    """B3~/E2~ at wave numbers ks (rad per cell) from lineouts E2row[i] (z = i) and B3row[i]
    (z = i + 1/2) of the leapfrog fields (B half a step later than E), window +-L cells about zp."""
    if ks is None:
        ks = np.linspace(0.05, 1.2, 24)
    ip = int(round(zp))
    idx = np.arange(ip - L, ip + L)
    w = 0.5 - 0.5 * np.cos(2 * np.pi * (idx - (ip - L)) / (2 * L))
    wb = 0.5 - 0.5 * np.cos(2 * np.pi * (idx + 0.5 - (ip - L)) / (2 * L))
    Ee = np.array([np.sum(w * E2row[idx] * np.exp(-1j * k * idx)) for k in ks])
    Bb = np.array([np.sum(wb * B3row[idx] * np.exp(-1j * k * (idx + 0.5))) for k in ks])
    return ks, Bb / Ee * np.exp(1j * ks * 0.5 / kappa)


def predicted_ratio(ks, kappa, CB, beta=1.0):
    """[beta k1]_t / [k]_B1 (Eq. EM) at k1 dz = ks, in units of dz = 1."""
    kh = ks / 2
    return kappa * np.sin(beta * kh / kappa) / fit.axial_symbol(CB, kh)


def band_means(ks, ratio, pred, kmin=0.7):
    band = ks >= kmin
    return float((ratio.real[band] - 1).mean()), float((pred[band] - 1).mean())
