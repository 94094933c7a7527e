"""FP64 CPU oracle for the relativistic-beam EM PIC step (arXiv:1910.13529).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference that the CUDA path is checked against.  Only tests/,
__graft_entry__.smoke() and bench.py's cpu_baseline / reference leg may import,
call, link or execute anything here; the product package never does, and the
two share no code.

Modules:
  pic_oracle.c  the PIC step in plain C loops (field advance, gather, Boris,
                Esirkepov deposit, current filter, current correction, Gauss
                residual, window)
  core.py       ctypes wrappers and the step driver (Sim)
  fit.py        Appendix C coefficient fit, Sec. 3 current-correction kernel, CFL
  kspace.py     Sec. 2-3 k-space integrals: self-force (with and without the current
                filter), kappa_r, on-axis E1, Appendix D closed forms
  spectral.py   the k-space field advance (Sec. 2.3 spectral solver, Sec. 3 [k]_1 = [k1]_t
                applied in k space, Appendix B PSATD) with numpy FFTs

Pins (tests/test_oracle_*.py): plane-wave dispersion of Eq. wave, Gauss's law kept
to round-off, Esirkepov continuity, Boris closed forms, the position update against
relativistic hyperbolic motion and the E x B drift with a different cell size on every axis
(test_oracle_motion.py), the whole step against a brute-force dense-matrix composition on
8 x 8 and 8 x 8 x 4 grids (test_oracle_dense.py), Table 1 re-fit, the self-force and kappa_r
values of Sec. 2-3.
The 5-pass current filter (named, not defined, in the paper) is pinned through its k-space
symbol to the three filtered self-forces of Table 2.  The split axial operators ([k]_E1 != [k]_B1,
Sec. 3) are pinned by the dispersion relation with the product of the two symbols, each side's
operator, div curl = 0 and Gauss's law with the B-side correction (tests/test_oracle_split.py).
The k-space advance is pinned to the finite-difference step (Yee and Appendix C symbols), the
leapfrog's single-mode closed form, phase velocity c for [k1]_t, Gauss's law with its current
scaling and its stability limits (tests/test_oracle_spectral.py).
"""
