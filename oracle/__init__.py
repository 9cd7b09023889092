"""CPU oracle for the log-determinant hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct FP64 implementations of what the CUDA path
computes, written from the paper (Aune & Simpson, "Parameter Estimation in
High Dimensional Gaussian Distributions"):

  matrices      the grid precision matrices Q as explicit sparse matrices
  closed_forms  eigenvalue closed forms; exact and probed values by DST/FFT
  hht           rational approximation nodes/weights of log (Eq. "eq_rat_app")
  cgm           multi-shift CG (CG-M / COCG-M), vector and projected forms
  probing       greedy distance-d colouring (plain C) and its validator
  method        banded Cholesky log det, selected inverse, exact shifted
                solves, and the method end to end (probing x f_N x CG-M)
  native.c      the plain C routines behind probing and method

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It shares no code, headers, tables or helpers with the
CUDA library and never imports it; the only common inputs come from the
seeded generators in `synth`.

Pins (tests/test_oracle_*.py, `-m "not gpu"`):
  * band Cholesky log det  == Fourier/sine eigenvalue closed forms, numpy slogdet;
  * selected inverse       == numpy inverse diagonal, sum 1/lambda closed form;
  * colouring              == i mod (d+1) on a path, checkerboard at d=1,
                              validity by (I+|A|)^d, one colour per vertex when
                              d >= diameter;
  * probed values          == circulant-symbol route (periodic), dense eigh,
                              exact log det under full probing;
  * HHT nodes              == scipy.linalg.logm on dense SPD matrices; error
                              within the 2 pi^2 N rate; elliptic identities;
  * CG-M                   == dense complex solves; projected == vector form.
"""
