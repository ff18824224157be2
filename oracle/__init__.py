"""FP64 CPU oracle for the Kadanoff-Baym time stepper.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, uncompressed
implementation of the discrete scheme, written from the paper (Sec. 2.1-2.4,
Eqs. KBEM-KBEL, Appendix A, Eq. Hybrid, Eq. SigmaF, Eq. Sigma2B).  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.  The CUDA library never imports, links or calls anything here,
and nothing here imports the library.

Modules
  weights  Appendix A weights in exact rational arithmetic
  dlr      DLR evaluation / reversal / product / convolution matrices (quadrature)
  models   self-energy functionals (Bethe, bath level, none)
  kbe      dense lower-triangular FP64 stepper (bootstrap + time steps)

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, exact rationals, brute-force global solves or invariants.
"""
