"""Plain FP64 CPU oracle for the domain-decomposed estimate of 1/det(M^dag M).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline leg are the
only code that may import this package.  It shares no code with the CUDA library and never
imports it.

* ``oracle.core``  -- ctypes binding of ``ddrw_oracle.c`` (operator, clover, CGNR, estimator,
  Philox noise), built with gcc by :func:`oracle.core.build`.
* ``oracle.dense`` -- dense linear algebra on tiny lattices (Eq. 1-6, the inverse of Sec. 1).
"""
