"""Plain CPU oracle of the shaken dynamics (arXiv:1904.06257).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import this package.  The
product (``paper_1904_06257_gb300``) never imports it and shares no code with
it.

* ``oracle.core``  -- ctypes wrapper of ``shaken_oracle.c`` (one site update at
  a time, fp64, the Philox stream and thresholds written out plainly).
* ``oracle.exact`` -- exact small-system solver in numpy: dense transition
  matrices of the half steps, the closed-form stationary measure of Thm 2.1,
  Gibbs measures and total-variation distances.
"""
