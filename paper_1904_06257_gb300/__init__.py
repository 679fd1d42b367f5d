"""GB300 (sm_103a) implementation of the per-half-step parallel update of the
shaken dynamics (Apollonio, D'Autilia, Scoppola, Scoppola, Troiani,
arXiv:1904.06257).

* ``paper_1904_06257_gb300.shaken``    -- Python binding of the C ABI (include/shaken.h);
                                          importing it loads libshaken.so (CUDA) or fails.
* ``paper_1904_06257_gb300.build``     -- builds libshaken.so in-tree with nvcc.
* ``paper_1904_06257_gb300.workloads`` -- seeded synthetic inputs (no method arithmetic).
"""
__all__ = ["build", "workloads"]
