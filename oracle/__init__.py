"""FP64 CPU oracle for the TFETI elastoplastic solver (test infrastructure only).

This package is a plain, slow, obviously-correct restatement of the paper's
method in numpy/scipy, in FP64.  It exists to check the CUDA path and is used
only by ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py``.  The product never imports it.  It
shares no code with the CUDA path; both take their inputs from ``workloads``.

Modules, each citing the passage it restates:

* ``material``  -- Hooke law, von Mises yield function, return mapping and the
  Clarke derivative T^o (Sec. 2.2-2.4 and their algebraic form in Sec. 3.1).
* ``fem``       -- hex8 strain-displacement matrices, element stiffness and
  internal force, traction loads (Sec. 3.1, eqs. (F_def), (K_def)).
* ``decomp``    -- box subdomains, orthonormal constraint matrix B, rigid-body
  kernel R, fixing-node generalised inverse (Sec. 4.1-4.2, Remark 1).
* ``tfeti``     -- Algorithm 3 (PCGP on the dual problem) with the lumped
  preconditioner.
* ``ssn``       -- Algorithms 2, 4 and 5 (semismooth Newton over load steps).
* ``direct``    -- undecomposed direct solve used only to pin the TFETI solve.

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants, brute force or the paper's printed values.
"""
