"""CPU oracle for the DisMech implicit DER step (arXiv 2311.18126, Sec. III).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
FP64 CPU restatement of the method: energies written once (``der.py``),
forces and Jacobians by automatic differentiation, LAPACK linear solves and
Newton's method on the backward-Euler residual (``system.py``), contact and
friction (``contact.py``).  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import or run it.  It shares no code
with the CUDA library and never imports it.

Parity pins: every function here is checked by ``tests/test_oracle_*.py``
against closed forms, invariances, finite differences, textbook beam results
and the friction law the paper prints.  The absolute values of the contact
stiffness k_c, the damping coefficient and the learned warm-start features
are readings, not values the paper fixes: for those, parity is unpinned
against the paper and only oracle-vs-GPU parity applies.
"""
from .system import OracleSystems, DEFAULT_PARAMS  # noqa: F401
from . import der, contact  # noqa: F401
