"""Plain FP64 CPU oracle of the orthogonalization-free Rayleigh-Ritz path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything under ``oracle/``.  The product path (the CUDA library and its Python
binding) never imports it and shares no code with it; the only module both
sides use is ``workloads``, which builds inputs and holds none of the method's
arithmetic.

Everything here is written from the paper's algorithms, in their order and
notation, in FP64 unless a function says otherwise.  Library primitives
(numpy matmul, numpy argmax, LAPACK's symmetric-definite eigensolver through
scipy) serve as single steps; there is no blocking, fusion or reordering.

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, invariants, textbook routines, brute
force).  Nothing here is "parity unpinned".
"""
from .ofrr import *  # noqa: F401,F403
