"""Test infrastructure only: the plain FP64 CPU oracle of the BCMG method.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this package.  The product path (``paper_2207_14208_gb300``) never
does.
"""

from .oracle import Oracle, build, dtau, blfa_G0, blfa_p  # noqa: F401
