"""FP64 CPU oracle of the static-subspace RPA path (test infrastructure only).

Imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py``; never by the product path.  See ``rpa_oracle`` for the
passages each function follows and for the one quantity left unpinned.
"""
from .rpa_oracle import *  # noqa: F401,F403
