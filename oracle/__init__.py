"""CPU oracle for the Magritte line-transfer hot path (arXiv 2411.03040).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import it.  It is independent
of the CUDA library (no shared code; only the seeded input generator is common).
"""
from .oracle import *  # noqa: F401,F403
from .oracle import build, _load  # noqa: F401
