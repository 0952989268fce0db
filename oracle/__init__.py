"""FP64 CPU oracle for Levenberg-Marquardt bundle adjustment.

TEST INFRASTRUCTURE ONLY.  The product path (the CUDA library and its Python
binding) never imports, calls or links anything under ``oracle/``; only the
tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` do.  The oracle shares no code with the CUDA
path: the two meet only in the seeded arrays that ``scenegen`` draws.
"""
from .ba_oracle import *  # noqa: F401,F403
from .ba_oracle import __all__  # noqa: F401
