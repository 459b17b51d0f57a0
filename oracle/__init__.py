"""FP64 CPU oracle of the plain-LRSTV ADMM iteration (arXiv 2204.12879).

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
reference the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it; the product path
(``paper_2204_12879_gb300``) never does.  It shares no code with the CUDA
path: the arithmetic lives in ``lrstv_oracle.c`` (plain C, FP64, OpenMP),
loaded here through ctypes, and, for the unrolled iteration and its
hand-derived adjoint, in ``adjoint.py`` (numpy, FP64), and for the Tucker
(HOOI) L-update of the full TDLRSTV model in ``tucker.py`` (numpy, FP64).
"""
from .oracle import *  # noqa: F401,F403
from .oracle import __all__  # noqa: F401
