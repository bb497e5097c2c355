"""FP64 CPU oracle for the neural multigrid solve -- test infrastructure.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library and its Python
binding never import it, and the two share no code.
"""
from .nmg_oracle import *  # noqa: F401,F403
from .classical import *  # noqa: F401,F403,E402
