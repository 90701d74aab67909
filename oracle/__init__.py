"""FP64 CPU oracle of the decoupled Fourier pose search -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(``cpu_baseline`` and ``--impl reference``) may import this package.  The CUDA library
never does, and the oracle never imports the library.
"""
from .fmbym_oracle import *  # noqa: F401,F403
from . import fmbym_oracle as core  # noqa: F401
