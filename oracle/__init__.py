"""FP64 CPU oracle of eMAGPIE (arXiv 2511.01793).  TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never imports, links or
calls it, and this package shares no code with the CUDA library: the two meet
only through the seeded input generators of ``synth``.
"""
from .emagpie import *  # noqa: F401,F403
from .emagpie import __all__  # noqa: F401
