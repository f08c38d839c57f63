"""FP64 CPU oracle of NS-RGS.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It imports nothing from the CUDA
library and the CUDA library never imports it; both sides receive their
inputs from the seeded generator in ``synth``.
"""
from .nsrgs_oracle import *  # noqa: F401,F403
from .nsrgs_oracle import __all__  # noqa: F401
