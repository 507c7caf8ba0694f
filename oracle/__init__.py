"""FP64 CPU oracle of the overlapping fragments method (test infrastructure).

Only tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  It shares no code with the CUDA path.
"""
from . import ofm_oracle  # noqa: F401
