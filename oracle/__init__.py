"""FP64 CPU oracle for masked LDDMM.

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the benchmark's
CPU-baseline leg.  The library never imports it; it shares no code with the CUDA path.
"""
from . import lddmm  # noqa: F401
from . import metrics  # noqa: F401
from . import preprocess  # noqa: F401
from . import shooting  # noqa: F401
