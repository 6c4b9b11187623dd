"""FP64 CPU oracle of the vector order-statistic filters (arXiv 1009.0959).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check and
the benchmark's CPU-baseline leg may import this package.  It shares no code,
header, table or constant generator with the CUDA path, and the CUDA path
never calls it.

  oracle.remez         Remez exchange (Sec. 2), FP64
  oracle.paper_tables  the coefficients and errors the paper prints
  oracle.approximants  target functions and approximants (Sec. 3.1 - 3.3)
  oracle.filters       the whole-image filters (C, FP64; oracle/vfo.c)
  oracle.metrics       MAE / MSE / NCD (Sec. 4) and PSNR
  oracle.gate          FP64 forward/backward of the impulse-detector network
"""
from . import approximants, metrics, paper_tables, remez  # noqa: F401
from .filters import Config, filter_image  # noqa: F401
