"""GB300 Monte Carlo X-ray scatter forward projection (arXiv 2201.13191).

Thin Python binding over the C ABI of ``libmc.so`` (declared in
``include/mc.h``).  The binding only marshals arguments: PyTorch provides
device memory and streams, and every step of the method runs in the CUDA
kernels of the library.  There is no CPU fallback: if the library cannot be
loaded, every call raises.
"""

from .binding import (  # noqa: F401
    MCError,
    Options,
    Tuning,
    CorrectParams,
    Context,
    library,
    library_path,
    STAT_NAMES,
    conv3x3,
    conv3x3_wgrad,
)
from .build import build  # noqa: F401
