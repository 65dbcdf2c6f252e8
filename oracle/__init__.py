"""FP64 CPU oracle for the coherent-dedispersion path (test infrastructure only).

Only tests, the smoke check and the benchmark's CPU-baseline leg may import this
package; the product path (the CUDA library and its binding) never does.
"""
from .cdd_oracle import *  # noqa: F401,F403
from .cdd_oracle import D_DISP_S_MHZ2, Geometry, TAPERS  # noqa: F401
