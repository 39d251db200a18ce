"""FP64 CPU oracle for Graph Convolution based Re-ranking (GCR) and GCRV.

This package is test infrastructure. It is imported only by the tests, by
``__graft_entry__.smoke()`` and by the CPU-baseline arm of ``bench.py``; the
library (``paper_2306_08792_gb300``) never imports or calls it, and it shares no
code with the CUDA path.
"""
from .gcr_oracle import *  # noqa: F401,F403
from .pvg_oracle import *  # noqa: F401,F403
from .serve_oracle import *  # noqa: F401,F403
from .dsfp_oracle import *  # noqa: F401,F403
from .eval_oracle import *  # noqa: F401,F403
