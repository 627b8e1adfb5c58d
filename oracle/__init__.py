"""FP64 CPU oracle of the bilayer product-quantization search path.

TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and bench.py's
CPU baseline.  The library never imports it; see bpq_oracle for details.
"""

from .bpq_oracle import *  # noqa: F401,F403
from . import bpq_oracle  # noqa: F401
