"""FP64 CPU oracle for the hybrid LB + Beris-Edwards step (arXiv:0901.3293).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py``; never by the product
library, which has no CPU fallback.  Shares no code with the CUDA path.
"""
from . import lbq, initial  # noqa: F401
