"""B300-native connected-sum engine for CoS++ (arXiv 2507.12349).

The computation runs in hand-written sm_103a CUDA kernels behind the C ABI of
``include/cos.h`` (``libcos.so``); ``binding`` exposes those calls with the same
names.  ``inputs`` holds the seeded synthetic workloads.
"""
from . import inputs  # noqa: F401

__all__ = ["inputs", "binding", "build"]
