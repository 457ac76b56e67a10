"""CPU FP64 oracle of the thermocapillary two-phase finite-volume step.

TEST INFRASTRUCTURE ONLY: this package checks the CUDA library and is used
by the tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg of
``bench.py``.  The product path never imports it, and it imports nothing
from the product package.
"""
from . import fvm_oracle  # noqa: F401
