"""GB300 (sm_103a) library for one explicit time step of the thermocapillary
two-phase finite-volume method (WENO5 transport, CSF + Marangoni surface
forces, density-weighted multigrid projection).  The compute path is the CUDA
library ``libfvm.so`` behind the C ABI in ``include/fvm.h``; this package is
its ctypes binding."""
from .fvm import (F64, MIXED, FvmError, Solver, fvm_workspace_size, load,  # noqa: F401
                  make_params, to_device)
