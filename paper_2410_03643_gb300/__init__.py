"""GB300 (sm_103a) tau-preconditioned GMRES time stepper for the Riesz fractional NLS
(arXiv 2410.03643).  The solver is the CUDA library librfnse.so (C ABI in include/rfnse.h);
`rfnse` is its ctypes binding and `build` compiles it in-tree."""
from .rfnse import (Solver, Batch, Params, RfnseError, NoConvergence, load_library, make_params,  # noqa: F401
                    rollout)
