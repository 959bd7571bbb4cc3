"""GB300 (sm_103a) entropy-stable discontinuous collocation residual for compressible Navier-Stokes.

The compute path is libesdc.so (hand-written CUDA, C ABI in include/esdc.h); `Solver` is a thin
torch front end.  `inputs` holds seeded synthetic meshes and initial states.  Importing the
package does not load the shared library; constructing a Solver does, and fails loudly without it.
"""
from . import inputs  # noqa: F401


def __getattr__(name):
    if name in ("Solver", "lgl"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
