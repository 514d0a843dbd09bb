"""GB300-native adaptive-multigrid solver for the even-odd preconditioned
Wilson-clover Dirac equation (Osborn et al., "Multigrid solver for clover
fermions", Lattice 2010).

* ``binding``  -- ctypes binding of the C ABI (``include/mgclover.h``)
* ``solver``   -- ``Solver`` convenience wrapper
* ``autograd`` -- differentiable solve (torch.autograd.Function) and gauge force
* ``inputs``   -- seeded synthetic gauge fields and sources
* ``build``    -- in-tree nvcc build of ``libmgclover.so`` for sm_103a

Importing the package does not load the CUDA library; the first ABI call does,
and fails loudly if it has not been built.
"""
__all__ = ["binding", "solver", "autograd", "inputs", "build"]
