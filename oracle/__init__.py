"""FP64 CPU oracle for the even-odd, multigrid-preconditioned GCR solve of the
Wilson-clover Dirac equation (Osborn et al., "Multigrid solver for clover
fermions", Lattice 2010).

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` may use it.  It shares no code with the CUDA path: every
operator, table and constant here is written out independently, in plain
numpy complex128, on whole-lattice arrays (no blocking, fusion or
reordering beyond what the definitions state).

Modules
-------
``dirac``     gamma matrices, Wilson hopping term, clover term, D, D_p, D_r,
              b_r and the even/odd reconstruction (Introduction, Eq. 1;
              "Red-black preconditioning", Eq. 2 and the D_r/b_r equations).
``krylov``    flexible GCR and minimal-residual relaxation ("Adaptive
              multigrid": GCR as the outer solver).
``philox``    Philox4x32-10 counter-based generator (Salmon et al., SC'11)
              and the Gaussian vectors the setup starts from.
``multigrid`` null-vector setup by inverse iteration ("Setup procedure"),
              chirality-split block Gram-Schmidt, R = P^dag, prolongation P,
              the Galerkin coarse operator R D_p P, coarse even-odd, and the
              recursive K-cycle MG-GCR ("Implementation").
``force``     gradient of Re<chi, D^{-1} eta> with respect to eta and the
              gauge links (not in the paper; a stated extension).

Readings of the paper where it is silent are listed in each module header.
"""
