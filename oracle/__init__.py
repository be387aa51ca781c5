"""FP64 CPU oracle for the collide-and-stream method on cell-centred non-uniform grids.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its Python
binding) imports, links or executes anything in this package.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg use it.

The oracle is a plain, slow, per-cell restatement of the method of Coreixas & Latt,
"GPU-based compressible lattice Boltzmann simulations on non-uniform grids using standard
C++ parallelism" (arXiv 2504.04465).  It shares no code with the CUDA path: it has its own
lattice tables, Hermite machinery, Newton solver, grid builder and time stepper, written
from the paper's equations in their printed order (collide, then stream; Section 2,
Eq. CollAndStream and Appendix A, Eqs. CollisionStep/StreamingStep).

Modules
    lattices   velocity sets and weights (Appendix A, Tab. lattices_structure)
    hermite    Hermite tensors, polynomial equilibria, BGK and recursive regularization
               (Appendix A, Eqs. GenEq, RecursivityEquilibrium, GenRegCollision, a1Rec)
    numerical  max-entropy equilibrium by Newton-Raphson with line search
               (Appendix A, Eqs. exponential, G0..G3yaa)
    grid       multi-level cell-centred grid with Rohde ghost layers (Sections 3.2, 4.3-4.4)
    solver     multi-level time stepping with coalescence/explosion (Section 4.5 and
               Eqs. coalescence/explosion_uniform), boundaries, DDF, shock sensor
    mlp        small multilayer perceptron forward/backward/Adam for the learned Newton guess
               (an extension beyond the paper; see its header)

Every function is pinned by a ``-m "not gpu"`` test against something other than itself
(printed values, closed forms, invariants, brute force); the one exception is listed in
the header of the module concerned as "parity unpinned".
"""
