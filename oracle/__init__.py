"""Plain FP64 CPU oracle for the hybrid scattered-regular meshless method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or call anything in this package.
The product path (the CUDA library and its Python binding) never imports it.

The oracle is written from the paper (arXiv:2303.01760) alone: it is slow and
direct, in float64, with library primitives (a dense or sparse solve, a sort, a
k-d tree query) used only as single steps.  It shares no code with the CUDA
path; the only input both sides consume is the seeded node-set generator.

Modules
  stencils  stencil selection (Section 2, "n neighbouring nodes")
  weights   MON and RBF-FD weights from Eq. 1 (Section 2 and 2.1)
  apply     operator application, Eq. 1
  stepper   explicit Boussinesq step with Chorin projection (Section 3)
  learned   consistency projection and the FP64 MLP (no counterpart in the
            paper: parity unpinned beyond the gradient and projection checks)
"""
