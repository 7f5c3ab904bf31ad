"""Plain FP64 CPU oracle for the domain-decomposed Wilson-Dirac hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, the smoke check of ``__graft_entry__`` and the CPU-baseline leg
of ``bench.py`` may use it.  It shares no code with the CUDA path (the seeded
input synthesis in ``paper_1112_1243_gb300.synthetic`` is the single common
module, and it holds none of the method's arithmetic).

Every function computes a definition of the paper (Leder, Finkenrath,
Knechtli, "Fermions as global correction in lattice QCD", Lattice 2011) in the
most direct form: dense matrices where the size allows, index-array stencils
in canonical site order otherwise, numpy complex128 throughout.  Where the
paper leaves a choice open, the reading taken is stated in the function's
docstring; the same readings are listed in the repository's design notes.

Modules
  geometry    lattice, neighbours, blocks, black/white colouring, block
              ordering, active links (Sec. 3, Fig. 1 and the active-link rule)
  gamma       Euclidean chiral gamma matrices
  dirac       Wilson-Dirac operator D = 1 - kappa*H, Dirichlet block operators,
              block-interaction terms, even-odd and domain Schur complements
              (Eq. domdec, Eq. ddfactor)
  philox      Philox4x32-10 counter-based generator (Salmon et al., SC'11)
  rng         uniforms, complex Gaussian noise, the method's stream keys
  solvers     textbook conjugate gradient on the normal equations
  estimator   stochastic determinant-ratio estimate (Sec. 4) and the
              interpolation factorisation (Eq. param)
  interp      geodesic link interpolation U_t = U (U^dag U')^t
  heatbath    Wilson plaquette action, Cabibbo-Marinari heat-bath with the
              Kennedy-Pendleton SU(2) sampler, over-relaxation
  accept      Metropolis acceptance steps (Eq. 2.1-2.3) and the Gaussian
              acceptance law (Eq. acceptance)
  chain       one step of the hierarchy (Sec. 5, Eq. 4step steps 0, 1, 3)
  recursive   one level of recursive decomposition (Eq. ddrec, step 2)
  gaugefix    relative gauge fixing of the proposal (Sec. 4)
  schwarz     Schwarz alternating procedure over the block decomposition
              and flexible GCR (the domain-decomposition solver the block
              decomposition comes from)

Parity status: every function here is pinned by a ``-m "not gpu"`` test to a
closed form, an identity of the paper, a published test vector or a library
routine; none is "parity unpinned".
"""
