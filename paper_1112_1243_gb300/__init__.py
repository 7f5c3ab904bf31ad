"""GB300 (sm_103a) library for the domain-decomposed Wilson-Dirac hot path of
the hierarchical acceptance algorithm of Leder, Finkenrath and Knechtli,
"Fermions as global correction in lattice QCD" (Lattice 2011).

The compute path is the CUDA library libdd.so (C ABI in include/dd.h); the
Python layer in ``api`` only marshals torch tensors into it.
"""
__all__ = ["api", "synthetic", "build"]
