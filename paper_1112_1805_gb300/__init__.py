"""GB300 (sm_103a) shearlet-regularised convex multi-label segmentation.

The ADMM of Haeuser & Steidl, "Convex Multiclass Segmentation with Shearlet
Regularization" (arXiv:1112.1805), as hand-written CUDA kernels behind the C
ABI declared in include/shearseg.h.  ``binding`` mirrors that ABI name for
name; ``api`` wraps it for torch tensors; ``synth`` generates seeded inputs.
Importing the package loads nothing; the first binding call loads (and if
needed builds) libshearseg.so and raises if that fails.
"""

__all__ = ["binding", "api", "synth", "build"]
