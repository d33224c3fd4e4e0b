"""GB300-native Levenberg-Marquardt graph optimiser (bundle adjustment and
visual-inertial BA) with a camera Schur complement, block-Jacobi preconditioned
conjugate gradients and point back-substitution, behind a C ABI (libgpo.so).

`paper_2509_26581_gb300.gpo` is the ctypes binding (same names as include/gpo.h);
`paper_2509_26581_gb300.synth` holds the seeded synthetic problem generators.
Nothing here loads the CUDA library until `gpo` is imported.
"""
__all__ = ["gpo", "synth"]
