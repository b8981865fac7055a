"""GB300-native kinetic Monte-Carlo hysteresis of magnetic nanoparticles in
lysosomes (Tan, Carrey & Respaud, arXiv:1407.2737).

The compute path is the CUDA library ``libkmc`` (``csrc/``) behind the C ABI
declared in ``include/kmc.h``; :mod:`.kmc` is its thin Python binding and
:mod:`.inputs` builds seeded synthetic lysosomes. Importing this package loads
nothing; the library is loaded on first use and a missing build is an error.
"""
__all__ = ["kmc", "inputs"]
