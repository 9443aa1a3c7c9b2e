"""GB300-native selected-inversion fermion drift for complex-Langevin QCD.

Bloch & Schenk, "Selected inversion as key to a stable Langevin evolution
across the QCD phase boundary" (arXiv:1707.08874).  The compute path is a
CUDA library behind a C ABI (``include/clselinv.h``); ``binding`` is the thin
Python layer over it.  ``inputs`` holds the seeded synthetic inputs.
"""
__all__ = ["inputs", "binding"]
