"""GB300-native lattice-Boltzmann flow + advection-diffusion-reaction solver
for catalytic fibrous membranes (Sitaru & Gekle, arXiv 2109.04455).

The compute path is the C-ABI library ``liblbm.so`` (hand-written sm_103a
CUDA); :mod:`paper_2109_04455_gb300.lbm` is its thin ctypes binding and
:mod:`paper_2109_04455_gb300.inputs` the seeded workload generator.  Nothing
is loaded at import time: the library is opened on first use and a missing
build raises instead of falling back to anything else.
"""
__all__ = ["inputs", "lbm"]
