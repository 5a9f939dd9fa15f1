"""B300 (sm_103a) Parareal with a PINN coarse propagator for the Black-Scholes equation.

The numerical path lives in the CUDA library ``libbsparareal.so`` (C ABI in
``include/bsparareal.h``); ``paper_2303_03848_b300.binding`` is the thin ctypes
layer over it.  Importing this package loads nothing; the library is loaded on
first use of the binding and the call fails loudly if it is missing.
"""
__all__ = ["binding", "synth"]
