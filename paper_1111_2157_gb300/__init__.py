"""GB300-native lattice Green's functions for charge-self-consistent LDA+DMFT.

The package wraps the CUDA library ``libgf.so`` (C-ABI declared in
``include/gf.h``) with a thin ctypes binding.  Importing the package loads
nothing; the library is loaded on first use and a missing library is an error.
"""
__all__ = ["gf", "autograd", "shard", "synth", "build"]
