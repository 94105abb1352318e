"""GB300-native sharp-interface IBM fractional step (arXiv 2606.09799).

`ibm` is the thin ctypes binding of the C-ABI CUDA library; `inputs` holds
the seeded workload generators.  Importing the package loads nothing.
"""
__all__ = ["ibm", "inputs"]
