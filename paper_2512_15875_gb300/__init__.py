"""GB300-native TTNO / TTNS hot path: environments, effective-Hamiltonian applies and block Gram
matrices for the tree-tensor-network vibrational eigensolver, behind a C ABI (``libttn.so``).

The compiled library is loaded lazily by :mod:`paper_2512_15875_gb300.ttn`; importing the package
itself pulls in nothing but NumPy.
"""
__all__ = ["inputs", "ttn"]
