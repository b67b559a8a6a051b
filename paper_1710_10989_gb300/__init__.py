"""GB300-native scaling-and-squaring matrix exponential with the reduced-product
Taylor scheme of Bader, Blanes and Casas (arXiv:1710.10989).

The compute path lives in the CUDA shared library built from ``csrc/``
(``libbbcexpm.so``); ``paper_1710_10989_gb300.api`` is its thin ctypes binding.
Importing this package does not load the library; ``api`` does, and fails
loudly if it is missing.
"""
__all__ = ["api", "workloads"]
