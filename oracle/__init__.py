"""CPU FP64 oracle for scaling-and-squaring exp(A) (Bader, Blanes, Casas, arXiv:1710.10989).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import anything from this package.
The CUDA library shares no code with it and never calls it.
"""
