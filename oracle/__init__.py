"""CPU oracle of the Wilson-Dirac hot path (FP64).

TEST INFRASTRUCTURE, not part of the product.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  ``oracle.wilson`` is the NumPy form of Eq. (1), Eq. (2), the Wilson and
even-odd operators and textbook CG/BiCGstab; ``oracle.c_oracle`` wraps a plain
C + OpenMP site loop of Eq. (1) used for large lattices and CPU timing.
"""
