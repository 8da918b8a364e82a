"""The oracle: a plain, slow, CPU FP64 implementation of the tiled BiDiag / R-BiDiag reduction, its
trees and its adjoint, written from the paper (arXiv 1611.06892) for checking the CUDA library.

ORACLE - test infrastructure only: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of
``bench.py`` import it.  It shares no code with the CUDA path, and the product path never calls it.
"""
