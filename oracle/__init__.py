"""Plain FP64 CPU oracle for HOTRG on the d-dimensional Ising model (arXiv:1906.06060, Sec. 2).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT. Only ``tests/``, ``__graft_entry__.smoke()``, and
the CPU-baseline leg and reference arm of ``bench.py`` may import anything from this package. The CUDA library
shares no code, table or helper with it.

Modules
-------
hotrg_ref   the method itself, step by step in the paper's order (FP64, NumPy/LAPACK).
exact       independent references that pin the oracle: brute-force enumeration of Z,
            Onsager's 2D solution, the 1D transfer matrix, closed forms.
"""
