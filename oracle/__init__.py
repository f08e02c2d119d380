"""Plain FP64 CPU oracle of the DD-alpha-AMG two-level method (Frommer et al., arXiv:1303.1377).

THIS PACKAGE IS TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test
suite, the smoke check and the CPU-baseline leg of the benchmark may import it.
The CUDA library never calls into it and shares no code, table or helper with it.

Every routine is written straight from the paper, in its order and notation,
vectorised with numpy over lattice sites but without any blocking, fusion or
reordering beyond what the paper states.  Section references are to the paper:
  Sec. 2.2  lattice, gamma basis, Wilson-clover operator D, Gamma5-symmetry
  Sec. 2.3  block decomposition and red-black multiplicative Schwarz (SAP)
  Sec. 3.1  aggregation-based interpolation P with local orthonormalisation
  Sec. 3.2  Gamma5-compatible standard aggregation, D_c = P^H D P (Lemma 3.x)
  Sec. 4.2  the V-cycle iteration matrix C^(nu)
  Sec. 4.3  Algorithm 1 (inexact deflation setup)
  Sec. 5    Algorithm 2 (DD-alpha-AMG setup), FGMRES with one V-cycle
  Sec. 6    odd-even preconditioning, Table 1 default parameters
  Sec. 3, 7 the recursion to more than two levels (multilevel.py, with the readings
            the paper leaves open stated in its docstring)

Pin status of each function is listed in the module docstrings; the pins
themselves live in tests/test_oracle_*.py.  Parity unpinned: iteration counts
and timings (the paper's gauge configurations are not available), and the GPU
adaptive setup entry-wise (tolerance-stopped inner solves diverge at rounding level).
"""
