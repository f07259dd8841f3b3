"""Plain CPU FP64 oracle for the block-sparse H_eff*psi path (test infrastructure).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  It shares no code with the CUDA library (``paper_2401_01921_gb300``) and
never imports it.

It restates, slowly and in the paper's order, what the method computes
(arXiv 2401.01921, "The Cytnx Library for Tensor Networks"):

* ``symtensor``  - symmetries, bonds with quantum numbers, zero-flux block
  enumeration in block-index order, densify / convert (Sec. 6 "UniTensor with
  Symmetries": 6.1 symmetries, 6.2 bonds, 6.3 symmetric UniTensor, 6.5 conversion).
* ``contract``   - pairwise contraction of block-sparse tensors over common
  labels with the bond checks, by explicit loops over matched block pairs, and
  the fused charge-sector tables (Sec. 7 "Tensor contraction"; bond combine of
  Sec. 6.2.2).
* ``network``    - the Network blueprint text format, PutUniTensor label
  mapping, ORDER parsing and the optimal-order search by dynamic programming
  with cost capping (Sec. 8 "Network", 8.1-8.3; Sec. 7 for the DP).
* ``lanczos``    - Lanczos on a linear operator with full reorthogonalisation
  and a Sturm-sequence bisection for the lowest eigenvalue (Sec. 9.3, the
  LinOp / Lanczos paragraph).
* ``brute``      - dense brute-force contraction with explicit index loops and
  dense exact diagonalisation, used only to pin the rest.

Parity status of every function is listed in its module header; the only
unpinned choices are the tie-break among equal-cost contraction orders (only
order independence of the result is pinned) and the Hubbard MPO sign
convention beyond the N <= 3 brute-force check.
"""
