"""CPU oracle for the metapath-query hot path. TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline and
reference legs may import anything from this package. The product path (the CUDA
library and its Python binding) never imports, links or runs it, and this package never
imports the product path; the two share nothing but the seeded input generators in
``gen``.

Contents, each citing the passage of the paper it follows:

* ``chain.c`` / ``chain.py`` -- the plain definition of a (constrained) metapath query
  result, A_m = M_1 A_1 M_2 ... A_{n-1} M_n over the integers (Sec. 2, Problem 1 and the
  constrained adjacency M_c * A after it), computed single-threaded with a dense uint64
  accumulator and overflow-checked arithmetic; plus the SpMV row/column-sum chains.
* ``hin.py`` -- typed 0/1 adjacency matrices (Sec. 2, Def. 1) and constraint masks
  (Def. 3) built with numpy from the generator's edge lists.
* ``planner.py`` -- the matrix-chain dynamic program of Eq. 1 with the dense cost of
  Sec. 3.1, the sparse cost of Eq. 2 and the average-case density estimator E_ac of
  Sec. 3.2, with the density matrix D.

Pins (tests/test_oracle_*.py) tie each function to something other than itself: brute
force path enumeration, closed forms, scipy.sparse, invariants and the paper's worked
numbers.
"""
