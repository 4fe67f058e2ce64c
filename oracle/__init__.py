"""CPU oracle for the HPS fast direct solver (arXiv 2503.17535).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package; only the tests, the smoke check and the benchmark's CPU
baseline leg use it.  It shares no code with the CUDA path.

Two independent programs live here:

* O1, ``oracle.hps``: a plain HPS implementation in NumPy (float64 and
  complex128) that follows the paper's steps in order: the leaf stage
  (Algorithms "2D DtN local solve" and "2D ItI local solve", and the 3D DtN
  variant of Appendix C), the merge stage (Algorithm "merge" with the block
  formulas of Appendices A.2, B.2 and C.2) and the downward pass
  (Algorithm "down pass").
* O2, ``oracle.composite``: a brute-force dense solve of the same composite
  collocation system, with no merges and no block formulas, used to pin O1 on
  small trees.

Readings of points the paper leaves open are listed at the top of each module.
"""
