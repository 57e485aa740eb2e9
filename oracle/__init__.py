"""CPU oracle for the H^2 local low-rank update -- TEST INFRASTRUCTURE ONLY.

A plain, slow, float64 numpy restatement of Boerm & Reimer, "Efficient
arithmetic operations for rank-structured matrices based on hierarchical
low-rank updates" (arXiv:1402.5056):

* ``oracle.tree``   -- cluster tree, block tree and admissible/inadmissible
  leaves (Section 2, Defs. "Cluster tree" and "Block tree");
* ``oracle.h2``     -- the H^2-matrix representation with nested cluster
  bases (Section 2, Def. "Cluster basis", Eq. (nested), Def. "H^2-matrix",
  Eq. (vsw)) and its dense assembly;
* ``oracle.update`` -- the local low-rank update
  Z|_{t0 x s0} <- trunc_eps(Z|_{t0 x s0} + A B^*) of Section 5, built from
  the recompression of Section 4 (Eq. (tildeZ_h2), the weight matrices,
  Eqs. (Qt_condensed), (Qt_nested), (hatQt_condensed)).
* ``oracle.matvec`` -- the H^2 matrix times a block of vectors (forward and
  backward transformations through the nested bases, Section 2);
* ``oracle.fem``    -- the P1 finite-element matrices of Section 7's model
  problem and their H^2 form;
* ``oracle.lr``     -- the H^2-LR factorisation, block substitutions, the
  product and the approximate inverse of Section 3, CG and Err of Section 7;
* ``oracle.chol``   -- the approximate Cholesky factorisation of Section 7's
  experiments, built with the algorithms of Section 3.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` (with the oracle timings it
reports beside its factorisation and inverse figures) may import this
package.  It shares
no code with the CUDA library and never imports it; library primitives
(numpy QR, SVD, matmul) serve as single steps.
"""
