"""CPU oracle of the HSS-structured multifrontal solver (arXiv 1502.07405).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA library.

Plain, slow and direct: float64 numpy, one front and one HSS node at a time,
each function following the paper's definitions and algorithms in the
paper's order (Sections 2-4 and 6.1).  Library primitives (matrix
products, LAPACK getrf/getrs, triangular solves, a complete QR) serve as
single steps; nothing is blocked, fused or reordered.

Modules
  philox        counter-based generator for the random sampling matrix R
  ordering      geometric nested dissection, separator reordering,
                symbolic factorization, HSS trees of the fronts
  hss           interpolative decomposition, HSS generators, mat-vec,
                element extraction, Algorithm 1 with the adaptive rank
                scheme, ULV-like factorization and solve
  multifrontal  dense and HSS multifrontal factorization and solves
  krylov        GMRES(30) with modified Gram-Schmidt and iterative
                refinement

Pinned by the ``-m "not gpu"`` tests; functions without a pin say
"parity unpinned" in their docstring.
"""
