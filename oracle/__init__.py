"""CPU FP64 oracle for the TNQE matrix-element path (arXiv 2404.10223).

This package is TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
the CPU-baseline leg of the benchmark may import it; the product library never
does, and it never imports the product library.

* ``oracle.fock`` -- exact dense Fock-space evaluation (Jordan-Wigner, Sec. II A;
  orbital rotations by the compound-matrix action of Thouless' theorem,
  Sec. II B) for small N.
* ``oracle.mps``  -- a plain CPU matrix-product-state implementation of the same
  path at any N: Givens factorisation of the relative rotation (Eq. 11),
  two-site gate application with SVD truncation (Eq. A5, Sec. II D), an exact
  MPO of Eq. 1, MPS-MPO-MPS transfer contraction and the canonical
  orthogonalisation solve (Sec. IV C, App. A2).
"""
