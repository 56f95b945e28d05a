"""CPU oracle for the three-way ACA hot path (complex128 / float64, numpy).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this package; the product path
(the CUDA library and its Python binding) never does, and this package
imports nothing from the product.  It is deliberately plain and slow:
every function follows the paper's definitions in the paper's order, with
library primitives (numpy/scipy: matrix products, QR, SVD, elliptic
functions) as its only building blocks.

Modules
  freqs       multistep-CQ and gCQ frequencies (Appendix A)
  quadrature  collocation entries of V and K (eq. (bie_semi_diri))
  galerkin    Galerkin entries of V (eq. (bie_semi_indirect))
  galerkin_p1 Galerkin D and K' with linear continuous elements
              (eq. (bie_semi_neum)), element-local 3 x 3 blocks
  tree        balanced cluster tree and geometric block partition
  aca3        the three-way ACA of Algorithm 1 with face ACA and
              QR+SVD recompression
  apply       dense and compressed application (eq. (product))
  gcq         the time-stepping consumer: history update and weights
              (eq. (gCQ_xn), eq. (gcq_formula)), implicit-Euler reading
"""
