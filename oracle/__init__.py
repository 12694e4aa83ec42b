"""Plain, slow FP64 CPU oracle for the helical-wave spectral method (Agarwal & Banerjee,
arXiv 2210.12252).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute anything
in this package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs use it.  It shares no code with the CUDA library; the two meet only
through the seeded inputs that ``paper_2210_12252_gb300.inputs`` draws (atom lists, random
coefficient blocks), which carry none of the method's arithmetic.

Modules
  basis        Bessel zeros, Gauss-Jacobi radial rule, radial tables, box/mask/index order
  potential    Gaussian-well potential summed over the helical group's images
  transforms   naive transforms (eqs. Naive_Inverse_Transform, Fast_fwd_transform_cont)
               and the fast ones of Algorithms 1-4
  hamiltonian  Algorithm 5 (H times a block), dense assembly, direct diagonalisation
  eigensolver  plain LOBPCG with the Teter-Payne-Allan preconditioner
  mlp          reference forward/backward of the per-mode preconditioner network
  density      electron density from converged states
  gradient     Cartesian gradients of functions expressed in helical waves (Appendix C)

Every function cites the passage of the paper it follows.  Readings of passages that are
silent or ambiguous are listed in the repository's design notes and restated at the function.
"""
