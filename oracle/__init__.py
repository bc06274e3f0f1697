"""CPU oracle for the matrix-free monolithic multigrid Stokes solver (FP64).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or links
this package: only the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference legs do.  It shares no code with the CUDA library; the
only common module is ``workloads`` (seeded input data, no method arithmetic).

What it computes, following the paper section by section:
  * fe.py        1D Gauss-Lobatto nodes, Gauss-Legendre quadrature, Lagrange bases
                 (Sec. 2: tensor-product Q_k / Q_{k-1} nodes, Fig. 1).
  * mesh.py      structured box hierarchy T_0..T_L, DoF numbering, Dirichlet mask
                 (Sec. 2, Sec. 3.1).
  * assemble.py  element matrices by plain quadrature, assembled CSR A, B, M_v, M_p,
                 K = [A B^T; B -C] (Eqs. a(u,v), b(v,q), Kx=f).
  * transfer.py  prolongation = canonical injection, restriction = transpose (Sec. 3.2).
  * smoother.py  Chebyshev-Jacobi Cheb(M, D, k), Lemma 1 scaling sigma/tau, the Schur
                 diagonal approximations d / p / loc, Algorithm 2, the inexact
                 symmetric Uzawa smoother in its compact form (Sec. 3.3.1).
  * mg.py        Algorithm 1 (V/W cycle), bordered coarse direct solve, stationary MG
                 driver with the rate q and T(eps) (Sec. 3.1, Sec. 4.1).
  * krylov.py    flexible GMRES with the multigrid cycle as right preconditioner
                 (outer FP64 loop; no counterpart in the paper).
  * mms.py       manufactured-solution errors (Sec. 2 error estimates).

Every function is pinned by tests against closed forms, textbook matrices,
dense direct solves or invariants (see tests/test_oracle_*.py).
"""
