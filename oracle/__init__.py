"""Plain FP64 CPU oracle of the space-time least-squares Schroedinger solver.

TEST INFRASTRUCTURE ONLY. This package is the slow, obviously-correct
restatement of the method of Bressan, Kushova, Sangalli and Tani
(arXiv 2311.18461) that the CUDA path is checked against. Only the tests,
`__graft_entry__.smoke()` and the `cpu_baseline` / `--impl reference` legs
of `bench.py` may import it. The CUDA library never calls into it and it
never calls into the CUDA library: the two share no code. Seeded input
generators live in the separate `inputs` package, which holds none of the
method's arithmetic.

Modules, each citing the passage of the paper it restates:
  bspline   -- open knot vectors, Cox-de Boor B-splines and derivatives (Sec. 3.1)
  matrices  -- univariate Galerkin matrices, Dirichlet/initial restriction (Eq. time_mat, Eq. space_mat, Sec. 3.2)
  system    -- Kronecker form of the least-squares matrix A (Eq. syst_mat),
               its separable-potential extension, mode products (Eq. kron_vec_multi)
  direct    -- independent (d+1)-dimensional quadrature of (S B_j, S B_i) (Sec. 4.3)
  fd        -- the preconditioner P-hat (Eq. prec_definition) and Algorithm 1; its potential-aware
               variant P_V for potentials that are sums of one-direction factors (an extension: the
               construction of Eq. prec_definition applied to i d_t + sum_l (-nu d_ll + v_l))
  geometry  -- the system on a mapped domain F((0,1)^d): physical-domain spatial matrices of Eq. space_mat
               by quadrature with the map's Jacobian and Hessian (Sec. 3.2, Eq. syst_mat; potential-free)
  pcg       -- preconditioned conjugate gradients (Sec. 5.3, Sec. 6); flexible CG for preconditioners
               applied inexactly (Notay 2000; not in the paper)
  rhs       -- load vector F(S B_i) and liftings of initial / boundary data (Sec. 2.2, Sec. 4.3)
  norms     -- L2 and V-norm errors (Sec. 2.1, Theorem 2)
  warmstart -- network, loss, gradient, Adam and randomized snapshot basis of the learned warm start
               (not in the paper: its PCG starts from zero, Sec. 6)

Parity status: every function here is pinned by a `-m "not gpu"` test against
closed forms, the paper's printed numbers, invariants or brute force. The
separable-potential terms (the paper has no potential) are pinned by
brute-force quadrature of the same sesquilinear form. The flexible CG used
with low-precision preconditioners (Notay's method, not in the paper) is
pinned by the invariants it fixes under a preconditioner that changes at every
iteration: A-orthogonal consecutive directions, exact line searches, a
non-increasing A-norm error, and plain PCG's iterates for a fixed one.
P_V is pinned by its spatial operators against brute-force Galerkin matrices and by Algorithm 1
against the dense inverse of P_V assembled from its definition; its ANOVA approximation for products of
factors by closed-form means and by its equality with P_V for additive potentials.
The warm-start module has no counterpart in the paper; its functions are pinned against finite
differences, closed forms and the SVD, but whether a trained warm start helps is judged only by PCG
iterations and final error against the cold start.
"""
