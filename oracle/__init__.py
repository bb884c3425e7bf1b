"""CPU FP64 oracle for the Radau-collocation interior-point Newton step.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
this package.  The product path (the CUDA library and its binding) never
does, and this package imports nothing from the product path except the
seeded input generator ``paper_2607_12201_gb300.workloads``, which holds none
of the method's arithmetic.

Plain, slow, obviously-correct restatement of the paper's method:

* ``radau``  - collocation nodes, Lagrange basis and differentiation weights
  (Eq. 3, "Collocation equation with condition independence").
* ``nlp``    - the simultaneous-method NLP of Eq. 2 / Eq. 3 for mass-action
  kinetics: objective, constraints, constraint Jacobian, Lagrangian Hessian.
* ``kkt``    - the regularised primal-dual KKT matrix, its inertia and its
  solution (dense Bunch-Kaufman or natural-order block elimination with
  pivoted dense LU), with FP64 iterative refinement.
* ``ipm``    - a filter line-search primal-dual interior-point method in the
  form of Waechter & Biegler (2006), the algorithm family of the solver the
  paper uses (Introduction: "a filter line-search interior point solver").
* ``lifted`` - the relaxed-equality ("lifted") form of the same method: slacks
  for the relaxed constraints, steps from the condensed positive-definite
  primal system W + Sigma + J^T D J by Cholesky (paper Section "Optimization
  framework configurations": the LiftedKKT form), pinned by brute-force
  solves of the whole primal-dual system, eigenvalue inertia and the limit of
  a vanishing relaxation.
* ``init``   - the initial state guess: an element-by-element collocation
  forward sweep at theta0 (paper: initial guesses from a forward solve at
  the nominal parameters, Section "Optimization framework configurations").

Pins (tests/test_oracle_*.py, all ``-m "not gpu"``): closed-form Radau
nodes; row sums / polynomial exactness of the differentiation weights; the
(2,3) Pade closed form of collocation on linear ODEs; the h^(2K-1) endpoint
order; finite-difference Jacobian and Hessian; brute-force dense solves and
eigenvalue inertia on tiny KKT systems; an independent reduced-space
Gauss-Newton solve of the linear-cascade estimation problem; and, for small
nonlinear mass-action networks (n <= 4, N = 12), an independent reduced-space
Levenberg-Marquardt solve over theta alone (Radau IIA stage equations from the
published Butcher matrix, Newton per element, a hand-written mass-action
right-hand side) whose optimum the full-space ``ipm.solve`` reproduces
(theta to 1e-7 / 1e-6, Phi to 1e-10); with noise-free cascade data, the
estimate converging to the true rate constants at the endpoint order h^5;
for the interior-point rules of Waechter & Biegler (2006): the inertia-correction
schedule call by call, the monotone barrier update, the fraction-to-boundary
step, the initial bound push, the condensed step against the unreduced
primal-dual Newton system, and filter acceptance of every accepted step.
Larger networks run the same code.  The Gauss-Legendre option (``radau.Tables``
with ``scheme="gauss"``) is pinned by closed-form nodes, quadrature and
polynomial exactness, the diagonal Pade closed form, the h^(2K) endpoint order,
finite differences, and a reduced-space fit through the closed-form K = 2 Gauss
Butcher tableau on a nonlinear network.
"""
