"""Oracle: a plain, slow, FP64 CPU restatement of the MC-PDIPM computations.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
--impl reference legs may import or run anything in this package.  It shares no code with the
CUDA path (paper_1310_6919_gb300/) and never imports it; the two meet only through the seeded
instances in `instances/` and through plain arrays a test hands to both.

Modules
  sdp         problem data as dense / sparse-list matrices, A(X), Y(z)           (Sec. 1)
  chordal     checks of an imported extended pattern E: PEO, E ⊇ aggregate, RIP  (Sec. 2.1)
  completion  max-determinant completion (Lemma 2.6 recursion, Sec. 3.1),
              Algorithm 1, and the definition L̂ = chol(X̂^{-1})
  scm         Schur complement matrix by its definition, eq. (SCM), and the HKM right side
  pdipm       dense HKM primal-dual interior-point method (Sec. 2.2, Steps 0-4) and the
              matrix-completion Newton step at a given iterate
  maxcut      closed forms and brute force used as pins
  diff        central-path point at fixed mu (Newton centring) and its implicit derivatives
              with respect to b, A_0 and A_k (an extension; not in the paper)
  certificate weak-duality bracket b^T z <= opt <= A_0 . X̄ for an iterate known on E
              (Grone's completion theorem, Sec. 2.1), for solves too large for the dense PDIPM

Parity status: every function above is pinned by tests in tests/test_oracle_*.py against closed
forms, invariants or brute force (see each function's docstring for its pin);
tests/test_oracle_mutants.py plants single-expression mistakes in this package's source and
checks that a pin fails for each.
"""
