"""Oracle: a plain, slow, FP64 CPU statement of what the joint gravity-magnetic
inversion hot path computes (arXiv 2112.15562, Secs. 2.1-2.8 and Appendix A).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link
this package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code, table or constant generator with
the CUDA library: the operator is assembled densely from the closed-form prism
fields, and the solver runs the RRCG steps one by one with dense matvecs.

Modules
  prism     closed-form vertical gravity and total-field magnetic anomaly of a
            right rectangular prism (Sec. 2.1)
  operator  dense sensitivity matrices, translation-invariant kernel tables and
            direct (FFT-free) sampled matvecs (Sec. 2.7.1)
  weights   depth, L1 (Eq. WL) and data weights, the noise model (Eq. noise)
  gramian   the Gramian and its ascent directions (Eq. Gramian, RRCG:2-3,
            Eq. steepestascenta/b)
  rrcg      the regularised reweighted CG joint solve (Eq. RRCG:1-8, Secs. 2.5,
            2.6, 2.8)

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
quadrature, closed forms, invariants or brute force, except the end-to-end solve
values on nonlinear cases, which only the paper's figures describe
("parity unpinned" for those values; the linear special case is pinned).
"""
