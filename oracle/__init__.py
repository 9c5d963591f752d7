"""FP64 CPU oracle of streaming GCP (arXiv 2110.14514), written from the paper.

TEST INFRASTRUCTURE ONLY.  The product path (the CUDA library and its Python
binding) never imports, links or runs anything in this package; only the
tests, the smoke check of ``__graft_entry__`` and the CPU-baseline leg of
``bench.py`` do.  It shares no code with the CUDA path: the only common
dependency is the seeded input generator package ``synthetic``.

Modules:
  philox  -- Philox4x32-10 (Salmon et al., SC'11) and the multiply-shift bounded integer
  gcp     -- losses, Kruskal model, exact and stratified-sampled gradients,
             objective estimate, history penalty (Sec. 2, Sec. 4.1-4.3, Alg. 5-6)
  solver  -- ADAM, WghtGcpSgd, FacGcpSgd, OnlineGCP, least-squares temporal
             solve, projected L-BFGS (Sec. 4.4, Alg. 1-4, Sec. 5)

Every function is pinned by tests in ``tests/test_oracle_*.py`` against
closed forms, brute force, finite differences and published test vectors.
"""
