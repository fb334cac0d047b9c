"""CPU oracle of the HSUMMA hot path -- TEST INFRASTRUCTURE.

A plain, slow, obviously correct CPU restatement of what the GPU path computes,
written from the paper (Quintin, Hasanov, Lastovetsky, "Hierarchical Parallel
Matrix Multiplication on Large-Scale Distributed Memory Platforms") and, for
the split-precision path and the learned cost model that the paper does not
contain, from the published methods each module names.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
or run anything here.  The product path (paper_1306_4161_gb300) never does, and
this package never imports the product: the two share only the seeded input
generator (workloads.py), which holds none of the method's arithmetic.

Modules
  native        binary64 triple-loop GEMM and Dot2 compensated entries (plain C)
  split         Ozaki-style slicing, exact pair products, exact recombination
  hsumma_sim    distributed SUMMA / HSUMMA simulation with broadcast counters,
                block-checkerboard and block-cyclic distributions
  cost_model    the paper's Hockney-model costs (Section IV)
  gpu_schedule  group resolution and the GPU panel-load counter model (block
                and block-cyclic layouts)
  mlp           float64 MLP forward / backward / Adam

Parity status: every function above is pinned by tests that do not reuse its
own code (brute force, closed forms, the paper's printed numbers, invariants);
see tests/test_oracle_*.py.
"""
