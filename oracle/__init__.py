"""FP64 CPU oracle for inverted-file spherical k-means (test infrastructure).

This package is test infrastructure, not part of the product.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  It shares no code with the CUDA path: both take
their inputs from ``paper_2002_09094_gb300.datagen`` and from nowhere else.

Modules
  spherical_kmeans  the method's definition: spherical Lloyd (Algorithm 2,
                    Eqs. 4-5, Eq. 8's sparse-object similarity) in FP64 with
                    dense or sparse per-cluster means; the lockstep checker.
  inverted_file     Algorithm 3 (IVF) written out step by step in FP64, used
                    to pin the paper's claim that IVF keeps Lloyd's solution.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute force, closed forms, invariants, a hand-derived worked example under
``tests/golden/``).  The paper prints no worked example of its own, so no
value here is pinned to a number printed in the paper.
"""
