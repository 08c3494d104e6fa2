"""FP64 CPU oracle for the FTK pose-scoring path (arXiv 1905.12317).

TEST INFRASTRUCTURE ONLY. Nothing in the library imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import or run it. It shares no code with the CUDA path.

Two oracles, both plain and slow, in float64:

* ``brute.bandlimited_inner_products`` (O1) -- the discretized bandlimited inner
  product X(delta, gamma) written out as its definition (eq. Xdg with the
  trapezoid Fourier transform eq. Ahattrap on the polar grid of Section 3.2).
* ``ftk_steps.ftk_scores`` (O2) -- the FTK algorithm of Section 4.5 taken step by
  step: radial quadrature (Section 3.1), per-Bessel-order operator SVD
  (eq. Jsvd, Remark r:svd), truncation (eq. svdtrunc), then Steps 1-3 of
  eq. (fbk3).

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
exact symmetries and the values printed in the paper.
"""
