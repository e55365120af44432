"""Plain, slow FP64 CPU oracle for direct Kohn-Sham minimisation on the
generalised Stiefel manifold X^T M X = I (Zhang, Zhu, Wen, Zhou,
"Gradient type optimization methods for electronic structure calculations").

TEST INFRASTRUCTURE ONLY.  The product path (the CUDA library and its Python
binding) never imports, links or runs anything in this package; only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` do.  The oracle shares no code with the CUDA path; both sides
take their seeded inputs from the separate ``ks_inputs`` module.

Modules
  fe       Q1 finite-element operators on a uniform cube (Sec. 2.3's L and B,
           restated for Q1 elements), exact sine-basis solves.
  energy   the discrete KS functional (Eq. EKS discretised, Sec. 2.3) and its
           derivative E_X (Eq. "partial deriv"), LDA exchange-correlation.
  stiefel  projected gradient (Eq. def-nablaE), Cayley retraction (Eqs. WY1,
           WY3, WY-1d), Cholesky-QR retraction (Eq. QR, Alg. ChQR), BB steps
           (Eq. bb-1), nonmonotone Armijo search (Eq. NMLS-Armijo) and
           Alg. ConOptM.
  brute    dense brute-force references for tiny grids (generalised
           eigensolves, damped SCF of Alg. SCF) used only to pin the above.

Every function of the oracle is pinned by a ``-m "not gpu"`` test against
something other than itself (closed forms, brute force, finite differences,
invariants); none is "parity unpinned".
"""
