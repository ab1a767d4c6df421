"""FP64 CPU oracle for reciprocity-aware tile low-rank (TLR) MDD.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import, call or execute
anything in this package.  The product path (the CUDA library under
``paper_2412_14973_gb300/`` and its Python binding) never imports it and
shares no code with it: no kernels, headers, helpers, tables or constant
generators.  The only shared module is ``tlr_synth`` (seeded random draws).

Every function is a plain, slow, FP64 numpy restatement of a definition in
arXiv 2412.14973 and cites the passage it follows:

* ``hilbert``  -- Hilbert-curve receiver reordering, eq. (10)-(14).
* ``layout``   -- stacked unknowns Z-bar, L-bar, R-bar (Tile Low-rank MDD),
                  for uniform tiles or any tile sizes d_i.
* ``operator`` -- dense-literal operator C(theta) -> X_h (eq. 6-9, 15), the
                  misfit f (eq. 17a), W and W' and the factor gradients
                  (eq. 25-27), the adjoint and the back-mapping (eq. 11).
* ``tlr``      -- the same quantities evaluated tile by tile without forming
                  X (associativity only); checked against ``operator``.
* ``solver``   -- ADMM (eq. 18-24) with an L-BFGS x-update, exact line
                  search, lambda continuation.
* ``benchmark``-- the preconditioned benchmark objective, eq. (4), solved by
                  conjugate gradients (a closed-form pin for one dense tile).
* ``warmstart``-- the tile rank rule, the entry count and tile-size choice,
                  and the SVD / Takagi warm start (hyper-parameter selection
                  and initialisation section; Examples section, steps 1-3).
* ``general``  -- the general (non-reciprocal) TLR form: every tile free,
                  its assembly, misfit, factor gradients, line quartic and
                  truncated-SVD warm start.
* ``fourier``  -- time <-> frequency stacks and the stack-wide alpha
                  (Numerical Examples; hyper-parameter selection section).

Pins for every function live in ``tests/test_oracle_*.py`` (CPU only).
"""
