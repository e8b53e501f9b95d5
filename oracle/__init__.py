"""CPU oracle for the SU(N) unfolding of a GKSL master equation (arXiv:1812.11626).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call,
link or run anything in this package. The product path (the CUDA library under
``paper_1812_11626_gb300/``) never touches it and shares no code with it.

The oracle is deliberately plain and slow. Every function states the passage
of the paper it follows. Where the paper reaches a result with a plain
definition, the oracle is that definition written out:

* the unfolded generator is the matrix of the Lindbladian in the orthonormal
  generator basis, ``Q_sm = Tr(F_s L(F_m))`` and ``K_s = Tr(F_s L(1/N))``
  (Eq. 1, Eq. 6, Eq. 9) -- ``lindblad.py`` (dense, small N) and
  ``csrc/oracle_unfold.c`` (sparse, any N);
* the structure constants are Eq. 5 evaluated on dense matrices
  (``structure.py``);
* the paper's own contraction formulas Eq. 7, Eq. 10, Eq. 11 are written out on
  dense f/d tensors for small N (``paper_formulas.py``), so the readings of the
  paper (the prefactor of Eq. 10, the rate in Eq. 11, the trace part of L) are
  pinned against the definition;
* propagation is the classical RK4 map on ``dv/dt = Q(t) v + K`` (Sec. IV,
  step 3.1), its discrete adjoint, and an independent density-matrix route
  through the matrix exponential of the vectorised Liouvillian (``propagate.py``).

Parity unpinned: none of the functions above; every one is pinned by a
``-m "not gpu"`` test against textbook values, closed forms, the paper's
printed nonzero counts (Sec. IV, step 2.2) or an independent route.
"""
