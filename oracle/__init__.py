"""FP64 CPU oracle for the WB-arSVD RZF precoder update (test infrastructure).

This package is the correctness reference for the CUDA library and nothing else.  Only the
test suite (``tests/``), ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg
of ``bench.py`` may import or run it; the product path (``paper_2512_16543_gb300``) never
does, and the two share no code.  Everything here is plain numpy in float64 / complex128,
written step by step from the paper so that a reader can check it against the equations:

  rzf       -- Gram matrix, direct inverses, RZF precoder, power normalisation and the
               sum-rate KPI (Section II eq. 5, Section VI eq. 15).
  lowrank   -- truncated SVD with the energy rule (Section IV eqs. 13-14) and the adaptive
               randomized SVD (Algorithm 1).
  woodbury  -- the Woodbury inverse update exactly as written in eq. 12 (Section III).
  method    -- the per-snapshot driver (Algorithm 2) over a trajectory, for full-inversion
               RZF and for WB with the exact SVD or with arSVD.
  philox    -- the Philox-4x32-10 counter-based generator (Salmon et al., SC'11) and the
               Box-Muller map that draw Algorithm 1's Gaussian test matrices.
  cost      -- the operation-count models of Tables I, II and IV.
  hybrid    -- hybrid beamforming of Section II (eq. 4 and eq. 5): the DFT codebook,
               best-power beams, the digital RZF precoder on H_eff = A F_RF, and the
               sum-rate of eq. 15 through the beams.

Parity status: every function is pinned by the CPU tests in ``tests/test_oracle_*.py``
against closed forms, brute force, invariants or published vectors; none is "parity
unpinned" except the reproduction of Table V / Fig. 2, which this package does not attempt.
"""
