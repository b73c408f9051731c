"""FP64 CPU oracle for the AGIS hot path (Lindegren et al. 2012, arXiv:1112.4139).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of the paper's method in NumPy, used to check the GPU library.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the GPU library never does, and this package never
imports the GPU library.  It shares no code with the CUDA path: the only thing
both consume is the seeded synthetic data from ``synth``.

Modules and the passages they follow:
  quat      App. A (Eqs. quatmult, quatconj, quatinv, qrot, quatframerot,
            quat2mat, diffrot2/3; Algorithm A.1)
  spline    App. B (Algorithm B.1, multiple end knots B.3)
  cholesky  App. C (Algorithms C.1-C.3, applied to dense and banded matrices)
  weights   Sect. 5.1.2 (Eqs. dw, dwH; the robust sigma from the intersextile range)
  model     Sects. 3.2-3.4, 3.6 and 5.1.3, 5.2.3-5.2.4 (observation model,
            residuals, partial derivatives)
  blocks    Sects. 5.1-5.3 and 6.1 (S, A, C blocks and the frame rotator)
  agis      Sect. 4.6 (the S[ACG] simple iteration)
  asi       Sect. 4.7 (the accelerated simple iteration)
  attnoise  Sect. 5.2.5 (the excess attitude noise, Eqs. excess, W, wl, e09)
  calgeneric Sects. 3.4 and 5.3 (the full geometric calibration: observation-line terms of
            Eq. etazeta, the block-diagonal update of Eqs. normC and calCon with the
            constraints of Eqs. cc1-cc3, the basic angle of Eq. DeltaGamma)
  mlp       the learned iteration proposal (not in the paper; analogue of the
            accelerated simple iteration of Sect. 4.7): network, loss, gradient,
            Adam, features and targets

Parity pins (tests/test_oracle_*.py) tie each part to the paper or to
mathematics rather than to itself.  Every function without such a pin says so.
"""
