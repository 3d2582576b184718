"""Plain, slow FP64 CPU oracle for the QTT Navier-Stokes time step.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library in ``paper_2406_17823_b300``; the two meet only at the seeded
input generators in ``qtt_inputs``.

Modules
-------
``oracle.qtt``    the QTT/MPS algorithm of the paper (Sec. II.B-II.C,
                  App. A-B) written out step by step with numpy FP64
                  (numpy's QR / SVD / tensordot serve as library primitives).
``oracle.dense``  the plain definition the QTT method approximates: the same
                  finite-difference scheme on the dense 2^n x 2^n grid, with
                  the penalty projection solved exactly in Fourier space.
"""
