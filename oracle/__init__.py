"""Plain FP64 CPU oracle for the staggered-grid P_N time step (StaRMAP, Section 2.1).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or constant generator with the CUDA library; the two meet only
through the seeded input arrays that ``paper_2004_02833_gb300.synth`` produces.

Modules
-------
sh       real spherical-harmonic basis, the coupling matrices Mx/My/Mz of Eq. (3)
         by exact spherical quadrature, and the sub-grid placement rule of Section 2.1.
stepper  media interpolation, the exact substep of Eq. (5), the Strang step of
         Eq. (6), the Fourier symbol of a step, and the discrete adjoint.

Every function states the passage it follows.  Readings of points the paper
leaves open are listed in the module docstrings; pins live in ``tests/``.
"""
