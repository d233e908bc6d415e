"""Plain CPU FP64 oracle for the finite-element P3M method (Beams, Olson, Freund).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA library under ``paper_1503_08509_gb300/``.

Every routine is written from the paper's equations, in FP64, with no blocking,
fusion or reordering beyond what the cited definition states.  Library
primitives (numpy matmul, scipy generalised eigensolver) serve as steps.

Modules
-------
fe1d     1-D Lagrange elements and periodic / Dirichlet assembly (Sec. 2.2).
screens  screen weights from the separable 1-D moment system (Eq. moment1d).
tables   FE basis-screen potential table (Remark in Sec. 4) and the continuum
         screen potential used for its boundary values (Eq. screenintegral).
fep3m    the whole method, Algorithm 1: binning, element-to-point coefficients,
         load vector, exact periodic FE solve, smooth-potential evaluation
         (Eq. evalsmooth), short-range sum with self term (Sec. 2.4-2.5), U
         (Eq. potentialenergy), and its hand-derived adjoint.
ewald    independent Ewald summation (the paper's "exact" comparison, Sec. 4).
"""
