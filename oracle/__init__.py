"""CPU oracle for multistage mixed-precision iterative refinement (MSIR).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct
restatement of the method of Oktay & Carson, "Multistage Mixed Precision
Iterative Refinement" (Algorithm 4 and Section 2.1), written with numpy in
float64 and with every lower precision simulated by explicit rounding.  It is
imported only by ``tests/``, by ``__graft_entry__.smoke()`` and by the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The product
path (``paper_2107_06200_gb300``) never imports it and shares no code with it.

Modules
-------
formats   number formats, unit roundoffs (Table 3), rounding, double-double
lu        blocked GEPP in precision u_f (Algorithm 4, first step)
trsv      triangular substitution models (Algorithm 4, SIR correction; x0)
residual  r = b - A x in u_r and the scaled residual (Algorithm 4, Sec. 2.1.2)
gmres     left-preconditioned GMRES for SGMRES-IR / GMRES-IR (Algorithms 2, 3)
squeeze   two-sided power-of-two scaling retried after a failed u_f LU (Sec. 2.1.2)
msir      the stage controller of Algorithm 4 with the criteria of Sec. 2.1.1
metrics   ferr / nbe / cbe (Section 2) and the reference solution x_ref

Readings of the paper that the text leaves open are listed in each module's
docstring; none of them is tuned to agree with the GPU path.
"""

from . import formats, lu, trsv, residual, gmres, squeeze, msir, metrics  # noqa: F401
