"""CPU oracle for the Burgers-Hopf characteristic-function solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library; the two
meet only in the seeded generators of the ``synthetic`` module.

Plain, slow, obviously correct float64 numpy/scipy code, each function citing
the passage of Rodgers & Venturi, "Tensor approximation of functional
differential equations" (arXiv 2403.04946) that it follows:

* ``model``       the 1-D Burgers instance of Eq. (hyper1): grids, difference
                  matrices, per-mode operators, the MPO of the generator,
                  cell moments of the Gaussian initial state.
* ``fullgrid``    the plain definition: the generator on the full n^d grid and
                  classical RK4 without truncation (Eq. ode, Eq.
                  discrete-flow-intro).
* ``tt``          tensor-train arithmetic (App. A): full contraction, sums,
                  scaling, flattenings, Alg. 1 (mirrored), Alg. 2 (mirrored),
                  the step-truncation RK4 step (Eq. discrete-flow-trunc-intro),
                  TT-SVD of a full tensor, moments, point evaluation.
* ``reference``   the linear closed form (nonlinear term off) and a Monte-Carlo
                  estimate from the discrete Burgers ODE.
* ``mlp``         the learned surrogate's network (not in the paper): forward
                  and backward passes, Adam, normalisation, ensemble bound.

Parity status of each function is listed in its docstring ("pinned by ..." or
"parity unpinned").
"""
