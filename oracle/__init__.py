"""Plain FP64 CPU oracle of the KNP-EMI implicit-explicit time step.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package. The product path (the CUDA library and its Python
binding) never calls it, and this package imports nothing from the product.

It restates the paper's method, Benedusi, Ellingsrud, Herlyng and Rognes,
"Scalable approximation and solvers for ionic electrodiffusion in cellular
geometries" (arXiv 2403.04491), step by step in numpy/scipy, in the paper's
notation, with no blocking, fusion or reordering beyond the definitions:

* ``topology``  - membrane facets, duplicated membrane nodes, DOF numbering (Section 3.3, Model A count of Section 5.1)
* ``fem``       - P1 mass/stiffness/weighted-stiffness and membrane matrices (Section 4.1)
* ``p2``        - P2 Lagrange elements: nodes, local matrices by barycentric moments, discretisation (Section 3.3 with p = 2)
* ``membrane``  - reversal potentials, alpha, Hodgkin-Huxley gates by Rush-Larsen, channel currents (Section 2.4, 3.2)
* ``system``    - the block operator A_{n-1}, right-hand side f_n, point pin and P_0 (Section 4.1, Remark 4.1, Eq. 4.4)
* ``solve``     - direct sparse solve and plain restarted GMRES (Section 6.2)
* ``step``      - the time loop (Section 3.2)

Parity status of each function is stated in its docstring; every function is
pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``.
"""
