"""FP64 CPU oracle for the porous D2Q8 MRT lattice Boltzmann method (Liu & He, arXiv 1311.7239).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package: only the tests,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``
may use it.  It shares no code with the CUDA path (no kernels, headers, tables or helpers) and
is written from the paper's equations in the paper's order, in numpy float64, with the 8x8 and
5x5 transforms applied as literal matrix products.

Modules
-------
mrt_d2q8     flow step: Eqs. 3-4, 6-22 (Sec. 2.2), streaming and wall rules (Sec. 3)
thermal_d2q5 temperature step: Appendix B (Eqs. B.1-B.7), buoyancy and Nusselt number (Sec. 3.4)
adjoint      discrete adjoint of the flow step by complex-step per-cell Jacobians

Pinned against closed forms, invariants and printed values by ``tests/test_oracle_*.py``.
"""
