"""Plain FP64 CPU oracle for the fractional-step immersed-boundary method.

TEST INFRASTRUCTURE ONLY. Nothing on the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` use it. It shares no code with the CUDA path
(the only common module is the seeded input generator, which holds none of
the method's arithmetic).

The oracle follows Sec. II.B of the paper step by step, written for a reader
to check by eye rather than for speed:

* ``mac``      staggered (MAC) grid operators: flux-form advection, Laplacian,
               gradient, divergence, boundary conditions (Sec. II.A/II.B).
* ``af``       Crank--Nicolson diffusion by approximate factorisation: one
               tridiagonal solve per direction (Sec. II.B).
* ``poisson``  pressure Poisson equation: plain O(N^2) DFTs in the periodic
               y, z directions and a tridiagonal (Thomas) solve along x.
* ``ib``       regularised delta-kernel interpolation and spreading (the
               moving-least-squares interpolation of Sec. II.B reduces to this
               on a uniform grid), bar-grid and flag markers.
* ``flag``     spring-network flag: stretching and dihedral-bending springs,
               forces by automatic differentiation of the energy, velocity
               Verlet sub-steps (Sec. II.B, last paragraphs).
* ``solver``   one full time step in the paper's order.
* ``generator`` the learned inflow generator (a stated reading of the
               synthetic-inflow perspective of Sec. V): periodic 3x3
               convolutions, residual network, its gradients, Adam, and the
               rollout renormalisation.

Every function states the passage it follows. Parity of each function is
pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``. The AB2
weights and the half-step time level of the pressure are pinned by the
temporal order of the step (``tests/test_oracle_time_order.py``); the
pressure update, with its correction term -(nu dt / 2) L_h phi, by the
Crank--Nicolson momentum balance that one step must satisfy at every
interior node (``tests/test_oracle_pressure_update.py``).
"""
