"""Plain CPU FP64 oracle for the partitioned poro-elastic + cohesive-fault solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import anything from here.
The GPU library never calls it and shares no code with it.

It restates, with assembled sparse matrices and library linear algebra, what the
paper (Gallyamov et al., "A Parallelized 3D Geomechanical Solver for
Fluid-induced Fault Slip in Poroelastic Media") defines:

  fem.py       Q1 element matrices (Sec. 3.2, App. A), fault geometry, the
               double-node fracture-flow operators (Sec. 3.1.2, 3.2.3, App. B)
               and global assembly.
  law.py       contact / Coulomb return map (Sec. 2.2.1, Eqs. normal_traction,
               yield_function, slip_split, plastic_slip_increment, corrector).
  solve.py     Newton on the incremental residuals (Sec. 3.3.1, Eqs.
               nonlinear_system, linear_system), dense LU, sparse direct and
               Prevost's partitioned CG (Sec. 3.3.2, Eqs. prevost_system,
               schur_system).
  analytic.py  closed forms used to pin the oracle: 1-D consolidation series,
               the line-source (Theis) fault pressure, the circular slip-front
               amplification lambda(T) (Sec. 4.2), Cryer's centre pressure
               (Sec. 4.1).
  tet.py       the paper's own discretisation without faults: P1 tetrahedra
               for displacement and pressure (Sec. 3.1), assembly and the
               backward-Euler monolithic step (Cryer's sphere, Sec. 4.1).
  tetfault.py  P1 tetrahedra with a fault: interface elements on the fault
               triangles (Sec. 3.1.1-3.1.2), nodal quadrature per pair, the
               triangle Laplacian; stepped by solve.py's Newton unchanged.
  adjoint.py   gradients of an objective of the converged steps (frozen
               fault states, consistent return-map derivative), one step and
               several steps with the inelastic slip as history.

Each module's header names the tests that pin it ("Pinned by: ...").  Parity
unpinned: the transient slip field at finite k_s on a finite box with Biot
coupling has no closed form; it is pinned only through the limits above and
the agreement of the independent solvers.
"""
