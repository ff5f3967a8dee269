"""FP64 CPU oracle for the DG + HABC explicit time step (arXiv 1610.05023).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute anything under ``oracle/``; only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.
The oracle shares no code with the CUDA path (its own reference elements,
mesh set-up, boundary algebra and time stepping are written here from the
paper and the textbook constructions it cites).

Modules
-------
jacobi    orthonormal Jacobi polynomials, Gauss / Gauss-Lobatto points
refelem   nodal reference line / triangle / tetrahedron (Sec. 3.2)
mesh      volume, surface and line meshes of a cuboid (Sec. 3.2, Table 1)
habc      Pade coefficients and the face / edge / corner algebra (Sec. 2, 3.1)
solver    DG right-hand sides, LSERK4, sources, energy (Sec. 3.2, Sec. 4.1)
closure   the learned closure's MLP (forward, gradient, finite differences)
          and the closed time step (ClosureSolver); not from the paper

Parity status: every function is pinned by a ``-m "not gpu"`` test.  The
numerical fluxes of the 2D / 1D auxiliary systems (the paper only says "the
same numerical scheme", Sec. 3.1 item 1; read as the upwind flux with the 3D
impedance rho c) are pinned by the exact energy rate of the semi-discrete
face and edge systems, a quadratic form of the interface jumps.
"""
