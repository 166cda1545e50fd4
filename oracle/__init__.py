"""CPU FP64 oracle for the rotor-stator matrix-free operator -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, independent restatement of the discrete method of
"High-order stabilized matrix-free simulation of rotating mixing devices using
the Mortar Element Method" (Sections 2-3).  It exists to check the CUDA library:
only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product (the CUDA library and its Python
binding) never imports, links or calls anything here, and this package never
imports the product.

Pieces (each function names the passage it follows):

* ``basis``   -- Gauss-Lobatto Lagrange bases of degree k, Gauss rules.
* ``fem``     -- isoparametric geometry, the stabilised ALE Navier-Stokes volume
                 terms (residual, Eq. Eq-NSweakComplete; Jacobian blocks A..D of
                 Section 2.3), element matrices (path A) and a per-point
                 matrix-free evaluation (path B).
* ``mortar``  -- rotor rotation (Section 3.1), mortar segments by sorted union
                 of both angular partitions and mapped Gauss rules (Section 3.2),
                 Hillewaert penalty (Eq. EqPenalty) and the mortar face terms of
                 Eq. Eq-NSweakWmortar.
* ``solve``   -- Dirichlet constraints, restarted GMRES / dense solves, Newton
                 (Eq. Eq-Newton-method).

Readings of passages that are silent or garbled are listed in the design doc of the
repository (S1..S21) and are the same ones the CUDA library takes.  Parity
status: every operator term is pinned by a test that does not re-derive it
(null space, conforming identity, assembled vs matrix-free, finite-difference
Jacobian, SIPG Stokes definiteness, quadrature invariants, manufactured-solution
convergence rates).
"""
