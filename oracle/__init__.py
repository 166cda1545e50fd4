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

Where the paper is silent or garbled, this package takes the same readings as
the CUDA library: the jump is own minus other with the own outward normal, the
face penalty is the larger of the two cells' values with F = 1, every
non-interface face enters the penalty with weight 1/2, h is the diameter of
the equal-volume circle (2D) or sphere (3D), k+1 Gauss points per direction,
Gauss-Lobatto nodes, mortar points on the exact circle with weights w R dphi
(dz), tau frozen in the Jacobian, no convective flux across the interface.
Parity status: every operator term is pinned by a test that does not re-derive
it (null space, conforming identity, assembled vs matrix-free, finite-difference
Jacobian, SIPG Stokes definiteness, quadrature invariants, rotation symmetry,
manufactured-solution convergence rates in 2D and 3D, a Taylor-Green step).
"""
