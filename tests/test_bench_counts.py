"""The bench's algorithmic work counts (the numerators of the roofline) against
the ncu measurements of the same kernel on the 16,384-hex Q2 cylinder
(profiles/k_cell_jac_fp64_3d_q2_mid.md): DRAM bytes of one FP64 cell-Jacobian
launch 134.740 MB read + 4.888 MB written; FP64 flop count of the kernel before
the flux folding 318.1 MFLOP (DFMA x 2 + DMUL + DADD).  Per-cell flops by hand
from the kernel's loops: Q2 3D 19,413, Q3 3D 54,464 (sum factorisation + point
physics per Gauss point times the points)."""
import synth
from synth.configs import CONFIGS

import bench


def test_algorithmic_counts_match_the_measured_kernel():
    c = CONFIGS["3d_q2_mid"]
    mesh = synth.rotor_stator_mesh(3, 2, c["m"], c["n_r"], c["n_s"], c["n_z"])
    assert (mesh.n_cells, mesh.n_nodes) == (16384, 141537)
    ncache = 35     # J^-1 (9), det J w, G (6), c~ (3), a (3), grad u* (9), R* (3), tau
    byts = bench.algorithmic_bytes_per_launch(3, 2, mesh.n_cells, mesh.n_nodes, ncache)
    measured = 134.739968e6 + 4.887808e6
    assert abs(byts / measured - 1.0) < 0.01, (byts, measured)
    assert bench.TRAFFIC_BYTES_PER_CELL_Q2_3D_FP64 * 16384 == measured
    assert bench.algorithmic_flops_per_cell(3, 2) == 19413
    assert abs(16384 * 19413 / 318.1e6 - 1.0) < 0.002
    assert bench.algorithmic_flops_per_cell(3, 3) == 54464
