"""The library's rotor-stator mesh generator (mf_mesh_rotor_stator, host
code, no GPU) against the seeded input generator that every other test uses:
identical connectivity, sides, walls and interface tables, coordinates equal
to roundoff, and the same coarsening maps (mf_mesh_coarsen_map)."""
import numpy as np
import pytest

import synth
from synth.mesh import coarsen

CASES = [
    dict(d=2, k=1, m=2, n_r=1, n_s=1),
    dict(d=2, k=2, m=16, n_r=5, n_s=12),
    dict(d=2, k=4, m=3, n_r=2, n_s=3),
    dict(d=3, k=2, m=4, n_r=2, n_s=2, n_z=3),
    dict(d=3, k=3, m=2, n_r=1, n_s=2, n_z=2),
    dict(d=3, k=2, m=8, n_r=4, n_s=4, n_z=8, blades=4),
    dict(d=3, k=3, m=6, n_r=3, n_s=2, n_z=5, blades=3),
]


@pytest.mark.parametrize("p", CASES, ids=lambda p: "-".join(f"{k}{v}" for k, v in p.items()))
def test_generator_matches_input_generator(p):
    from paper_2608_27423_b300 import rotor_stator_mesh
    ref = synth.rotor_stator_mesh(p["d"], p["k"], p["m"], p["n_r"], p["n_s"], p.get("n_z", 1),
                                  blades=p.get("blades", 0))
    got = rotor_stator_mesh(**p)
    assert got.x0.shape == ref.x0.shape and got.cells.shape == ref.cells.shape
    for key in ("cells", "cell_side", "node_side", "wall", "iface_rotor", "iface_stator"):
        assert np.array_equal(getattr(got, key), getattr(ref, key)), key
    assert np.abs(got.x0 - ref.x0).max() < 1e-14
    assert (got.R, got.n_R, got.n_z, got.H) == (ref.R, ref.n_R, ref.n_z, ref.H)
    assert abs(got.phi0 - ref.phi0) < 1e-16
    # interface nodes of both sides lie on the circle
    for tab in (got.iface_rotor, got.iface_stator):
        nodes = got.cells[tab.ravel()]
        r = np.hypot(got.x0[nodes, 0], got.x0[nodes, 1])
        assert np.sum(np.abs(r - got.R) < 1e-15) >= tab.size * (p["k"] + 1) ** (p["d"] - 1)


@pytest.mark.parametrize("p", [dict(d=2, k=2, m=4, n_r=2, n_s=4), dict(d=3, k=2, m=4, n_r=2, n_s=2, n_z=4)])
def test_coarsen_map_matches_input_generator(p):
    from paper_2608_27423_b300 import coarsen_map
    cp, parent, child = coarsen_map(**p)
    rp, rparent, rchild = coarsen(dict(p, n_z=p.get("n_z", 1)))
    for key in ("m", "n_r", "n_s"):
        assert cp[key] == rp[key]
    if p["d"] == 3:
        assert cp["n_z"] == rp["n_z"]
    assert np.array_equal(parent, rparent) and np.array_equal(child, rchild)


def test_generator_rejects_bad_parameters():
    from paper_2608_27423_b300 import rotor_stator_mesh, coarsen_map, MfError
    for bad in (dict(d=4), dict(k=0), dict(m=0), dict(R=1.2), dict(sq=0.8), dict(d=2, blades=2), dict(n_z=0)):
        with pytest.raises(MfError):
            rotor_stator_mesh(**bad)
    with pytest.raises(MfError):
        coarsen_map(d=2, k=2, m=3, n_r=2, n_s=2)
    with pytest.raises(TypeError):
        rotor_stator_mesh(radius=1.0)


def _node_count(d, k, m, n_r, n_s, n_z):
    """Nodes of the generated mesh: O-grid square, rotor rings, stator rings
    (interface duplicated), times the node layers in z."""
    mk, nRk = m * k, 4 * m * k
    n2 = (mk + 1) ** 2 + n_r * k * nRk + (n_s * k + 1) * nRk
    return n2 * (n_z * k + 1 if d == 3 else 1)


def test_dof_per_cell_ratio_matches_the_papers_meshes():
    """Table of the paper's scalability meshes (Section 4.3): DoFs / cells is
    32.2-33.1 at Q2Q2 and 105-110 at Q3Q3 (d+1 fields on k^3 nodes per cell plus
    surface terms); the synthetic cylinders of the workloads fall in the same
    band.  The node-count formula is checked against the generator first."""
    from paper_2608_27423_b300 import rotor_stator_mesh
    from synth.configs import CONFIGS
    for p in (dict(d=3, k=2, m=4, n_r=2, n_s=2, n_z=3), dict(d=3, k=3, m=6, n_r=3, n_s=2, n_z=5),
              dict(d=2, k=2, m=16, n_r=5, n_s=12, n_z=1)):
        assert rotor_stator_mesh(**p).n_nodes == _node_count(**p)
    bands = {2: (32.0, 34.0), 3: (105.0, 113.0)}
    for name in ("3d_q2", "3d_q3", "3d_q3_1m"):
        c = CONFIGS[name]
        cells = (c["m"] ** 2 + 4 * c["m"] * (c["n_r"] + c["n_s"])) * c["n_z"]
        dofs = 4 * _node_count(3, c["k"], c["m"], c["n_r"], c["n_s"], c["n_z"])
        lo, hi = bands[c["k"]]
        assert lo <= dofs / cells <= hi, (name, cells, dofs, dofs / cells)


@pytest.mark.parametrize("p", [dict(d=2, k=2, m=4, n_r=2, n_s=3, n_R_stator=12),
                               dict(d=3, k=3, m=2, n_r=1, n_s=2, n_z=2, n_R_stator=11)],
                         ids=["2d-12", "3d-11"])
def test_generator_unequal_partitions_match_input_generator(p):
    """Stator with its own number of interface cells: same arrays as the input
    generator; the operator refuses such meshes (no mortar kernel for them yet)."""
    from paper_2608_27423_b300 import rotor_stator_mesh, RotorStatorOperator, MfError
    q = dict(p)
    n_Rs = q.pop("n_R_stator")
    ref = synth.rotor_stator_mesh(q["d"], q["k"], q["m"], q["n_r"], q["n_s"], q.get("n_z", 1), n_R_stator=n_Rs)
    got = rotor_stator_mesh(**p)
    assert got.n_R_stator == n_Rs and got.iface_stator.shape == ref.iface_stator.shape
    for key in ("cells", "cell_side", "node_side", "wall", "iface_rotor", "iface_stator"):
        assert np.array_equal(getattr(got, key), getattr(ref, key)), key
    assert np.abs(got.x0 - ref.x0).max() < 1e-14
