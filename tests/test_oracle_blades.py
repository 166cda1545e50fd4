"""Blades: walls moving with the rotor (wall = 2) in the seeded mesh and the
oracle's Dirichlet data on them (the wall velocity equals the mesh velocity
omega e_z x x of Section 3.1 at the current angle)."""
import numpy as np

import synth
from tests.oracle_helpers import make_op


def test_blade_nodes_are_interior_rotor_nodes():
    mesh = synth.rotor_stator_mesh(3, 2, 2, 4, 2, 4, blades=4)
    b = mesh.wall == 2
    assert b.sum() > 0
    assert np.all(mesh.node_side[b] == 0)                         # rotor nodes only
    r = np.hypot(mesh.x0[b, 0], mesh.x0[b, 1])
    assert r.max() < mesh.R - 1e-9                                 # off the sliding interface
    z = mesh.x0[b, 2]
    assert z.min() >= 0.25 - 1e-12 and z.max() <= 0.75 + 1e-12    # middle half of the height
    # four blades at equally spaced angles: the blade-node angle set is invariant under a quarter turn
    ang = np.round(np.mod(np.arctan2(mesh.x0[b, 1], mesh.x0[b, 0]), 2 * np.pi) / (np.pi / 2), 9)
    frac = np.unique(np.mod(ang, 1.0))
    assert len(np.unique(np.floor(ang) % 4)) == 4 and len(frac) < len(np.unique(ang))
    # no blades without the option, and stationary walls unchanged by it
    plain = synth.rotor_stator_mesh(3, 2, 2, 4, 2, 4)
    assert not np.any(plain.wall == 2)
    assert np.array_equal(plain.wall == 1, mesh.wall == 1)


def test_moving_wall_dirichlet_is_the_rotated_rigid_velocity():
    theta, omega = 0.7, 1.3
    mesh, prm, f = synth.make_config(d=3, k=2, m=2, n_r=4, n_s=2, n_z=4, nu=0.05, omega=omega, dt=0.01, bdf=1,
                                     theta=theta, seed=4, blades=4)
    op = make_op(mesh, prm, f)
    b = mesh.wall == 2
    # node positions at angle theta, rotated here from the reference coordinates
    c, s = np.cos(theta), np.sin(theta)
    x = mesh.x0[b, 0] * c - mesh.x0[b, 1] * s
    y = mesh.x0[b, 0] * s + mesh.x0[b, 1] * c
    up = np.array(f["up_star"])
    r = op.residual(up)
    assert np.allclose(r[b, 0], up[b, 0] + omega * y, atol=1e-13)
    assert np.allclose(r[b, 1], up[b, 1] - omega * x, atol=1e-13)
    assert np.allclose(r[b, 2], up[b, 2], atol=1e-13)
    # a state equal to the rigid rotation on the blades leaves zero residual there
    up[b, 0], up[b, 1], up[b, 2] = -omega * y, omega * x, 0.0
    assert np.abs(op.residual(up)[b, :3]).max() < 1e-13
    # speed omega r, tangential
    g = op.g[b]
    assert np.allclose(np.hypot(g[:, 0], g[:, 1]), omega * np.hypot(x, y), rtol=1e-13)
    assert np.abs(g[:, 0] * x + g[:, 1] * y).max() < 1e-13
