"""Oracle pins for the energy budget terms (kinetic energy 1/2 int |u|^2,
viscous dissipation nu int grad u : grad u of Eq. 1's Laplacian viscous form
and the paper's -tau : grad u with tau = -nu (grad u + grad u^T)) on the
rotor-stator disk / cylinder of radius 1, height 1, and for the wall loads
(torque from the consistent reactions) against Taylor-Couette flow.

Closed forms: a rigid rotation u = e_z x x has 1/2 int |u|^2 = 1/2 int r^2 =
pi/4 per unit height and grad u : grad u = 2; a linear field u = A x has
grad u : grad u = |A|_F^2; a uniform field has 1/2 |u|^2 area.  The discrete
values differ only by the isoparametric boundary's area error, which falls
as h^(2k)."""
import numpy as np
import pytest

import synth
from oracle.fem import Problem

NU = 0.1


def _fields(d, k, m, theta=0.3):
    mesh = synth.rotor_stator_mesh(d, k, m, max(1, m // 2), m, 2 if d == 3 else 1)
    pr = Problem(mesh, NU, 1.0, 0.01, 1, theta)
    x = pr.x
    rot = np.zeros((mesh.n_nodes, d + 1))
    rot[:, 0], rot[:, 1] = -x[:, 1], x[:, 0]
    A = (np.arange(1, d * d + 1).reshape(d, d) - 2.5) * 0.3
    lin = np.zeros_like(rot)
    lin[:, :d] = x @ A.T
    uni = np.zeros_like(rot)
    uni[:, 0] = 1.0
    return pr, rot, lin, A, uni


def _errors(d, k, m):
    pr, rot, lin, A, uni = _fields(d, k, m)
    ke_r, di_r, ds_r = pr.energy(rot)
    _, di_l, ds_l = pr.energy(lin)
    ke_u, di_u, ds_u = pr.energy(uni)
    # (grad u + grad u^T) : grad u = |A|^2 + tr(A A) for u = A x; zero for a rigid rotation
    return dict(ke_rot=ke_r / (np.pi / 4) - 1, di_rot=di_r / (2 * NU * np.pi) - 1,
                di_lin=di_l / (NU * (A ** 2).sum() * np.pi) - 1, ke_uni=ke_u / (np.pi / 2) - 1,
                ds_lin=ds_l / (NU * ((A ** 2).sum() + np.trace(A @ A)) * np.pi) - 1,
                di_uni=di_u, ds_uni=ds_u, ds_rot=ds_r)


@pytest.mark.parametrize("k", [2, 3])
def test_energy_closed_forms_and_boundary_rate(k):
    e2, e4 = _errors(2, k, 2), _errors(2, k, 4)
    for key in ("ke_rot", "di_rot", "di_lin", "ke_uni", "ds_lin"):
        assert abs(e2[key]) < 2e-3, (key, e2)
        # isoparametric circle: area error O(h^(2k)) -> rate about 2k between m = 2 and 4
        rate = np.log2(abs(e2[key]) / abs(e4[key]))
        assert rate > 2 * k - 0.5, (key, rate, e2, e4)
    assert abs(e2["di_uni"]) < 1e-13 and abs(e2["ds_uni"]) < 1e-13 and abs(e2["ds_rot"]) < 1e-13


def test_energy_3d_cylinder_and_pressure_ignored():
    pr, rot, lin, A, uni = _fields(3, 3, 2)
    ke_r, di_r, ds_r = pr.energy(rot)
    assert abs(ke_r / (np.pi / 4) - 1) < 1e-5 and abs(di_r / (2 * NU * np.pi) - 1) < 1e-5 and abs(ds_r) < 1e-13
    # the pressure component does not enter; the terms are quadratic in u
    noisy = lin.copy()
    noisy[:, 3] = np.random.default_rng(3).standard_normal(rot.shape[0])
    e = pr.energy(lin)
    assert np.allclose(pr.energy(noisy), e, rtol=1e-14)
    assert np.allclose(pr.energy(2.0 * lin), 4 * np.array(e), rtol=1e-14)


def _couette(k, m, nu=0.2, Om=1.0, theta=0.1):
    """Steady Taylor-Couette flow in the stator annulus: the stator's first ring
    of cells (R <= r <= r1) is a rigid body turning at Om (stationary walls with
    Dirichlet data Om e_z x x), the outer wall r = 1 is at rest, the rotor is
    fluid enclosed by the rigid ring (no mesh motion, omega = 0)."""
    import dataclasses
    import scipy.sparse.linalg as spla
    from oracle.solve import Operator
    n_s = 2 * m
    mesh = synth.rotor_stator_mesh(2, k, m, max(1, m // 2), n_s)
    r1 = mesh.R + (1.0 - mesh.R) / n_s
    body = (mesh.node_side == 1) & (np.hypot(mesh.x0[:, 0], mesh.x0[:, 1]) <= r1 + 1e-12)
    wall = mesh.wall.copy()
    wall[body] = 1
    mesh = dataclasses.replace(mesh, wall=wall)
    x = Problem(mesh, nu, 0.0, 0.0, 1, theta).x
    g = np.zeros((mesh.n_nodes, 2))
    g[body, 0], g[body, 1] = -Om * x[body, 1], Om * x[body, 0]
    op = Operator(mesh, nu, 0.0, 0.0, 1, theta, g=g)
    up = np.zeros((mesh.n_nodes, 3))
    for _ in range(12):
        r = op.residual(up)
        if np.linalg.norm(r) < 1e-11:
            break
        op.set_linearization(up)
        up += spla.spsolve(op.assemble().tocsc(), -r.ravel()).reshape(up.shape)
    assert np.linalg.norm(op.residual(up)) < 1e-10
    group = np.where(body, 0, 1)
    loads = op.wall_loads(up, group=group, n_groups=2)
    # closed form: torque per unit depth the inner cylinder exerts on the fluid,
    # 4 pi nu Om r1^2 b^2 / (b^2 - r1^2), b = 1; the outer wall exerts the opposite
    T = 4 * np.pi * nu * Om * r1 ** 2 / (1.0 - r1 ** 2)
    return loads, T, Om


@pytest.mark.parametrize("k", [2, 3])
def test_wall_loads_taylor_couette_torque(k):
    errs = []
    for m in (2, 4):
        loads, T, Om = _couette(k, m)
        assert np.abs(loads[:, :2]).max() < 1e-12 * T        # no net force (symmetric flow)
        e_in, e_out = loads[0, 2] / T - 1, loads[1, 2] / (-T) - 1
        assert abs(e_in) < 2e-3 and abs(e_out) < 2e-3, (m, e_in, e_out)
        # the rigid body's power is its torque times its angular velocity; the resting wall does no work
        assert abs(loads[0, 3] - Om * loads[0, 2]) < 1e-12 * T and abs(loads[1, 3]) < 1e-12 * T
        errs.append(max(abs(e_in), abs(e_out)))
    assert np.log2(errs[0] / errs[1]) > 2 * k - 1.5, errs


def test_wall_loads_default_groups_follow_wall_type():
    """group=None sums stationary walls into row 0 and walls moving with the rotor into row 1."""
    from tests.oracle_helpers import make_op
    mesh, prm, f = synth.make_config(d=3, k=2, m=2, n_r=4, n_s=2, n_z=4, nu=0.05, omega=1.3, dt=0.01, bdf=1,
                                     theta=0.7, seed=4, blades=4)
    op = make_op(mesh, prm, f)
    up = f["up_star"]
    a = op.wall_loads(up)
    grp = np.where(mesh.wall == 2, 1, 0)
    b = op.wall_loads(up, group=grp, n_groups=2)
    assert np.allclose(a, b, rtol=1e-14, atol=0)
    # one group holding every wall = the sum of the two
    c = op.wall_loads(up, group=np.zeros(mesh.n_nodes, int), n_groups=1)
    assert np.allclose(c[0], a.sum(0), rtol=1e-12)
