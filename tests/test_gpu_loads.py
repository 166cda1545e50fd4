"""Wall loads on the GPU: steady Taylor-Couette flow (a rigid ring of stator
cells turning at Om inside a resting outer wall; the enclosed rotor is fluid),
the same set-up as the oracle's pin.  The discrete solution comes from the
oracle's direct solve, so the test isolates mf_wall_loads: its force, torque
and power per wall group must equal the oracle's consistent reactions of the
same state, and the torque must approach the closed form at the rate the
oracle pin fixes."""
import dataclasses

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def couette_state(k, m, nu, Om, theta):
    """Mesh, wall groups and the converged discrete state (oracle, sparse LU)."""
    import scipy.sparse.linalg as spla
    from oracle.fem import Problem
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
    ref = Operator(mesh, nu, 0.0, 0.0, 1, theta, g=g)
    up = np.zeros((mesh.n_nodes, 3))
    for _ in range(12):
        r = ref.residual(up)
        if np.linalg.norm(r) < 1e-11:
            break
        ref.set_linearization(up)
        up += spla.spsolve(ref.assemble().tocsc(), -r.ravel()).reshape(up.shape)
    group = np.where(body, 0, 1).astype(np.uint8)
    return mesh, g, up, group, ref, r1


@pytest.mark.parametrize("k", [2, 3])
def test_taylor_couette_wall_loads_on_gpu(k):
    from paper_2608_27423_b300 import RotorStatorOperator
    nu, Om, theta = 0.2, 1.0, 0.1
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    errs = []
    for m in (2, 4):
        mesh, g, up, group, ref, r1 = couette_state(k, m, nu, Om, theta)
        op = RotorStatorOperator(mesh, nu, 0.0, 0.0, 1)
        op.set_angle(theta)
        op.set_dirichlet(T(g))
        op.set_linearization(T(up), theta)
        out = torch.empty((2, 4), dtype=torch.float64, device="cuda")
        op.wall_loads(T(up), out, group=torch.tensor(group, device="cuda"), n_groups=2)
        loads = out.cpu().numpy()
        loads_ref = ref.wall_loads(up, group=group.astype(np.int64), n_groups=2)
        Tq = 4 * np.pi * nu * Om * r1 ** 2 / (1.0 - r1 ** 2)
        # parity with the oracle's reactions of the same state
        assert np.abs(loads - loads_ref).max() < 1e-11 * Tq, (loads, loads_ref)
        # closed form, no net force, power = Om * torque on the ring, none on the resting wall
        e_in, e_out = loads[0, 2] / Tq - 1, loads[1, 2] / (-Tq) - 1
        assert abs(e_in) < 2e-3 and abs(e_out) < 2e-3, (m, e_in, e_out)
        assert np.abs(loads[:, :2]).max() < 1e-10 * Tq
        assert abs(loads[0, 3] - Om * loads[0, 2]) < 1e-10 * Tq and abs(loads[1, 3]) < 1e-10 * Tq
        errs.append(max(abs(e_in), abs(e_out)))
    assert np.log2(errs[0] / errs[1]) > 2 * k - 1.5, errs
