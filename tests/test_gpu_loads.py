"""Wall loads end to end on the GPU: steady Taylor-Couette flow solved by
mf_solve_step, torque by mf_wall_loads, against the closed form (the same
set-up as the oracle's pin): a rigid ring of stator cells turning at Om inside
a resting outer wall; the enclosed rotor is fluid."""
import dataclasses

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def couette_gpu(k, m, nu=0.2, Om=1.0, theta=0.1):
    from paper_2608_27423_b300 import RotorStatorOperator, solver_defaults, MF_PC_JACOBI, MF_FP64
    n_s = 2 * m
    mesh = synth.rotor_stator_mesh(2, k, m, max(1, m // 2), n_s)
    r1 = mesh.R + (1.0 - mesh.R) / n_s
    body = (mesh.node_side == 1) & (np.hypot(mesh.x0[:, 0], mesh.x0[:, 1]) <= r1 + 1e-12)
    wall = mesh.wall.copy()
    wall[body] = 1
    mesh = dataclasses.replace(mesh, wall=wall)
    op = RotorStatorOperator(mesh, nu, 0.0, 0.0, 1)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    op.set_angle(theta)
    xyz = torch.empty((mesh.n_nodes, 2), dtype=torch.float64, device="cuda")
    op.node_coords(xyz)
    x = xyz.cpu().numpy()
    g = np.zeros((mesh.n_nodes, 2))
    g[body, 0], g[body, 1] = -Om * x[body, 1], Om * x[body, 0]
    op.set_dirichlet(T(g))
    up = torch.zeros((mesh.n_nodes, 3), dtype=torch.float64, device="cuda")
    st, rep = op.solve_step(up, solver_defaults(theta=theta, pc=MF_PC_JACOBI, pc_precision=MF_FP64, newton_rtol=1e-12,
                                                newton_atol=1e-12, lin_rtol=1e-10, max_newton=30, restart=200,
                                                max_lin_iters=20000))
    assert st == 0, op.last_error()
    out = torch.empty((2, 4), dtype=torch.float64, device="cuda")
    op.wall_loads(up, out, group=torch.tensor(np.where(body, 0, 1).astype(np.uint8), device="cuda"), n_groups=2)
    Tq = 4 * np.pi * nu * Om * r1 ** 2 / (1.0 - r1 ** 2)
    return out.cpu().numpy(), Tq, Om


@pytest.mark.parametrize("k", [2, 3])
def test_taylor_couette_torque_on_gpu(k):
    errs = []
    for m in (2, 4):
        loads, Tq, Om = couette_gpu(k, m)
        e_in, e_out = loads[0, 2] / Tq - 1, loads[1, 2] / (-Tq) - 1
        assert abs(e_in) < 2e-3 and abs(e_out) < 2e-3, (m, e_in, e_out)
        assert np.abs(loads[:, :2]).max() < 1e-8 * Tq
        assert abs(loads[0, 3] - Om * loads[0, 2]) < 1e-10 * Tq and abs(loads[1, 3]) < 1e-10 * Tq
        errs.append(max(abs(e_in), abs(e_out)))
    assert np.log2(errs[0] / errs[1]) > 2 * k - 1.5, errs
