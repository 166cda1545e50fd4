"""Transient path end to end (Section 4.2, Taylor-Green vortex): BDF2 time
steps with the rotor rotating at omega, the mortar remapped and Dirichlet data
updated every step, each step solved by mf_solve_step.  Checked against the
analytic solution: velocity error converges at high order under refinement and
rotating the rotor changes the error little (the paper's finding)."""
import numpy as np
import pytest

import synth
from oracle.fem import Problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NU = 1.0


def exact(x, t):
    u = np.exp(-2 * NU * t) * np.cos(x[:, 0]) * np.sin(x[:, 1])
    v = -np.exp(-2 * NU * t) * np.sin(x[:, 0]) * np.cos(x[:, 1])
    p = -0.25 * (np.cos(2 * x[:, 0]) + np.cos(2 * x[:, 1])) * np.exp(-4 * NU * t)
    return np.stack([u, v, p], 1)


def run_tgv(k, m, omega, dt, steps):
    from paper_2608_27423_b300 import RotorStatorOperator, solver_defaults, MF_PC_JACOBI, MF_FP64
    mesh = synth.rotor_stator_mesh(2, k, m, max(1, m // 2), m)
    op = RotorStatorOperator(mesh, NU, omega, dt, 2)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    xyz = torch.empty((mesh.n_nodes, 2), dtype=torch.float64, device="cuda")

    def coords(theta):
        op.set_angle(theta)
        op.node_coords(xyz)
        return xyz.cpu().numpy()

    # history at t = -dt and t = 0, at the node positions of those times
    u_m1 = exact(coords(-omega * dt), -dt)
    u_0 = exact(coords(0.0), 0.0)
    wall = mesh.wall.astype(bool)
    prev, cur = u_m1, u_0
    t = 0.0
    for n in range(steps):
        t = (n + 1) * dt
        theta = omega * t
        xn = coords(theta)
        g = np.zeros((mesh.n_nodes, 2))
        g[wall] = exact(xn[wall], t)[:, :2]
        op.set_dirichlet(T(g))
        op.set_history(T(cur[:, :2]), T(prev[:, :2]))
        up = T(cur)
        st, rep = op.solve_step(up, solver_defaults(theta=theta, pc=MF_PC_JACOBI, pc_precision=MF_FP64,
                                                    newton_rtol=1e-10, newton_atol=1e-12, lin_rtol=1e-8,
                                                    max_newton=20, restart=100, max_lin_iters=3000))
        assert st == 0, (n, st, op.last_error())
        prev, cur = cur, up.cpu().numpy()
    # velocity L2 error at t by the oracle's quadrature on the final geometry
    pr = Problem(mesh, NU, omega, dt, 2, omega * t)
    cl = np.arange(mesh.n_cells)
    geo = pr.geometry(cl)
    uh = np.einsum("qa,Kai->Kqi", pr.phi, cur[pr.cells][..., :2])
    ex = exact(geo["xq"].reshape(-1, 2), t).reshape(len(cl), -1, 3)
    return float(np.sqrt((geo["W"][..., None] * (uh - ex[..., :2]) ** 2).sum()))


def test_tgv_convergence_and_rotation_invariance():
    dt, steps = 2e-4, 25
    e = {(m, w): run_tgv(3, m, w, dt, steps) for m in (2, 4) for w in (0.0, 1.0)}
    rate0 = np.log2(e[(2, 0.0)] / e[(4, 0.0)])
    rate1 = np.log2(e[(2, 1.0)] / e[(4, 1.0)])
    assert rate0 > 3.0 and rate1 > 3.0, (e, rate0, rate1)
    assert abs(e[(4, 1.0)] / e[(4, 0.0)] - 1.0) < 0.5, e
