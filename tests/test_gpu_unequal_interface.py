"""General interfaces on the GPU: rotor and stator split the circle into
different numbers of cells (n_R != n_Rs), so a cell meets several mortar
segments (the paper restricts itself to equal partitions, Section 3.1 and its
conclusions).  The library's mortar cells are then the n_R + n_Rs segments
per layer between consecutive rotor and stator vertices, built on the device
at every angle.  Parity against the oracle's general mortar (the sorted union
of both vertex sets): Jacobian in FP64, FP32 and double-float, residual,
diagonal, and a Newton solve."""
import numpy as np
import pytest

import synth
from oracle.solve import Operator

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return max(float(np.linalg.norm(a - b) / np.linalg.norm(b)), float(np.abs(a - b).max() / np.abs(b).max()))


def _case(d, k, n_Rs, theta, m=4, seed=41):
    from paper_2608_27423_b300 import RotorStatorOperator
    n_z = 2 if d == 3 else 1
    mesh = synth.rotor_stator_mesh(d, k, m, 1, 2, n_z, n_R_stator=n_Rs)
    rng = np.random.default_rng(seed)
    up = rng.uniform(-1, 1, (mesh.n_nodes, d + 1))
    un = rng.uniform(-1, 1, (mesh.n_nodes, d))
    unm1 = rng.uniform(-1, 1, (mesh.n_nodes, d))
    x = rng.uniform(-1, 1, (mesh.n_nodes, d + 1))
    x[mesh.wall.astype(bool), :d] = 0.0
    ref = Operator(mesh, 0.05, 1.0, 0.01, 2, theta, up_star=up, u_n=un, u_nm1=unm1)
    g = RotorStatorOperator(mesh, 0.05, 1.0, 0.01, 2)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g.set_history(T(un), T(unm1))
    g.set_linearization(T(up), theta)
    return mesh, ref, g, T, up, x


CASES = [(2, 2, 12, 0.137), (2, 2, 23, -2.5), (2, 3, 7, 0.4), (3, 2, 5, 0.9), (3, 2, 11, 9.0), (3, 3, 6, 0.3),
         (2, 2, 8, 2 * np.pi / 16 * 3)]      # last: every other rotor vertex on a stator vertex (zero-length segments)


@pytest.mark.parametrize("d,k,n_Rs,theta", CASES)
def test_unequal_interface_apply_residual_diagonal_match_oracle(d, k, n_Rs, theta):
    from paper_2608_27423_b300 import MF_FP32, MF_DF64
    mesh, ref, g, T, up, x = _case(d, k, n_Rs, theta)
    assert mesh.iface_stator.shape[1] == n_Rs
    yr = ref.apply(x)
    y = torch.empty_like(T(x))
    g.apply_jacobian(T(x), y)
    assert rel(y.cpu().numpy(), yr) <= 1e-12
    ydf = torch.empty_like(y)
    g.apply_jacobian(T(x), ydf, prec=MF_DF64)
    assert rel(ydf.cpu().numpy(), yr) <= 1e-12
    y32 = torch.empty_like(y, dtype=torch.float32)
    g.apply_jacobian(T(x).float(), y32, prec=MF_FP32)
    assert rel(y32.double().cpu().numpy(), yr) <= 1e-5
    u = up * 0.7 + 0.1
    r = torch.empty_like(y)
    g.residual(T(u), r)
    assert rel(r.cpu().numpy(), ref.residual(u)) <= 1e-12
    dg = torch.empty_like(y)
    g.diagonal(dg)
    assert rel(dg.cpu().numpy(), ref.diagonal()) <= 1e-12


def test_unequal_interface_newton_matches_oracle():
    """Jacobi-FGMRES Newton on a 2D mesh with 16 rotor and 12 stator interface
    cells: the solution equals the oracle's direct Newton solution."""
    from paper_2608_27423_b300 import RotorStatorOperator, solver_defaults, MF_PC_JACOBI, MF_FP64
    from tests.test_gpu_solver import _oracle_solution, _compare
    mesh = synth.rotor_stator_mesh(2, 2, 4, 2, 3, n_R_stator=12)
    prm = dict(nu=0.05, omega=1.0, dt=0.01, bdf=1, theta=0.137)
    rng = np.random.default_rng(5)
    un = rng.uniform(-1, 1, (mesh.n_nodes, 2))
    u0 = np.zeros((mesh.n_nodes, 3))
    u0[:, :2] = un
    u0[mesh.wall.astype(bool), :2] = 0.0
    f = dict(u_n=un, u_nm1=None, u_n_full=u0)
    ref, red = _oracle_solution(mesh, prm, f)
    assert red < 1e-12
    g = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g.set_history(T(un))
    up = T(u0)
    st, rep = g.solve_step(up, solver_defaults(theta=prm["theta"], pc=MF_PC_JACOBI, pc_precision=MF_FP64,
                                               newton_rtol=1e-11, lin_rtol=1e-6, max_newton=60, restart=80,
                                               max_lin_iters=2000))
    assert st == 0, (st, g.last_error())
    du, dp = _compare(up.cpu().numpy(), ref)
    assert du < 1e-8 and dp < 1e-6, (du, dp)
