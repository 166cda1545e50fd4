"""Additive Schwarz smoother on the GPU (Section 3.4 ASM; local matrices of
Algorithm 2 reconstructed column by column from the matrix-free kernels, FP32
inverses): one application against the oracle's (oracle/asm.py), and the
multigrid-preconditioned Newton solve with ASM smoothing against the oracle's
direct Newton solution."""
import numpy as np
import pytest

import synth
from oracle import asm as oasm
from oracle.solve import Operator

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("d,k,n_Rs", [(2, 2, None), (2, 3, None), (3, 2, None), (3, 1, None), (2, 2, 12)])
def test_asm_apply_matches_oracle(d, k, n_Rs):
    """Tolerance: the FP32 Gauss-Jordan inverses of the local matrices carry
    about cond(A_K) x 6e-8 relative error; 2e-4 covers the condition numbers of
    these cells (measured below 1e3)."""
    from paper_2608_27423_b300 import RotorStatorOperator
    m = 4 if d == 2 else 2
    mesh = synth.rotor_stator_mesh(d, k, m, 1, 2, 2 if d == 3 else 1, n_R_stator=n_Rs)
    rng = np.random.default_rng(9)
    up = rng.uniform(-1, 1, (mesh.n_nodes, d + 1))
    un = rng.uniform(-1, 1, (mesh.n_nodes, d))
    theta = 0.137
    ref = Operator(mesh, 0.05, 1.0, 0.01, 1, theta, up_star=up, u_n=un)
    r = rng.uniform(-1, 1, (mesh.n_nodes, d + 1))
    z_ref = oasm.asm_apply(ref, r)
    g = RotorStatorOperator(mesh, 0.05, 1.0, 0.01, 1)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g.set_history(T(un))
    g.set_linearization(T(up), theta)
    assert g.asm_setup() == 0
    z = torch.full((mesh.n_nodes, d + 1), float("nan"), dtype=torch.float32, device="cuda")
    g.asm_apply(T(r).float(), z)
    got = z.double().cpu().numpy()
    e_nw = np.linalg.norm(got - z_ref) / np.linalg.norm(z_ref)
    e_max = np.abs(got - z_ref).max() / np.abs(z_ref).max()
    assert e_nw <= 2e-4 and e_max <= 2e-4, (e_nw, e_max)


def test_asm_smoothed_multigrid_newton_matches_oracle():
    """Three-level 2D h-hierarchy, V-cycle with GMRES smoothing right-
    preconditioned by ASM on every level: the Newton solution equals the
    oracle's (the iteration counts of both smoothers are reported, not
    compared: with element-matrix patches the inverse diagonal needs fewer)."""
    from paper_2608_27423_b300 import RotorStatorOperator, solver_defaults, MF_PC_MG, MF_FP32, MF_SMOOTH_ASM, \
        MF_SMOOTH_JACOBI
    from tests.test_gpu_solver import _oracle_solution, _compare
    prm = dict(nu=0.05, omega=1.0, dt=0.01, bdf=1, theta=0.137)
    hier = synth.mesh.hierarchy(dict(d=2, k=2, m=8, n_r=4, n_s=4, n_z=1), 3)
    ops = [RotorStatorOperator(mm, prm["nu"], prm["omega"], prm["dt"], prm["bdf"]) for mm, _, _ in hier]
    for lev in range(2):
        ops[lev].mg_attach(ops[lev + 1], hier[lev][1], hier[lev][2])
    mesh = hier[0][0]
    f = synth.make_config(d=2, k=2, m=8, n_r=4, n_s=4, seed=21, **prm)[2]
    u0 = np.zeros((mesh.n_nodes, 3))
    u0[:, :2] = f["u_n"]
    u0[mesh.wall.astype(bool), :2] = 0.0
    f = dict(f, u_n_full=u0)
    ref, red = _oracle_solution(mesh, prm, f)
    g = ops[0]
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g.set_history(T(f["u_n"]))
    its = {}
    for name, sm in (("asm", MF_SMOOTH_ASM), ("jacobi", MF_SMOOTH_JACOBI)):
        up = T(u0)
        st, rep = g.solve_step(up, solver_defaults(theta=prm["theta"], pc=MF_PC_MG, pc_precision=MF_FP32,
                                                   mg_smoother=sm, newton_rtol=1e-11, lin_rtol=1e-6, max_newton=40,
                                                   restart=30, max_lin_iters=300, mg_smooth=3, mg_coarse_iters=30))
        assert st == 0, (name, st, g.last_error())
        du, dp = _compare(up.cpu().numpy(), ref)
        assert du < 1e-8 and dp < 1e-6, (name, du, dp)
        its[name] = rep.lin_iters_total
    print("FGMRES iterations", its)


def test_asm_smoothed_multigrid_newton_matches_oracle_3d():
    """Two-level 3D Q2 h-hierarchy with ASM smoothing on both levels: the
    Newton solution equals the oracle's direct Newton solution."""
    from paper_2608_27423_b300 import RotorStatorOperator, solver_defaults, MF_PC_MG, MF_FP32, MF_SMOOTH_ASM
    from tests.test_gpu_solver import _oracle_solution, _compare
    prm = dict(nu=0.05, omega=1.0, dt=0.01, bdf=1, theta=0.137)
    hier = synth.mesh.hierarchy(dict(d=3, k=2, m=4, n_r=2, n_s=2, n_z=2), 2)
    ops = [RotorStatorOperator(mm, prm["nu"], prm["omega"], prm["dt"], prm["bdf"]) for mm, _, _ in hier]
    ops[0].mg_attach(ops[1], hier[0][1], hier[0][2])
    mesh = hier[0][0]
    f = synth.make_config(d=3, k=2, m=4, n_r=2, n_s=2, n_z=2, seed=22, **prm)[2]
    u0 = np.zeros((mesh.n_nodes, 4))
    u0[:, :3] = f["u_n"]
    u0[mesh.wall.astype(bool), :3] = 0.0
    f = dict(f, u_n_full=u0)
    ref, red = _oracle_solution(mesh, prm, f)
    g = ops[0]
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g.set_history(T(f["u_n"]))
    up = T(u0)
    st, rep = g.solve_step(up, solver_defaults(theta=prm["theta"], pc=MF_PC_MG, pc_precision=MF_FP32,
                                               mg_smoother=MF_SMOOTH_ASM, newton_rtol=1e-11, lin_rtol=1e-6,
                                               max_newton=40, restart=30, max_lin_iters=300, mg_smooth=3,
                                               mg_coarse_iters=30))
    assert st == 0, (st, g.last_error(), list(rep.res_norm[:rep.newton_iters + 1]))
    du, dp = _compare(up.cpu().numpy(), ref)
    assert du < 1e-8 and dp < 1e-6, (du, dp)
    print("FGMRES iterations", rep.lin_iters_total)
