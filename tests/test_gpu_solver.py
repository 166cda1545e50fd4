"""GPU Newton/FGMRES solve against the oracle's solution of R(u) = 0 (Eq.
Eq-Newton-method), all-FP64 and mixed precision (FP32 Chebyshev-Jacobi)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _solve_gpu(mesh, prm, f, **opts):
    from paper_2608_27423_b300 import RotorStatorOperator, solver_defaults
    g = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g.set_history(T(f["u_n"]), T(f["u_nm1"]) if f["u_nm1"] is not None else None)
    up = T(f["u_n_full"])
    st, rep = g.solve_step(up, solver_defaults(theta=prm["theta"], **opts))
    return st, rep, up.cpu().numpy()


@pytest.fixture(scope="module")
def case():
    mesh, prm, f = synth.make_config(d=2, k=2, m=4, n_r=2, n_s=3, nu=0.05, omega=1.0, dt=0.01, bdf=1,
                                     theta=0.137, seed=21)
    # initial guess: previous velocity, zero pressure, wall values zero
    u0 = np.zeros((mesh.n_nodes, 3))
    u0[:, :2] = f["u_n"]
    u0[mesh.wall.astype(bool), :2] = 0.0
    f = dict(f, u_n_full=u0)
    return mesh, prm, f


def _oracle_solution(mesh, prm, f):
    from oracle.solve import Operator
    import scipy.sparse.linalg as spla
    op = Operator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], prm["theta"], u_n=f["u_n"],
                  u_nm1=f["u_nm1"])
    up = f["u_n_full"].copy()
    r0 = np.linalg.norm(op.residual(up))
    for _ in range(60):
        r = op.residual(up)
        if np.linalg.norm(r) <= 1e-13 * r0:
            break
        op.set_linearization(up)
        up = up + spla.spsolve(op.assemble().tocsc(), -r.ravel()).reshape(up.shape)
    return up, np.linalg.norm(op.residual(up)) / r0


def _compare(a, b):
    du = np.linalg.norm(a[:, :2] - b[:, :2]) / np.linalg.norm(b[:, :2])
    pa = a[:, 2] - a[:, 2].mean()
    pb = b[:, 2] - b[:, 2].mean()
    dp = np.linalg.norm(pa - pb) / np.linalg.norm(pb)
    return du, dp


def test_fp64_jacobi_newton_matches_oracle(case):
    from paper_2608_27423_b300 import MF_PC_JACOBI, MF_FP64
    mesh, prm, f = case
    ref, red = _oracle_solution(mesh, prm, f)
    assert red < 1e-12
    st, rep, up = _solve_gpu(mesh, prm, f, pc=MF_PC_JACOBI, pc_precision=MF_FP64, newton_rtol=1e-11,
                             lin_rtol=1e-6, max_newton=60, restart=80, max_lin_iters=2000)
    assert st == 0, (st, rep.newton_iters, list(rep.res_norm[:rep.newton_iters + 1]))
    du, dp = _compare(up, ref)
    assert du < 1e-8 and dp < 1e-6, (du, dp)


@pytest.mark.parametrize("inner", [20, 80])
def test_mixed_precision_nested_gmres_matches_oracle(case, inner):
    """FP32 inner GMRES inside the FP64 FGMRES reaches the oracle's solution."""
    from paper_2608_27423_b300 import MF_PC_GMRES, MF_FP32
    mesh, prm, f = case
    ref, _ = _oracle_solution(mesh, prm, f)
    st, rep, up = _solve_gpu(mesh, prm, f, pc=MF_PC_GMRES, pc_precision=MF_FP32, inner_iters=inner,
                             newton_rtol=1e-11, lin_rtol=1e-6, max_newton=60, restart=30, max_lin_iters=400)
    assert st == 0, (st, rep.newton_iters)
    du, dp = _compare(up, ref)
    assert du < 1e-8 and dp < 1e-6, (du, dp)


def test_chebyshev_preconditioner_reduces_residual(case):
    from paper_2608_27423_b300 import MF_PC_CHEBYSHEV, MF_FP32
    mesh, prm, f = case
    st, rep, up = _solve_gpu(mesh, prm, f, pc=MF_PC_CHEBYSHEV, pc_precision=MF_FP32, cheb_degree=3,
                             newton_rtol=1e-6, lin_rtol=1e-3, max_newton=10, restart=50, max_lin_iters=500)
    assert rep.lambda_max > 0
    assert rep.res_norm[rep.newton_iters] < 1e-3 * rep.res_norm[0]


def test_newton_reports_iteration_limit(case):
    """A forced cap of one Newton step returns MF_ERR_NOT_CONVERGED with the
    residual history, and leaves the device usable."""
    from paper_2608_27423_b300 import MF_PC_JACOBI
    mesh, prm, f = case
    st, rep, up = _solve_gpu(mesh, prm, f, pc=MF_PC_JACOBI, newton_rtol=1e-14, max_newton=1)
    assert st == 6 and rep.newton_iters == 1
    assert rep.res_norm[1] < rep.res_norm[0]
    torch.cuda.synchronize()


def test_nan_input_is_reported(case):
    from paper_2608_27423_b300 import MF_PC_JACOBI
    mesh, prm, f = case
    f2 = dict(f)
    u0 = f["u_n_full"].copy()
    u0[5, 0] = np.nan
    f2["u_n_full"] = u0
    st, rep, up = _solve_gpu(mesh, prm, f2, pc=MF_PC_JACOBI)
    assert st == 5


def test_2d_workload_jacobi_newton_to_1e10():
    """The 2D rotor-stator workload (576 + 768 Q2 quads, non-matching mortar at
    0.137 rad, nu = 0.01, omega = 1, BDF1 dt = 0.01): Newton with FGMRES whose
    preconditioner is 80 steps of Jacobi-preconditioned GMRES, to a 1e-10
    relative residual, equal to the oracle's Newton solution.  (Plain Jacobi as
    the FGMRES preconditioner stalls near 1e-9 here: the PSPG pressure block is
    elliptic.)"""
    from paper_2608_27423_b300 import MF_PC_GMRES, MF_FP64
    mesh, prm, f = synth.make_config("2d_q2")
    u0 = np.zeros((mesh.n_nodes, 3))
    u0[:, :2] = f["u_n"]
    u0[mesh.wall.astype(bool), :2] = 0.0
    f = dict(f, u_n_full=u0)
    ref, red = _oracle_solution(mesh, prm, f)
    assert red < 1e-12
    st, rep, up = _solve_gpu(mesh, prm, f, pc=MF_PC_GMRES, pc_precision=MF_FP64, inner_iters=80, newton_rtol=1e-10,
                             lin_rtol=1e-6, max_newton=30, restart=30, max_lin_iters=300)
    assert st == 0, (st, rep.newton_iters)
    assert rep.res_norm[rep.newton_iters] <= 1e-10 * rep.res_norm[0]
    du, dp = _compare(up, ref)
    assert du < 1e-7 and dp < 1e-5, (du, dp)


def test_metrics_log_records_solves(case, tmp_path):
    """With mf_log_open set, mf_solve_step and mf_run_transient append one JSON
    line each; the solve's line carries the report's residual history."""
    import json
    import torch as _t
    from paper_2608_27423_b300 import log_open, MF_PC_JACOBI, MF_FP64, solver_defaults
    mesh, prm, f = case
    path = tmp_path / "calls.jsonl"
    log_open(path)
    try:
        st, rep, up = _solve_gpu(mesh, prm, f, pc=MF_PC_JACOBI, pc_precision=MF_FP64, newton_rtol=1e-8,
                                 lin_rtol=1e-6, max_newton=20, restart=80, max_lin_iters=2000)
        from paper_2608_27423_b300 import RotorStatorOperator, MF_PC_GMRES, MF_FP32
        g = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
        un = _t.tensor(np.ascontiguousarray(f["u_n_full"]), dtype=_t.float64, device="cuda")
        g.run_transient(un, None, 2, prm["theta"], newton_iters=2, krylov_iters=6,
                        opts=solver_defaults(pc=MF_PC_GMRES, pc_precision=MF_FP32, inner_iters=10))
    finally:
        log_open(None)
    recs = [json.loads(line) for line in open(path)]
    calls = [r["call"] for r in recs]
    assert calls == ["mf_solve_step", "mf_run_transient"], calls
    s = recs[0]
    assert s["status"] == st == 0 and s["newton_iters"] == rep.newton_iters and s["n_dofs"] == mesh.n_dofs
    assert np.allclose(s["res_norm"], list(rep.res_norm[:rep.newton_iters + 1]), rtol=1e-15)
    assert recs[1]["n_steps"] == 2 and recs[1]["graph"] == 1 and recs[1]["theta_end"] > recs[1]["theta0"]
