"""Batched nonlinear step (mf_batch_solve_step) of uneven independent
instances: every instance reaches the oracle's Newton solution of its own
R(u) = 0 (Eq. Eq-Newton-method), the batched mode (per-instance streams, one
persistent Jacobian launch for all instances, CUDA graph) and the sequential
mode (one instance after another, eager) agree, and the reported residual
norms are the oracle's residual norms of the returned states."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (m, n_r, n_s, Re, theta, seed): 2D Q2 rotor-stator meshes of 28 .. 180 quads
SPECS = [(4, 2, 3, 10.0, 0.137, 31), (6, 2, 4, 20.0, 0.9, 32), (2, 1, 2, 1.0, 2.3, 33), (4, 1, 4, 50.0, 0.05, 34)]


def _instance(m, n_r, n_s, re, theta, seed):
    nu = 1.0 / (2.0 * np.pi * re)
    mesh, prm, f = synth.make_config(d=2, k=2, m=m, n_r=n_r, n_s=n_s, nu=nu, omega=1.0, dt=0.01, bdf=2,
                                     theta=theta, seed=seed)
    u0 = np.zeros((mesh.n_nodes, 3))
    u0[:, :2] = f["u_n"]
    u0[mesh.wall.astype(bool), :2] = 0.0
    return mesh, prm, f, u0


def _oracle(mesh, prm, f, u0):
    from oracle.solve import Operator
    import scipy.sparse.linalg as spla
    op = Operator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], prm["theta"], u_n=f["u_n"],
                  u_nm1=f["u_nm1"])
    up = u0.copy()
    r0 = np.linalg.norm(op.residual(up))
    for _ in range(60):
        r = op.residual(up)
        if np.linalg.norm(r) <= 1e-13 * r0:
            break
        op.set_linearization(up)
        up = up + spla.spsolve(op.assemble().tocsc(), -r.ravel()).reshape(up.shape)
    return op, up


def _rel(a, b):
    du = np.linalg.norm(a[:, :2] - b[:, :2]) / np.linalg.norm(b[:, :2])
    pa, pb = a[:, 2] - a[:, 2].mean(), b[:, 2] - b[:, 2].mean()
    return du, np.linalg.norm(pa - pb) / np.linalg.norm(pb)


@pytest.fixture(scope="module")
def cases():
    out = []
    for s in SPECS:
        mesh, prm, f, u0 = _instance(*s)
        op, ref = _oracle(mesh, prm, f, u0)
        out.append((mesh, prm, f, u0, op, ref))
    return out


def _run(cases, batched, use_graph):
    from paper_2608_27423_b300 import RotorStatorOperator, BatchedOperators, solver_defaults, MF_PC_GMRES, MF_FP32
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    ops, ups = [], []
    for mesh, prm, f, u0, _, _ in cases:
        g = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
        g.set_history(T(f["u_n"]), T(f["u_nm1"]))
        ops.append(g)
        ups.append(T(u0))
    batch = BatchedOperators(ops)
    # full Newton steps with a strong linear solve: the test is about agreement, not globalisation
    o = solver_defaults(pc=MF_PC_GMRES, pc_precision=MF_FP32, inner_iters=40, newton_rtol=1e-12, max_newton=40,
                        line_search=0)
    st, reps = batch.solve_step(ups, [c[1]["theta"] for c in cases], o, krylov_iters=16, batched=batched,
                                use_graph=use_graph)
    torch.cuda.synchronize()
    return st, reps, [u.cpu().numpy() for u in ups], (batch, ops)


def test_batched_solve_reaches_oracle_solutions(cases):
    st, reps, ups, keep = _run(cases, batched=True, use_graph=True)
    assert st == 0, [(r.status, r.newton_iters, r.res_norm[r.newton_iters] / r.res_norm[0]) for r in reps]
    for (mesh, prm, f, u0, op, ref), rep, up in zip(cases, reps, ups):
        it = rep.newton_iters
        assert 1 <= it <= 40 and rep.status == 0
        r0 = np.linalg.norm(op.residual(u0))
        assert abs(rep.res_norm[0] - r0) <= 1e-12 * r0
        # the reported final norm is the oracle's residual norm of the returned
        # state, up to the rounding of the two residual evaluations (~1e-13 R_0)
        rf = np.linalg.norm(op.residual(up))
        assert rf <= 1e-12 * r0 + 1e-13 * r0 and abs(rep.res_norm[it] - rf) <= 1e-3 * rf + 1e-13 * r0
        du, dp = _rel(up, ref)
        assert du < 1e-8 and dp < 1e-6, (du, dp)


def test_batched_and_sequential_modes_agree(cases):
    st_b, reps_b, ups_b, keep_b = _run(cases, batched=True, use_graph=True)
    st_s, reps_s, ups_s, keep_s = _run(cases, batched=False, use_graph=False)
    assert st_b == 0 and st_s == 0
    for a, b in zip(ups_b, ups_s):
        du, dp = _rel(a, b)
        assert du < 1e-8 and dp < 1e-6, (du, dp)
    st_g, reps_g, ups_g, keep_g = _run(cases, batched=False, use_graph=True)
    assert st_g == 0
    for a, b in zip(ups_g, ups_s):
        du, dp = _rel(a, b)
        assert du < 1e-8 and dp < 1e-6, (du, dp)


def test_batched_solve_iteration_cap_reports_not_converged(cases):
    from paper_2608_27423_b300 import RotorStatorOperator, BatchedOperators, solver_defaults, MF_PC_JACOBI, MF_FP64
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    ops, ups = [], []
    for mesh, prm, f, u0, _, _ in cases[:2]:
        g = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
        g.set_history(T(f["u_n"]), T(f["u_nm1"]))
        ops.append(g)
        ups.append(T(u0))
    batch = BatchedOperators(ops)
    o = solver_defaults(pc=MF_PC_JACOBI, pc_precision=MF_FP64, newton_rtol=1e-14, max_newton=2, batch_fallback=0)
    st, reps = batch.solve_step(ups, [c[1]["theta"] for c in cases[:2]], o, krylov_iters=4)
    assert st == 6
    for r in reps:
        assert r.newton_iters == 2 and r.status == 6 and r.res_norm[2] < r.res_norm[0]
        assert r.fallback_newton_iters == 0


def test_batched_solve_fallback_finishes_instances(cases):
    """An iteration cap that stops the batched steps above tolerance: with the
    adaptive fallback (the default) every instance continues alone with
    mf_solve_step from its last iterate and reaches the tolerance relative to
    its initial residual; the report counts both parts."""
    from paper_2608_27423_b300 import RotorStatorOperator, BatchedOperators, solver_defaults, MF_PC_GMRES, MF_FP32
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    ops, ups = [], []
    for mesh, prm, f, u0, _, _ in cases[:2]:
        g = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
        g.set_history(T(f["u_n"]), T(f["u_nm1"]))
        ops.append(g)
        ups.append(T(u0))
    batch = BatchedOperators(ops)
    tol = 1e-9
    o = solver_defaults(pc=MF_PC_GMRES, pc_precision=MF_FP32, inner_iters=40, newton_rtol=tol, max_newton=2,
                        restart=30, lin_rtol=1e-6, max_lin_iters=300)
    st, reps = batch.solve_step(ups, [c[1]["theta"] for c in cases[:2]], o, krylov_iters=4)
    assert st == 0, [r.status for r in reps]
    for r in reps:
        k = r.newton_iters
        assert r.status == 0 and r.fallback_newton_iters >= 1 and k == 2 + r.fallback_newton_iters
        assert r.res_norm[k] <= tol * r.res_norm[0] * (1 + 1e-12)
        # the fallback starts over from the initial guess unless the batched
        # iterations got within sqrt(newton_rtol) of the target
        best = min(r.res_norm[1], r.res_norm[2], r.res_norm[0])
        assert r.fallback_restarted == (0 if best <= np.sqrt(tol) * r.res_norm[0] else 1)
