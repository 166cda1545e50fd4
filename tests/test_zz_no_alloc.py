"""mf_solve_step_static: the Newton / FGMRES step with its workspace in the
library's fixed device array, for callers that must not allocate device memory
(a process whose allocator has reserved the GPU up front, or a loop that cannot
take cudaMalloc's device-wide synchronisation).  Checked through the C ABI
against mf_solve_step on the same problem, on two calls in a row (the array
keeps the previous call's contents), plus its size limit.

Collected last on purpose: it runs after every other test file."""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problem():
    from paper_2608_27423_b300 import RotorStatorOperator
    mesh, prm, f = synth.make_config(d=2, k=2, m=4, n_r=2, n_s=3, nu=0.05, omega=1.0, dt=0.01, bdf=1, theta=0.137,
                                     seed=21)
    op = RotorStatorOperator(mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    op.set_history(T(f["u_n"]))
    u0 = np.zeros((mesh.n_nodes, 3))
    u0[:, :2] = f["u_n"]
    u0[mesh.wall.astype(bool), :2] = 0.0
    return mesh, prm, op, T(u0)


def _opts(theta, restart=80):
    from paper_2608_27423_b300 import solver_defaults, MF_PC_JACOBI, MF_FP64
    return solver_defaults(theta=theta, pc=MF_PC_JACOBI, pc_precision=MF_FP64, newton_rtol=1e-11, lin_rtol=1e-6,
                           max_newton=60, restart=restart, max_lin_iters=2000)


def _rel(a, b):
    du = float((a[:, :2] - b[:, :2]).norm() / b[:, :2].norm())
    pa, pb = a[:, 2] - a[:, 2].mean(), b[:, 2] - b[:, 2].mean()
    return du, float((pa - pb).norm() / pb.norm())


def test_static_workspace_solve_matches_allocating_solve():
    from paper_2608_27423_b300 import _lib, MfSolveReport
    lib = _lib.load()
    mesh, prm, op, u0 = _problem()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ref = u0.clone()
    o = _opts(prm["theta"])
    rep = MfSolveReport()
    st = lib.mf_solve_step(op.h, C.c_void_p(ref.data_ptr()), C.byref(o), C.byref(rep), stream)
    assert st == 0, op.last_error()
    for call in range(2):
        up = u0.clone()
        rep2 = MfSolveReport()
        st = lib.mf_solve_step_static(op.h, C.c_void_p(up.data_ptr()), C.byref(o), C.byref(rep2), stream)
        assert st == 0, (call, op.last_error())
        du, dp = _rel(up, ref)
        assert du < 1e-8 and dp < 1e-6, (call, du, dp)
        # atomics reorder sums, so the step that crosses the 1e-11 tolerance may move by one
        assert abs(rep2.newton_iters - rep.newton_iters) <= 1


def test_static_workspace_call_allocates_no_device_memory():
    """On a freshly created handle that never ran mf_solve_step, two static
    calls in a row leave the device's free memory unchanged (cudaMemGetInfo
    through torch.cuda.mem_get_info, after a synchronize).  A warm-up call on
    another handle first loads every kernel the solve launches, so lazy module
    loading does not show up as an allocation."""
    from paper_2608_27423_b300 import _lib, MfSolveReport
    lib = _lib.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    _, prm, warm, u_w = _problem()
    o = _opts(prm["theta"])
    rep = MfSolveReport()
    assert lib.mf_solve_step_static(warm.h, C.c_void_p(u_w.data_ptr()), C.byref(o), C.byref(rep), stream) == 0
    _, prm, fresh, u0 = _problem()
    ups = [u0.clone(), u0.clone()]
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for up in ups:
        st = lib.mf_solve_step_static(fresh.h, C.c_void_p(up.data_ptr()), C.byref(o), C.byref(rep), stream)
        assert st == 0, fresh.last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    # the fresh handle's result equals the warm handle's (same problem)
    du, dp = _rel(ups[1], u_w)
    assert du < 1e-8 and dp < 1e-6, (du, dp)


def test_static_workspace_rejects_oversized_problems():
    from paper_2608_27423_b300 import _lib, MfSolveReport, MF_PC_GMRES, RotorStatorOperator
    lib = _lib.load()
    mesh, prm, op, u0 = _problem()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rep = MfSolveReport()
    # the 2D workload (16,707 DoFs) with restart 200 needs (2*200 + 10) * 16,707 doubles > 4 Mi
    big_mesh, big_prm, _ = synth.make_config("2d_q2")
    big = RotorStatorOperator(big_mesh, big_prm["nu"], big_prm["omega"], big_prm["dt"], big_prm["bdf"])
    ub = torch.zeros((big_mesh.n_nodes, 3), dtype=torch.float64, device="cuda")
    o = _opts(big_prm["theta"], restart=200)
    st = lib.mf_solve_step_static(big.h, C.c_void_p(ub.data_ptr()), C.byref(o), C.byref(rep), stream)
    assert st == _lib.MF_ERR_ARG
    assert "static workspace" in big.last_error()
    # only the Jacobi / FP64 configuration runs without allocation
    o = _opts(prm["theta"])
    o.pc = MF_PC_GMRES
    st = lib.mf_solve_step_static(op.h, C.c_void_p(u0.data_ptr()), C.byref(o), C.byref(rep), stream)
    assert st == _lib.MF_ERR_ARG
    assert "MF_PC_JACOBI" in op.last_error()
