"""Multigrid transfers and the MF_PC_MG solve (Section 3.4: geometric and
polynomial coarsening).  Prolongation = coarse finite-element function at the
fine nodes (oracle basis), restriction = its transpose (adjoint identity),
interpolation = fine function at the coarse nodes."""
import numpy as np
import pytest

import synth
from synth.mesh import coarsen
from oracle.basis import tensor_basis, gll_nodes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ops(fine_mesh, coarse_mesh, parent, child, prm):
    from paper_2608_27423_b300 import RotorStatorOperator
    f = RotorStatorOperator(fine_mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
    c = RotorStatorOperator(coarse_mesh, prm["nu"], prm["omega"], prm["dt"], prm["bdf"])
    f.mg_attach(c, parent, child)
    return f, c


def _ref_coords_in_parent(k, d, child_bits, hcoarse):
    g = gll_nodes(k)
    n = k + 1
    idx = np.array(np.unravel_index(np.arange(n ** d), (n,) * d, order="F")).T
    xi = g[idx]
    if not hcoarse:
        return xi
    o = np.array([(child_bits >> r) & 1 for r in range(d)], dtype=float)
    return (o[None, :] + xi) / 2.0


CASES = [dict(d=2, k=2, h=True), dict(d=3, k=2, h=True), dict(d=2, k=3, h=False), dict(d=3, k=3, h=False)]


@pytest.mark.parametrize("c", CASES, ids=lambda c: f"d{c['d']}k{c['k']}{'h' if c['h'] else 'p'}")
def test_transfers(c):
    d, k = c["d"], c["k"]
    p = dict(d=d, k=k, m=4, n_r=2, n_s=2, n_z=2 if d == 3 else 1)
    prm = dict(nu=0.01, omega=1.0, dt=0.01, bdf=1)
    fm = synth.rotor_stator_mesh(d, k, p["m"], p["n_r"], p["n_s"], p["n_z"])
    if c["h"]:
        cp, parent, child = coarsen(p)
        cm = synth.rotor_stator_mesh(d, k, cp["m"], cp["n_r"], cp["n_s"], cp["n_z"])
        kc = k
    else:
        cm = synth.rotor_stator_mesh(d, k - 1, p["m"], p["n_r"], p["n_s"], p["n_z"])
        parent = child = None
        kc = k - 1
    f, co = _ops(fm, cm, parent, child, prm)
    rng = np.random.default_rng(3)
    xc = rng.uniform(-1, 1, (cm.n_nodes, d + 1))
    xf = rng.uniform(-1, 1, (fm.n_nodes, d + 1))
    T = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    out_f = torch.zeros((fm.n_nodes, d + 1), dtype=torch.float64, device="cuda")
    f.mg_prolongate(T(xc), out_f)
    out_c = torch.zeros((cm.n_nodes, d + 1), dtype=torch.float64, device="cuda")
    f.mg_restrict(T(xf), out_c)
    # prolongation against the coarse basis evaluated at the fine nodes
    ref = np.full((fm.n_nodes, d + 1), np.nan)
    cells_f, cells_c = np.asarray(fm.cells), np.asarray(cm.cells)
    for cell in range(fm.n_cells):
        pc = parent[cell] if parent is not None else cell
        xi = _ref_coords_in_parent(k, d, int(child[cell]) if child is not None else 0, parent is not None)
        phi, _, _ = tensor_basis(kc, d, xi)
        ref[cells_f[cell]] = phi @ xc[cells_c[pc]]
    pf = out_f.cpu().numpy()
    assert np.abs(pf - ref).max() < 1e-12
    # restriction is the transpose of the prolongation
    lhs = float((out_c.cpu().numpy() * xc).sum())
    rhs = float((xf * pf).sum())
    assert abs(lhs - rhs) < 1e-11 * abs(rhs)


def test_interpolation_reproduces_coarse_space():
    """Interpolating the prolongation of a coarse field gives the field back."""
    d, k = 3, 2
    p = dict(d=d, k=k, m=4, n_r=2, n_s=2, n_z=2)
    fm = synth.rotor_stator_mesh(d, k, 4, 2, 2, 2)
    cp, parent, child = coarsen(p)
    cm = synth.rotor_stator_mesh(d, k, cp["m"], cp["n_r"], cp["n_s"], cp["n_z"])
    f, co = _ops(fm, cm, parent, child, dict(nu=0.01, omega=1.0, dt=0.01, bdf=1))
    xc = torch.tensor(np.random.default_rng(1).uniform(-1, 1, (cm.n_nodes, 4)), device="cuda")
    xf = torch.zeros((fm.n_nodes, 4), dtype=torch.float64, device="cuda")
    f.mg_prolongate(xc, xf)
    back = torch.full_like(xc, float("nan"))
    f.mg_interpolate(xf, back)
    assert float((back - xc).abs().max()) < 1e-12


def test_multigrid_preconditioned_newton_matches_oracle():
    """Three-level h-hierarchy (2D) as the FGMRES preconditioner: the Newton
    solution equals the oracle's."""
    from paper_2608_27423_b300 import RotorStatorOperator, solver_defaults, MF_PC_MG
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
    up = T(u0)
    st, rep = g.solve_step(up, solver_defaults(theta=prm["theta"], pc=MF_PC_MG, newton_rtol=1e-11, lin_rtol=1e-6,
                                               max_newton=40, restart=30, max_lin_iters=300, mg_smooth=3,
                                               mg_coarse_iters=30))
    assert st == 0, (st, g.last_error(), list(rep.res_norm[:rep.newton_iters + 1]))
    du, dp = _compare(up.cpu().numpy(), ref)
    assert du < 1e-8 and dp < 1e-6, (du, dp)


@pytest.fixture(scope="module")
def q3_case():
    """3D Q3 cylinder (72 hexes, 10,108 DoFs), BDF2, and the oracle's direct
    Newton solution of its step (computed once for both precisions)."""
    from tests.test_gpu_solver import _oracle_solution
    prm = dict(nu=0.05, omega=1.0, dt=0.01, bdf=2, theta=0.137)
    cfg = dict(d=3, k=3, m=2, n_r=2, n_s=2, n_z=2)
    mesh, _, f = synth.make_config(**cfg, seed=23, **prm)
    u0 = np.zeros((mesh.n_nodes, 4))
    u0[:, :3] = f["u_n"]
    u0[mesh.wall.astype(bool), :3] = 0.0
    f = dict(f, u_n_full=u0)
    ref, red = _oracle_solution(mesh, prm, f)
    assert red < 1e-12
    return cfg, prm, mesh, f, ref


@pytest.mark.parametrize("pc_prec", ["fp32", "fp64"])
def test_polynomial_multigrid_q3_newton_matches_oracle(q3_case, pc_prec):
    """The polynomial level of the mixed solve (Q3 -> Q2 on the same cells) and
    one geometric level below it (Q2, every block halved): FGMRES in FP64
    preconditioned by the V-cycle with FP32 (mixed) or FP64 operator applies.
    The Newton solution equals the oracle's direct Newton solution (sparse LU
    of the assembled Jacobian at every step)."""
    from paper_2608_27423_b300 import RotorStatorOperator, solver_defaults, MF_PC_MG, MF_FP32, MF_FP64
    from tests.test_gpu_solver import _compare
    cfg, prm, mesh, f, ref = q3_case
    pmesh = synth.rotor_stator_mesh(3, 2, cfg["m"], cfg["n_r"], cfg["n_s"], cfg["n_z"])
    cp, parent, child = coarsen(dict(cfg, k=2))
    cmesh = synth.rotor_stator_mesh(3, 2, cp["m"], cp["n_r"], cp["n_s"], cp["n_z"])
    ops = [RotorStatorOperator(mm, prm["nu"], prm["omega"], prm["dt"], prm["bdf"]) for mm in (mesh, pmesh, cmesh)]
    ops[0].mg_attach(ops[1])                      # polynomial: Q3 -> Q2, same cells
    ops[1].mg_attach(ops[2], parent, child)       # geometric: Q2 -> Q2 on the halved mesh
    g = ops[0]
    T = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    g.set_history(T(f["u_n"]), T(f["u_nm1"]))
    up = T(f["u_n_full"])
    st, rep = g.solve_step(up, solver_defaults(theta=prm["theta"], pc=MF_PC_MG,
                                               pc_precision=MF_FP32 if pc_prec == "fp32" else MF_FP64,
                                               newton_rtol=1e-11, lin_rtol=1e-6, max_newton=40, restart=30,
                                               max_lin_iters=300, mg_smooth=3, mg_coarse_iters=30))
    assert st == 0, (st, g.last_error(), list(rep.res_norm[:rep.newton_iters + 1]))
    du, dp = _compare(up.cpu().numpy(), ref)
    assert du < 1e-8 and dp < 1e-6, (du, dp)
