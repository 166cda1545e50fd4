"""Pins of the oracle's discrete operator against properties the method fixes
(Section 2: weak form, mortar terms, stabilisation, Newton Jacobian)."""
import numpy as np
import pytest

from oracle.fem import Problem, rotation_matrix
from oracle.mortar import Mortar, mortar_segments
from tests.oracle_helpers import small_case, make_op, merge_interface


CASES = [dict(d=2, k=2), dict(d=2, k=3, m=1), dict(d=3, k=2, m=1, n_z=2), dict(d=3, k=3, m=1, n_s=1, n_z=1)]


@pytest.mark.parametrize("c", CASES)
def test_P3_assembled_equals_matrix_free(c):
    mesh, prm, f = small_case(bdf=2, **c)
    op = make_op(mesh, prm, f)
    A = op.assemble()
    y1 = op.apply(f["x"])
    y2 = (A @ f["x"].ravel()).reshape(y1.shape)
    assert np.linalg.norm(y1 - y2) <= 1e-13 * np.linalg.norm(y2)


@pytest.mark.parametrize("c", [dict(d=2, k=2), dict(d=3, k=2, m=1, n_z=2)])
def test_P4_finite_difference_jacobian(c):
    """J v = (R(x*+eps v) - R(x*-eps v)) / (2 eps) + O(eps^2), tau frozen (S8)."""
    mesh, prm, f = small_case(bdf=2, **c)
    op = make_op(mesh, prm, f)
    us = f["up_star"].copy()
    us[op.cmask] = 0.0
    op.set_linearization(us)
    v = f["x"]
    jv = op.apply(v)
    errs = []
    for eps in (1e-2, 1e-3):
        fd = (op.residual(us + eps * v, tau_up=us) - op.residual(us - eps * v, tau_up=us)) / (2 * eps)
        errs.append(np.linalg.norm(fd - jv) / np.linalg.norm(jv))
    assert errs[1] < 1e-6
    assert errs[0] / errs[1] > 80.0          # second order in eps


def test_P4_residual_is_frozen_tau_consistent():
    """Without the frozen tau the FD derivative differs (tau depends on u), so the
    test above really exercises the frozen-tau reading."""
    mesh, prm, f = small_case()
    op = make_op(mesh, prm, f)
    us = f["up_star"].copy()
    us[op.cmask] = 0.0
    op.set_linearization(us)
    v = f["x"]
    eps = 1e-5
    fd = (op.residual(us + eps * v) - op.residual(us - eps * v)) / (2 * eps)
    jv = op.apply(v)
    assert np.linalg.norm(fd - jv) / np.linalg.norm(jv) > 1e-6


def test_P5_sipg_stokes_block_symmetric_positive():
    """u* = 0, omega = 0, steady, tau = 0: the viscous block is symmetric and
    positive definite on constrained vectors and the divergence block is minus
    the transpose of the gradient block (textbook SIPG Stokes)."""
    mesh, prm, f = small_case(theta=0.21)
    from oracle.solve import Operator
    op = Operator(mesh, 1.0, 0.0, 0.0, 1, 0.21, up_star=np.zeros_like(f["up_star"]), stab=False)
    A = op.assemble().toarray()
    nd = A.shape[0]
    comp = np.arange(nd) % 3
    free_v = (~op.cmask).ravel() & (comp < 2)
    K = A[np.ix_(free_v, free_v)]
    assert np.abs(K - K.T).max() < 1e-13 * np.abs(K).max()
    assert np.linalg.eigvalsh(0.5 * (K + K.T)).min() > 0.0
    pm = comp == 2
    B = A[np.ix_(free_v, pm)]
    C = A[np.ix_(pm, free_v)]
    assert np.abs(B + C.T).max() < 1e-14 * np.abs(B).max() * 100
    assert np.abs(A[np.ix_(pm, pm)]).max() == 0.0


@pytest.mark.parametrize("c", [dict(d=2, k=2, m=2), dict(d=3, k=2, m=1, n_z=2)])
def test_P1_constant_pressure_interior_rows(c):
    """J [0; 1_p] vanishes on every row whose test function does not reach the
    interface (divergence theorem on the isoparametric cells, exact quadrature)."""
    mesh, prm, f = small_case(**c)
    op = make_op(mesh, prm, f)
    e = np.zeros((op.nn, op.d + 1))
    e[:, op.d] = 1.0
    y = op.apply(e)
    cells = np.asarray(mesh.cells)
    if_cells = np.concatenate([mesh.iface_rotor.ravel(), mesh.iface_stator.ravel()])
    near = np.zeros(op.nn, bool)
    near[cells[if_cells].ravel()] = True
    scale = np.abs(op.apply(f["x"])).max()
    assert np.abs(y[~near]).max() < 1e-13 * scale
    assert np.abs(y[:, op.d]).max() < 1e-13 * scale          # pressure rows: exact everywhere


def test_P1_constant_pressure_interface_defect_converges():
    """On interface rows the defect is the mismatch between the polynomial cell
    faces and the exact circle used by the mortar rule (readings S10, S13): the
    face normal errs by O(h^k), each row integrates it over a face of length h
    and there are O(1/h) rows, so the summed defect vanishes at order k.  A sign
    error in the mortar pressure term would leave an O(1) sum (rate 0)."""
    defects = []
    for m in (2, 4, 8):
        mesh, prm, f = small_case(d=2, k=2, m=m, n_r=m // 2, n_s=m // 2)
        op = make_op(mesh, prm, f)
        e = np.zeros((op.nn, 3))
        e[:, 2] = 1.0
        y = op.apply(e)
        defects.append(np.abs(y[:, :2]).sum())
    rates = np.log2(np.array(defects[:-1]) / np.array(defects[1:]))
    assert rates.min() > 1.8, (defects, rates)


@pytest.mark.parametrize("c", [dict(d=2, k=2, m=2, j=3), dict(d=2, k=3, m=1, j=1),
                               dict(d=3, k=2, m=1, n_z=2, j=2)])
def test_P2_conforming_angle_reproduces_merged_mesh(c):
    """At theta = j 2 pi / n_R the mortar operator restricted to continuous
    vectors equals the conforming operator on the merged mesh (all mortar
    terms cancel pointwise)."""
    c = dict(c)
    j = c.pop("j")
    mesh, prm, f = small_case(**c)
    theta = j * 2 * np.pi / mesh.n_R
    prm = dict(prm, theta=theta)
    op = make_op(mesh, prm, f)
    P, cm = merge_interface(op)
    nm = P.max() + 1
    d = op.d
    rng = np.random.default_rng(3)
    z_star = rng.uniform(-1, 1, (nm, d + 1))
    z = rng.uniform(-1, 1, (nm, d + 1))
    un = rng.uniform(-1, 1, (nm, d))
    op = make_op(mesh, prm, dict(f, u_n=un[P]))
    op.set_linearization(z_star[P])
    ym = op.apply(z[P])
    yPt = np.zeros((nm, d + 1))
    np.add.at(yPt, P, ym)
    pc = Problem(cm, prm["nu"], prm["omega"], prm["dt"], prm["bdf"], 0.0)
    pc.set_history(un)
    wall = np.asarray(cm.wall).astype(bool)
    zc = z.copy()
    zc[wall, :d] = 0.0
    yc = pc.volume_apply(z_star, zc)
    free = np.ones((nm, d + 1), bool)
    free[wall, :d] = False
    scale = np.abs(yc).max()
    assert np.abs(yc[free] - yPt[free]).max() < 1e-12 * scale


def test_P9_linearity_and_zero():
    mesh, prm, f = small_case()
    op = make_op(mesh, prm, f)
    x, y = f["x"], np.roll(f["x"], 5, axis=0)
    lhs = op.apply(2.0 * x - 0.5 * y)
    rhs = 2.0 * op.apply(x) - 0.5 * op.apply(y)
    assert np.linalg.norm(lhs - rhs) < 1e-13 * np.linalg.norm(rhs)
    assert np.abs(op.apply(np.zeros_like(x))).max() == 0.0


def test_tau_limits():
    """Tezduyar tau (Eq. Eq-stab-param) tends to dt, h/(2|a|) and h^2/(12 nu) when
    the transient, convective or diffusive part dominates."""
    mesh, prm, f = small_case()
    h = 0.1
    for (dt, nu, a, expect) in [(1e-6, 1e-3, 1.0, 1e-6), (0.0, 1e-9, 100.0, h / 200.0),
                                (0.0, 10.0, 1e-9, h * h / 120.0)]:
        p = Problem(mesh, nu, 0.0, dt, 1, 0.0)
        p.h = np.full(mesh.n_cells, h)
        t = p.tau(np.array([[[a, 0.0]]]), np.array([0]))
        assert abs(t[0, 0] / expect - 1.0) < 1e-4
