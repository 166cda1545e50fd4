"""Unequal interface partitions (the rotor and the stator split the circle into
different numbers of cells, so a cell can meet several mortar pieces): the
paper restricts itself to equal partitions; these pins check the oracle's
general mortar before any GPU path uses it.  Segment coverage and weights
(P8), assembled = matrix-free (P3), the constant-pressure rows (P1), the
Jacobian against finite differences (P4) and manufactured-solution
convergence (P7) at the equal-partition rate."""
import numpy as np
import pytest

import synth
from oracle.fem import Problem
from oracle.mortar import Mortar, mortar_segments
from oracle.solve import Operator


@pytest.mark.parametrize("n_Rs", [12, 20, 7, 16])
@pytest.mark.parametrize("theta", [0.0, 0.137, -2.5, 9.0])
def test_segments_cover_every_cell_of_both_sides(n_Rs, theta):
    n_R = 16
    segs = mortar_segments(theta, n_R, n_Rs)
    cover_r, cover_s = np.zeros(n_R), np.zeros(n_Rs)
    for a, L, jr, js in segs:
        assert L > 0
        cover_r[jr] += L
        cover_s[js] += L
    assert np.allclose(cover_r, 2 * np.pi / n_R, atol=1e-13)
    assert np.allclose(cover_s, 2 * np.pi / n_Rs, atol=1e-13)
    assert len(segs) <= n_R + n_Rs


def _case(d=2, k=2, n_Rs=12, theta=0.137, seed=3):
    m = 4 if d == 2 else 2
    mesh = synth.rotor_stator_mesh(d, k, m, 1, 2, 2 if d == 3 else 1, n_R_stator=n_Rs)
    rng = np.random.default_rng(seed)
    up = rng.uniform(-1, 1, (mesh.n_nodes, d + 1))
    un = rng.uniform(-1, 1, (mesh.n_nodes, d))
    x = rng.uniform(-1, 1, (mesh.n_nodes, d + 1))
    x[mesh.wall.astype(bool), :d] = 0.0
    op = Operator(mesh, 0.1, 1.0, 0.01, 1, theta, up_star=up, u_n=un)
    return mesh, op, up, x


@pytest.mark.parametrize("d,n_Rs", [(2, 12), (2, 23), (3, 5)])
def test_unequal_weights_and_assembled_equals_matrix_free(d, n_Rs):
    mesh, op, up, x = _case(d=d, n_Rs=n_Rs)
    assert mesh.iface_stator.shape[1] == n_Rs and mesh.iface_rotor.shape[1] == mesh.n_R != n_Rs
    total = sum(float(np.sum(r["w"])) for r in op.mortar.recs)
    assert abs(total / (2 * np.pi * mesh.R * (mesh.H if d == 3 else 1.0)) - 1.0) < 1e-13
    A = op.assemble()
    y1 = op.apply(x)
    y2 = (A @ x.ravel()).reshape(y1.shape)
    assert np.linalg.norm(y1 - y2) <= 1e-13 * np.linalg.norm(y2)


def test_unequal_constant_pressure_rows_and_fd_jacobian():
    mesh, op, up, x = _case(d=2, n_Rs=12)
    e = np.zeros((op.nn, op.d + 1))
    e[:, op.d] = 1.0
    y = op.apply(e)
    cells = np.asarray(mesh.cells)
    near = np.zeros(op.nn, bool)
    near[cells[np.concatenate([mesh.iface_rotor.ravel(), mesh.iface_stator.ravel()])].ravel()] = True
    scale = np.abs(op.apply(x)).max()
    assert np.abs(y[~near]).max() < 1e-13 * scale and np.abs(y[:, op.d]).max() < 1e-13 * scale
    us = up.copy()
    us[op.cmask] = 0.0
    op.set_linearization(us)
    jv = op.apply(x)
    errs = []
    for eps in (1e-2, 1e-3):
        fd = (op.residual(us + eps * x, tau_up=us) - op.residual(us - eps * x, tau_up=us)) / (2 * eps)
        errs.append(np.linalg.norm(fd - jv) / np.linalg.norm(jv))
    assert errs[1] < 1e-6 and errs[0] / errs[1] > 80.0


@pytest.mark.slow
def test_unequal_mms_converges_like_equal_partitions():
    from tests.test_oracle_mms import load_mms
    from oracle.solve import chord_solve
    nu, src, exact = load_mms()

    def err(m, n_Rs):
        mesh = synth.rotor_stator_mesh(2, 2, m, max(1, m // 2), m, n_R_stator=n_Rs)
        prm = dict(nu=nu, omega=0.0, dt=0.0, bdf=1, theta=0.2)
        pr = Problem(mesh, nu, 0.0, 0.0, 1, 0.2)
        g = exact(pr.x)[:, :2]
        up, hist = chord_solve(mesh, prm, np.zeros((mesh.n_nodes, 3)), source=src, g=g)
        geo = pr.geometry(np.arange(mesh.n_cells))
        uh = np.einsum("qa,Kai->Kqi", pr.phi, up[pr.cells][..., :2])
        ex = exact(geo["xq"].reshape(-1, 2)).reshape(mesh.n_cells, -1, 3)
        return float(np.sqrt((geo["W"][..., None] * (uh - ex[..., :2]) ** 2).sum()))

    # stator 3m cells against the rotor's 4m: the same optimal rate as equal partitions (measured 3.16 against
    # 3.22 from m = 8 to 16); the error level is higher because this stator is 25% coarser
    e_un = [err(m, 3 * m) for m in (8, 16)]
    e_eq = [err(m, 4 * m) for m in (8, 16)]
    r_un, r_eq = np.log2(e_un[0] / e_un[1]), np.log2(e_eq[0] / e_eq[1])
    assert r_un > 2 + 1 - 0.35 and abs(r_un - r_eq) < 0.3, (e_un, e_eq)


@pytest.mark.parametrize("n_R,n_Rs", [(16, 16), (16, 12), (16, 20), (8, 7), (64, 48)])
def test_library_segments_equal_the_oracles(n_R, n_Rs):
    """The library's host-side segment builder (mf_mortar_segments) gives the
    oracle's segments: same pieces, cells and lengths (to roundoff)."""
    from paper_2608_27423_b300 import mortar_segments as lib_segments
    rng = np.random.default_rng(n_R * 100 + n_Rs)
    for theta in [0.0, 1e-12, 2 * np.pi / n_R * 3, -0.4, 7.3] + list(rng.uniform(-10, 10, 5)):
        ref = mortar_segments(theta, n_R, n_Rs)
        a, L, jr, js = lib_segments(n_R, n_Rs, theta)
        assert len(ref) == len(a), (theta, len(ref), len(a))
        for (ra, rL, rjr, rjs), x, y, p, q in zip(ref, a, L, jr, js):
            assert (rjr, rjs) == (p, q) and abs(rL - y) < 1e-13 and abs(np.mod(ra - x + 1, 2 * np.pi) - 1) < 1e-13
        assert abs(L.sum() - 2 * np.pi) < 1e-12
