"""Pins P6 and P8 of the oracle (no implementation compared, only facts the
geometry fixes):
P8  the mortar weights of every rotor angle sum to the interface length 2 pi R
    (times H in 3D) exactly, and the cells' det J w sum to the domain area
    (volume) with the isoparametric boundary error falling at a high rate;
P6  the O-grid rotor maps onto itself under a quarter turn, so the Jacobian at
    theta + pi/2 equals the Jacobian at theta with the rotor nodes permuted
    (linearisation state and history given as functions of position); the
    Jacobian is continuous in theta through a conforming angle."""
import numpy as np
import pytest

import synth
from oracle.fem import Problem
from oracle.mortar import Mortar
from oracle.solve import Operator


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("theta", [0.0, 0.137, 3 * 2 * np.pi / 16 + 1e-11, -0.4, 7.0])
def test_P8_mortar_weights_sum_to_interface_length(d, theta):
    mesh = synth.rotor_stator_mesh(d, 2, 4, 2, 2, 3 if d == 3 else 1)
    pr = Problem(mesh, 0.01, 1.0, 0.01, 1, theta)
    mt = Mortar(pr)
    total = sum(float(np.sum(r["w"])) for r in mt.recs)
    exact = 2 * np.pi * mesh.R * (mesh.H if d == 3 else 1.0)
    assert abs(total / exact - 1.0) < 1e-13, (total, exact)


@pytest.mark.parametrize("k", [2, 3])
def test_P8_cell_weights_approach_domain_measure(k):
    errs = []
    for m in (4, 8):
        mesh = synth.rotor_stator_mesh(2, k, m, 2, m)
        pr = Problem(mesh, 0.01, 0.0, 0.0, 1, 0.0)
        area = float(pr.geometry(np.arange(mesh.n_cells))["W"].sum())
        errs.append(abs(area - np.pi))
    assert errs[0] < 1e-3 and np.log2(errs[0] / errs[1]) > 2 * k - 0.5, errs
    mesh = synth.rotor_stator_mesh(3, 2, 8, 2, 8, 2, H=0.7)
    pr = Problem(mesh, 0.01, 0.0, 0.0, 1, 0.0)
    vol = float(pr.geometry(np.arange(mesh.n_cells))["W"].sum())
    assert abs(vol / (0.7 * np.pi) - 1.0) < 1e-4


def _fields(x):
    up = np.stack([np.sin(x[:, 0] + 2 * x[:, 1]), np.cos(3 * x[:, 0] - x[:, 1]), x[:, 0] * x[:, 1]], 1)
    un = np.stack([np.cos(x[:, 0] - x[:, 1]), np.sin(2 * x[:, 0] * x[:, 1])], 1)
    return up, un


def _jacobian(mesh, theta):
    x = Problem(mesh, 0.05, 1.0, 0.01, 1, theta).x
    up, un = _fields(x)
    return Operator(mesh, 0.05, 1.0, 0.01, 1, theta, up_star=up, u_n=un).assemble().tocsr(), x


def test_P6_quarter_turn_permutes_rotor_nodes():
    mesh = synth.rotor_stator_mesh(2, 2, 2, 1, 2)
    th0 = 0.137
    A0, x0 = _jacobian(mesh, th0)
    A1, x1 = _jacobian(mesh, th0 + 0.5 * np.pi)
    # node i at th0 + pi/2 sits where node perm[i] of the same side sat at th0
    perm = np.arange(mesh.n_nodes)
    side = np.asarray(mesh.node_side)
    key = lambda x: np.round(x, 9)
    lookup = {(int(s),) + tuple(key(p)): j for j, (s, p) in enumerate(zip(side, x0))}
    for i in range(mesh.n_nodes):
        perm[i] = lookup[(int(side[i]),) + tuple(key(x1[i]))]
    assert np.any(perm != np.arange(mesh.n_nodes)) and len(set(perm)) == mesh.n_nodes
    nf = 3
    P = (perm[:, None] * nf + np.arange(nf)[None, :]).ravel()
    B = A0[P][:, P]
    diff = abs(A1 - B).max()
    assert diff < 1e-11 * abs(A0).max(), diff


def test_P6_jacobian_continuous_through_conforming_angle():
    mesh = synth.rotor_stator_mesh(2, 2, 2, 1, 2)
    D = 2 * np.pi / mesh.n_R
    for th in (0.0, 3 * D):
        A, _ = _jacobian(mesh, th)
        for eps in (1e-10, -1e-10):
            Ae, _ = _jacobian(mesh, th + eps)
            assert abs(Ae - A).max() < 1e-7 * abs(A).max()
