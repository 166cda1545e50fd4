"""Oracle pins for the energy budget terms (kinetic energy 1/2 int |u|^2 and
viscous dissipation nu int grad u : grad u of Eq. 1's Laplacian viscous form)
on the rotor-stator disk / cylinder of radius 1, height 1.

Closed forms: a rigid rotation u = e_z x x has 1/2 int |u|^2 = 1/2 int r^2 =
pi/4 per unit height and grad u : grad u = 2; a linear field u = A x has
grad u : grad u = |A|_F^2; a uniform field has 1/2 |u|^2 area.  The discrete
values differ only by the isoparametric boundary's area error, which falls
as h^(2k)."""
import numpy as np
import pytest

import synth
from oracle.fem import Problem

NU = 0.1


def _fields(d, k, m, theta=0.3):
    mesh = synth.rotor_stator_mesh(d, k, m, max(1, m // 2), m, 2 if d == 3 else 1)
    pr = Problem(mesh, NU, 1.0, 0.01, 1, theta)
    x = pr.x
    rot = np.zeros((mesh.n_nodes, d + 1))
    rot[:, 0], rot[:, 1] = -x[:, 1], x[:, 0]
    A = (np.arange(1, d * d + 1).reshape(d, d) - 2.5) * 0.3
    lin = np.zeros_like(rot)
    lin[:, :d] = x @ A.T
    uni = np.zeros_like(rot)
    uni[:, 0] = 1.0
    return pr, rot, lin, A, uni


def _errors(d, k, m):
    pr, rot, lin, A, uni = _fields(d, k, m)
    ke_r, di_r = pr.energy(rot)
    _, di_l = pr.energy(lin)
    ke_u, di_u = pr.energy(uni)
    return dict(ke_rot=ke_r / (np.pi / 4) - 1, di_rot=di_r / (2 * NU * np.pi) - 1,
                di_lin=di_l / (NU * (A ** 2).sum() * np.pi) - 1, ke_uni=ke_u / (np.pi / 2) - 1, di_uni=di_u)


@pytest.mark.parametrize("k", [2, 3])
def test_energy_closed_forms_and_boundary_rate(k):
    e2, e4 = _errors(2, k, 2), _errors(2, k, 4)
    for key in ("ke_rot", "di_rot", "di_lin", "ke_uni"):
        assert abs(e2[key]) < 2e-3, (key, e2)
        # isoparametric circle: area error O(h^(2k)) -> rate about 2k between m = 2 and 4
        rate = np.log2(abs(e2[key]) / abs(e4[key]))
        assert rate > 2 * k - 0.5, (key, rate, e2, e4)
    assert abs(e2["di_uni"]) < 1e-13


def test_energy_3d_cylinder_and_pressure_ignored():
    pr, rot, lin, A, uni = _fields(3, 3, 2)
    ke_r, di_r = pr.energy(rot)
    assert abs(ke_r / (np.pi / 4) - 1) < 1e-5 and abs(di_r / (2 * NU * np.pi) - 1) < 1e-5
    # the pressure component does not enter; the terms are quadratic in u
    noisy = rot.copy()
    noisy[:, 3] = np.random.default_rng(3).standard_normal(rot.shape[0])
    assert np.allclose(pr.energy(noisy), (ke_r, di_r), rtol=1e-14)
    assert np.allclose(pr.energy(2.0 * rot), (4 * ke_r, 4 * di_r), rtol=1e-14)
