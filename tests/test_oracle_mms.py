"""P7: manufactured-solution convergence of the oracle's full operator
(Section 4.1): velocity L2 error O(h^{k+1}), pressure O(h^k), mortar errors
independent of the rotor angle and equal to the conforming ones."""
import os

import numpy as np
import pytest
import sympy as sp

import synth
from oracle.fem import Problem
from oracle.solve import chord_solve

HERE = os.path.dirname(os.path.abspath(__file__))


def load_mms():
    exprs = {}
    for line in open(os.path.join(HERE, "golden", "mms2d_steady.txt")):
        if line.startswith("#") or "=" not in line:
            continue
        k, v = [t.strip() for t in line.split("=", 1)]
        exprs[k] = v
    X, Y = sp.symbols("x y")
    ns = {"x": X, "y": Y, "pi": sp.pi, "sin": sp.sin, "cos": sp.cos}
    u, v, p = (sp.sympify(exprs[k], locals=ns) for k in ("u", "v", "p"))
    nu = float(exprs["nu"])
    fx = u * sp.diff(u, X) + v * sp.diff(u, Y) + sp.diff(p, X) - nu * (sp.diff(u, X, 2) + sp.diff(u, Y, 2))
    fy = u * sp.diff(v, X) + v * sp.diff(v, Y) + sp.diff(p, Y) - nu * (sp.diff(v, X, 2) + sp.diff(v, Y, 2))
    F = sp.lambdify((X, Y), [fx, fy], "numpy")
    U = sp.lambdify((X, Y), [u, v, p], "numpy")

    def src(x):
        r = F(x[:, 0], x[:, 1])
        return np.stack([np.broadcast_to(r[0], x[:, 0].shape), np.broadcast_to(r[1], x[:, 0].shape)], 1)

    def exact(x):
        r = U(x[:, 0], x[:, 1])
        return np.stack([np.broadcast_to(c, x[:, 0].shape) for c in r], 1)
    return nu, src, exact


def mms_errors(k, m, theta):
    nu, src, exact = load_mms()
    mesh = synth.rotor_stator_mesh(2, k, m, max(1, m // 2), m)
    prm = dict(nu=nu, omega=0.0, dt=0.0, bdf=1, theta=theta)
    pr = Problem(mesh, nu, 0.0, 0.0, 1, theta)
    g = exact(pr.x)[:, :2]
    up, hist = chord_solve(mesh, prm, np.zeros((mesh.n_nodes, 3)), source=src, g=g)
    assert hist[-1] <= 1e-11 * hist[0] or hist[-1] < 1e-14
    cl = np.arange(mesh.n_cells)
    geo = pr.geometry(cl)
    vals = up[pr.cells]
    uh = np.einsum("qa,Kai->Kqi", pr.phi, vals[..., :2])
    ph = np.einsum("qa,Ka->Kq", pr.phi, vals[..., 2])
    ex = exact(geo["xq"].reshape(-1, 2)).reshape(len(cl), -1, 3)
    W = geo["W"]
    eu = np.sqrt((W[..., None] * (uh - ex[..., :2]) ** 2).sum())
    dp = ph - ex[..., 2]
    dp -= (W * dp).sum() / W.sum()
    ep = np.sqrt((W * dp ** 2).sum())
    return eu, ep


@pytest.mark.slow
def test_P7_mms_rates_with_mortar():
    k = 2
    errs = np.array([mms_errors(k, m, 0.2) for m in (4, 8, 16)])
    rates = np.log2(errs[:-1] / errs[1:])
    assert rates[-1, 0] > k + 1 - 0.35, (errs, rates)
    assert rates[-1, 1] > k - 0.35, (errs, rates)


def test_P7_mortar_error_independent_of_angle():
    """Error at a non-matching angle equals the matching-angle error to a few %."""
    e0 = np.array(mms_errors(2, 4, 0.0))
    e1 = np.array(mms_errors(2, 4, 0.137))
    e2 = np.array(mms_errors(2, 4, np.pi / 8 - 0.01))
    assert np.all(np.abs(e1 / e0 - 1.0) < 0.05), (e0, e1)
    assert np.all(np.abs(e2 / e0 - 1.0) < 0.05), (e0, e2)
