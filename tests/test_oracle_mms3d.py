"""P7 in 3D: manufactured-solution convergence of the oracle's full operator
on the rotor-stator cylinder (steady, nu = 1, omega = 0, non-matching mortar
angle): velocity L2 error O(h^{k+1}).  The solution is the curl of a smooth
potential (divergence free by construction; tests/golden/mms3d_curl.txt),
the momentum source and the wall data follow from it."""
import os

import numpy as np
import pytest
import sympy as sp

import synth
from oracle.fem import Problem
from oracle.solve import chord_solve

HERE = os.path.dirname(os.path.abspath(__file__))


def load_mms3d():
    exprs = {}
    for line in open(os.path.join(HERE, "golden", "mms3d_curl.txt")):
        if line.startswith("#") or "=" not in line:
            continue
        k, v = [t.strip() for t in line.split("=", 1)]
        exprs[k] = v
    X, Y, Z = sp.symbols("x y z")
    ns = {"x": X, "y": Y, "z": Z, "pi": sp.pi, "sin": sp.sin, "cos": sp.cos}
    A = [sp.sympify(exprs[k], locals=ns) for k in ("Ax", "Ay", "Az")]
    p = sp.sympify(exprs["p"], locals=ns)
    nu = float(exprs["nu"])
    xs = (X, Y, Z)
    u = [sp.diff(A[2], Y) - sp.diff(A[1], Z), sp.diff(A[0], Z) - sp.diff(A[2], X), sp.diff(A[1], X) - sp.diff(A[0], Y)]
    assert sp.simplify(sum(sp.diff(u[i], xs[i]) for i in range(3))) == 0
    f = [sum(u[j] * sp.diff(u[i], xs[j]) for j in range(3)) + sp.diff(p, xs[i])
         - nu * sum(sp.diff(u[i], xs[j], 2) for j in range(3)) for i in range(3)]
    F = sp.lambdify(xs, f, "numpy")
    U = sp.lambdify(xs, u + [p], "numpy")

    def stack(r, x):
        return np.stack([np.broadcast_to(c, x[:, 0].shape) for c in r], 1)
    return nu, (lambda x: stack(F(x[:, 0], x[:, 1], x[:, 2]), x)), (lambda x: stack(U(x[:, 0], x[:, 1], x[:, 2]), x))


def mms3d_errors(k, m, theta):
    nu, src, exact = load_mms3d()
    mesh = synth.rotor_stator_mesh(3, k, m, max(1, m // 2), max(1, m // 2), m)
    prm = dict(nu=nu, omega=0.0, dt=0.0, bdf=1, theta=theta)
    pr = Problem(mesh, nu, 0.0, 0.0, 1, theta)
    g = exact(pr.x)[:, :3]
    up, hist = chord_solve(mesh, prm, np.zeros((mesh.n_nodes, 4)), source=src, g=g)
    assert hist[-1] <= 1e-10 * hist[0] or hist[-1] < 1e-13
    cl = np.arange(mesh.n_cells)
    geo = pr.geometry(cl)
    vals = up[pr.cells]
    uh = np.einsum("qa,Kai->Kqi", pr.phi, vals[..., :3])
    ex = exact(geo["xq"].reshape(-1, 3)).reshape(len(cl), -1, 4)
    W = geo["W"]
    return float(np.sqrt((W[..., None] * (uh - ex[..., :3]) ** 2).sum()))


@pytest.mark.slow
def test_P7_3d_velocity_rate_with_mortar():
    k = 2
    e = [mms3d_errors(k, m, 0.3) for m in (2, 4)]
    rate = np.log2(e[0] / e[1])
    assert rate > k + 1 - 0.5, (e, rate)
