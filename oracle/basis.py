"""Q_k Lagrange bases on Gauss-Lobatto nodes and Gauss-Legendre rules on [0,1].

Equal-order Q_k shape functions for velocity and pressure: Eq. Eq-shape-functions
(Section 2.3); node placement (Gauss-Lobatto) is reading S12; Gauss rules with
k+1 points per direction are reading S11.
"""
import numpy as np
from numpy.polynomial import legendre as L


def gll_nodes(k):
    """k+1 Gauss-Lobatto-Legendre points on [0,1]: ends plus roots of P_k'."""
    c = np.zeros(k + 1)
    c[k] = 1.0
    inner = np.sort(np.real(L.legroots(L.legder(c)))) if k >= 2 else np.zeros(0)
    x = np.concatenate([[-1.0], inner, [1.0]])
    x = 0.5 * (x - x[::-1])                 # exact symmetry
    return 0.5 * (x + 1.0)


def gauss_rule(q):
    """q-point Gauss-Legendre rule on [0,1]; weights sum to 1."""
    x, w = L.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_1d(nodes, x):
    """Values, first and second derivatives of the Lagrange polynomials.

    Returns arrays [len(x), len(nodes)] computed directly from the product
    formula l_a(x) = prod_{b != a} (x - x_b) / (x_a - x_b).
    """
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    val = np.ones((len(x), n))
    d1 = np.zeros((len(x), n))
    d2 = np.zeros((len(x), n))
    for a in range(n):
        others = [b for b in range(n) if b != a]
        den = np.prod([nodes[a] - nodes[b] for b in others])
        val[:, a] = np.prod([x - nodes[b] for b in others], axis=0) / den if others else 1.0
        for c in others:
            rest = [b for b in others if b != c]
            term = np.prod([x - nodes[b] for b in rest], axis=0) if rest else np.ones_like(x)
            d1[:, a] += term / den
            for e in rest:
                rest2 = [b for b in rest if b != e]
                t2 = np.prod([x - nodes[b] for b in rest2], axis=0) if rest2 else np.ones_like(x)
                d2[:, a] += t2 / den
    return val, d1, d2


def tensor_basis(k, d, pts):
    """Q_k basis on [0,1]^d at points pts [P, d].

    Node index a = i_0 + n i_1 + n^2 i_2 (xi_0 fastest), n = k+1.
    Returns phi [P, N], dphi [P, N, d] (reference gradient),
    hphi [P, N, d, d] (reference Hessian).
    """
    nodes = gll_nodes(k)
    n = k + 1
    N = n ** d
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, d)
    P = pts.shape[0]
    tabs = [lagrange_1d(nodes, pts[:, r]) for r in range(d)]   # each (val, d1, d2) [P, n]
    idx = np.array(np.unravel_index(np.arange(N), (n,) * d, order="F")).T   # [N, d], col r = i_r
    phi = np.ones((P, N))
    for r in range(d):
        phi *= tabs[r][0][:, idx[:, r]]
    dphi = np.ones((P, N, d))
    hphi = np.ones((P, N, d, d))
    for s in range(d):
        for r in range(d):
            dphi[:, :, s] *= (tabs[r][1] if r == s else tabs[r][0])[:, idx[:, r]]
        for t in range(d):
            for r in range(d):
                if s == t:
                    f = tabs[r][2] if r == s else tabs[r][0]
                else:
                    f = tabs[r][1] if r in (s, t) else tabs[r][0]
                hphi[:, :, s, t] *= f[:, idx[:, r]]
    return phi, dphi, hphi


def tensor_gauss(k, d):
    """Tensor Gauss points [(k+1)^d, d] (xi_0 fastest) and weights."""
    x, w = gauss_rule(k + 1)
    n = k + 1
    idx = np.array(np.unravel_index(np.arange(n ** d), (n,) * d, order="F")).T
    return x[idx], np.prod(w[idx], axis=1)
