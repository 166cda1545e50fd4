"""Pins of the oracle's bases and quadrature against closed forms (Section 2.3,
equal-order Q_k Lagrange bases; readings S11, S12)."""
import numpy as np
import pytest

from oracle.basis import gll_nodes, gauss_rule, lagrange_1d, tensor_basis, tensor_gauss


def test_gll_closed_forms():
    assert np.allclose(gll_nodes(1), [0, 1], atol=1e-15)
    assert np.allclose(gll_nodes(2), [0, 0.5, 1], atol=1e-15)
    r5 = 1 / np.sqrt(5.0)
    assert np.allclose(gll_nodes(3), [0, (1 - r5) / 2, (1 + r5) / 2, 1], atol=1e-15)
    r37 = np.sqrt(3.0 / 7.0)
    assert np.allclose(gll_nodes(4), [0, (1 - r37) / 2, 0.5, (1 + r37) / 2, 1], atol=1e-15)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6])
def test_gauss_exactness(q):
    x, w = gauss_rule(q)
    for p in range(2 * q):
        assert abs((w * x ** p).sum() - 1.0 / (p + 1)) < 1e-13
    assert abs((w * x ** (2 * q)).sum() - 1.0 / (2 * q + 1)) > 1e-9


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_lagrange_interpolation_and_derivatives(k):
    nodes = gll_nodes(k)
    v, d1, d2 = lagrange_1d(nodes, nodes)
    assert np.allclose(v, np.eye(k + 1), atol=1e-13)
    xs = np.linspace(0.03, 0.97, 11)
    v, d1, d2 = lagrange_1d(nodes, xs)
    # polynomials of degree <= k are reproduced with their derivatives
    for p in range(k + 1):
        c = nodes ** p
        assert np.allclose(v @ c, xs ** p, atol=1e-12)
        assert np.allclose(d1 @ c, p * xs ** max(p - 1, 0) if p else 0 * xs, atol=1e-10)
        assert np.allclose(d2 @ c, p * (p - 1) * xs ** max(p - 2, 0) if p > 1 else 0 * xs, atol=1e-9)
    # derivatives against central differences
    h = 1e-5
    vp, _, _ = lagrange_1d(nodes, xs + h)
    vm, _, _ = lagrange_1d(nodes, xs - h)
    v0, d1, _ = lagrange_1d(nodes, xs)
    assert np.allclose((vp - vm) / (2 * h), d1, atol=1e-7)
    _, d1p, _ = lagrange_1d(nodes, xs + h)
    _, d1m, d2 = lagrange_1d(nodes, xs - h)[0], lagrange_1d(nodes, xs - h)[1], lagrange_1d(nodes, xs)[2]
    assert np.allclose((d1p - d1m) / (2 * h), d2, atol=1e-5)


@pytest.mark.parametrize("d,k", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_tensor_basis_reproduces_tensor_polynomials(d, k):
    rng = np.random.default_rng(1)
    pts = rng.random((7, d))
    phi, dphi, hphi = tensor_basis(k, d, pts)
    n = k + 1
    nodes = gll_nodes(k)
    idx = np.array(np.unravel_index(np.arange(n ** d), (n,) * d, order="F")).T
    X = nodes[idx]                                  # node coordinates, xi_0 fastest
    # f = xi_0^k * xi_1^(k-1) * (xi_2^1) lies in Q_k
    e = [k, k - 1, 1][:d]
    f = np.prod(X ** np.array(e), axis=1)
    val = np.prod(pts ** np.array(e), axis=1)
    assert np.allclose(phi @ f, val, atol=1e-12)
    for s in range(d):
        es = np.array(e, dtype=float)
        g = es[s] * pts[:, s] ** max(e[s] - 1, 0) * np.prod(np.delete(pts ** np.array(e), s, axis=1), axis=1)
        assert np.allclose(np.einsum("pa,a->p", dphi[:, :, s], f), g, atol=1e-10)
    # mixed second derivative d0 d1
    g01 = e[0] * e[1] * pts[:, 0] ** (e[0] - 1) * pts[:, 1] ** max(e[1] - 1, 0)
    if d == 3:
        g01 = g01 * pts[:, 2] ** e[2]
    assert np.allclose(np.einsum("pa,a->p", hphi[:, :, 0, 1], f), g01, atol=1e-9)
    assert np.allclose(hphi, np.swapaxes(hphi, 2, 3), atol=1e-12)
    # partition of unity
    assert np.allclose(phi.sum(1), 1.0, atol=1e-13)
    assert np.abs(dphi.sum(1)).max() < 1e-11


def test_tensor_gauss_weights():
    for d in (2, 3):
        for k in (1, 2, 3):
            x, w = tensor_gauss(k, d)
            assert x.shape == ((k + 1) ** d, d)
            assert abs(w.sum() - 1.0) < 1e-14
