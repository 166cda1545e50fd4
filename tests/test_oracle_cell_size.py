"""Pin of the oracle's element size h (Eq. Eq-stab-param; 3D reading S9).

h enters tau, so a wrong constant (a radius in place of a diameter, a missing
4/pi) changes tau by a fixed factor: every consistency pin (FD Jacobian, MMS,
conforming identity) still passes because both paths use the same h.  These
checks compare h against closed forms instead: single cells whose volume is
known exactly (unit square and cube, a box, curved Q2 cells with a polynomial
Jacobian that the (k+1)-point Gauss rule integrates exactly), and the
diameter of the area- / volume-equivalent circle / sphere,
  2D: h = sqrt(4 V / pi),   3D: h = (6 V / pi)^(1/3).
A planted mistake of each kind fails the same check."""
import numpy as np
import pytest

from oracle.basis import gll_nodes
from oracle.fem import Problem


class _OneCell:
    """A one-cell mesh whose nodes sit at x = phi(GLL point) for a map phi."""

    def __init__(self, d, k, phi):
        self.d, self.k = d, k
        g = gll_nodes(k)
        n = k + 1
        idx = np.array(np.unravel_index(np.arange(n ** d), (n,) * d, order="F")).T
        ref = g[idx]                                        # [N, d], xi_0 fastest
        self.x0 = np.array([phi(p) for p in ref], dtype=np.float64)
        self.cells = np.arange(n ** d, dtype=np.int32)[None]
        self.cell_side = np.ones(1, np.uint8)               # stator: no rotation applied
        self.node_side = np.ones(n ** d, np.uint8)
        self.wall = np.zeros(n ** d, np.uint8)
        self.n_cells = 1


# (d, k, map, exact volume)
CASES = [
    (2, 1, lambda p: p, 1.0),                                          # unit square
    (2, 2, lambda p: np.array([2.0 * p[0], p[1] * (1.0 + p[0])]), 3.0),  # trapezoid, det J = 2(1 + xi)
    (2, 2, lambda p: np.array([p[0], p[1] * (1.0 + p[0] ** 2)]), 4.0 / 3.0),  # curved top, det J = 1 + xi^2
    (2, 3, lambda p: np.array([p[0] + 0.3 * p[1], 0.5 * p[1]]), 0.5),   # parallelogram
    (3, 1, lambda p: p, 1.0),                                          # unit cube
    (3, 2, lambda p: np.array([2.0 * p[0], p[1], 0.5 * p[2]]), 1.0),    # box 2 x 1 x 1/2
    (3, 2, lambda p: np.array([p[0], p[1], p[2] * (1.0 + p[0] ** 2)]), 4.0 / 3.0),  # curved top face
    (3, 3, lambda p: np.array([p[0], p[1] * (2.0 + p[0]), 3.0 * p[2]]), 7.5),  # det J = 3(2 + xi)
]


def _expected_h(d, V):
    return np.sqrt(4.0 * V / np.pi) if d == 2 else (6.0 * V / np.pi) ** (1.0 / 3.0)


def _pin_holds(problem_cls):
    for d, k, phi, V in CASES:
        p = problem_cls(_OneCell(d, k, phi), 0.01, 0.0, 0.0, 1, 0.0)
        h = float(p.cell_size(np.array([0]))[0])
        if abs(h / _expected_h(d, V) - 1.0) > 1e-13:
            return False
    return True


@pytest.mark.parametrize("case", range(len(CASES)))
def test_cell_size_matches_equivalent_circle_or_sphere(case):
    d, k, phi, V = CASES[case]
    p = Problem(_OneCell(d, k, phi), 0.01, 0.0, 0.0, 1, 0.0)
    h = float(p.cell_size(np.array([0]))[0])
    assert abs(h / _expected_h(d, V) - 1.0) < 1e-13, (h, _expected_h(d, V))
    # the constructor's per-cell h is the same value (it is what tau reads)
    assert abs(p.h[0] / h - 1.0) < 1e-15


def test_cell_size_closed_form_numbers():
    """Numbers written out: unit square 2/sqrt(pi), unit cube (6/pi)^(1/3)."""
    sq = Problem(_OneCell(2, 1, lambda p: p), 0.01, 0.0, 0.0, 1, 0.0).h[0]
    cu = Problem(_OneCell(3, 1, lambda p: p), 0.01, 0.0, 0.0, 1, 0.0).h[0]
    assert abs(sq - 1.1283791670955126) < 1e-15
    assert abs(cu - 1.2407009817988002) < 1e-15


def test_tau_uses_pinned_h():
    """tau at a point of the unit cube in the diffusive limit equals
    h^2 / (12 nu) with h = (6/pi)^(1/3): the pinned h is the one tau sees."""
    p = Problem(_OneCell(3, 1, lambda q: q), 10.0, 0.0, 0.0, 1, 0.0)
    t = p.tau(np.array([[[1e-12, 0.0, 0.0]]]), np.array([0]))[0, 0]
    h = (6.0 / np.pi) ** (1.0 / 3.0)
    assert abs(t / (h * h / 120.0) - 1.0) < 1e-12


class _Radius(Problem):
    """Planted mistake: radius instead of diameter of the equivalent circle."""

    def cell_size(self, cl):
        return 0.5 * Problem.cell_size(self, cl)


class _No4OverPi(Problem):
    """Planted mistake: h = sqrt(V) (2D) / cbrt(V) (3D), no 4/pi or 6/pi."""

    def cell_size(self, cl):
        h = Problem.cell_size(self, cl)
        V = h ** self.d * (np.pi / 4.0 if self.d == 2 else np.pi / 6.0)
        return V ** (1.0 / self.d)


class _DividedByK(Problem):
    """Planted mistake: h divided by the degree (the rejected reading of S9)."""

    def cell_size(self, cl):
        return Problem.cell_size(self, cl) / self.k


def test_planted_mistakes_fail_the_pin():
    assert _pin_holds(Problem)
    for bad in (_Radius, _No4OverPi, _DividedByK):
        assert not _pin_holds(bad), bad.__name__
