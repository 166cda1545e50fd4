"""Mortar interface of the rotor-stator mesh, plain FP64.

* Mortar cells (Section 2.1, Fig. mortar, Section 3.2): the interface circle is
  cut at every rotor vertex (rotated by theta) and every stator vertex; each
  piece of the sorted union is a mortar segment, and a reference Gauss rule is
  mapped into it.  Weight of a point: w_hat * R * (segment angle) [* w_z * dz]
  (reading S10 of the garbled det J = R delta_0 delta_1).  Point on the exact
  circle with the exact normal (reading S13); each side's reference coordinate
  along the face is linear in the angle.
* Penalty tau_k of Eq. EqPenalty (Hillewaert), with S2 (face value = max of the
  two cells), S3 (F = 1 by default) and S4 (all non-interface faces halved).
* Face terms of Eq. Eq-NSweakWmortar with reading S1: on side s, the jump is
  own minus other and n is the side's own outward normal:
      - (q, 1/2 [[u]].n) + (v, {p} n) - (grad v : nu/2 [[u]] (x) n)
      - (v, nu {grad u} n) + (v, nu tau [[u]]).
"""
import numpy as np
from .basis import tensor_basis, gauss_rule, tensor_gauss


def mortar_segments(theta, n_R, n_Rs=None):
    """Sorted union of rotor vertices theta + 2 pi i / n_R and stator vertices
    2 pi j / n_Rs (n_Rs = n_R: the paper's equal partitions) on the circle,
    angles relative to the partition origin phi0.  Returns (start angle,
    length, rotor cell index, stator cell index) for every piece of positive
    length; with unequal partitions a cell may meet several pieces."""
    two_pi = 2.0 * np.pi
    n_Rs = n_R if n_Rs is None else int(n_Rs)
    Dr, Ds = two_pi / n_R, two_pi / n_Rs
    rv = np.mod(theta + Dr * np.arange(n_R), two_pi)
    sv = np.mod(Ds * np.arange(n_Rs), two_pi)
    cuts = np.sort(np.concatenate([rv, sv]))
    segs = []
    for i in range(len(cuts)):
        a = cuts[i]
        b = cuts[i + 1] if i + 1 < len(cuts) else cuts[0] + two_pi
        L = b - a
        if L <= 1e-13:
            continue
        mid = a + 0.5 * L
        jr = int(np.floor(np.mod(mid - theta, two_pi) / Dr)) % n_R
        js = int(np.floor(np.mod(mid, two_pi) / Ds)) % n_Rs
        segs.append((a, L, jr, js))
    return segs


def face_coordinate(phi, start, n_R):
    """Reference coordinate along a side's face: the angle from the cell's first
    vertex (modulo 2 pi) divided by the cell's angular size (reading S13)."""
    D = 2.0 * np.pi / n_R
    return np.mod(phi - start, 2.0 * np.pi) / D


def face_area(prob, cell, r, side, q):
    """Area (3D) or length (2D) of the face xi_r = side of a cell by a q-point
    Gauss rule on the face of the isoparametric map."""
    d = prob.d
    x, w = gauss_rule(q)
    if d == 2:
        pts = np.zeros((q, 2))
        pts[:, r] = side
        pts[:, 1 - r] = x
        wt = w
    else:
        t = [s for s in range(3) if s != r]
        X1, X2 = np.meshgrid(x, x, indexing="ij")
        W1, W2 = np.meshgrid(w, w, indexing="ij")
        pts = np.zeros((q * q, 3))
        pts[:, r] = side
        pts[:, t[0]] = X1.ravel()
        pts[:, t[1]] = X2.ravel()
        wt = (W1 * W2).ravel()
    _, dphi, _ = tensor_basis(prob.k, d, pts)
    X = prob.x[prob.cells[cell]]
    J = np.einsum("am,par->pmr", X, dphi)
    if d == 2:
        t = 1 - r
        da = np.linalg.norm(J[:, :, t], axis=1)
    else:
        t = [s for s in range(3) if s != r]
        da = np.linalg.norm(np.cross(J[:, :, t[0]], J[:, :, t[1]]), axis=1)
    return float((da * wt).sum())


def penalty(prob, cell, iface_side):
    """tau_k = F (k+1)^2 (A(other faces)/2 + A(interface face)) / V (Eq. EqPenalty).
    The interface face of rotor cells is xi_0 = 1, of stator cells xi_0 = 0."""
    q = prob.k + 1
    areas = {}
    for r in range(prob.d):
        for s in (0.0, 1.0):
            areas[(r, s)] = face_area(prob, cell, r, s, q)
    a_if = areas[(0, iface_side)]
    a_other = sum(v for key, v in areas.items() if key != (0, iface_side))
    g = prob.geometry(np.array([cell]))
    V = float(g["W"].sum())
    return prob.F * (prob.k + 1) ** 2 * (0.5 * a_other + a_if) / V


class Mortar:
    """Mortar points of the interface at the problem's rotor angle."""

    def __init__(self, prob, layers=None):
        """layers: z-layers to build (default all); a subset serves sampled checks."""
        m = prob.mesh
        self.prob = prob
        d = prob.d
        self.R = float(m.R)
        self.n_R = int(m.n_R)
        self.n_Rs = int(getattr(m, "n_R_stator", 0) or self.n_R)     # stator partition (default: equal)
        self.n_z = int(m.n_z)
        D = 2.0 * np.pi / self.n_R
        Ds = 2.0 * np.pi / self.n_Rs
        sg, wg = gauss_rule(prob.k + 1)
        segs = mortar_segments(prob.theta, self.n_R, self.n_Rs)
        phi0 = float(m.phi0)
        self.tau_cell = {}
        recs = []
        for lz in (range(self.n_z) if layers is None else layers):
            for (pa, L, jr, js) in segs:
                cr = int(m.iface_rotor[lz, jr])
                cs = int(m.iface_stator[lz, js])
                rel = pa + sg * L
                xr = face_coordinate(rel, prob.theta + jr * D, self.n_R)
                xs = face_coordinate(rel, js * Ds, self.n_Rs)
                phis = phi0 + rel
                w = wg * self.R * L
                if d == 2:
                    pr = np.stack([np.ones_like(xr), xr], axis=1)
                    ps = np.stack([np.zeros_like(xs), xs], axis=1)
                    wq = w
                    nrm = np.stack([np.cos(phis), np.sin(phis)], axis=1)
                else:
                    dz = m.H / self.n_z
                    A, Z = np.meshgrid(np.arange(len(sg)), np.arange(len(sg)), indexing="xy")
                    A, Z = A.ravel(), Z.ravel()        # angular index fastest
                    pr = np.stack([np.ones(len(A)), xr[A], sg[Z]], axis=1)
                    ps = np.stack([np.zeros(len(A)), xs[A], sg[Z]], axis=1)
                    wq = w[A] * wg[Z] * dz
                    nrm = np.stack([np.cos(phis[A]), np.sin(phis[A]), np.zeros(len(A))], axis=1)
                recs.append(dict(cells=(cr, cs), pts=(pr, ps), w=wq, n=nrm))
                for c_, s_ in ((cr, 1.0), (cs, 0.0)):
                    if c_ not in self.tau_cell:
                        self.tau_cell[c_] = penalty(prob, c_, s_)
        self.recs = recs

    def side_eval(self, cell, pts):
        """Basis values and physical gradients of a cell at reference points."""
        prob = self.prob
        phi, dphi, _ = tensor_basis(prob.k, prob.d, pts)
        X = prob.x[prob.cells[cell]]
        J = np.einsum("am,par->pmr", X, dphi)
        Jinv = np.linalg.inv(J)
        grad = np.einsum("par,prm->pam", dphi, Jinv)
        return phi, grad

    def pair_matrix(self, rec):
        """Face element matrix M[s, a, f, t, b, e] of one mortar cell: test side s
        node a field f, trial side t node b field e (side 0 rotor, 1 stator)."""
        prob = self.prob
        d, N, nu = prob.d, prob.N, prob.nu
        cr, cs = rec["cells"]
        tau_f = max(self.tau_cell[cr], self.tau_cell[cs])
        ev = [self.side_eval(cr, rec["pts"][0]), self.side_eval(cs, rec["pts"][1])]
        nr = [rec["n"], -rec["n"]]
        w = rec["w"]
        M = np.zeros((2, N, d + 1, 2, N, d + 1))
        for s in range(2):
            phs, grs = ev[s]
            ns = nr[s]
            for t in range(2):
                pht, grt = ev[t]
                sg = 1.0 if s == t else -1.0
                # (v, {p} n_s)
                M[s, :, :d, t, :, d] += 0.5 * np.einsum("p,pa,pb,pi->aib", w, phs, pht, ns)
                # -(q, 1/2 [[u]] . n_s)
                M[s, :, d, t, :, :d] += -0.5 * sg * np.einsum("p,pa,pb,pj->abj", w, phs, pht, ns)
                # -(grad v : nu/2 [[u]] (x) n_s) - (v, nu {grad u} n_s) + (v, nu tau [[u]])
                vv = (-0.5 * nu * sg * np.einsum("p,pam,pm,pb->ab", w, grs, ns, pht)
                      - 0.5 * nu * np.einsum("p,pa,pbm,pm->ab", w, phs, grt, ns)
                      + nu * tau_f * sg * np.einsum("p,pa,pb->ab", w, phs, pht))
                for i in range(d):
                    M[s, :, i, t, :, i] += vv
        return M

    def apply(self, w_vec, out=None, recs=None):
        """Face terms applied to the nodal vector w_vec [N_n, d+1] by per-point
        evaluation of traces, averages and jumps (matrix-free form)."""
        prob = self.prob
        d, nu = prob.d, prob.nu
        out = np.zeros((prob.nn, d + 1)) if out is None else out
        for rec in (self.recs if recs is None else recs):
            cr, cs = rec["cells"]
            tau_f = max(self.tau_cell[cr], self.tau_cell[cs])
            ev = [self.side_eval(cr, rec["pts"][0]), self.side_eval(cs, rec["pts"][1])]
            vals = [w_vec[prob.cells[cr]], w_vec[prob.cells[cs]]]
            u = [np.einsum("pa,ai->pi", ev[s][0], vals[s][:, :d]) for s in range(2)]
            gu = [np.einsum("pam,ai->pim", ev[s][1], vals[s][:, :d]) for s in range(2)]
            p = [ev[s][0] @ vals[s][:, d] for s in range(2)]
            nr = [rec["n"], -rec["n"]]
            w = rec["w"]
            pavg = 0.5 * (p[0] + p[1])
            gavg = 0.5 * (gu[0] + gu[1])
            for s in range(2):
                o = 1 - s
                jump = u[s] - u[o]
                ns = nr[s]
                fv = pavg[:, None] * ns - nu * np.einsum("pim,pm->pi", gavg, ns) + nu * tau_f * jump
                Fv = -0.5 * nu * jump[:, :, None] * ns[:, None, :]
                fq = -0.5 * (jump * ns).sum(1)
                phs, grs = ev[s]
                loc = np.zeros((prob.N, d + 1))
                loc[:, :d] = (np.einsum("p,pa,pi->ai", w, phs, fv)
                              + np.einsum("p,pam,pim->ai", w, grs, Fv))
                loc[:, d] = np.einsum("p,pa,p->a", w, phs, fq)
                np.add.at(out, prob.cells[rec["cells"][s]], loc)
        return out
