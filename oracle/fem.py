"""Volume terms of the stabilised ALE Navier-Stokes operator, plain FP64.

Follows Section 2 of the paper:
* weak form Eq. EqNSweak with the pressure and viscous terms integrated by parts
  (Eqs. EqMortarPre, EqMortarDiff), i.e. the volume part of Eq. Eq-NSweakWmortar;
* SUPG/PSPG terms of Eq. Eq-NSweakComplete with the strong residual of
  Eq. Eq-strong-residual and the Tezduyar parameter of Eq. Eq-stab-param;
* the Newton Jacobian blocks of Section 2.3 (A-hat .. D-hat) with the readings
  S5 (SUPG test direction derivative (phi_j . grad) phi_i), S6 (B-hat pairs
  tau a.grad(phi_i) with grad psi_j), S7 (d/dt phi_j -> alpha_0/dt phi_j) and
  S8 (tau frozen).

Two independent evaluation paths: element matrices by naive quadrature loops
over points x test x trial (path A, ``element_matrices``) and per-point field
evaluation followed by test-function integration (path B, ``volume_apply`` and
``volume_residual``).  Geometry: Q_k isoparametric map, physical gradient
J^{-T} grad_xi, physical Hessian J^{-T}(H_xi phi - sum_m (grad phi)_m H_xi x_m) J^{-1}
(reading S15), element size h from the cell volume (Eq. Eq-stab-param with
reading S9).
"""
import numpy as np
from .basis import tensor_basis, tensor_gauss

BDF = {1: (1.0, -1.0, 0.0), 2: (1.5, -2.0, 0.5)}


def rotation_matrix(d, theta):
    """Rotor rotation of Section 3.1: the 2D matrix, or the 3D formula
    R = cos(t) I + sin(t) W + (1 - cos(t)) r (x) r with axis r = e_z and W the
    skew tensor of r (W v = r x v)."""
    c, s = np.cos(theta), np.sin(theta)
    if d == 2:
        return np.array([[c, -s], [s, c]])
    r = np.array([0.0, 0.0, 1.0])
    W = np.array([[0.0, -r[2], r[1]], [r[2], 0.0, -r[0]], [-r[1], r[0], 0.0]])
    return c * np.eye(3) + s * W + (1.0 - c) * np.outer(r, r)


class Problem:
    """Mesh + physical parameters at one rotor angle.

    mesh: synth.RotorStatorMesh-like object; nu, omega, dt (0 = steady), bdf
    (1|2), theta (rotor angle), F (penalty factor, reading S3), source: callable
    f(x [P,d]) -> [P,d] or None (f = 0).
    """

    def __init__(self, mesh, nu, omega, dt, bdf, theta, F=1.0, source=None, stab=True):
        self.mesh = mesh
        self.d = mesh.d
        self.k = mesh.k
        self.n = mesh.k + 1
        self.N = self.n ** self.d
        self.nu = float(nu)
        self.omega = float(omega)
        self.dt = float(dt)
        self.bdf = int(bdf)
        self.theta = float(theta)
        self.F = float(F)
        self.source = source
        self.stab = bool(stab)
        self.cells = np.asarray(mesh.cells, dtype=np.int64)
        self.cell_side = np.asarray(mesh.cell_side)
        self.nn = mesh.x0.shape[0]
        Rm = rotation_matrix(self.d, self.theta)
        x = np.array(mesh.x0, dtype=np.float64)
        rot = np.asarray(mesh.node_side) == 0
        x[rot] = x[rot] @ Rm.T
        self.x = x
        self.wall = np.asarray(mesh.wall).astype(bool)
        self.qpts, self.qw = tensor_gauss(self.k, self.d)
        self.phi, self.dphi, self.hphi = tensor_basis(self.k, self.d, self.qpts)
        self.alpha = BDF[self.bdf]
        self.a0dt = self.alpha[0] / self.dt if self.dt > 0 else 0.0
        self.ht = np.zeros((self.nn, self.d))
        self.h = self.cell_size(np.arange(self.cells.shape[0]))

    # ------------------------------------------------------------------ state
    def set_history(self, u_n, u_nm1=None):
        """h_t = (alpha_1 u^n + alpha_2 u^{n-1}) / dt at the nodes (BDF, Section 4)."""
        if self.dt <= 0:
            self.ht = np.zeros((self.nn, self.d))
            return
        a = self.alpha
        ht = a[1] * np.asarray(u_n, dtype=np.float64)
        if self.bdf == 2:
            ht = ht + a[2] * np.asarray(u_nm1, dtype=np.float64)
        self.ht = ht / self.dt

    # --------------------------------------------------------------- geometry
    def geometry(self, cl):
        """Per cell in cl and Gauss point: J [C,Q,d,d] (J[m,r] = dx_m/dxi_r),
        det J, J^{-1} [C,Q,r,m], W = det J * w_q, physical basis gradient
        [C,Q,N,d], physical basis Laplacian [C,Q,N], physical points [C,Q,d]."""
        X = self.x[self.cells[cl]]                                     # [C,N,d]
        J = np.einsum("Kam,qar->Kqmr", X, self.dphi)
        HX = np.einsum("Kam,qars->Kqmrs", X, self.hphi)
        detJ = np.linalg.det(J)
        Jinv = np.linalg.inv(J)                                         # [C,Q,r,m]
        grad = np.einsum("qar,Kqrm->Kqam", self.dphi, Jinv)
        hcorr = self.hphi[None] - np.einsum("Kqam,Kqmrs->Kqars", grad, HX)
        G = np.einsum("Kqrm,Kqsm->Kqrs", Jinv, Jinv)
        lap = np.einsum("Kqars,Kqrs->Kqa", hcorr, G)
        W = detJ * self.qw[None]
        xq = np.einsum("Kam,qa->Kqm", X, self.phi)
        return dict(J=J, detJ=detJ, Jinv=Jinv, W=W, grad=grad, lap=lap, xq=xq)

    def energy(self, up):
        """Energy budget terms of the discrete velocity u_h at the current
        geometry, by the operator's Gauss rule (Section 4.5.2, energy balance):
        kinetic energy 1/2 int |u_h|^2; viscous dissipation of the Laplacian
        viscous form, nu int grad u_h : grad u_h; and the paper's dissipation
        -tau : grad u with the deviatoric stress tau = -nu (grad u + grad u^T),
        i.e. nu int (grad u_h + grad u_h^T) : grad u_h.  Wall values count."""
        up = np.asarray(up, dtype=np.float64).reshape(self.nn, -1)
        d = self.d
        ke = diss = diss_sym = 0.0
        nc = self.cells.shape[0]
        for s0 in range(0, nc, 512):
            cl = np.arange(s0, min(nc, s0 + 512))
            g = self.geometry(cl)
            U = up[self.cells[cl]][..., :d]                              # [C,N,d]
            uq = np.einsum("qa,Kai->Kqi", self.phi, U)
            gu = np.einsum("Kqam,Kai->Kqim", g["grad"], U)               # gu[i, m] = d u_i / d x_m
            ke += 0.5 * float((g["W"] * (uq ** 2).sum(-1)).sum())
            diss += self.nu * float((g["W"] * (gu ** 2).sum((-1, -2))).sum())
            sym = gu + np.swapaxes(gu, -1, -2)
            diss_sym += self.nu * float((g["W"] * (sym * gu).sum((-1, -2))).sum())
        return ke, diss, diss_sym

    def cell_size(self, cl):
        """h = diameter of the area- (2D) / volume- (3D) equivalent circle/sphere
        (Eq. Eq-stab-param; 3D reading S9)."""
        h = np.empty(len(cl))
        for s0 in range(0, len(cl), 2048):
            c = cl[s0:s0 + 2048]
            X = self.x[self.cells[c]]
            J = np.einsum("Kam,qar->Kqmr", X, self.dphi)
            V = (np.linalg.det(J) * self.qw[None]).sum(1)
            h[s0:s0 + 2048] = np.sqrt(4.0 * V / np.pi) if self.d == 2 else np.cbrt(6.0 * V / np.pi)
        return h

    def u_ale(self, cl, xq):
        """Mesh velocity omega e_z x x in rotor cells, 0 in stator cells (Eq. EqNS)."""
        u = np.zeros_like(xq)
        rot = (self.cell_side[cl] == 0)[:, None]
        u[..., 0] = np.where(rot, -self.omega * xq[..., 1], 0.0)
        u[..., 1] = np.where(rot, self.omega * xq[..., 0], 0.0)
        return u

    def tau(self, a, cl):
        """Tezduyar tau_u of Eq. Eq-stab-param at each point; a = u - u_ALE.
        With stab=False the SUPG/PSPG terms are switched off (tau = 0)."""
        if not self.stab:
            return np.zeros(a.shape[:-1])
        h = self.h[cl][:, None]
        s = (2.0 * np.linalg.norm(a, axis=-1) / h) ** 2 + 9.0 * (4.0 * self.nu / h ** 2) ** 2
        if self.dt > 0:
            s = s + (1.0 / self.dt) ** 2
        return 1.0 / np.sqrt(s)

    def fsrc(self, xq):
        if self.source is None:
            return np.zeros_like(xq)
        return self.source(xq.reshape(-1, self.d)).reshape(xq.shape)

    # ---------------------------------------------------------- point state
    def state(self, cl, g, up, tau_up=None):
        """Velocity value/gradient/Laplacian, pressure value/gradient, history
        term, mesh velocity, advection a = u - u_ALE, tau and the strong residual
        R (Eq. Eq-strong-residual) at the Gauss points of cells cl.  tau is taken
        at the state tau_up when given (frozen-tau residual, reading S8)."""
        d = self.d
        vals = up[self.cells[cl]]                                      # [C,N,d+1]
        U = np.einsum("qa,Kai->Kqi", self.phi, vals[..., :d])
        gU = np.einsum("Kqam,Kai->Kqim", g["grad"], vals[..., :d])     # [C,Q,c,m]
        lU = np.einsum("Kqa,Kai->Kqi", g["lap"], vals[..., :d])
        P = np.einsum("qa,Ka->Kq", self.phi, vals[..., d])
        gP = np.einsum("Kqam,Ka->Kqm", g["grad"], vals[..., d])
        ht = np.einsum("qa,Kai->Kqi", self.phi, self.ht[self.cells[cl]])
        ua = self.u_ale(cl, g["xq"])
        a = U - ua
        if tau_up is None:
            tau = self.tau(a, cl)
        else:
            Ut = np.einsum("qa,Kai->Kqi", self.phi, tau_up[self.cells[cl]][..., :d])
            tau = self.tau(Ut - ua, cl)
        Rs = (self.a0dt * U + ht + np.einsum("Kqm,Kqim->Kqi", a, gU) + gP
              - self.nu * lU - self.fsrc(g["xq"]))
        return dict(U=U, gU=gU, lU=lU, P=P, gP=gP, ht=ht, a=a, tau=tau, R=Rs)

    # -------------------------------------------------- path B: matrix-free
    def volume_residual(self, up, cl=None, out=None, tau_up=None):
        """Volume part of the stabilised weak residual (Eq. Eq-NSweakComplete with
        the integrated-by-parts pressure and viscous terms of Eq. Eq-NSweakWmortar)
        at the state up [N_n, d+1], accumulated into out [N_n, d+1]."""
        d = self.d
        cl = np.arange(self.cells.shape[0]) if cl is None else np.asarray(cl)
        out = np.zeros((self.nn, d + 1)) if out is None else out
        for s0 in range(0, len(cl), 512):
            c = cl[s0:s0 + 512]
            g = self.geometry(c)
            st = self.state(c, g, up, tau_up)
            W = g["W"]
            # value flux of v: d_t u + (a . grad) u - f ; gradient flux of v:
            # nu grad u - p I + tau a (x) R ; value flux of q: div u ; gradient flux of q: tau R
            fv = (self.a0dt * st["U"] + st["ht"] + np.einsum("Kqm,Kqim->Kqi", st["a"], st["gU"])
                  - self.fsrc(g["xq"]))
            Fv = self.nu * st["gU"] - st["P"][..., None, None] * np.eye(d)[None, None]
            Fv = Fv + st["tau"][..., None, None] * st["R"][..., :, None] * st["a"][..., None, :]
            fq = np.einsum("Kqii->Kq", st["gU"])
            Fq = st["tau"][..., None] * st["R"]
            loc = np.zeros((len(c), self.N, d + 1))
            loc[..., :d] = (np.einsum("Kq,qa,Kqi->Kai", W, self.phi, fv)
                            + np.einsum("Kq,Kqam,Kqim->Kai", W, g["grad"], Fv))
            loc[..., d] = (np.einsum("Kq,qa,Kq->Ka", W, self.phi, fq)
                           + np.einsum("Kq,Kqam,Kqm->Ka", W, g["grad"], Fq))
            np.add.at(out, self.cells[c].ravel(), loc.reshape(-1, d + 1))
        return out

    def volume_apply(self, up_star, w, cl=None, out=None):
        """Volume part of the Jacobian applied to w [N_n, d+1] (increments of
        velocity and pressure), linearised at up_star; the Gateaux derivative of
        ``volume_residual`` with tau frozen (blocks A-hat..D-hat, Section 2.3)."""
        d = self.d
        cl = np.arange(self.cells.shape[0]) if cl is None else np.asarray(cl)
        out = np.zeros((self.nn, d + 1)) if out is None else out
        for s0 in range(0, len(cl), 512):
            c = cl[s0:s0 + 512]
            g = self.geometry(c)
            st = self.state(c, g, up_star)
            W = g["W"]
            vals = w[self.cells[c]]
            Wv = np.einsum("qa,Kai->Kqi", self.phi, vals[..., :d])
            gW = np.einsum("Kqam,Kai->Kqim", g["grad"], vals[..., :d])
            lW = np.einsum("Kqa,Kai->Kqi", g["lap"], vals[..., :d])
            Pr = np.einsum("qa,Ka->Kq", self.phi, vals[..., d])
            gPr = np.einsum("Kqam,Ka->Kqm", g["grad"], vals[..., d])
            a, tau = st["a"], st["tau"]
            gal = (self.a0dt * Wv + np.einsum("Kqm,Kqim->Kqi", Wv, st["gU"])
                   + np.einsum("Kqm,Kqim->Kqi", a, gW))
            Rl = gal + gPr - self.nu * lW
            fv = gal
            Fv = self.nu * gW - Pr[..., None, None] * np.eye(d)[None, None]
            Fv = Fv + tau[..., None, None] * (Rl[..., :, None] * a[..., None, :]
                                                + st["R"][..., :, None] * Wv[..., None, :])
            fq = np.einsum("Kqii->Kq", gW)
            Fq = tau[..., None] * Rl
            loc = np.zeros((len(c), self.N, d + 1))
            loc[..., :d] = (np.einsum("Kq,qa,Kqi->Kai", W, self.phi, fv)
                            + np.einsum("Kq,Kqam,Kqim->Kai", W, g["grad"], Fv))
            loc[..., d] = (np.einsum("Kq,qa,Kq->Ka", W, self.phi, fq)
                           + np.einsum("Kq,Kqam,Kqm->Ka", W, g["grad"], Fq))
            np.add.at(out, self.cells[c].ravel(), loc.reshape(-1, d + 1))
        return out

    # -------------------------------------------------- path A: element matrices
    def element_matrices(self, up_star, cl):
        """Element Jacobian matrices E[c, a, f, b, e] (test node a field f, trial
        node b field e; fields 0..d-1 velocity, d pressure) by naive quadrature of
        the blocks A-hat, B-hat, C-hat, D-hat written entry by entry."""
        d = self.d
        cl = np.asarray(cl)
        g = self.geometry(cl)
        st = self.state(cl, g, up_star)
        W, phi, grad, lap = g["W"], self.phi, g["grad"], g["lap"]
        a, tau, gU, Rs = st["a"], st["tau"], st["gU"], st["R"]
        C, N = len(cl), self.N
        sa = np.einsum("Kqm,Kqam->Kqa", a, grad)                      # a . grad(phi_a)
        Lb = self.a0dt * phi[None] + sa - self.nu * lap               # d_t phi + a.grad phi - nu lap phi
        E = np.zeros((C, N, d + 1, N, d + 1))
        # velocity-velocity, diagonal in components
        diag = (np.einsum("Kq,qa,qb->Kab", W, phi, self.a0dt * phi)
                + np.einsum("Kq,qa,Kqb->Kab", W, phi, sa)
                + self.nu * np.einsum("Kq,Kqam,Kqbm->Kab", W, grad, grad)
                + np.einsum("Kq,Kq,Kqa,Kqb->Kab", W, tau, sa, Lb))
        for c_ in range(d):
            E[:, :, c_, :, c_] += diag
        # velocity-velocity, coupling through grad U* and R*
        E[:, :, :d, :, :d] += np.einsum("Kq,qa,qb,Kqij->Kaibj", W, phi, phi, gU)
        E[:, :, :d, :, :d] += np.einsum("Kq,Kq,Kqa,qb,Kqij->Kaibj", W, tau, sa, phi, gU)
        E[:, :, :d, :, :d] += np.einsum("Kq,Kq,qb,Kqaj,Kqi->Kaibj", W, tau, phi, grad, Rs)
        # velocity test, pressure trial: -(div phi_i, psi_j) + (tau a.grad phi_i, grad psi_j)
        E[:, :, :d, :, d] += (-np.einsum("Kq,Kqai,qb->Kaib", W, grad, phi)
                              + np.einsum("Kq,Kq,Kqa,Kqbi->Kaib", W, tau, sa, grad))
        # pressure test, velocity trial: (psi_i, div phi_j) + (tau grad psi_i, R'(phi_j))
        E[:, :, d, :, :d] += (np.einsum("Kq,qa,Kqbj->Kabj", W, phi, grad)
                              + np.einsum("Kq,Kq,Kqaj,Kqb->Kabj", W, tau, grad, Lb)
                              + np.einsum("Kq,Kq,Kqai,qb,Kqij->Kabj", W, tau, grad, phi, gU))
        # pressure-pressure: (tau grad psi_i, grad psi_j)
        E[:, :, d, :, d] += np.einsum("Kq,Kq,Kqam,Kqbm->Kab", W, tau, grad, grad)
        return E
